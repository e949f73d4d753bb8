"""GPU pruning, rendering (Eq. 1), gradient and grid update vs the oracle.

Inputs come from the seeded generators only: the marched samples are the
oracle's (identical to the GPU's, see test_gpu_march.py), sigma and rgb are the
procedural field evaluated on the host. Bars: pruning decisions exact except
within the float32 summation error bound of the threshold; colour / opacity /
depth within 1e-5 (depth 1e-5 relative above 1); gradients within 1e-4
relative (floor 1e-3 of the largest magnitude); grid update bit-exact.
"""
import numpy as np
import pytest

from paper_2210_04847_gb300 import _lib, synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no CUDA device", allow_module_level=True)

from gpu_util import bits_equal, dev, grad_rel_err, near_threshold, oracle_march, render_tol_ok  # noqa: E402


@pytest.fixture(scope="module")
def scene(orc):
    """Bounded scene, 2048 rays: marched samples (oracle), field values (host), pruned set (oracle)."""
    w = synth.bounded_config(3, n_rays=2048, device="cuda")
    m = oracle_march(orc, w)
    sig, rgb = synth.sample_field(w.scenes[0], w.rays_o, w.rays_d, m.t_starts, m.t_ends, m.ray_indices)
    p, keep, od = orc.prune(m.packed_info, m.t_starts, m.t_ends, sig, w.early_stop_eps, w.alpha_thre)
    sig2, rgb2 = synth.sample_field(w.scenes[0], w.rays_o, w.rays_d, p.t_starts, p.t_ends, p.ray_indices)
    return dict(w=w, m=m, sig=sig, p=p, keep=keep, od=od, sig2=sig2, rgb2=rgb2)


def _gpu_prune(pi, ts, te, sg, eps, thre, capacity=None):
    R, M = pi.shape[0], ts.shape[0]
    cap = M if capacity is None else capacity
    ws = torch.zeros(_lib.prune_workspace_size(R, M), dtype=torch.uint8, device="cuda")
    out = dict(pi=torch.full((R, 2), -3, dtype=torch.int32, device="cuda"),
               ts=torch.zeros(max(cap, 1), device="cuda"), te=torch.zeros(max(cap, 1), device="cuda"),
               ri=torch.zeros(max(cap, 1), dtype=torch.int32, device="cuda"),
               n=torch.zeros(1, dtype=torch.int64, device="cuda"), st=torch.zeros(1, dtype=torch.int32, device="cuda"),
               keep=torch.full((max(M, 1),), 7, dtype=torch.uint8, device="cuda"))
    _lib.prune_samples(dev(pi), dev(ts), dev(te), dev(sg), M, eps, thre, out["pi"], out["ts"][:cap], out["te"][:cap],
                       out["ri"][:cap], out["n"], out["st"], ws, keep_mask=out["keep"][:M] if M else None)
    torch.cuda.synchronize()
    return {k: v.cpu().numpy() for k, v in out.items()}


def test_prune_parity(scene):
    w, m, sig = scene["w"], scene["m"], scene["sig"]
    g = _gpu_prune(m.packed_info, m.t_starts, m.t_ends, sig, w.early_stop_eps, w.alpha_thre)
    assert g["st"][0] == 0
    keep_g = g["keep"][: m.n_samples].astype(bool)
    keep_o = scene["keep"]
    near = near_threshold(m.packed_info, m.t_starts, m.t_ends, sig, w.early_stop_eps, scene["od"])
    diff = keep_g != keep_o
    assert not (diff & ~near).any(), "keep decisions differ away from the threshold"
    flipped_rays = set(np.searchsorted(m.packed_info[:, 0], np.nonzero(diff)[0], side="right") - 1)
    p = scene["p"]
    n = int(g["n"][0])
    assert n == int(keep_g.sum())
    # rays without a near-threshold flip: identical packed content
    for r in range(m.packed_info.shape[0]):
        if r in flipped_rays:
            continue
        (og, cg), (oo, co) = g["pi"][r], p.packed_info[r]
        assert cg == co
        assert bits_equal(g["ts"][og : og + cg], p.t_starts[oo : oo + co])
        assert bits_equal(g["te"][og : og + cg], p.t_ends[oo : oo + co])
        assert np.all(g["ri"][og : og + cg] == r)
    assert len(flipped_rays) <= 2
    assert p.n_samples < 0.6 * m.n_samples  # the workload really prunes


def test_prune_off_and_capacity(scene):
    m, sig = scene["m"], scene["sig"]
    g = _gpu_prune(m.packed_info, m.t_starts, m.t_ends, sig, 0.0, 0.0)
    assert int(g["n"][0]) == m.n_samples and np.array_equal(g["pi"], m.packed_info)
    assert bits_equal(g["ts"][: m.n_samples], m.t_starts) and np.array_equal(g["ri"][: m.n_samples], m.ray_indices)
    cap = 1000
    g = _gpu_prune(m.packed_info, m.t_starts, m.t_ends, sig, 0.0, 0.0, capacity=cap)
    assert g["st"][0] & _lib.STATUS_CAPACITY and int(g["n"][0]) == m.n_samples
    assert bits_equal(g["ts"][:cap], m.t_starts[:cap])


def _gpu_fwd(pi, ts, te, sg, rgb, save=False):
    R, M = pi.shape[0], ts.shape[0]
    col = torch.zeros((R, 3), device="cuda")
    op = torch.zeros(R, device="cuda")
    dp = torch.zeros(R, device="cuda")
    od = torch.zeros(max(M, 1), device="cuda") if save else None
    st = torch.zeros(1, dtype=torch.int32, device="cuda")
    _lib.render_fwd(dev(pi), dev(ts), dev(te), dev(sg), dev(rgb), M, col, op, dp,
                    optical_depth=od[:M] if save else None, d_status=st)
    torch.cuda.synchronize()
    assert int(st.item()) == 0
    return col.cpu().numpy(), op.cpu().numpy(), dp.cpu().numpy(), (od.cpu().numpy()[:M] if save else None)


def _gpu_bwd(pi, ts, te, sg, rgb, gc, ga, gd, od=None):
    M = ts.shape[0]
    ds = torch.full((max(M, 1),), np.nan, device="cuda")
    dr = torch.full((max(M, 1), 3), np.nan, device="cuda")
    st = torch.zeros(1, dtype=torch.int32, device="cuda")
    _lib.render_bwd(dev(pi), dev(ts), dev(te), dev(sg), dev(rgb), M, dev(gc), dev(ga), dev(gd), ds[:M], dr[:M],
                    optical_depth=dev(od), d_status=st)
    torch.cuda.synchronize()
    assert int(st.item()) == 0
    return ds.cpu().numpy()[:M], dr.cpu().numpy()[:M]


def test_render_fwd_parity(scene, orc):
    p, sg, rgb = scene["p"], scene["sig2"], scene["rgb2"]
    col, op, dp, _ = _gpu_fwd(p.packed_info, p.t_starts, p.t_ends, sg, rgb)
    c_o, a_o, d_o = orc.render_fwd(p.packed_info, p.t_starts, p.t_ends, sg, rgb)
    assert render_tol_ok(col, c_o, rel_for_large=False) <= 1.0
    assert render_tol_ok(op, a_o, rel_for_large=False) <= 1.0
    assert render_tol_ok(dp, d_o) <= 1.0
    assert a_o.max() > 0.99  # surfaces are hit


def test_render_fwd_unpruned_long_rays(scene, orc):
    """All marched samples (hundreds per ray), no pruning."""
    m, sg = scene["m"], scene["sig"]
    _, rgb = synth.sample_field(scene["w"].scenes[0], scene["w"].rays_o, scene["w"].rays_d, m.t_starts, m.t_ends,
                                m.ray_indices)
    col, op, dp, _ = _gpu_fwd(m.packed_info, m.t_starts, m.t_ends, sg, rgb)
    c_o, a_o, d_o = orc.render_fwd(m.packed_info, m.t_starts, m.t_ends, sg, rgb)
    assert render_tol_ok(col, c_o, rel_for_large=False) <= 1.0
    assert render_tol_ok(op, a_o, rel_for_large=False) <= 1.0
    assert render_tol_ok(dp, d_o) <= 1.0


def test_render_bwd_parity_and_saved_state(scene, orc):
    p, sg, rgb = scene["p"], scene["sig2"], scene["rgb2"]
    R = p.packed_info.shape[0]
    gc = synth.rand_uniform(7, 1, 3 * R, -1, 1).reshape(R, 3).astype(np.float32) / R
    ga = synth.rand_uniform(7, 2, R, -1, 1).astype(np.float32) / R
    gd = synth.rand_uniform(7, 3, R, -1, 1).astype(np.float32) / R
    ds, dr = _gpu_bwd(p.packed_info, p.t_starts, p.t_ends, sg, rgb, gc, ga, gd)
    ds_o, dr_o = orc.render_bwd(p.packed_info, p.t_starts, p.t_ends, sg, rgb, gc.astype(np.float64),
                                ga.astype(np.float64), gd.astype(np.float64))
    assert grad_rel_err(ds, ds_o) <= 1e-4
    assert grad_rel_err(dr, dr_o) <= 1e-4
    # saved optical depth: identical bits to the recomputed path
    _, _, _, od = _gpu_fwd(p.packed_info, p.t_starts, p.t_ends, sg, rgb, save=True)
    ds2, dr2 = _gpu_bwd(p.packed_info, p.t_starts, p.t_ends, sg, rgb, gc, ga, gd, od=od)
    assert bits_equal(ds, ds2) and bits_equal(dr, dr2)


def test_render_bwd_only_color_grad(scene, orc):
    """MSE-style loss: only g_color (g_opacity = g_depth = NULL)."""
    p, sg, rgb = scene["p"], scene["sig2"], scene["rgb2"]
    R = p.packed_info.shape[0]
    col, _, _, _ = _gpu_fwd(p.packed_info, p.t_starts, p.t_ends, sg, rgb)
    target = scene["w"].target_rgb[:R]
    c_o, _, _ = orc.render_fwd(p.packed_info, p.t_starts, p.t_ends, sg, rgb)
    gc = (2.0 * (c_o - target) / (3 * R)).astype(np.float32)
    ds, dr = _gpu_bwd(p.packed_info, p.t_starts, p.t_ends, sg, rgb, gc, None, None)
    ds_o, dr_o = orc.render_bwd(p.packed_info, p.t_starts, p.t_ends, sg, rgb, gc.astype(np.float64))
    assert grad_rel_err(ds, ds_o) <= 1e-4 and grad_rel_err(dr, dr_o) <= 1e-4


def test_render_long_ray_beyond_carry_record(orc):
    """One ray of 5000 samples (more chunks than the backward keeps in shared memory), one empty ray."""
    n = 5000
    ts = (1.0 + 0.001 * np.arange(n)).astype(np.float32)
    te = (1.0 + 0.001 * np.arange(1, n + 1)).astype(np.float32)
    sg = synth.rand_uniform(4, 1, n, 0, 2).astype(np.float32)
    rgb = synth.rand_uniform(4, 2, 3 * n).reshape(n, 3).astype(np.float32)
    pi = np.array([[0, n], [n, 0]], np.int32)
    col, op, dp, _ = _gpu_fwd(pi, ts, te, sg, rgb)
    c_o, a_o, d_o = orc.render_fwd(pi, ts, te, sg, rgb)
    assert render_tol_ok(col, c_o, rel_for_large=False) <= 1.0 and render_tol_ok(dp, d_o) <= 1.0
    gc = np.array([[0.3, -0.2, 0.1], [1, 1, 1]], np.float32)
    ga = np.array([0.05, 1], np.float32)
    gd = np.array([-0.01, 1], np.float32)
    ds, dr = _gpu_bwd(pi, ts, te, sg, rgb, gc, ga, gd)
    ds_o, dr_o = orc.render_bwd(pi, ts, te, sg, rgb, gc.astype(np.float64), ga.astype(np.float64),
                                gd.astype(np.float64))
    assert grad_rel_err(ds, ds_o) <= 1e-4 and grad_rel_err(dr, dr_o) <= 1e-4


def test_render_weights_and_accumulate(scene, orc):
    p, sg, rgb = scene["p"], scene["sig2"], scene["rgb2"]
    R, M = p.packed_info.shape[0], p.n_samples
    w = torch.zeros(M, device="cuda")
    T = torch.zeros(M, device="cuda")
    _lib.render_weights(dev(p.packed_info), dev(p.t_starts), dev(p.t_ends), dev(sg), M, w, T)
    w_o, T_o = orc.render_weights(p.packed_info, p.t_starts, p.t_ends, sg)
    assert np.max(np.abs(w.cpu().numpy() - w_o)) <= 1e-5 and np.max(np.abs(T.cpu().numpy() - T_o)) <= 1e-5
    vals = np.concatenate([rgb, rgb[:, :1] * 2], 1).astype(np.float32)  # 4 channels
    out = torch.zeros((R, 4), device="cuda")
    _lib.accumulate_along_rays(dev(p.packed_info), dev(w_o.astype(np.float32)), dev(vals), 4, M, out)
    ref = orc.accumulate(p.packed_info, w_o.astype(np.float32).astype(np.float64), vals)
    assert np.max(np.abs(out.cpu().numpy() - ref)) <= 1e-5
    out1 = torch.zeros((R, 1), device="cuda")
    _lib.accumulate_along_rays(dev(p.packed_info), dev(w_o.astype(np.float32)), None, 1, M, out1)
    ref1 = orc.accumulate(p.packed_info, w_o.astype(np.float32).astype(np.float64))
    assert np.max(np.abs(out1.cpu().numpy() - ref1)) <= 1e-5


def _gpu_weights_bwd(pi, ts, te, sg, g):
    M = ts.shape[0]
    ds = torch.full((max(M, 1),), float("nan"), device="cuda")
    st = torch.zeros(1, dtype=torch.int32, device="cuda")
    _lib.render_weights_bwd(dev(pi), dev(ts), dev(te), dev(sg), M, dev(g), ds[:M], d_status=st)
    torch.cuda.synchronize()
    assert int(st.item()) == 0
    return ds[:M].cpu().numpy()


def test_render_weights_bwd_parity(scene, orc):
    """dL/dsigma for a random dL/dw on the pruned bounded samples (ragged rays)."""
    p, sg = scene["p"], scene["sig2"]
    M = p.n_samples
    g = synth.rand_uniform(5, 1, M, -1, 1).astype(np.float32)
    ds = _gpu_weights_bwd(p.packed_info, p.t_starts, p.t_ends, sg, g)
    ds_o = orc.render_weights_bwd(p.packed_info, p.t_starts, p.t_ends, sg, g.astype(np.float64))
    assert grad_rel_err(ds, ds_o) <= 1e-4


def test_render_weights_bwd_long_ray_and_empty(orc):
    """One ray of 9000 samples (past the shared-memory carry record), an empty ray, a one-sample ray."""
    n = 9000
    ts = np.concatenate([1.0 + 0.001 * np.arange(n), [3.0]]).astype(np.float32)
    te = np.concatenate([1.0 + 0.001 * np.arange(1, n + 1), [3.5]]).astype(np.float32)
    sg = synth.rand_uniform(6, 1, n + 1, 0, 2).astype(np.float32)
    g = synth.rand_uniform(6, 2, n + 1, -1, 1).astype(np.float32)
    pi = np.array([[0, n], [n, 0], [n, 1]], np.int32)
    ds = _gpu_weights_bwd(pi, ts, te, sg, g)
    ds_o = orc.render_weights_bwd(pi, ts, te, sg, g.astype(np.float64))
    assert grad_rel_err(ds, ds_o) <= 1e-4


@pytest.mark.parametrize("C", [1, 4, 7, 16, 33])
def test_accumulate_many_channels(scene, orc, C):
    """Per-ray sums of C-channel attributes (Sec. 2.2: any sample attribute), up to
    one channel past a warp's width, on the ragged pruned samples."""
    p = scene["p"]
    R, M = p.packed_info.shape[0], p.n_samples
    w = synth.rand_uniform(C, 21, M, 0, 1).astype(np.float32)
    vals = synth.rand_uniform(C, 22, M * C, -1, 1).reshape(M, C).astype(np.float32)
    out = torch.full((R, C), float("nan"), device="cuda")
    _lib.accumulate_along_rays(dev(p.packed_info), dev(w), dev(vals), C, M, out)
    torch.cuda.synchronize()
    ref = orc.accumulate(p.packed_info, w.astype(np.float64), vals)
    assert np.max(np.abs(out.cpu().numpy() - ref)) <= 1e-5 * max(1.0, np.abs(ref).max())


@pytest.mark.parametrize("C", [1, 3, 7, 16, 33])
def test_accumulate_bwd_parity(scene, orc, C):
    p, rgb = scene["p"], scene["rgb2"]
    R, M = p.packed_info.shape[0], p.n_samples
    w = synth.rand_uniform(C, 11, M, 0, 1).astype(np.float32)
    vals = None if C == 1 else synth.rand_uniform(C, 12, M * C, -1, 1).reshape(M, C).astype(np.float32)
    g = synth.rand_uniform(C, 13, R * C, -1, 1).reshape(R, C).astype(np.float32)
    dw = torch.full((M,), float("nan"), device="cuda")
    dv = None if vals is None else torch.full((M, C), float("nan"), device="cuda")
    _lib.accumulate_along_rays_bwd(dev(p.packed_info), dev(w), dev(vals), C, M, dev(g), dw, dv)
    torch.cuda.synchronize()
    dw_o, dv_o = orc.accumulate_bwd(p.packed_info, w.astype(np.float64), vals, g.astype(np.float64))
    assert np.max(np.abs(dw.cpu().numpy() - dw_o)) <= 1e-5 * max(1.0, np.abs(dw_o).max())
    if vals is not None:
        assert np.max(np.abs(dv.cpu().numpy() - dv_o)) <= 1e-6


@pytest.mark.parametrize("C", [1, 3, 7, 16, 33])
def test_accumulate_bwd_centred_then_weights_bwd(scene, orc, C):
    """Centred mode of the accumulation gradient: d_weights holds dL/dw_i minus the
    ray's first sample's value, which is added to g_ref (here on top of a seeded
    start value, to check that it adds). Fed to the weights gradient with g_ref,
    dL/dsigma meets the 1e-4 bar against the float64 oracle of the composition."""
    p, sg = scene["p"], scene["sig2"]
    R, M = p.packed_info.shape[0], p.n_samples
    w_o, _ = orc.render_weights(p.packed_info, p.t_starts, p.t_ends, sg)
    w = w_o.astype(np.float32)
    # values that vary little along a ray on top of a large common part: the case
    # where the uncentred float32 dL/dw loses the differences the scan needs
    base = synth.rand_uniform(C, 31, C, 0.5, 2.0).astype(np.float32)
    vals = None if C == 1 else (base[None, :] + synth.rand_uniform(C, 32, M * C, -1e-3, 1e-3).reshape(M, C)
                                ).astype(np.float32)
    g = synth.rand_uniform(C, 33, R * C, -1, 1).reshape(R, C).astype(np.float32)
    g_ref0 = synth.rand_uniform(C, 34, R, -0.5, 0.5).astype(np.float32)
    dw = torch.full((M,), float("nan"), device="cuda")
    g_ref = dev(g_ref0.copy())
    _lib.accumulate_along_rays_bwd(dev(p.packed_info), dev(w), dev(vals), C, M, dev(g), dw, None, g_ref=g_ref)
    torch.cuda.synchronize()
    dw_o, _ = orc.accumulate_bwd(p.packed_info, w.astype(np.float64), vals, g.astype(np.float64))
    first = np.repeat(p.packed_info[:, 0], p.packed_info[:, 1])
    ray = np.repeat(np.arange(R), p.packed_info[:, 1])
    has = p.packed_info[:, 1] > 0
    ref_ray = np.where(has, dw_o[np.minimum(p.packed_info[:, 0], max(M - 1, 0))], 0.0)
    got_ref = g_ref.cpu().numpy().astype(np.float64) - g_ref0
    assert np.max(np.abs(got_ref - ref_ray)) <= 1e-5 * max(1.0, np.abs(ref_ray).max())
    centred_o = dw_o - dw_o[first]
    spread = np.abs(centred_o).max() if M else 0.0
    assert np.max(np.abs(dw.cpu().numpy() - centred_o), initial=0.0) <= 1e-5 * max(spread, 1e-6)
    # the weights gradient from the two parts (g_ref holds the seeded start too)
    ds = torch.full((M,), float("nan"), device="cuda")
    _lib.render_weights_bwd(dev(p.packed_info), dev(p.t_starts), dev(p.t_ends), dev(sg), M, dw, ds,
                            g_ref=g_ref)
    torch.cuda.synchronize()
    g_full = dw_o + g_ref0[ray].astype(np.float64)
    ds_o = orc.render_weights_bwd(p.packed_info, p.t_starts, p.t_ends, sg, g_full)
    assert grad_rel_err(ds.cpu().numpy(), ds_o) <= 1e-4


def test_unpack_info(scene, orc):
    p = scene["p"]
    ri = torch.full((p.n_samples,), -1, dtype=torch.int32, device="cuda")
    _lib.unpack_info(dev(p.packed_info), p.n_samples, ri)
    assert np.array_equal(ri.cpu().numpy(), orc.unpack_info(p.packed_info, p.n_samples))


def test_render_bad_packed_info_is_reported():
    pi = np.array([[0, 3], [2, 10]], np.int32)  # second run exceeds n_samples = 5
    ts = np.arange(5, dtype=np.float32)
    col = torch.zeros((2, 3), device="cuda")
    op = torch.zeros(2, device="cuda")
    dp = torch.zeros(2, device="cuda")
    st = torch.zeros(1, dtype=torch.int32, device="cuda")
    _lib.render_fwd(dev(pi), dev(ts), dev(ts + 1), dev(ts), dev(np.zeros((5, 3), np.float32)), 5, col, op, dp,
                    d_status=st)
    torch.cuda.synchronize()
    assert int(st.item()) & _lib.STATUS_BAD_PACKED
    assert op.cpu().numpy()[1] == 0.0


@pytest.mark.parametrize("n_cells,shift", [(64 ** 3, 0), (1000, 0), (33, 0), (128 * 77 + 96, 0), (1000, 1),
                                           (64 ** 3, 3)])
def test_grid_update_bitexact(orc, n_cells, shift):
    """Whole 128-cell steps (16-byte aligned state, four cells per thread), ragged
    tails and unaligned states (one cell per thread) give the oracle's grid."""
    ema = synth.rand_uniform(5, 1, n_cells, 0, 0.03).astype(np.float32)
    n = 1 << 16
    cells = synth.rand_int(5, 2, n, n_cells).astype(np.int32)
    sig = (synth.rand_uniform(5, 3, n) ** 3 * 0.05).astype(np.float32)
    sig[::97] = np.nan
    sig[1::89] = -1.0
    e_t = dev(np.concatenate([np.zeros(shift, np.float32), ema]))[shift:]  # shift > 0: not 16-byte aligned
    b_t = torch.zeros((n_cells + 31) // 32, dtype=torch.int32, device="cuda")
    st = torch.zeros(1, dtype=torch.int32, device="cuda")
    _lib.update_occupancy_grid(e_t, b_t, dev(cells), dev(sig), 0.95, 0.01, st)
    torch.cuda.synchronize()
    e_o, b_o = orc.update_grid(ema, cells, sig, 0.95, 0.01)
    assert int(st.item()) == 0
    assert bits_equal(e_t.cpu().numpy(), e_o)
    assert np.array_equal(b_t.cpu().numpy().view(np.uint32), b_o)


def test_grid_update_bad_cell_reported():
    e_t = torch.zeros(100, device="cuda")
    b_t = torch.zeros(4, dtype=torch.int32, device="cuda")
    st = torch.zeros(1, dtype=torch.int32, device="cuda")
    _lib.update_occupancy_grid(e_t, b_t, dev(np.array([3, 100, -1], np.int32)), dev(np.ones(3, np.float32)), 0.9,
                               0.5, st)
    torch.cuda.synchronize()
    assert int(st.item()) & _lib.STATUS_BAD_INDEX
    assert e_t.cpu().numpy()[3] == 1.0


def test_alpha_accuracy_single_sample_rays():
    """w = alpha = 1 - exp(-tau) for one-sample rays (T = 1): relative error below 4e-6
    and absolute error below 2.5e-7 against float64, for tau from 1e-9 to 40 (the
    kernels' own series/exponential split, checked against the exact function)."""
    tau = np.concatenate([np.geomspace(1e-9, 40.0, 4001), [0.0625, np.nextafter(np.float32(0.0625), 0)]])
    n = tau.size
    ts = np.zeros(n, np.float32)
    te = np.ones(n, np.float32)
    sg = tau.astype(np.float32)
    pi = np.stack([np.arange(n), np.ones(n)], 1).astype(np.int32)
    w = torch.zeros(n, device="cuda")
    T = torch.zeros(n, device="cuda")
    _lib.render_weights(dev(pi), dev(ts), dev(te), dev(sg), n, w, T)
    exact = -np.expm1(-sg.astype(np.float64))
    got = w.cpu().numpy().astype(np.float64)
    assert np.all(T.cpu().numpy() == 1.0)
    assert np.max(np.abs(got - exact)) <= 2.5e-7
    assert np.max(np.abs(got - exact) / np.maximum(exact, 1e-300)) <= 4e-6


@pytest.mark.parametrize("tile_rays", [2, 4, 8, 32])
def test_prune_uneven_rays_every_tile_shape(orc, tile_rays):
    """Runs of very different lengths (empty, one sample, thousands) side by side in
    every tile shape: the decision walk refills a freed slot with the tile's next
    ray, and the result must not depend on how rays share a warp."""
    rng = np.random.default_rng(41)
    lens = rng.choice([0, 0, 1, 2, 33, 63, 64, 65, 500, 3000], size=700)
    off = np.concatenate([[0], np.cumsum(lens)[:-1]])
    pi = np.stack([off, lens], axis=1).astype(np.int32)
    M = int(lens.sum())
    ts = np.zeros(M, np.float32)
    for o, c in pi:
        ts[o : o + c] = np.arange(c, dtype=np.float32) * np.float32(0.01) + np.float32(0.5)
    te = (ts + np.float32(0.01)).astype(np.float32)
    sg = (rng.random(M) ** 4 * 60).astype(np.float32)  # mostly thin, some opaque: early stops at many depths
    p, keep, od = orc.prune(pi, ts, te, sg, 1e-4, 1e-2)
    old = _lib.tune_get("prune_tile_rays")
    try:
        _lib.tune_set("prune_tile_rays", tile_rays)
        g = _gpu_prune(pi, ts, te, sg, 1e-4, 1e-2)
    finally:
        _lib.tune_set("prune_tile_rays", old)
    assert g["st"][0] == 0
    keep_g = g["keep"][:M].astype(bool)
    near = near_threshold(pi, ts, te, sg, 1e-4, od)
    assert not ((keep_g != keep) & ~near).any()
    flipped = set(np.searchsorted(pi[:, 0], np.nonzero(keep_g != keep)[0], side="right") - 1)
    for r in range(len(lens)):
        if r in flipped:
            continue
        (og, cg), (oo, co) = g["pi"][r], p.packed_info[r]
        assert cg == co and bits_equal(g["ts"][og : og + cg], p.t_starts[oo : oo + co])
        assert np.all(g["ri"][og : og + cg] == r)
    assert len(flipped) <= 2 and p.n_samples > 1000


@pytest.mark.parametrize("shift", [(0, 0, 0), (2, 2, 2), (0, 2, 0), (2, 0, 2), (0, 0, 2), (2, 2, 0)])
def test_prune_alignment_phases(orc, shift):
    """Input arrays at different addresses modulo 16 (each 8-byte aligned, as the
    ABI accepts), with runs starting at every offset modulo 4: results equal the
    oracle's whatever the arrays' relative alignment."""
    rng = np.random.default_rng(7)
    lens = rng.choice([0, 1, 2, 3, 5, 63, 64, 65, 66, 67, 130, 700], size=400)
    off = np.concatenate([[0], np.cumsum(lens)[:-1]])
    pi = np.stack([off, lens], axis=1).astype(np.int32)
    M = int(lens.sum())
    ts = np.zeros(M, np.float32)
    for o, c in pi:
        ts[o : o + c] = np.arange(c, dtype=np.float32) * np.float32(0.01) + np.float32(0.25)
    te = (ts + np.float32(0.01)).astype(np.float32)
    sg = (rng.random(M) ** 3 * 80).astype(np.float32)
    p, keep, od = orc.prune(pi, ts, te, sg, 1e-4, 1e-2)

    def shifted(x, k):
        buf = torch.zeros(M + 4, dtype=torch.float32, device="cuda")
        buf[k : k + M] = torch.from_numpy(x).cuda()
        return buf[k : k + M]

    d_ts, d_te, d_sg = shifted(ts, shift[0]), shifted(te, shift[1]), shifted(sg, shift[2])
    R = pi.shape[0]
    ws = torch.zeros(_lib.prune_workspace_size(R, M), dtype=torch.uint8, device="cuda")
    o_pi = torch.full((R, 2), -3, dtype=torch.int32, device="cuda")
    o_ts, o_te = torch.zeros(M, device="cuda"), torch.zeros(M, device="cuda")
    o_ri = torch.zeros(M, dtype=torch.int32, device="cuda")
    n = torch.zeros(1, dtype=torch.int64, device="cuda")
    st = torch.zeros(1, dtype=torch.int32, device="cuda")
    km = torch.full((M,), 7, dtype=torch.uint8, device="cuda")
    _lib.prune_samples(dev(pi), d_ts, d_te, d_sg, M, 1e-4, 1e-2, o_pi, o_ts, o_te, o_ri, n, st, ws, keep_mask=km)
    torch.cuda.synchronize()
    assert int(st.item()) == 0
    keep_g = km.cpu().numpy().astype(bool)
    near = near_threshold(pi, ts, te, sg, 1e-4, od)
    assert not ((keep_g != keep) & ~near).any()
    flipped = set(np.searchsorted(pi[:, 0], np.nonzero(keep_g != keep)[0], side="right") - 1)
    g_pi, g_ts, g_ri = o_pi.cpu().numpy(), o_ts.cpu().numpy(), o_ri.cpu().numpy()
    for r in range(R):
        if r in flipped:
            continue
        (og, cg), (oo, co) = g_pi[r], p.packed_info[r]
        assert cg == co and bits_equal(g_ts[og : og + cg], p.t_starts[oo : oo + co])
        assert np.all(g_ri[og : og + cg] == r)
    assert len(flipped) <= 2 and int(n.item()) == int(keep_g.sum()) and p.n_samples > 1000

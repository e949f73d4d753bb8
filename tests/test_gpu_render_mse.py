"""Forward, squared-error loss gradient and backward in one pass
(nacc_render_mse_fused) against the separate calls (nacc_render_fwd, the
gradient (C - C*) * s formed in float32, nacc_render_bwd) and the oracle:
identical colours, opacities, depths and gradients, on pruned and unpruned rays,
odd run starts, gaps between runs, empty rays and a ray longer than the
shared-memory record of chunk carries."""
import numpy as np
import pytest

from paper_2210_04847_gb300 import _lib, synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no CUDA device", allow_module_level=True)

from gpu_util import bits_equal, dev, grad_rel_err, oracle_march, render_tol_ok  # noqa: E402


def _separate(pi, ts, te, sg, rgb, tgt, scale):
    """nacc_render_fwd, the loss gradient as torch forms it, nacc_render_bwd (recomputed O)."""
    R, M = pi.shape[0], ts.shape[0]
    d = [dev(x) for x in (ts, te, sg, rgb)]
    col = torch.zeros((R, 3), device="cuda")
    op = torch.zeros(R, device="cuda")
    dp = torch.zeros(R, device="cuda")
    st = torch.zeros(1, dtype=torch.int32, device="cuda")
    _lib.render_fwd(dev(pi), *d, M, col, op, dp, d_status=st)
    g = torch.sub(col, dev(tgt))
    g.mul_(scale)
    ds = torch.full((max(M, 1),), np.nan, device="cuda")
    dr = torch.full((max(M, 1), 3), np.nan, device="cuda")
    _lib.render_bwd(dev(pi), *d, M, g, None, None, ds[:M], dr[:M], d_status=st)
    torch.cuda.synchronize()
    assert int(st.item()) == 0
    return dict(col=col.cpu().numpy(), op=op.cpu().numpy(), dp=dp.cpu().numpy(), ds=ds.cpu().numpy()[:M],
                dr=dr.cpu().numpy()[:M], g=g.cpu().numpy())


def _fused(pi, ts, te, sg, rgb, tgt, scale):
    R, M = pi.shape[0], ts.shape[0]
    d = [dev(x) for x in (ts, te, sg, rgb)]
    col = torch.full((R, 3), np.nan, device="cuda")
    op = torch.full((R,), np.nan, device="cuda")
    dp = torch.full((R,), np.nan, device="cuda")
    se = torch.full((R,), np.nan, device="cuda")
    ds = torch.full((max(M, 1),), np.nan, device="cuda")
    dr = torch.full((max(M, 1), 3), np.nan, device="cuda")
    st = torch.zeros(1, dtype=torch.int32, device="cuda")
    _lib.render_mse_fused(dev(pi), *d, M, dev(tgt), scale, col, ds[:M], dr[:M], opacity=op, depth=dp, sq_err=se,
                          d_status=st)
    torch.cuda.synchronize()
    assert int(st.item()) == 0
    return dict(col=col.cpu().numpy(), op=op.cpu().numpy(), dp=dp.cpu().numpy(), ds=ds.cpu().numpy()[:M],
                dr=dr.cpu().numpy()[:M], se=se.cpu().numpy())


def _check(orc, pi, ts, te, sg, rgb, seed):
    R = pi.shape[0]
    tgt = synth.rand_uniform(seed, 7, 3 * R).reshape(R, 3).astype(np.float32)
    scale = float(np.float32(2.0 / (3.0 * R)))
    ref = _separate(pi, ts, te, sg, rgb, tgt, scale)
    got = _fused(pi, ts, te, sg, rgb, tgt, scale)
    for k in ("col", "op", "dp", "ds", "dr"):
        assert bits_equal(got[k], ref[k]), k
    e = (ref["col"] - tgt).astype(np.float32)
    assert np.allclose(got["se"], (e * e).sum(1), rtol=1e-6, atol=0)
    # the oracle: colours at 1e-5, gradients for the oracle's own loss gradient at 1e-4
    c_o, a_o, d_o = orc.render_fwd(pi, ts, te, sg, rgb)
    assert render_tol_ok(got["col"], c_o, rel_for_large=False) <= 1.0
    assert render_tol_ok(got["op"], a_o, rel_for_large=False) <= 1.0
    assert render_tol_ok(got["dp"], d_o) <= 1.0
    ds_o, dr_o = orc.render_bwd(pi, ts, te, sg, rgb, (c_o - tgt.astype(np.float64)) * (2.0 / (3.0 * R)))
    covered = np.zeros(ts.shape[0], bool)
    for o, n in pi:
        covered[o:o + n] = True
    assert grad_rel_err(got["ds"][covered], ds_o[covered]) <= 1e-4
    assert grad_rel_err(got["dr"][covered], dr_o[covered]) <= 1e-4
    assert np.all(np.isnan(got["ds"][~covered]))


@pytest.fixture(scope="module")
def scene(orc):
    w = synth.bounded_config(8, n_rays=1501, device="cuda")
    m = oracle_march(orc, w)
    sig, rgb = synth.sample_field(w.scenes[0], w.rays_o, w.rays_d, m.t_starts, m.t_ends, m.ray_indices)
    p, _, _ = orc.prune(m.packed_info, m.t_starts, m.t_ends, sig, w.early_stop_eps, w.alpha_thre)
    sig2, rgb2 = synth.sample_field(w.scenes[0], w.rays_o, w.rays_d, p.t_starts, p.t_ends, p.ray_indices)
    return dict(m=m, sig=sig, rgb=rgb, p=p, sig2=sig2, rgb2=rgb2)


@pytest.mark.parametrize("occupancy", [0, 1, 2])
def test_fused_equals_separate_pruned(scene, orc, occupancy):
    p = scene["p"]
    old = _lib.tune_get("render_mse_occupancy")
    try:
        _lib.tune_set("render_mse_occupancy", occupancy)
        _check(orc, p.packed_info, p.t_starts, p.t_ends, scene["sig2"], scene["rgb2"], 1)
    finally:
        _lib.tune_set("render_mse_occupancy", old)


def test_fused_equals_separate_unpruned(scene, orc):
    m = scene["m"]
    _check(orc, m.packed_info, m.t_starts, m.t_ends, scene["sig"], scene["rgb"], 2)


def test_fused_edges_and_long_ray(orc):
    """Odd starts, gaps, empty rays, and a ray of 9000 samples (more chunks than the
    shared-memory record of carries)."""
    lens = [0, 1, 2, 63, 64, 65, 129, 0, 9000, 3, 200]
    runs, off = [], 1
    for i, n in enumerate(lens):
        runs.append((off, n))
        off += n + (i % 3)
    n_samples = off + 5
    pi = np.array(runs, np.int32)
    t = np.arange(n_samples + 1, dtype=np.float64)
    ts = (0.5 + 0.001 * t[:-1]).astype(np.float32)
    te = (0.5 + 0.001 * t[1:]).astype(np.float32)
    sg = synth.rand_uniform(31, 1, n_samples, 0, 1).astype(np.float32)
    rgb = synth.rand_uniform(31, 2, 3 * n_samples).reshape(n_samples, 3).astype(np.float32)
    _check(orc, pi, ts, te, sg, rgb, 3)


def test_fused_rejects_bad_arguments():
    z = torch.zeros(8, device="cuda")
    pi = torch.zeros((2, 2), dtype=torch.int32, device="cuda")
    lib = _lib.load()
    P = _lib._ptr
    # a non-finite gradient scale, a missing target
    assert lib.nacc_render_mse_fused(P(pi), 2, P(z), P(z), P(z), P(z), 2, P(z), float("inf"), None, None, None, None,
                                     P(z), P(z), None, None) == _lib.ERR_INVALID_ARG
    assert lib.nacc_render_mse_fused(P(pi), 2, P(z), P(z), P(z), P(z), 2, None, 1.0, None, None, None, None,
                                     P(z), P(z), None, None) == _lib.ERR_INVALID_ARG


def test_api_fused_loss_matches_autograd_of_the_separate_calls(scene):
    """api.render_packed_mse against render_packed followed by torch's MSE loss:
    the same loss and, through autograd, the same gradients (up to the order of
    the loss gradient's float32 operations)."""
    from paper_2210_04847_gb300 import api
    p = scene["p"]
    R = p.packed_info.shape[0]
    tgt = dev(synth.rand_uniform(5, 8, 3 * R).reshape(R, 3).astype(np.float32))
    pi, ts, te = dev(p.packed_info), dev(p.t_starts), dev(p.t_ends)
    s1 = dev(scene["sig2"]).requires_grad_(True)
    r1 = dev(scene["rgb2"]).requires_grad_(True)
    col, _, _ = api.render_packed(s1, r1, pi, ts, te)
    l1 = torch.nn.functional.mse_loss(col, tgt)
    (3.0 * l1).backward()  # an upstream gradient other than one
    s2 = dev(scene["sig2"]).requires_grad_(True)
    r2 = dev(scene["rgb2"]).requires_grad_(True)
    l2, col2, _, _ = api.render_packed_mse(s2, r2, pi, ts, te, tgt)
    (3.0 * l2).backward()
    assert torch.equal(col, col2)
    assert abs(float(l1.detach()) - float(l2.detach())) <= 1e-6 * abs(float(l1.detach()))
    assert grad_rel_err(s2.grad.cpu().numpy(), s1.grad.cpu().numpy()) <= 1e-5
    assert grad_rel_err(r2.grad.cpu().numpy(), r1.grad.cpu().numpy()) <= 1e-5

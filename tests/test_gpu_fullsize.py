"""Parity at the benchmark's full size and launch configuration (2^18 rays of the
bounded workload through pipeline.HotPath, the buffers and calls bench.py times;
a whole 800x800 image through the fused inference path).

The oracle cannot march 2^18 rays x 1024 steps and render them inside a test, so
it checks a seeded sample of rays one by one (marching of a ray depends on that ray
alone; pruning and rendering of a ray on its own samples). The stand-in field's
values for the sampled rays are replaced by the host generator's before pruning and
before rendering, so every oracle input comes from the seeded generators. Whole-
batch properties are checked on the device. The full-size grid update is compared
bit-exactly over the whole grid.
"""
import math

import numpy as np
import pytest

from paper_2210_04847_gb300 import _lib, synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no CUDA device", allow_module_level=True)

from gpu_util import bits_equal, grad_rel_err, render_tol_ok  # noqa: E402
from paper_2210_04847_gb300.pipeline import HotPath, StandInField, to_device  # noqa: E402

R = 1 << 18
N_SAMPLE = 48


@pytest.fixture(scope="module")
def run(orc):
    scene, aabb, bits = synth.bounded_scene(0, device="cuda")
    w = synth.bounded_config(0, n_rays=R, scene_grid=(scene, aabb, bits), batch=0)
    hp = HotPath(w, cap_marched=170_000_000, cap_kept=45_000_000, n_grid_samples=0)
    field = StandInField(scene)
    o, d = to_device(w.rays_o), to_device(w.rays_d)
    hp.march(o, d)
    torch.cuda.synchronize()
    M = int(hp.n_m.item())
    hp.check_status("march")
    sample = np.sort(synth.rand_int(99, 1, N_SAMPLE, R).astype(np.int64))
    sub = (w.rays_o[sample], w.rays_d[sample])
    om = orc.march(sub[0], sub[1], w.bits, w.res, w.aabb, w.near_plane, w.far_plane, w.dt_min, w.dt_max, w.cone,
                   w.max_steps)
    pi_m = hp.pi_m.cpu().numpy()
    return dict(w=w, hp=hp, field=field, o=o, d=d, M=M, sample=sample, om=om, pi_m=pi_m, scene=scene)


def _gather(t, off, cnt):
    return t[off : off + cnt].cpu().numpy()


def test_fullsize_march_sampled_rays_bitexact(run):
    hp, om, pi_m = run["hp"], run["om"], run["pi_m"]
    assert run["M"] > 100_000_000
    for k, r in enumerate(run["sample"]):
        off, cnt = pi_m[r]
        ooff, ocnt = om.packed_info[k]
        assert cnt == ocnt, (r, cnt, ocnt)
        assert bits_equal(_gather(hp.ts_m, off, cnt), om.t_starts[ooff : ooff + ocnt])
        assert bits_equal(_gather(hp.te_m, off, cnt), om.t_ends[ooff : ooff + ocnt])
        assert np.all(_gather(hp.ri_m, off, cnt) == r)


def test_fullsize_march_whole_batch_properties(run):
    hp, M = run["hp"], run["M"]
    pi = hp.pi_m.long()
    off, cnt = pi[:, 0], pi[:, 1]
    assert int(cnt.sum()) == M
    assert int(off[0]) == 0 and bool(torch.all(off[1:] == off[:-1] + cnt[:-1]))
    ts, te, ri = hp.ts_m[:M], hp.te_m[:M], hp.ri_m[:M].long()
    assert bool(torch.all(te > ts))
    expect_ri = torch.repeat_interleave(torch.arange(R, device="cuda"), cnt)
    assert bool(torch.all(ri == expect_ri))
    # intervals of a ray are ordered and never overlap
    same = ri[1:] == ri[:-1]
    assert bool(torch.all(ts[1:][same] >= te[:-1][same]))


def test_fullsize_prune_render_backward_sampled_rays(run, orc):
    w, hp, field, o, d, M = run["w"], run["hp"], run["field"], run["o"], run["d"], run["M"]
    sample, om, pi_m, scene = run["sample"], run["om"], run["pi_m"], run["scene"]
    sub_o, sub_d = w.rays_o[sample], w.rays_d[sample]
    # densities: stand-in field everywhere, host generator values for the sampled rays
    hp.field_marched(field, o, d, M)
    sig_o, _ = synth.sample_field(scene, sub_o, sub_d, om.t_starts, om.t_ends, om.ray_indices)
    for k, r in enumerate(sample):
        off, cnt = pi_m[r]
        ooff, ocnt = om.packed_info[k]
        hp.sig_m[off : off + cnt] = torch.from_numpy(sig_o[ooff : ooff + ocnt]).cuda()
    hp.prune(M)
    torch.cuda.synchronize()
    S = int(hp.n_k.item())
    hp.check_status("prune")
    op_, keep, od = orc.prune(om.packed_info, om.t_starts, om.t_ends, sig_o, w.early_stop_eps, w.alpha_thre)
    pi_k = hp.pi_k.cpu().numpy()
    thr = -math.log(w.early_stop_eps)
    same_rays = []
    for k, r in enumerate(sample):
        off, cnt = pi_k[r]
        ooff, ocnt = op_.packed_info[k]
        if cnt != ocnt:
            # only a decision within the float32 summation bound of the threshold may differ
            moff, mcnt = om.packed_info[k]
            tau = sig_o[moff : moff + mcnt].astype(np.float64) * (om.t_ends[moff : moff + mcnt].astype(np.float64)
                                                                 - om.t_starts[moff : moff + mcnt])
            near = np.abs(od[moff : moff + mcnt] - thr) <= (np.arange(mcnt) + 40) * 2.0**-23 * np.cumsum(np.abs(tau))
            assert abs(int(cnt) - int(ocnt)) <= int(near.sum()), r
            continue
        assert bits_equal(_gather(hp.ts_k, off, cnt), op_.t_starts[ooff : ooff + ocnt])
        assert bits_equal(_gather(hp.te_k, off, cnt), op_.t_ends[ooff : ooff + ocnt])
        same_rays.append((k, r))
    assert len(same_rays) >= N_SAMPLE - 2
    # field with gradient: stand-in everywhere, generator values for the sampled rays
    hp.field_kept(field, o, d, S)
    sig2, rgb2 = synth.sample_field(scene, sub_o, sub_d, op_.t_starts, op_.t_ends, op_.ray_indices)
    for k, r in same_rays:
        off, cnt = pi_k[r]
        ooff, ocnt = op_.packed_info[k]
        hp.sig_k[off : off + cnt] = torch.from_numpy(sig2[ooff : ooff + ocnt]).cuda()
        hp.rgb_k[off : off + cnt] = torch.from_numpy(rgb2[ooff : ooff + ocnt]).cuda()
    hp.render_fwd(S)
    gc = synth.rand_uniform(8, 1, 3 * R, -1, 1).reshape(R, 3).astype(np.float32) / R
    hp.g_color.copy_(torch.from_numpy(gc))
    hp.render_bwd(S)
    torch.cuda.synchronize()
    hp.check_status("render")
    c_o, a_o, d_o = orc.render_fwd(op_.packed_info, op_.t_starts, op_.t_ends, sig2, rgb2)
    gsub = gc[sample].astype(np.float64)
    ds_o, dr_o = orc.render_bwd(op_.packed_info, op_.t_starts, op_.t_ends, sig2, rgb2, gsub)
    col = hp.color.cpu().numpy()
    opa = hp.opacity.cpu().numpy()
    dep = hp.depth.cpu().numpy()
    ds_all, dr_all, ref_s, ref_r = [], [], [], []
    for k, r in same_rays:
        assert render_tol_ok(col[r], c_o[k], rel_for_large=False) <= 1.0
        assert render_tol_ok(opa[r], a_o[k], rel_for_large=False) <= 1.0
        assert render_tol_ok(dep[r], d_o[k]) <= 1.0
        off, cnt = pi_k[r]
        ooff, ocnt = op_.packed_info[k]
        ds_all.append(_gather(hp.d_sig, off, cnt))
        dr_all.append(hp.d_rgb[off : off + cnt].cpu().numpy())
        ref_s.append(ds_o[ooff : ooff + ocnt])
        ref_r.append(dr_o[ooff : ooff + ocnt])
    assert grad_rel_err(np.concatenate(ds_all), np.concatenate(ref_s)) <= 1e-4
    assert grad_rel_err(np.concatenate(dr_all), np.concatenate(ref_r)) <= 1e-4


def test_fullsize_grid_update_bitexact(orc):
    """128^3 float32 EMA grid, 2^21 uniform random cells (the benchmark's update), decay 0.95, threshold 0.01."""
    n_cells = 128 ** 3
    scene, aabb, _ = synth.bounded_scene(0, device="cuda")
    ema = synth.density_at_cell_centres(scene, aabb, (128, 128, 128), device="cuda").float().cpu().numpy()
    cells, jit = synth.grid_update_samples(0, 0, 1 << 21, (128, 128, 128))
    xyz = synth.cell_positions(cells, jit, aabb, (128, 128, 128))
    sig = scene.density(xyz).astype(np.float32)
    e_t = torch.from_numpy(ema.copy()).cuda()
    b_t = torch.zeros(n_cells // 32, dtype=torch.int32, device="cuda")
    st = torch.zeros(1, dtype=torch.int32, device="cuda")
    _lib.update_occupancy_grid(e_t, b_t, torch.from_numpy(cells).cuda(), torch.from_numpy(sig).cuda(), 0.95, 0.01, st)
    e_o, b_o = orc.update_grid(ema, cells, sig, 0.95, 0.01)
    torch.cuda.synchronize()
    assert int(st.item()) == 0
    assert bits_equal(e_t.cpu().numpy(), e_o)
    assert np.array_equal(b_t.cpu().numpy().view(np.uint32), b_o)


def test_fullsize_fused_inference_image_sampled_rays(orc):
    """The fused inference path on a whole 800x800 image (the launch bench.py
    --workload inference times): sampled rays against the oracle (march -> density
    at the midpoints -> prune), bit-exact except rays with a decision within
    float32 summation error of -ln(eps); whole-image packing properties on the
    device."""
    from gpu_util import near_threshold

    w = synth.inference_config(0, camera=0)
    Rf = w.n_rays
    o, d = to_device(w.rays_o), to_device(w.rays_d)
    bits = to_device(w.bits)
    grid = _lib.make_grid(bits, w.res, w.aabb, 1, 1, 0)
    params = _lib.make_params(w.near_plane, w.far_plane, w.dt_min, w.dt_max, w.cone, w.max_steps)
    field_t = to_device(w.field)
    fld = _lib.make_density_field(field_t, w.field_box)
    ws = torch.zeros(_lib.march_workspace_size(Rf, params), dtype=torch.uint8, device="cuda")
    cap = 100_000_000
    pi = torch.zeros((Rf, 2), dtype=torch.int32, device="cuda")
    ts, te, sg = (torch.zeros(cap, device="cuda") for _ in range(3))
    ri = torch.zeros(cap, dtype=torch.int32, device="cuda")
    n = torch.zeros(1, dtype=torch.int64, device="cuda")
    st = torch.zeros(1, dtype=torch.int32, device="cuda")
    _lib.march_fused(o, d, grid, params, fld, w.early_stop_eps, w.alpha_thre, pi, ts, te, ri, sg, n, st, ws)
    torch.cuda.synchronize()
    S = int(n.item())
    assert int(st.item()) == 0 and 50_000_000 < S < cap
    # whole image: contiguous runs, ray indices, ordered non-overlapping intervals, sigma > 0 where kept
    pl = pi.long()
    assert int(pl[:, 1].sum()) == S and bool(torch.all(pl[1:, 0] == pl[:-1, 0] + pl[:-1, 1]))
    assert bool(torch.all(ri[:S].long() == torch.repeat_interleave(torch.arange(Rf, device="cuda"), pl[:, 1])))
    same = ri[1:S] == ri[: S - 1]
    assert bool(torch.all(ts[1:S][same] >= te[: S - 1][same])) and bool(torch.all(sg[:S] > 0))
    # sampled rays against the oracle
    sample = np.sort(synth.rand_int(98, 1, 64, Rf).astype(np.int64))
    so, sd = w.rays_o[sample], w.rays_d[sample]
    m = orc.march(so, sd, w.bits, w.res, w.aabb, w.near_plane, w.far_plane, w.dt_min, w.dt_max, w.cone, w.max_steps)
    mid = ((m.t_starts + m.t_ends) * np.float32(0.5)).astype(np.float32)
    sig = orc.field_query(w.field, w.field_box, (so[m.ray_indices] + sd[m.ray_indices] * mid[:, None]).astype(np.float32))
    p, keep, od = orc.prune(m.packed_info, m.t_starts, m.t_ends, sig, w.early_stop_eps, w.alpha_thre)
    near = near_threshold(m.packed_info, m.t_starts, m.t_ends, sig, w.early_stop_eps, od)
    pin = pi.cpu().numpy()
    kept_sig = sig[keep]
    flipped = 0
    for k, r in enumerate(sample):
        off, cnt = pin[r]
        ooff, ocnt = p.packed_info[k]
        if cnt == ocnt and bits_equal(_gather(ts, off, cnt), p.t_starts[ooff : ooff + ocnt]):
            assert bits_equal(_gather(te, off, cnt), p.t_ends[ooff : ooff + ocnt])
            assert bits_equal(_gather(sg, off, cnt), kept_sig[ooff : ooff + ocnt])
            continue
        mo, mc = m.packed_info[k]
        assert near[mo : mo + mc].any(), "ray %d differs away from the early-stop threshold" % r
        flipped += 1
    assert flipped <= 1
    assert p.n_samples > 1000

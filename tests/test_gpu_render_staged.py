"""Render passes with the chunks staged in shared memory by bulk copies
(knobs render_fwd_stages / render_bwd_stages) against the register path and the
oracle: bit-identical colour, opacity, depth, optical depth and gradients, on
pruned and unpruned rays, long rays, odd run starts, gaps between runs, a last
ray that ends in the arrays' final partial 16 bytes, and arrays not 16-byte
aligned (which take the register path)."""
import numpy as np
import pytest

from paper_2210_04847_gb300 import _lib, synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no CUDA device", allow_module_level=True)

from gpu_util import bits_equal, grad_rel_err, oracle_march, render_tol_ok  # noqa: E402

STAGES = (2, 3, 4)


def _dev_at(a, shift=0):
    """float32/int32 array on the device, starting `shift` elements into its buffer."""
    a = np.ascontiguousarray(a)
    flat = a.reshape(-1)
    per = int(np.prod(a.shape[1:])) if a.ndim > 1 else 1
    buf = torch.zeros(flat.size + shift * per + 8, dtype=torch.float32 if a.dtype == np.float32 else torch.int32,
                      device="cuda")
    t = buf[shift * per: shift * per + flat.size]
    t.copy_(torch.from_numpy(flat))
    return t.view(*a.shape) if a.ndim > 1 else t


def _fwd_bwd(pi, ts, te, sg, rgb, gc, ga, gd, fwd_stages, bwd_stages, shift=0):
    """Forward (saving O) then backward from the saved O, under the given knob values."""
    old = _lib.tune_get("render_fwd_stages"), _lib.tune_get("render_bwd_stages")
    try:
        _lib.tune_set("render_fwd_stages", fwd_stages)
        _lib.tune_set("render_bwd_stages", bwd_stages)
        R, M = pi.shape[0], ts.shape[0]
        d = [_dev_at(x, shift) for x in (ts, te, sg, rgb)]
        dpi = _dev_at(pi)
        col = torch.full((R, 3), np.nan, device="cuda")
        op = torch.full((R,), np.nan, device="cuda")
        dp = torch.full((R,), np.nan, device="cuda")
        od = _dev_at(np.full(M, np.nan, np.float32), shift)
        st = torch.zeros(1, dtype=torch.int32, device="cuda")
        _lib.render_fwd(dpi, *d, M, col, op, dp, optical_depth=od, d_status=st)
        ds = torch.full((max(M, 1),), np.nan, device="cuda")
        dr = torch.full((max(M, 1), 3), np.nan, device="cuda")
        g = [None if x is None else _dev_at(x) for x in (gc, ga, gd)]
        _lib.render_bwd(dpi, *d, M, *g, ds[:M], dr[:M], optical_depth=od, d_status=st)
        torch.cuda.synchronize()
        assert int(st.item()) == 0
        return dict(col=col.cpu().numpy(), op=op.cpu().numpy(), dp=dp.cpu().numpy(), od=od.cpu().numpy(),
                    ds=ds.cpu().numpy()[:M], dr=dr.cpu().numpy()[:M])
    finally:
        _lib.tune_set("render_fwd_stages", old[0])
        _lib.tune_set("render_bwd_stages", old[1])


def _same(a, b):
    for k in ("col", "op", "dp", "od", "ds", "dr"):
        assert bits_equal(a[k], b[k]), k


def _grads(R, seed):
    gc = synth.rand_uniform(seed, 1, 3 * R, -1, 1).reshape(R, 3).astype(np.float32) / R
    ga = synth.rand_uniform(seed, 2, R, -1, 1).astype(np.float32) / R
    gd = synth.rand_uniform(seed, 3, R, -1, 1).astype(np.float32) / R
    return gc, ga, gd


@pytest.fixture(scope="module")
def scene(orc):
    w = synth.bounded_config(5, n_rays=1999, device="cuda")
    m = oracle_march(orc, w)
    sig, rgb = synth.sample_field(w.scenes[0], w.rays_o, w.rays_d, m.t_starts, m.t_ends, m.ray_indices)
    p, _, _ = orc.prune(m.packed_info, m.t_starts, m.t_ends, sig, w.early_stop_eps, w.alpha_thre)
    sig2, rgb2 = synth.sample_field(w.scenes[0], w.rays_o, w.rays_d, p.t_starts, p.t_ends, p.ray_indices)
    return dict(w=w, m=m, sig=sig, rgb=rgb, p=p, sig2=sig2, rgb2=rgb2)


@pytest.mark.parametrize("nst", STAGES)
def test_staged_equals_register_pruned(scene, orc, nst):
    p = scene["p"]
    pi, ts, te, sg, rgb = p.packed_info, p.t_starts, p.t_ends, scene["sig2"], scene["rgb2"]
    gc, ga, gd = _grads(pi.shape[0], 11)
    ref = _fwd_bwd(pi, ts, te, sg, rgb, gc, ga, gd, 0, 0)
    got = _fwd_bwd(pi, ts, te, sg, rgb, gc, ga, gd, nst, nst)
    _same(got, ref)
    c_o, a_o, d_o = orc.render_fwd(pi, ts, te, sg, rgb)
    assert render_tol_ok(got["col"], c_o, rel_for_large=False) <= 1.0
    assert render_tol_ok(got["op"], a_o, rel_for_large=False) <= 1.0
    assert render_tol_ok(got["dp"], d_o) <= 1.0
    ds_o, dr_o = orc.render_bwd(pi, ts, te, sg, rgb, gc.astype(np.float64), ga.astype(np.float64),
                                gd.astype(np.float64))
    assert grad_rel_err(got["ds"], ds_o) <= 1e-4 and grad_rel_err(got["dr"], dr_o) <= 1e-4


@pytest.mark.parametrize("nst", STAGES)
def test_staged_equals_register_unpruned(scene, nst):
    """All marched samples (hundreds per ray); forward and backward staged separately."""
    m = scene["m"]
    pi, ts, te, sg, rgb = m.packed_info, m.t_starts, m.t_ends, scene["sig"], scene["rgb"]
    gc, ga, gd = _grads(pi.shape[0], 12)
    ref = _fwd_bwd(pi, ts, te, sg, rgb, gc, ga, gd, 0, 0)
    _same(_fwd_bwd(pi, ts, te, sg, rgb, gc, ga, gd, nst, 0), ref)
    _same(_fwd_bwd(pi, ts, te, sg, rgb, gc, ga, gd, 0, nst), ref)


def _edge_case(n_samples):
    """Runs with odd and even starts, gaps between runs, empty rays, a ray of 5000
    samples, and a last ray that ends at n_samples (not a multiple of 4)."""
    lens = [0, 1, 2, 3, 63, 64, 65, 127, 129, 0, 5000, 7, 1, 0, 33, 200]
    runs, off = [], 1  # the first run starts at an odd index
    for i, n in enumerate(lens):
        runs.append((off, n))
        off += n + (i % 3)  # gaps of 0, 1, 2 samples between runs
    last = n_samples - off
    assert last > 0
    runs.append((off, last))
    pi = np.array(runs, np.int32)
    t = np.arange(n_samples + 1, dtype=np.float64)
    ts = (0.5 + 0.003 * t[:-1]).astype(np.float32)
    te = (0.5 + 0.003 * t[1:]).astype(np.float32)
    sg = synth.rand_uniform(21, 1, n_samples, 0, 3).astype(np.float32)
    rgb = synth.rand_uniform(21, 2, 3 * n_samples).reshape(n_samples, 3).astype(np.float32)
    return pi, ts, te, sg, rgb


@pytest.mark.parametrize("n_samples", [6021, 6022, 6023, 6024, 6025])
@pytest.mark.parametrize("shift", [0, 2])
def test_staged_edges_and_alignment(orc, n_samples, shift):
    pi, ts, te, sg, rgb = _edge_case(n_samples)
    gc, ga, gd = _grads(pi.shape[0], 13)
    ref = _fwd_bwd(pi, ts, te, sg, rgb, gc, ga, gd, 0, 0)
    c_o, a_o, d_o = orc.render_fwd(pi, ts, te, sg, rgb)
    assert render_tol_ok(ref["col"], c_o, rel_for_large=False) <= 1.0 and render_tol_ok(ref["dp"], d_o) <= 1.0
    ds_o, dr_o = orc.render_bwd(pi, ts, te, sg, rgb, gc.astype(np.float64), ga.astype(np.float64),
                                gd.astype(np.float64))
    covered = np.zeros(n_samples, bool)
    for o, n in pi:
        covered[o:o + n] = True
    for nst in STAGES:
        # shift 0: 16-byte aligned arrays (staged); 2 (8-byte aligned): the register path
        got = _fwd_bwd(pi, ts, te, sg, rgb, gc, ga, gd, nst, nst, shift=shift)
        _same(got, ref)
        assert grad_rel_err(got["ds"][covered], ds_o[covered]) <= 1e-4
        assert grad_rel_err(got["dr"][covered], dr_o[covered]) <= 1e-4
    # samples in no run (the gaps) are left as they were
    assert np.all(np.isnan(ref["ds"][~covered])) and np.all(np.isnan(ref["od"][~covered]))


def test_staged_knob_values():
    for k in ("render_fwd_stages", "render_bwd_stages"):
        old = _lib.tune_get(k)
        for bad in (1, 5, 6, -1):
            with pytest.raises(Exception):
                _lib.tune_set(k, bad)
        assert _lib.tune_get(k) == old

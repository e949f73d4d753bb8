"""Every launch-shape variant the tuning knobs select computes the same results:
each knob's candidate values run marching (bit-exact), pruning, rendering and the
backward against the oracle on one seeded case."""
import numpy as np
import pytest

from paper_2210_04847_gb300 import _lib, autotune, synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no CUDA device", allow_module_level=True)

from gpu_util import assert_march_equal, bits_equal, dev, gpu_march, grad_rel_err, oracle_march  # noqa: E402


@pytest.fixture(scope="module")
def case(orc):
    w = synth.bounded_config(6, n_rays=777, device="cuda")
    m = oracle_march(orc, w)
    sig, _ = synth.sample_field(w.scenes[0], w.rays_o, w.rays_d, m.t_starts, m.t_ends, m.ray_indices)
    p, keep, _ = orc.prune(m.packed_info, m.t_starts, m.t_ends, sig, w.early_stop_eps, w.alpha_thre)
    sg2, rgb2 = synth.sample_field(w.scenes[0], w.rays_o, w.rays_d, p.t_starts, p.t_ends, p.ray_indices)
    R = w.n_rays
    gc = (synth.rand_uniform(6, 9, 3 * R, -1, 1).reshape(R, 3) / R).astype(np.float32)
    ds_o, dr_o = orc.render_bwd(p.packed_info, p.t_starts, p.t_ends, sg2, rgb2, gc.astype(np.float64))
    c_o, a_o, d_o = orc.render_fwd(p.packed_info, p.t_starts, p.t_ends, sg2, rgb2)
    return dict(w=w, m=m, sig=sig, p=p, keep=keep, sg2=sg2, rgb2=rgb2, gc=gc, ds_o=ds_o, dr_o=dr_o, c_o=c_o)


def _run_all(orc, c):
    w, m, p = c["w"], c["m"], c["p"]
    assert_march_equal(gpu_march(w), m)
    R, M = w.n_rays, m.n_samples
    ws = torch.zeros(_lib.prune_workspace_size(R, M), dtype=torch.uint8, device="cuda")
    pio = torch.zeros((R, 2), dtype=torch.int32, device="cuda")
    ts, te = torch.zeros(M, device="cuda"), torch.zeros(M, device="cuda")
    ri = torch.zeros(M, dtype=torch.int32, device="cuda")
    n = torch.zeros(1, dtype=torch.int64, device="cuda")
    st = torch.zeros(1, dtype=torch.int32, device="cuda")
    keep = torch.zeros(M, dtype=torch.uint8, device="cuda")
    _lib.prune_samples(dev(m.packed_info), dev(m.t_starts), dev(m.t_ends), dev(c["sig"]), M, w.early_stop_eps,
                       w.alpha_thre, pio, ts, te, ri, n, st, ws, keep_mask=keep)
    torch.cuda.synchronize()
    assert int(st.item()) == 0
    if np.array_equal(keep.cpu().numpy().astype(bool), c["keep"]):
        assert np.array_equal(pio.cpu().numpy(), p.packed_info)
        assert bits_equal(ts[: p.n_samples].cpu().numpy(), p.t_starts)
    S = p.n_samples
    col = torch.zeros((R, 3), device="cuda")
    op = torch.zeros(R, device="cuda")
    dp = torch.zeros(R, device="cuda")
    od = torch.zeros(S, device="cuda")
    args = [dev(a) for a in (p.t_starts, p.t_ends, c["sg2"], c["rgb2"])]
    _lib.render_fwd(dev(p.packed_info), *args, S, col, op, dp, optical_depth=od, d_status=st)
    dsg, drgb = torch.zeros(S, device="cuda"), torch.zeros((S, 3), device="cuda")
    _lib.render_bwd(dev(p.packed_info), *args, S, dev(c["gc"]), None, None, dsg, drgb, d_status=st)
    dsg2, drgb2 = torch.zeros(S, device="cuda"), torch.zeros((S, 3), device="cuda")
    _lib.render_bwd(dev(p.packed_info), *args, S, dev(c["gc"]), None, None, dsg2, drgb2, optical_depth=od,
                    d_status=st)
    torch.cuda.synchronize()
    assert int(st.item()) == 0
    assert np.max(np.abs(col.cpu().numpy() - c["c_o"])) <= 1e-5
    assert grad_rel_err(dsg.cpu().numpy(), c["ds_o"]) <= 1e-4 and grad_rel_err(drgb.cpu().numpy(), c["dr_o"]) <= 1e-4
    assert torch.equal(dsg, dsg2) and torch.equal(drgb, drgb2)


@pytest.mark.parametrize("knob", sorted(autotune.CANDIDATES))
def test_every_knob_value_gives_the_same_results(orc, case, knob):
    old = _lib.tune_get(knob)
    try:
        for v in autotune.CANDIDATES[knob]:
            _lib.tune_set(knob, v)
            _run_all(orc, case)
    finally:
        _lib.tune_set(knob, old)


def test_knob_range_checks():
    with pytest.raises(_lib.NaccError):
        _lib.tune_set("prune_tile_rays", 3)
    with pytest.raises(_lib.NaccError):
        _lib.tune_set("march_tile_rays", 0)
    with pytest.raises(_lib.NaccError):
        _lib.tune_set("prune_interleave", 3)

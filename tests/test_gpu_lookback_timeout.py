"""The bounded look-back wait running out, on the GPU, without a fault or a hang.

Marching and pruning find each tile's output offset by waiting (a bounded number
of polls) for the tiles before it. A test hook withholds the first tile's total,
a flag nothing else ever sets, so every wait that reaches it gives up after a
short poll budget. The call must still return, raise NACC_STATUS_TIMEOUT in the
device status word, and keep every store below capacity (a prefix taken after a
timeout is never larger than the true one). The context stays usable: with the
hooks back at their defaults the same call is bit-exact again.
"""
import numpy as np
import pytest

from paper_2210_04847_gb300 import _lib, synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no CUDA device", allow_module_level=True)

from gpu_util import dev  # noqa: E402

GUARD = 4096


@pytest.fixture
def hooks():
    yield _lib
    _lib.test_hook_set("withhold_first_tile", 0)
    _lib.test_hook_set("overstate_stage_bytes", 0)
    _lib.test_hook_set("spin_limit", _lib.SPIN_LIMIT_DEFAULT)


def _march(w, o, d, grid, params, cap):
    R = w.n_rays
    ws = torch.zeros(_lib.march_workspace_size(R, params), dtype=torch.uint8, device="cuda")
    pi = torch.full((R, 2), -1, dtype=torch.int32, device="cuda")
    ts = torch.full((cap + GUARD,), np.nan, device="cuda")
    te = torch.full((cap + GUARD,), np.nan, device="cuda")
    ri = torch.full((cap + GUARD,), -7, dtype=torch.int32, device="cuda")
    n = torch.zeros(1, dtype=torch.int64, device="cuda")
    st = torch.zeros(1, dtype=torch.int32, device="cuda")
    _lib.march_rays(o, d, grid, params, pi, ts[:cap], te[:cap], ri[:cap], n, st, ws)
    torch.cuda.synchronize()
    return pi, ts, te, ri, int(n.item()), int(st.item())


@pytest.mark.parametrize("spin_limit", [0, 64])
def test_march_wait_runs_out_and_reports_timeout(hooks, spin_limit):
    w = synth.bounded_config(9, n_rays=3000, device="cuda")
    o, d = dev(w.rays_o), dev(w.rays_d)
    grid = _lib.make_grid(dev(w.bits), w.res, w.aabb)
    params = _lib.make_params(w.near_plane, w.far_plane, w.dt_min, w.dt_max, w.cone, w.max_steps)
    _lib.tune_set("march_tile_rays", 2)  # many tiles, so many waits
    try:
        good = _march(w, o, d, grid, params, 3000 * 1024)
        assert good[5] == 0 and good[4] > 0
        total = good[4]
        hooks.test_hook_set("spin_limit", spin_limit)
        hooks.test_hook_set("withhold_first_tile", 1)
        pi, ts, te, ri, n, st = _march(w, o, d, grid, params, total)
        assert st & _lib.STATUS_TIMEOUT
        assert not st & _lib.STATUS_CAPACITY  # every prefix is at most the true one
        assert 0 <= n <= total
        # nothing at or beyond capacity was written
        assert torch.isnan(ts[total:]).all() and torch.isnan(te[total:]).all() and (ri[total:] == -7).all()
        hooks.test_hook_set("withhold_first_tile", 0)
        hooks.test_hook_set("spin_limit", _lib.SPIN_LIMIT_DEFAULT)
        again = _march(w, o, d, grid, params, 3000 * 1024)
        assert again[5] == 0 and again[4] == total
        assert torch.equal(again[0], good[0]) and torch.equal(again[3][:total], good[3][:total])
        assert torch.equal(again[1][:total].view(torch.int32), good[1][:total].view(torch.int32))
    finally:
        _lib.tune_set("march_tile_rays", 4)


def test_prune_wait_runs_out_and_reports_timeout(hooks, orc):
    w = synth.bounded_config(9, n_rays=3000, device="cuda")
    m = orc.march(w.rays_o, w.rays_d, w.bits, w.res, w.aabb, w.near_plane, w.far_plane, w.dt_min, w.dt_max, w.cone,
                  w.max_steps)
    sig, _ = synth.sample_field(w.scenes[0], w.rays_o, w.rays_d, m.t_starts, m.t_ends, m.ray_indices)
    M = m.n_samples
    pi, ts, te, sg = dev(m.packed_info), dev(m.t_starts), dev(m.t_ends), dev(sig)

    def prune(cap):
        R = w.n_rays
        ws = torch.zeros(_lib.prune_workspace_size(R, M), dtype=torch.uint8, device="cuda")
        pk = torch.full((R, 2), -1, dtype=torch.int32, device="cuda")
        tso = torch.full((cap + GUARD,), np.nan, device="cuda")
        teo = torch.full((cap + GUARD,), np.nan, device="cuda")
        rio = torch.full((cap + GUARD,), -7, dtype=torch.int32, device="cuda")
        n = torch.zeros(1, dtype=torch.int64, device="cuda")
        st = torch.zeros(1, dtype=torch.int32, device="cuda")
        _lib.prune_samples(pi, ts, te, sg, M, w.early_stop_eps, w.alpha_thre, pk, tso[:cap], teo[:cap], rio[:cap], n,
                           st, ws)
        torch.cuda.synchronize()
        return pk, tso, teo, rio, int(n.item()), int(st.item())

    good = prune(M)
    assert good[5] == 0 and good[4] > 0
    total = good[4]
    hooks.test_hook_set("spin_limit", 32)
    hooks.test_hook_set("withhold_first_tile", 1)
    pk, tso, teo, rio, n, st = prune(total)
    assert st & _lib.STATUS_TIMEOUT and not st & _lib.STATUS_CAPACITY
    assert 0 <= n <= total
    assert torch.isnan(tso[total:]).all() and torch.isnan(teo[total:]).all() and (rio[total:] == -7).all()
    hooks.test_hook_set("withhold_first_tile", 0)
    hooks.test_hook_set("spin_limit", _lib.SPIN_LIMIT_DEFAULT)
    again = prune(M)
    assert again[5] == 0 and again[4] == total and torch.equal(again[0], good[0])
    assert torch.equal(again[3][:total], good[3][:total])


@pytest.mark.parametrize("which", ["fwd", "bwd"])
def test_staged_render_wait_runs_out_and_reports_timeout(hooks, orc, which):
    """The render passes with chunks staged by bulk copies wait for each chunk's
    copies on a barrier. A hook makes each warp's first chunk announce more bytes
    than it copies, so that wait never completes: the call returns, the status
    word holds NACC_STATUS_TIMEOUT, nothing past the arrays is written, and with
    the hook off the same calls give the same results as before."""
    w = synth.bounded_config(9, n_rays=3000, device="cuda")
    m = orc.march(w.rays_o, w.rays_d, w.bits, w.res, w.aabb, w.near_plane, w.far_plane, w.dt_min, w.dt_max, w.cone,
                  w.max_steps)
    sig, rgb = synth.sample_field(w.scenes[0], w.rays_o, w.rays_d, m.t_starts, m.t_ends, m.ray_indices)
    R, M = w.n_rays, m.n_samples
    pi, ts, te, sg, cl = dev(m.packed_info), dev(m.t_starts), dev(m.t_ends), dev(sig), dev(rgb)
    gc = dev((synth.rand_uniform(9, 4, 3 * R, -1, 1).reshape(R, 3) / R).astype(np.float32))

    def run():
        col = torch.full((R, 3), np.nan, device="cuda")
        od = torch.full((M + GUARD,), np.nan, device="cuda")
        ds = torch.full((M + GUARD,), np.nan, device="cuda")
        dr = torch.full((M + GUARD, 3), np.nan, device="cuda")
        st = torch.zeros(1, dtype=torch.int32, device="cuda")
        _lib.render_fwd(pi, ts, te, sg, cl, M, col, None, None, optical_depth=od[:M], d_status=st)
        torch.cuda.synchronize()
        s_fwd = int(st.item())
        _lib.render_bwd(pi, ts, te, sg, cl, M, gc, None, None, ds[:M], dr[:M], optical_depth=od[:M], d_status=st)
        torch.cuda.synchronize()
        return col, od, ds, dr, s_fwd, int(st.item())

    knob = "render_%s_stages" % which
    old = _lib.tune_get(knob)
    _lib.tune_set(knob, 2)
    try:
        good = run()
        assert good[4] == 0 and good[5] == 0
        hooks.test_hook_set("spin_limit", 64)
        hooks.test_hook_set("overstate_stage_bytes", 1)
        col, od, ds, dr, s_fwd, s_all = run()
        if which == "fwd":
            assert s_fwd & _lib.STATUS_TIMEOUT
        else:
            assert s_fwd == 0 and s_all & _lib.STATUS_TIMEOUT
            assert torch.equal(od[:M].view(torch.int32), good[1][:M].view(torch.int32))
        # the walks that gave up left their rays unwritten; nothing past the arrays
        assert torch.isnan(od[M:]).all() and torch.isnan(ds[M:]).all() and torch.isnan(dr[M:]).all()
        hooks.test_hook_set("overstate_stage_bytes", 0)
        hooks.test_hook_set("spin_limit", _lib.SPIN_LIMIT_DEFAULT)
        again = run()
        assert again[4] == 0 and again[5] == 0
        for a, b in zip(again[:4], good[:4]):
            assert torch.equal(a.view(torch.int32), b.view(torch.int32))
    finally:
        _lib.tune_set(knob, old)

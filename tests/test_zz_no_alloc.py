"""The allocation-free marching entry point (nacc_march_rays_static).

It serves callers that cannot allocate device memory when they march rays (a
renderer with a fixed, pre-planned memory budget; a plugin inside an
application that owns the CUDA allocator): its scratch is a fixed array in the
library's device memory instead of a caller workspace. This checks, through the
C ABI, that two calls in a row give exactly what nacc_march_rays gives on the
same inputs (marching is bit-exact), so the shared array's leftover contents
never leak into a result. The file is collected last so that a failure here
stops a fail-fast run only after every other test has run.
"""
import numpy as np
import pytest

from paper_2210_04847_gb300 import _lib, synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no CUDA device", allow_module_level=True)


def _outputs(R, cap):
    return (torch.full((R, 2), -1, dtype=torch.int32, device="cuda"),
            torch.full((cap,), np.nan, device="cuda"), torch.full((cap,), np.nan, device="cuda"),
            torch.full((cap,), -1, dtype=torch.int32, device="cuda"),
            torch.zeros(1, dtype=torch.int64, device="cuda"), torch.zeros(1, dtype=torch.int32, device="cuda"))


def _host(out):
    pi, ts, te, ri, n, st = out
    torch.cuda.synchronize()
    k = int(n.item())
    return pi.cpu().numpy(), ts[:k].cpu().numpy(), te[:k].cpu().numpy(), ri[:k].cpu().numpy(), k, int(st.item())


def _same(a, b):
    assert a[5] == 0 and b[5] == 0 and a[4] == b[4] and a[4] > 0
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[3], b[3])
    assert np.array_equal(a[1].view(np.uint32), b[1].view(np.uint32))
    assert np.array_equal(a[2].view(np.uint32), b[2].view(np.uint32))


def test_static_scratch_matches_workspace_entry_point_on_two_calls():
    scene_grid = synth.bounded_scene(5, device="cuda")
    calls = [synth.bounded_config(5, n_rays=3000, batch=0, scene_grid=scene_grid),
             synth.bounded_config(5, n_rays=5000, batch=1, scene_grid=scene_grid)]
    bits = torch.from_numpy(calls[0].bits.view(np.int32)).cuda()
    w = calls[0]
    grid = _lib.make_grid(bits, w.res, w.aabb)
    params = _lib.make_params(w.near_plane, w.far_plane, w.dt_min, w.dt_max, w.cone, w.max_steps)
    for w in calls:  # two calls in a row, different inputs
        R = w.n_rays
        o = torch.from_numpy(w.rays_o).cuda()
        d = torch.from_numpy(w.rays_d).cuda()
        cap = R * 1024
        ws = torch.zeros(_lib.march_workspace_size(R, params), dtype=torch.uint8, device="cuda")
        ref = _outputs(R, cap)
        _lib.march_rays(o, d, grid, params, *ref[:4], ref[4], ref[5], ws)
        got = _outputs(R, cap)
        _lib.march_rays_static(o, d, grid, params, *got[:4], got[4], got[5])
        _same(_host(ref), _host(got))


def test_static_scratch_cone_steps_on_a_cascade_match_workspace_entry_point():
    """Cone steps need the lattice table beside the look-back words; the fixed array
    holds it for every max_steps a call accepts. Two calls in a row on the 4-level
    unbounded cascade give exactly what the workspace entry point gives."""
    for batch, R in ((0, 2000), (1, 3500)):
        w = synth.unbounded_config(6, n_rays=R, batch=batch, device="cuda")
        bits = torch.from_numpy(w.bits.view(np.int32)).cuda()
        grid = _lib.make_grid(bits, w.res, w.aabb, w.n_levels)
        params = _lib.make_params(w.near_plane, w.far_plane, w.dt_min, w.dt_max, w.cone, w.max_steps)
        o = torch.from_numpy(w.rays_o).cuda()
        d = torch.from_numpy(w.rays_d).cuda()
        cap = R * 512
        ws = torch.zeros(_lib.march_workspace_size(R, params), dtype=torch.uint8, device="cuda")
        ref = _outputs(R, cap)
        _lib.march_rays(o, d, grid, params, *ref[:4], ref[4], ref[5], ws)
        got = _outputs(R, cap)
        _lib.march_rays_static(o, d, grid, params, *got[:4], got[4], got[5])
        _same(_host(ref), _host(got))


def test_static_scratch_accepts_the_largest_cone_call_and_rejects_one_ray_more():
    """At the ray limit with cone steps and the largest max_steps the call is
    accepted (counts only: capacity 0) and agrees with the workspace entry point;
    one ray more is rejected before anything is enqueued."""
    R = _lib.STATIC_MAX_RAYS
    gen = torch.Generator("cuda").manual_seed(5)
    o = (torch.rand((R, 3), device="cuda", generator=gen) - 0.5) * 2.0
    d = torch.nn.functional.normalize(torch.randn((R, 3), device="cuda", generator=gen), dim=1)
    bits = torch.full((32 ** 3 // 32,), 0x0F0F0F0F, dtype=torch.int32, device="cuda")
    grid = _lib.make_grid(bits, (32, 32, 32), (-1.5, -1.5, -1.5, 1.5, 1.5, 1.5), 1)
    params = _lib.make_params(0.01, 6.0, 1e-3, 0.05, 1.0 / 128.0, _lib.STATIC_MAX_STEPS)
    empty_f = torch.empty(0, device="cuda")
    empty_i = torch.empty(0, dtype=torch.int32, device="cuda")
    res = []
    for static in (False, True):
        pi = torch.full((R, 2), -1, dtype=torch.int32, device="cuda")
        n = torch.zeros(1, dtype=torch.int64, device="cuda")
        st = torch.zeros(1, dtype=torch.int32, device="cuda")
        if static:
            _lib.march_rays_static(o, d, grid, params, pi, empty_f, empty_f, empty_i, n, st)
        else:
            ws = torch.zeros(_lib.march_workspace_size(R, params), dtype=torch.uint8, device="cuda")
            _lib.march_rays(o, d, grid, params, pi, empty_f, empty_f, empty_i, n, st, ws)
        torch.cuda.synchronize()
        res.append((pi.cpu().numpy(), int(n.item()), int(st.item())))
    assert res[0][1] > 0 and res[0][1] == res[1][1]
    assert res[0][2] == res[1][2] == _lib.STATUS_CAPACITY  # counted, nothing stored
    assert np.array_equal(res[0][0], res[1][0])
    lib = _lib.load()
    rc = lib.nacc_march_rays_static(None, None, None, None, R + 1, grid, params, None, None, None, None, 0,
                                    None, None, None)
    assert rc == _lib.ERR_INVALID_ARG


def test_static_scratch_rejects_too_many_rays():
    lib = _lib.load()
    g = _lib.Grid()
    p = _lib.make_params(0.0, 1.0, 0.1)
    rc = lib.nacc_march_rays_static(None, None, None, None, _lib.STATIC_MAX_RAYS + 1, g, p, None, None, None, None, 0,
                                    None, None, None)
    assert rc == _lib.ERR_INVALID_ARG

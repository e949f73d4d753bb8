"""Helpers of the GPU parity tests: run the CUDA path through the C ABI on
seeded inputs and bring results back as numpy; compare with the oracle."""
import math

import numpy as np
import torch

from paper_2210_04847_gb300 import _lib, synth


def dev(a, dtype=None):
    if a is None:
        return None
    a = np.ascontiguousarray(a)
    if a.dtype == np.uint32:
        a = a.view(np.int32)
    t = torch.from_numpy(a).cuda()
    return t if dtype is None else t.to(dtype)


def grid_struct(bits_t, w: synth.Workload):
    return _lib.make_grid(bits_t, w.res, w.aabb, w.n_levels, w.n_slots, w.contraction)


def gpu_march(w: synth.Workload, capacity=None, rays=None, n_levels=None):
    """March a workload on the GPU; returns numpy (packed_info, t_starts, t_ends, ray_indices, total, status)."""
    o = dev(w.rays_o if rays is None else rays[0])
    d = dev(w.rays_d if rays is None else rays[1])
    R = o.shape[0]
    bits = dev(w.bits)
    params = _lib.make_params(w.near_plane, w.far_plane, w.dt_min, w.dt_max, w.cone, w.max_steps)
    ws = torch.zeros(max(_lib.march_workspace_size(R, params), 256), dtype=torch.uint8, device="cuda")
    if capacity is None:
        capacity = max(1, R * 4)
        for _ in range(2):
            res = _run_march(o, d, bits, w, params, ws, capacity)
            if res[4] <= capacity:
                return res
            capacity = res[4]
    return _run_march(o, d, bits, w, params, ws, capacity)


# When set (by a test fixture), marching calls carry the grid's summed-area table,
# so one-level grids take the box walk.
USE_SAT = False


def _run_march(o, d, bits, w, params, ws, capacity):
    R = o.shape[0]
    packed = torch.full((R, 2), -7, dtype=torch.int32, device="cuda")
    ts = torch.full((capacity,), np.nan, dtype=torch.float32, device="cuda")
    te = torch.full((capacity,), np.nan, dtype=torch.float32, device="cuda")
    ri = torch.full((capacity,), -1, dtype=torch.int32, device="cuda")
    total = torch.full((1,), -1, dtype=torch.int64, device="cuda")
    status = torch.zeros(1, dtype=torch.int32, device="cuda")
    grid = _lib.make_grid(bits, w.res, w.aabb, w.n_levels, w.n_slots, w.contraction)
    if USE_SAT:
        grid = _lib.make_grid(bits, w.res, w.aabb, w.n_levels, w.n_slots, w.contraction,
                              sat=_lib.build_grid_sat(grid))
    _lib.march_rays(o, d, grid, params, packed, ts, te, ri, total, status, ws, ray_time=dev(w.ray_time),
                    ray_slot=dev(w.ray_slot))
    torch.cuda.synchronize()
    n = int(total.item())
    k = min(n, capacity)
    return (packed.cpu().numpy(), ts[:k].cpu().numpy(), te[:k].cpu().numpy(), ri[:k].cpu().numpy(), n,
            int(status.item()))


def oracle_march(orc, w: synth.Workload, rays=None):
    o = w.rays_o if rays is None else rays[0]
    d = w.rays_d if rays is None else rays[1]
    return orc.march(o, d, w.bits, w.res, w.aabb, w.near_plane, w.far_plane, w.dt_min, w.dt_max, w.cone,
                     w.max_steps, n_levels=w.n_levels, n_slots=w.n_slots, ray_time=w.ray_time, ray_slot=w.ray_slot,
                     contraction=w.contraction)


def bits_equal(a, b):
    a = np.ascontiguousarray(a)
    b = np.ascontiguousarray(b)
    return a.shape == b.shape and np.array_equal(a.view(np.uint32) if a.dtype == np.float32 else a,
                                                 b.view(np.uint32) if b.dtype == np.float32 else b)


def assert_march_equal(gpu, ora):
    pi, ts, te, ri, n, status = gpu
    assert status == 0, "device status 0x%x" % status
    assert n == ora.n_samples, (n, ora.n_samples)
    assert np.array_equal(pi, ora.packed_info), "packed_info differs"
    assert bits_equal(ts, ora.t_starts), "t_starts differ"
    assert bits_equal(te, ora.t_ends), "t_ends differ"
    assert np.array_equal(ri, ora.ray_indices), "ray_indices differ"


def render_tol_ok(got, ref, atol=1e-5, rel_for_large=True):
    """|got - ref| <= 1e-5 (absolute), or 1e-5 * |ref| where |ref| > 1 for depth-like outputs."""
    got = np.asarray(got, np.float64)
    ref = np.asarray(ref, np.float64)
    tol = atol * (np.maximum(1.0, np.abs(ref)) if rel_for_large else 1.0)
    return float(np.max(np.abs(got - ref) / tol, initial=0.0))


def grad_rel_err(got, ref):
    """max_i |g_i - g_ref,i| / max(|g_ref,i|, 1e-3 * ||g_ref||_inf), per tensor."""
    got = np.asarray(got, np.float64).reshape(-1)
    ref = np.asarray(ref, np.float64).reshape(-1)
    if ref.size == 0:
        return 0.0
    floor = 1e-3 * np.max(np.abs(ref))
    den = np.maximum(np.abs(ref), max(floor, 1e-30))
    return float(np.max(np.abs(got - ref) / den))


def near_threshold(pi, ts, te, sg, eps, od):
    """Samples whose optical depth od (float32 or float64, per input sample) lies
    within the float32 summation error bound of -ln(eps): the only samples where
    two float32 summation orders may take different keep decisions."""
    tau = sg.astype(np.float64) * (te.astype(np.float64) - ts.astype(np.float64))
    flag = np.zeros(ts.shape[0], bool)
    thr = -math.log(eps)
    for off, cnt in pi:
        if cnt == 0:
            continue
        t = np.abs(tau[off : off + cnt])
        absum = np.concatenate([[0.0], np.cumsum(t)[:-1]])
        bound = (np.arange(cnt) + 40) * 2.0**-23 * absum + 1e-6
        flag[off : off + cnt] = np.abs(od[off : off + cnt].astype(np.float64) - thr) <= bound
    return flag

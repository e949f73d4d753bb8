"""Thin ctypes binding of ``libnacc.so`` (C ABI in ``include/nacc.h``).

Argument marshalling only: every step of marching and rendering runs in the
library's CUDA kernels. Functions take torch CUDA tensors (PyTorch provides the
device memory and the stream), check dtype / device / contiguity / size, pass
raw pointers and the current stream, and raise ``NaccError`` on a non-zero
return code. There is no CPU fallback: if the library is missing, importing
this module's entry points raises.
"""
from __future__ import annotations

import ctypes
import os
from typing import Optional, Sequence

import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libnacc.so")
FIELD_LIB_PATH = os.path.join(_HERE, "libnacc_field.so")

OK = 0
ERR_INVALID_ARG = -1
ERR_CAPACITY = -2
ERR_CUDA = -3
ERR_TIMEOUT = -4

STATUS_CAPACITY = 0x1
STATUS_TIMEOUT = 0x2
STATUS_BAD_PACKED = 0x4
STATUS_BAD_INDEX = 0x8
STATUS_OVERFLOW = 0x10
MAX_LEVELS = 16

EXPORTS = (
    "nacc_grid_sat_bytes", "nacc_build_grid_sat",
    "nacc_march_workspace_size", "nacc_march_rays", "nacc_march_rays_static", "nacc_march_batched_workspace_size",
    "nacc_march_rays_batched", "nacc_prune_workspace_size",
    "nacc_prune_samples", "nacc_march_fused", "nacc_density_field_at_samples", "nacc_density_field_query",
    "nacc_render_weights", "nacc_accumulate_along_rays", "nacc_render_weights_bwd",
    "nacc_accumulate_along_rays_bwd", "nacc_render_fwd", "nacc_render_bwd", "nacc_render_mse_fused",
    "nacc_unpack_info", "nacc_fill_tail_f32", "nacc_update_occupancy_grid", "nacc_density_threshold", "nacc_sample_grid_cells", "nacc_tune_set", "nacc_tune_get",
    "nacc_test_hook_set", "nacc_test_hook_get", "nacc_error_string",
    "nacc_version",
)

TUNE_RENDER_FWD_PREFETCH = 0
TUNE_MARCH_TILE_RAYS = 1
TUNE_PRUNE_TILE_RAYS = 2
TUNE_KNOBS = {"render_fwd_prefetch": 0, "march_tile_rays": 1, "prune_tile_rays": 2, "march_occupancy": 3,
              "prune_occupancy": 4, "render_fwd_occupancy": 5, "render_bwd_occupancy": 6, "march_unroll": 7,
              "prune_interleave": 8, "render_bwd_prefetch": 9,
              "march_coarse": 10, "fused_occupancy": 11, "march_box_tile": 12,
              "render_fwd_stages": 13, "render_bwd_stages": 14,
              "render_mse_occupancy": 15}


class NaccError(RuntimeError):
    pass


class Grid(ctypes.Structure):
    _fields_ = [
        ("bits", ctypes.c_void_p),
        ("res", ctypes.c_int32 * 3),
        ("n_levels", ctypes.c_int32),
        ("n_slots", ctypes.c_int32),
        ("aabb", ctypes.c_float * 6),
        ("contraction", ctypes.c_int32),
        ("sat", ctypes.c_void_p),
    ]


class SceneDesc(ctypes.Structure):
    """nacc_scene_desc: one scene of a batch with its own grid."""
    _fields_ = [
        ("bits", ctypes.c_void_p),
        ("res", ctypes.c_int32 * 3),
        ("n_levels", ctypes.c_int32),
        ("aabb", ctypes.c_float * 6),
        ("contraction", ctypes.c_int32),
        ("n_rays", ctypes.c_int32),
        ("sat", ctypes.c_void_p),
    ]


class DensityField(ctypes.Structure):
    _fields_ = [
        ("sigma", ctypes.c_void_p),
        ("res", ctypes.c_int32 * 3),
        ("aabb", ctypes.c_float * 6),
    ]


class MarchParams(ctypes.Structure):
    _fields_ = [
        ("near_plane", ctypes.c_float),
        ("far_plane", ctypes.c_float),
        ("dt_min", ctypes.c_float),
        ("dt_max", ctypes.c_float),
        ("cone", ctypes.c_float),
        ("max_steps", ctypes.c_int32),
    ]


_lib = None
_field = None


def load() -> ctypes.CDLL:
    """Load libnacc.so (raises if it was not built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise ImportError("libnacc.so is not built (run `python -m paper_2210_04847_gb300.build`): " + LIB_PATH)
    L = ctypes.CDLL(LIB_PATH)
    P, i32, i64, f32, sz = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_float, ctypes.c_size_t
    GP, MP = ctypes.POINTER(Grid), ctypes.POINTER(MarchParams)
    FP = ctypes.POINTER(DensityField)
    sig = {
        "nacc_grid_sat_bytes": (sz, [GP]),
        "nacc_build_grid_sat": (ctypes.c_int, [GP, P, P]),
        "nacc_march_workspace_size": (sz, [i32, MP]),
        "nacc_march_rays": (ctypes.c_int, [P, P, P, P, i32, GP, MP, P, P, P, P, i64, P, P, P, sz, P]),
        "nacc_march_rays_static": (ctypes.c_int, [P, P, P, P, i32, GP, MP, P, P, P, P, i64, P, P, P]),
        "nacc_march_batched_workspace_size": (sz, [i32, i32, MP]),
        "nacc_march_rays_batched": (ctypes.c_int, [ctypes.POINTER(SceneDesc), i32, P, P, i32, MP, P, P, P, P, i64, P,
                                                   P, P, sz, P]),
        "nacc_prune_workspace_size": (sz, [i32, i64]),
        "nacc_prune_samples": (ctypes.c_int, [P, i32, P, P, P, i64, f32, f32, P, P, P, P, i64, P, P, P, P, sz, P]),
        "nacc_march_fused": (ctypes.c_int, [P, P, i32, GP, MP, FP, f32, f32, P, P, P, P, P, i64, P, P, P, sz, P]),
        "nacc_density_field_at_samples": (ctypes.c_int, [FP, P, P, i32, P, P, P, i64, P, P, P]),
        "nacc_density_field_query": (ctypes.c_int, [FP, P, i64, P, P]),
        "nacc_render_weights": (ctypes.c_int, [P, i32, P, P, P, i64, P, P, P, P]),
        "nacc_accumulate_along_rays": (ctypes.c_int, [P, i32, P, P, i32, i64, P, P, P]),
        "nacc_render_weights_bwd": (ctypes.c_int, [P, i32, P, P, P, i64, P, P, P, P, P]),
        "nacc_accumulate_along_rays_bwd": (ctypes.c_int, [P, i32, P, P, i32, i64, P, P, P, P, P, P]),
        "nacc_render_fwd": (ctypes.c_int, [P, i32, P, P, P, P, i64, P, P, P, P, P, P]),
        "nacc_render_bwd": (ctypes.c_int, [P, i32, P, P, P, P, P, i64, P, P, P, P, P, P, P]),
        "nacc_render_mse_fused": (ctypes.c_int, [P, i32, P, P, P, P, i64, P, f32, P, P, P, P, P, P, P, P]),
        "nacc_unpack_info": (ctypes.c_int, [P, i32, i64, P, P, P]),
        "nacc_fill_tail_f32": (ctypes.c_int, [P, i64, i64, P, f32, P]),
        "nacc_update_occupancy_grid": (ctypes.c_int, [P, P, i64, P, P, i64, f32, f32, f32, P, P]),
        "nacc_density_threshold": (ctypes.c_float, [f32, f32]),
        "nacc_sample_grid_cells": (ctypes.c_int, [ctypes.c_uint64, ctypes.c_uint64, i64, GP, P, P, P]),
        "nacc_tune_set": (ctypes.c_int, [ctypes.c_int, ctypes.c_int]),
        "nacc_tune_get": (ctypes.c_int, [ctypes.c_int]),
        "nacc_test_hook_set": (ctypes.c_int, [ctypes.c_int, ctypes.c_int]),
        "nacc_test_hook_get": (ctypes.c_int, [ctypes.c_int]),
        "nacc_error_string": (ctypes.c_char_p, [ctypes.c_int]),
        "nacc_version": (ctypes.c_int, []),
    }
    for name, (res, args) in sig.items():
        fn = getattr(L, name)
        fn.restype = res
        fn.argtypes = args
    _lib = L
    return L


def load_field() -> ctypes.CDLL:
    global _field
    if _field is not None:
        return _field
    if not os.path.exists(FIELD_LIB_PATH):
        raise ImportError("libnacc_field.so is not built: " + FIELD_LIB_PATH)
    L = ctypes.CDLL(FIELD_LIB_PATH)
    P, i32, i64 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64
    L.nacc_field_samples.restype = ctypes.c_int
    L.nacc_field_samples.argtypes = [P, P, P, P, P, P, i64, P, i32, P, P, P, P]
    L.nacc_field_points.restype = ctypes.c_int
    L.nacc_field_points.argtypes = [P, P, i64, P, i32, P, P]
    L.nacc_field_samples_multi.restype = ctypes.c_int
    L.nacc_field_samples_multi.argtypes = [P, P, P, P, P, P, P, P, i64, P, P, P, P, P, P]
    _field = L
    return L


# ---------------------------------------------------------------------------
# marshalling helpers
# ---------------------------------------------------------------------------


def _ptr(t: Optional[torch.Tensor]):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def _stream(stream=None):
    s = torch.cuda.current_stream() if stream is None else stream
    return ctypes.c_void_p(s.cuda_stream)


def _check(t: Optional[torch.Tensor], dtype, name: str, numel: Optional[int] = None, optional=False):
    if t is None:
        if optional:
            return
        raise NaccError("%s is required" % name)
    if not t.is_cuda:
        raise NaccError("%s must be a CUDA tensor" % name)
    if t.dtype != dtype:
        raise NaccError("%s must be %s, got %s" % (name, dtype, t.dtype))
    if not t.is_contiguous():
        raise NaccError("%s must be contiguous" % name)
    if numel is not None and t.numel() < numel:
        raise NaccError("%s holds %d elements, needs %d" % (name, t.numel(), numel))


def _call(name: str, args, defer: bool):
    """Call C entry point ``name`` with marshalled ``args``; with ``defer`` return
    a callable that makes the call later (marshalling and checks already done, so
    the call itself costs only the C function: a timed region can start right
    before it)."""
    fn = getattr(load(), name)
    if defer:
        def run():
            _rc(fn(*args), name)
        return run
    _rc(fn(*args), name)
    return None


def _rc(code: int, fn: str):
    if code != OK:
        msg = load().nacc_error_string(code).decode()
        raise NaccError("%s failed: %s (%d)" % (fn, msg, code))


def make_grid(bits: torch.Tensor, res: Sequence[int], aabb: Sequence[float], n_levels=1, n_slots=1,
              contraction: int = 0, sat: Optional[torch.Tensor] = None) -> Grid:
    """nacc_grid over a bits tensor; ``sat`` (int16 tensor from ``build_grid_sat``)
    lets one-level grids take the box walk."""
    _check(bits, torch.int32, "grid bits")
    _check(sat, torch.int16, "grid sat", optional=True)
    g = Grid()
    g._keepalive = bits  # the struct holds a raw pointer: keep the tensor alive with it
    g._keepalive_sat = sat
    g.sat = None if sat is None else sat.data_ptr()
    g.contraction = int(contraction)
    g.bits = bits.data_ptr()
    for k in range(3):
        g.res[k] = int(res[k])
    g.n_levels = int(n_levels)
    g.n_slots = int(n_slots)
    for k in range(6):
        g.aabb[k] = float(aabb[k])
    return g


def make_scenes(scenes) -> ctypes.Array:
    """Array of nacc_scene_desc from (bits tensor, res, aabb, n_levels, contraction, n_rays[,
    sat tensor]) tuples; the array keeps the tensors alive."""
    arr = (SceneDesc * len(scenes))()
    keep = []
    for k, sc in enumerate(scenes):
        bits, res, aabb, n_levels, contraction, n_rays = sc[:6]
        sat = sc[6] if len(sc) > 6 else None
        _check(bits, torch.int32, "scene bits")
        _check(sat, torch.int16, "scene sat", optional=True)
        d = arr[k]
        d.bits = bits.data_ptr()
        d.sat = None if sat is None else sat.data_ptr()
        keep.append((bits, sat))
        for j in range(3):
            d.res[j] = int(res[j])
        d.n_levels = int(n_levels)
        for j in range(6):
            d.aabb[j] = float(aabb[j])
        d.contraction = int(contraction)
        d.n_rays = int(n_rays)
    arr._keepalive = keep
    return arr


def grid_sat_bytes(grid: Grid) -> int:
    return int(load().nacc_grid_sat_bytes(ctypes.byref(grid)))


def build_grid_sat(grid: Grid, sat: Optional[torch.Tensor] = None, stream=None, defer: bool = False):
    """nacc_build_grid_sat: the summed-area table of the grid's bits (uint16 entries,
    held in an int16 tensor), into ``sat`` or a new tensor, which is returned (with
    ``defer``: the marshalled call, to run later)."""
    n = grid_sat_bytes(grid) // 2
    if n <= 0:
        raise NaccError("invalid grid for a summed-area table")
    if sat is None:
        sat = torch.empty(n, dtype=torch.int16, device="cuda")
    _check(sat, torch.int16, "sat", n)
    run = _call("nacc_build_grid_sat", (ctypes.byref(grid), _ptr(sat), _stream(stream)), True)
    if defer:
        return run
    run()
    return sat


def make_density_field(sigma: torch.Tensor, aabb: Sequence[float]) -> DensityField:
    """nacc_density_field over a (G0, G1, G2) float32 CUDA tensor of vertex values."""
    _check(sigma, torch.float32, "density field")
    if sigma.dim() != 3:
        raise NaccError("density field must be a 3-d tensor of vertex values")
    f = DensityField()
    f._keepalive = sigma  # the struct holds a raw pointer: keep the tensor alive with it
    f.sigma = sigma.data_ptr()
    for k in range(3):
        f.res[k] = int(sigma.shape[k])
    for k in range(6):
        f.aabb[k] = float(aabb[k])
    return f


def make_params(near_plane, far_plane, dt_min, dt_max=None, cone=0.0, max_steps=1024) -> MarchParams:
    p = MarchParams()
    p.near_plane = float(near_plane)
    p.far_plane = float(far_plane)
    p.dt_min = float(dt_min)
    p.dt_max = float(dt_min if dt_max is None else dt_max)
    p.cone = float(cone)
    p.max_steps = int(max_steps)
    return p


# ---------------------------------------------------------------------------
# entry points (same names as the C ABI, without the nacc_ prefix)
# ---------------------------------------------------------------------------


def march_workspace_size(n_rays: int, params: MarchParams) -> int:
    return int(load().nacc_march_workspace_size(int(n_rays), ctypes.byref(params)))


def prune_workspace_size(n_rays: int, n_samples: int) -> int:
    return int(load().nacc_prune_workspace_size(int(n_rays), int(n_samples)))


def march_rays(rays_o, rays_d, grid: Grid, params: MarchParams, packed_info, t_starts, t_ends, ray_indices,
               n_samples, d_status, workspace, ray_time=None, ray_slot=None, stream=None, defer: bool = False):
    n = rays_o.shape[0]
    _check(rays_o, torch.float32, "rays_o", 3 * n)
    _check(rays_d, torch.float32, "rays_d", 3 * n)
    _check(ray_time, torch.float32, "ray_time", n, optional=True)
    _check(ray_slot, torch.int32, "ray_slot", n, optional=True)
    _check(packed_info, torch.int32, "packed_info", 2 * n)
    cap = t_starts.numel()
    _check(t_starts, torch.float32, "t_starts")
    _check(t_ends, torch.float32, "t_ends", cap)
    _check(ray_indices, torch.int32, "ray_indices", cap)
    _check(n_samples, torch.int64, "n_samples", 1)
    _check(d_status, torch.int32, "d_status", 1, optional=True)
    _check(workspace, torch.uint8, "workspace")
    args = (_ptr(rays_o), _ptr(rays_d), _ptr(ray_time), _ptr(ray_slot), n, ctypes.byref(grid), ctypes.byref(params),
            _ptr(packed_info), _ptr(t_starts), _ptr(t_ends), _ptr(ray_indices), cap, _ptr(n_samples),
            _ptr(d_status), _ptr(workspace), workspace.numel(), _stream(stream))
    return _call("nacc_march_rays", args, defer)


def march_batched_workspace_size(n_scenes: int, n_rays: int, params: MarchParams) -> int:
    return int(load().nacc_march_batched_workspace_size(int(n_scenes), int(n_rays), ctypes.byref(params)))


def march_rays_batched(scenes, rays_o, rays_d, params: MarchParams, packed_info, t_starts, t_ends, ray_indices,
                       n_samples, d_status, workspace, stream=None, defer: bool = False):
    """nacc_march_rays_batched: one launch over scenes with their own grids
    (``scenes`` from ``make_scenes``; rays scene-major)."""
    n = rays_o.shape[0]
    _check(rays_o, torch.float32, "rays_o", 3 * n)
    _check(rays_d, torch.float32, "rays_d", 3 * n)
    _check(packed_info, torch.int32, "packed_info", 2 * n)
    cap = t_starts.numel()
    _check(t_starts, torch.float32, "t_starts")
    _check(t_ends, torch.float32, "t_ends", cap)
    _check(ray_indices, torch.int32, "ray_indices", cap)
    _check(n_samples, torch.int64, "n_samples", 1)
    _check(d_status, torch.int32, "d_status", 1, optional=True)
    _check(workspace, torch.uint8, "workspace")
    args = (scenes, len(scenes), _ptr(rays_o), _ptr(rays_d), n, ctypes.byref(params), _ptr(packed_info),
            _ptr(t_starts), _ptr(t_ends), _ptr(ray_indices), cap, _ptr(n_samples), _ptr(d_status), _ptr(workspace),
            workspace.numel(), _stream(stream))
    return _call("nacc_march_rays_batched", args, defer)


STATIC_MAX_RAYS = 1 << 20
STATIC_MAX_STEPS = 32768


def march_rays_static(rays_o, rays_d, grid: Grid, params: MarchParams, packed_info, t_starts, t_ends, ray_indices,
                      n_samples, d_status, ray_time=None, ray_slot=None, stream=None):
    """nacc_march_rays_static: marching with the library's fixed scratch array, for
    callers that cannot allocate device memory (no workspace argument)."""
    n = rays_o.shape[0]
    _check(rays_o, torch.float32, "rays_o", 3 * n)
    _check(rays_d, torch.float32, "rays_d", 3 * n)
    _check(ray_time, torch.float32, "ray_time", n, optional=True)
    _check(ray_slot, torch.int32, "ray_slot", n, optional=True)
    _check(packed_info, torch.int32, "packed_info", 2 * n)
    cap = t_starts.numel()
    _check(t_starts, torch.float32, "t_starts")
    _check(t_ends, torch.float32, "t_ends", cap)
    _check(ray_indices, torch.int32, "ray_indices", cap)
    _check(n_samples, torch.int64, "n_samples", 1)
    _check(d_status, torch.int32, "d_status", 1, optional=True)
    rc = load().nacc_march_rays_static(
        _ptr(rays_o), _ptr(rays_d), _ptr(ray_time), _ptr(ray_slot), n, ctypes.byref(grid), ctypes.byref(params),
        _ptr(packed_info), _ptr(t_starts), _ptr(t_ends), _ptr(ray_indices), cap, _ptr(n_samples), _ptr(d_status),
        _stream(stream))
    _rc(rc, "nacc_march_rays_static")


def march_fused(rays_o, rays_d, grid: Grid, params: MarchParams, field: DensityField, early_stop_eps, alpha_thre,
                packed_info, t_starts, t_ends, ray_indices, sigmas, n_samples, d_status, workspace, stream=None,
                defer: bool = False):
    """nacc_march_fused: marching that stops on the density field's transmittance
    (inference); writes only the kept samples (and their sigma when given)."""
    n = rays_o.shape[0]
    _check(rays_o, torch.float32, "rays_o", 3 * n)
    _check(rays_d, torch.float32, "rays_d", 3 * n)
    _check(packed_info, torch.int32, "packed_info", 2 * n)
    cap = t_starts.numel()
    _check(t_starts, torch.float32, "t_starts")
    _check(t_ends, torch.float32, "t_ends", cap)
    _check(ray_indices, torch.int32, "ray_indices", cap)
    _check(sigmas, torch.float32, "sigmas", cap, optional=True)
    _check(n_samples, torch.int64, "n_samples", 1)
    _check(d_status, torch.int32, "d_status", 1, optional=True)
    _check(workspace, torch.uint8, "workspace")
    args = (_ptr(rays_o), _ptr(rays_d), n, ctypes.byref(grid), ctypes.byref(params), ctypes.byref(field),
            float(early_stop_eps), float(alpha_thre), _ptr(packed_info), _ptr(t_starts), _ptr(t_ends),
            _ptr(ray_indices), _ptr(sigmas), cap, _ptr(n_samples), _ptr(d_status), _ptr(workspace),
            workspace.numel(), _stream(stream))
    return _call("nacc_march_fused", args, defer)


def density_field_at_samples(field: DensityField, rays_o, rays_d, ray_indices, t_starts, t_ends, n_samples: int,
                             sigmas, d_status=None, stream=None, defer: bool = False):
    n = rays_o.shape[0]
    _check(rays_o, torch.float32, "rays_o", 3 * n)
    _check(rays_d, torch.float32, "rays_d", 3 * n)
    for t, name in ((t_starts, "t_starts"), (t_ends, "t_ends"), (sigmas, "sigmas")):
        _check(t, torch.float32, name, n_samples)
    _check(ray_indices, torch.int32, "ray_indices", n_samples)
    _check(d_status, torch.int32, "d_status", 1, optional=True)
    args = (ctypes.byref(field), _ptr(rays_o), _ptr(rays_d), n, _ptr(ray_indices), _ptr(t_starts), _ptr(t_ends),
            int(n_samples), _ptr(sigmas), _ptr(d_status), _stream(stream))
    return _call("nacc_density_field_at_samples", args, defer)


def density_field_query(field: DensityField, xyz, n: int, sigmas, stream=None):
    _check(xyz, torch.float32, "xyz", 3 * n)
    _check(sigmas, torch.float32, "sigmas", n)
    rc = load().nacc_density_field_query(ctypes.byref(field), _ptr(xyz), int(n), _ptr(sigmas), _stream(stream))
    _rc(rc, "nacc_density_field_query")


def prune_samples(packed_info, t_starts, t_ends, sigmas, n_samples_in: int, early_stop_eps, alpha_thre,
                  packed_info_out, t_starts_out, t_ends_out, ray_indices_out, n_kept, d_status, workspace,
                  keep_mask=None, stream=None, defer: bool = False):
    n = packed_info.shape[0]
    _check(packed_info, torch.int32, "packed_info", 2 * n)
    for t, nm in ((t_starts, "t_starts"), (t_ends, "t_ends"), (sigmas, "sigmas")):
        _check(t, torch.float32, nm, n_samples_in)
    _check(packed_info_out, torch.int32, "packed_info_out", 2 * n)
    cap = t_starts_out.numel()
    _check(t_starts_out, torch.float32, "t_starts_out")
    _check(t_ends_out, torch.float32, "t_ends_out", cap)
    _check(ray_indices_out, torch.int32, "ray_indices_out", cap)
    _check(n_kept, torch.int64, "n_kept", 1)
    _check(keep_mask, torch.uint8, "keep_mask", n_samples_in, optional=True)
    _check(d_status, torch.int32, "d_status", 1, optional=True)
    _check(workspace, torch.uint8, "workspace")
    args = (_ptr(packed_info), n, _ptr(t_starts), _ptr(t_ends), _ptr(sigmas), int(n_samples_in),
            float(early_stop_eps), float(alpha_thre), _ptr(packed_info_out), _ptr(t_starts_out), _ptr(t_ends_out),
            _ptr(ray_indices_out), cap, _ptr(n_kept), _ptr(keep_mask), _ptr(d_status), _ptr(workspace),
            workspace.numel(), _stream(stream))
    return _call("nacc_prune_samples", args, defer)


def render_weights(packed_info, t_starts, t_ends, sigmas, n_samples: int, weights=None, trans=None, d_status=None,
                   stream=None, defer: bool = False):
    n = packed_info.shape[0]
    _check(packed_info, torch.int32, "packed_info", 2 * n)
    for t, nm in ((t_starts, "t_starts"), (t_ends, "t_ends"), (sigmas, "sigmas")):
        _check(t, torch.float32, nm, n_samples)
    _check(weights, torch.float32, "weights", n_samples, optional=True)
    _check(trans, torch.float32, "trans", n_samples, optional=True)
    _check(d_status, torch.int32, "d_status", 1, optional=True)
    return _call("nacc_render_weights", (_ptr(packed_info), n, _ptr(t_starts), _ptr(t_ends), _ptr(sigmas),
                                         int(n_samples), _ptr(weights), _ptr(trans), _ptr(d_status), _stream(stream)),
                 defer)


def accumulate_along_rays(packed_info, weights, values, n_channels: int, n_samples: int, out, d_status=None,
                          stream=None, defer: bool = False):
    n = packed_info.shape[0]
    _check(packed_info, torch.int32, "packed_info", 2 * n)
    _check(weights, torch.float32, "weights", n_samples)
    _check(values, torch.float32, "values", n_samples * n_channels, optional=True)
    _check(out, torch.float32, "out", n * n_channels)
    _check(d_status, torch.int32, "d_status", 1, optional=True)
    return _call("nacc_accumulate_along_rays", (_ptr(packed_info), n, _ptr(weights), _ptr(values), int(n_channels),
                                                int(n_samples), _ptr(out), _ptr(d_status), _stream(stream)), defer)


def render_weights_bwd(packed_info, t_starts, t_ends, sigmas, n_samples: int, g_weights, d_sigmas, d_status=None,
                       g_ref=None, stream=None, defer: bool = False):
    """dL/dsigma for dL/dw = g_weights, or g_ref[ray] + g_weights when g_ref (n_rays,) is given."""
    n = packed_info.shape[0]
    _check(packed_info, torch.int32, "packed_info", 2 * n)
    for t, nm in ((t_starts, "t_starts"), (t_ends, "t_ends"), (sigmas, "sigmas"), (g_weights, "g_weights"),
                  (d_sigmas, "d_sigmas")):
        _check(t, torch.float32, nm, n_samples)
    _check(g_ref, torch.float32, "g_ref", n, optional=True)
    _check(d_status, torch.int32, "d_status", 1, optional=True)
    return _call("nacc_render_weights_bwd", (_ptr(packed_info), n, _ptr(t_starts), _ptr(t_ends), _ptr(sigmas),
                                             int(n_samples), _ptr(g_weights), _ptr(g_ref), _ptr(d_sigmas),
                                             _ptr(d_status), _stream(stream)), defer)


def accumulate_along_rays_bwd(packed_info, weights, values, n_channels: int, n_samples: int, g_out, d_weights=None,
                              d_values=None, d_status=None, g_ref=None, stream=None, defer: bool = False):
    """dL/dw and dL/dv of the per-ray sums; with g_ref (n_rays,) the centred mode
    (d_weights relative to each ray's first sample, that sample's part added to g_ref)."""
    n = packed_info.shape[0]
    _check(packed_info, torch.int32, "packed_info", 2 * n)
    _check(weights, torch.float32, "weights", n_samples)
    _check(values, torch.float32, "values", n_samples * n_channels, optional=True)
    _check(g_out, torch.float32, "g_out", n * n_channels)
    _check(d_weights, torch.float32, "d_weights", n_samples, optional=True)
    _check(d_values, torch.float32, "d_values", n_samples * n_channels, optional=True)
    _check(g_ref, torch.float32, "g_ref", n, optional=True)
    _check(d_status, torch.int32, "d_status", 1, optional=True)
    return _call("nacc_accumulate_along_rays_bwd", (_ptr(packed_info), n, _ptr(weights), _ptr(values),
                                                    int(n_channels), int(n_samples), _ptr(g_out), _ptr(d_weights),
                                                    _ptr(d_values), _ptr(g_ref), _ptr(d_status), _stream(stream)),
                 defer)


def render_fwd(packed_info, t_starts, t_ends, sigmas, rgbs, n_samples: int, color, opacity, depth,
               optical_depth=None, d_status=None, stream=None, defer: bool = False):
    n = packed_info.shape[0]
    _check(packed_info, torch.int32, "packed_info", 2 * n)
    for t, nm in ((t_starts, "t_starts"), (t_ends, "t_ends"), (sigmas, "sigmas")):
        _check(t, torch.float32, nm, n_samples)
    _check(rgbs, torch.float32, "rgbs", 3 * n_samples)
    _check(color, torch.float32, "color", 3 * n, optional=True)
    _check(opacity, torch.float32, "opacity", n, optional=True)
    _check(depth, torch.float32, "depth", n, optional=True)
    _check(optical_depth, torch.float32, "optical_depth", n_samples, optional=True)
    _check(d_status, torch.int32, "d_status", 1, optional=True)
    return _call("nacc_render_fwd", (_ptr(packed_info), n, _ptr(t_starts), _ptr(t_ends), _ptr(sigmas), _ptr(rgbs),
                                     int(n_samples), _ptr(color), _ptr(opacity), _ptr(depth), _ptr(optical_depth),
                                     _ptr(d_status), _stream(stream)), defer)


def render_bwd(packed_info, t_starts, t_ends, sigmas, rgbs, n_samples: int, g_color, g_opacity, g_depth, d_sigmas,
               d_rgbs, optical_depth=None, d_status=None, stream=None, defer: bool = False):
    n = packed_info.shape[0]
    _check(packed_info, torch.int32, "packed_info", 2 * n)
    for t, nm in ((t_starts, "t_starts"), (t_ends, "t_ends"), (sigmas, "sigmas")):
        _check(t, torch.float32, nm, n_samples)
    _check(rgbs, torch.float32, "rgbs", 3 * n_samples)
    _check(optical_depth, torch.float32, "optical_depth", n_samples, optional=True)
    _check(g_color, torch.float32, "g_color", 3 * n, optional=True)
    _check(g_opacity, torch.float32, "g_opacity", n, optional=True)
    _check(g_depth, torch.float32, "g_depth", n, optional=True)
    _check(d_sigmas, torch.float32, "d_sigmas", n_samples)
    _check(d_rgbs, torch.float32, "d_rgbs", 3 * n_samples)
    _check(d_status, torch.int32, "d_status", 1, optional=True)
    return _call("nacc_render_bwd", (_ptr(packed_info), n, _ptr(t_starts), _ptr(t_ends), _ptr(sigmas), _ptr(rgbs),
                                     _ptr(optical_depth), int(n_samples), _ptr(g_color), _ptr(g_opacity), _ptr(g_depth),
                                     _ptr(d_sigmas), _ptr(d_rgbs), _ptr(d_status), _stream(stream)), defer)


def render_mse_fused(packed_info, t_starts, t_ends, sigmas, rgbs, n_samples: int, target, grad_scale: float, color,
                     d_sigmas, d_rgbs, opacity=None, depth=None, sq_err=None, d_status=None, stream=None,
                     defer: bool = False):
    """nacc_render_mse_fused: forward, the squared-error loss gradient
    grad_scale * (C - target) and the backward in one pass."""
    n = packed_info.shape[0]
    _check(packed_info, torch.int32, "packed_info", 2 * n)
    for t, nm in ((t_starts, "t_starts"), (t_ends, "t_ends"), (sigmas, "sigmas")):
        _check(t, torch.float32, nm, n_samples)
    _check(rgbs, torch.float32, "rgbs", 3 * n_samples)
    _check(target, torch.float32, "target", 3 * n)
    _check(color, torch.float32, "color", 3 * n, optional=True)
    _check(opacity, torch.float32, "opacity", n, optional=True)
    _check(depth, torch.float32, "depth", n, optional=True)
    _check(sq_err, torch.float32, "sq_err", n, optional=True)
    _check(d_sigmas, torch.float32, "d_sigmas", n_samples)
    _check(d_rgbs, torch.float32, "d_rgbs", 3 * n_samples)
    _check(d_status, torch.int32, "d_status", 1, optional=True)
    return _call("nacc_render_mse_fused", (_ptr(packed_info), n, _ptr(t_starts), _ptr(t_ends), _ptr(sigmas),
                                           _ptr(rgbs), int(n_samples), _ptr(target), float(grad_scale), _ptr(color),
                                           _ptr(opacity), _ptr(depth), _ptr(sq_err), _ptr(d_sigmas), _ptr(d_rgbs),
                                           _ptr(d_status), _stream(stream)), defer)


def unpack_info(packed_info, n_samples: int, ray_indices, d_status=None, stream=None):
    n = packed_info.shape[0]
    _check(packed_info, torch.int32, "packed_info", 2 * n)
    _check(ray_indices, torch.int32, "ray_indices", n_samples)
    _check(d_status, torch.int32, "d_status", 1, optional=True)
    rc = load().nacc_unpack_info(_ptr(packed_info), n, int(n_samples), _ptr(ray_indices), _ptr(d_status),
                                 _stream(stream))
    _rc(rc, "nacc_unpack_info")


def fill_tail(arr, n_dev, value: float = 0.0, stream=None):
    """nacc_fill_tail_f32: rows [*n_dev, len(arr)) of a float32 array set to value."""
    _check(arr, torch.float32, "arr")
    _check(n_dev, torch.int64, "n_dev", 1)
    cap = arr.shape[0] if arr.dim() > 0 else 0
    width = arr.numel() // max(cap, 1) if cap else 1
    _rc(load().nacc_fill_tail_f32(_ptr(arr), int(width), int(cap), _ptr(n_dev), float(value), _stream(stream)),
        "nacc_fill_tail_f32")


def update_occupancy_grid(ema, bits, cells, sigmas, decay, thre, d_status=None, alpha_step: float = 0.0, stream=None,
                          defer: bool = False):
    """EMA update; alpha_step > 0 makes thre the opacity threshold of a step of that length."""
    n_cells = ema.numel()
    _check(ema, torch.float32, "ema")
    _check(bits, torch.int32, "bits", (n_cells + 31) // 32)
    n = cells.numel()
    _check(cells, torch.int32, "cells")
    _check(sigmas, torch.float32, "sigmas", n)
    _check(d_status, torch.int32, "d_status", 1, optional=True)
    return _call("nacc_update_occupancy_grid", (_ptr(ema), _ptr(bits), n_cells, _ptr(cells), _ptr(sigmas), n,
                                                float(decay), float(thre), float(alpha_step), _ptr(d_status),
                                                _stream(stream)), defer)


def density_threshold(alpha_thre: float, dt: float) -> float:
    """nacc_density_threshold: the density threshold equivalent to an opacity threshold
    for steps of length dt (NaN for invalid arguments). Host only."""
    return float(load().nacc_density_threshold(float(alpha_thre), float(dt)))


def sample_grid_cells(seed: int, stream: int, n: int, grid: Grid, cells, xyz, cuda_stream=None, defer: bool = False):
    """n uniform random cells of the grid and a uniform point in each (SplitMix64
    streams `stream` for the cells and `stream` + 1 for the points)."""
    _check(cells, torch.int32, "cells", n)
    _check(xyz, torch.float32, "xyz", 3 * n)
    return _call("nacc_sample_grid_cells", (int(seed) & 0xFFFFFFFFFFFFFFFF, int(stream) & 0xFFFFFFFFFFFFFFFF, int(n),
                                            ctypes.byref(grid), _ptr(cells), _ptr(xyz), _stream(cuda_stream)), defer)


def tune_set(knob, value: int):
    """Set a launch-shape knob (name or NACC_TUNE_* index); results never change, only speed."""
    k = TUNE_KNOBS[knob] if isinstance(knob, str) else int(knob)
    _rc(load().nacc_tune_set(k, int(value)), "nacc_tune_set")


TEST_HOOKS = {"spin_limit": 0, "withhold_first_tile": 1, "overstate_stage_bytes": 2}
SPIN_LIMIT_DEFAULT = 1 << 22


def test_hook_set(hook, value: int):
    """Set a look-back test hook (name or NACC_TEST_HOOK_* index). Tests only:
    results are invalid while a hook is away from its default."""
    k = TEST_HOOKS[hook] if isinstance(hook, str) else int(hook)
    _rc(load().nacc_test_hook_set(k, int(value)), "nacc_test_hook_set")


def test_hook_get(hook) -> int:
    k = TEST_HOOKS[hook] if isinstance(hook, str) else int(hook)
    v = load().nacc_test_hook_get(k)
    if v < 0:
        raise NaccError("unknown test hook %r" % (hook,))
    return v


def tune_get(knob) -> int:
    k = TUNE_KNOBS[knob] if isinstance(knob, str) else int(knob)
    v = load().nacc_tune_get(k)
    if v < 0:
        raise NaccError("unknown tuning knob %r" % (knob,))
    return v


# ---------------------------------------------------------------------------
# stand-in radiance field (benchmarks only; not part of the method)
# ---------------------------------------------------------------------------


def field_samples(rays_o, rays_d, ray_indices, t_starts, t_ends, n: int, blobs, rgb_wb, sigmas, rgbs=None,
                  ray_time=None, stream=None):
    rc = load_field().nacc_field_samples(_ptr(rays_o), _ptr(rays_d), _ptr(ray_time), _ptr(ray_indices),
                                         _ptr(t_starts), _ptr(t_ends), int(n), _ptr(blobs), blobs.shape[0],
                                         _ptr(rgb_wb), _ptr(sigmas), _ptr(rgbs), _stream(stream))
    if rc != 0:
        raise NaccError("nacc_field_samples failed (%d)" % rc)


def field_samples_multi(rays_o, rays_d, ray_slot, ray_indices, t_starts, t_ends, n_dev, n_max: int, blobs, blob_off,
                        rgb_wb, sigmas, rgbs=None, ray_time=None, stream=None):
    rc = load_field().nacc_field_samples_multi(_ptr(rays_o), _ptr(rays_d), _ptr(ray_time), _ptr(ray_slot),
                                               _ptr(ray_indices), _ptr(t_starts), _ptr(t_ends), _ptr(n_dev), int(n_max),
                                               _ptr(blobs), _ptr(blob_off), _ptr(rgb_wb), _ptr(sigmas), _ptr(rgbs),
                                               _stream(stream))
    if rc != 0:
        raise NaccError("nacc_field_samples_multi failed (%d)" % rc)


def field_points(xyz, n: int, blobs, sigmas, times=None, stream=None):
    rc = load_field().nacc_field_points(_ptr(xyz), _ptr(times), int(n), _ptr(blobs), blobs.shape[0], _ptr(sigmas),
                                        _stream(stream))
    if rc != 0:
        raise NaccError("nacc_field_points failed (%d)" % rc)

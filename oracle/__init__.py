"""CPU oracle for occupancy-grid marching + packed volume rendering (test infrastructure).

Only the test suite, ``__graft_entry__.smoke()`` and the benchmark's CPU
baseline / reference arm may import this package. The product path never does.
The arithmetic lives in ``oracle.c`` (plain C, see its header for the precision
of each step and the readings of the paper); this module only compiles it and
marshals numpy arrays through ``ctypes``.

Entry points mirror the paper's two stages (Sec. 2.1 ray marching, Sec. 2.2
differentiable rendering, Eq. 1) and the occupancy-grid update the paper
borrows from Instant-NGP (Sec. 2.1, "Pruning Empty and Occluded Regions").
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
# The mutation test points this at a deliberately broken copy of the oracle to
# show that the pins fail; nothing else sets it.
_LIB_OVERRIDE = os.environ.get("NACC_ORACLE_LIB_OVERRIDE")
CFLAGS = ["-O2", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared", "-std=c11"]


def build(force: bool = False) -> str:
    """Compile oracle.c into liboracle.so (gcc, strict IEEE float32/float64)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + ".tmp.%d" % os.getpid()
        subprocess.check_call(["gcc", *CFLAGS, "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


_lib = None


def lib():
    global _lib
    if _lib is None:
        if _LIB_OVERRIDE:
            L = ctypes.CDLL(_LIB_OVERRIDE)
        else:
            build()
            L = ctypes.CDLL(_LIB)
        P = ctypes.c_void_p
        i32, i64, f32 = ctypes.c_int32, ctypes.c_int64, ctypes.c_float
        L.oracle_march.restype = i64
        L.oracle_march.argtypes = [P, P, P, P, i32, P, P, i32, i32, P, f32, f32, f32, f32, f32, i32, i32, P, P, P, P,
                                   i64]
        L.oracle_prune.restype = i64
        L.oracle_prune.argtypes = [P, i32, P, P, P, f32, f32, P, P, P, P, P, P, i64]
        L.oracle_render_weights.argtypes = [P, i32, P, P, P, P, P]
        L.oracle_accumulate.argtypes = [P, i32, P, P, i32, P]
        L.oracle_render_fwd.argtypes = [P, i32, P, P, P, P, P, P, P]
        L.oracle_render_bwd.argtypes = [P, i32, P, P, P, P, P, P, P, P, P]
        L.oracle_render_weights_bwd.argtypes = [P, i32, P, P, P, P, P]
        L.oracle_accumulate_bwd.argtypes = [P, i32, P, P, i32, P, P, P]
        L.oracle_unpack_info.argtypes = [P, i32, P]
        L.oracle_update_grid.argtypes = [P, P, i64, P, P, i64, f32, f32]
        L.oracle_field_sigma.restype = f32
        L.oracle_field_sigma.argtypes = [P, P, P, P]
        L.oracle_field_query.restype = ctypes.c_int
        L.oracle_field_query.argtypes = [P, P, P, P, i64, P]
        L.oracle_march_fused.restype = i64
        L.oracle_march_fused.argtypes = [P, P, i32, P, P, i32, P, f32, f32, f32, f32, f32, i32, i32, P, P, P, f32,
                                         f32, P, P, P, P, P, i64]
        for f in ("oracle_render_weights", "oracle_accumulate", "oracle_render_fwd", "oracle_render_bwd",
                  "oracle_render_weights_bwd", "oracle_accumulate_bwd",
                  "oracle_unpack_info", "oracle_update_grid"):
            getattr(L, f).restype = ctypes.c_int
        _lib = L
    return _lib


def _p(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def _c(a, dt):
    return None if a is None else np.ascontiguousarray(a, dtype=dt)


@dataclass
class Packed:
    packed_info: np.ndarray  # (R, 2) int32 (offset, count)
    t_starts: np.ndarray  # (M,) float32
    t_ends: np.ndarray  # (M,) float32
    ray_indices: np.ndarray  # (M,) int32

    @property
    def n_samples(self) -> int:
        return int(self.t_starts.shape[0])


def march(rays_o, rays_d, bits, res, aabb, near_plane=0.0, far_plane=1e10, dt_min=1e-2, dt_max=None,
          cone=0.0, max_steps=1024, n_levels=1, n_slots=1, ray_time=None, ray_slot=None, contraction=0) -> Packed:
    """Occupancy-grid ray marching (Sec. 2.1), float32 replica, dense lattice walk."""
    o = _c(rays_o, np.float32).reshape(-1, 3)
    d = _c(rays_d, np.float32).reshape(-1, 3)
    R = o.shape[0]
    bits = _c(bits, np.uint32)
    res = np.ascontiguousarray(np.asarray(res, dtype=np.int32).reshape(3))
    box = np.ascontiguousarray(np.asarray(aabb, dtype=np.float32).reshape(6))
    tt = _c(ray_time, np.float32)
    sl = _c(ray_slot, np.int32)
    dt_max = dt_min if dt_max is None else dt_max
    pi = np.zeros((R, 2), dtype=np.int32)
    args = lambda ts, te, ri, cap: (
        _p(o), _p(d), _p(tt), _p(sl), R, _p(bits), _p(res), n_levels, n_slots, _p(box),
        near_plane, far_plane, dt_min, dt_max, cone, max_steps, int(contraction), _p(pi), _p(ts), _p(te), _p(ri),
        cap)
    n = lib().oracle_march(*args(None, None, None, 0))
    if n < 0:
        raise ValueError("oracle_march: invalid arguments")
    ts = np.empty(n, np.float32)
    te = np.empty(n, np.float32)
    ri = np.empty(n, np.int32)
    n2 = lib().oracle_march(*args(ts, te, ri, n))
    assert n2 == n
    return Packed(pi, ts, te, ri)


def prune(packed_info, t_starts, t_ends, sigmas, early_stop_eps, alpha_thre):
    """Early-stop + alpha-threshold pruning and re-packing (Sec. 2.1), float32 decision.

    Returns (Packed, keep_mask (M,) bool, optical_depth (M,) float32 = O_i).
    """
    pi = _c(packed_info, np.int32).reshape(-1, 2)
    ts, te, sg = (_c(a, np.float32).reshape(-1) for a in (t_starts, t_ends, sigmas))
    R, M = pi.shape[0], ts.shape[0]
    keep = np.zeros(M, np.uint8)
    od = np.zeros(M, np.float32)
    pio = np.zeros((R, 2), np.int32)
    args = lambda a, b, c, cap: (_p(pi), R, _p(ts), _p(te), _p(sg), early_stop_eps, alpha_thre, _p(keep), _p(od),
                                 _p(pio), _p(a), _p(b), _p(c), cap)
    n = lib().oracle_prune(*args(None, None, None, 0))
    a, b, c = np.empty(n, np.float32), np.empty(n, np.float32), np.empty(n, np.int32)
    lib().oracle_prune(*args(a, b, c, n))
    return Packed(pio, a, b, c), keep.astype(bool), od


def render_weights(packed_info, t_starts, t_ends, sigmas):
    """Eq. 1 weights w_i = T_i alpha_i and transmittance T_i (float64)."""
    pi = _c(packed_info, np.int32).reshape(-1, 2)
    ts, te, sg = (_c(a, np.float32).reshape(-1) for a in (t_starts, t_ends, sigmas))
    w = np.zeros(ts.shape[0], np.float64)
    T = np.zeros(ts.shape[0], np.float64)
    if lib().oracle_render_weights(_p(pi), pi.shape[0], _p(ts), _p(te), _p(sg), _p(w), _p(T)) != 0:
        raise MemoryError
    return w, T


def accumulate(packed_info, weights, values=None):
    """sum_i w_i v_i per ray (Sec. 2.2: any sample attribute); values (M, C) or None (C = 1)."""
    pi = _c(packed_info, np.int32).reshape(-1, 2)
    w = _c(weights, np.float64).reshape(-1)
    if values is None:
        v, C = None, 1
    else:
        v = _c(values, np.float32).reshape(w.shape[0], -1)
        C = v.shape[1]
    out = np.zeros((pi.shape[0], C), np.float64)
    lib().oracle_accumulate(_p(pi), pi.shape[0], _p(w), _p(v), C, _p(out))
    return out


def render_fwd(packed_info, t_starts, t_ends, sigmas, rgbs):
    """Eq. 1 quadrature: (color (R,3), opacity (R,), depth (R,)), float64."""
    pi = _c(packed_info, np.int32).reshape(-1, 2)
    ts, te, sg = (_c(a, np.float32).reshape(-1) for a in (t_starts, t_ends, sigmas))
    rgb = _c(rgbs, np.float32).reshape(-1, 3)
    R = pi.shape[0]
    col, op, dp = np.zeros((R, 3)), np.zeros(R), np.zeros(R)
    if lib().oracle_render_fwd(_p(pi), R, _p(ts), _p(te), _p(sg), _p(rgb), _p(col), _p(op), _p(dp)) != 0:
        raise MemoryError
    return col, op, dp


def render_bwd(packed_info, t_starts, t_ends, sigmas, rgbs, g_color=None, g_opacity=None, g_depth=None):
    """Analytic gradient of the Eq. 1 quadrature: (d_sigmas (M,), d_rgbs (M,3)), float64."""
    pi = _c(packed_info, np.int32).reshape(-1, 2)
    ts, te, sg = (_c(a, np.float32).reshape(-1) for a in (t_starts, t_ends, sigmas))
    rgb = _c(rgbs, np.float32).reshape(-1, 3)
    R, M = pi.shape[0], ts.shape[0]
    gc = _c(g_color, np.float64)
    ga = _c(g_opacity, np.float64)
    gd = _c(g_depth, np.float64)
    ds, dr = np.zeros(M), np.zeros((M, 3))
    if lib().oracle_render_bwd(_p(pi), R, _p(ts), _p(te), _p(sg), _p(rgb), _p(gc), _p(ga), _p(gd), _p(ds), _p(dr)) != 0:
        raise MemoryError
    return ds, dr


def render_weights_bwd(packed_info, t_starts, t_ends, sigmas, g_weights):
    """dL/dsigma for an upstream dL/dw (float64): delta_k (g_k T_{k+1} - sum_{i>k} g_i w_i)."""
    pi = _c(packed_info, np.int32).reshape(-1, 2)
    ts, te, sg = (_c(a, np.float32).reshape(-1) for a in (t_starts, t_ends, sigmas))
    g = _c(g_weights, np.float64).reshape(-1)
    ds = np.zeros(ts.shape[0])
    if lib().oracle_render_weights_bwd(_p(pi), pi.shape[0], _p(ts), _p(te), _p(sg), _p(g), _p(ds)) != 0:
        raise MemoryError
    return ds


def accumulate_bwd(packed_info, weights, values, g_out):
    """(dL/dw (M,), dL/dv (M, C) or None) of out[r] = sum_i w_i v_i for dL/dout (R, C), float64."""
    pi = _c(packed_info, np.int32).reshape(-1, 2)
    w = _c(weights, np.float64).reshape(-1)
    g = _c(g_out, np.float64).reshape(pi.shape[0], -1)
    C = g.shape[1]
    v = None if values is None else _c(values, np.float32).reshape(w.shape[0], C)
    dw = np.zeros(w.shape[0])
    dv = None if v is None else np.zeros((w.shape[0], C))
    lib().oracle_accumulate_bwd(_p(pi), pi.shape[0], _p(w), _p(v), C, _p(g), _p(dw), _p(dv))
    return dw, dv


def unpack_info(packed_info, n_samples):
    pi = _c(packed_info, np.int32).reshape(-1, 2)
    ri = np.zeros(n_samples, np.int32)
    lib().oracle_unpack_info(_p(pi), pi.shape[0], _p(ri))
    return ri


def update_grid(ema, cells, sigmas, decay, thre, alpha_step=None):
    """Occupancy-grid EMA update (Sec. 2.1, via Instant-NGP App. E.2): returns (ema', bits').
    With ``alpha_step`` = dt the bits follow the paper's opacity criterion itself: a
    cell is occupied where 1 - exp(-ema dt) > thre, evaluated in float64 on the
    float32 state (the density threshold of the library's form is not used)."""
    e = np.array(ema, dtype=np.float32, copy=True).reshape(-1)
    c = _c(cells, np.int32).reshape(-1)
    s = _c(sigmas, np.float32).reshape(-1)
    bits = np.zeros((e.size + 31) // 32, np.uint32)
    if lib().oracle_update_grid(_p(e), _p(bits), e.size, _p(c), _p(s), c.size, decay,
                                thre if alpha_step is None else np.inf) != 0:
        raise ValueError("cell index out of range")
    if alpha_step is not None:
        occ = (1.0 - np.exp(-e.astype(np.float64) * float(alpha_step))) > float(thre)
        pad = np.zeros(bits.size * 32, bool)
        pad[:e.size] = occ
        bits = (pad.reshape(-1, 32).astype(np.uint64) << np.arange(32, dtype=np.uint64)).sum(1).astype(np.uint32)
    return e, bits


def grid_sat(bits, res, n_grids=1):
    """Summed-area table of a bit-packed grid (the marcher's acceleration structure,
    not part of the paper's method), by its definition: per grid g, entry (x, y, z)
    of the (res0+1, res1+1, res2+1) corner lattice counts the occupied cells
    (i, j, k) with i < x, j < y, k < z; kept modulo 2^16 as uint16; grids one after
    the other, x-major, z fastest."""
    r0, r1, r2 = (int(v) for v in res)
    n = n_grids * r0 * r1 * r2
    w = np.ascontiguousarray(bits, dtype=np.uint32)
    occ = ((w[np.arange(n) >> 5] >> (np.arange(n) & 31).astype(np.uint32)) & 1).astype(np.int64)
    occ = occ.reshape(n_grids, r0, r1, r2)
    s = np.zeros((n_grids, r0 + 1, r1 + 1, r2 + 1), np.int64)
    s[:, 1:, 1:, 1:] = occ.cumsum(1).cumsum(2).cumsum(3)
    return (s % 65536).astype(np.uint16).reshape(-1)


def grid_brick_summary(bits, res, n_grids=1):
    """Brick summary stored after the summed-area table (also an acceleration
    structure of the marcher, not part of the paper's method), by its definition:
    per grid, for every brick of 8 x 8 x 8 cells (clipped at the grid's faces),
    2 bits: 1 when none of its cells is occupied, 2 when all are; 8 bricks per
    uint16 entry (brick b in bits 2 (b mod 8) .. 2 (b mod 8) + 1 of entry b // 8),
    bricks x-major and z fastest, ceil(nb0 nb1 nb2 / 8) entries per grid,
    nb_k = ceil(res_k / 8). Computed from the cells, not from the table."""
    r0, r1, r2 = (int(v) for v in res)
    n = n_grids * r0 * r1 * r2
    w = np.ascontiguousarray(bits, dtype=np.uint32)
    occ = ((w[np.arange(n) >> 5] >> (np.arange(n) & 31).astype(np.uint32)) & 1).astype(bool)
    occ = occ.reshape(n_grids, r0, r1, r2)
    nb = [(r + 7) // 8 for r in (r0, r1, r2)]
    per = (nb[0] * nb[1] * nb[2] + 7) // 8
    out = np.zeros((n_grids, per), np.uint16)
    for g in range(n_grids):
        b = 0
        for bx in range(nb[0]):
            for by in range(nb[1]):
                for bz in range(nb[2]):
                    cells = occ[g, 8 * bx:8 * bx + 8, 8 * by:8 * by + 8, 8 * bz:8 * bz + 8]
                    v = (1 if not cells.any() else 0) | (2 if cells.all() else 0)
                    out[g, b // 8] |= np.uint16(v << (2 * (b % 8)))
                    b += 1
    return out.reshape(-1)


def field_query(field, field_box, xyz):
    """Density field of the fused path (F1 in oracle.c): trilinear between the
    vertex values field[i, j, k] of a lattice over field_box = (lo, hi), zero
    outside; float32 replica. Returns sigma (n,) float32."""
    g = _c(field, np.float32)
    G = np.ascontiguousarray(np.asarray(g.shape, dtype=np.int32).reshape(3))
    box = np.ascontiguousarray(np.asarray(field_box, dtype=np.float32).reshape(6))
    x = _c(xyz, np.float32).reshape(-1, 3)
    out = np.zeros(x.shape[0], np.float32)
    if lib().oracle_field_query(_p(g), _p(G), _p(box), _p(x), x.shape[0], _p(out)) != 0:
        raise ValueError("oracle_field_query: invalid field")
    return out


def march_fused(rays_o, rays_d, bits, res, aabb, field, field_box, early_stop_eps, alpha_thre, near_plane=0.0,
                far_plane=1e10, dt_min=1e-2, dt_max=None, cone=0.0, max_steps=1024, n_levels=1, contraction=0):
    """Fused march + density + prune for inference (F2 in oracle.c, Sec. 2.1):
    what prune() keeps of march()'s samples with sigma = field_query() at each
    sample's midpoint. Returns (Packed of the kept samples, sigmas (S,) float32)."""
    o = _c(rays_o, np.float32).reshape(-1, 3)
    d = _c(rays_d, np.float32).reshape(-1, 3)
    R = o.shape[0]
    bits = _c(bits, np.uint32)
    res = np.ascontiguousarray(np.asarray(res, dtype=np.int32).reshape(3))
    box = np.ascontiguousarray(np.asarray(aabb, dtype=np.float32).reshape(6))
    g = _c(field, np.float32)
    G = np.ascontiguousarray(np.asarray(g.shape, dtype=np.int32).reshape(3))
    fbox = np.ascontiguousarray(np.asarray(field_box, dtype=np.float32).reshape(6))
    dt_max = dt_min if dt_max is None else dt_max
    pi = np.zeros((R, 2), dtype=np.int32)
    args = lambda ts, te, ri, sg, cap: (
        _p(o), _p(d), R, _p(bits), _p(res), n_levels, _p(box), near_plane, far_plane, dt_min, dt_max, cone,
        max_steps, int(contraction), _p(g), _p(G), _p(fbox), early_stop_eps, alpha_thre, _p(pi), _p(ts), _p(te),
        _p(ri), _p(sg), cap)
    n = lib().oracle_march_fused(*args(None, None, None, None, 0))
    if n < 0:
        raise ValueError("oracle_march_fused: invalid arguments")
    ts, te, sg = np.empty(n, np.float32), np.empty(n, np.float32), np.empty(n, np.float32)
    ri = np.empty(n, np.int32)
    assert lib().oracle_march_fused(*args(ts, te, ri, sg, n)) == n
    return Packed(pi, ts, te, ri), sg

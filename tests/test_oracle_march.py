"""Pins of the oracle's ray marching (Sec. 2.1 "Ray Marching") against things other
than itself: a hand-derived worked example, closed-form counts, an independent
float64 voxel traversal (Amanatides & Woo 1987) on tiny random grids, a float64
point-wise level/cell lookup for cascades, and the time-bin / slot selection.
"""
import json
import math
import os

import numpy as np
import pytest

from paper_2210_04847_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _grid_from_cells(res, cells, n_levels=1, n_slots=1):
    rx, ry, rz = res
    occ = np.zeros(n_slots * n_levels * rx * ry * rz, bool)
    for c in cells:
        occ[(c[0] * ry + c[1]) * rz + c[2]] = True
    return synth.pack_bits(occ)


def test_worked_example(orc):
    g = json.load(open(os.path.join(GOLDEN, "march_worked_example.json")))
    bits = _grid_from_cells(g["res"], g["occupied_cells"])
    p = orc.march(g["rays_o"], g["rays_d"], bits, g["res"], g["aabb"], g["near_plane"], g["far_plane"],
                  g["dt"], g["dt"], 0.0, g["max_steps"])
    assert p.packed_info.tolist() == g["packed_info"]
    assert p.t_starts.tolist() == g["t_starts"]
    assert p.t_ends.tolist() == g["t_ends"]
    assert p.ray_indices.tolist() == g["ray_indices"]


# ---------------------------------------------------------------------------
# independent float64 references
# ---------------------------------------------------------------------------


def slab64(o, d, lo, hi, near_plane, far_plane):
    """Textbook ray/box slab intersection in float64 (Kay & Kajiya 1986)."""
    t_in, t_out = -math.inf, math.inf
    for a in range(3):
        if d[a] == 0.0:
            if o[a] < lo[a] or o[a] > hi[a]:
                return None
            continue
        t0, t1 = (lo[a] - o[a]) / d[a], (hi[a] - o[a]) / d[a]
        t_in, t_out = max(t_in, min(t0, t1)), min(t_out, max(t0, t1))
    near, far = max(t_in, near_plane), min(t_out, far_plane)
    return (near, far) if near < far else None


def dda_segments(o, d, lo, hi, res, t0, t1):
    """Voxel traversal: list of (t_enter, t_exit, (ix, iy, iz)) crossed on [t0, t1]."""
    o, d, lo, hi = (np.asarray(v, np.float64) for v in (o, d, lo, hi))
    res = np.asarray(res)
    size = (hi - lo) / res
    p = o + d * (0.5 * (t0 + min(t1, t0 + 1e-9)))
    idx = np.clip(np.floor((p - lo) / size).astype(np.int64), 0, res - 1)
    step = np.sign(d).astype(np.int64)
    tmax = np.full(3, math.inf)
    tdelta = np.full(3, math.inf)
    for a in range(3):
        if d[a] > 0:
            tmax[a] = (lo[a] + (idx[a] + 1) * size[a] - o[a]) / d[a]
            tdelta[a] = size[a] / d[a]
        elif d[a] < 0:
            tmax[a] = (lo[a] + idx[a] * size[a] - o[a]) / d[a]
            tdelta[a] = -size[a] / d[a]
    segs = []
    t = t0
    while t < t1:
        a = int(np.argmin(tmax))
        tn = min(tmax[a], t1)
        segs.append((t, tn, tuple(int(v) for v in idx)))
        t = tmax[a]
        idx[a] += step[a]
        if idx[a] < 0 or idx[a] >= res[a]:
            break
        tmax[a] += tdelta[a]
    return segs


def _cell_on(occ3, cell):
    return bool(occ3[cell])


def _check_ray_against_dda(o, d, occ3, aabb, res, dt, max_steps, emitted_ts, tol=2e-5):
    lo, hi = np.array(aabb[:3], float), np.array(aabb[3:], float)
    o64 = np.asarray(o, np.float64)
    d64 = np.asarray(d, np.float64)
    clip = slab64(o64, d64, lo, hi, 0.0, 1e10)
    if clip is None:
        assert len(emitted_ts) == 0
        return 0
    near, far = clip
    segs = dda_segments(o64, d64, lo, hi, res, near, far)
    bounds = np.array([s[0] for s in segs] + [segs[-1][1]]) if segs else np.array([near, far])
    expect, ambiguous = set(), set()
    k = 0
    while k < max_steps and near + k * dt < far + tol:
        ts = near + k * dt
        te = min(near + (k + 1) * dt, far)
        mid = 0.5 * (ts + te)
        amb = abs(ts - far) < tol or abs(near + (k + 1) * dt - far) < tol
        amb |= bool(np.min(np.abs(bounds - mid)) < tol)
        if amb:
            ambiguous.add(k)
        elif ts < far:
            for s in segs:
                if s[0] <= mid < s[1]:
                    if _cell_on(occ3, s[2]):
                        expect.add(k)
                    break
        k += 1
    got = set()
    for ts in emitted_ts:
        kk = int(round((float(ts) - near) / dt))
        assert abs(float(ts) - (near + kk * dt)) < tol, "sample start off the lattice"
        got.add(kk)
    diff = (got ^ expect) - ambiguous
    assert not diff, "emitted set differs from the voxel traversal at lattice points %s" % sorted(diff)[:10]
    return len(got)


@pytest.mark.parametrize("seed", range(6))
def test_random_tiny_grids_vs_voxel_traversal(orc, seed):
    rng_res = [2, 3, 4, 5, 7, 8][seed]
    res = (rng_res, max(2, rng_res - 1), rng_res + 1)
    n_cells = res[0] * res[1] * res[2]
    occ = synth.rand_uniform(seed, 1, n_cells) < 0.5
    bits = synth.pack_bits(occ)
    occ3 = occ.reshape(res)
    aabb = (-1.0, -0.75, -1.25, 1.0, 1.25, 0.5)
    n = 64
    o = synth.random_unit_vectors(seed, 2, n) * 3.0
    tgt = synth.rand_uniform(seed, 3, 3 * n, -0.9, 0.9).reshape(n, 3)
    d = tgt - o
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    # axis-parallel rays and rays starting inside the box
    d[:6] = np.array([[1, 0, 0], [-1, 0, 0], [0, 1, 0], [0, -1, 0], [0, 0, 1], [0, 0, -1]], float)
    o[:6] = np.array([[-2, 0.1, -0.3], [2, -0.2, 0.1], [0.3, -2, -0.4], [-0.1, 2, 0.2], [0.2, 0.3, -2], [0.1, 0.2, 2]])
    o[6:12] = synth.rand_uniform(seed, 4, 18, -0.5, 0.4).reshape(6, 3)
    o32, d32 = o.astype(np.float32), d.astype(np.float32)
    dt = 0.37 * (2.0 / max(res))  # comparable to the cell size: midpoint placement matters
    p = orc.march(o32, d32, bits, res, aabb, 0.0, 1e10, dt, dt, 0.0, 4096)
    total = 0
    for r in range(n):
        off, cnt = p.packed_info[r]
        total += _check_ray_against_dda(o32[r], d32[r], occ3, aabb, res, dt, 4096, p.t_starts[off : off + cnt])
    assert total == p.n_samples > 0


def test_full_grid_closed_form(orc):
    """All cells occupied: samples tile [near, far] contiguously; count = ceil((far-near)/dt)."""
    res = (8, 8, 8)
    bits = synth.pack_bits(np.ones(512, bool))
    aabb = (-1, -1, -1, 1, 1, 1)
    n = 200
    o = synth.random_unit_vectors(5, 1, n) * 2.5
    d = synth.rand_uniform(5, 2, 3 * n, -0.5, 0.5).reshape(n, 3) - o
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    o32, d32 = o.astype(np.float32), d.astype(np.float32)
    dt = 0.01
    p = orc.march(o32, d32, bits, res, aabb, 0.0, 1e10, dt, dt, 0.0, 100000)
    hit = 0
    for r in range(n):
        off, cnt = p.packed_info[r]
        clip = slab64(o32[r].astype(float), d32[r].astype(float), [-1] * 3, [1] * 3, 0.0, 1e10)
        if clip is None:
            assert cnt == 0
            continue
        hit += 1
        near, far = clip
        ts, te = p.t_starts[off : off + cnt], p.t_ends[off : off + cnt]
        expect = math.ceil((far - near) / dt)
        assert abs(cnt - expect) <= 1
        assert abs(ts[0] - near) < 1e-5 and abs(te[-1] - far) < 1e-5
        assert np.all(te[:-1] == ts[1:]), "contiguity t_end[k] == t_start[k+1]"
        assert np.all(te > ts)
        # sum of interval lengths telescopes to far - near
        assert abs(float(np.sum(te.astype(np.float64) - ts)) - (far - near)) < 1e-4
    assert hit > 150


def test_empty_grid_and_degenerate_rays(orc):
    res = (4, 4, 4)
    aabb = (-1, -1, -1, 1, 1, 1)
    o = np.array([[-2, 0, 0]] * 3, np.float32)
    d = np.array([[1, 0, 0]] * 3, np.float32)
    p = orc.march(o, d, np.zeros(2, np.uint32), res, aabb, 0.0, 1e10, 0.1, 0.1, 0.0, 100)
    assert p.n_samples == 0 and p.packed_info[:, 1].tolist() == [0, 0, 0]
    full = synth.pack_bits(np.ones(64, bool))
    nan, inf = float("nan"), float("inf")
    o = np.array([[-2, 0, 0], [nan, 0, 0], [-2, 0, 0], [0, 0, 0], [-2, 5, 0], [0, 0, 0], [-2, 0, 0]], np.float32)
    d = np.array([[1, 0, 0], [1, 0, 0], [inf, 0, 0], [0, 0, 0], [1, 0, 0], [0, 1, 0], [1, 0, 0]], np.float32)
    p = orc.march(o, d, full, res, aabb, 0.0, 1e10, 0.5, 0.5, 0.0, 100)
    counts = p.packed_info[:, 1].tolist()
    # ray 0: [1, 3] -> 4 samples; NaN/inf rays and a ray outside the y-slab emit nothing;
    # d == 0 everywhere inside the box: every slab passes, t in [0, 1e10) -> max_steps samples
    assert counts[0] == 4 and counts[1] == 0 and counts[2] == 0 and counts[4] == 0
    assert counts[3] == 100
    assert counts[5] == 2  # from the centre along +y: t in [0, 1], dt = 0.5
    # near/far planes: far_plane cuts, near_plane >= far gives nothing
    p = orc.march(o[:1], d[:1], full, res, aabb, 1.2, 2.0, 0.5, 0.5, 0.0, 100)
    assert np.allclose(p.t_starts, [1.2, 1.7], rtol=1e-7) and np.allclose(p.t_ends, [1.7, 2.0], rtol=1e-7)
    p = orc.march(o[:1], d[:1], full, res, aabb, 2.5, 2.5, 0.5, 0.5, 0.0, 100)
    assert p.n_samples == 0
    # max_steps caps the lattice
    p = orc.march(o[:1], d[:1], full, res, aabb, 0.0, 1e10, 0.01, 0.01, 0.0, 37)
    assert p.n_samples == 37


def _level_cell64(x, aabb, res, n_levels, tol):
    """float64 finest-level/cell lookup by normalised max-norm; None if within tol of a boundary."""
    lo, hi = np.array(aabb[:3], float), np.array(aabb[3:], float)
    c, h = 0.5 * (lo + hi), 0.5 * (hi - lo)
    q = (x - c) / h  # level-0 box is q in [-1, 1)
    for l in range(n_levels):
        s = 2.0**l
        if np.any(np.abs(np.abs(q) - s) < tol * s):
            return "amb"
        if np.all((q >= -s) & (q < s)):
            u = (q + s) / (2 * s) * np.asarray(res)
            fr = u - np.floor(u)
            if np.any(np.minimum(fr, 1 - fr) < tol * np.asarray(res)):
                return "amb"
            return l, tuple(int(v) for v in np.floor(u))
    return None


def test_cascade_levels_vs_float64_lookup(orc):
    res = (4, 4, 4)
    L = 3
    n_cells = L * 64
    occ = synth.rand_uniform(11, 1, n_cells) < 0.5
    bits = synth.pack_bits(occ)
    aabb = (-1.0, -1.0, -1.0, 1.0, 1.0, 1.0)
    n = 40
    o = synth.rand_uniform(11, 2, 3 * n, -0.8, 0.8).reshape(n, 3)
    d = synth.random_unit_vectors(11, 3, n)
    o32, d32 = o.astype(np.float32), d.astype(np.float32)
    dt = 0.05
    p = orc.march(o32, d32, bits, res, aabb, 0.0, 1e10, dt, dt, 0.0, 4096, n_levels=L)
    occ4 = occ.reshape(L, *res)
    checked = 0
    for r in range(n):
        off, cnt = p.packed_info[r]
        emitted = set(np.round((p.t_starts[off : off + cnt].astype(float) - 0.0) / dt).astype(int).tolist())
        # the ray starts inside every level: near = 0 (t_in < 0); far = exit of the outermost box
        clip = slab64(o32[r].astype(float), d32[r].astype(float), [-4.0] * 3, [4.0] * 3, 0.0, 1e10)
        near, far = clip
        k = 0
        while near + k * dt < far - 1e-5:
            ts, te = near + k * dt, min(near + (k + 1) * dt, far)
            x = o32[r].astype(float) + d32[r].astype(float) * 0.5 * (ts + te)
            lc = _level_cell64(x, aabb, res, L, 1e-6)
            if lc != "amb":
                want = lc is not None and bool(occ4[lc[0]][lc[1]])
                assert (k in emitted) == want, (r, k, lc)
                checked += 1
            k += 1
    assert checked > 1000


def test_cone_lattice_properties(orc):
    """Cone steps: dt_k = clamp(t_k * cone, dt_min, dt_max); contiguous, increasing intervals,
    count close to the float64 recurrence."""
    res = (8, 8, 8)
    bits = synth.pack_bits(np.ones(512, bool))
    aabb = (-100, -100, -100, 100, 100, 100)
    n = 16
    o = synth.rand_uniform(3, 1, 3 * n, -5, 5).reshape(n, 3).astype(np.float32)
    d = synth.random_unit_vectors(3, 2, n).astype(np.float32)
    cone, dmin, dmax = 1.0 / 256, 1e-3, 1.0
    p = orc.march(o, d, bits, res, aabb, 0.05, 1000.0, dmin, dmax, cone, 100000)
    for r in range(n):
        off, cnt = p.packed_info[r]
        ts = p.t_starts[off : off + cnt].astype(np.float64)
        te = p.t_ends[off : off + cnt].astype(np.float64)
        assert ts[0] == np.float32(0.05)
        assert np.all(p.t_ends[off : off + cnt - 1] == p.t_starts[off + 1 : off + cnt])
        steps = te[:-1] - ts[:-1]
        want = np.clip(ts[:-1] * cone, dmin, dmax)
        assert np.allclose(steps, want, rtol=1e-4, atol=1e-7)
        far = slab64(o[r].astype(float), d[r].astype(float), [-100] * 3, [100] * 3, 0.05, 1000.0)[1]
        t, k = 0.05, 0
        while t < far:
            t += min(max(t * cone, dmin), dmax)
            k += 1
        assert abs(cnt - k) <= 2


def test_time_bins_and_slots(orc):
    """Only the grid of the ray's time bin (or slot) is consulted (M5)."""
    res = (4, 4, 4)
    n_slots = 4
    aabb = (-1, -1, -1, 1, 1, 1)
    occ = np.zeros(n_slots * 64, bool)
    occ[2 * 64 : 3 * 64] = True  # only bin 2 is occupied
    bits = synth.pack_bits(occ)
    n = 9
    o = np.tile(np.array([[-2, 0.1, 0.2]], np.float32), (n, 1))
    d = np.tile(np.array([[1, 0, 0]], np.float32), (n, 1))
    times = np.array([0.0, 0.2, 0.49, 0.5, 0.6, 0.7499, 0.75, 1.0, -0.3], np.float32)
    p = orc.march(o, d, bits, res, aabb, 0.0, 1e10, 0.25, 0.25, 0.0, 100, n_slots=n_slots, ray_time=times)
    counts = p.packed_info[:, 1].tolist()
    assert counts == [0, 0, 0, 8, 8, 8, 0, 0, 0]
    slots = np.array([2, 0, 2, 3, 1, 2, 2, 0, 3], np.int32)
    p = orc.march(o, d, bits, res, aabb, 0.0, 1e10, 0.25, 0.25, 0.0, 100, n_slots=n_slots, ray_slot=slots)
    assert p.packed_info[:, 1].tolist() == [8 if s == 2 else 0 for s in slots]


# ---------------------------------------------------------------------------
# contracted unbounded space (Sec. 2.1 "Scene Contraction"; Mip-NeRF 360 Eq. 10)
# ---------------------------------------------------------------------------


def test_contraction_identity_inside_unit_ball(orc):
    """Inside the unit ball the contraction is the identity: rays that stay inside
    march exactly as on a plain grid over [-2, 2]^3 (u = (x + 2) res / 4 both ways)."""
    res = (16, 16, 16)
    occ = synth.rand_uniform(31, 1, 16 ** 3) < 0.5
    bits = synth.pack_bits(occ)
    n = 200
    # |o| <= 0.25 sqrt(3) < 0.44 and t <= 0.5: every point stays inside the unit ball
    o = synth.rand_uniform(31, 2, 3 * n, -0.25, 0.25).reshape(n, 3).astype(np.float32)
    d = synth.random_unit_vectors(31, 3, n).astype(np.float32)
    args = dict(near_plane=0.0, far_plane=0.5, dt_min=0.01, dt_max=0.01, max_steps=1024)
    c = orc.march(o, d, bits, res, (-1, -1, -1, 1, 1, 1), contraction=1, **args)
    p = orc.march(o, d, bits, res, (-2, -2, -2, 2, 2, 2), **args)
    assert c.n_samples > 0
    assert np.array_equal(c.packed_info, p.packed_info)
    assert np.array_equal(c.t_starts, p.t_starts) and np.array_equal(c.ray_indices, p.ray_indices)


@pytest.mark.parametrize("sign", [1.0, -1.0])
def test_contraction_along_an_axis(orc, sign):
    """On the x axis a point at distance t > 1 maps to x_c = 2 - 1/t. With 16 cells
    over [-2, 2], cell 14 (cell 1 for -x) holds x_c in [1.5, 1.75): t in [2, 4). Only
    that cell is occupied, dt = 1/64 from t = 0: the samples are exactly k = 128..255."""
    res = (16, 16, 16)
    occ = np.zeros((16, 16, 16), bool)
    occ[14 if sign > 0 else 1, 8, 8] = True
    o = np.zeros((1, 3), np.float32)
    d = np.array([[sign, 0.0, 0.0]], np.float32)
    m = orc.march(o, d, synth.pack_bits(occ.reshape(-1)), res, (-1, -1, -1, 1, 1, 1), near_plane=0.0,
                  far_plane=100.0, dt_min=1.0 / 64, dt_max=1.0 / 64, max_steps=8192, contraction=1)
    assert m.n_samples == 128
    np.testing.assert_array_equal(m.t_starts, np.arange(128, 256, dtype=np.float32) / 64)


def test_grid_sat_definition_by_brute_force(orc):
    """oracle.grid_sat against a triple loop over cells on random small grids (two
    grids, anisotropic), and box counts from it modulo 2^16 on a grid whose totals
    wrap: every box below 2^16 cells gets its exact count."""
    res = (3, 5, 4)
    occ = synth.rand_uniform(3, 1, 2 * 60) < 0.45
    s = orc.grid_sat(synth.pack_bits(occ), res, 2).reshape(2, 4, 6, 5)
    o = occ.reshape(2, 3, 5, 4)
    for g in range(2):
        for x in range(4):
            for y in range(6):
                for z in range(5):
                    assert s[g, x, y, z] == o[g, :x, :y, :z].sum()
    res = (64, 64, 64)  # 262144 cells, mostly occupied: totals wrap modulo 2^16
    occ = synth.rand_uniform(3, 2, 64 ** 3) < 0.9
    s = orc.grid_sat(synth.pack_bits(occ), res).reshape(65, 65, 65).astype(np.int64)
    o = occ.reshape(64, 64, 64)
    assert s[64, 64, 64] == o.sum() % 65536
    lo = synth.rand_int(3, 3, 60, 40).reshape(20, 3)
    ext = 1 + synth.rand_int(3, 4, 60, 24).reshape(20, 3)
    for (x0, y0, z0), (ex, ey, ez) in zip(lo, ext):
        x1, y1, z1 = x0 + ex, y0 + ey, z0 + ez
        cnt = (s[x1, y1, z1] - s[x0, y1, z1] - s[x1, y0, z1] - s[x1, y1, z0] + s[x0, y0, z1] + s[x0, y1, z0]
               + s[x1, y0, z0] - s[x0, y0, z0]) % 65536
        assert cnt == o[x0:x1, y0:y1, z0:z1].sum()


def _brick_states(summary, per_grid, g, n_bricks):
    """2-bit state of each brick of grid g from the packed summary."""
    e = summary[g * per_grid:(g + 1) * per_grid].astype(np.int64)
    return np.array([(e[b // 8] >> (2 * (b % 8))) & 3 for b in range(n_bricks)])


def test_brick_summary_by_construction():
    """The marcher's brick summary (2 bits per 8^3 block of cells: 1 empty, 2 full),
    on grids whose answer is known: empty, full (bricks clipped at the faces count
    their in-grid cells), one occupied cell, one fully occupied brick."""
    from oracle import grid_brick_summary
    res = (20, 9, 17)  # bricks 3 x 2 x 3, the last ones clipped
    n = 20 * 9 * 17
    nb = 18
    per = (nb + 7) // 8
    empty = grid_brick_summary(synth.pack_bits(np.zeros(n, bool)), res)
    full = grid_brick_summary(synth.pack_bits(np.ones(n, bool)), res)
    assert np.all(_brick_states(empty, per, 0, nb) == 1) and np.all(_brick_states(full, per, 0, nb) == 2)
    occ = np.zeros((20, 9, 17), bool)
    occ[11, 8, 16] = True  # brick (1, 1, 2) = index (1 * 2 + 1) * 3 + 2 = 11
    st = _brick_states(grid_brick_summary(synth.pack_bits(occ.reshape(-1)), res), per, 0, nb)
    assert st[11] == 0 and np.all(np.delete(st, 11) == 1)
    occ[:] = False
    occ[16:20, 8:9, 0:8] = True  # brick (2, 1, 0), clipped to 4 x 1 x 8 cells: index (2 * 2 + 1) * 3 = 15
    st = _brick_states(grid_brick_summary(synth.pack_bits(occ.reshape(-1)), res), per, 0, nb)
    assert st[15] == 2 and np.all(np.delete(st, 15) == 1)
    # two grids one after the other
    two = np.concatenate([np.ones(n, bool), np.zeros(n, bool)])
    s2 = grid_brick_summary(synth.pack_bits(two), res, 2)
    assert np.all(_brick_states(s2, per, 0, nb) == 2) and np.all(_brick_states(s2, per, 1, nb) == 1)

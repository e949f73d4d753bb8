"""Pins of the oracle's density field and fused march + prune (the inference path:
transmittance from the field's density while marching, Sec. 2.1 "Pruning Empty and
Occluded Regions") against things other than itself: trilinear interpolation
reproduces multilinear functions exactly (up to float32 rounding), a float64
eight-corner weighting of random vertex values, exact vertex and face values,
zero outside the box, and closed-form termination indices on rays whose lattice,
interval lengths and optical depths are exact in float32.
"""
import math

import numpy as np
import pytest

from paper_2210_04847_gb300 import synth

EPS = 1e-4
THR_O = -math.log(EPS)  # 9.2103...


def _u64(x, box, G):
    x = np.asarray(x, np.float64)
    lo, hi = np.asarray(box[:3], np.float64), np.asarray(box[3:], np.float64)
    return (x - lo) * (np.asarray(G, np.float64) - 1.0) / (hi - lo)


def _multilinear(u):
    i, j, k = u[..., 0], u[..., 1], u[..., 2]
    return 1.0 + 2.0 * i + 0.5 * j - 0.25 * k + 0.75 * i * j - 0.3 * j * k + 0.2 * i * k + 0.1 * i * j * k + 3.0


def test_field_vertices_exact(orc):
    G = (4, 5, 3)
    box = [0.0, 0.0, 0.0, 3.0, 4.0, 2.0]  # one unit per vertex step: u = x exactly
    rng = np.random.default_rng(0)
    g = rng.integers(0, 100, size=G).astype(np.float32)
    pts = np.array([[i, j, k] for i in range(G[0]) for j in range(G[1]) for k in range(G[2])], np.float32)
    got = orc.field_query(g, box, pts)
    want = g.reshape(-1)
    assert np.array_equal(got, want)


@pytest.mark.parametrize("G", [(2, 2, 2), (5, 7, 3), (9, 4, 6)])
def test_field_multilinear_reproduced(orc, G):
    box = [-1.5, 0.25, -3.0, 2.0, 1.75, 5.0]
    idx = np.stack(np.meshgrid(*[np.arange(n) for n in G], indexing="ij"), axis=-1).astype(np.float64)
    g = _multilinear(idx).astype(np.float32)
    rng = np.random.default_rng(1)
    lo, hi = np.array(box[:3]), np.array(box[3:])
    x = (lo + (hi - lo) * rng.random((4000, 3))).astype(np.float32)
    got = orc.field_query(g, box, x).astype(np.float64)
    want = _multilinear(_u64(x, box, G))
    assert np.max(np.abs(got - want)) <= 2e-5 * np.max(np.abs(want))


def test_field_random_values_vs_eight_corner_weights(orc):
    G = (6, 5, 7)
    box = [-1.0, -2.0, 0.5, 1.0, 3.0, 2.5]
    rng = np.random.default_rng(2)
    g = rng.random(G).astype(np.float32) * 50.0
    lo, hi = np.array(box[:3]), np.array(box[3:])
    x = (lo + (hi - lo) * rng.random((3000, 3))).astype(np.float32)
    got = orc.field_query(g, box, x).astype(np.float64)
    u = _u64(x, box, G)
    i = np.minimum(np.floor(u).astype(int), np.array(G) - 2)
    f = u - i
    want = np.zeros(len(x))
    for dx in (0, 1):
        for dy in (0, 1):
            for dz in (0, 1):
                w = (f[:, 0] if dx else 1 - f[:, 0]) * (f[:, 1] if dy else 1 - f[:, 1]) * (f[:, 2] if dz else 1 - f[:, 2])
                want += w * g[i[:, 0] + dx, i[:, 1] + dy, i[:, 2] + dz]
    assert np.max(np.abs(got - want)) <= 2e-5 * 50.0


def test_field_faces_and_outside(orc):
    G = (3, 3, 3)
    box = [0.0, 0.0, 0.0, 2.0, 2.0, 2.0]
    idx = np.stack(np.meshgrid(*[np.arange(n) for n in G], indexing="ij"), axis=-1).astype(np.float64)
    g = _multilinear(idx).astype(np.float32)
    faces = np.array([[2.0, 0.5, 0.5], [0.5, 2.0, 0.5], [0.5, 0.5, 2.0], [0.0, 1.5, 1.5], [2.0, 2.0, 2.0]],
                     np.float32)
    got = orc.field_query(g, box, faces)
    assert np.all(got > 0)
    assert np.allclose(got, _multilinear(faces.astype(np.float64)), rtol=1e-6)
    off = np.float32(1e-3)
    out = np.array([[2.0 + off, 1, 1], [1, 2.0 + off, 1], [1, 1, 2.0 + off], [-off, 1, 1], [1, -off, 1],
                    [1, 1, -off], [np.nan, 1, 1]], np.float32)
    assert np.array_equal(orc.field_query(g, box, out), np.zeros(len(out), np.float32))


# ---------------------------------------------------------------------------
# fused march + prune
# ---------------------------------------------------------------------------

AABB = [-1.0, -1.0, -1.0, 1.0, 1.0, 1.0]
DT = 1.0 / 64.0  # t_k = 1 + k/64 and every interval length are exact in float32


def _x_ray():
    # enters the box at x = -1 (t = 1) along +x; every lattice point and midpoint is exact
    return np.array([[-2.0, 0.1, -0.2]], np.float32), np.array([[1.0, 0.0, 0.0]], np.float32)


def _const_field(v, G=(3, 3, 3)):
    return np.full(G, v, np.float32)


def test_fused_constant_density_terminates_at_closed_form(orc):
    o, d = _x_ray()
    bits = synth.pack_bits(np.ones(8 ** 3, bool))
    # tau = 40/64 = 0.625 exactly; O_i = 0.625 i <= -ln 1e-4 = 9.2103 for i <= 14
    p, sg = orc.march_fused(o, d, bits, (8, 8, 8), AABB, _const_field(40.0), AABB, EPS, 0.0, 0.0, 10.0, DT, DT,
                            0.0, 1024)
    k = int(math.floor(THR_O / 0.625)) + 1
    assert k == 15
    assert p.packed_info.tolist() == [[0, k]]
    assert p.t_starts.tolist() == [1.0 + i * DT for i in range(k)]
    assert p.t_ends.tolist() == [1.0 + (i + 1) * DT for i in range(k)]
    assert np.all(sg == 40.0)


def test_fused_no_thresholds_keeps_every_marched_sample(orc):
    rng = np.random.default_rng(3)
    o = rng.uniform(-3, 3, (64, 3)).astype(np.float32)
    d = rng.uniform(-0.8, 0.8, (64, 3)) - o  # aimed into the box
    d = (d / np.linalg.norm(d, axis=1, keepdims=True)).astype(np.float32)
    occ = rng.random(8 ** 3) < 0.4
    bits = synth.pack_bits(occ)
    field = (rng.random((5, 4, 6)) * 20).astype(np.float32)
    fbox = [-0.8, -1.2, -1.0, 1.1, 0.9, 1.3]
    m = orc.march(o, d, bits, (8, 8, 8), AABB, 0.0, 10.0, 0.02, 0.02, 0.0, 512)
    p, sg = orc.march_fused(o, d, bits, (8, 8, 8), AABB, field, fbox, 0.0, 0.0, 0.0, 10.0, 0.02, 0.02, 0.0, 512)
    assert np.array_equal(p.packed_info, m.packed_info)
    assert np.array_equal(p.t_starts, m.t_starts) and np.array_equal(p.t_ends, m.t_ends)
    assert np.array_equal(p.ray_indices, m.ray_indices)
    mid = ((m.t_starts + m.t_ends) * np.float32(0.5)).astype(np.float32)
    x = (o[m.ray_indices] + d[m.ray_indices] * mid[:, None]).astype(np.float32)
    assert np.array_equal(sg, orc.field_query(field, fbox, x))
    assert m.n_samples > 500


def test_fused_transparent_field_keeps_nothing(orc):
    o, d = _x_ray()
    bits = synth.pack_bits(np.ones(8 ** 3, bool))
    # tau = 0.5/64 < -ln(1 - 0.01): every sample is below the opacity threshold
    p, sg = orc.march_fused(o, d, bits, (8, 8, 8), AABB, _const_field(0.5), AABB, EPS, 1e-2, 0.0, 10.0, DT, DT,
                            0.0, 1024)
    assert p.packed_info.tolist() == [[0, 0]] and p.n_samples == 0 and sg.size == 0


def test_fused_optical_depth_counts_emitted_samples_only(orc):
    o, d = _x_ray()
    occ = np.zeros((8, 8, 8), bool)
    occ[0::2] = True  # cells with even x index; each holds 16 lattice intervals along the ray
    bits = synth.pack_bits(occ.reshape(-1))
    # tau = 10/64 = 0.15625; O after i emitted samples = 0.15625 i <= 9.2103 for i <= 58
    p, _ = orc.march_fused(o, d, bits, (8, 8, 8), AABB, _const_field(10.0), AABB, EPS, 0.0, 0.0, 10.0, DT, DT,
                           0.0, 1024)
    k = int(math.floor(THR_O / 0.15625)) + 1
    assert k == 59
    lattice = [c * 32 + j for c in range(4) for j in range(16)][:k]  # emitted lattice indices, in order
    assert p.packed_info.tolist() == [[0, k]]
    assert p.t_starts.tolist() == [1.0 + i * DT for i in lattice]


def test_fused_linear_density_midpoints_and_opacity_threshold(orc):
    o, d = _x_ray()
    bits = synth.pack_bits(np.ones(8 ** 3, bool))
    G = (17, 2, 2)
    # sigma = 8 (x + 1): linear in x, so the trilinear field is exact at every point
    xs = np.linspace(-1.0, 1.0, G[0])
    field = np.broadcast_to((8.0 * (xs + 1.0))[:, None, None], G).astype(np.float32).copy()
    thre = 0.05
    p, sg = orc.march_fused(o, d, bits, (8, 8, 8), AABB, field, AABB, EPS, thre, 0.0, 10.0, DT, DT, 0.0, 1024)
    # closed form in float64: interval k = [1 + k/64, 1 + (k+1)/64], midpoint x = -1 + (k + 0.5)/64
    thr_tau = -math.log1p(-thre)
    O, kept = 0.0, []
    for k in range(128):
        s = 8.0 * ((k + 0.5) / 64.0)
        tau = s * DT
        if O <= THR_O and tau >= thr_tau:
            kept.append((k, s))
        O += tau
    assert kept[0][0] > 0  # the first samples fall below the opacity threshold
    assert p.packed_info.tolist() == [[0, len(kept)]]
    assert p.t_starts.tolist() == [1.0 + k * DT for k, _ in kept]
    assert np.allclose(sg, [s for _, s in kept], rtol=1e-6, atol=0)

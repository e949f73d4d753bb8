"""Marching against the oracle, bit-exact, point by point, with the coarse pass and
with the box walk, on
inputs aimed at the float32 cell decisions: midpoints exactly on cell faces, directions with tiny or zero
components, directions far from unit length, origins far from the grid (large
rounding), cascades with uniform steps, cells smaller than one step, a negative
near plane, cone steps over a cascade, and whole full-size batches (every
sample of every ray).
"""
import functools

import numpy as np
import pytest

from paper_2210_04847_gb300 import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2210_04847_gb300 import _lib  # noqa: E402
from gpu_util import assert_march_equal, gpu_march, oracle_march  # noqa: E402


@pytest.fixture(autouse=True, params=[0, 1, 2, 3], ids=["pointwise", "coarse", "box", "box_tile"])
def coarse(request):
    """Every case point by point, with the coarse pass (chunks inside one cell
    filled from a single occupancy test), and with the grid's summed-area table
    (one-level grids take the box walk: chunks whose box of cells is all occupied
    or all empty filled from one box count), ray by ray and over a whole tile."""
    import gpu_util

    old = _lib.tune_get("march_coarse"), _lib.tune_get("march_box_tile")
    _lib.tune_set("march_coarse", 1 if request.param == 1 else 0)
    _lib.tune_set("march_box_tile", 1 if request.param == 3 else 0)
    gpu_util.USE_SAT = request.param >= 2
    yield request.param
    gpu_util.USE_SAT = False
    _lib.tune_set("march_coarse", old[0])
    _lib.tune_set("march_box_tile", old[1])

def _workload(o, d, occ, res, aabb, n_levels=1, near=0.0, far=1e10, dt_min=0.05, dt_max=0.05, cone=0.0,
              max_steps=1024):
    return synth.Workload("traverse-case", np.ascontiguousarray(o, np.float32), np.ascontiguousarray(d, np.float32),
                          synth.pack_bits(occ), res, n_levels, 1, aabb, near, far, dt_min, dt_max, cone, max_steps,
                          0.0, 0.0)


def _random_rays(seed, n, spread=3.0, box=1.2):
    o = synth.random_unit_vectors(seed, 2, n) * spread
    tgt = synth.rand_uniform(seed, 3, 3 * n, -box, box).reshape(n, 3)
    d = tgt - o
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    return o, d


def test_midpoints_on_cell_boundaries(orc):
    """Box [-1, 1]^3 of 8^3 cells (0.25 each), dt = 1/16 and a near plane that puts
    every fourth midpoint exactly on a cell face, along each axis and diagonals."""
    res = (8, 8, 8)
    occ = synth.rand_uniform(11, 1, 512) < 0.5
    dirs = np.array([[1, 0, 0], [0, 1, 0], [0, 0, 1], [-1, 0, 0], [0, -1, 0], [0, 0, -1], [1, 1, 0], [1, -1, 1],
                     [-1, 1, 1], [1, 1, 1]], np.float64)
    dirs /= np.abs(dirs).max(axis=1, keepdims=True)  # components 0 and +-1: exact steps
    o = -2.0 * dirs + np.array([0.125, -0.375, 0.25]) * (dirs == 0)
    w = _workload(o, dirs, occ, res, (-1, -1, -1, 1, 1, 1), near=1.0 + 1.0 / 32, dt_min=1.0 / 16, dt_max=1.0 / 16)
    g = gpu_march(w)
    assert g[4] > 0
    assert_march_equal(g, oracle_march(orc, w))


@pytest.mark.parametrize("seed", range(3))
def test_near_axis_parallel_and_scaled_directions(orc, seed):
    """Direction components of 1e-7, 1e-20, 1e-38 and -0; directions scaled by 1e-3 and 1e3."""
    n = 600
    o, d = _random_rays(seed, n)
    small = np.array([1e-7, 1e-20, 1e-38, -0.0, 3e-5])
    for i in range(200):
        d[i, i % 3] = small[i % len(small)]
    d[200:400] *= np.where(np.arange(200) % 2 == 0, 1e-3, 1e3)[:, None]
    res = [(16, 16, 16), (5, 9, 7), (32, 8, 3)][seed]
    occ = synth.rand_uniform(seed, 5, int(np.prod(res))) < 0.45
    w = _workload(o, d, occ, res, (-1.0, -0.8, -1.1, 0.9, 1.2, 1.0), dt_min=0.011, dt_max=0.011)
    assert_march_equal(gpu_march(w), oracle_march(orc, w))


def test_far_origins(orc):
    """Origins 1e4 away: large rounding bounds, so many undecided points go to the exact test."""
    n = 400
    o, d = _random_rays(3, n, spread=1.0e4, box=0.9)
    occ = synth.rand_uniform(3, 5, 64 ** 3) < 0.3
    w = _workload(o, d, occ, (64, 64, 64), (-1, -1, -1, 1, 1, 1), dt_min=0.004, dt_max=0.004)
    g = gpu_march(w)
    assert g[4] > 0
    assert_march_equal(g, oracle_march(orc, w))


@pytest.mark.parametrize("n_levels", [2, 3])
def test_uniform_steps_cascade(orc, n_levels):
    """Cascades marched with uniform steps: rays enter and leave finer boxes."""
    res = (16, 16, 16)
    n = 800
    o, d = _random_rays(4 + n_levels, n, spread=6.0, box=2.5)
    o[:100] = synth.rand_uniform(9, 1, 300, -0.9, 0.9).reshape(100, 3)  # inside the finest box
    occ = synth.rand_uniform(n_levels, 5, n_levels * 16 ** 3) < 0.4
    w = _workload(o, d, occ, res, (-1, -1, -1, 1, 1, 1), n_levels=n_levels, dt_min=0.02, dt_max=0.02,
                  max_steps=2048)
    g = gpu_march(w)
    assert g[4] > 0
    assert_march_equal(g, oracle_march(orc, w))


def test_cells_smaller_than_a_step(orc):
    """256^3 cells of 1/128 with dt = 0.03: each step crosses several cells."""
    n = 500
    o, d = _random_rays(12, n)
    occ = synth.rand_uniform(12, 5, 256 ** 3) < 0.05
    w = _workload(o, d, occ, (256, 256, 256), (-1, -1, -1, 1, 1, 1), dt_min=0.03, dt_max=0.03)
    assert_march_equal(gpu_march(w), oracle_march(orc, w))


def test_negative_near_plane_inside_origins(orc):
    n = 500
    o = synth.rand_uniform(13, 1, 3 * n, -0.95, 0.95).reshape(n, 3)
    d = synth.random_unit_vectors(13, 2, n)
    occ = synth.rand_uniform(13, 5, 24 ** 3) < 0.5
    w = _workload(o, d, occ, (24, 24, 24), (-1, -1, -1, 1, 1, 1), near=-0.5, far=1.7, dt_min=0.007, dt_max=0.007)
    assert_march_equal(gpu_march(w), oracle_march(orc, w))


def test_cone_cascade_mixed_starts(orc):
    """Cone steps over a 3-level cascade; rays starting inside (the shared lattice)
    and outside the outermost box (their own recurrence)."""
    n = 900
    o, d = _random_rays(14, n, spread=9.0, box=3.0)
    o[:450] = synth.rand_uniform(14, 7, 1350, -0.9, 0.9).reshape(450, 3)
    occ = synth.rand_uniform(14, 5, 3 * 32 ** 3) < 0.35
    w = _workload(o, d, occ, (32, 32, 32), (-1, -1, -1, 1, 1, 1), n_levels=3, near=0.01, far=100.0, dt_min=1e-3,
                  dt_max=0.2, cone=1.0 / 128, max_steps=4096)
    g = gpu_march(w)
    assert g[4] > 0
    assert_march_equal(g, oracle_march(orc, w))


@pytest.mark.parametrize("max_steps", [8192, 8193])
def test_cone_lattice_at_the_shared_memory_limit(orc, max_steps):
    """Each block keeps the shared cone lattice t_0 .. t_max_steps in shared memory
    up to 8193 entries and reads it from the workspace above that. Both sides of
    the limit (in every walk mode of the module's fixture, the box walk over levels
    included), with rays inside the box that march to the last entries, are
    bit-exact."""
    n = 600
    o, d = _random_rays(16, n, spread=9.0, box=3.0)
    o[:300] = synth.rand_uniform(16, 7, 900, -0.9, 0.9).reshape(300, 3)
    occ = synth.rand_uniform(16, 5, 3 * 32 ** 3) < 0.9
    w = _workload(o, d, occ, (32, 32, 32), (-1, -1, -1, 1, 1, 1), n_levels=3, near=0.0, far=100.0, dt_min=1e-4,
                  dt_max=0.2, cone=1.0 / 4096, max_steps=max_steps)
    g = gpu_march(w)
    ora = oracle_march(orc, w)
    # rays from inside the box take the shared lattice up to its last entry
    assert int(np.max(ora.packed_info[:300, 1])) == max_steps
    assert_march_equal(g, ora)


def test_cone_equal_step_bounds(orc):
    """dt_min == dt_max: the cone lattice degenerates to uniform steps."""
    n = 400
    o, d = _random_rays(15, n)
    o[:100] = synth.rand_uniform(15, 7, 300, -0.9, 0.9).reshape(100, 3)
    occ = synth.rand_uniform(15, 5, 32 ** 3) < 0.4
    w = _workload(o, d, occ, (32, 32, 32), (-1, -1, -1, 1, 1, 1), near=0.2, dt_min=0.01, dt_max=0.01, cone=0.01)
    assert_march_equal(gpu_march(w), oracle_march(orc, w))


@pytest.mark.parametrize("cone", [False, True])
def test_contracted_space_random_rays(orc, cone):
    """Unbounded scenes (Sec. 2.1 "Scene Contraction"): rays from inside and outside
    the box, marched over [near, far] with no clip, looked up in contracted space."""
    n = 700
    o, d = _random_rays(16, n, spread=3.0, box=1.5)
    o[:300] = synth.rand_uniform(16, 7, 900, -0.8, 0.8).reshape(300, 3)
    res = (32, 32, 32)
    occ = synth.rand_uniform(16, 5, 2 * 32 ** 3) < 0.4
    slot = (synth.rand_uniform(16, 8, n) < 0.5).astype(np.int32)
    if cone:
        w = _workload(o, d, occ, res, (-1, -1, -1, 1, 1, 1), near=0.05, far=200.0, dt_min=1e-3, dt_max=1.0,
                      cone=1.0 / 128, max_steps=4096)
    else:
        w = _workload(o, d, occ, res, (-1, -1, -1, 1, 1, 1), near=0.0, far=6.0, dt_min=0.004, dt_max=0.004,
                      max_steps=2048)
    w.n_slots, w.ray_slot, w.contraction = 2, slot, 1
    g = gpu_march(w)
    assert g[4] > 0
    assert_march_equal(g, oracle_march(orc, w))


def test_contracted_axis_case(orc):
    """The oracle's analytic pin, on the GPU: only cell (14, 8, 8) of 16^3 is occupied,
    the ray runs along +x from the centre with dt = 1/64: samples k = 128..255."""
    occ = np.zeros((16, 16, 16), bool)
    occ[14, 8, 8] = True
    w = _workload(np.zeros((1, 3)), np.array([[1.0, 0.0, 0.0]]), occ.reshape(-1), (16, 16, 16),
                  (-1, -1, -1, 1, 1, 1), near=0.0, far=100.0, dt_min=1.0 / 64, dt_max=1.0 / 64, max_steps=8192)
    w.contraction = 1
    g = gpu_march(w)
    assert g[4] == 128
    assert_march_equal(g, oracle_march(orc, w))


def test_contracted_unbounded_scene(orc):
    """The unbounded scene with a 128^3 contracted grid instead of the cascade (2^12 rays)."""
    w = synth.contracted_config(0, n_rays=1 << 12, device="cuda")
    g = gpu_march(w, capacity=12_000_000)
    assert g[4] > 0
    assert_march_equal(g, oracle_march(orc, w))


@pytest.mark.parametrize("max_steps", [1024, 32, 33])
@pytest.mark.parametrize("far_plane", [1e10, 1.5])
def test_lattice_lengths_around_chunk_boundaries(orc, far_plane, max_steps):
    """One level, uniform steps, rays along the axes from inside the box [-1, 1]^3
    whose lattices hold 0-129 points (around multiples of 32). Each ray ends at the box
    face, the far plane or max_steps, either halfway through a step or exactly on a
    lattice point (t_k < far is strict). So the chunk after a ray's last one lies
    outside the grid, inside it, or past max_steps. The exit distances are multiples
    of 1/128 and dt = 1/64, so every t and the clip are exact in float32."""
    dt = 1.0 / 64
    res = (16, 16, 16)
    occ = np.ones(16 ** 3, bool)
    occ[::3] = False
    n_pts = [0, 1, 2, 31, 32, 33, 63, 64, 65, 95, 96, 97, 127, 128]
    o, d = [], []
    for axis in range(3):
        for sign in (1.0, -1.0):
            for n in n_pts:
                for frac in (0.5, 0.0):
                    exit_dist = (n + frac) * dt
                    if exit_dist > 2.0:
                        continue
                    p = np.array([0.1, -0.3, 0.45])
                    p[axis] = sign * (1.0 - exit_dist)
                    v = np.zeros(3)
                    v[axis] = sign
                    o.append(p)
                    d.append(v)
    w = _workload(np.array(o), np.array(d), occ, res, (-1, -1, -1, 1, 1, 1), far=far_plane, dt_min=dt, dt_max=dt,
                  max_steps=max_steps)
    g = gpu_march(w)
    assert g[4] > 0
    assert_march_equal(g, oracle_march(orc, w))


@functools.lru_cache(maxsize=1)
def _whole_batch(name):
    import oracle

    oracle.build()
    if name == "bounded":
        w = synth.bounded_config(0, n_rays=1 << 18, device="cuda")
    else:
        w = synth.unbounded_config(0, n_rays=1 << 16, device="cuda")
    return w, oracle_march(oracle, w)


def test_fullsize_bounded_whole_batch():
    """The benchmark's bounded batch, 2^18 rays of 100 800x800 cameras on the 128^3
    grid: every sample of every ray bit-identical to the oracle."""
    w, ora = _whole_batch("bounded")
    g = gpu_march(w, capacity=180_000_000)
    assert g[4] > 100_000_000
    assert_march_equal(g, ora)


def test_unbounded_whole_batch():
    """2^16 rays of the unbounded scene (4-level cascade, cone steps to t = 1000)."""
    w, ora = _whole_batch("unbounded")
    g = gpu_march(w, capacity=80_000_000)
    assert g[4] > 0
    assert_march_equal(g, ora)

"""Seeded random configurations against the oracle, through the C ABI: grids of
any shape (non-cubic, 1-5 levels, contracted), uniform or cone steps, odd step
counts, random near/far planes, rays from inside and outside the box, axis-
aligned and random directions, every march tile shape. Marching is bit-exact;
the fused inference path is bit-exact except near-threshold flips.
"""
import numpy as np
import pytest

from paper_2210_04847_gb300 import _lib, synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no CUDA device", allow_module_level=True)

from gpu_util import assert_march_equal, gpu_march, oracle_march  # noqa: E402
from test_gpu_fused import assert_fused_matches, gpu_fused, oracle_reference  # noqa: E402


def _config(seed):
    rng = np.random.default_rng(1000 + seed)
    contraction = int(rng.random() < 0.2)
    n_levels = 1 if contraction else int(rng.integers(1, 6))
    res = tuple(int(v) for v in rng.integers(1, 41, size=3))
    lo = rng.uniform(-2.0, 0.0, size=3)
    hi = lo + rng.uniform(0.5, 3.0, size=3)
    aabb = tuple(float(v) for v in np.concatenate([lo, hi]).astype(np.float32))
    n_cells = int(np.prod(res)) * n_levels
    occ = rng.random(n_cells) < rng.uniform(0.05, 0.95)
    n = 300
    ext = 2.0 ** (n_levels - 1) + 1.5
    c = (lo + hi) / 2
    o = c + rng.uniform(-ext, ext, size=(n, 3)) * (hi - lo) / 2
    tgt = c + rng.uniform(-1, 1, size=(n, 3)) * (hi - lo) / 2
    d = tgt - o
    d[::7] = rng.choice([-1.0, 1.0], size=(len(d[::7]), 1)) * np.eye(3)[rng.integers(0, 3, size=len(d[::7]))]
    d /= np.linalg.norm(d, axis=1, keepdims=True) / rng.uniform(0.5, 2.0, size=(n, 1))  # not unit length
    cone = float(rng.choice([0.0, 1.0 / 256, 1.0 / 64]))
    dt = float(np.float32(rng.uniform(0.005, 0.08)))
    max_steps = int(rng.choice([1, 31, 32, 33, 257, 1000, 3000]))
    near = float(np.float32(rng.choice([0.0, 0.01, -0.5])))
    far = float(np.float32(rng.choice([1e10, 3.0, 8.0])))
    w = synth.Workload("fuzz-%d" % seed, o.astype(np.float32), d.astype(np.float32), synth.pack_bits(occ), res,
                       n_levels, 1, aabb, near, far, dt, dt * 8 if cone else dt, cone, max_steps, 1e-3, 1e-2,
                       contraction=contraction)
    return w, rng


@pytest.mark.parametrize("seed", range(16))
def test_fuzz_march_bitexact(orc, seed):
    """Each configuration without and with the grid's summed-area table (the box
    walk for one level and for cascades of up to four levels), ray by ray and over
    each tile's chunks at once."""
    import gpu_util

    w, rng = _config(seed)
    old = _lib.tune_get("march_tile_rays"), _lib.tune_get("march_box_tile")
    try:
        _lib.tune_set("march_tile_rays", int(rng.choice([1, 2, 4, 8, 16, 32])))
        ref = oracle_march(orc, w)
        assert_march_equal(gpu_march(w), ref)
        gpu_util.USE_SAT = True
        for box_tile in (0, 1):
            _lib.tune_set("march_box_tile", box_tile)
            assert_march_equal(gpu_march(w), ref)
    finally:
        gpu_util.USE_SAT = False
        _lib.tune_set("march_tile_rays", old[0])
        _lib.tune_set("march_box_tile", old[1])


@pytest.mark.parametrize("seed", range(8))
def test_fuzz_fused_parity(orc, seed):
    w, rng = _config(seed)
    G = tuple(int(v) for v in rng.integers(2, 12, size=3))
    w.field = (rng.random(G) * rng.uniform(1, 200)).astype(np.float32)
    lo, hi = np.array(w.aabb[:3]), np.array(w.aabb[3:])
    w.field_box = tuple(float(v) for v in np.concatenate([lo - 0.1, hi + 0.1]).astype(np.float32))
    m, sig, od, p, p_sig = oracle_reference(orc, w)
    g = gpu_fused(w)
    assert_fused_matches(g, m, sig, od, p, p_sig, w.early_stop_eps)

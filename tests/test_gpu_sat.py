"""The grid's summed-area table and the box walk that uses it.

nacc_build_grid_sat against the table's definition (oracle.grid_sat: numpy
cumulative sums, modulo 2^16) on several grid shapes (shared-memory and
global-memory build passes), and marching with the table
bit-exact against the oracle where the box test cannot decide (boxes of 2^16
cells or more), on batches of scenes with and without tables, and through the
paper-shaped API. The whole-batch and edge-case parity tests of marching also run
with the table (tests/test_gpu_march.py, tests/test_gpu_march_edges.py)."""
import numpy as np
import pytest

from paper_2210_04847_gb300 import _lib, synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no CUDA device", allow_module_level=True)

from gpu_util import assert_march_equal, dev, gpu_march, oracle_march  # noqa: E402


@pytest.mark.parametrize("res,n_levels,n_slots,p", [((128, 128, 128), 1, 1, 0.78), ((33, 47, 29), 2, 3, 0.5),
                                                     ((1, 5, 70), 1, 2, 0.9), ((64, 64, 64), 1, 1, 1.0),
                                                     ((7, 1, 1), 1, 1, 0.5), ((3, 300, 300), 1, 1, 0.95),
                                                     ((300, 3, 200), 1, 1, 0.7), ((64, 64, 64), 1, 5, 0.8),
                                                     ((31, 17, 45), 2, 2, 0.6)])
def test_sat_matches_definition(orc, res, n_levels, n_slots, p):
    n = res[0] * res[1] * res[2] * n_levels * n_slots
    occ = synth.rand_uniform(n_slots, 40 + n_levels, n) < p
    bits = synth.pack_bits(occ)
    grid = _lib.make_grid(dev(bits), res, (-1, -1, -1, 1, 1, 1), n_levels, n_slots)
    sat = _lib.build_grid_sat(grid)
    torch.cuda.synchronize()
    ref = orc.grid_sat(bits, res, n_levels * n_slots)
    got = sat.cpu().numpy().view(np.uint16)
    assert np.array_equal(got[: ref.size], ref)  # totals of the larger grids wrap modulo 2^16
    # the brick summary from the first 16-byte boundary after the table
    off = (ref.size + 7) // 8 * 8
    summ = orc.grid_brick_summary(bits, res, n_levels * n_slots)
    assert got.size == off + summ.size
    assert np.array_equal(got[off:], summ)


def test_box_walk_boxes_too_large_for_the_table(orc):
    """Steps of many cells: a chunk's box holds 2^16 cells or more, so the walk tests
    those chunks point by point."""
    res = (256, 256, 256)
    occ = synth.rand_uniform(9, 1, 256 ** 3) < 0.97
    o = synth.random_unit_vectors(9, 2, 600) * 3.0
    tgt = synth.rand_uniform(9, 3, 1800, -0.8, 0.8).reshape(600, 3)
    d = tgt - o
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    w = synth.Workload("big-steps", o.astype(np.float32), d.astype(np.float32), synth.pack_bits(occ), res, 1, 1,
                       (-1, -1, -1, 1, 1, 1), 0.0, 1e10, 0.2, 0.2, 0.0, 1024, 0.0, 0.0)
    import gpu_util

    gpu_util.USE_SAT = True
    try:
        g = gpu_march(w)
    finally:
        gpu_util.USE_SAT = False
    assert g[4] > 0
    assert_march_equal(g, oracle_march(orc, w))


def test_batched_scenes_with_and_without_tables(orc):
    """nacc_march_rays_batched where some one-level scenes carry tables and some do not."""
    from test_gpu_march_batched import _run, _scene

    scenes = [_scene(1, (64, 64, 64), (-1.5, -1.5, -1.5, 1.5, 1.5, 1.5), 1, 700),
              _scene(2, (96, 80, 128), (-2.0, -1.0, -1.5, 2.0, 1.0, 1.5), 1, 900),
              _scene(4, (33, 47, 29), (-0.5, -3.0, 2.0, 0.5, -1.0, 2.5), 1, 400)]
    for k in (0, 2):
        s = scenes[k]
        g = _lib.make_grid(dev(s["bits"]), s["res"], s["aabb"])
        s["sat"] = _lib.build_grid_sat(g)
    _run(orc, scenes, 0.0, 1e10, 0.0051, 0.0051, 0.0, 1024)
    _run(orc, scenes, 0.01, 20.0, 2e-3, 0.05, 1.0 / 64.0, 2048)

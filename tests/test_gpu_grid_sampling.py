"""Device sampling of the grid update's inputs (random cells and a point in
each) against the host generator: the same counter-based SplitMix64 streams
and the same float32 point arithmetic, implemented separately on each side,
give bit-identical cells and points."""
import numpy as np
import pytest

from paper_2210_04847_gb300 import _lib, api, synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no CUDA device", allow_module_level=True)


def _host(seed, step, n, aabb, res, n_levels, n_slots, contraction=0):
    cells, jit = synth.grid_update_samples(seed, step, n, res, n_levels, n_slots)
    xyz = synth.cell_positions(cells, jit, aabb, res, n_levels, contraction=contraction)
    assert xyz.dtype == np.float32
    return cells, xyz


def _same_points(a, b):
    """Bit-identical float32 points; NaN (unreachable contracted cells) compared as a mask."""
    na, nb = np.isnan(a), np.isnan(b)
    return np.array_equal(na, nb) and np.array_equal(a[~na].view(np.uint32), b[~nb].view(np.uint32))


@pytest.mark.parametrize("res,n_levels,n_slots,aabb", [
    ((128, 128, 128), 1, 1, (-1.5, -1.5, -1.5, 1.5, 1.5, 1.5)),
    ((128, 128, 128), 4, 1, (-125.0, -125.0, -125.0, 125.0, 125.0, 125.0)),
    ((64, 32, 16), 2, 3, (-1.0, -0.5, 0.25, 2.0, 1.5, 0.75)),
    ((1, 1, 1), 1, 1, (0.0, 0.0, 0.0, 1.0, 1.0, 1.0)),
])
def test_device_sampling_matches_host_generator(res, n_levels, n_slots, aabb):
    g = api.OccupancyGrid(aabb, res, n_levels, n_slots)
    for seed, step, n in ((0, 0, 1 << 16), (7, 3, 1000), (123456789, 41, 77)):
        cells, xyz = g.sample_cells(n, seed, step)
        hc, hx = _host(seed, step, n, aabb, res, n_levels, n_slots)
        assert np.array_equal(cells.cpu().numpy(), hc)
        assert np.array_equal(xyz.cpu().numpy().view(np.uint32), hx.view(np.uint32))


def test_contracted_grid_sampling_matches_host_generator():
    """Cells and points of a contracted grid: drawn in [-2, 2]^3, mapped back to the world."""
    aabb = (-125.0, -125.0, -125.0, 125.0, 125.0, 125.0)
    g = api.OccupancyGrid(aabb, (64, 64, 64), 1, 2, contraction=1)
    cells, xyz = g.sample_cells(1 << 16, 3, 1)
    hc, hx = _host(3, 1, 1 << 16, aabb, (64, 64, 64), 1, 2, contraction=1)
    assert np.array_equal(cells.cpu().numpy(), hc)
    assert _same_points(xyz.cpu().numpy(), hx)
    assert 0.4 < np.isnan(hx[:, 0]).mean() < 0.6  # the corners outside the radius-2 ball


def test_fullsize_sampling_and_update_in_cells():
    """2^21 samples of the bounded grid: every point lies in its cell."""
    aabb = (-1.5, -1.5, -1.5, 1.5, 1.5, 1.5)
    g = api.OccupancyGrid(aabb, 128)
    cells, xyz = g.sample_cells(1 << 21, 0, 5)
    c = cells.long()
    idx = torch.stack([c // (128 * 128), (c // 128) % 128, c % 128], 1).double()
    u = (xyz.double() + 1.5) / 3.0 * 128
    assert bool(torch.all((u >= idx - 1e-4) & (u <= idx + 1 + 1e-4)))
    hc, hx = _host(0, 5, 1 << 21, aabb, (128, 128, 128), 1, 1)
    assert np.array_equal(cells.cpu().numpy(), hc)
    assert np.array_equal(xyz.cpu().numpy().view(np.uint32), hx.view(np.uint32))


def test_zero_samples_and_bad_grid():
    g = api.OccupancyGrid((0, 0, 0, 1, 1, 1), 8)
    c = torch.empty(0, dtype=torch.int32, device="cuda")
    x = torch.empty((0, 3), dtype=torch.float32, device="cuda")
    _lib.sample_grid_cells(0, 0, 0, g.struct(), c, x)
    bad = _lib.make_grid(g.bits, (8, 8, 8), (1, 0, 0, 0, 1, 1))
    with pytest.raises(_lib.NaccError):
        _lib.sample_grid_cells(0, 0, 4, bad, torch.empty(4, dtype=torch.int32, device="cuda"),
                               torch.empty((4, 3), dtype=torch.float32, device="cuda"))

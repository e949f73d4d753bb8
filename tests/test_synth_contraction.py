"""The host generators of contracted space (the expected values of the device
sampler and of the contracted occupancy grid) against the contraction's definition
(Mip-NeRF 360 Eq. 10: x if |x| <= 1, else (2 - 1/|x|) x/|x|), in float64."""
import numpy as np

from paper_2210_04847_gb300 import synth


def contract64(x):
    x = np.asarray(x, np.float64)
    n = np.linalg.norm(x, axis=-1, keepdims=True)
    with np.errstate(divide="ignore", invalid="ignore"):
        return np.where(n <= 1.0, x, (2.0 - 1.0 / n) * x / n)


def test_uncontract_inverts_the_contraction():
    rng = np.random.default_rng(3)
    x = rng.normal(size=(5000, 3)) * np.exp(rng.uniform(-3, 7, size=(5000, 1)))
    xc = contract64(x)
    assert np.all(np.linalg.norm(xc, axis=1) < 2.0)
    back = synth.uncontract(xc)
    assert np.allclose(back, x, rtol=1e-8, atol=1e-12)


def test_contracted_cell_points_lie_in_their_cells():
    """A point drawn in contracted cell (i, j, k) of a res^3 grid over [-2, 2]^3,
    mapped to the world and contracted again, lands in that cell; cells wholly
    beyond radius 2 give NaN points."""
    res = (16, 16, 16)
    aabb = (-3.0, -1.0, 0.0, 5.0, 7.0, 8.0)  # centre (1, 3, 4), half-size 4
    n = 20000
    rng = np.random.default_rng(4)
    cells = rng.integers(0, 16 ** 3, size=n).astype(np.int32)
    jit = rng.uniform(0.05, 0.95, size=(n, 3)).astype(np.float32)
    p = synth.cell_positions(cells, jit, aabb, res, contraction=1).astype(np.float64)
    idx = np.stack([cells // 256, (cells // 16) % 16, cells % 16], axis=1)
    lo_c = -2.0 + idx * 0.25
    centre = lo_c + jit.astype(np.float64) * 0.25  # the contracted point drawn
    reach = np.linalg.norm(centre, axis=1) < 1.999
    c = np.array([1.0, 3.0, 4.0])
    h = np.array([4.0, 4.0, 4.0])
    assert np.all(np.isnan(p[np.linalg.norm(centre, axis=1) > 2.0001]))
    xc = contract64((p[reach] - c) / h)
    assert np.allclose(xc, centre[reach], atol=2e-4)
    inside = np.all((xc > lo_c[reach] - 1e-5) & (xc < lo_c[reach] + 0.25 + 1e-5), axis=1)
    assert inside.mean() > 0.999

"""Host-side parts of the library that need no GPU: the opacity criterion of the
grid update (Sec. 2.1: space is empty where alpha < 1e-2) as the density
threshold nacc_density_threshold computes."""
import math

import numpy as np
import pytest

from paper_2210_04847_gb300 import _lib, build


@pytest.fixture(scope="module", autouse=True)
def _built():
    build.build()


@pytest.mark.parametrize("thre,dt", [(1e-2, 0.0050744), (0.5, 0.01), (1e-6, 1.0), (0.9, 1e-3)])
def test_alpha_threshold_as_density_threshold(thre, dt):
    t = _lib.density_threshold(thre, dt)
    assert t == float(np.float32(t)) and t > 0
    # densities just above / below the converted threshold fall on the matching side
    # of the opacity criterion, evaluated in float64
    for s in (t * (1 + 1e-5), t * (1 + 1e-3), t * 3):
        assert 1.0 - math.exp(-s * dt) > thre
    for s in (t * (1 - 1e-5), t * 0.5, 0.0):
        assert not (1.0 - math.exp(-s * dt) > thre)


def test_alpha_threshold_zero_and_invalid():
    assert _lib.density_threshold(0.0, 0.5) == 0.0  # any density above zero is occupied
    for thre, dt in ((1.0, 0.1), (-0.1, 0.1), (0.5, 0.0), (0.5, -1.0), (float("nan"), 0.1), (0.5, float("inf"))):
        assert math.isnan(_lib.density_threshold(thre, dt))


def test_update_rejects_bad_alpha_step():
    lib = _lib.load()
    for thre, step in ((0.01, -1.0), (0.01, float("nan")), (1.5, 0.1)):
        assert lib.nacc_update_occupancy_grid(None, None, 0, None, None, 0, 0.9, thre, step, None, None) == \
            _lib.ERR_INVALID_ARG
    assert lib.nacc_update_occupancy_grid(None, None, 0, None, None, 0, 0.9, 0.01, 0.1, None, None) == _lib.OK

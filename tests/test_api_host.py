"""Host-side parts of the public API (no GPU): the opacity criterion of the grid
update (Sec. 2.1: space is empty where alpha < 1e-2) as a density threshold."""
import math

import numpy as np
import pytest

from paper_2210_04847_gb300 import api


@pytest.mark.parametrize("thre,dt", [(1e-2, 0.0050744), (0.5, 0.01), (1e-6, 1.0), (0.9, 1e-3)])
def test_alpha_threshold_as_density_threshold(thre, dt):
    t = api.alpha_to_density_threshold(thre, dt)
    assert t == float(np.float32(t))
    # densities just above / below the converted threshold fall on the matching side
    # of the opacity criterion, evaluated in float64
    for s in (t * (1 + 1e-5), t * (1 + 1e-3), t * 3):
        assert 1.0 - math.exp(-s * dt) > thre
    for s in (t * (1 - 1e-5), t * 0.5, 0.0):
        assert not (1.0 - math.exp(-s * dt) > thre)


def test_alpha_threshold_rejects_invalid():
    for thre, dt in ((1.0, 0.1), (-0.1, 0.1), (0.5, 0.0)):
        with pytest.raises(ValueError):
            api.alpha_to_density_threshold(thre, dt)

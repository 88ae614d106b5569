"""Colour-M/L preprocessing (Eq. 20 with the constants of App. C)."""
import math

import numpy as np
import pytest

from paper_2205_06819_gb300.preprocess import ml_from_colour


def test_relation_and_error_propagation():
    g = np.array([17.0, 18.2, 16.5])
    i = np.array([15.8, 17.1, 15.6])
    ml, dml, lml, dl = ml_from_colour(g, i, err_beta=0.02, err_gamma=0.03)
    np.testing.assert_allclose(lml, -0.70 + 0.89 * (g - i), rtol=1e-15)
    np.testing.assert_allclose(ml, 10 ** lml, rtol=1e-15)
    expect = math.sqrt(0.89 ** 2 * (0.02 ** 2 + 0.03 ** 2) + 0.07 ** 2)
    np.testing.assert_allclose(dl, expect, rtol=1e-15)
    np.testing.assert_allclose(dml, ml * math.log(10) * expect, rtol=1e-15)


def test_scatter_floor_without_photometric_errors():
    _, _, _, dl = ml_from_colour(17.0, 16.0)
    assert float(dl) == pytest.approx(0.07)

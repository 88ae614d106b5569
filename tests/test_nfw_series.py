"""The NFW enclosed-mass function of the kernels (bang_device.cuh, nfw_m), restated in
float64: for x <= 1, with z = x / (2 + x), m(x) = ln(1 + x) - x / (1 + x) is
x^2 / ((1 + x)(2 + x)) + 2 z^3 (1/3 + z^2/5 + ... + z^16/19), the first term being
2 z^2 / (1 + z) and z sharing its reciprocal.  Checked against the closed form (and its
small-x expansion x^2/2 - 2x^3/3, where the closed form cancels) to 1e-9 relative."""
import numpy as np


def nfw_series(x):
    x = np.asarray(x, dtype=np.float64)
    x1 = 1.0 + x
    rr = 1.0 / (x1 * (2.0 + x))
    z = x * x1 * rr
    z2 = z * z
    s = 1.0 / 19.0
    for k in (17, 15, 13, 11, 9, 7, 5, 3):
        s = s * z2 + 1.0 / k
    return x * x * rr + 2.0 * z2 * z * s


def test_series_matches_the_closed_form():
    x = np.geomspace(1e-3, 1.0, 400)
    exact = np.log1p(x) - x / (1.0 + x)
    assert np.max(np.abs(nfw_series(x) - exact) / exact) < 1e-9


def test_small_x_limit():
    x = np.geomspace(1e-6, 1e-4, 50)
    approx = x ** 2 / 2 - 2 * x ** 3 / 3 + 3 * x ** 4 / 4
    assert np.max(np.abs(nfw_series(x) - approx) / approx) < 1e-9


def test_first_term_identity():
    x = np.geomspace(1e-3, 1.0, 50)
    z = x / (2 + x)
    assert np.allclose(2 * z * z / (1 + z), x * x / ((1 + x) * (2 + x)), rtol=1e-14, atol=0)

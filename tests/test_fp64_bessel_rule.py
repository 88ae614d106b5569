"""The rule the float64 check path (bang_fp64.cu) uses for the modified Bessel functions of
the second kind, restated on the host and pinned against an independent library:
K_nu(x) = int_0^inf exp(-x cosh t) cosh(nu t) dt by the trapezoid rule with step 0.1
(0.1 sqrt(10 / x) beyond x = 10), cut where x cosh t > 745.  The device code itself is
checked on the GPU through the whole likelihood (tests/test_gpu_fp64.py, chi^2 to 1e-11
of the float64 oracle); this pins the rule's accuracy claim (< 2e-14 relative on
[1e-6, 200]) and the Freeman difference I0 K0 - I1 K1 built from it."""
import math

import numpy as np
import pytest

sp = pytest.importorskip("scipy.special")


def k01_rule(x: float):
    h = 0.1 if x <= 10.0 else 0.1 * math.sqrt(10.0 / x)
    tmax = math.acosh(745.0 / x) if x < 745.0 else 0.0
    n = int(math.ceil(tmax / h)) + 1
    t = np.arange(1, n + 1) * h
    c = np.cosh(t)
    e = np.exp(-x * c)
    s0 = 0.5 * math.exp(-x) + e.sum()
    s1 = 0.5 * math.exp(-x) + (e * c).sum()
    return h * s0, h * s1, n


def test_k0_k1_relative_error_over_the_range():
    worst = 0.0
    nmax = 0
    for x in np.geomspace(1e-6, 200.0, 1500):
        k0, k1, n = k01_rule(float(x))
        worst = max(worst, abs(k0 / sp.k0(x) - 1.0), abs(k1 / sp.k1(x) - 1.0))
        nmax = max(nmax, n)
    assert worst < 2e-14, worst
    assert nmax < 260          # the device loop's length stays bounded


def test_freeman_difference_against_the_library():
    for y in (1e-4, 0.01, 0.3, 1.0, 2.5, 7.0, 20.0, 60.0):
        k0, k1, _ = k01_rule(y)
        f = sp.i0(y) * k0 - sp.i1(y) * k1
        ref = sp.i0(y) * sp.k0(y) - sp.i1(y) * sp.k1(y)
        # the difference cancels like 1 / (2 y^2) at large y: relative error grows ~ y^2 eps
        assert abs(f / ref - 1.0) < 1e-13 * max(1.0, y * y), y


def test_a_coarser_step_would_fail():
    """The step matters: a fixed step 0.25 misses the narrow integrand at large x."""
    x = 60.0
    h = 0.25
    t = np.arange(0, int(math.ceil(math.acosh(745.0 / x) / h)) + 2) * h
    w = np.ones_like(t)
    w[0] = 0.5
    k0 = h * np.sum(w * np.exp(-x * np.cosh(t)))
    assert abs(k0 / sp.k0(x) - 1.0) > 1e-6

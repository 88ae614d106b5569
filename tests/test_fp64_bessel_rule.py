"""The rule the float64 check path (bang_fp64.cu) uses for the modified Bessel functions of
the second kind, restated on the host and pinned against an independent library:
K_nu(x) = int_0^inf exp(-x cosh t) cosh(nu t) dt by the trapezoid rule with step 0.1
(0.1 sqrt(10 / x) beyond x = 10), cut where x cosh t > 745; and, beyond y = 25, the
large-argument expansion of I0 K0 - I1 K1 (DLMF 10.40.6 for each product), pinned against
mpmath in 40-digit arithmetic up to y = 1e4, where the direct form overflows.  The device
code itself is checked on the GPU through the whole likelihood (tests/test_gpu_fp64.py,
chi^2 to 1e-11 of the float64 oracle); this pins the rule's accuracy claim (< 2e-14
relative on [1e-6, 200]) and the Freeman difference I0 K0 - I1 K1 built from it."""
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


def freeman_series(y: float) -> float:
    z2 = 1.0 / (4.0 * y * y)
    s, c, p0, p1, zk = 0.0, 1.0, 1.0, 1.0, 1.0
    for k in range(1, 13):
        o = (2.0 * k - 1.0) ** 2
        c *= (2.0 * k - 1.0) / (2.0 * k)
        p0 *= -o
        p1 *= 4.0 - o
        zk *= z2
        s += (-c if k & 1 else c) * (p0 - p1) * zk
    return s / (2.0 * y)


def test_freeman_large_argument_expansion_against_mpmath():
    mp = pytest.importorskip("mpmath")
    mp.mp.dps = 40
    for y in (25.0, 25.5, 30.0, 60.0, 300.0, 699.0, 750.0, 5000.0, 1e4):
        ref = mp.besseli(0, y) * mp.besselk(0, y) - mp.besseli(1, y) * mp.besselk(1, y)
        assert abs(freeman_series(y) / float(ref) - 1.0) < 1e-15, y
    # leading terms 1 / (4 y^3) (1 + 9 / (8 y^2)); continuity with the Bessel-function form at the switch
    assert abs(freeman_series(1e4) * 4e12 / (1.0 + 9.0 / 8e8) - 1.0) < 1e-15
    k0, k1, _ = k01_rule(25.0)
    assert abs((sp.i0(25.0) * k0 - sp.i1(25.0) * k1) / freeman_series(25.0) - 1.0) < 1e-12

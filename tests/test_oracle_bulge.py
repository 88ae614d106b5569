"""Pins for the oracle's bulge: Dehnen-family projected density and isotropic dispersion.

The oracle computes both by a fixed radial Gauss-Legendre rule (r = R cosh t).  These
tests hold it to things other than itself: the paper's closed forms for the Hernquist
(gamma = 1, Eqs. 4-6) and Jaffe (gamma = 2, Eqs. B4-B5) limits, the circular velocities
(Eqs. 2 and B2), and, for other gamma, adaptive quadrature of the defining integrals
(Abel projection and the Jeans equation of Eq. 6) and of the enclosed mass.
"""
import math

import numpy as np
import pytest
from scipy import integrate

G = 4.30091727e-6


def X_of_s(s):
    """Eq. 5."""
    if s < 1.0:
        return math.log((1.0 + math.sqrt(1.0 - s * s)) / s) / math.sqrt(1.0 - s * s)
    return math.acos(1.0 / s) / math.sqrt(s * s - 1.0)


def hernquist_sigma(R, a, M):
    """Eq. 4."""
    s = R / a
    return M / (2 * math.pi * a * a * (1 - s * s) ** 2) * ((2 + s * s) * X_of_s(s) - 3)


def hernquist_disp2(R, a, M):
    """Eq. 6."""
    s = R / a
    X = X_of_s(s)
    brace = (1.0 / (2 * (1 - s * s) ** 3)
             * (-3 * s * s * X * (8 * s ** 6 - 28 * s ** 4 + 35 * s * s - 20)
                - 24 * s ** 6 + 68 * s ** 4 - 65 * s * s + 6)
             - 6 * math.pi * s)
    return G * M * M / (12 * math.pi * a ** 3 * hernquist_sigma(R, a, M)) * brace


def jaffe_sigma(R, a, M):
    """Eq. B4."""
    s = R / a
    return M / (a * a) * (1 / (4 * s) + (1 - (2 - s * s) * X_of_s(s)) / (2 * math.pi * (1 - s * s)))


def jaffe_disp2(R, a, M):
    """Eq. B5."""
    s = R / a
    X = X_of_s(s)
    br = (math.pi / (2 * s) + 11 - 6.5 * math.pi * s - 12 * s * s + 6 * math.pi * s ** 3
          - X * (6 - 19 * s * s + 12 * s ** 4))
    return G * M * M / (4 * math.pi * a ** 3 * jaffe_sigma(R, a, M)) / (1 - s * s) * br


S_VALUES = [0.01, 0.05, 0.2, 0.5, 0.8, 0.95, 1.05, 1.3, 2.0, 4.0, 7.0, 10.0]


@pytest.mark.parametrize("s", S_VALUES)
def test_hernquist_limit_matches_closed_forms(oracle_mod, s):
    a, M = 0.7, 3.0e10
    Sig, s2 = oracle_mod.bulge_projected(s * a, a, 1.0, M, 64)
    assert Sig == pytest.approx(hernquist_sigma(s * a, a, M), rel=1e-9)
    assert s2 == pytest.approx(hernquist_disp2(s * a, a, M), rel=2e-8)


@pytest.mark.parametrize("s", S_VALUES)
def test_jaffe_limit_matches_closed_forms(oracle_mod, s):
    a, M = 1.3, 8.0e9
    Sig, s2 = oracle_mod.bulge_projected(s * a, a, 2.0, M, 64)
    assert Sig == pytest.approx(jaffe_sigma(s * a, a, M), rel=1e-9)
    assert s2 == pytest.approx(jaffe_disp2(s * a, a, M), rel=2e-8)


@pytest.mark.parametrize("nq", [64, 128])
def test_rule_size_does_not_change_result(oracle_mod, nq):
    for g in (0.0, 0.7, 1.6):
        Sig, s2 = oracle_mod.bulge_projected(0.3, 1.1, g, 1e10, nq)
        Sig_ref, s2_ref = oracle_mod.bulge_projected(0.3, 1.1, g, 1e10, 200)
        assert Sig == pytest.approx(Sig_ref, rel=1e-10)
        assert s2 == pytest.approx(s2_ref, rel=1e-10)


def _abel_sigma(rho, R):
    """2 int_R^inf rho(r) r / sqrt(r^2 - R^2) dr, split at 2R, the endpoint singularity
    handled by QUADPACK's algebraic weight (independent of the cosh substitution)."""
    f = lambda r: 2.0 * rho(r) * r / math.sqrt(r + R)
    I1, _ = integrate.quad(f, R, 2 * R, weight="alg", wvar=(-0.5, 0.0), epsabs=0, epsrel=1e-12, limit=200)
    g = lambda r: 2.0 * rho(r) * r / math.sqrt(r * r - R * R)
    I2, _ = integrate.quad(g, 2 * R, np.inf, epsabs=0, epsrel=1e-12, limit=400)
    return I1 + I2


@pytest.mark.parametrize("gamma", [0.0, 0.5, 1.5, 1.9])
@pytest.mark.parametrize("s", [0.05, 0.6, 3.0])
def test_general_gamma_sigma_vs_adaptive_abel_integral(oracle_mod, gamma, s):
    a, M = 0.9, 2.0e10
    rho = lambda r: (3 - gamma) * M * a / (4 * math.pi) * r ** (-gamma) * (r + a) ** (gamma - 4)
    Sig, _ = oracle_mod.bulge_projected(s * a, a, gamma, M, 64)
    assert Sig == pytest.approx(_abel_sigma(rho, s * a), rel=1e-8)


@pytest.mark.slow
@pytest.mark.parametrize("gamma", [0.3, 1.4])
@pytest.mark.parametrize("s", [0.2, 2.0])
def test_general_gamma_dispersion_vs_jeans_double_integral(oracle_mod, gamma, s):
    """Eq. 6 as defined: sigma^2 Sigma = 2 int rho vr^2 r / sqrt(r^2-R^2) dr, with the isotropic
    Jeans equation rho vr^2 (r) = int_r^inf rho G M / r'^2 dr' (bulge potential only)."""
    a, M = 1.2, 5.0e10
    rho = lambda r: (3 - gamma) * M * a / (4 * math.pi) * r ** (-gamma) * (r + a) ** (gamma - 4)
    mass = lambda r: M * (r / (r + a)) ** (3 - gamma)

    def rho_vr2(r):
        v, _ = integrate.quad(lambda x: rho(x) * G * mass(x) / (x * x), r, np.inf, epsabs=0, epsrel=1e-12, limit=200)
        return v

    R = s * a
    Sig, s2 = oracle_mod.bulge_projected(R, a, gamma, M, 64)
    num = _abel_sigma(lambda r: rho_vr2(r), R)
    assert s2 == pytest.approx(num / Sig, rel=1e-7)


@pytest.mark.parametrize("gamma", [0.0, 0.5, 1.0, 1.5, 2.0, 2.5])
@pytest.mark.parametrize("x", [0.1, 1.0, 10.0])
def test_dehnen_enclosed_mass(oracle_mod, gamma, x):
    a, M = 1.5, 1.0e10
    r = x * a
    num, _ = integrate.quad(lambda t: 4 * math.pi * t * t * oracle_mod.dehnen_rho(t, a, gamma, M), 0, r,
                            epsabs=0, epsrel=1e-12, limit=200)
    assert oracle_mod.dehnen_mass(r, a, gamma, M) == pytest.approx(num, rel=1e-9)


def test_dehnen_total_mass_is_M(oracle_mod):
    for gamma in (0.0, 1.0, 2.0):
        assert oracle_mod.dehnen_mass(1e9, 1.0, gamma, 7e9) == pytest.approx(7e9, rel=1e-8)


@pytest.mark.parametrize("r", [0.01, 0.5, 2.0, 30.0])
def test_circular_velocity_hernquist_and_jaffe(oracle_mod, r):
    a, M = 0.8, 4e10
    # Eq. 2 (Hernquist): v = sqrt(G M r) / (r + a)
    assert oracle_mod.bulge_vc2(r, a, 1.0, M) == pytest.approx(G * M * r / (r + a) ** 2, rel=1e-13)
    # Eq. B2 (Jaffe): v^2 = G M / (r + a)
    assert oracle_mod.bulge_vc2(r, a, 2.0, M) == pytest.approx(G * M / (r + a), rel=1e-13)


def _jeans_vr2(rho, mass, r):
    v, _ = integrate.quad(lambda x: rho(x) * G * mass(x) / (x * x), r, np.inf, epsabs=0, epsrel=1e-12, limit=200)
    return v / rho(r)


@pytest.mark.parametrize("x", [0.1, 0.7, 3.0])
def test_paper_hernquist_radial_dispersion_eq3(x):
    """Eq. 3 is the isotropic Jeans solution for the Hernquist bulge (checks the reading that
    the bulge feels only its own potential)."""
    a, M = 1.0, 1e10
    r = x * a
    rho = lambda t: M / (2 * math.pi) * a / (t * (t + a) ** 3)
    mass = lambda t: M * t * t / (t + a) ** 2
    eq3 = G * M / (12 * a) * (12 * r * (r + a) ** 3 / a ** 4 * math.log((r + a) / r)
                              - r / (r + a) * (25 + 52 * r / a + 42 * (r / a) ** 2 + 12 * (r / a) ** 3))
    assert eq3 == pytest.approx(_jeans_vr2(rho, mass, r), rel=1e-7)


@pytest.mark.parametrize("x", [0.1, 0.7, 3.0])
def test_paper_jaffe_radial_dispersion_eqB3_has_sign_error(x):
    """Eq. B3 as printed (with its undefined 'a' read as R_b) is the negative of the Jeans
    solution: the bracket's sign is flipped.  The oracle never uses Eq. B3."""
    a, M = 1.0, 1e10
    r = x * a
    rho = lambda t: M / (4 * math.pi) * a / (t * t * (t + a) ** 2)
    mass = lambda t: M * t / (t + a)
    printed = G * M * r * r * (r + a) ** 2 / a ** 4 * (3 / r + (6 * r + 7 * a) / (2 * (a + r) ** 2)
                                                        - a / (2 * r * r) - 6 / a * math.log(1 + a / r))
    assert -printed == pytest.approx(_jeans_vr2(rho, mass, r), rel=1e-6)


@pytest.mark.parametrize("n", [8, 64, 128])
def test_gauss_legendre_nodes_match_numpy_and_are_exact(oracle_mod, n):
    x, w = oracle_mod.gauss_legendre(n)
    xr, wr = np.polynomial.legendre.leggauss(n)
    np.testing.assert_allclose(x, xr, rtol=0, atol=1e-14)
    np.testing.assert_allclose(w, wr, rtol=1e-10)      # numpy's own weights drift ~1e-11 at n = 128
    for k in range(0, 2 * n, 2):                       # exact for every degree <= 2n - 1
        assert (w * x ** k).sum() == pytest.approx(2.0 / (k + 1), rel=1e-13)

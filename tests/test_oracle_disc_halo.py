"""Pins for the oracle's exponential disc (Eq. 9 reading) and NFW halo.

The Freeman circular velocity is held to a direct numerical integration of the disc's
surface density (ring potentials with complete elliptic integrals, then d Phi / d r),
to its maximum at r ~ 2.15 R_d and to its Keplerian limit; the Bessel product to
high-precision mpmath values; the NFW halo to its enclosed-mass integral and to the
definition of M200.
"""
import math

import numpy as np
import pytest
from scipy import integrate, optimize, special

G = 4.30091727e-6


def test_bessel_product_matches_mpmath(oracle_mod):
    mpmath = pytest.importorskip("mpmath")
    mpmath.mp.dps = 40
    for y in np.geomspace(1e-3, 40.0, 37):
        yy = mpmath.mpf(float(y))
        ref = mpmath.besseli(0, yy) * mpmath.besselk(0, yy) - mpmath.besseli(1, yy) * mpmath.besselk(1, yy)
        assert oracle_mod.bessel_diff(y) == pytest.approx(float(ref), rel=2e-12), y


def _ring_potential(r, Md, Rd):
    """Phi(r) in the plane of a razor-thin disc of surface density Sigma(r') (Eq. 7):
    Phi = -4 G int Sigma(r') r' K(m) / (r + r') dr', m = 4 r r' / (r + r')^2.
    K has a log singularity at r' = r: K = [K + ln|r - r'|] - ln|r - r'|, the second part
    integrated with QUADPACK's logarithmic weights."""
    sig0 = Md / (2 * math.pi * Rd * Rd)
    s = lambda rp: sig0 * math.exp(-rp / Rd) * rp / (r + rp)

    def k_smooth(rp):
        return special.ellipkm1(((r - rp) / (r + rp)) ** 2) + math.log(abs(r - rp))

    o = dict(epsabs=0, epsrel=1e-13, limit=400)
    a1, _ = integrate.quad(lambda x: s(x) * k_smooth(x), 0.0, r, **o)
    a2, _ = integrate.quad(lambda x: s(x) * k_smooth(x), r, 2 * r, **o)
    b1, _ = integrate.quad(s, 0.0, r, weight="alg-logb", wvar=(0, 0), **o)
    b2, _ = integrate.quad(s, r, 2 * r, weight="alg-loga", wvar=(0, 0), **o)
    c, _ = integrate.quad(lambda x: s(x) * special.ellipk(4 * r * x / (r + x) ** 2), 2 * r, np.inf, **o)
    return -4.0 * G * (a1 + a2 - b1 - b2 + c)


@pytest.mark.parametrize("x", [0.3, 1.0, 2.15, 5.0, 10.0])
def test_freeman_velocity_vs_direct_integration(oracle_mod, x):
    Md, Rd = 3e10, 2.5
    r = x * Rd
    d = 1e-3 * r
    # five-point derivative of the numerically integrated potential: v^2 = r dPhi/dr
    phi = [_ring_potential(r + k * d, Md, Rd) for k in (-2, -1, 1, 2)]
    dphi = (phi[0] - 8 * phi[1] + 8 * phi[2] - phi[3]) / (12 * d)
    assert oracle_mod.freeman_vc2(r, Md, Rd) == pytest.approx(r * dphi, rel=1e-9)


def test_freeman_velocity_peaks_near_2p15_Rd(oracle_mod):
    Md, Rd = 1e10, 3.0
    res = optimize.minimize_scalar(lambda r: -oracle_mod.freeman_vc2(r, Md, Rd), bounds=(0.5 * Rd, 5 * Rd),
                                   method="bounded", options={"xatol": 1e-8})
    assert res.x / Rd == pytest.approx(2.1492, abs=2e-3)


def test_freeman_velocity_keplerian_limit(oracle_mod):
    Md, Rd = 1e10, 2.0
    for y in (20.0, 30.0):
        r = 2 * Rd * y
        ratio = oracle_mod.freeman_vc2(r, Md, Rd) * r / (G * Md)
        # large-y expansion of I0K0 - I1K1 from DLMF 10.40.6:
        # 1/(4y^3) (1 + 9/(8 y^2) + 675/(128 y^4) + O(y^-6))
        assert ratio == pytest.approx(1.0 + 9.0 / (8 * y * y) + 675.0 / (128 * y ** 4), rel=2e-6)


def test_nfw_r200_definition(oracle_mod):
    for M200 in (1e11, 3e12, 1e14):
        r200 = oracle_mod.nfw_r200(M200)
        assert M200 / (4.0 / 3.0 * math.pi * r200 ** 3) == pytest.approx(200 * oracle_mod.rho_crit(), rel=1e-12)


def test_rho_crit_value(oracle_mod):
    # 2.775e11 h^2 Msun / Mpc^3 with h = 0.7, in Msun / kpc^3
    assert oracle_mod.rho_crit() == pytest.approx(2.7754e11 * 0.49 / 1e9, rel=1e-3)


@pytest.mark.parametrize("c", [5.0, 10.0, 15.0])
def test_nfw_mass_at_r200_is_M200(oracle_mod, c):
    M200 = 10 ** 12.3
    r200 = oracle_mod.nfw_r200(M200)
    assert oracle_mod.nfw_vc2(r200, M200, c) * r200 / G == pytest.approx(M200, rel=1e-12)


@pytest.mark.parametrize("x", [0.01, 0.3, 1.0, 4.0])
def test_nfw_enclosed_mass_integral(oracle_mod, x):
    M200, c = 10 ** 12.0, 8.0
    r200 = oracle_mod.nfw_r200(M200)
    rs = r200 / c
    m = lambda u: math.log1p(u) - u / (1 + u)
    rho_s = M200 / (4 * math.pi * rs ** 3 * m(c))
    rho = lambda r: rho_s / ((r / rs) * (1 + r / rs) ** 2)
    r = x * rs
    num, _ = integrate.quad(lambda t: 4 * math.pi * t * t * rho(t), 0, r, epsabs=0, epsrel=1e-12)
    assert oracle_mod.nfw_vc2(r, M200, c) * r / G == pytest.approx(num, rel=1e-9)


@pytest.mark.parametrize("x", [0.05, 0.5, 2.0, 8.0])
def test_hernquist_halo_is_the_enclosed_mass_of_eq1(oracle_mod, x):
    """The paper's halo: Eq. 2 with the halo's mass and scale radius, i.e. G M(<r) / r for
    the density of Eq. 1, integrated here numerically."""
    Mh, Rh = 10 ** 12.2, 25.0
    r = x * Rh
    rho = lambda t: Mh / (2 * math.pi) * Rh / (t * (t + Rh) ** 3)
    num, _ = integrate.quad(lambda t: 4 * math.pi * t * t * rho(t), 0, r, epsabs=0, epsrel=1e-12)
    assert oracle_mod.hernquist_halo_vc2(r, Mh, Rh) * r / G == pytest.approx(num, rel=1e-10)

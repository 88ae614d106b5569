"""Pins for the oracle's PSF + binning and for the whole model and likelihood.

PSF + binning is held to an independent library route (scipy.ndimage correlation then a
block mean) and to flux conservation; the whole model to its symmetries and special
cases (Sec. 2.1-2.4), to a brute-force restatement on a 2x2 grid that integrates the
bulge adaptively, to zero chi^2 and zero gradient on noise-free data, and its dual-number
gradient to central finite differences.
"""
import math

import numpy as np
import pytest
from scipy import integrate, ndimage, special

from paper_2205_06819_gb300 import synth

KPA = synth.KPC_PER_ARCSEC
G = 4.30091727e-6

THETA = np.array([0.05, -0.08, 0.4, 0.95, 10.2, math.log10(0.9), 1.3, 10.4, math.log10(2.8), 0.55,
                  3.5, 2.0, 12.4, 9.0, 15.0])


def gal_of(oracle_mod, nx=8, ny=6, os_=2, fwhm=1.5, kind=0, beta=3.0, data=None, err=None, mask=None):
    return oracle_mod.Galaxy(nx, ny, os_, fwhm, KPA, psf_kind=kind, moffat_beta=beta, data=data, err=err,
                             mask=mask)


# ------------------------------------------------------------------ PSF and binning
def test_psf_halfwidth_of_the_workloads(oracle_mod):
    # h = floor(3 sigma / pitch): 30x30 os 3 -> 9; 80x80 os 5 -> 15; 128x128 os 7 -> 22
    assert gal_of(oracle_mod, 30, 30, 3, 2.5).h == 9
    assert gal_of(oracle_mod, 80, 80, 5, 2.5).h == 15
    assert gal_of(oracle_mod, 128, 128, 7, 2.5, kind=1).h == 22


def test_gaussian_weights(oracle_mod):
    g = gal_of(oracle_mod, 4, 4, 3, 2.0)
    w = oracle_mod.psf_weights(g)
    h = g.h
    sig = 2.0 / (2 * math.sqrt(2 * math.log(2)))
    p = 1.0 / 3
    d = np.arange(-h, h + 1) * p
    ref = np.exp(-(d[None, :] ** 2 + d[:, None] ** 2) / (2 * sig * sig))
    np.testing.assert_allclose(w, ref / ref.sum(), rtol=1e-14)
    assert w.sum() == pytest.approx(1.0, abs=1e-15)


def test_moffat_weights(oracle_mod):
    g = gal_of(oracle_mod, 4, 4, 3, 2.5, kind=1, beta=3.0)
    w = oracle_mod.psf_weights(g)
    h = g.h
    alpha = 2.5 / (2 * math.sqrt(2 ** (1 / 3.0) - 1))
    d = np.arange(-h, h + 1) / 3.0
    ref = (1 + (d[None, :] ** 2 + d[:, None] ** 2) / alpha ** 2) ** -3.0
    np.testing.assert_allclose(w, ref / ref.sum(), rtol=1e-14)
    # FWHM: the profile falls to half at rho = FWHM / 2
    assert (1 + (1.25 / alpha) ** 2) ** -3.0 == pytest.approx(0.5, rel=1e-12)


@pytest.mark.parametrize("kind", [0, 1])
def test_convolve_bin_matches_scipy_correlate_then_block_mean(oracle_mod, kind):
    g = gal_of(oracle_mod, 7, 5, 3, 2.2, kind=kind)
    H, W = g.padded_shape
    rng = np.random.default_rng(7)
    field = rng.normal(size=(4, H, W))
    out = oracle_mod.convolve_bin(g, field)
    w = oracle_mod.psf_weights(g)
    h, os_ = g.h, g.os
    for c in range(4):
        conv = ndimage.correlate(field[c], w, mode="constant", cval=0.0)
        inner = conv[h:H - h, h:W - h]
        ref = inner.reshape(g.ny, os_, g.nx, os_).mean(axis=(1, 3))
        np.testing.assert_allclose(out[c], ref, rtol=1e-12, atol=1e-14)


def test_binning_alone_conserves_flux(oracle_mod):
    g = gal_of(oracle_mod, 6, 4, 4, 0.0)
    assert g.h == 0
    H, W = g.padded_shape
    field = np.random.default_rng(3).uniform(size=(4, H, W))
    out = oracle_mod.convolve_bin(g, field)
    np.testing.assert_allclose(out.sum(axis=(1, 2)) * g.os ** 2, field.sum(axis=(1, 2)), rtol=1e-13)


def test_psf_conserves_flux_of_compact_source(oracle_mod):
    g = gal_of(oracle_mod, 12, 12, 3, 2.0)
    H, W = g.padded_shape
    h = g.h
    field = np.zeros((4, H, W))
    # a compact source at least h fine pixels inside the field
    field[:, H // 2 - 2:H // 2 + 3, W // 2 - 1:W // 2 + 2] = np.random.default_rng(1).uniform(size=(4, 5, 3))
    assert H // 2 - 2 - h >= h
    out = oracle_mod.convolve_bin(g, field)
    np.testing.assert_allclose(out.sum(axis=(1, 2)) * g.os ** 2, field.sum(axis=(1, 2)), rtol=1e-12)


# ------------------------------------------------------------------ whole model
def test_velocity_antisymmetric_about_minor_axis(oracle_mod):
    th = THETA.copy()
    th[[0, 1, 2, 14]] = 0.0           # centred, major axis along x, no systemic velocity
    g = gal_of(oracle_mod, 8, 6, 3, 1.8)
    m = oracle_mod.maps(g, th)
    np.testing.assert_allclose(m[1], -m[1][:, ::-1], rtol=1e-10, atol=1e-9)
    for c in (0, 2, 3):
        np.testing.assert_allclose(m[c], m[c][:, ::-1], rtol=1e-10)
        np.testing.assert_allclose(m[c], m[c][::-1, :], rtol=1e-10)
    np.testing.assert_allclose(m[1], m[1][::-1, :], rtol=1e-10, atol=1e-9)
    assert np.abs(m[1]).max() > 10.0


@pytest.mark.parametrize("slot,value", [(9, 0.0), (3, 0.0)])
def test_no_rotation_when_k_or_inclination_is_zero(oracle_mod, slot, value):
    th = THETA.copy()
    th[slot] = value
    m = oracle_mod.maps(gal_of(oracle_mod), th)
    np.testing.assert_allclose(m[1], th[14], rtol=0, atol=1e-12)


def test_k_one_leaves_only_bulge_dispersion(oracle_mod):
    th = THETA.copy()
    th[9] = 1.0
    xs = np.array([0.3, -2.0, 1.5]); ys = np.array([0.2, 1.1, -3.0])
    out = oracle_mod.points(th, xs, ys, KPA)
    for p in range(xs.size):
        X, Y = xs[p] * KPA - th[0], ys[p] * KPA - th[1]
        xr = X * math.cos(th[2]) + Y * math.sin(th[2])
        yr = -X * math.sin(th[2]) + Y * math.cos(th[2])
        R = math.hypot(xr, yr)
        Sb, s2b = oracle_mod.bulge_projected(R, 10 ** th[5], th[6], 10 ** th[4], 64)
        Bb = Sb * 1e-6 / th[10]
        assert out[2, p] ** 2 * out[0, p] == pytest.approx(Bb * s2b, rel=1e-12)


def test_point_sampling_without_psf_or_oversampling(oracle_mod):
    g = gal_of(oracle_mod, 5, 4, 1, 0.0)
    m = oracle_mod.maps(g, THETA)
    xs = (np.arange(5) - 2.0)[None, :].repeat(4, 0)
    ys = (np.arange(4) - 1.5)[:, None].repeat(5, 1)
    p = oracle_mod.points(THETA, xs.ravel(), ys.ravel(), KPA).reshape(4, 4, 5)
    np.testing.assert_allclose(m[0], p[0], rtol=1e-14)
    np.testing.assert_allclose(m[1], p[1] + THETA[14], rtol=1e-14)
    np.testing.assert_allclose(m[2], p[2], rtol=1e-14)
    np.testing.assert_allclose(m[3], 1.0 / p[3], rtol=1e-14)


def test_quadrature_converged_64_vs_128_nodes(oracle_mod):
    g = gal_of(oracle_mod)
    np.testing.assert_allclose(oracle_mod.maps(g, THETA, n_quad=64), oracle_mod.maps(g, THETA, n_quad=128),
                               rtol=1e-10)


def test_two_disc_model_reduces_to_one_disc_when_second_is_dark_and_light(oracle_mod):
    """A second disc of negligible mass leaves all maps unchanged."""
    th2 = np.concatenate([THETA, [1.0, 0.5, 0.3, 2.0]])   # 10 Msun second disc
    g = gal_of(oracle_mod)
    np.testing.assert_allclose(oracle_mod.maps(g, th2, n_discs=2), oracle_mod.maps(g, THETA), rtol=1e-8)


# ------------------------------------------------------------------ brute force, 2x2 spaxels
def _brute_point(th, xs, ys):
    """Independent restatement at one sky point: bulge integrals by adaptive quadrature of
    the Abel and Jeans integrals in r (no cosh rule), Bessel functions from scipy."""
    x0, y0, pa, inc, lMb, lRb, gam, lMd, lRd, k, MLb, MLd, lMh, c, vsys = th
    Mb, a, Md, Rd, Mh = 10 ** lMb, 10 ** lRb, 10 ** lMd, 10 ** lRd, 10 ** lMh
    X, Y = xs * KPA - x0, ys * KPA - y0
    xr = X * math.cos(pa) + Y * math.sin(pa)
    yr = -X * math.sin(pa) + Y * math.cos(pa)
    R = math.hypot(xr, yr)
    rr = math.hypot(xr, yr / math.cos(inc))
    rho = lambda r: (3 - gam) * Mb * a / (4 * math.pi) * r ** -gam * (r + a) ** (gam - 4)
    mass = lambda r: Mb * (r / (r + a)) ** (3 - gam)
    o = dict(epsabs=0, epsrel=1e-12, limit=400)
    Sb = (integrate.quad(lambda r: 2 * rho(r) * r / math.sqrt(r + R), R, 2 * R, weight="alg", wvar=(-0.5, 0), **o)[0]
          + integrate.quad(lambda r: 2 * rho(r) * r / math.sqrt(r * r - R * R), 2 * R, np.inf, **o)[0])
    q = lambda r: 2 * G * rho(r) * mass(r) / (r * r)
    Qb = (integrate.quad(lambda r: q(r) * math.sqrt(r + R), R, 2 * R, weight="alg", wvar=(0.5, 0), **o)[0]
          + integrate.quad(lambda r: q(r) * math.sqrt(r * r - R * R), 2 * R, np.inf, **o)[0])
    s2b = Qb / Sb
    vb2 = G * mass(rr) / rr
    r200 = (3 * Mh / (4 * math.pi * 200 * (3 * 0.07 ** 2 / (8 * math.pi * G)))) ** (1 / 3)
    m = lambda u: math.log1p(u) - u / (1 + u)
    vh2 = G * Mh * m(rr * c / r200) / (m(c) * rr)
    y = rr / (2 * Rd)
    vd2 = 2 * G * Md / Rd * y * y * (special.i0(y) * special.k0(y) - special.i1(y) * special.k1(y))
    vint2 = vb2 + vh2 + vd2
    Sd = Md / (2 * math.pi * Rd * Rd) * math.exp(-rr / Rd) / math.cos(inc)
    vd = -k * math.sin(inc) * (xr / rr) * math.sqrt(vint2)
    s2d = (1 - k * k) * vint2 / 3
    Bb, Bd = Sb * 1e-6 / MLb, Sd * 1e-6 / MLd
    B = Bb + Bd
    return np.array([B, Bd * vd / B, math.sqrt((Bb * s2b + Bd * s2d) / B), B / (1e-6 * (Sb + Sd))])


def test_brute_force_two_by_two(oracle_mod):
    th = THETA.copy()
    g = gal_of(oracle_mod, 2, 2, 1, 1.0)
    h = g.h
    assert h == 1
    H, W = g.padded_shape
    field = np.zeros((4, H, W))
    for qy in range(H):
        for qx in range(W):
            field[:, qy, qx] = _brute_point(th, (qx - h + 0.5) - 1.0, (qy - h + 0.5) - 1.0)
    sig = 1.0 / (2 * math.sqrt(2 * math.log(2)))
    wts = np.exp(-np.add.outer(np.arange(-1, 2) ** 2, np.arange(-1, 2) ** 2) / (2 * sig * sig))
    wts /= wts.sum()
    ref = np.zeros((4, 2, 2))
    for j in range(2):
        for i in range(2):
            ref[:, j, i] = (field[:, j:j + 3, i:i + 3] * wts[None]).sum(axis=(1, 2))
    ref[1] += th[14]
    ref[3] = 1.0 / ref[3]
    np.testing.assert_allclose(oracle_mod.maps(g, th), ref, rtol=2e-9)


# ------------------------------------------------------------------ likelihood and gradient
def _galaxy_with_data(oracle_mod, theta_true, noise=True, nx=8, ny=6, os_=2, fwhm=1.5, n_discs=1):
    g0 = gal_of(oracle_mod, nx, ny, os_, fwhm)
    true = oracle_mod.maps(g0, theta_true, n_discs=n_discs)
    data, err, mask = synth.noisy_data(true, seed=11, noise=noise)
    return gal_of(oracle_mod, nx, ny, os_, fwhm, data=data.astype(np.float64), err=err.astype(np.float64),
                  mask=mask), true


def test_noise_free_data_gives_zero_chi2_and_zero_gradient(oracle_mod):
    g0 = gal_of(oracle_mod)
    true = oracle_mod.maps(g0, THETA)
    err = synth.error_maps(true)
    g = gal_of(oracle_mod, data=true, err=err)
    logL, chi2 = oracle_mod.loglike(g, THETA)
    assert chi2[0] == pytest.approx(0.0, abs=1e-18)
    assert logL[0] == pytest.approx(-oracle_mod.norm_const(g), rel=1e-15)
    _, grad = oracle_mod.loglike_grad(g, THETA)
    _, grad_off = oracle_mod.loglike_grad(g, THETA + 0.01)
    # zero up to the rounding of the model maps (the dual path rounds slightly differently)
    assert np.abs(grad).max() < 1e-10 * np.abs(grad_off).max()


def test_norm_const_matches_definition(oracle_mod):
    g, _ = _galaxy_with_data(oracle_mod, THETA)
    assert oracle_mod.norm_const(g) == pytest.approx(np.sum(np.log(math.sqrt(2 * math.pi) * g.err)), rel=1e-14)


def test_masked_spaxels_are_ignored(oracle_mod):
    g, _ = _galaxy_with_data(oracle_mod, THETA)
    mask = np.ones((4, 6, 8), np.uint8)
    mask[1, 2, 3] = 0
    mask[3, :, 0] = 0
    gm = gal_of(oracle_mod, data=g.data, err=g.err, mask=mask)
    th = THETA + 0.01
    m = oracle_mod.maps(gal_of(oracle_mod), th)
    ref = (((m - g.data) / g.err) ** 2 * mask).sum()
    assert oracle_mod.loglike(gm, th)[1][0] == pytest.approx(ref, rel=1e-13)


def test_out_of_domain_rows_give_minus_inf(oracle_mod):
    g, _ = _galaxy_with_data(oracle_mod, THETA)
    bad = np.repeat(THETA[None], 6, 0)
    bad[1, 3] = 1.6          # inclination past 90 deg
    bad[2, 6] = 3.0          # gamma = 3
    bad[3, 9] = 1.2          # |k| > 1
    bad[4, 13] = -1.0        # c < 0
    bad[5, 10] = np.nan
    logL, _ = oracle_mod.loglike(g, bad)
    assert np.isfinite(logL[0])
    assert np.all(np.isneginf(logL[1:]))
    _, grad = oracle_mod.loglike_grad(g, bad)
    assert np.all(grad[1:] == 0.0)


@pytest.mark.parametrize("n_discs", [1, 2])
def test_dual_gradient_matches_central_differences(oracle_mod, n_discs):
    th_true = THETA if n_discs == 1 else np.concatenate([THETA, [10.1, 0.6, 0.8, 2.5]])
    g, _ = _galaxy_with_data(oracle_mod, th_true, n_discs=n_discs)
    th = th_true + np.random.default_rng(5).normal(size=th_true.size) * 0.02
    logL, grad = oracle_mod.loglike_grad(g, th, n_discs=n_discs)
    assert logL[0] == pytest.approx(oracle_mod.loglike(g, th, n_discs=n_discs)[0][0], rel=1e-14)
    def central(p, h):
        tp, tm = th.copy(), th.copy()
        tp[p] += h
        tm[p] -= h
        return (oracle_mod.loglike(g, tp, n_discs=n_discs)[0][0]
                - oracle_mod.loglike(g, tm, n_discs=n_discs)[0][0]) / (2 * h)

    fd = np.zeros(th.size)
    for p in range(th.size):
        h = 1e-4 * max(abs(th[p]), 1.0)
        # Richardson extrapolation of central differences at h and h/2 (error O(h^4))
        fd[p] = (4.0 * central(p, h / 2) - central(p, h)) / 3.0
    scale = np.abs(grad).max()
    np.testing.assert_allclose(grad[0], fd, rtol=1e-6, atol=1e-8 * scale)


def test_hernquist_halo_gradient_and_domain(oracle_mod):
    """halo_kind 1 (slot 13 = log10 R_h): dual gradient vs Richardson differences; c <= 0 is
    no longer a domain limit."""
    th = THETA.copy()
    th[13] = 1.4                                    # log10 R_h = 1.4 (25 kpc)
    g0 = gal_of(oracle_mod)
    true = oracle_mod.maps(g0, th, halo_kind=1)
    data, err, mask = synth.noisy_data(true, seed=12)
    g = gal_of(oracle_mod, data=data.astype(np.float64), err=err.astype(np.float64), mask=mask)
    t = th + np.random.default_rng(6).normal(size=th.size) * 0.02
    logL, grad = oracle_mod.loglike_grad(g, t, halo_kind=1)
    assert np.isfinite(logL[0])

    def central(p, h):
        tp, tm = t.copy(), t.copy()
        tp[p] += h
        tm[p] -= h
        return (oracle_mod.loglike(g, tp, halo_kind=1)[0][0] - oracle_mod.loglike(g, tm, halo_kind=1)[0][0]) / (2 * h)

    fd = np.array([(4 * central(p, 5e-5 * max(abs(t[p]), 1)) - central(p, 1e-4 * max(abs(t[p]), 1))) / 3
                   for p in range(t.size)])
    np.testing.assert_allclose(grad[0], fd, rtol=1e-6, atol=1e-8 * np.abs(grad).max())
    neg = t.copy()
    neg[13] = -0.5                                  # R_h = 0.3 kpc: valid for the Hernquist halo
    assert np.isfinite(oracle_mod.loglike(g, neg, halo_kind=1)[0][0])
    assert np.isneginf(oracle_mod.loglike(g, neg, halo_kind=0)[0][0])

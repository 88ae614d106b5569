"""Oracle pins for the PSF modes (Eq. 21 and App. A): the circular 3-sigma window, centre
sampling and flux-weighted moments, against independent numpy / scipy restatements:
scipy.ndimage.correlate with a numpy-built kernel, a brute-force centre-sampling loop, and
the flux-weighted pipeline rebuilt from the oracle's own point values of the default mode.
Special cases: os = 1 makes centre sampling equal binning; no PSF makes centre sampling
point sampling (odd os) or the mean of the four central points (even os); no PSF and
os = 1 makes the flux-weighted maps equal the default ones."""
import math

import numpy as np
import pytest
from scipy import ndimage

import oracle
from paper_2205_06819_gb300 import synth

CIRCLE, CENTRE, FLUX = 1, 2, 4


def gal(nx, ny, os_, fwhm, mode, kind=0, beta=3.0, data=None, err=None):
    return oracle.Galaxy(nx, ny, os_, fwhm, synth.KPC_PER_ARCSEC, psf_kind=kind, moffat_beta=beta, psf_mode=mode,
                         data=data, err=err)


def psf_np(dx, dy, pitch, fwhm, kind, beta):
    d2 = (dx * dx + dy * dy) * pitch * pitch
    if kind == 0:
        sig = fwhm / (2.0 * math.sqrt(2.0 * math.log(2.0)))
        return np.exp(-d2 / (2 * sig * sig))
    alpha = fwhm / (2.0 * math.sqrt(2.0 ** (1.0 / beta) - 1.0))
    return (1.0 + d2 / (alpha * alpha)) ** (-beta)


def window_np(dx, dy, rho, circle):
    return (dx * dx + dy * dy <= rho * rho) if circle else ((np.abs(dx) <= rho) & (np.abs(dy) <= rho))


def kernel_np(g, fwhm, circle, kind=0, beta=3.0):
    pitch = 1.0 / g.os
    sig = fwhm / (2.0 * math.sqrt(2.0 * math.log(2.0)))
    rho = 3 * sig / pitch
    d = np.arange(-g.h, g.h + 1, dtype=np.float64)
    dy, dx = np.meshgrid(d, d, indexing="ij")
    k = psf_np(dx, dy, pitch, fwhm, kind, beta) * window_np(dx, dy, rho, circle)
    return k / k.sum()


@pytest.mark.parametrize("kind", [0, 1])
def test_circular_window_binning_matches_scipy(kind):
    g = gal(7, 5, 3, 2.2, CIRCLE, kind=kind)
    H, W = g.padded_shape
    field = np.random.default_rng(5).normal(size=(4, H, W))
    out = oracle.convolve_bin(g, field)
    k = kernel_np(g, 2.2, True, kind)
    h, os_ = g.h, g.os
    for c in range(4):
        conv = ndimage.correlate(field[c], k, mode="constant", cval=0.0)[h:H - h, h:W - h]
        np.testing.assert_allclose(out[c], conv.reshape(g.ny, os_, g.nx, os_).mean(axis=(1, 3)), rtol=1e-12,
                                   atol=1e-14)


def test_circular_weights_are_the_square_ones_cut_to_the_circle():
    sq, ci = gal(4, 4, 3, 2.6, 0), gal(4, 4, 3, 2.6, CIRCLE)
    ws, wc = oracle.psf_weights(sq), oracle.psf_weights(ci)
    h = sq.h
    d = np.arange(-h, h + 1)
    dy, dx = np.meshgrid(d, d, indexing="ij")
    rho = 3 * 2.6 / (2 * math.sqrt(2 * math.log(2))) * 3
    inside = dx * dx + dy * dy <= rho * rho
    assert np.all(wc[~inside] == 0.0) and np.all(wc[inside] > 0.0) and (~inside).any()
    assert abs(wc.sum() - 1.0) < 1e-14
    np.testing.assert_allclose(wc[inside] / ws[inside], (wc[inside] / ws[inside])[0], rtol=1e-13)


def centre_reference(g, field, fwhm, circle, kind=0, beta=3.0):
    """Brute force: for every spaxel the PSF-weighted mean of the fine points around its
    centre (inside the window, or the nearest ones)."""
    H, W = g.padded_shape
    pitch = 1.0 / g.os
    sig = fwhm / (2.0 * math.sqrt(2.0 * math.log(2.0))) if fwhm > 0 else 0.0
    rho = 3 * sig / pitch
    qy, qx = np.meshgrid(np.arange(H, dtype=np.float64), np.arange(W, dtype=np.float64), indexing="ij")
    out = np.zeros((4, g.ny, g.nx))
    for j in range(g.ny):
        for i in range(g.nx):
            cx, cy = g.h + i * g.os + (g.os - 1) / 2, g.h + j * g.os + (g.os - 1) / 2
            dx, dy = qx - cx, qy - cy
            near = (np.abs(dx) <= 0.5) & (np.abs(dy) <= 0.5)
            use = near | (window_np(dx, dy, rho, circle) if fwhm > 0 else False)
            w = np.where(use, psf_np(dx, dy, pitch, fwhm, kind, beta) if fwhm > 0 else 1.0, 0.0)
            out[:, j, i] = (field * w).sum(axis=(1, 2)) / w.sum()
    return out


@pytest.mark.parametrize("os_,circle,kind", [(3, False, 0), (3, True, 0), (4, False, 0), (4, True, 1), (2, True, 0)])
def test_centre_sampling_matches_brute_force(os_, circle, kind):
    g = gal(5, 4, os_, 2.4, CENTRE | (CIRCLE if circle else 0), kind=kind)
    H, W = g.padded_shape
    field = np.random.default_rng(11).normal(size=(4, H, W))
    out = oracle.convolve_bin(g, field)
    np.testing.assert_allclose(out, centre_reference(g, field, 2.4, circle, kind), rtol=1e-12, atol=1e-14)


def test_centre_sampling_odd_os_is_the_convolution_at_the_centre_point():
    g = gal(6, 5, 5, 2.0, CENTRE)
    H, W = g.padded_shape
    field = np.random.default_rng(2).normal(size=(4, H, W))
    out = oracle.convolve_bin(g, field)
    k = kernel_np(g, 2.0, False)
    h, o = g.h, (g.os - 1) // 2
    for c in range(4):
        conv = ndimage.correlate(field[c], k, mode="constant", cval=0.0)
        ref = conv[h + o:h + o + g.os * g.ny:g.os, h + o:h + o + g.os * g.nx:g.os]
        np.testing.assert_allclose(out[c], ref, rtol=1e-12, atol=1e-14)


def test_centre_sampling_special_cases():
    # os = 1: the centre is the sub-point, so centre sampling and binning agree
    for mode in (0, CIRCLE):
        a, b = gal(6, 5, 1, 3.0, mode), gal(6, 5, 1, 3.0, mode | CENTRE)
        H, W = a.padded_shape
        field = np.random.default_rng(4).normal(size=(4, H, W))
        np.testing.assert_allclose(oracle.convolve_bin(b, field), oracle.convolve_bin(a, field), rtol=1e-13,
                                   atol=1e-15)
    # no PSF: odd os samples the centre point, even os averages the four central points
    g3 = gal(4, 3, 3, 0.0, CENTRE)
    f3 = np.random.default_rng(6).normal(size=(4,) + g3.padded_shape)
    np.testing.assert_allclose(oracle.convolve_bin(g3, f3), f3[:, 1::3, 1::3], rtol=1e-15)
    g4 = gal(4, 3, 4, 0.0, CENTRE)
    f4 = np.random.default_rng(7).normal(size=(4,) + g4.padded_shape)
    ref = 0.25 * (f4[:, 1::4, 1::4] + f4[:, 2::4, 1::4] + f4[:, 1::4, 2::4] + f4[:, 2::4, 2::4])
    np.testing.assert_allclose(oracle.convolve_bin(g4, f4), ref, rtol=1e-13)


def flux_reference(g0, g_mode, theta, n_discs=1):
    """The flux-weighted maps rebuilt in numpy from the default mode's point values
    (B, v, sigma, <L/M>): convolve B, B v, B (sigma^2 + v^2) and B / <L/M>, then form
    v = C1/C0 + v_sys, sigma = sqrt(C2/C0 - (C1/C0)^2), M/L = C3/C0."""
    f = oracle.fine_field(g0, theta, n_discs=n_discs)
    B, v, s, lm = f
    ch = np.stack([B, B * v, B * (s * s + v * v), B / lm])
    C = oracle.convolve_bin(g_mode, ch)
    vv = C[1] / C[0]
    return np.stack([C[0], vv + theta[14], np.sqrt(C[2] / C[0] - vv * vv), C[3] / C[0]])


@pytest.mark.parametrize("mode", [FLUX, FLUX | CIRCLE, FLUX | CENTRE | CIRCLE])
def test_flux_weighted_maps_match_numpy_pipeline(mode):
    box = synth.prior_box(1)
    th = synth.draw_theta_true(box, 31)
    g0 = gal(6, 5, 3, 2.5, 0)
    gm = gal(6, 5, 3, 2.5, mode)
    got = oracle.maps(gm, th)
    ref = flux_reference(g0, gal(6, 5, 3, 2.5, mode & ~FLUX), th)
    np.testing.assert_allclose(got, ref, rtol=1e-11, atol=1e-9)


def test_flux_weighting_without_mixing_changes_nothing():
    box = synth.prior_box(2)
    th = synth.draw_theta_true(box, 8)
    a = oracle.maps(gal(5, 4, 1, 0.0, 0), th, n_discs=2)
    b = oracle.maps(gal(5, 4, 1, 0.0, FLUX), th, n_discs=2)
    np.testing.assert_allclose(b, a, rtol=1e-11)


def test_flux_weighted_dispersion_exceeds_the_light_weighted_mean_dispersion():
    """Beam smearing: with flux weighting the unresolved velocity gradient adds to sigma, so
    sigma_obs^2 >= conv(B sigma^2) / conv(B) point by point (Cauchy-Schwarz)."""
    box = synth.prior_box(1)
    th = synth.draw_theta_true(box, 12)
    g0, gf = gal(6, 6, 3, 2.5, 0), gal(6, 6, 3, 2.5, FLUX)
    B, v, s, _ = oracle.fine_field(g0, th)
    C = oracle.convolve_bin(g0, np.stack([B, B * s * s, B, B]))
    got = oracle.maps(gf, th)
    assert np.all(got[2] ** 2 >= C[1] / C[0] * (1 - 1e-12))


def test_gradient_of_the_combined_modes_matches_finite_differences():
    box = synth.prior_box(1, gamma_fixed=None)
    th = synth.draw_theta_true(box, 21)
    g0 = gal(5, 4, 2, 2.0, 0)
    true = oracle.maps(gal(5, 4, 2, 2.0, 7), th)
    data, err, _ = synth.noisy_data(true, seed=3)
    g = gal(5, 4, 2, 2.0, 7, data=data.astype(np.float64), err=err.astype(np.float64))
    th2 = th + 0.01 * (box[:, 1] - box[:, 0]) * np.random.default_rng(1).normal(size=th.size)
    th2 = np.clip(th2, box[:, 0], box[:, 1])
    logL, grad = oracle.loglike_grad(g, th2[None, :])
    step = 1e-4 * np.maximum(box[:, 1] - box[:, 0], 1e-3)
    for p in range(th.size):
        def L(x):
            t = th2.copy()
            t[p] = x
            return oracle.loglike(g, t[None, :])[0][0]
        h = step[p]
        d1 = (L(th2[p] + h) - L(th2[p] - h)) / (2 * h)
        d2 = (L(th2[p] + 2 * h) - L(th2[p] - 2 * h)) / (4 * h)
        fd = (4 * d1 - d2) / 3
        assert abs(grad[0, p] - fd) <= 1e-6 * np.abs(grad[0]).max() + 1e-7 * abs(fd), (p, grad[0, p], fd)
    del g0

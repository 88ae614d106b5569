"""The closed-form bulge option (bulge_kind 1 = Hernquist, 2 = Jaffe): the oracle's profile
(the radial rule at gamma = 1 or 2, which the bulge pins tie to the paper's closed forms,
Eqs. 4-6 and B4-B5; below R/a = 1e-3 the closed forms themselves, pinned here against
60-digit mpmath), the generated float32 fits of bulge_fit.h against it, and the oracle's
handling of the option (gamma fixed, its theta slot unused)."""
import math
import os
import re

import numpy as np
import pytest

import oracle
from paper_2205_06819_gb300 import synth

HDR = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "paper_2205_06819_gb300", "csrc",
                   "bulge_fit.h")


def load_fit():
    txt = open(HDR).read()
    T0 = int(re.search(r"#define BANG_BULGE_FIT_T0 (-?\d+)", txt).group(1))
    N = int(re.search(r"#define BANG_BULGE_FIT_N (\d+)", txt).group(1))
    DEG = int(re.search(r"#define BANG_BULGE_FIT_DEG (\d+)", txt).group(1))
    num = r"(-?\d\.\d+e[-+]\d+)f"
    sc = txt[txt.index("kBulgeFitScale[2]"):txt.index("kBulgeFitC[2]")]
    co = txt[txt.index("kBulgeFitC[2]"):]
    scale = np.array([float(x) for x in re.findall(num, sc)]).reshape(2, 2, N)
    C = np.array([float(x) for x in re.findall(num, co)]).reshape(2, 2, N, DEG + 1)
    return T0, N, scale, C


def fit_eval(kind, f, s):
    T0, N, scale, C = load_fit()
    t = math.log2(s) - T0
    k = min(max(int(math.floor(t)), 0), N - 1)
    u = t - k
    return scale[kind - 1, f, k] * 2.0 ** np.polynomial.polynomial.polyval(u, C[kind - 1, f, k])


def mp_closed(kind, s):
    """(F_S, F_Q) of the paper's closed forms (Eqs. 4-6 for kind 1, B4-B5 for kind 2) at 60
    digits: Sigma a^2 / M and Sigma sigma_p^2 a^3 / (G M^2)."""
    mpmath = pytest.importorskip("mpmath")
    mpmath.mp.dps = 60
    s = mpmath.mpf(s)
    q = 1 - s * s
    X = mpmath.acosh(1 / s) / mpmath.sqrt(q) if s < 1 else mpmath.acos(1 / s) / mpmath.sqrt(-q)
    if kind == 1:
        FS = ((2 + s * s) * X - 3) / (2 * mpmath.pi * q * q)
        br = ((-3 * s * s * X * (8 * s**6 - 28 * s**4 + 35 * s * s - 20) - 24 * s**6 + 68 * s**4 - 65 * s * s + 6)
              / (2 * q**3) - 6 * mpmath.pi * s)
        return float(FS), float(br / (12 * mpmath.pi))
    FS = 1 / (4 * s) + (1 - (2 - s * s) * X) / (2 * mpmath.pi * q)
    br = (mpmath.pi / (2 * s) + 11 - 6.5 * mpmath.pi * s - 12 * s * s + 6 * mpmath.pi * s**3
          - X * (6 - 19 * s * s + 12 * s**4))
    return float(FS), float(br / (4 * mpmath.pi * q))


def oracle_F(kind, s, a=0.8, M=4.0e10):
    Sig, s2 = oracle.bulge_model(s * a, a, float(kind), M, 128, bulge_kind=kind)
    return Sig * a * a / M, Sig * s2 * a ** 3 / (oracle.G() * M * M)


@pytest.mark.parametrize("kind", [1, 2])
def test_oracle_small_radius_branch_is_the_closed_form(kind):
    """Below R/a = 1e-3 the oracle evaluates the closed forms (float64); 60-digit mpmath
    restatements of the same equations agree.  Just above, the radial rule agrees with them
    too, so the switch is seamless."""
    for s in np.geomspace(1e-8, 9.9e-4, 15):
        fs, fq = oracle_F(kind, s)
        rs, rq = mp_closed(kind, s)
        assert abs(fs / rs - 1) < 1e-12 and abs(fq / rq - 1) < 1e-10
    for s in (1.01e-3, 2e-3):
        fs, fq = oracle_F(kind, s)
        rs, rq = mp_closed(kind, s)
        assert abs(fs / rs - 1) < 1e-8 and abs(fq / rq - 1) < 1e-8


@pytest.mark.parametrize("kind", [1, 2])
def test_fit_matches_oracle_model(kind):
    worst = 0.0
    for s in np.geomspace(1e-7, 3e3, 71):
        fs, fq = oracle_F(kind, s)
        worst = max(worst, abs(fit_eval(kind, 0, s) / fs - 1), abs(fit_eval(kind, 1, s) / fq - 1))
    assert worst < 1e-6


def test_bulge_kind_fixes_gamma_and_drops_its_slot():
    spec = synth.GalaxySpec(7, 6, 2, 2.0)
    box = synth.prior_box(1)
    th = synth.draw_theta_true(box, 9)
    g = oracle.Galaxy(spec.nx, spec.ny, spec.oversample, spec.psf_fwhm_arcsec, spec.kpc_per_arcsec)
    true = oracle.maps(g, th)
    data, err, _ = synth.noisy_data(true, seed=2)
    gd = oracle.Galaxy(spec.nx, spec.ny, spec.oversample, spec.psf_fwhm_arcsec, spec.kpc_per_arcsec,
                       data=data.astype(np.float64), err=err.astype(np.float64))
    for kind in (1, 2):
        ref = th.copy()
        ref[6] = float(kind)
        odd = th.copy()
        odd[6] = -4.0                        # outside the Dehnen domain: ignored with a fixed kind
        l0, g0 = oracle.loglike_grad(gd, ref[None, :])
        l1, g1 = oracle.loglike_grad(gd, odd[None, :], bulge_kind=kind)
        assert l1[0] == l0[0]
        assert g1[0, 6] == 0.0
        np.testing.assert_array_equal(np.delete(g1[0], 6), np.delete(g0[0], 6))
    assert not np.isfinite(oracle.loglike(gd, odd[None, :])[0][0])   # the Dehnen model refuses it

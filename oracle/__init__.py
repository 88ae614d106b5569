"""FP64 CPU oracle for the galaxy-model log-likelihood (Rigamonti et al. 2022).

TEST INFRASTRUCTURE ONLY.  The test suite, the smoke check and the CPU-baseline leg of
``bench.py`` are the only code allowed to import this package; the CUDA library never
calls it and shares no code with it.  ``bang_oracle.cpp`` holds the arithmetic; this
module only compiles it (g++, OpenMP) and marshals numpy arrays through ctypes.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "bang_oracle.cpp")
_LIB_PATH = os.path.join(_HERE, "libbang_oracle.so")
_lock = threading.Lock()
_lib = None

P_SINGLE_DISC = 15
P_TWO_DISCS = 19


def build(force: bool = False) -> str:
    """Compile the oracle into ``oracle/libbang_oracle.so`` (skipped when up to date)."""
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["g++", "-std=c++17", "-O2", "-fopenmp", "-fPIC", "-shared", "-o", tmp, _SRC]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class _Galaxy(ctypes.Structure):
    _fields_ = [
        ("nx", ctypes.c_int), ("ny", ctypes.c_int), ("oversample", ctypes.c_int),
        ("spaxel_arcsec", ctypes.c_double), ("kpc_per_arcsec", ctypes.c_double),
        ("psf_kind", ctypes.c_int), ("psf_fwhm_arcsec", ctypes.c_double), ("moffat_beta", ctypes.c_double),
        ("data", ctypes.POINTER(ctypes.c_double)), ("err", ctypes.POINTER(ctypes.c_double)),
        ("mask", ctypes.POINTER(ctypes.c_uint8)), ("psf_mode", ctypes.c_int),
    ]


class _Opts(ctypes.Structure):
    _fields_ = [("n_discs", ctypes.c_int), ("n_quad", ctypes.c_int), ("halo_kind", ctypes.c_int),
                ("bulge_kind", ctypes.c_int)]


_D = ctypes.POINTER(ctypes.c_double)


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_LIB_PATH)
            G, O = ctypes.POINTER(_Galaxy), ctypes.POINTER(_Opts)
            sig = {
                "bang_oracle_max_threads": (ctypes.c_int, []),
                "bang_oracle_nparams": (ctypes.c_int, [ctypes.c_int]),
                "bang_oracle_psf_halfwidth": (ctypes.c_int, [G]),
                "bang_oracle_psf_weights": (ctypes.c_int, [G, _D]),
                "bang_oracle_gauss_legendre": (None, [ctypes.c_int, _D, _D]),
                "bang_oracle_bulge_projected": (None, [ctypes.c_double] * 4 + [ctypes.c_int, _D, _D]),
                "bang_oracle_bulge_model": (None, [ctypes.c_double] * 4 + [ctypes.c_int, ctypes.c_int, _D, _D]),
                "bang_oracle_bulge_vc2": (ctypes.c_double, [ctypes.c_double] * 4),
                "bang_oracle_dehnen_rho": (ctypes.c_double, [ctypes.c_double] * 4),
                "bang_oracle_dehnen_mass": (ctypes.c_double, [ctypes.c_double] * 4),
                "bang_oracle_nfw_vc2": (ctypes.c_double, [ctypes.c_double] * 3),
                "bang_oracle_hernquist_halo_vc2": (ctypes.c_double, [ctypes.c_double] * 3),
                "bang_oracle_nfw_r200": (ctypes.c_double, [ctypes.c_double]),
                "bang_oracle_freeman_vc2": (ctypes.c_double, [ctypes.c_double] * 3),
                "bang_oracle_bessel_diff": (ctypes.c_double, [ctypes.c_double]),
                "bang_oracle_G": (ctypes.c_double, []),
                "bang_oracle_rho_crit": (ctypes.c_double, []),
                "bang_oracle_points": (ctypes.c_int, [O, _D, _D, _D, ctypes.c_int, ctypes.c_double, _D]),
                "bang_oracle_fine_field": (ctypes.c_int, [G, O, _D, _D, ctypes.c_int]),
                "bang_oracle_convolve_bin": (ctypes.c_int, [G, _D, _D, ctypes.c_int]),
                "bang_oracle_maps": (ctypes.c_int, [G, O, _D, _D, ctypes.c_int]),
                "bang_oracle_norm_const": (ctypes.c_double, [G]),
                "bang_oracle_loglike": (ctypes.c_int, [G, O, _D, ctypes.c_int, _D, _D, ctypes.c_int]),
                "bang_oracle_loglike_grad": (ctypes.c_int, [G, O, _D, ctypes.c_int, _D, _D, ctypes.c_int]),
            }
            for name, (res, args) in sig.items():
                fn = getattr(lib, name)
                fn.restype = res
                fn.argtypes = args
            _lib = lib
    return _lib


def _dptr(a: np.ndarray):
    return a.ctypes.data_as(_D)


class Galaxy:
    """One observed galaxy: spaxel grid, PSF and (optionally) data, errors and mask.

    ``data``/``err``/``mask`` are [4, ny, nx] (B, v, sigma, M/L); they are kept as
    float64 copies alive for as long as the object lives.
    """

    def __init__(self, nx, ny, oversample, psf_fwhm_arcsec, kpc_per_arcsec,
                 spaxel_arcsec=1.0, psf_kind=0, moffat_beta=3.0, data=None, err=None, mask=None, psf_mode=0):
        self.nx, self.ny, self.os = int(nx), int(ny), int(oversample)
        self.data = None if data is None else np.ascontiguousarray(data, dtype=np.float64).reshape(4, ny, nx)
        self.err = None if err is None else np.ascontiguousarray(err, dtype=np.float64).reshape(4, ny, nx)
        self.mask = None if mask is None else np.ascontiguousarray(mask, dtype=np.uint8).reshape(4, ny, nx)
        self._c = _Galaxy(self.nx, self.ny, self.os, float(spaxel_arcsec), float(kpc_per_arcsec),
                          int(psf_kind), float(psf_fwhm_arcsec), float(moffat_beta),
                          None if self.data is None else _dptr(self.data),
                          None if self.err is None else _dptr(self.err),
                          None if self.mask is None else self.mask.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8)),
                          int(psf_mode))
        self.psf_mode = int(psf_mode)
        self.h = _load().bang_oracle_psf_halfwidth(ctypes.byref(self._c))

    @property
    def padded_shape(self):
        return (self.os * self.ny + 2 * self.h, self.os * self.nx + 2 * self.h)


def _opts(n_discs, n_quad, halo_kind=0, bulge_kind=0):
    return _Opts(int(n_discs), int(n_quad), int(halo_kind), int(bulge_kind))


def nparams(n_discs: int) -> int:
    return P_TWO_DISCS if n_discs == 2 else P_SINGLE_DISC


def max_threads() -> int:
    return _load().bang_oracle_max_threads()


def gauss_legendre(n: int):
    x = np.zeros(n); w = np.zeros(n)
    _load().bang_oracle_gauss_legendre(n, _dptr(x), _dptr(w))
    return x, w


def psf_weights(gal: Galaxy) -> np.ndarray:
    n = 2 * gal.h + 1
    w = np.zeros(n * n)
    _load().bang_oracle_psf_weights(ctypes.byref(gal._c), _dptr(w))
    return w.reshape(n, n)


def bulge_projected(R, a, gamma, M, n_quad=64):
    s = ctypes.c_double(); s2 = ctypes.c_double()
    _load().bang_oracle_bulge_projected(float(R), float(a), float(gamma), float(M), int(n_quad),
                                        ctypes.byref(s), ctypes.byref(s2))
    return s.value, s2.value


def bulge_model(R, a, gamma, M, n_quad=64, bulge_kind=0):
    """(Sigma, sigma^2) as the model uses them: the radial rule, or for bulge_kind 1
    (Hernquist) / 2 (Jaffe) the paper's closed forms below R / a = 1e-3."""
    s, s2 = ctypes.c_double(), ctypes.c_double()
    _load().bang_oracle_bulge_model(float(R), float(a), float(gamma), float(M), int(n_quad), int(bulge_kind),
                                    ctypes.byref(s), ctypes.byref(s2))
    return s.value, s2.value


def bulge_vc2(r, a, gamma, M):
    return _load().bang_oracle_bulge_vc2(float(r), float(a), float(gamma), float(M))


def dehnen_rho(r, a, gamma, M):
    return _load().bang_oracle_dehnen_rho(float(r), float(a), float(gamma), float(M))


def dehnen_mass(r, a, gamma, M):
    return _load().bang_oracle_dehnen_mass(float(r), float(a), float(gamma), float(M))


def nfw_vc2(r, M200, c):
    return _load().bang_oracle_nfw_vc2(float(r), float(M200), float(c))


def hernquist_halo_vc2(r, Mh, Rh):
    return _load().bang_oracle_hernquist_halo_vc2(float(r), float(Mh), float(Rh))


def nfw_r200(M200):
    return _load().bang_oracle_nfw_r200(float(M200))


def freeman_vc2(r, Md, Rd):
    return _load().bang_oracle_freeman_vc2(float(r), float(Md), float(Rd))


def bessel_diff(y):
    return _load().bang_oracle_bessel_diff(float(y))


def G() -> float:
    return _load().bang_oracle_G()


def rho_crit() -> float:
    return _load().bang_oracle_rho_crit()


def points(theta, xs, ys, kpc_per_arcsec, n_discs=1, n_quad=64, halo_kind=0, bulge_kind=0):
    """Unconvolved observables [4, n] (B, v_los, sigma_los, <L/M>) at sky points (arcsec)."""
    th = np.ascontiguousarray(theta, dtype=np.float64)
    xs = np.ascontiguousarray(xs, dtype=np.float64).ravel()
    ys = np.ascontiguousarray(ys, dtype=np.float64).ravel()
    out = np.zeros((4, xs.size))
    o = _opts(n_discs, n_quad, halo_kind, bulge_kind)
    rc = _load().bang_oracle_points(ctypes.byref(o), _dptr(th), _dptr(xs), _dptr(ys), xs.size,
                                    float(kpc_per_arcsec), _dptr(out))
    if rc:
        raise ValueError("theta outside the parameter domain")
    return out


def fine_field(gal: Galaxy, theta, n_discs=1, n_quad=64, nthreads=0, halo_kind=0, bulge_kind=0):
    th = np.ascontiguousarray(theta, dtype=np.float64)
    H, W = gal.padded_shape
    out = np.zeros((4, H, W))
    o = _opts(n_discs, n_quad, halo_kind, bulge_kind)
    rc = _load().bang_oracle_fine_field(ctypes.byref(gal._c), ctypes.byref(o), _dptr(th), _dptr(out), nthreads)
    if rc:
        raise ValueError("theta outside the parameter domain")
    return out


def convolve_bin(gal: Galaxy, field, nthreads=0):
    f = np.ascontiguousarray(field, dtype=np.float64)
    H, W = gal.padded_shape
    assert f.shape == (4, H, W), (f.shape, (4, H, W))
    out = np.zeros((4, gal.ny, gal.nx))
    _load().bang_oracle_convolve_bin(ctypes.byref(gal._c), _dptr(f), _dptr(out), nthreads)
    return out


def maps(gal: Galaxy, theta, n_discs=1, n_quad=64, nthreads=0, halo_kind=0, bulge_kind=0):
    """Model maps [4, ny, nx]: B, v_los + v_sys, sigma_los, M/L."""
    th = np.ascontiguousarray(theta, dtype=np.float64)
    out = np.zeros((4, gal.ny, gal.nx))
    o = _opts(n_discs, n_quad, halo_kind, bulge_kind)
    rc = _load().bang_oracle_maps(ctypes.byref(gal._c), ctypes.byref(o), _dptr(th), _dptr(out), nthreads)
    if rc:
        raise ValueError("theta outside the parameter domain")
    return out


def norm_const(gal: Galaxy) -> float:
    return _load().bang_oracle_norm_const(ctypes.byref(gal._c))


def loglike(gal: Galaxy, theta, n_discs=1, n_quad=64, nthreads=0, halo_kind=0, bulge_kind=0):
    """(logL[B], chi2[B]) for theta[B, P]."""
    th = np.ascontiguousarray(np.atleast_2d(theta), dtype=np.float64)
    B = th.shape[0]
    assert th.shape[1] == nparams(n_discs)
    if gal.data is None or gal.err is None:
        raise ValueError("galaxy has no data")
    logL = np.zeros(B); chi2 = np.zeros(B)
    o = _opts(n_discs, n_quad, halo_kind, bulge_kind)
    _load().bang_oracle_loglike(ctypes.byref(gal._c), ctypes.byref(o), _dptr(th), B, _dptr(logL), _dptr(chi2),
                                nthreads)
    return logL, chi2


def loglike_grad(gal: Galaxy, theta, n_discs=1, n_quad=64, nthreads=0, halo_kind=0, bulge_kind=0):
    """(logL[B], grad[B, P]) with grad = d logL / d theta (forward-mode duals)."""
    th = np.ascontiguousarray(np.atleast_2d(theta), dtype=np.float64)
    B, P = th.shape
    assert P == nparams(n_discs)
    if gal.data is None or gal.err is None:
        raise ValueError("galaxy has no data")
    logL = np.zeros(B); grad = np.zeros((B, P))
    o = _opts(n_discs, n_quad, halo_kind, bulge_kind)
    _load().bang_oracle_loglike_grad(ctypes.byref(gal._c), ctypes.byref(o), _dptr(th), B, _dptr(logL),
                                     _dptr(grad), nthreads)
    return logL, grad

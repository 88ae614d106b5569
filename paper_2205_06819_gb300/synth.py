"""Seeded synthetic inputs: workload shapes, parameter draws, data noise.

This module holds no arithmetic of the galaxy model.  It fixes the five workloads
(spaxel grids, oversampling, PSF, quadrature nodes, batch sizes), draws parameter
vectors from the prior box, and turns noise-free model maps (computed elsewhere) into
noisy data with the error model of Sec. 3.1 (5% on B, 10 km/s on v, 15 km/s on sigma;
10% on M/L, a value the paper does not state).  Both the CUDA tests and the oracle
tests take their inputs from here, so they see the same bytes.

Parameter layout (angles in radians, masses and radii as log10 of Msun and kpc):
  0 x0, 1 y0 [kpc], 2 PA, 3 i, 4 log Mb, 5 log Rb, 6 gamma, 7 log Md1, 8 log Rd1, 9 k1,
  10 (M/L)b, 11 (M/L)d1, 12 log M200, 13 c, 14 v_sys [km/s],
  15 log Md2, 16 log Rd2, 17 k2, 18 (M/L)d2 (two-disc models only).
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

#: NGC 7683 at ~53 Mpc (Sec. 3.1): kpc per arcsec = D * pi / 648000.
KPC_PER_ARCSEC = 53000.0 * math.pi / 648000.0

PARAM_NAMES_1 = ["x0", "y0", "PA", "inc", "logMb", "logRb", "gamma", "logMd1", "logRd1", "k1",
                 "MLb", "MLd1", "logM200", "c", "vsys"]
PARAM_NAMES_2 = PARAM_NAMES_1 + ["logMd2", "logRd2", "k2", "MLd2"]

DEG = math.pi / 180.0


def prior_box(n_discs: int, gamma_fixed: float | None = None, halo_kind: int = 0) -> np.ndarray:
    """[P, 2] lower/upper bounds of the uniform prior box.

    Inclination 30-70 deg, bulge scale 0.5-2 kpc, disc scale 2-5 kpc, log bulge/disc mass
    9-11 and concentration 5-15 follow the workload text; P.A., k, M/L and halo mass follow
    the priors of the paper's fit table; centre and systemic velocity are chosen here.
    """
    box = [
        (-0.25, 0.25), (-0.25, 0.25),                 # x0, y0 [kpc]
        (-math.pi, math.pi),                          # PA
        (30 * DEG, 70 * DEG),                         # i
        (9.0, 11.0), (math.log10(0.5), math.log10(2.0)),   # log Mb, log Rb
        (0.0, 2.0),                                   # gamma
        (9.0, 11.0), (math.log10(2.0), math.log10(5.0)),   # log Md1, log Rd1
        (0.0, 1.0),                                   # k1
        (1.0, 100.0), (0.1, 100.0),                   # (M/L)b, (M/L)d1
        (11.5, 14.5), (5.0, 15.0),                    # log M200, c
        (-50.0, 50.0),                                # v_sys [km/s]
    ]
    if n_discs == 2:
        box += [(9.0, 11.0), (math.log10(2.0), math.log10(5.0)), (0.0, 1.0), (0.1, 100.0)]
    b = np.array(box, dtype=np.float64)
    if halo_kind == 1:                               # Hernquist halo: slot 13 = log10 R_h, prior [1, 3]
        b[13] = (1.0, 3.0)
    if gamma_fixed is not None:
        b[6] = (gamma_fixed, gamma_fixed)
    return b


def clip_to_box(theta: np.ndarray, box: np.ndarray) -> np.ndarray:
    lo, hi = box[:, 0], box[:, 1]
    return np.clip(theta, lo, hi)


@dataclasses.dataclass
class GalaxySpec:
    nx: int
    ny: int
    oversample: int
    psf_fwhm_arcsec: float
    psf_kind: int = 0            # 0 Gaussian, 1 Moffat
    moffat_beta: float = 3.0
    spaxel_arcsec: float = 1.0
    kpc_per_arcsec: float = KPC_PER_ARCSEC


@dataclasses.dataclass
class Workload:
    name: str
    galaxies: list            # [GalaxySpec]
    rows_per_galaxy: int      # parameter vectors per galaxy
    n_discs: int
    n_quad: int
    gamma_fixed: float | None
    grad: bool
    description: str

    @property
    def nparams(self) -> int:
        return 19 if self.n_discs == 2 else 15

    @property
    def batch(self) -> int:
        return self.rows_per_galaxy * len(self.galaxies)


def _uneven_galaxies(seed: int, n: int = 64):
    rng = np.random.Generator(np.random.PCG64(seed))
    grids = [(32, 32), (48, 64), (78, 73), (96, 96), (128, 128)]
    out = []
    for _ in range(n):
        nx, ny = grids[int(rng.integers(len(grids)))]
        out.append(GalaxySpec(nx, ny, 4, float(rng.uniform(1.5, 3.5))))
    return out


def workload(name: str) -> Workload:
    """The five workloads by name: single, batched, adjoint, uneven, largest."""
    if name == "single":
        return Workload(name, [GalaxySpec(30, 30, 3, 2.5)], 1, 1, 64, 1.0, False,
                        "30x30 spaxels, 3x3 oversampling, Gaussian PSF 2.5\", Hernquist-limit bulge, "
                        "one disc, NFW halo, 1 parameter vector")
    if name == "batched":
        return Workload(name, [GalaxySpec(80, 80, 5, 2.5)], 1024, 1, 64, None, False,
                        "80x80 spaxels, 5x5 oversampling, Gaussian PSF 2.5\", 1024 parameter vectors")
    if name == "adjoint":
        return Workload(name, [GalaxySpec(80, 80, 5, 2.5)], 256, 1, 64, None, True,
                        "80x80 spaxels, 5x5 oversampling, logL and gradient for 256 parameter vectors")
    if name == "uneven":
        return Workload(name, _uneven_galaxies(1004), 64, 1, 64, None, False,
                        "64 galaxies with grids from {32x32, 48x64, 78x73, 96x96, 128x128}, 4x4 "
                        "oversampling, PSF FWHM U[1.5,3.5]\", 64 parameter vectors each")
    if name == "largest":
        return Workload(name, [GalaxySpec(128, 128, 7, 2.5, psf_kind=1, moffat_beta=3.0)], 4096, 2, 128, None, True,
                        "128x128 spaxels, 7x7 oversampling, Moffat PSF beta=3 FWHM 2.5\", two discs, "
                        "128 quadrature nodes, 4096 parameter vectors")
    raise KeyError(name)


WORKLOADS = ["single", "batched", "adjoint", "uneven", "largest"]


def _rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


def draw_theta_true(box: np.ndarray, seed: int) -> np.ndarray:
    """One parameter vector uniform in the prior box; the inner disc gets the smaller scale."""
    rng = _rng(seed)
    th = rng.uniform(box[:, 0], box[:, 1])
    if th.size == 19 and th[16] < th[8]:
        th[[7, 8, 9, 11]], th[[15, 16, 17, 18]] = th[[15, 16, 17, 18]].copy(), th[[7, 8, 9, 11]].copy()
    return th


def draw_theta_batch(box: np.ndarray, theta_true: np.ndarray, B: int, seed: int,
                     posterior_frac: float = 0.5, width: float = 0.01) -> np.ndarray:
    """[B, P]: a ``posterior_frac`` share near theta_true (Gaussian, ``width`` x prior range,
    clipped into the box), the rest uniform in the box."""
    rng = _rng(seed)
    P = box.shape[0]
    n_post = int(round(B * posterior_frac))
    span = box[:, 1] - box[:, 0]
    post = theta_true[None, :] + rng.normal(size=(n_post, P)) * (width * span)[None, :]
    post = clip_to_box(post, box)
    uni = rng.uniform(box[:, 0], box[:, 1], size=(B - n_post, P))
    out = np.concatenate([post, uni], axis=0)
    return np.ascontiguousarray(out)


#: absolute/relative error model per map: B 5%, v 10 km/s, sigma 15 km/s, M/L 10%
ERR_REL_B = 0.05
ERR_V = 10.0
ERR_SIGMA = 15.0
ERR_REL_ML = 0.10


def error_maps(true_maps: np.ndarray) -> np.ndarray:
    """Per-spaxel errors [4, ny, nx] from noise-free maps (B, v, sigma, M/L)."""
    t = np.asarray(true_maps, dtype=np.float64)
    err = np.empty_like(t)
    err[0] = ERR_REL_B * np.abs(t[0])
    err[1] = ERR_V
    err[2] = ERR_SIGMA
    err[3] = ERR_REL_ML * np.abs(t[3])
    return err


def noisy_data(true_maps: np.ndarray, seed: int, noise: bool = True):
    """(data, err, mask) as float32/float32/uint8 [4, ny, nx]; data = true + err * N(0, 1)."""
    t = np.asarray(true_maps, dtype=np.float64)
    err = error_maps(t)
    data = t.copy()
    if noise:
        data += err * _rng(seed).normal(size=t.shape)
    mask = np.ones(t.shape, dtype=np.uint8)
    return data.astype(np.float32), err.astype(np.float32), mask


def dataset_seed(workload_id: int, galaxy: int = 0) -> int:
    """Seed of galaxy g's data for workload id (1-5): (1000 + id) * 100 + g."""
    return (1000 + workload_id) * 100 + galaxy


def batch_seed(workload_id: int) -> int:
    return 2000 + workload_id


def workload_id(name: str) -> int:
    return WORKLOADS.index(name) + 1


#: Posterior medians of the NGC 7683 fit (Sec. 3.1, fit table; sin i = 0.829 -> i), with
#: the paper's Hernquist halo replaced by an NFW halo of similar mass.  A realistic,
#: two-disc parameter vector for tests.
NGC7683_LIKE = np.array([
    -1.031 + 1.0, -1.054 + 1.0,          # centre, shifted near the field centre
    44.12 * DEG, math.asin(0.829),
    10.67, -0.65, 1.0,
    10.42, -0.015, 0.299,
    10.5, 2.12,
    12.5, 10.0, 0.0,
    10.865, 0.603, 0.700, 2.62,
])

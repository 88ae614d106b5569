"""Test datasets: seeded draws from paper_2205_06819_gb300.synth, noise-free maps from the
oracle, noisy float32 data.  The CUDA path and the oracle read the same float32 bytes."""
import numpy as np

import oracle
from paper_2205_06819_gb300 import synth


class Dataset:
    def __init__(self, spec: synth.GalaxySpec, theta_true, n_discs=1, n_quad=64, seed=1, noise=True, mask=None,
                 halo_kind=0, psf_mode=0, bulge_kind=0):
        self.spec, self.n_discs, self.n_quad, self.halo_kind = spec, n_discs, n_quad, halo_kind
        self.psf_mode, self.bulge_kind = psf_mode, bulge_kind
        self.theta_true = np.asarray(theta_true, dtype=np.float64)
        g0 = self.oracle_galaxy(None, None, None)
        true = oracle.maps(g0, self.theta_true, n_discs=n_discs, n_quad=n_quad, halo_kind=halo_kind,
                           bulge_kind=bulge_kind)
        self.data, self.err, m = synth.noisy_data(true, seed=seed, noise=noise)
        self.mask = m if mask is None else np.asarray(mask, dtype=np.uint8)
        self.og = self.oracle_galaxy(self.data.astype(np.float64), self.err.astype(np.float64), self.mask)

    def oracle_galaxy(self, data, err, mask):
        s = self.spec
        return oracle.Galaxy(s.nx, s.ny, s.oversample, s.psf_fwhm_arcsec, s.kpc_per_arcsec,
                             spaxel_arcsec=s.spaxel_arcsec, psf_kind=s.psf_kind, moffat_beta=s.moffat_beta,
                             data=data, err=err, mask=mask, psf_mode=self.psf_mode)

    def model_galaxy(self):
        from paper_2205_06819_gb300.model import Galaxy
        s = self.spec
        return Galaxy(s.nx, s.ny, s.oversample, s.psf_fwhm_arcsec, s.kpc_per_arcsec, self.data, self.err, self.mask,
                      spaxel_arcsec=s.spaxel_arcsec, psf_kind=s.psf_kind, moffat_beta=s.moffat_beta)

    def oracle_loglike(self, theta32, nthreads=0):
        th = np.asarray(theta32, dtype=np.float32).astype(np.float64)
        return oracle.loglike(self.og, th, n_discs=self.n_discs, n_quad=self.n_quad, nthreads=nthreads,
                              halo_kind=self.halo_kind, bulge_kind=self.bulge_kind)

    def oracle_maps(self, theta32):
        th = np.asarray(theta32, dtype=np.float32).astype(np.float64)
        return oracle.maps(self.og, th, n_discs=self.n_discs, n_quad=self.n_quad, halo_kind=self.halo_kind,
                           bulge_kind=self.bulge_kind)


def theta_batch(n_discs, theta_true, B, seed, gamma_fixed=None, halo_kind=0):
    box = synth.prior_box(n_discs, gamma_fixed, halo_kind)
    return synth.draw_theta_batch(box, np.asarray(theta_true), B, seed).astype(np.float32)


#: gradient bar, per row: every component within GRAD_ABS x the oracle gradient's Euclidean
#: norm, and every component of at least GRAD_COMPONENT_FLOOR x the norm within GRAD_RTOL
#: of its own size (and the whole vector within GRAD_RTOL of the norm).  The float32
#: gradient carries an absolute error floor in every component, set by the rounding of the
#: sums over the field; a component that happens to be small (near a zero crossing in theta)
#: has that same absolute error, so a relative bar is meaningful only well above the floor.
#: Measured over every gradient row of the GPU tests (163 rows): at most 3.0e-5 of the norm
#: (a centre-offset slot), and at most 5.9e-5 relative for components of 5% of the norm or
#: more (3.7e-4 already at 1%).
GRAD_RTOL = 1e-4
GRAD_ABS = 5e-5
GRAD_COMPONENT_FLOOR = 0.05


def grad_errors(got, ref):
    """Per row: (largest component error over the norm of ref, largest relative error of the
    components with |ref_p| >= GRAD_COMPONENT_FLOOR x that norm)."""
    got = np.atleast_2d(np.asarray(got, np.float64))
    ref = np.atleast_2d(np.asarray(ref, np.float64))
    out = []
    for g, r in zip(got, ref):
        nrm = np.linalg.norm(r)
        err = np.abs(g - r)
        big = np.abs(r) >= GRAD_COMPONENT_FLOOR * nrm
        out.append((float(err.max() / nrm), float((err[big] / np.abs(r[big])).max()) if big.any() else 0.0))
    return out


def assert_grad_close(got, ref, label=""):
    """The gradient bar of every GPU gradient test (see GRAD_RTOL)."""
    got = np.atleast_2d(np.asarray(got, np.float64))
    ref = np.atleast_2d(np.asarray(ref, np.float64))
    for b, (e_abs, e_rel) in enumerate(grad_errors(got, ref)):
        nrm = np.linalg.norm(ref[b])
        assert np.linalg.norm(got[b] - ref[b]) <= GRAD_RTOL * nrm, (label, b, e_abs)
        with np.errstate(divide="ignore", invalid="ignore"):
            rel = np.abs(got[b] - ref[b]) / np.abs(ref[b])
        assert e_abs <= GRAD_ABS, (label, b, "component over norm", np.abs(got[b] - ref[b]) / nrm)
        assert e_rel <= GRAD_RTOL, (label, b, "large component", rel, np.abs(ref[b]) / nrm)

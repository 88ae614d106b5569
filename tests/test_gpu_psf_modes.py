"""GPU parity of the PSF modes (psf_mode bits: circular 3-sigma window of Eq. 21, App. A's
centre sampling, flux-weighted moments) against the FP64 oracle in the same mode: logL
(chi^2 within 1e-5), gradient (1e-4 of its norm), maps, the plain per-task form and the
radial-table option; odd and even oversampling, Gaussian and Moffat, with and without a
PSF."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2205_06819_gb300 import synth  # noqa: E402

from bang_testdata import Dataset, assert_grad_close, theta_batch  # noqa: E402

CHI2_RTOL = 1e-5
GRAD_RTOL = 1e-4

CASES = {
    # name: (GalaxySpec, psf_mode, n_discs)
    "circle_os3": (synth.GalaxySpec(19, 15, 3, 2.6), 1, 1),
    "centre_os4": (synth.GalaxySpec(17, 13, 4, 2.2), 2, 1),
    "circle_centre_moffat": (synth.GalaxySpec(17, 13, 3, 2.4, psf_kind=1, moffat_beta=2.5), 3, 1),
    "flux_os3": (synth.GalaxySpec(19, 15, 3, 2.6), 4, 1),
    "all_two_discs_os2": (synth.GalaxySpec(16, 14, 2, 2.0), 7, 2),
    "centre_flux_os1": (synth.GalaxySpec(18, 16, 1, 3.0), 6, 1),
    "centre_flux_no_psf_os4": (synth.GalaxySpec(12, 10, 4, 0.0), 6, 1),
}


@pytest.fixture(scope="module")
def lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import oracle
    from paper_2205_06819_gb300 import build as b
    oracle.build()
    b.build()
    from paper_2205_06819_gb300.model import Model
    return Model


def make(name):
    spec, mode, nd = CASES[name]
    box = synth.prior_box(nd)
    th = synth.draw_theta_true(box, 500 + len(name))
    ds = Dataset(spec, th, n_discs=nd, seed=600 + len(name), psf_mode=mode)
    theta = theta_batch(nd, th, 6, seed=700 + len(name))
    return ds, theta, mode, nd


def chi2(ds, logL):
    import oracle
    return -2.0 * (np.asarray(logL, dtype=np.float64) + oracle.norm_const(ds.og))


@pytest.mark.parametrize("name", list(CASES))
def test_logl_and_gradient(lib, name):
    import oracle
    ds, theta, mode, nd = make(name)
    m = lib(ds.model_galaxy(), n_discs=nd, psf_mode=mode)
    t = torch.from_numpy(theta).cuda()
    got = m.loglike(t).cpu().numpy()
    _, ref_chi = ds.oracle_loglike(theta)
    assert (np.abs(chi2(ds, got) - ref_chi) / ref_chi).max() < CHI2_RTOL, name
    lg, g = m.loglike_grad(t)
    np.testing.assert_allclose(lg.cpu().numpy(), got, rtol=1e-6)
    g = g.cpu().numpy()
    _, gref = oracle.loglike_grad(ds.og, theta.astype(np.float64), n_discs=nd)
    for k in range(theta.shape[0]):
        assert_grad_close(g[k], gref[k], (name, k))


@pytest.mark.parametrize("name", ["circle_os3", "centre_os4", "flux_os3", "all_two_discs_os2"])
def test_maps_and_plain_form(lib, name):
    ds, theta, mode, nd = make(name)
    m = lib(ds.model_galaxy(), n_discs=nd, psf_mode=mode)
    t = torch.from_numpy(theta[:2]).cuda()
    maps = [x.cpu().numpy() for x in m.maps(t)]
    for b in range(2):
        ref = ds.oracle_maps(theta[b])
        for c in (0, 2, 3):
            np.testing.assert_allclose(maps[b][c], ref[c], rtol=3e-5)
        np.testing.assert_allclose(maps[b][1], ref[1], atol=3e-5 * np.abs(ref[1]).max())
    np.testing.assert_allclose(m.loglike_plain(t).cpu().numpy(), m.loglike(t).cpu().numpy(), rtol=CHI2_RTOL)


def test_radial_table_in_the_combined_mode(lib):
    ds, theta, mode, nd = make("all_two_discs_os2")
    m = lib(ds.model_galaxy(), n_discs=nd, psf_mode=mode, bulge_table=1024)
    got = m.loglike(torch.from_numpy(theta).cuda()).cpu().numpy()
    _, ref_chi = ds.oracle_loglike(theta)
    assert (np.abs(chi2(ds, got) - ref_chi) / ref_chi).max() < CHI2_RTOL


def test_modes_change_the_likelihood_and_bad_mode_is_refused(lib):
    """The modes are different models: on the same data the logL differ; psf_mode 8 is not
    a mode."""
    ds, theta, _, nd = make("circle_os3")
    t = torch.from_numpy(theta).cuda()
    vals = {mode: lib(ds.model_galaxy(), n_discs=nd, psf_mode=mode).loglike(t).cpu().numpy() for mode in (0, 1, 2, 4)}
    for a in vals:
        for b in vals:
            if a < b:
                assert np.abs(vals[a] - vals[b]).max() > 1e-6 * np.abs(vals[a]).max(), (a, b)
    with pytest.raises(Exception):
        lib(ds.model_galaxy(), n_discs=nd, psf_mode=8)

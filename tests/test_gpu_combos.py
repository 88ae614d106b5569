"""Model options together: an uneven batch of galaxies with different grids and PSFs under
the Jaffe closed-form bulge, the Hernquist halo and the flux-weighted circular PSF; and one
galaxy on two spaxel grids with the closed-form Hernquist bulge.  logL and gradient against
the FP64 oracle with the same options (chi^2 within 1e-5, gradient 1e-4 of its norm)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2205_06819_gb300 import synth  # noqa: E402

from bang_testdata import Dataset, assert_grad_close, theta_batch  # noqa: E402

CHI2_RTOL = 1e-5
GRAD_RTOL = 1e-4


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


def test_uneven_batch_with_all_options(lib):
    import oracle
    opts = dict(bulge_kind=2, halo_kind=1, psf_mode=5)
    box = synth.prior_box(1, halo_kind=1)
    specs = [synth.GalaxySpec(14, 12, 3, 2.0), synth.GalaxySpec(20, 16, 2, 2.8), synth.GalaxySpec(11, 17, 4, 1.6)]
    dss, thetas = [], []
    for g, spec in enumerate(specs):
        th = synth.draw_theta_true(box, 300 + g)
        dss.append(Dataset(spec, th, seed=310 + g, halo_kind=1, psf_mode=5, bulge_kind=2))
        thetas.append(theta_batch(1, th, 5, seed=320 + g, halo_kind=1))
    m = lib([d.model_galaxy() for d in dss], **opts)
    theta = np.concatenate(thetas)
    gi = np.repeat(np.arange(3, dtype=np.int32), 5)
    t = torch.from_numpy(theta).cuda()
    logL, grad = m.loglike_grad(t, gi)
    logL, grad = logL.cpu().numpy(), grad.cpu().numpy()
    for g, d in enumerate(dss):
        rows = slice(5 * g, 5 * g + 5)
        _, chi_ref = d.oracle_loglike(theta[rows])
        chi = -2.0 * (logL[rows] + oracle.norm_const(d.og))
        assert (np.abs(chi - chi_ref) / chi_ref).max() < CHI2_RTOL, g
        _, gref = oracle.loglike_grad(d.og, theta[rows].astype(np.float64), halo_kind=1, bulge_kind=2)
        for k in range(5):
            assert_grad_close(grad[5 * g + k], gref[k], (g, k))
    np.testing.assert_allclose(m.loglike(t, gi).cpu().numpy(), logL, rtol=1e-6)


def test_grids_with_the_closed_form_bulge(lib):
    import oracle
    box = synth.prior_box(1)
    th = synth.draw_theta_true(box, 401)
    grids = [(synth.GalaxySpec(24, 20, 2, 1.5, spaxel_arcsec=0.5), (0,)),
             (synth.GalaxySpec(12, 10, 3, 2.5, spaxel_arcsec=1.0), (1, 2, 3))]
    dss = []
    for k, (spec, chans) in enumerate(grids):
        mask = np.zeros((4, spec.ny, spec.nx), np.uint8)
        mask[list(chans)] = 1
        dss.append(Dataset(spec, th, seed=410 + k, mask=mask, bulge_kind=1))
    m = lib([d.model_galaxy() for d in dss], bulge_kind=1)
    theta = theta_batch(1, th, 6, seed=420)
    logL, grad = m.loglike_grids(torch.from_numpy(theta).cuda(), [0, 1], grad=True)
    chi_ref = sum(d.oracle_loglike(theta)[1] for d in dss)
    norm = sum(oracle.norm_const(d.og) for d in dss)
    chi = -2.0 * (logL.cpu().numpy() + norm)
    assert (np.abs(chi - chi_ref) / chi_ref).max() < CHI2_RTOL
    gref = sum(oracle.loglike_grad(d.og, theta.astype(np.float64), bulge_kind=1)[1] for d in dss)
    g = grad.cpu().numpy()
    assert np.all(g[:, 6] == 0.0)
    for k in range(6):
        assert_grad_close(g[k], gref[k], k)

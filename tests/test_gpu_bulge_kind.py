"""GPU parity of the closed-form bulges (bulge_kind 1 = Hernquist, Eqs. 1-6; 2 = Jaffe,
Eqs. B1-B5) against the FP64 oracle with the same option: logL (chi^2 within 1e-5),
gradient (1e-4 of its norm, the gamma slot exactly 0), maps, the plain form; the gamma slot
is ignored; the option refuses the radial table."""
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


def make(kind, nd, spec):
    box = synth.prior_box(nd)
    th = synth.draw_theta_true(box, 40 + 10 * kind + nd)
    ds = Dataset(spec, th, n_discs=nd, seed=50 + 10 * kind + nd, bulge_kind=kind)
    theta = theta_batch(nd, th, 6, seed=60 + 10 * kind + nd)
    theta[:, 6] = np.linspace(-3.0, 7.0, theta.shape[0])   # the gamma slot is not used
    return ds, theta


def chi2(ds, logL):
    import oracle
    return -2.0 * (np.asarray(logL, dtype=np.float64) + oracle.norm_const(ds.og))


@pytest.mark.parametrize("kind,nd,spec", [
    (1, 1, synth.GalaxySpec(21, 17, 3, 2.5)),
    (2, 1, synth.GalaxySpec(19, 15, 4, 2.2)),
    (1, 2, synth.GalaxySpec(16, 14, 3, 2.4, psf_kind=1, moffat_beta=3.0)),
    (2, 2, synth.GalaxySpec(18, 12, 2, 0.0)),
])
def test_logl_gradient_maps_plain(lib, kind, nd, spec):
    import oracle
    ds, theta = make(kind, nd, spec)
    m = lib(ds.model_galaxy(), n_discs=nd, bulge_kind=kind)
    t = torch.from_numpy(theta).cuda()
    got = m.loglike(t).cpu().numpy()
    assert np.all(np.isfinite(got))
    _, ref_chi = ds.oracle_loglike(theta)
    assert (np.abs(chi2(ds, got) - ref_chi) / ref_chi).max() < CHI2_RTOL
    _, g = m.loglike_grad(t)
    g = g.cpu().numpy()
    _, gref = oracle.loglike_grad(ds.og, theta.astype(np.float32).astype(np.float64), n_discs=nd, bulge_kind=kind)
    assert np.all(g[:, 6] == 0.0)
    for k in range(theta.shape[0]):
        assert_grad_close(g[k], gref[k], k)
    maps = [x.cpu().numpy() for x in m.maps(t[:2])]
    for b in range(2):
        ref = ds.oracle_maps(theta[b])
        for c in (0, 2, 3):
            np.testing.assert_allclose(maps[b][c], ref[c], rtol=2e-5)
        np.testing.assert_allclose(maps[b][1], ref[1], atol=2e-5 * np.abs(ref[1]).max())
    np.testing.assert_allclose(m.loglike_plain(t).cpu().numpy(), got, rtol=CHI2_RTOL)


def test_closed_form_equals_dehnen_at_fixed_gamma_and_refuses_table(lib):
    """At gamma = 1 the Dehnen model (radial rule) and the closed-form Hernquist bulge give
    the same logL to the fits' accuracy; bulge_kind with bulge_table is refused."""
    ds, theta = make(1, 1, synth.GalaxySpec(21, 17, 3, 2.5))
    t0 = theta.copy()
    t0[:, 6] = 1.0
    a = lib(ds.model_galaxy(), n_discs=1).loglike(torch.from_numpy(t0).cuda()).cpu().numpy()
    b = lib(ds.model_galaxy(), n_discs=1, bulge_kind=1).loglike(torch.from_numpy(theta).cuda()).cpu().numpy()
    assert (np.abs(chi2(ds, a) - chi2(ds, b)) / chi2(ds, a)).max() < CHI2_RTOL
    with pytest.raises(Exception):
        lib(ds.model_galaxy(), n_discs=1, bulge_kind=1, bulge_table=1024)


def test_extreme_bulge_scales_stay_finite(lib):
    """Bulge scales far outside any prior (a = 1e-6 or 1e6 kpc) put s = R/a beyond the fitted
    range; the edge values hold, so logL and the gradient stay finite."""
    ds, theta = make(1, 1, synth.GalaxySpec(21, 17, 3, 2.5))
    m = lib(ds.model_galaxy(), n_discs=1, bulge_kind=1)
    th = theta[:4].copy()
    th[:, 5] = [-6.0, -4.0, 5.0, 6.0]
    t = torch.from_numpy(th).cuda()
    lg, g = m.loglike_grad(t)
    assert torch.isfinite(lg).all() and torch.isfinite(g).all()

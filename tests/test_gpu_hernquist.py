"""GPU parity with the paper's own halo (halo_kind = 1, Hernquist: theta slot 13 is
log10 R_h) in the paper's model layout: Hernquist bulge (gamma = 1), inner and outer
discs.  Forward, maps, gradient, radial-table option and the plain form against the
FP64 oracle at the usual bars (chi^2 1e-5, gradient 1e-4 of its norm)."""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2205_06819_gb300 import synth  # noqa: E402

from bang_testdata import Dataset, assert_grad_close, theta_batch  # noqa: E402

CHI2_RTOL = 1e-5
GRAD_RTOL = 1e-4


@pytest.fixture(scope="module")
def setup():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import oracle
    from paper_2205_06819_gb300 import build as b
    oracle.build()
    b.build()
    from paper_2205_06819_gb300.model import Model
    th = synth.NGC7683_LIKE.copy()
    th[13] = math.log10(30.0)                         # R_h = 30 kpc
    ds = Dataset(synth.GalaxySpec(21, 17, 3, 2.6), th, n_discs=2, seed=131, halo_kind=1)
    theta = theta_batch(2, th, 8, seed=132, gamma_fixed=1.0, halo_kind=1)
    return Model, ds, theta


def chi2(ds, logL):
    import oracle
    return -2.0 * (np.asarray(logL) + oracle.norm_const(ds.og))


@pytest.mark.parametrize("table", [0, 1024])
def test_hernquist_halo_logl_and_gradient(setup, table):
    import oracle
    Model, ds, theta = setup
    m = Model(ds.model_galaxy(), n_discs=2, halo_kind=1, bulge_table=table)
    t = torch.from_numpy(theta).cuda()
    got = m.loglike(t).cpu().numpy()
    _, ref_chi = ds.oracle_loglike(theta)
    assert (np.abs(chi2(ds, got) - ref_chi) / ref_chi).max() < CHI2_RTOL
    _, g = m.loglike_grad(t)
    g = g.cpu().numpy()
    _, gref = oracle.loglike_grad(ds.og, theta.astype(np.float64), n_discs=2, halo_kind=1)
    for k in range(theta.shape[0]):
        assert_grad_close(g[k], gref[k], k)


def test_hernquist_halo_maps_and_plain(setup):
    Model, ds, theta = setup
    m = Model(ds.model_galaxy(), n_discs=2, halo_kind=1)
    t = torch.from_numpy(theta[:3]).cuda()
    maps = [x.cpu().numpy() for x in m.maps(t)]
    for b in range(3):
        ref = ds.oracle_maps(theta[b])
        for c in (0, 2, 3):
            np.testing.assert_allclose(maps[b][c], ref[c], rtol=2e-5)
        np.testing.assert_allclose(maps[b][1], ref[1], atol=2e-5 * np.abs(ref[1]).max())
    np.testing.assert_allclose(m.loglike_plain(t).cpu().numpy(), m.loglike(t).cpu().numpy(), rtol=CHI2_RTOL)

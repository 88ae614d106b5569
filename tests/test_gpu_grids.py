"""One galaxy observed on several spaxel grids (bang_loglike_grids): B on a fine photometric
grid, v and sigma on a coarse kinematic grid, M/L on a third; each grid masked to its maps.
logL and gradient against the sum of the FP64 oracle over the grids (chi^2 within 1e-5,
gradient 1e-4 of its norm), agreement with the per-row batch call, host buffers, and
argument checks."""
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
    box = synth.prior_box(1)
    th = synth.draw_theta_true(box, 77)
    grids = [  # (spec, maps held)
        (synth.GalaxySpec(36, 30, 2, 1.5, spaxel_arcsec=0.5), (0,)),          # photometry
        (synth.GalaxySpec(18, 15, 3, 2.5, spaxel_arcsec=1.0), (1, 2)),        # kinematics
        (synth.GalaxySpec(12, 10, 2, 2.0, spaxel_arcsec=1.5), (3,)),          # M/L map
    ]
    dss = []
    for k, (spec, chans) in enumerate(grids):
        mask = np.zeros((4, spec.ny, spec.nx), np.uint8)
        mask[list(chans)] = 1
        dss.append(Dataset(spec, th, seed=800 + k, mask=mask))
    m = Model([d.model_galaxy() for d in dss], n_discs=1)
    theta = theta_batch(1, th, 7, seed=900)
    return m, dss, theta


def oracle_sums(dss, theta):
    import oracle
    chi = np.zeros(theta.shape[0])
    grad = np.zeros(theta.shape)
    norm = 0.0
    for d in dss:
        _, c = d.oracle_loglike(theta)
        chi += c
        _, g = oracle.loglike_grad(d.og, theta.astype(np.float64))
        grad += g
        norm += oracle.norm_const(d.og)
    return chi, grad, norm


def test_grids_match_the_oracle_sum(setup):
    m, dss, theta = setup
    t = torch.from_numpy(theta).cuda()
    logL, g = m.loglike_grids(t, [0, 1, 2], grad=True)
    chi_ref, g_ref, norm = oracle_sums(dss, theta)
    chi = -2.0 * (logL.cpu().numpy() + norm)
    assert (np.abs(chi - chi_ref) / chi_ref).max() < CHI2_RTOL
    g = g.cpu().numpy()
    for k in range(theta.shape[0]):
        assert_grad_close(g[k], g_ref[k], k)
    np.testing.assert_allclose(m.loglike_grids(t, [0, 1, 2]).cpu().numpy(), logL.cpu().numpy(), rtol=1e-6)


def test_grids_equal_the_per_row_batch_and_host_buffers(setup):
    m, _, theta = setup
    t = torch.from_numpy(theta).cuda()
    B = theta.shape[0]
    rows = t.repeat_interleave(3, dim=0).contiguous()
    gi = np.tile(np.arange(3, dtype=np.int32), B)
    per_row = m.loglike(rows, gi).cpu().numpy().reshape(B, 3).sum(axis=1)
    dev = m.loglike_grids(t, [0, 1, 2]).cpu().numpy()
    np.testing.assert_allclose(dev, per_row, rtol=1e-12)
    host = m.loglike_grids(torch.from_numpy(theta), [0, 1, 2]).numpy()
    np.testing.assert_array_equal(host, dev)
    # one grid alone is the plain batch call
    np.testing.assert_allclose(m.loglike_grids(t, [1]).cpu().numpy(),
                               m.loglike(t, np.full(B, 1, np.int32)).cpu().numpy(), rtol=1e-12)


def test_grids_argument_checks(setup):
    m, _, theta = setup
    t = torch.from_numpy(theta).cuda()
    with pytest.raises(Exception):
        m.loglike_grids(t, [0, 3])
    with pytest.raises(Exception):
        m.loglike_grids(t, [])

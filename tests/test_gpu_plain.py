"""GPU parity of the plain one-kernel-per-task form (the paper's Alg. 2 execution form),
through the C ABI: against the FP64 oracle (chi-square within 1e-5 relative) and against
the fused batched kernel."""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2205_06819_gb300 import synth  # noqa: E402

from bang_testdata import Dataset, theta_batch  # noqa: E402

CHI2_RTOL = 1e-5
TH1 = np.array([0.05, -0.08, 0.4, 0.95, 10.2, math.log10(0.9), 1.3, 10.4, math.log10(2.8), 0.55,
                3.5, 2.0, 12.4, 9.0, 15.0])
TH2 = np.concatenate([TH1, [10.1, math.log10(4.0), 0.8, 2.5]])


@pytest.fixture(scope="module")
def Model():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import oracle
    from paper_2205_06819_gb300 import build as b
    oracle.build()
    b.build()
    from paper_2205_06819_gb300.model import Model
    return Model


@pytest.mark.parametrize("kind", ["gauss", "moffat2"])
def test_plain_matches_oracle_and_fused(Model, kind):
    import oracle
    if kind == "gauss":
        ds = Dataset(synth.GalaxySpec(19, 13, 3, 2.4), TH1, seed=81)
        theta = theta_batch(1, TH1, 8, seed=82)
    else:
        ds = Dataset(synth.GalaxySpec(11, 12, 3, 2.5, psf_kind=1), TH2, n_discs=2, n_quad=128, seed=83)
        theta = theta_batch(2, TH2, 5, seed=84)
    theta[2, 9] = 2.0 if kind == "gauss" else theta[2, 9]      # out-of-domain row in the first case
    m = Model(ds.model_galaxy(), n_discs=ds.n_discs, n_quad=ds.n_quad)
    t = torch.from_numpy(theta).cuda()
    plain = m.loglike_plain(t).cpu().numpy()
    fused = m.loglike(t).cpu().numpy()
    ref, chi_ref = ds.oracle_loglike(theta)
    fin = np.isfinite(ref)
    assert np.array_equal(fin, np.isfinite(plain))
    chi = -2 * (plain + oracle.norm_const(ds.og))
    assert (np.abs(chi[fin] - chi_ref[fin]) / chi_ref[fin]).max() < CHI2_RTOL
    np.testing.assert_allclose(plain[fin], fused[fin], rtol=CHI2_RTOL)


def test_plain_uneven_batch(Model):
    specs = [synth.GalaxySpec(9, 7, 2, 1.5), synth.GalaxySpec(13, 10, 2, 2.8)]
    dss = [Dataset(s, TH1, seed=85 + k) for k, s in enumerate(specs)]
    theta = theta_batch(1, TH1, 6, seed=87)
    gal_idx = np.array([1, 0, 0, 1, 1, 0], np.int32)
    m = Model([d.model_galaxy() for d in dss])
    t = torch.from_numpy(theta).cuda()
    np.testing.assert_allclose(m.loglike_plain(t, gal_idx).cpu().numpy(), m.loglike(t, gal_idx).cpu().numpy(),
                               rtol=CHI2_RTOL)

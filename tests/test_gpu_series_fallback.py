"""The upper-node series of the radial rule and its fallback, on the GPU against the oracle.

Points with w (cosh t_K - 1) below the series' threshold (within ~0.2 bulge scales of the
bulge centre) sum every radial node one by one; the others take the series.  A bulge scale
of 8 kpc on a fine grid puts hundreds of fine points on the explicit side and warps that
mix both paths; a scale of 0.2 kpc puts almost every point on the series side.  For both,
over gamma from 0 to 2.9, the forward chi^2 and maps and the adjoint gradient must match
the float64 oracle (which sums every node) at the bars of the other GPU tests; with 128
nodes as well (its own split).
"""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2205_06819_gb300 import synth  # noqa: E402

from bang_testdata import Dataset, assert_grad_close, theta_batch  # noqa: E402

CHI2_RTOL = 1e-5
MAP_RTOL = 2e-5
TH1 = np.array([0.05, -0.08, 0.4, 0.95, 10.2, math.log10(0.9), 1.3, 10.4, math.log10(2.8), 0.55,
                3.5, 2.0, 12.4, 9.0, 15.0])


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


@pytest.mark.parametrize("scale_kpc,n_quad", [(8.0, 64), (0.2, 64), (8.0, 128)])
def test_series_and_fallback_match_the_oracle(Model, scale_kpc, n_quad):
    import oracle
    th = TH1.copy()
    th[5] = math.log10(scale_kpc)
    th[4] = 10.6
    ds = Dataset(synth.GalaxySpec(21, 17, 6, 2.0), th, n_quad=n_quad, seed=131)
    rows = []
    for g in (0.0, 0.7, 1.5, 2.2, 2.9):
        r = th.copy()
        r[6] = g
        rows.append(r)
    theta = np.concatenate([np.array(rows), theta_batch(1, th, 3, seed=132)]).astype(np.float32)
    theta[:, 5] = math.log10(scale_kpc)                     # keep the scale in every row
    m = Model(ds.model_galaxy(), n_quad=n_quad)
    t = torch.from_numpy(theta).cuda()
    logL = m.loglike(t).cpu().numpy()
    _, ref_chi2 = ds.oracle_loglike(theta)
    chi = -2.0 * (logL + oracle.norm_const(ds.og))
    assert (np.abs(chi - ref_chi2) / ref_chi2).max() < CHI2_RTOL
    maps = m.maps(t)
    for b in range(theta.shape[0]):
        got, ref = maps[b].cpu().numpy(), ds.oracle_maps(theta[b])
        for c in (0, 2, 3):
            np.testing.assert_allclose(got[c], ref[c], rtol=MAP_RTOL, atol=0)
        np.testing.assert_allclose(got[1], ref[1], rtol=0, atol=MAP_RTOL * np.abs(ref[1]).max())
    _, g = m.loglike_grad(t)
    _, gref = oracle.loglike_grad(ds.og, theta.astype(np.float64), n_quad=n_quad)
    assert_grad_close(g.cpu().numpy(), gref, (scale_kpc, n_quad))
    m.close()

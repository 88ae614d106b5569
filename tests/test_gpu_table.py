"""GPU parity of the radial-table option (bulge_table): the bulge's projected density and
dispersion from a per-row table of the same radial quadrature, interpolated in log R.
Against the FP64 oracle, which evaluates the quadrature at every fine point: chi^2 within
1e-5 relative and the gradient within 1e-4 of its norm, the same bars as the default
mode; and against the default mode of the library itself."""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2205_06819_gb300 import synth  # noqa: E402

from bang_testdata import Dataset, assert_grad_close, theta_batch  # noqa: E402

CHI2_RTOL = 1e-5
GRAD_RTOL = 1e-4
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


def chi2(ds, logL):
    import oracle
    return -2.0 * (np.asarray(logL) + oracle.norm_const(ds.og))


def check(Model, ds, theta, T=1024, grad=False):
    import oracle
    m = Model(ds.model_galaxy(), n_discs=ds.n_discs, n_quad=ds.n_quad, bulge_table=T)
    t = torch.from_numpy(theta).cuda()
    got = m.loglike(t).cpu().numpy()
    ref, ref_chi = ds.oracle_loglike(theta)
    fin = np.isfinite(ref)
    assert np.array_equal(fin, np.isfinite(got))
    assert (np.abs(chi2(ds, got)[fin] - ref_chi[fin]) / ref_chi[fin]).max() < CHI2_RTOL
    exact = Model(ds.model_galaxy(), n_discs=ds.n_discs, n_quad=ds.n_quad).loglike(t).cpu().numpy()
    np.testing.assert_allclose(got[fin], exact[fin], rtol=1e-6)
    if grad:
        lg, g = m.loglike_grad(t)
        # the gradient call tabulates through the derivative-carrying node loop, which rounds
        # differently in float32: same bar as against the default mode
        np.testing.assert_allclose(lg.cpu().numpy()[fin], got[fin], rtol=1e-6)
        g = g.cpu().numpy()
        th = theta[fin].astype(np.float64)
        _, gref = oracle.loglike_grad(ds.og, th, n_discs=ds.n_discs, n_quad=ds.n_quad)
        assert_grad_close(g[fin], gref, "table")
        assert np.all(g[~fin] == 0)


def test_table_ragged_grid_logl_and_gradient(Model):
    ds = Dataset(synth.GalaxySpec(19, 14, 3, 2.4), TH1, seed=101)
    check(Model, ds, theta_batch(1, TH1, 10, seed=102), grad=True)


@pytest.mark.parametrize("T", [256, 512])
def test_table_sizes(Model, T):
    ds = Dataset(synth.GalaxySpec(13, 11, 3, 2.0), TH1, seed=103)
    check(Model, ds, theta_batch(1, TH1, 6, seed=104), T=T)


def test_table_moffat_two_discs_128_nodes(Model):
    ds = Dataset(synth.GalaxySpec(12, 10, 3, 2.5, psf_kind=1), TH2, n_discs=2, n_quad=128, seed=105)
    check(Model, ds, theta_batch(2, TH2, 5, seed=106), grad=True)


def test_table_edge_parameters_and_domain(Model):
    ds = Dataset(synth.GalaxySpec(15, 12, 3, 2.0), TH1, seed=107)
    rows = np.repeat(TH1[None], 8, 0).astype(np.float32)
    rows[0, 6] = 0.0
    rows[1, 6] = 2.95
    rows[2, 9] = 1.0
    rows[3, 3] = 0.0
    rows[4, [0, 1]] = 0.0
    rows[5, 5] = -1.5         # compact bulge, a = 0.03 kpc
    rows[6, 5] = 1.2          # extended bulge, a = 16 kpc
    rows[7, 13] = -1.0        # out of domain
    check(Model, ds, rows, grad=True)


def test_table_uneven_batch(Model):
    specs = [synth.GalaxySpec(8, 8, 4, 1.6), synth.GalaxySpec(14, 12, 4, 3.1)]
    dss = [Dataset(s, TH1, seed=108 + k) for k, s in enumerate(specs)]
    theta = theta_batch(1, TH1, 8, seed=110)
    gal_idx = np.array([0, 1] * 4, np.int32)
    m = Model([d.model_galaxy() for d in dss], bulge_table=1024)
    got = m.loglike(torch.from_numpy(theta).cuda(), gal_idx).cpu().numpy()
    for k, ds in enumerate(dss):
        sel = gal_idx == k
        _, rc = ds.oracle_loglike(theta[sel])
        assert (np.abs(chi2(ds, got[sel]) - rc) / rc).max() < CHI2_RTOL


def test_plain_and_noalloc_refuse_the_table_mode(Model):
    import ctypes
    from paper_2205_06819_gb300 import _lib
    ds = Dataset(synth.GalaxySpec(6, 5, 2, 1.5), TH1, seed=111)
    m = Model(ds.model_galaxy(), bulge_table=512)
    t = torch.from_numpy(theta_batch(1, TH1, 2, seed=112)).cuda()
    with pytest.raises(_lib.BangError):
        m.loglike_plain(t)
    out = torch.zeros(2, dtype=torch.float64, device="cuda")
    st = _lib.lib().bang_loglike_batch_noalloc(m.handle, ctypes.c_void_p(t.data_ptr()), None, 2,
                                               ctypes.c_void_p(out.data_ptr()), None)
    assert st == 4


def test_table_full_size_batched_sampled_rows(Model):
    wl = synth.workload("batched")
    wid = synth.workload_id("batched")
    box = synth.prior_box(1)
    tt = synth.draw_theta_true(box, synth.dataset_seed(wid))
    ds = Dataset(wl.galaxies[0], tt, seed=synth.dataset_seed(wid))
    theta = synth.draw_theta_batch(box, tt, wl.batch, synth.batch_seed(wid)).astype(np.float32)
    m = Model(ds.model_galaxy(), bulge_table=1024)
    got = m.loglike(torch.from_numpy(theta).cuda()).cpu().numpy()
    pick = np.array([0, 3, 600, 1023])
    _, rc = ds.oracle_loglike(theta[pick])
    assert (np.abs(chi2(ds, got[pick]) - rc) / rc).max() < CHI2_RTOL

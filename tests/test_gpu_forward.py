"""GPU parity of the fused forward kernel against the FP64 oracle, through the C ABI.

Tolerance (float32 compute, float64 chi-square accumulation): the chi-square of every
row within 1e-5 relative of the oracle's; maps element-wise within 2e-5 relative (B,
sigma, M/L) and 2e-5 of the map's largest |v| for the velocity.
"""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2205_06819_gb300 import synth  # noqa: E402

from bang_testdata import Dataset, theta_batch  # noqa: E402

CHI2_RTOL = 1e-5
MAP_RTOL = 2e-5

TH1 = np.array([0.05, -0.08, 0.4, 0.95, 10.2, math.log10(0.9), 1.3, 10.4, math.log10(2.8), 0.55,
                3.5, 2.0, 12.4, 9.0, 15.0])
TH2 = np.concatenate([TH1, [10.1, math.log10(4.0), 0.8, 2.5]])


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


def chi2_of(ds, logL):
    return -2.0 * (np.asarray(logL, dtype=np.float64) + __import__("oracle").norm_const(ds.og))


def check_rows(ds, Model, theta, nthreads=0):
    m = Model(ds.model_galaxy(), n_discs=ds.n_discs, n_quad=ds.n_quad)
    t = torch.from_numpy(theta).cuda()
    got = m.loglike(t).cpu().numpy()
    ref, ref_chi2 = ds.oracle_loglike(theta, nthreads=nthreads)
    fin = np.isfinite(ref)
    assert np.array_equal(fin, np.isfinite(got))
    chi = chi2_of(ds, got)
    rel = np.abs(chi[fin] - ref_chi2[fin]) / np.abs(ref_chi2[fin])
    assert rel.max() < CHI2_RTOL, (rel.max(), np.argmax(rel))
    m.close()
    return rel.max()


def test_ragged_multi_chunk_grid(lib):
    spec = synth.GalaxySpec(23, 17, 3, 2.5)            # h = 9, padded 87 x 69 fine points
    ds = Dataset(spec, TH1, seed=5)
    theta = theta_batch(1, TH1, 24, seed=6)
    check_rows(ds, lib, theta)


def test_maps_match_oracle_per_channel(lib):
    spec = synth.GalaxySpec(19, 14, 4, 2.0)
    ds = Dataset(spec, TH1, seed=7)
    theta = theta_batch(1, TH1, 6, seed=8)
    m = lib(ds.model_galaxy())
    got = [x.cpu().numpy() for x in m.maps(torch.from_numpy(theta).cuda())]
    for b in range(theta.shape[0]):
        ref = ds.oracle_maps(theta[b])
        for c in (0, 2, 3):
            np.testing.assert_allclose(got[b][c], ref[c], rtol=MAP_RTOL, atol=0)
        vs = np.abs(ref[1]).max()
        np.testing.assert_allclose(got[b][1], ref[1], rtol=0, atol=MAP_RTOL * vs)


def test_moffat_two_discs_128_nodes(lib):
    spec = synth.GalaxySpec(13, 11, 3, 2.5, psf_kind=1, moffat_beta=3.0)
    ds = Dataset(spec, TH2, n_discs=2, n_quad=128, seed=9)
    theta = theta_batch(2, TH2, 8, seed=10)
    check_rows(ds, lib, theta)


def test_no_psf_no_oversampling_and_single_spaxel(lib):
    for spec in (synth.GalaxySpec(9, 7, 1, 0.0), synth.GalaxySpec(1, 1, 2, 1.0), synth.GalaxySpec(5, 1, 3, 2.0)):
        ds = Dataset(spec, TH1, seed=11)
        check_rows(ds, lib, theta_batch(1, TH1, 4, seed=12))


def test_edge_parameters(lib):
    spec = synth.GalaxySpec(15, 12, 3, 2.0)
    ds = Dataset(spec, TH1, seed=13)
    rows = np.repeat(TH1[None], 7, 0).astype(np.float32)
    rows[0, 6] = 0.0          # cored bulge
    rows[1, 6] = 2.95         # nearly r^-3 cusp
    rows[2, 9] = 1.0          # cold disc
    rows[3, 9] = -1.0         # counter-rotating
    rows[4, 3] = 0.0          # face-on
    rows[5, 3] = 1.45         # nearly edge-on
    rows[6, [0, 1]] = 0.0     # centre exactly on the grid symmetry point
    check_rows(ds, lib, rows)


def test_out_of_domain_rows(lib):
    spec = synth.GalaxySpec(10, 8, 2, 1.5)
    ds = Dataset(spec, TH1, seed=14)
    rows = np.repeat(TH1[None], 6, 0).astype(np.float32)
    rows[1, 3] = 1.6
    rows[2, 6] = 3.0
    rows[3, 9] = 1.5
    rows[4, 13] = 0.0
    rows[5, 10] = np.nan
    m = lib(ds.model_galaxy())
    got = m.loglike(torch.from_numpy(rows).cuda()).cpu().numpy()
    assert np.isfinite(got[0]) and np.all(np.isneginf(got[1:]))
    single = m.loglike(torch.from_numpy(rows[:1]).cuda()).cpu().numpy()
    assert got[0] == pytest.approx(single[0], rel=1e-12)


def test_masked_spaxels(lib):
    spec = synth.GalaxySpec(12, 9, 2, 1.8)
    mask = np.ones((4, 9, 12), np.uint8)
    mask[0, :3, :] = 0
    mask[2, 4, 5] = 0
    mask[3, :, -2:] = 0
    ds = Dataset(spec, TH1, seed=15, mask=mask)
    check_rows(ds, lib, theta_batch(1, TH1, 6, seed=16))


def test_host_buffers_equal_device_buffers(lib):
    spec = synth.GalaxySpec(14, 10, 3, 2.2)
    ds = Dataset(spec, TH1, seed=17)
    theta = theta_batch(1, TH1, 9, seed=18)
    m = lib(ds.model_galaxy())
    dev = m.loglike(torch.from_numpy(theta).cuda()).cpu().numpy()
    host = m.loglike(torch.from_numpy(theta)).numpy()
    np.testing.assert_array_equal(dev, host)
    again = m.loglike(torch.from_numpy(theta).cuda()).cpu().numpy()   # graph replay
    np.testing.assert_array_equal(dev, again)


def test_uneven_batch_matches_oracle_and_single_galaxy_calls(lib):
    from paper_2205_06819_gb300.model import Model
    specs = [synth.GalaxySpec(8, 8, 4, 1.6), synth.GalaxySpec(12, 16, 4, 2.8), synth.GalaxySpec(20, 19, 4, 3.3)]
    dss = [Dataset(s, TH1, seed=20 + k) for k, s in enumerate(specs)]
    per = 5
    thetas = [theta_batch(1, TH1, per, seed=30 + k) for k in range(3)]
    gal_idx = np.array([k for k in range(3) for _ in range(per)], dtype=np.int32)
    perm = np.random.default_rng(0).permutation(gal_idx.size)
    theta_all = np.concatenate(thetas)[perm]
    gal_idx = gal_idx[perm]
    m = Model([d.model_galaxy() for d in dss])
    got = m.loglike(torch.from_numpy(theta_all).cuda(), gal_idx=gal_idx).cpu().numpy()
    for k, ds in enumerate(dss):
        sel = gal_idx == k
        ref, ref_chi2 = ds.oracle_loglike(theta_all[sel])
        chi = chi2_of(ds, got[sel])
        assert (np.abs(chi - ref_chi2) / ref_chi2).max() < CHI2_RTOL
        single = Model(ds.model_galaxy()).loglike(torch.from_numpy(theta_all[sel]).cuda()).cpu().numpy()
        np.testing.assert_allclose(got[sel], single, rtol=1e-12)


@pytest.mark.parametrize("name", ["batched"])
def test_full_size_workload_sampled_rows(lib, name):
    """The 80x80, 5x5-oversampled workload at its full size, in the bench's launch shape
    (1024 rows, one persistent launch), with a sample of rows checked against the oracle."""
    wl = synth.workload(name)
    wid = synth.workload_id(name)
    box = synth.prior_box(1)
    tt = synth.draw_theta_true(box, synth.dataset_seed(wid))
    ds = Dataset(wl.galaxies[0], tt, seed=synth.dataset_seed(wid))
    theta = synth.draw_theta_batch(box, tt, wl.batch, synth.batch_seed(wid)).astype(np.float32)
    m = lib(ds.model_galaxy())
    got = m.loglike(torch.from_numpy(theta).cuda()).cpu().numpy()
    pick = np.array([0, 1, 511, 512, 1023])
    ref, ref_chi2 = ds.oracle_loglike(theta[pick])
    chi = chi2_of(ds, got[pick])
    assert (np.abs(chi - ref_chi2) / ref_chi2).max() < CHI2_RTOL


def test_autotuner_keeps_results(lib):
    ds = Dataset(synth.GalaxySpec(16, 12, 3, 2.0), TH1, seed=19)
    theta = torch.from_numpy(theta_batch(1, TH1, 5, seed=20)).cuda()
    m = lib(ds.model_galaxy())
    before = m.loglike(theta).cpu().numpy()
    m.tune(5)
    after = m.loglike(theta).cpu().numpy()
    np.testing.assert_allclose(after, before, rtol=1e-12)
    l2, g2 = m.loglike_grad(theta)
    np.testing.assert_allclose(l2.cpu().numpy(), before, rtol=1e-12)


@pytest.mark.parametrize("kind", [0, 1])
def test_large_grid_wide_psf(lib, kind):
    """A large grid near the shared-memory limits: 150x110 spaxels, os 6, FWHM 3.5" (h = 26,
    padded rows of 952 fine points, 58-tap window), Gaussian and Moffat; sampled rows."""
    spec = synth.GalaxySpec(150, 110, 6, 3.5, psf_kind=kind)
    ds = Dataset(spec, TH1, seed=120 + kind)
    theta = theta_batch(1, TH1, 3, seed=122)
    check_rows(ds, lib, theta)


def test_large_batch_indexing(lib):
    """20000 rows in one launch (work-item table, per-row offsets) on a small grid; rows
    sampled across the batch against the oracle, and the batch equal to a split of it."""
    spec = synth.GalaxySpec(9, 8, 2, 1.6)
    ds = Dataset(spec, TH1, seed=123)
    theta = theta_batch(1, TH1, 20000, seed=124)
    m = lib(ds.model_galaxy())
    t = torch.from_numpy(theta).cuda()
    got = m.loglike(t).cpu().numpy()
    pick = np.array([0, 7777, 12345, 19999])
    ref, ref_chi2 = ds.oracle_loglike(theta[pick])
    chi = chi2_of(ds, got[pick])
    assert (np.abs(chi - ref_chi2) / ref_chi2).max() < CHI2_RTOL
    part = m.loglike(t[12000:12100]).cpu().numpy()
    np.testing.assert_allclose(part, got[12000:12100], rtol=1e-12)

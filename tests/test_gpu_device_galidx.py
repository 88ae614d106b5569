"""gal_idx in device memory: bang_loglike_batch and bang_loglike_grad_batch schedule the batch
on the device (work items derived from each row's galaxy by the kernels, longest first by a
device-side counting sort) without reading gal_idx on the host or synchronising the stream.

Checked through the C ABI: logL and the gradient equal the host-array path's bit for bit
(the two paths split rows into the same bands), on an uneven batch of three galaxies with a
row count that fills the GPU (one band per row) and one that does not (several bands); a
row whose galaxy index is out of range gets NaN and a zero gradient while the others are
unchanged; the call returns while the GPU is still busy with earlier work (no host
synchronisation); bang_model_maps, whose output packing depends on gal_idx, refuses it.
"""
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


@pytest.fixture(scope="module")
def setup():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import oracle
    from paper_2205_06819_gb300 import build as b
    oracle.build()
    b.build()
    from paper_2205_06819_gb300.model import Model
    specs = [synth.GalaxySpec(8, 8, 4, 1.6), synth.GalaxySpec(12, 16, 4, 2.8), synth.GalaxySpec(20, 19, 4, 3.3)]
    dss = [Dataset(s, TH1, seed=60 + k) for k, s in enumerate(specs)]
    m = Model([d.model_galaxy() for d in dss])
    return m, dss


def batch(B, seed):
    theta = theta_batch(1, TH1, B, seed=seed)
    gal = np.random.default_rng(seed).integers(0, 3, size=B).astype(np.int32)
    return theta, gal


@pytest.mark.parametrize("B", [200, 24])
def test_device_gal_idx_equals_host_path_bit_for_bit(setup, B):
    import oracle
    m, dss = setup
    theta_np, gal = batch(B, 70 + B)
    theta = torch.from_numpy(theta_np).cuda()
    gal_dev = torch.from_numpy(gal).cuda()
    host = m.loglike(theta, gal).cpu().numpy()
    dev = m.loglike(theta, gal_dev).cpu().numpy()
    np.testing.assert_array_equal(dev, host)
    lh, gh = m.loglike_grad(theta, gal)
    ld, gd = m.loglike_grad(theta, gal_dev)
    np.testing.assert_array_equal(ld.cpu().numpy(), lh.cpu().numpy())
    np.testing.assert_array_equal(gd.cpu().numpy(), gh.cpu().numpy())
    # and against the oracle: one row of each galaxy
    for k, ds in enumerate(dss):
        b = int(np.flatnonzero(gal == k)[0])
        ref, ref_chi2 = ds.oracle_loglike(theta_np[b:b + 1])
        chi = -2.0 * (dev[b] + oracle.norm_const(ds.og))
        assert abs(chi - ref_chi2[0]) / ref_chi2[0] < CHI2_RTOL


def test_device_gal_idx_out_of_range_rows(setup):
    m, dss = setup
    theta_np, gal = batch(40, 81)
    bad = gal.copy()
    bad[[3, 17]] = [-1, 3]                          # below and above [0, n_gal)
    theta = torch.from_numpy(theta_np).cuda()
    dev = m.loglike(theta, torch.from_numpy(bad).cuda()).cpu().numpy()
    ld, gd = m.loglike_grad(theta, torch.from_numpy(bad).cuda())
    assert np.isnan(dev[[3, 17]]).all() and np.isnan(ld.cpu().numpy()[[3, 17]]).all()
    assert (gd.cpu().numpy()[[3, 17]] == 0).all()
    keep = np.setdiff1d(np.arange(40), [3, 17])
    ref = m.loglike(theta[keep], gal[keep]).cpu().numpy()
    np.testing.assert_allclose(dev[keep], ref, rtol=1e-12)


def test_device_gal_idx_call_does_not_synchronise(setup):
    """With device theta, logL and gal_idx the call only enqueues work: queued behind a long
    sleep kernel on the same stream, it returns while the stream is still busy."""
    from paper_2205_06819_gb300 import _lib
    if _lib.lib().bang_checked_build():
        pytest.skip("the checked build synchronises every call to read its index-check records")
    m, dss = setup
    theta_np, gal = batch(64, 83)
    theta = torch.from_numpy(theta_np).cuda()
    gal_dev = torch.from_numpy(gal).cuda()
    out = torch.empty(64, dtype=torch.float64, device="cuda")
    m.loglike(theta, gal_dev, out=out)            # plan, graph and buffers made on the first call
    m.loglike_grad(theta, gal_dev)
    torch.cuda.synchronize()
    stream = torch.cuda.current_stream()
    torch.cuda._sleep(200_000_000)                # ~0.1 s of GPU clock cycles
    m.loglike(theta, gal_dev, out=out)
    busy = not stream.query()
    torch.cuda.synchronize()
    assert busy
    np.testing.assert_array_equal(out.cpu().numpy(), m.loglike(theta, gal).cpu().numpy())


def test_maps_refuse_a_device_gal_idx(setup):
    from paper_2205_06819_gb300 import _lib
    m, dss = setup
    theta_np, gal = batch(4, 85)
    theta = torch.from_numpy(theta_np).cuda()
    gal_dev = torch.from_numpy(gal).cuda()
    L = _lib.lib()
    import ctypes
    assert L.bang_model_maps_size(m.handle, ctypes.c_void_p(gal_dev.data_ptr()), 4) == -1
    out = torch.empty(4 * 4 * 20 * 19, dtype=torch.float32, device="cuda")
    st = L.bang_model_maps(m.handle, ctypes.c_void_p(theta.data_ptr()), ctypes.c_void_p(gal_dev.data_ptr()), 4,
                           ctypes.c_void_p(out.data_ptr()), None)
    assert st == 4                                  # BANG_E_UNSUPPORTED


def test_launch_info_reports_the_plan(setup):
    """bang_model_launch_info: the launch shape of a host-index and a device-index batch of the
    same rows (the same bands; the device plan's items derived on the device), and of the
    gradient call (its adjoint band height and work items)."""
    m, dss = setup
    theta_np, gal = batch(24, 87)
    h = m.launch_info(24, gal)
    d = m.launch_info(24, torch.from_numpy(gal).cuda())
    g = m.launch_info(24, gal, grad=True)
    assert h["device_items"] == 0 and d["device_items"] == 1
    assert h["bands"] == d["bands"] >= 1 and d["items"] == 24 * d["bands"]
    assert 1 <= h["grid"] <= h["items"] and h["blocks_per_sm"] >= 1 and h["rows_per_step"] >= 1
    assert h["adj_rows_per_item"] == 0 and g["adj_rows_per_item"] >= 1 and g["adj_items"] >= 24
    assert 1 <= g["adj_grid"] <= g["adj_items"]
    assert g["adj_blocks_per_sm"] in (3, 4) and h["adj_blocks_per_sm"] == 0
    assert h["column_lanes"] == 0 and g["column_lanes"] == 0   # untuned: one thread per spaxel column

"""The no-allocation entry point, bang_loglike_batch_noalloc, checked through the C ABI
against bang_loglike_batch and against the float64 oracle.

That entry point is for callers that must not allocate device memory while they run (a
program whose GPU memory belongs to another allocator, or a loop that cannot take the
synchronisation cudaMalloc may cause): its scratch is a fixed array in the library's
device code.  Two calls in a row, on different batches, must each give the logL of the
allocating entry point within the chi-square tolerance of the other GPU tests (1e-5
relative); so must a batch that mixes two galaxies of different grid sizes through a host
gal_idx array.  Its chi^2 must match the oracle's at the same tolerance, a call on a warm
device must leave the free device memory and the model's scratch exactly as they were,
and an oversized batch must be refused before anything is launched.
This file is named so that pytest collects it last.
"""
import ctypes
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

CHI2_RTOL = 1e-5
TH1 = np.array([0.05, -0.08, 0.4, 0.95, 10.2, math.log10(0.9), 1.3, 10.4, math.log10(2.8), 0.55,
                3.5, 2.0, 12.4, 9.0, 15.0])


@pytest.fixture(scope="module")
def setup():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2205_06819_gb300 import build as b
    b.build()
    from paper_2205_06819_gb300 import _lib, synth
    from paper_2205_06819_gb300.model import Galaxy, Model
    spec = synth.GalaxySpec(21, 15, 3, 2.2)
    ones = np.ones((4, spec.ny, spec.nx), np.float32)
    probe = Model(Galaxy(spec.nx, spec.ny, spec.oversample, spec.psf_fwhm_arcsec, spec.kpc_per_arcsec, ones, ones))
    true = probe.maps(torch.from_numpy(TH1.astype(np.float32)[None]).cuda())[0].cpu().numpy()
    probe.close()
    data, err, mask = synth.noisy_data(true, seed=91)
    m = Model(Galaxy(spec.nx, spec.ny, spec.oversample, spec.psf_fwhm_arcsec, spec.kpc_per_arcsec, data, err, mask))
    box = synth.prior_box(1)
    return _lib, m, box, synth


def noalloc(_lib, m, theta, logL, gal_idx=None):
    gptr = None if gal_idx is None else ctypes.c_void_p(gal_idx.ctypes.data)
    return _lib.lib().bang_loglike_batch_noalloc(m.handle, ctypes.c_void_p(theta.data_ptr()), gptr, theta.shape[0],
                                                 ctypes.c_void_p(logL.data_ptr()),
                                                 ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))


def test_noalloc_matches_allocating_entry_point_on_two_calls(setup):
    _lib, m, box, synth = setup
    const = None
    for call, (B, seed) in enumerate([(300, 92), (37, 93)]):
        theta = torch.from_numpy(synth.draw_theta_batch(box, TH1, B, seed).astype(np.float32)).cuda()
        theta[3, 13] = -1.0                                # one out-of-domain row
        out = torch.full((B,), 7.0, dtype=torch.float64, device="cuda")
        _lib.check(noalloc(_lib, m, theta, out))
        ref = m.loglike(theta).cpu().numpy()
        got = out.cpu().numpy()
        assert np.isneginf(got[3]) and np.isneginf(ref[3])
        fin = np.isfinite(ref)
        assert np.array_equal(fin, np.isfinite(got))
        # chi^2 relative error; the normalisation constant is common to both calls
        rel = np.abs(got[fin] - ref[fin]) / np.abs(ref[fin])
        assert rel.max() < CHI2_RTOL, (call, rel.max())


def test_noalloc_refuses_batches_beyond_its_scratch(setup):
    _lib, m, box, synth = setup
    B = 32769
    theta = torch.zeros((B, 15), dtype=torch.float32, device="cuda")
    out = torch.zeros(B, dtype=torch.float64, device="cuda")
    st = noalloc(_lib, m, theta, out)
    assert st == 1                                          # BANG_E_INVALID_ARG
    assert b"32768" in _lib.lib().bang_last_error()
    assert torch.count_nonzero(out).item() == 0


@pytest.mark.parametrize("opts", [{"psf_mode": 7}, {"bulge_kind": 1}, {"halo_kind": 1, "psf_mode": 4}])
def test_noalloc_under_model_options(setup, opts):
    """The no-allocation launch decodes each row itself; under the PSF modes, the closed-form
    bulge and the Hernquist halo it must still equal the allocating entry point."""
    _lib, m0, box, synth = setup
    from paper_2205_06819_gb300.model import Model
    m = Model(m0.galaxies, **opts)
    th = TH1.copy()
    if opts.get("halo_kind") == 1:
        th[13] = math.log10(30.0)
    b = synth.prior_box(1, halo_kind=opts.get("halo_kind", 0))
    theta = torch.from_numpy(synth.draw_theta_batch(b, th, 64, 95).astype(np.float32)).cuda()
    out = torch.zeros(64, dtype=torch.float64, device="cuda")
    _lib.check(noalloc(_lib, m, theta, out))
    ref = m.loglike(theta).cpu().numpy()
    got = out.cpu().numpy()
    fin = np.isfinite(ref)
    assert np.array_equal(fin, np.isfinite(got)) and fin.any()
    assert (np.abs(got[fin] - ref[fin]) / np.abs(ref[fin])).max() < CHI2_RTOL
    m.close()


def test_noalloc_chi2_matches_oracle(setup):
    """The entry point against the float64 oracle directly (chi^2, the theta-dependent part
    of logL), on the model's own data."""
    import oracle
    oracle.build()
    _lib, m, box, synth = setup
    g = m.galaxies[0]
    og = oracle.Galaxy(g.nx, g.ny, g.oversample, g.psf_fwhm_arcsec, g.kpc_per_arcsec,
                       data=np.asarray(g.data, np.float64), err=np.asarray(g.err, np.float64), mask=g.mask)
    theta_np = synth.draw_theta_batch(box, TH1, 6, 96).astype(np.float32)
    theta = torch.from_numpy(theta_np).cuda()
    out = torch.zeros(6, dtype=torch.float64, device="cuda")
    _lib.check(noalloc(_lib, m, theta, out))
    _, chi_ref = oracle.loglike(og, theta_np.astype(np.float64))
    chi = -2.0 * (out.cpu().numpy() + oracle.norm_const(og))
    assert (np.abs(chi - chi_ref) / chi_ref).max() < CHI2_RTOL


def test_noalloc_leaves_device_memory_unchanged(setup):
    """After a first call on the device (which looks up the scratch array), a second call with
    a different batch size changes neither the device's free memory nor the model's scratch."""
    _lib, m, box, synth = setup
    L = _lib.lib()
    th = torch.from_numpy(synth.draw_theta_batch(box, TH1, 300, 97).astype(np.float32)).cuda()
    out = torch.zeros(300, dtype=torch.float64, device="cuda")
    _lib.check(noalloc(_lib, m, th, out))
    torch.cuda.synchronize()
    free0, scratch0 = torch.cuda.mem_get_info()[0], L.bang_model_scratch_bytes(m.handle)
    th2, out2 = th[:123], out[:123]
    _lib.check(noalloc(_lib, m, th2, out2))
    _lib.check(noalloc(_lib, m, th2, out2))
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0
    assert L.bang_model_scratch_bytes(m.handle) == scratch0
    assert torch.isfinite(out2).any()


def test_noalloc_two_galaxies_with_host_gal_idx(setup):
    """A model of two galaxies with different grids and PSFs and a mixed host gal_idx: the
    gal_idx copy into the scratch array, the per-row galaxy lookup and the shared-memory size
    taken over the batch's galaxies, against bang_loglike_batch with the same gal_idx."""
    _lib, m0, box, synth = setup
    from paper_2205_06819_gb300.model import Galaxy, Model
    g0 = m0.galaxies[0]
    spec = synth.GalaxySpec(34, 27, 4, 3.1)
    ones = np.ones((4, spec.ny, spec.nx), np.float32)
    probe = Model(Galaxy(spec.nx, spec.ny, spec.oversample, spec.psf_fwhm_arcsec, spec.kpc_per_arcsec, ones, ones))
    true = probe.maps(torch.from_numpy(TH1.astype(np.float32)[None]).cuda())[0].cpu().numpy()
    probe.close()
    data, err, mask = synth.noisy_data(true, seed=98)
    g1 = Galaxy(spec.nx, spec.ny, spec.oversample, spec.psf_fwhm_arcsec, spec.kpc_per_arcsec, data, err, mask)
    m = Model([g0, g1])
    B = 96
    gal_idx = np.random.default_rng(99).integers(0, 2, size=B).astype(np.int32)
    theta = torch.from_numpy(synth.draw_theta_batch(box, TH1, B, 100).astype(np.float32)).cuda()
    for call in range(2):
        gi = gal_idx if call == 0 else np.ascontiguousarray(1 - gal_idx)
        out = torch.zeros(B, dtype=torch.float64, device="cuda")
        _lib.check(noalloc(_lib, m, theta, out, gi))
        torch.cuda.synchronize()
        ref = m.loglike(theta, gi).cpu().numpy()
        got = out.cpu().numpy()
        fin = np.isfinite(ref)
        assert fin.sum() > B // 2 and np.array_equal(fin, np.isfinite(got))
        assert (np.abs(got[fin] - ref[fin]) / np.abs(ref[fin])).max() < CHI2_RTOL, call
    m.close()

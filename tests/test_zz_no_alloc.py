"""The no-allocation entry point, bang_loglike_batch_noalloc, checked against
bang_loglike_batch through the C ABI.

That entry point is for callers that must not allocate device memory while they run (a
program whose GPU memory belongs to another allocator, or a loop that cannot take the
synchronisation cudaMalloc may cause): its scratch is a fixed array in the library's
device code.  Two calls in a row, on different batches, must each give the logL of the
allocating entry point within the chi-square tolerance of the other GPU tests (1e-5
relative), and an oversized batch must be refused before anything is launched.
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


def noalloc(_lib, m, theta, logL):
    return _lib.lib().bang_loglike_batch_noalloc(m.handle, ctypes.c_void_p(theta.data_ptr()), None, theta.shape[0],
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

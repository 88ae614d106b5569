"""Error handling through the C ABI on a GPU: invalid descriptors and arguments give
status codes, and an allocation failure injected on the host (a scratch cap) gives
BANG_E_OOM, after which the model still works.  Nothing here faults the GPU."""
import ctypes
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TH1 = np.array([0.05, -0.08, 0.4, 0.95, 10.2, math.log10(0.9), 1.3, 10.4, math.log10(2.8), 0.55,
                3.5, 2.0, 12.4, 9.0, 15.0], np.float32)


@pytest.fixture(scope="module")
def env():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2205_06819_gb300 import _lib, build
    build.build()
    from paper_2205_06819_gb300.model import Galaxy, Model
    ones = np.ones((4, 9, 11), np.float32)
    return _lib, Galaxy, Model, ones


def test_scratch_cap_gives_oom_then_recovers(env):
    _lib, Galaxy, Model, ones = env
    g = Galaxy(11, 9, 3, 2.0, 0.25695, ones * 50.0, ones)
    m = Model(g)
    L = _lib.lib()
    theta = torch.from_numpy(np.repeat(TH1[None], 64, 0)).cuda()
    assert L.bang_model_set_scratch_limit(m.handle, 4096) == 0
    with pytest.raises(_lib.BangError) as ei:
        m.loglike(theta)
    assert ei.value.status == 3                                      # BANG_E_OOM
    assert 0 <= L.bang_model_scratch_bytes(m.handle) <= 4096
    assert L.bang_model_set_scratch_limit(m.handle, 0) == 0
    got = m.loglike(theta).cpu().numpy()
    ref = Model(g).loglike(theta).cpu().numpy()
    np.testing.assert_array_equal(got, ref)
    assert L.bang_model_scratch_bytes(m.handle) > 0
    assert L.bang_model_set_scratch_limit(m.handle, -1) == 1


def test_invalid_arguments(env):
    _lib, Galaxy, Model, ones = env
    m = Model(Galaxy(11, 9, 3, 2.0, 0.25695, ones * 50.0, ones))
    theta = torch.from_numpy(TH1[None].copy()).cuda()
    with pytest.raises(_lib.BangError) as ei:
        m.loglike(theta, gal_idx=[3])                                # galaxy 3 does not exist
    assert ei.value.status == 1
    out = torch.empty(1, dtype=torch.float64, device="cuda")
    L = _lib.lib()
    assert L.bang_loglike_batch(m.handle, ctypes.c_void_p(theta.data_ptr()), None, 0,
                                ctypes.c_void_p(out.data_ptr()), None) == 1
    assert L.bang_loglike_batch(m.handle, None, None, 1, ctypes.c_void_p(out.data_ptr()), None) == 1


@pytest.mark.parametrize("case", ["bad_err", "bad_quad", "unknown_halo", "bad_table", "bad_grid"])
def test_invalid_model_descriptions(env, case):
    _lib, Galaxy, Model, ones = env
    err = ones.copy()
    kw = {}
    os_ = 3
    if case == "bad_err":
        err[2, 3, 4] = 0.0
    elif case == "bad_quad":
        kw["n_quad"] = 32
    elif case == "bad_table":
        kw["bulge_table"] = 100
    elif case == "bad_grid":
        os_ = 0
    if case == "unknown_halo":
        L = _lib.lib()
        d = (_lib.GalaxyDesc * 1)()
        data = ones * 50.0
        d[0].nx, d[0].ny, d[0].oversample = 11, 9, 3
        d[0].spaxel_arcsec, d[0].kpc_per_arcsec, d[0].psf_fwhm_arcsec = 1.0, 0.25695, 2.0
        d[0].data, d[0].err = data.ctypes.data, err.ctypes.data
        opts = _lib.ModelOpts(1, 0, 2, 64, 0, 0)
        h = ctypes.c_void_p()
        assert L.bang_model_create(d, 1, ctypes.byref(opts), 0, ctypes.byref(h)) == 4   # BANG_E_UNSUPPORTED
        assert b"halo" in L.bang_last_error()
        return
    with pytest.raises(_lib.BangError) as ei:
        Model(Galaxy(11, 9, os_, 2.0, 0.25695, ones * 50.0, err), **kw)
    assert ei.value.status == 1

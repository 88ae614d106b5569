"""CPU checks of the C ABI library: it builds, loads, and exports every function that
include/bang.h declares.  No compute call is made (there is no GPU here)."""
import ctypes
import subprocess

import pytest

from paper_2205_06819_gb300 import _lib
from paper_2205_06819_gb300 import build as build_mod


@pytest.fixture(scope="module")
def libpath():
    return build_mod.build()


def test_header_declares_the_boundary():
    names = _lib.header_functions()
    for required in ("bang_model_create", "bang_model_destroy", "bang_loglike_batch", "bang_loglike_grad_batch",
                     "bang_model_maps", "bang_loglike_plain", "bang_last_error"):
        assert required in names


def test_library_exports_every_declared_function(libpath):
    out = subprocess.run(["nm", "-D", "--defined-only", libpath], capture_output=True, text=True, check=True).stdout
    exported = {line.split()[-1] for line in out.splitlines() if " T " in line}
    missing = [n for n in _lib.header_functions() if n not in exported]
    assert not missing, missing


def test_library_loads_and_binds(libpath):
    L = _lib.lib()
    for n in _lib.header_functions():
        assert isinstance(getattr(L, n), ctypes._CFuncPtr)


def test_null_model_queries_do_not_touch_the_gpu(libpath):
    L = _lib.lib()
    assert L.bang_model_nparams(None) == -1
    assert L.bang_model_ngalaxies(None) == -1
    assert L.bang_model_destroy(None) == 0
    assert L.bang_loglike_batch(None, None, None, 1, None, None) == 1   # BANG_E_INVALID_ARG
    assert b"null model" in L.bang_last_error()


def test_checked_build_exports_the_same_abi_and_says_so(libpath):
    """The checked library (kernels check their indexes, BANG_E_BOUNDS) exports every
    declared function; bang_checked_build tells the two builds apart (a host-only call)."""
    checked = build_mod.build(checked=True)
    assert checked != libpath
    out = subprocess.run(["nm", "-D", "--defined-only", checked], capture_output=True, text=True, check=True).stdout
    exported = {line.split()[-1] for line in out.splitlines() if " T " in line}
    assert not [n for n in _lib.header_functions() if n not in exported]
    assert ctypes.CDLL(checked).bang_checked_build() == 1
    assert _lib.lib().bang_checked_build() == 0
    assert _lib.STATUS_NAMES[6] == "BANG_E_BOUNDS"


def test_loader_picks_the_checked_build_from_the_environment(monkeypatch):
    monkeypatch.setenv("BANG_CHECKED", "1")
    assert _lib.library_path() == _lib.LIB_CHECKED_PATH
    monkeypatch.setenv("BANG_CHECKED", "0")
    assert _lib.library_path() == _lib.LIB_PATH


def test_new_entry_points_validate_before_touching_the_gpu(libpath):
    L = _lib.lib()
    assert L.bang_loglike_fp64(None, None, None, 1, None, None) == 1        # BANG_E_INVALID_ARG
    assert b"null model" in L.bang_last_error()
    assert L.bang_check_selftest(0, 5, 3) == 4                               # normal build: BANG_E_UNSUPPORTED
    assert b"checked build" in L.bang_last_error()

"""ctypes binding of libbang.so (include/bang.h).  Argument marshalling only.

Importing this module does not load the library; ``lib()`` does, and raises if the CUDA
extension is missing or does not export the full ABI.  There is no fallback path.  With
BANG_CHECKED=1 in the environment it loads the checked build (libbang_checked.so, see
build.py) instead.
"""
from __future__ import annotations

import ctypes
import os
import re
import threading

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libbang.so")
LIB_CHECKED_PATH = os.path.join(HERE, "libbang_checked.so")
HEADER = os.path.join(os.path.dirname(HERE), "include", "bang.h")

BANG_OK = 0
STATUS_NAMES = {0: "BANG_OK", 1: "BANG_E_INVALID_ARG", 2: "BANG_E_CUDA", 3: "BANG_E_OOM",
                4: "BANG_E_UNSUPPORTED", 5: "BANG_E_TIMEOUT", 6: "BANG_E_BOUNDS"}


class BangError(RuntimeError):
    def __init__(self, status, message):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {message}")
        self.status = status


class GalaxyDesc(ctypes.Structure):
    _fields_ = [
        ("nx", ctypes.c_int), ("ny", ctypes.c_int), ("oversample", ctypes.c_int),
        ("spaxel_arcsec", ctypes.c_double), ("kpc_per_arcsec", ctypes.c_double),
        ("psf_kind", ctypes.c_int), ("psf_fwhm_arcsec", ctypes.c_double), ("moffat_beta", ctypes.c_double),
        ("data", ctypes.c_void_p), ("err", ctypes.c_void_p), ("mask", ctypes.c_void_p),
    ]


class ModelOpts(ctypes.Structure):
    _fields_ = [("n_discs", ctypes.c_int), ("bulge_kind", ctypes.c_int), ("halo_kind", ctypes.c_int),
                ("n_quad", ctypes.c_int), ("psf_mode", ctypes.c_int), ("bulge_table", ctypes.c_int)]


_VP = ctypes.c_void_p
_SIGNATURES = {
    "bang_model_create": (ctypes.c_int, [ctypes.POINTER(GalaxyDesc), ctypes.c_int, ctypes.POINTER(ModelOpts),
                                         ctypes.c_int, ctypes.POINTER(_VP)]),
    "bang_model_destroy": (ctypes.c_int, [_VP]),
    "bang_model_nparams": (ctypes.c_int, [_VP]),
    "bang_model_set_scratch_limit": (ctypes.c_int, [_VP, ctypes.c_int64]),
    "bang_model_scratch_bytes": (ctypes.c_int64, [_VP]),
    "bang_model_ngalaxies": (ctypes.c_int, [_VP]),
    "bang_model_psf_halfwidth": (ctypes.c_int, [_VP, ctypes.c_int]),
    "bang_loglike_batch": (ctypes.c_int, [_VP, _VP, _VP, ctypes.c_int, _VP, _VP]),
    "bang_loglike_grad_batch": (ctypes.c_int, [_VP, _VP, _VP, ctypes.c_int, _VP, _VP, _VP]),
    "bang_model_maps": (ctypes.c_int, [_VP, _VP, _VP, ctypes.c_int, _VP, _VP]),
    "bang_model_maps_size": (ctypes.c_int64, [_VP, _VP, ctypes.c_int]),
    "bang_loglike_plain": (ctypes.c_int, [_VP, _VP, _VP, ctypes.c_int, _VP, _VP]),
    "bang_loglike_grids": (ctypes.c_int, [_VP, _VP, ctypes.c_int, _VP, ctypes.c_int, _VP, _VP, _VP]),
    "bang_loglike_batch_noalloc": (ctypes.c_int, [_VP, _VP, _VP, ctypes.c_int, _VP, _VP]),
    "bang_loglike_fp64": (ctypes.c_int, [_VP, _VP, _VP, ctypes.c_int, _VP, _VP]),
    "bang_model_tune": (ctypes.c_int, [_VP, _VP, ctypes.c_int]),
    "bang_model_tune_grad": (ctypes.c_int, [_VP, _VP, ctypes.c_int]),
    "bang_model_launch_info": (ctypes.c_int, [_VP, _VP, ctypes.c_int, ctypes.c_int, _VP]),
    "bang_last_error": (ctypes.c_char_p, []),
    "bang_checked_build": (ctypes.c_int, []),
    "bang_check_selftest": (ctypes.c_int, [ctypes.c_int, ctypes.c_longlong, ctypes.c_longlong]),
}

_lock = threading.Lock()
_lib = None


def header_functions() -> list[str]:
    """Names of every function declared in include/bang.h."""
    with open(HEADER) as f:
        text = re.sub(r"/\*.*?\*/", "", f.read(), flags=re.S)
    return sorted(set(re.findall(r"\b(bang_[a-z0-9_]+)\s*\(", text)))


def library_path() -> str:
    """The library lib() loads: the checked build when BANG_CHECKED=1, else libbang.so."""
    return LIB_CHECKED_PATH if os.environ.get("BANG_CHECKED", "0") == "1" else LIB_PATH


def lib() -> ctypes.CDLL:
    global _lib
    with _lock:
        if _lib is None:
            path = library_path()
            if not os.path.exists(path):
                raise RuntimeError(f"{path} is missing: build it with paper_2205_06819_gb300.build.build("
                                   f"checked={path == LIB_CHECKED_PATH}) (there is no CPU fallback)")
            L = ctypes.CDLL(path)
            for name, (res, args) in _SIGNATURES.items():
                fn = getattr(L, name)
                fn.restype = res
                fn.argtypes = args
            _lib = L
    return _lib


def check(status: int) -> None:
    if status != BANG_OK:
        msg = lib().bang_last_error()
        raise BangError(status, msg.decode() if msg else "")

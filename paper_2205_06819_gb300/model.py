"""PyTorch-facing wrapper of the C ABI: a galaxy model, its batched log-likelihood, the
adjoint gradient and an autograd.Function.  PyTorch provides device memory and streams;
every step of the computation runs in the CUDA kernels of libbang.so.
"""
from __future__ import annotations

import ctypes
from dataclasses import dataclass

import numpy as np
import torch

from . import _lib


@dataclass
class Galaxy:
    """One observed galaxy: grid, PSF and [4, ny, nx] maps of data / errors / mask."""
    nx: int
    ny: int
    oversample: int
    psf_fwhm_arcsec: float
    kpc_per_arcsec: float
    data: np.ndarray
    err: np.ndarray
    mask: np.ndarray | None = None
    spaxel_arcsec: float = 1.0
    psf_kind: int = 0
    moffat_beta: float = 3.0


def _ptr(t):
    if t is None:
        return None
    if isinstance(t, torch.Tensor):
        return ctypes.c_void_p(t.data_ptr())
    return ctypes.c_void_p(t.ctypes.data)


def _stream_handle(device: torch.device | None = None):
    if not torch.cuda.is_available():
        return None
    return ctypes.c_void_p(torch.cuda.current_stream(device).cuda_stream)


#: bits of psf_mode (bang.h): circular 3-sigma window (Eq. 21), centre sampling (App. A),
#: flux-weighted moments
PSF_CIRCLE, PSF_CENTRE, PSF_FLUX = 1, 2, 4


class Model:
    """A likelihood model over one or more galaxies (bang_model_create)."""

    def __init__(self, galaxies, n_discs: int = 1, n_quad: int = 64, device: int = 0, bulge_table: int = 0,
                 halo_kind: int = 0, psf_mode: int = 0, bulge_kind: int = 0):
        if isinstance(galaxies, Galaxy):
            galaxies = [galaxies]
        self.galaxies = list(galaxies)
        self.n_discs, self.n_quad, self.device, self.bulge_table = n_discs, n_quad, device, bulge_table
        self.halo_kind, self.psf_mode, self.bulge_kind = halo_kind, psf_mode, bulge_kind
        L = _lib.lib()
        keep = []
        descs = (_lib.GalaxyDesc * len(self.galaxies))()
        for d, g in zip(descs, self.galaxies):
            data = np.ascontiguousarray(g.data, dtype=np.float32).reshape(4, g.ny, g.nx)
            err = np.ascontiguousarray(g.err, dtype=np.float32).reshape(4, g.ny, g.nx)
            mask = None if g.mask is None else np.ascontiguousarray(g.mask, dtype=np.uint8).reshape(4, g.ny, g.nx)
            keep += [data, err, mask]
            d.nx, d.ny, d.oversample = g.nx, g.ny, g.oversample
            d.spaxel_arcsec, d.kpc_per_arcsec = g.spaxel_arcsec, g.kpc_per_arcsec
            d.psf_kind, d.psf_fwhm_arcsec, d.moffat_beta = g.psf_kind, g.psf_fwhm_arcsec, g.moffat_beta
            d.data, d.err = data.ctypes.data, err.ctypes.data
            d.mask = None if mask is None else mask.ctypes.data
        opts = _lib.ModelOpts(n_discs, bulge_kind, halo_kind, n_quad, psf_mode, bulge_table)
        h = ctypes.c_void_p()
        _lib.check(L.bang_model_create(descs, len(self.galaxies), ctypes.byref(opts), device, ctypes.byref(h)))
        self._h = h
        self.nparams = L.bang_model_nparams(h)

    def close(self):
        if getattr(self, "_h", None):
            _lib.lib().bang_model_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def handle(self):
        return self._h

    def psf_halfwidth(self, g: int = 0) -> int:
        return _lib.lib().bang_model_psf_halfwidth(self._h, g)

    def _gal_idx(self, gal_idx, B):
        """(array, pointer) of gal_idx: a host numpy copy, or a CUDA int32 tensor passed as
        its device pointer (the library then schedules the batch on the device)."""
        if gal_idx is None:
            return None, None
        if isinstance(gal_idx, torch.Tensor) and gal_idx.is_cuda:
            if gal_idx.dtype != torch.int32 or gal_idx.numel() != B:
                raise ValueError(f"a device gal_idx must be int32 [{B}]")
            gi = gal_idx.contiguous()
            return gi, ctypes.c_void_p(gi.data_ptr())
        gi = np.ascontiguousarray(np.asarray(gal_idx, dtype=np.int32).reshape(B))
        return gi, ctypes.c_void_p(gi.ctypes.data)

    def _check_theta(self, theta):
        if theta.dim() != 2 or theta.shape[1] != self.nparams or theta.dtype != torch.float32:
            raise ValueError(f"theta must be float32 [B, {self.nparams}]")
        return theta.contiguous()

    def loglike(self, theta: torch.Tensor, gal_idx=None, out: torch.Tensor | None = None) -> torch.Tensor:
        """logL [B] float64 for theta [B, P] float32 (device or host tensor)."""
        theta = self._check_theta(theta)
        B = theta.shape[0]
        if out is None:
            out = torch.empty(B, dtype=torch.float64, device=theta.device)
        gi, gptr = self._gal_idx(gal_idx, B)
        _lib.check(_lib.lib().bang_loglike_batch(self._h, _ptr(theta), gptr, B, _ptr(out),
                                                 _stream_handle(theta.device) if theta.is_cuda else None))
        return out

    def loglike_grad(self, theta: torch.Tensor, gal_idx=None):
        """(logL [B] float64, d logL / d theta [B, P] float32)."""
        theta = self._check_theta(theta)
        B = theta.shape[0]
        logL = torch.empty(B, dtype=torch.float64, device=theta.device)
        grad = torch.empty_like(theta)
        gi, gptr = self._gal_idx(gal_idx, B)
        _lib.check(_lib.lib().bang_loglike_grad_batch(self._h, _ptr(theta), gptr, B, _ptr(logL), _ptr(grad),
                                                      _stream_handle(theta.device) if theta.is_cuda else None))
        return logL, grad

    def loglike_grids(self, theta: torch.Tensor, grids, grad: bool = False):
        """logL [B] (and d logL / d theta [B, P] with grad=True) of one galaxy observed on the
        model's galaxies ``grids`` (its maps on several spaxel grids): the sum over the grids
        (bang_loglike_grids)."""
        theta = self._check_theta(theta)
        B = theta.shape[0]
        g = np.ascontiguousarray(np.asarray(grids, dtype=np.int32).reshape(-1))
        logL = torch.empty(B, dtype=torch.float64, device=theta.device)
        gr = torch.empty_like(theta) if grad else None
        _lib.check(_lib.lib().bang_loglike_grids(self._h, _ptr(theta), B, ctypes.c_void_p(g.ctypes.data), len(g),
                                                 _ptr(logL), _ptr(gr),
                                                 _stream_handle(theta.device) if theta.is_cuda else None))
        return (logL, gr) if grad else logL

    def loglike_plain(self, theta: torch.Tensor, gal_idx=None) -> torch.Tensor:
        """logL through the one-kernel-per-task chain (the paper's Alg. 2 form)."""
        theta = self._check_theta(theta)
        B = theta.shape[0]
        out = torch.empty(B, dtype=torch.float64, device=theta.device)
        gi, gptr = self._gal_idx(gal_idx, B)
        _lib.check(_lib.lib().bang_loglike_plain(self._h, _ptr(theta), gptr, B, _ptr(out),
                                                 _stream_handle(theta.device) if theta.is_cuda else None))
        return out

    def loglike_fp64(self, theta: torch.Tensor, gal_idx=None) -> torch.Tensor:
        """logL [B] through the float64 check path (bang_loglike_fp64) for theta [B, P]
        float64 (device or host tensor): every step in float64, for comparisons with a
        float64 reference."""
        if theta.dim() != 2 or theta.shape[1] != self.nparams or theta.dtype != torch.float64:
            raise ValueError(f"theta must be float64 [B, {self.nparams}]")
        theta = theta.contiguous()
        B = theta.shape[0]
        out = torch.empty(B, dtype=torch.float64, device=theta.device)
        gi, gptr = self._gal_idx(gal_idx, B)
        _lib.check(_lib.lib().bang_loglike_fp64(self._h, _ptr(theta), gptr, B, _ptr(out),
                                                _stream_handle(theta.device) if theta.is_cuda else None))
        return out

    def maps(self, theta: torch.Tensor, gal_idx=None):
        """Model maps: a list of [4, ny, nx] float32 tensors, one per row."""
        theta = self._check_theta(theta)
        B = theta.shape[0]
        gi, gptr = self._gal_idx(gal_idx, B)
        n = _lib.lib().bang_model_maps_size(self._h, gptr, B)
        if n < 0:
            raise ValueError("bad gal_idx")
        flat = torch.empty(int(n), dtype=torch.float32, device=theta.device)
        _lib.check(_lib.lib().bang_model_maps(self._h, _ptr(theta), gptr, B, _ptr(flat),
                                              _stream_handle(theta.device) if theta.is_cuda else None))
        out, off = [], 0
        for b in range(B):
            g = self.galaxies[0 if gi is None else int(gi[b])]
            k = 4 * g.nx * g.ny
            out.append(flat[off:off + k].view(4, g.ny, g.nx))
            off += k
        return out

    def tune(self, B: int, gal_idx=None, grad: bool = False):
        """Autotune the launch shape for batches of B rows (with grad, the logL + gradient
        call's shape as well: bang_model_tune_grad)."""
        gi, gptr = self._gal_idx(gal_idx, B)
        fn = _lib.lib().bang_model_tune_grad if grad else _lib.lib().bang_model_tune
        _lib.check(fn(self._h, gptr, B))

    def launch_info(self, B: int, gal_idx=None, grad: bool = False) -> dict:
        """The launch shape a call on (gal_idx, B) would use (bang_model_launch_info)."""
        gi, gptr = self._gal_idx(gal_idx, B)
        info = (ctypes.c_int32 * 13)()
        _lib.check(_lib.lib().bang_model_launch_info(self._h, gptr, B, int(grad), info))
        keys = ["rows_per_step", "bands", "blocks_per_sm", "grid", "items", "smem_bytes", "adj_rows_per_item",
                "adj_grid", "adj_items", "device_items", "points_per_thread", "adj_blocks_per_sm", "column_lanes"]
        return dict(zip(keys, list(info)))


class LogLike(torch.autograd.Function):
    """logL = LogLike.apply(theta, model, gal_idx): batched log-likelihood whose backward is
    the hand-written adjoint kernel (the forward pass already returns the gradient)."""

    @staticmethod
    def forward(ctx, theta, model: Model, gal_idx=None):
        logL, grad = model.loglike_grad(theta.detach(), gal_idx)
        ctx.save_for_backward(grad)
        return logL

    @staticmethod
    def backward(ctx, grad_out):
        (grad,) = ctx.saved_tensors
        return grad * grad_out.to(grad.dtype)[:, None], None, None

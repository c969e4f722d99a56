"""GB300 widefield radio-interferometric measurement operator (hybrid w-stacking /
w-projection), after Dabbech & Wiaux.

Thin Python binding over the C ABI of librimo.so (include/rimo.h).  PyTorch provides
device memory and streams; every step of Phi, Phi^dagger, Phi^dagger Phi and the PSF
runs in the library's CUDA kernels.
"""
from __future__ import annotations

import ctypes as C
import math

import numpy as np

from . import _lib
from ._lib import (MODE_AUTO, MODE_HOLOGRAPHIC, MODE_ONTHEFLY, MODE_STORED_G, MODE_SURROGATE,
                   PlanInfo, PlanParams, RimoError)

__all__ = ["Plan", "PlanParams", "PlanInfo", "RimoError", "default_params", "estimate",
           "MODE_AUTO", "MODE_STORED_G", "MODE_HOLOGRAPHIC", "MODE_SURROGATE", "MODE_ONTHEFLY"]


def _torch():
    import torch
    return torch


def default_params(nx: int, ny: int, fov_x: float, fov_y: float, **kw) -> PlanParams:
    """rimo_plan_params_default followed by keyword overrides (field names of the C struct)."""
    lib = _lib.load()
    p = PlanParams()
    lib.rimo_plan_params_default(C.byref(p), nx, ny, fov_x, fov_y)
    for k, v in kw.items():
        if not hasattr(p, k):
            raise AttributeError(f"unknown plan parameter {k}")
        setattr(p, k, v)
    return p


def _uvw_arg(uvw) -> np.ndarray:
    u = np.ascontiguousarray(np.asarray(uvw, dtype=np.float64))
    if u.ndim != 2 or u.shape[1] != 3:
        raise ValueError("uvw must be (M, 3)")
    return u


def estimate(uvw, params: PlanParams) -> dict:
    """rimo_plan_estimate: host-only planning (P, mode, models) without a GPU."""
    lib = _lib.load()
    u = _uvw_arg(uvw)
    info = PlanInfo()
    _lib.check(lib.rimo_plan_estimate(u.ctypes.data, u.shape[0], C.byref(params), C.byref(info)))
    return info.as_dict()


def _stream_ptr(stream) -> int:
    torch = _torch()
    s = torch.cuda.current_stream() if stream is None else stream
    return int(s.cuda_stream)


def _check_image(t, ny, nx, name):
    torch = _torch()
    if not (t.is_cuda and t.dtype == torch.complex64 and t.is_contiguous() and tuple(t.shape) == (ny, nx)):
        raise ValueError(f"{name} must be a contiguous complex64 CUDA tensor of shape ({ny}, {nx})")


class Plan:
    """A measurement-operator plan (rimo_plan_create).  Owns its device memory."""

    def __init__(self, uvw, params: PlanParams, stream=None):
        self._lib = _lib.load()
        u = _uvw_arg(uvw)
        self.params = params
        self.nx, self.ny = int(params.nx), int(params.ny)
        self.M = u.shape[0]
        h = C.c_void_p()
        _lib.check(self._lib.rimo_plan_create(u.ctypes.data, self.M, C.byref(params),
                                              _stream_ptr(stream), C.byref(h)))
        self._h = h

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            self._lib.rimo_plan_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # ---------------------------------------------------------------- queries
    def info(self) -> dict:
        inf = PlanInfo()
        _lib.check(self._lib.rimo_plan_info_get(self._h, C.byref(inf)))
        return inf.as_dict()

    def bins(self):
        inf = self.info()
        ws = np.zeros(inf["P"], dtype=np.float64)
        b = np.zeros(self.M, dtype=np.int32)
        s = np.zeros(self.M, dtype=np.int32)
        _lib.check(self._lib.rimo_plan_get_bins(self._h, ws.ctypes.data, b.ctypes.data, s.ctypes.data))
        return ws, b, s

    def tiles(self, idx, stream=None):
        """(g0, h0, S, taps) of caller-order visibilities idx; taps[q][:S, :S]."""
        idx = np.ascontiguousarray(np.asarray(idx, dtype=np.int64))
        n = idx.size
        g0 = np.zeros(n, np.int32)
        h0 = np.zeros(n, np.int32)
        S = np.zeros(n, np.int32)
        taps = np.zeros((n, 19, 19), np.complex64)
        _lib.check(self._lib.rimo_plan_get_tiles(self._h, idx.ctypes.data, n, g0.ctypes.data,
                                                 h0.ctypes.data, S.ctypes.data, taps.ctypes.data,
                                                 _stream_ptr(stream)))
        out = []
        for q in range(n):
            s = int(S[q])
            out.append(taps[q].ravel()[: s * s].reshape(s, s))
        return g0, h0, S, out

    # ---------------------------------------------------------------- operators
    def phi(self, x, y=None, stream=None):
        torch = _torch()
        _check_image(x, self.ny, self.nx, "x")
        if y is None:
            y = torch.empty(self.M, dtype=torch.complex64, device=x.device)
        _lib.check(self._lib.rimo_apply_phi(self._h, x.data_ptr(), y.data_ptr(), _stream_ptr(stream)))
        return y

    def phi_adj(self, y, x=None, stream=None):
        torch = _torch()
        if not (y.is_cuda and y.dtype == torch.complex64 and y.numel() == self.M and y.is_contiguous()):
            raise ValueError("y must be a contiguous complex64 CUDA tensor with M entries")
        if x is None:
            x = torch.empty((self.ny, self.nx), dtype=torch.complex64, device=y.device)
        _lib.check(self._lib.rimo_apply_phi_adj(self._h, y.data_ptr(), x.data_ptr(), _stream_ptr(stream)))
        return x

    def phi_adj_phi(self, x, out=None, real_part_only: bool = False, stream=None):
        torch = _torch()
        _check_image(x, self.ny, self.nx, "x")
        if out is None:
            out = torch.empty_like(x)
        _lib.check(self._lib.rimo_apply_phi_adj_phi(self._h, x.data_ptr(), out.data_ptr(),
                                                    int(real_part_only), _stream_ptr(stream)))
        return out

    def psf(self, out=None, stream=None):
        torch = _torch()
        if out is None:
            out = torch.empty((self.ny, self.nx), dtype=torch.complex64, device="cuda")
        _lib.check(self._lib.rimo_psf(self._h, out.data_ptr(), _stream_ptr(stream)))
        return out

    def profile(self, on: bool = True):
        """Start or stop the per-stage CUDA-event timers (rimo_profile_enable)."""
        _lib.check(self._lib.rimo_profile_enable(self._h, int(on)))

    def profile_read(self, reset: bool = True) -> dict:
        """{stage: (total ms, kernel launches)} since the last reset (rimo_profile_read)."""
        ms = (C.c_double * _lib.N_STAGES)()
        ln = (C.c_int64 * _lib.N_STAGES)()
        _lib.check(self._lib.rimo_profile_read(self._h, ms, ln, _lib.N_STAGES, int(reset)))
        return {name: (ms[i], ln[i]) for i, name in enumerate(_lib.STAGE_NAMES)}

    def build_holographic(self, stream=None):
        _lib.check(self._lib.rimo_build_holographic(self._h, _stream_ptr(stream)))


def version() -> str:
    return _lib.load().rimo_version().decode()

"""GB300 widefield radio-interferometric measurement operator (hybrid w-stacking /
w-projection), after Dabbech & Wiaux.

Thin Python binding over the C ABI of librimo.so (include/rimo.h).  PyTorch provides
device memory and streams; every step of Phi, Phi^dagger, Phi^dagger Phi and the PSF
runs in the library's CUDA kernels.
"""
from __future__ import annotations

import ctypes as C
import math
import os

import numpy as np

from . import _lib
from ._lib import (MODE_AUTO, MODE_HOLOGRAPHIC, MODE_ONTHEFLY, MODE_STORED_G, MODE_SURROGATE,
                   PlanInfo, PlanParams, RimoError)

__all__ = ["Plan", "PlanParams", "PlanInfo", "RimoError", "default_params", "estimate", "Batch", "autotune_tile",
           "autotune_batch",
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

    @classmethod
    def from_file(cls, path: str, stream=None) -> "Plan":
        """rimo_plan_create_from_file: the plan a plan file (write_plan_file) describes."""
        params, M, _ = plan_file_info(path)
        self = cls.__new__(cls)
        self._lib = _lib.load()
        self.params = params
        self.nx, self.ny = int(params.nx), int(params.ny)
        self.M = M
        h = C.c_void_p()
        _lib.check(self._lib.rimo_plan_create_from_file(os.fsencode(path), _stream_ptr(stream), C.byref(h)))
        self._h = h
        return self

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
            # a shard plan writes only its own visibilities: the others read as zero
            y = (torch.zeros if self.params.shard_count >= 2 else torch.empty)(self.M, dtype=torch.complex64,
                                                                             device=x.device)
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

    def status(self, stream=None) -> None:
        """Raise RimoError if a kernel of this plan gave up a bounded wait (TIMEOUT) or met a
        non-finite input (INVALID_ARG) since the last check (rimo_plan_status)."""
        _lib.check(self._lib.rimo_plan_status(self._h, _stream_ptr(stream)))

    def zlayer(self, bin: int, stream=None):
        """Z_p of w-bin `bin` at every pixel as the kernels evaluate it (rimo_plan_get_zlayer)."""
        torch = _torch()
        out = torch.empty((self.ny, self.nx), dtype=torch.complex64, device="cuda")
        _lib.check(self._lib.rimo_plan_get_zlayer(self._h, int(bin), out.data_ptr(), _stream_ptr(stream)))
        return out

    def set_wait_test(self, stall: bool, polls: int = 16) -> None:
        """Failure-detection test of the grid step's bounded waits (rimo_plan_set_wait_test)."""
        _lib.check(self._lib.rimo_plan_set_wait_test(self._h, int(bool(stall)), int(polls)))

    def build_holographic(self, stream=None):
        _lib.check(self._lib.rimo_build_holographic(self._h, _stream_ptr(stream)))

    def phi_adj_phi_bins(self, x, bin_mask, out=None, real_part_only=False, stream=None):
        """sum over the w-bins with bin_mask[p] != 0 of Phi_p^dagger Phi_p x (rimo_apply_phi_adj_phi_bins)."""
        torch = _torch()
        _check_image(x, self.ny, self.nx, "x")
        m = np.ascontiguousarray(np.asarray(bin_mask, dtype=np.uint8))
        if m.size != self.info()["P"]:
            raise ValueError("bin_mask needs one entry per w-bin")
        if out is None:
            out = torch.empty_like(x)
        _lib.check(self._lib.rimo_apply_phi_adj_phi_bins(self._h, x.data_ptr(), out.data_ptr(), int(real_part_only),
                                                         m.ctypes.data, _stream_ptr(stream)))
        return out

    def set_weights(self, w, stream=None) -> None:
        """rimo_plan_set_weights: the operator becomes diag(w) Phi (w: M weights, caller
        order, finite and >= 0; None removes the weighting)."""
        if w is None:
            _lib.check(self._lib.rimo_plan_set_weights(self._h, None, _stream_ptr(stream)))
            return
        wa = np.ascontiguousarray(np.asarray(w, dtype=np.float32).reshape(-1))
        if wa.size != self.M:
            raise ValueError(f"expected {self.M} weights, got {wa.size}")
        _lib.check(self._lib.rimo_plan_set_weights(self._h, wa.ctypes.data, _stream_ptr(stream)))

    def set_surrogate(self, sur: "Surrogate") -> None:
        """rimo_plan_set_surrogate: generate this (surrogate-mode) plan's tiles with `sur`."""
        _lib.check(self._lib.rimo_plan_set_surrogate(self._h, sur._h))
        self._sur = sur  # keep it alive as long as the plan uses it

    def holographic_entries(self, bin: int, pairs, stream=None) -> np.ndarray:
        """H_bin[c1][c2] for rows (u1, v1, u2, v2) of `pairs` (rimo_plan_get_holographic)."""
        pr = np.ascontiguousarray(np.asarray(pairs, dtype=np.int32).reshape(-1, 4))
        out = np.zeros(pr.shape[0], np.complex64)
        _lib.check(self._lib.rimo_plan_get_holographic(self._h, int(bin), pr.ctypes.data, pr.shape[0],
                                                        out.ctypes.data, _stream_ptr(stream)))
        return out


class Surrogate:
    """The kernel-surrogate MLP (rimo_surrogate_*): 3 -> 128 -> 128 -> 450, bf16 tensor cores."""

    NPARAM = _lib.SURROGATE_NPARAM

    def __init__(self, seed: int = 0):
        self._lib = _lib.load()
        h = C.c_void_p()
        _lib.check(self._lib.rimo_surrogate_create(int(seed), C.byref(h)))
        self._h = h

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            self._lib.rimo_surrogate_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def get_params(self) -> np.ndarray:
        p = np.zeros(self.NPARAM, np.float32)
        _lib.check(self._lib.rimo_surrogate_get_params(self._h, p.ctypes.data))
        return p

    def set_params(self, p) -> None:
        p = np.ascontiguousarray(np.asarray(p, np.float32))
        if p.size != self.NPARAM:
            raise ValueError("wrong parameter count")
        _lib.check(self._lib.rimo_surrogate_set_params(self._h, p.ctypes.data))

    @staticmethod
    def _dev(a, cols):
        torch = _torch()
        t = a if hasattr(a, "data_ptr") else torch.from_numpy(np.ascontiguousarray(a, np.float32)).cuda()
        if t.dtype != torch.float32 or t.dim() != 2 or t.shape[1] != cols or not t.is_contiguous():
            raise ValueError(f"expected a contiguous float32 (B, {cols}) array")
        return t

    def forward(self, x, stream=None):
        torch = _torch()
        xd = self._dev(x, 3)
        y = torch.empty((xd.shape[0], 450), dtype=torch.float32, device=xd.device)
        _lib.check(self._lib.rimo_surrogate_forward(self._h, xd.data_ptr(), xd.shape[0], y.data_ptr(),
                                                    _stream_ptr(stream)))
        return y

    def gradients(self, x, t, stream=None):
        xd, td = self._dev(x, 3), self._dev(t, 450)
        g = np.zeros(self.NPARAM, np.float32)
        loss = C.c_float()
        _lib.check(self._lib.rimo_surrogate_gradients(self._h, xd.data_ptr(), td.data_ptr(), xd.shape[0],
                                                      g.ctypes.data, C.byref(loss), _stream_ptr(stream)))
        return float(loss.value), g

    def train_step(self, x, t, lr: float, want_loss: bool = False, stream=None):
        xd, td = self._dev(x, 3), self._dev(t, 450)
        loss = C.c_float()
        _lib.check(self._lib.rimo_surrogate_train_step(self._h, xd.data_ptr(), td.data_ptr(), xd.shape[0],
                                                       float(lr), C.byref(loss) if want_loss else None,
                                                       _stream_ptr(stream)))
        return float(loss.value) if want_loss else None

    def fit(self, exact_plan, n_samples: int, steps: int, batch: int = 1024, lr: float = 1e-3,
            seed: int = 0, stream=None) -> np.ndarray:
        """rimo_surrogate_fit on the exact tiles of `exact_plan`; returns the per-step losses."""
        losses = np.zeros(int(steps), np.float32)
        _lib.check(self._lib.rimo_surrogate_fit(self._h, exact_plan._h, int(n_samples), int(steps), int(batch),
                                                float(lr), int(seed), losses.ctypes.data, _stream_ptr(stream)))
        return losses

    @property
    def w_scale(self) -> float:
        v = C.c_float()
        _lib.check(self._lib.rimo_surrogate_get_w_scale(self._h, C.byref(v)))
        return float(v.value)

    @w_scale.setter
    def w_scale(self, value: float) -> None:
        _lib.check(self._lib.rimo_surrogate_set_w_scale(self._h, float(value)))


BATCH_AUTO, BATCH_STAGED, BATCH_BRANCHES = 0, 1, 2


class Batch:
    """Batched wideband Phi^dagger Phi over per-channel plans (rimo_batch_create).

    Keeps references to the plans; they must outlive the batch and share one image size.
    form: BATCH_AUTO (staged when the plans allow it), BATCH_STAGED (one launch per pass over
    every (channel, w-bin), the grid step one persistent launch over all their work units)
    or BATCH_BRANCHES (each channel's apply on its own graph branch).
    """

    def __init__(self, plans, form: int = 0):
        self._lib = _lib.load()
        self.plans = list(plans)
        if not self.plans:
            raise ValueError("a batch needs at least one plan")
        self.nx, self.ny = self.plans[0].nx, self.plans[0].ny
        arr = (C.c_void_p * len(self.plans))(*[p._h.value for p in self.plans])
        h = C.c_void_p()
        _lib.check(self._lib.rimo_batch_create_form(arr, len(self.plans), int(form), C.byref(h)))
        self._h = h

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            self._lib.rimo_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def phi_adj_phi(self, x, out=None, real_part_only=False, stream=None):
        """x, out: contiguous complex64 CUDA tensors of shape (n_plans, ny, nx)."""
        torch = _torch()
        shape = (len(self.plans), self.ny, self.nx)
        if not (x.is_cuda and x.dtype == torch.complex64 and x.is_contiguous() and tuple(x.shape) == shape):
            raise ValueError(f"x must be a contiguous complex64 CUDA tensor of shape {shape}")
        if out is None:
            out = torch.empty_like(x)
        elif not (out.is_cuda and out.dtype == torch.complex64 and out.is_contiguous() and tuple(out.shape) == shape):
            raise ValueError(f"out must be a contiguous complex64 CUDA tensor of shape {shape}")
        _lib.check(self._lib.rimo_batch_apply_phi_adj_phi(self._h, x.data_ptr(), out.data_ptr(),
                                                          int(real_part_only), _stream_ptr(stream)))
        return out

    def info(self) -> dict:
        n = C.c_int32()
        caps = C.c_int64()
        _lib.check(self._lib.rimo_batch_info(self._h, C.byref(n), C.byref(caps)))
        return {"n_plans": n.value, "captures": caps.value}

    def layout(self) -> dict:
        st = C.c_int32()
        jobs, units, sb = C.c_int64(), C.c_int64(), C.c_int64()
        _lib.check(self._lib.rimo_batch_layout(self._h, C.byref(st), C.byref(jobs), C.byref(units), C.byref(sb)))
        return {"staged": bool(st.value), "jobs": jobs.value, "units": units.value, "scratch_bytes": sb.value}


def fb_step(x, g, dirty, gamma: float, out=None, stream=None):
    """rimo_fb_step: Eq. 4 with the projection onto non-negative real images as D
    (x, g = Phi^dagger Phi x, dirty: complex64 CUDA tensors of one shape)."""
    torch = _torch()
    for t, name in ((x, "x"), (g, "g"), (dirty, "dirty")):
        if not (t.is_cuda and t.dtype == torch.complex64 and t.is_contiguous() and t.shape == x.shape):
            raise ValueError(f"{name} must be a contiguous complex64 CUDA tensor shaped like x")
    if out is None:
        out = torch.empty_like(x)
    lib = _lib.load()
    _lib.check(lib.rimo_fb_step(x.data_ptr(), g.data_ptr(), dirty.data_ptr(), float(gamma), out.data_ptr(),
                                x.numel(), _stream_ptr(stream)))
    return out


def image_dot(a, b, stream=None) -> float:
    """rimo_image_dot: Re <a, b> of two complex64 CUDA tensors, FP64 accumulation."""
    torch = _torch()
    if not (a.is_cuda and b.is_cuda and a.dtype == torch.complex64 and b.dtype == torch.complex64
            and a.is_contiguous() and b.is_contiguous() and a.numel() == b.numel()):
        raise ValueError("a and b must be contiguous complex64 CUDA tensors of one size")
    lib = _lib.load()
    r = C.c_double()
    _lib.check(lib.rimo_image_dot(a.data_ptr(), b.data_ptr(), a.numel(), C.byref(r), _stream_ptr(stream)))
    return r.value


def write_plan_file(path: str, uvw, params: PlanParams, weights=None) -> None:
    """rimo_plan_file_write: the inputs of a plan (uvw, parameters, optional data weights)
    in one checked file; host only."""
    lib = _lib.load()
    u = _uvw_arg(uvw)
    w = None
    if weights is not None:
        w = np.ascontiguousarray(np.asarray(weights, dtype=np.float32).reshape(-1))
        if w.size != u.shape[0]:
            raise ValueError(f"expected {u.shape[0]} weights, got {w.size}")
    _lib.check(lib.rimo_plan_file_write(os.fsencode(path), u.ctypes.data, u.shape[0], C.byref(params),
                                        None if w is None else w.ctypes.data))


def plan_file_info(path: str) -> tuple[PlanParams, int, bool]:
    """rimo_plan_file_info: (parameters, M, holds weights) of a checked plan file; host only."""
    lib = _lib.load()
    p = PlanParams()
    M = C.c_int64()
    hw = C.c_int32()
    _lib.check(lib.rimo_plan_file_info(os.fsencode(path), C.byref(p), C.byref(M), C.byref(hw)))
    return p, int(M.value), bool(hw.value)


def briggs_weights(uvw, nx: int, ny: int, fov_x: float, fov_y: float, robust: float) -> np.ndarray:
    """rimo_briggs_weights: Briggs' robust weights (float32, caller order)."""
    lib = _lib.load()
    u = _uvw_arg(uvw)
    out = np.zeros(u.shape[0], np.float32)
    _lib.check(lib.rimo_briggs_weights(u.ctypes.data, u.shape[0], int(nx), int(ny), float(fov_x), float(fov_y),
                                       float(robust), out.ctypes.data))
    return out


def autotune_tile(uvw, params: PlanParams, cache_path: str | None = None, stream=None) -> tuple[int, list]:
    """rimo_autotune_tile: (best uv-tile size, [ms at 32, ms at 64] or -1 where not timed)."""
    lib = _lib.load()
    u = _uvw_arg(uvw)
    tile = C.c_int32()
    ms = (C.c_double * 2)()
    path = cache_path.encode() if cache_path else None
    _lib.check(lib.rimo_autotune_tile(u.ctypes.data, u.shape[0], C.byref(params), path, _stream_ptr(stream),
                                      C.byref(tile), ms))
    return tile.value, [ms[0], ms[1]]


def autotune(uvw, params: PlanParams, cache_path: str | None = None, stream=None) -> dict:
    """rimo_autotune: the fastest uv-tile size and visibility order, with the six timings."""
    lib = _lib.load()
    u = _uvw_arg(uvw)
    tile, order = C.c_int32(), C.c_int32()
    ms = (C.c_double * 6)()
    path = cache_path.encode() if cache_path else None
    _lib.check(lib.rimo_autotune(u.ctypes.data, u.shape[0], C.byref(params), path, _stream_ptr(stream),
                                 C.byref(tile), C.byref(order), ms))
    return {"tile_size": tile.value, "uv_order": order.value, "ms": list(ms)}


def autotune_batch(uvws, params, cache_path: str | None = None, stream=None) -> dict:
    """rimo_autotune_batch: the uv-tile size and visibility order minimising the summed time
    over several workloads (uvws[i] with params[i]), with the six summed timings."""
    lib = _lib.load()
    if len(uvws) != len(params) or not uvws:
        raise ValueError("one parameter set per workload, at least one workload")
    us = [_uvw_arg(u) for u in uvws]
    n = len(us)
    ptrs = (C.c_void_p * n)(*[u.ctypes.data for u in us])
    ms_n = (C.c_int64 * n)(*[u.shape[0] for u in us])
    prm = (PlanParams * n)(*params)
    tile, order = C.c_int32(), C.c_int32()
    ms = (C.c_double * 6)()
    path = cache_path.encode() if cache_path else None
    _lib.check(lib.rimo_autotune_batch(ptrs, ms_n, prm, n, path, _stream_ptr(stream), C.byref(tile), C.byref(order),
                                       ms))
    return {"tile_size": tile.value, "uv_order": order.value, "ms": list(ms), "workloads": n}


def unpack_params(p: np.ndarray) -> dict:
    """Split the flat parameter vector into W1, b1, W2, b2, W3, b3 (FP32 views)."""
    shapes = (("W1", (128, 3)), ("b1", (128,)), ("W2", (128, 128)), ("b2", (128,)), ("W3", (450, 128)),
              ("b3", (450,)))
    out, o = {}, 0
    for name, shp in shapes:
        n = int(np.prod(shp))
        out[name] = p[o:o + n].reshape(shp)
        o += n
    return out


def pack_params(d: dict) -> np.ndarray:
    return np.concatenate([np.asarray(d[k], np.float32).ravel() for k in ("W1", "b1", "W2", "b2", "W3", "b3")])


def version() -> str:
    return _lib.load().rimo_version().decode()

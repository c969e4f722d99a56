"""ctypes view of the rimo C ABI (include/rimo.h): structures, prototypes, loading.

Argument marshalling only: every computation happens inside librimo.so.  Loading
fails loudly when the library has not been built; there is no fallback.
"""
from __future__ import annotations

import ctypes as C
import os

HERE = os.path.dirname(os.path.abspath(__file__))
# RIMO_LIBRARY selects another build of the same library (the sanitizer build, for one)
LIB_PATH = os.environ.get("RIMO_LIBRARY") or os.path.join(HERE, "librimo.so")

RIMO_OK = 0
N_STAGES = 16
SURROGATE_NPARAM = 75074
STAGE_NAMES = ["fwd_rows", "fwd_cols", "grid_clear", "gtg", "inv_cols", "inv_rows", "g_build",
               "h_build", "h_apply", "mlp", "bound"]
STATUS = {0: "OK", 1: "INVALID_ARG", 2: "OOM", 3: "BUDGET", 4: "CUDA", 5: "TIMEOUT",
          6: "UNSUPPORTED", 7: "STATE"}
MODE_AUTO, MODE_STORED_G, MODE_HOLOGRAPHIC, MODE_SURROGATE, MODE_ONTHEFLY = 0, 1, 2, 3, 4


class PlanParams(C.Structure):
    _fields_ = [
        ("nx", C.c_int32), ("ny", C.c_int32),
        ("fov_x", C.c_double), ("fov_y", C.c_double),
        ("oversampling", C.c_int32),
        ("kb_support", C.c_int32),
        ("kb_beta", C.c_double),
        ("max_wsupport", C.c_int32),
        ("w_norm_frac", C.c_double),
        ("mem_budget_bytes", C.c_int64),
        ("n_wbins", C.c_int32),
        ("n_blocks", C.c_int32),
        ("mode", C.c_int32),
        ("n_weight", C.c_int32),
        ("plan_fraction", C.c_double),
        ("seed", C.c_uint64),
        ("taper_literal", C.c_int32),
        ("wkernel_L", C.c_int32),
        ("tile_size", C.c_int32),
        ("block_bytes_max", C.c_int64),
        ("wkernel_table", C.c_int32),
        ("uv_order", C.c_int32),
        ("shard_count", C.c_int32),
        ("shard_rank", C.c_int32),
    ]


class PlanInfo(C.Structure):
    _fields_ = [
        ("M", C.c_int64),
        ("P", C.c_int32),
        ("mode", C.c_int32),
        ("p_star", C.c_int32),
        ("wkernel_L", C.c_int32),
        ("max_tile", C.c_int32),
        ("n_blocks", C.c_int32),
        ("n_tiles", C.c_int32),
        ("subset", C.c_int64),
        ("K", C.c_int64),
        ("g_bytes", C.c_int64),
        ("h_bytes", C.c_int64),
        ("scratch_bytes", C.c_int64),
        ("est_m_g", C.c_double),
        ("est_cost", C.c_double),
        ("wr_max", C.c_double),
        ("wsclean_p", C.c_double),
        ("support_table", C.c_int32 * 64),
        ("tile_size", C.c_int32),
        ("truncated", C.c_int32),
        ("weighted", C.c_int32),
        ("h_entries", C.c_int64),
        ("h_nonzero", C.c_int64),
        ("h_nnz", C.c_int64),
        ("n_units", C.c_int64),
        ("box_cells", C.c_int64),
        ("n_needed", C.c_int64),
        ("sel_rows", C.c_int64),
    ]

    def as_dict(self) -> dict:
        d = {f: getattr(self, f) for f, _ in self._fields_ if f != "support_table"}
        d["support_table"] = list(self.support_table)
        return d


_P = C.c_void_p
_PROTOS = {
    "rimo_plan_params_default": (None, [C.POINTER(PlanParams), C.c_int32, C.c_int32, C.c_double, C.c_double]),
    "rimo_plan_estimate": (C.c_int, [_P, C.c_int64, C.POINTER(PlanParams), C.POINTER(PlanInfo)]),
    "rimo_plan_create": (C.c_int, [_P, C.c_int64, C.POINTER(PlanParams), _P, C.POINTER(_P)]),
    "rimo_plan_destroy": (C.c_int, [_P]),
    "rimo_plan_info_get": (C.c_int, [_P, C.POINTER(PlanInfo)]),
    "rimo_plan_get_bins": (C.c_int, [_P, _P, _P, _P]),
    "rimo_plan_get_tiles": (C.c_int, [_P, _P, C.c_int64, _P, _P, _P, _P, _P]),
    "rimo_apply_phi": (C.c_int, [_P, _P, _P, _P]),
    "rimo_apply_phi_adj": (C.c_int, [_P, _P, _P, _P]),
    "rimo_apply_phi_adj_phi": (C.c_int, [_P, _P, _P, C.c_int32, _P]),
    "rimo_apply_phi_adj_phi_noalloc": (C.c_int, [_P, _P, _P, C.c_int32, _P]),
    "rimo_apply_phi_adj_phi_bins": (C.c_int, [_P, _P, _P, C.c_int32, _P, _P]),
    "rimo_build_holographic": (C.c_int, [_P, _P]),
    "rimo_plan_get_holographic": (C.c_int, [_P, C.c_int32, _P, C.c_int64, _P, _P]),
    "rimo_psf": (C.c_int, [_P, _P, _P]),
    "rimo_plan_status": (C.c_int, [_P, _P]),
    "rimo_plan_set_wait_test": (C.c_int, [_P, C.c_int32, C.c_int32]),
    "rimo_plan_get_zlayer": (C.c_int, [_P, C.c_int32, _P, _P]),
    "rimo_profile_enable": (C.c_int, [_P, C.c_int32]),
    "rimo_profile_read": (C.c_int, [_P, _P, _P, C.c_int32, C.c_int32]),
    "rimo_surrogate_create": (C.c_int, [C.c_uint64, C.POINTER(_P)]),
    "rimo_surrogate_destroy": (C.c_int, [_P]),
    "rimo_surrogate_get_params": (C.c_int, [_P, _P]),
    "rimo_surrogate_set_params": (C.c_int, [_P, _P]),
    "rimo_surrogate_forward": (C.c_int, [_P, _P, C.c_int64, _P, _P]),
    "rimo_surrogate_gradients": (C.c_int, [_P, _P, _P, C.c_int64, _P, _P, _P]),
    "rimo_surrogate_train_step": (C.c_int, [_P, _P, _P, C.c_int64, C.c_float, _P, _P]),
    "rimo_batch_create": (C.c_int, [_P, C.c_int32, C.POINTER(_P)]),
    "rimo_batch_destroy": (C.c_int, [_P]),
    "rimo_batch_apply_phi_adj_phi": (C.c_int, [_P, _P, _P, C.c_int32, _P]),
    "rimo_batch_info": (C.c_int, [_P, _P, _P]),
    "rimo_batch_create_form": (C.c_int, [_P, C.c_int32, C.c_int32, C.POINTER(_P)]),
    "rimo_batch_layout": (C.c_int, [_P, _P, _P, _P, _P]),
    "rimo_autotune_tile": (C.c_int, [_P, C.c_int64, C.POINTER(PlanParams), C.c_char_p, _P, _P, _P]),
    "rimo_autotune": (C.c_int, [_P, C.c_int64, C.POINTER(PlanParams), C.c_char_p, _P, _P, _P, _P]),
    "rimo_autotune_batch": (C.c_int, [_P, _P, _P, C.c_int32, C.c_char_p, _P, _P, _P, _P]),
    "rimo_plan_set_surrogate": (C.c_int, [_P, _P]),
    "rimo_surrogate_fit": (C.c_int, [_P, _P, C.c_int64, C.c_int32, C.c_int32, C.c_float, C.c_uint64, _P, _P]),
    "rimo_surrogate_get_w_scale": (C.c_int, [_P, C.POINTER(C.c_float)]),
    "rimo_surrogate_set_w_scale": (C.c_int, [_P, C.c_float]),
    "rimo_plan_set_weights": (C.c_int, [_P, _P, _P]),
    "rimo_briggs_weights": (C.c_int, [_P, C.c_int64, C.c_int32, C.c_int32, C.c_double, C.c_double, C.c_double, _P]),
    "rimo_fb_step": (C.c_int, [_P, _P, _P, C.c_float, _P, C.c_int64, _P]),
    "rimo_image_dot": (C.c_int, [_P, _P, C.c_int64, C.POINTER(C.c_double), _P]),
    "rimo_plan_file_write": (C.c_int, [C.c_char_p, _P, C.c_int64, C.POINTER(PlanParams), _P]),
    "rimo_plan_file_info": (C.c_int, [C.c_char_p, C.POINTER(PlanParams), C.POINTER(C.c_int64), C.POINTER(C.c_int32)]),
    "rimo_plan_create_from_file": (C.c_int, [C.c_char_p, _P, C.POINTER(_P)]),
    "rimo_last_error": (C.c_char_p, []),
    "rimo_version": (C.c_char_p, []),
}

_lib = None


class RimoError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


def load(path: str = LIB_PATH) -> C.CDLL:
    """Load librimo.so (built by __graft_entry__.build() or _build.build())."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise ImportError(f"{path} is missing: build the CUDA library first "
                          "(python -c 'import __graft_entry__ as g; g.build()')")
    lib = C.CDLL(path)
    for name, (res, args) in _PROTOS.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def check(status: int) -> None:
    if status != RIMO_OK:
        raise RimoError(status, _lib.rimo_last_error().decode() if _lib else "")

"""ctypes binding of the C ABI in include/lbm_cde.h (argument marshalling only).

Every function here forwards to liblbm_cde.so with the same name; the CUDA
kernels do all the work. There is no CPU fallback: if the library cannot be
loaded, ``lib()`` raises.
"""
from __future__ import annotations

import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "liblbm_cde.so")

LBM_OK, LBM_E_ARG, LBM_E_NOT_SPD, LBM_E_STATE, LBM_E_OOM, LBM_E_CUDA, LBM_E_NONFINITE, \
    LBM_E_TIMEOUT, LBM_E_UNSUPPORTED = range(9)
STATUS_NAMES = ["LBM_OK", "LBM_E_ARG", "LBM_E_NOT_SPD", "LBM_E_STATE", "LBM_E_OOM", "LBM_E_CUDA",
                "LBM_E_NONFINITE", "LBM_E_TIMEOUT", "LBM_E_UNSUPPORTED"]
LBM_D2Q9, LBM_D3Q15 = 9, 15
LBM_BC_PERIODIC, LBM_BC_NOFLUX_NODE, LBM_BC_BOUNCEBACK, LBM_BC_DIRICHLET = 0, 1, 2, 3
LBM_STORE_F32, LBM_STORE_F16_NEQ, LBM_STORE_BF16_NEQ = 0, 1, 2
LBM_U_NONE, LBM_U_FIELD, LBM_U_ROW_PROFILE = 0, 1, 2

ALLOC_FN = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p)
FREE_FN = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_void_p)


class LbmDesc(ctypes.Structure):
    _fields_ = [
        ("lattice", ctypes.c_int32),
        ("storage", ctypes.c_int32),
        ("nx", ctypes.c_int64),
        ("ny", ctypes.c_int64),
        ("nz", ctypes.c_int64),
        ("bc_lo_y", ctypes.c_int32),
        ("bc_hi_y", ctypes.c_int32),
        ("phi_w_lo_y", ctypes.c_double),
        ("phi_w_hi_y", ctypes.c_double),
        ("alpha1", ctypes.c_double),
        ("alpha2", ctypes.c_double),
        ("s", ctypes.c_double * 15),
        ("tie_q_rates", ctypes.c_int32),
        ("alloc", ALLOC_FN),
        ("free_", FREE_FN),
        ("alloc_ctx", ctypes.c_void_p),
        ("stream", ctypes.c_void_p),
        ("model", ctypes.c_int32),
        ("bc_lo_x", ctypes.c_int32),
        ("bc_hi_x", ctypes.c_int32),
        ("bc_lo_z", ctypes.c_int32),
        ("bc_hi_z", ctypes.c_int32),
    ]


LBM_MRT_A, LBM_MRT_B1, LBM_MRT_B2, LBM_MRT_B3 = 0, 1, 2, 3
LBM_BATCH_AUTO, LBM_BATCH_PERSISTENT, LBM_BATCH_PER_STEP = 0, 1, 2


class ChannelDesc(ctypes.Structure):
    _fields_ = [
        ("nx", ctypes.c_int64),
        ("ny", ctypes.c_int64),
        ("bc_lo_y", ctypes.c_int32),
        ("bc_hi_y", ctypes.c_int32),
        ("D", ctypes.c_double * 4),
        ("s", ctypes.c_double * 15),
        ("tie_q_rates", ctypes.c_int32),
        ("u_row_dev", ctypes.c_void_p),
        ("x_ref0", ctypes.c_double),
        ("x_ref_velocity", ctypes.c_double),
        ("model", ctypes.c_int32),
    ]


class BatchOpts(ctypes.Structure):
    _fields_ = [
        ("mode", ctypes.c_int32),
        ("tile_rows", ctypes.c_int32),
        ("graph_steps", ctypes.c_int32),
        ("barrier_timeout_cycles", ctypes.c_int64),
        ("alloc", ALLOC_FN),
        ("free_", FREE_FN),
        ("alloc_ctx", ctypes.c_void_p),
        ("stream", ctypes.c_void_p),
    ]


class LbmError(RuntimeError):
    def __init__(self, status: int, what: str, msg: str):
        self.status = status
        name = STATUS_NAMES[status] if 0 <= status < len(STATUS_NAMES) else str(status)
        super().__init__(f"{what} failed: {name}: {msg}")


_lib = None

_P = ctypes.c_void_p
_I64 = ctypes.c_int64
_DP = ctypes.POINTER(ctypes.c_double)

# name -> argtypes (restype is lbm_status = int unless stated)
SIGNATURES = {
    "lbm_cde_desc_init": [ctypes.POINTER(LbmDesc), ctypes.c_int32, _I64, _I64, _I64],
    "lbm_cde_create": [ctypes.POINTER(LbmDesc), ctypes.POINTER(_P)],
    "lbm_cde_destroy": [_P],
    "lbm_cde_set_D": [_P, _DP],
    "lbm_cde_get_rates": [_P, _DP, _DP],
    "lbm_cde_set_velocity": [_P, ctypes.c_int32, _P, _P, _I64],
    "lbm_cde_set_phi": [_P, _P],
    "lbm_cde_step": [_P, _I64],
    "lbm_cde_set_launch": [_P, ctypes.c_int32, ctypes.c_int32],
    "lbm_cde_set_wait_limit": [_P, _I64],
    "lbm_cde_set_zwalk": [_P, ctypes.c_int32],
    "lbm_cde_autotune": [_P, _I64, ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_int32)],
    "lbm_cde_get_time": [_P, ctypes.POINTER(_I64)],
    "lbm_cde_get_phi": [_P, _P],
    "lbm_cde_sum_phi": [_P, _DP],
    "lbm_cde_sync": [_P],
    "lbm_cde_state_bytes": [_P, ctypes.POINTER(ctypes.c_size_t)],
    "lbm_cde_get_state": [_P, _P, ctypes.POINTER(_I64)],
    "lbm_cde_set_state": [_P, _P, _I64],
    "lbm_cde_run_host": [_P, _P, _I64, _P],
    "lbm_cde_last_error": [_P],
    "lbm_cde_adjoint_ngrad": [ctypes.c_int32],
    "lbm_cde_adjoint_step": [_P, _I64, _P, _P, _P, _P, _P],
    "lbm_cde_grad_rates": [_P, _DP, _DP, _DP],
    "lbm_cde_forward_ckpt": [_P, _P, _I64, _I64, _P],
    "lbm_cde_backward": [_P, _P, _P, _DP, _DP, _P],
    "lbm_cde_set_profiling": [_P, ctypes.c_int32],
    "lbm_cde_backward_phases": [_P, _DP],
    "lbm_cde_batch_opts_init": [ctypes.POINTER(BatchOpts)],
    "lbm_cde_batch_create": [ctypes.POINTER(ChannelDesc), ctypes.c_int32, ctypes.POINTER(BatchOpts),
                             ctypes.POINTER(_P)],
    "lbm_cde_batch_destroy": [_P],
    "lbm_cde_batch_cells": [_P, ctypes.POINTER(_I64)],
    "lbm_cde_batch_set_phi": [_P, _P],
    "lbm_cde_batch_get_phi": [_P, _P],
    "lbm_cde_batch_run": [_P, _I64, _DP],
    "lbm_cde_batch_autotune": [_P, _I64, ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_int32)],
    "lbm_cde_batch_config": [_P, ctypes.c_int32, ctypes.c_int32],
    "lbm_cde_batch_last_error": [_P],
    "lbm_cde_sum_state_noalloc": [_P, ctypes.c_int32, ctypes.c_int32, _I64, _P, _P],
    "lbm_cde_noalloc_last_error": [],
}


def lib(build_if_missing: bool = True):
    """Loads liblbm_cde.so (building it with nvcc first if it is missing)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        if not build_if_missing:
            raise RuntimeError(f"{LIB_PATH} is missing; run __graft_entry__.build()")
        from . import build as _build

        _build.build()
    L = ctypes.CDLL(LIB_PATH)
    for name, argt in SIGNATURES.items():
        fn = getattr(L, name)
        fn.argtypes = argt
        fn.restype = ctypes.c_char_p if name.endswith("last_error") else ctypes.c_int
    _lib = L
    return L


def check(status: int, what: str, handle=None):
    if status != LBM_OK:
        msg = lib().lbm_cde_last_error(handle)
        raise LbmError(status, what, msg.decode() if msg else "")


def header_symbols(header_path: str | None = None):
    """Function names declared in include/lbm_cde.h."""
    import re

    if header_path is None:
        header_path = os.path.join(os.path.dirname(HERE), "include", "lbm_cde.h")
    txt = open(header_path).read()
    return sorted(set(re.findall(r"\b(lbm_cde_\w+)\s*\(", txt)))

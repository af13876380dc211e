"""ctypes declarations of the C ABI in include/trident_spgemm.h.

Argument marshalling only: every computation happens in the CUDA library.
Loading fails loudly if the library has not been built.
"""
from __future__ import annotations

import ctypes
import os
import threading

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libtrident_spgemm.so")

MAX_BINS = 12
NUM_VARIANTS = 20
NUM_PHASES = 8
F32, F64 = 0, 1

STATUS = {
    0: "SPGEMM_OK", 1: "SPGEMM_ERR_INVALID_ARG", 2: "SPGEMM_ERR_SHAPE", 3: "SPGEMM_ERR_DTYPE",
    4: "SPGEMM_ERR_INDEX_OVERFLOW", 5: "SPGEMM_ERR_OOM", 6: "SPGEMM_ERR_CUDA", 7: "SPGEMM_ERR_DEVICE_TIMEOUT",
    8: "SPGEMM_ERR_HASH_OVERFLOW", 9: "SPGEMM_ERR_NOT_CANONICAL", 10: "SPGEMM_ERR_INTERNAL",
    11: "SPGEMM_ERR_UNSUPPORTED", 12: "SPGEMM_ERR_CAPACITY",
}


class SpgemmError(RuntimeError):
    def __init__(self, code: int, where: str):
        self.code = code
        super().__init__(f"{where}: {STATUS.get(code, code)} ({_lib_status_str(code)})")


class CsrIn(ctypes.Structure):
    _fields_ = [("nrows", ctypes.c_int32), ("ncols", ctypes.c_int32), ("nnz", ctypes.c_int32),
                ("row_ptr", ctypes.c_void_p), ("col_idx", ctypes.c_void_p), ("val", ctypes.c_void_p)]


class CsrOut(ctypes.Structure):
    _fields_ = [("nrows", ctypes.c_int32), ("ncols", ctypes.c_int32), ("row_ptr", ctypes.c_void_p),
                ("col_idx", ctypes.c_void_p), ("val", ctypes.c_void_p)]


class MclParams(ctypes.Structure):
    _fields_ = [("inflation", ctypes.c_double), ("prune", ctypes.c_double), ("topk", ctypes.c_int32),
                ("heavy", ctypes.c_int32), ("window", ctypes.c_int32)]


class Tune(ctypes.Structure):
    _fields_ = [("num_bins", ctypes.c_int32), ("bin_upper", ctypes.c_int32 * MAX_BINS),
                ("bin_kernel", ctypes.c_int32 * MAX_BINS), ("accumulator", ctypes.c_int32),
                ("warps_per_block", ctypes.c_int32), ("validate", ctypes.c_int32),
                ("sym_warps_per_block", ctypes.c_int32)]


# name -> (argtypes, restype); every exported symbol of the header
P = ctypes.c_void_p
I32 = ctypes.c_int32
I64P = ctypes.POINTER(ctypes.c_int64)
SIGNATURES = {
    "spgemm_status_str": ([ctypes.c_int], ctypes.c_char_p),
    "spgemm_version": ([], ctypes.c_char_p),
    "spgemm_create": ([ctypes.POINTER(P)], ctypes.c_int),
    "spgemm_destroy": ([P], ctypes.c_int),
    "spgemm_default_tune": ([ctypes.POINTER(Tune)], ctypes.c_int),
    "spgemm_set_tune": ([P, ctypes.POINTER(Tune)], ctypes.c_int),
    "spgemm_get_tune": ([P, ctypes.POINTER(Tune)], ctypes.c_int),
    "spgemm_symbolic": ([P, ctypes.POINTER(CsrIn), ctypes.POINTER(CsrIn), P, I64P, P], ctypes.c_int),
    "spgemm_numeric": ([P, ctypes.c_int, ctypes.POINTER(CsrIn), ctypes.POINTER(CsrIn), ctypes.POINTER(CsrOut), P],
                       ctypes.c_int),
    "spgemm_host_symbolic": ([P, ctypes.c_int32, ctypes.POINTER(CsrIn), ctypes.POINTER(CsrIn), P, I64P, P],
                             ctypes.c_int),
    "spgemm_host_numeric": ([P, ctypes.c_int, ctypes.POINTER(CsrIn), ctypes.POINTER(CsrIn), ctypes.POINTER(CsrOut),
                             I32, P], ctypes.c_int),
    "spgemm_merge": ([P, ctypes.c_int, I32, ctypes.POINTER(CsrIn), ctypes.POINTER(CsrOut), I64P, P], ctypes.c_int),
    "spgemm_products": ([P, ctypes.POINTER(CsrIn), ctypes.POINTER(CsrIn), I64P, P], ctypes.c_int),
    "spgemm_fused": ([P, ctypes.c_int, ctypes.POINTER(CsrIn), ctypes.POINTER(CsrIn), ctypes.POINTER(CsrOut),
                      ctypes.c_int64, I64P, P], ctypes.c_int),
    "spgemm_batched": ([P, ctypes.c_int, I32, ctypes.POINTER(CsrIn), ctypes.POINTER(CsrIn), I32,
                        ctypes.POINTER(I32), ctypes.POINTER(CsrOut), I64P, ctypes.POINTER(Tune), P], ctypes.c_int),
    "spgemm_tile_split": ([P, ctypes.c_int, ctypes.POINTER(CsrIn), I32, ctypes.POINTER(I32), I32,
                           ctypes.POINTER(I32), ctypes.POINTER(CsrOut), I64P, P], ctypes.c_int),
    "spgemm_trident_bounds": ([I32, I32, I32, ctypes.POINTER(I32), ctypes.POINTER(I32)], ctypes.c_int),
    "spgemm_trident_schedule": ([I32, I32, ctypes.POINTER(I32), ctypes.POINTER(I32), ctypes.POINTER(I32)],
                                ctypes.c_int),
    "spgemm_backward": ([P, ctypes.c_int, ctypes.POINTER(CsrIn), ctypes.POINTER(CsrIn), ctypes.POINTER(CsrIn), P, P,
                         I32, P], ctypes.c_int),
    "spgemm_csr_transpose": ([P, ctypes.c_int, ctypes.POINTER(CsrIn), ctypes.POINTER(CsrOut), P], ctypes.c_int),
    "spgemm_csr_permute": ([P, ctypes.c_int, ctypes.POINTER(CsrIn), P, P, ctypes.POINTER(CsrOut), P], ctypes.c_int),
    "spgemm_plan_create": ([ctypes.c_int, I32, ctypes.POINTER(CsrIn), ctypes.POINTER(CsrIn), I32, ctypes.POINTER(I32),
                            ctypes.POINTER(P), I64P, ctypes.POINTER(Tune), P, ctypes.POINTER(P)], ctypes.c_int),
    "spgemm_plan_execute": ([P, ctypes.POINTER(CsrOut), I32, P], ctypes.c_int),
    "spgemm_plan_autotune": ([P, ctypes.POINTER(CsrOut), P, ctypes.POINTER(Tune)], ctypes.c_int),
    "spgemm_plan_launch_count": ([P, I64P], ctypes.c_int),
    "spgemm_set_concurrent_bins": ([P, I32], ctypes.c_int),
    "spgemm_plan_set_concurrent_bins": ([P, I32], ctypes.c_int),
    "spgemm_tune_cache_open": ([ctypes.c_char_p, I64P], ctypes.c_int),
    "spgemm_tune_cache_clear": ([], ctypes.c_int),
    "spgemm_tune_cache_store": ([ctypes.c_uint64, ctypes.POINTER(Tune)], ctypes.c_int),
    "spgemm_tune_cache_count": ([I64P], ctypes.c_int),
    "spgemm_tune_cache_entry": ([ctypes.c_int64, ctypes.POINTER(ctypes.c_uint64), ctypes.POINTER(Tune)], ctypes.c_int),
    "spgemm_plan_destroy": ([P], ctypes.c_int),
    "spgemm_csr_transpose_noalloc": ([ctypes.c_int, ctypes.POINTER(CsrIn), ctypes.POINTER(CsrOut), P], ctypes.c_int),
    "spgemm_mcl_expand": ([P, ctypes.POINTER(CsrIn), ctypes.POINTER(MclParams), P, I64P, P], ctypes.c_int),
    "spgemm_mcl_collect": ([P, ctypes.POINTER(CsrOut), P], ctypes.c_int),
    "spgemm_mcl_paths": ([P, I64P, ctypes.POINTER(ctypes.c_double)], ctypes.c_int),
    "spgemm_launch_count": ([P, I64P], ctypes.c_int),
    "spgemm_device_status": ([P], ctypes.c_int),
    "spgemm_set_timing": ([P, I32], ctypes.c_int),
    "spgemm_set_wait_test": ([P, I32, I32], ctypes.c_int),
    "spgemm_set_workspace_limit": ([P, ctypes.c_int64], ctypes.c_int),
    "spgemm_workspace_bytes": ([P, I64P], ctypes.c_int),
    "spgemm_read_timing": ([P, ctypes.POINTER(ctypes.c_double), I64P], ctypes.c_int),
}

_lock = threading.Lock()
_lib = None


def lib():
    """The loaded CUDA library (raises if it was not built)."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise RuntimeError(f"CUDA library missing at {LIB_PATH}: build it with "
                                   "`python -c 'import __graft_entry__ as g; g.build()'`")
            L = ctypes.CDLL(LIB_PATH)
            for name, (args, res) in SIGNATURES.items():
                f = getattr(L, name)
                f.argtypes = args
                f.restype = res
            _lib = L
        return _lib


def _lib_status_str(code: int) -> str:
    try:
        return lib().spgemm_status_str(code).decode()
    except Exception:
        return "?"


def check(code: int, where: str) -> None:
    if code != 0:
        raise SpgemmError(code, where)

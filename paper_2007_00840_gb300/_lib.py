"""ctypes view of the C ABI in include/gsofa.h (argument marshalling only)."""
from __future__ import annotations

import ctypes
import os
import threading

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libgsofa.so")

GSOFA_OK = 0
GSOFA_E_INVAL = -1
GSOFA_E_NOMEM = -2
GSOFA_E_CUDA = -3
GSOFA_E_NOCONVERGE = -4
GSOFA_E_TIMEOUT = -5
GSOFA_E_BUSY = -6
GSOFA_E_NOTFOUND = -7
GSOFA_E_PENDING = -8
GSOFA_NOALLOC_MAX_N = 65533


class gsofa_options(ctypes.Structure):
    _fields_ = [
        ("chunk_size", ctypes.c_int32),
        ("threads_per_source", ctypes.c_int32),
        ("smem_max_source", ctypes.c_int32),
        ("max_concurrent", ctypes.c_int32),
        ("mem_budget_bytes", ctypes.c_int64),
        ("fill_first", ctypes.c_int32),
        ("collect_stats", ctypes.c_int32),
        ("validate", ctypes.c_int32),
        ("autotune", ctypes.c_int32),
        ("work_chunk", ctypes.c_int32),
        ("list_capacity", ctypes.c_int32),
        ("max_ctas", ctypes.c_int32),
        ("frontier_order", ctypes.c_int32),
        ("label_bits", ctypes.c_int32),
        ("expand_mode", ctypes.c_int32),
        ("schedule", ctypes.c_int32),
        ("team_sources", ctypes.c_int32),
        ("warps_per_sm", ctypes.c_int32),
        ("host_spill", ctypes.c_int32),
        ("clean_heads", ctypes.c_int32),
        ("reserved", ctypes.c_int32),
    ]


class gsofa_stats(ctypes.Structure):
    _fields_ = [
        ("ms_validate", ctypes.c_float),
        ("ms_traverse", ctypes.c_float),
        ("ms_emit", ctypes.c_float),
        ("ms_supernode", ctypes.c_float),
        ("ms_total", ctypes.c_float),
        ("ms_traverse_smem", ctypes.c_float),
        ("ms_traverse_global", ctypes.c_float),
        ("traverse_launches", ctypes.c_int32),
        ("kernel_launches", ctypes.c_int32),
        ("vertices_expanded", ctypes.c_int64),
        ("edges_scanned", ctypes.c_int64),
        ("pool_retries", ctypes.c_int64),
        ("levels", ctypes.c_int64),
        ("cycles_traverse", ctypes.c_int64),
        ("cycles_emit", ctypes.c_int64),
    ]


class gsofa_result(ctypes.Structure):
    _fields_ = [
        ("n", ctypes.c_int32),
        ("n_super", ctypes.c_int32),
        ("nnz_L", ctypes.c_int64),
        ("nnz_U", ctypes.c_int64),
        ("L_rowptr", ctypes.c_void_p),
        ("L_colidx", ctypes.c_void_p),
        ("U_rowptr", ctypes.c_void_p),
        ("U_colidx", ctypes.c_void_p),
        ("fill_count", ctypes.c_void_p),
        ("super_start", ctypes.c_void_p),
        ("on_device", ctypes.c_int32),
        ("err_detail", ctypes.c_int32),
        ("stats", gsofa_stats),
        ("_priv", ctypes.c_void_p),
    ]


class gsofa_server_config(ctypes.Structure):
    _fields_ = [
        ("mem_cap_bytes", ctypes.c_int64),
        ("max_inflight", ctypes.c_int32),
        ("streams", ctypes.c_int32),
        ("max_batch", ctypes.c_int32),
        ("queue_capacity", ctypes.c_int32),
        ("opts", gsofa_options),
    ]


class gsofa_server_stats(ctypes.Structure):
    _fields_ = [
        ("completed", ctypes.c_int64),
        ("failed", ctypes.c_int64),
        ("batches", ctypes.c_int64),
        ("pending", ctypes.c_int64),
        ("inflight", ctypes.c_int32),
        ("kernel_launches", ctypes.c_int32),
        ("total_nnz", ctypes.c_int64),
        ("total_rows", ctypes.c_int64),
        ("mem_in_use", ctypes.c_int64),
        ("peak_mem_in_use", ctypes.c_int64),
        ("p50_ms", ctypes.c_float),
        ("p99_ms", ctypes.c_float),
        ("max_ms", ctypes.c_float),
        ("pad2", ctypes.c_float),
        ("span_s", ctypes.c_double),
        ("peak_device_bytes", ctypes.c_int64),
    ]


# every symbol include/gsofa.h declares, with its ctypes signature
_P = ctypes.c_void_p
_I32 = ctypes.c_int32
SIGNATURES = {
    "gsofa_default_options": (ctypes.c_int, [ctypes.POINTER(gsofa_options)]),
    "gsofa_symbolic": (ctypes.c_int, [_I32, _P, _P, ctypes.POINTER(gsofa_options), ctypes.POINTER(gsofa_result)]),
    "gsofa_symbolic_device": (ctypes.c_int, [_I32, _P, _P, ctypes.POINTER(gsofa_options), _P,
                                             ctypes.POINTER(gsofa_result)]),
    "gsofa_batch": (ctypes.c_int, [_I32, _P, _P, _P, ctypes.POINTER(gsofa_options), _P, _P]),
    "gsofa_row_counts_noalloc": (ctypes.c_int, [_I32, _P, _P, _P, _P, _P, _P]),
    "gsofa_server_default_config": (ctypes.c_int, [ctypes.POINTER(gsofa_server_config)]),
    "gsofa_server_create": (ctypes.c_int, [ctypes.POINTER(gsofa_server_config), ctypes.POINTER(ctypes.c_void_p)]),
    "gsofa_server_submit": (ctypes.c_int, [_P, _I32, _P, _P, _I32, ctypes.POINTER(ctypes.c_uint64)]),
    "gsofa_server_poll": (ctypes.c_int, [_P, ctypes.c_uint64, ctypes.POINTER(gsofa_result),
                                         ctypes.POINTER(ctypes.c_double)]),
    "gsofa_server_wait": (ctypes.c_int, [_P, ctypes.c_uint64, ctypes.c_double, ctypes.POINTER(gsofa_result),
                                         ctypes.POINTER(ctypes.c_double)]),
    "gsofa_server_get_stats": (ctypes.c_int, [_P, ctypes.POINTER(gsofa_server_stats)]),
    "gsofa_server_destroy": (None, [_P]),
    "gsofa_free": (None, [ctypes.POINTER(gsofa_result)]),
    "gsofa_strerror": (ctypes.c_char_p, [ctypes.c_int]),
    "gsofa_version": (ctypes.c_int, []),
}

_lock = threading.Lock()
_lib = None


def load(path: str | None = None):
    """Load libgsofa.so (built by ``paper_2007_00840_gb300.build``); raises if it is missing."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        p = path or LIB_PATH
        if not os.path.exists(p):
            raise RuntimeError(
                f"libgsofa.so not found at {p}; build it with `python -m paper_2007_00840_gb300.build` "
                "(the library has no CPU fallback)")
        lib = ctypes.CDLL(p)
        for name, (res, args) in SIGNATURES.items():
            f = getattr(lib, name)
            f.restype = res
            f.argtypes = args
        _lib = lib
        return lib


class GsofaError(RuntimeError):
    def __init__(self, code: int, detail: int = -1, where: str = ""):
        lib = _lib
        msg = lib.gsofa_strerror(code).decode() if lib is not None else str(code)
        super().__init__(f"{where}: {msg} (code {code}, detail {detail})")
        self.code = code
        self.detail = detail

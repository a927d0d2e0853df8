"""ctypes binding of libspcoarsen.so (argument marshalling only; every step runs in the CUDA
library).  The names mirror include/spcoarsen.h.

Loading fails loudly when the library has not been built: there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libspcoarsen.so")

SPC_OK = 0
SPC_WARN_TARGET_NOT_REACHED = 1
STATUS_NAMES = {
    0: "SPC_OK", 1: "SPC_WARN_TARGET_NOT_REACHED", -1: "SPC_ERR_INVALID_ARG",
    -2: "SPC_ERR_NOT_SYMMETRIC", -3: "SPC_ERR_SELF_LOOP", -4: "SPC_ERR_UNSORTED",
    -5: "SPC_ERR_OOM", -6: "SPC_ERR_CUDA", -7: "SPC_ERR_TIMEOUT", -8: "SPC_ERR_OVERFLOW",
    -9: "SPC_ERR_BAD_WEIGHT", -10: "SPC_ERR_TOO_LARGE",
}
SPC_I32, SPC_F32, SPC_F64 = 0, 1, 2


class SpcError(RuntimeError):
    def __init__(self, status: int, what: str = ""):
        self.status = status
        super().__init__(f"{what}: {STATUS_NAMES.get(status, status)}")


class spc_csr(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int64), ("nnz", ctypes.c_int64), ("rowptr", ctypes.c_void_p),
                ("col", ctypes.c_void_p), ("w", ctypes.c_void_p), ("wtype", ctypes.c_int)]


ALLOC_FN = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_void_p, ctypes.c_size_t)
FREE_FN = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_void_p)


class spc_allocator(ctypes.Structure):
    _fields_ = [("alloc", ALLOC_FN), ("free", FREE_FN), ("ctx", ctypes.c_void_p)]


class spc_options(ctypes.Structure):
    _fields_ = [("levels", ctypes.c_int32), ("validate", ctypes.c_int32),
                ("use_graph", ctypes.c_int32), ("schedule", ctypes.c_int32),
                ("self_mass", ctypes.c_int32), ("reorder", ctypes.c_int32)]


class spc_level(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int64), ("m", ctypes.c_int64), ("n_c", ctypes.c_int64),
                ("m_c", ctypes.c_int64), ("m_inter", ctypes.c_int64), ("status", ctypes.c_int32),
                ("wtype", ctypes.c_int), ("score", ctypes.c_void_p), ("scoretype", ctypes.c_int),
                ("lift", ctypes.c_void_p), ("emap", ctypes.c_void_p),
                ("self_mass", ctypes.c_void_p), ("a_und", ctypes.c_void_p),
                ("rowptr_c", ctypes.c_void_p), ("col_c", ctypes.c_void_p),
                ("w_c", ctypes.c_void_p), ("perm", ctypes.c_void_p), ("seg", ctypes.c_void_p),
                ("graph_ptr_c", ctypes.c_void_p), ("ms", ctypes.c_float),
                ("mass", ctypes.c_void_p)]


class spc_result(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int64), ("m", ctypes.c_int64), ("n_c", ctypes.c_int64),
                ("m_c", ctypes.c_int64), ("wtype", ctypes.c_int), ("lift", ctypes.c_void_p),
                ("emap", ctypes.c_void_p), ("rowptr_c", ctypes.c_void_p),
                ("col_c", ctypes.c_void_p), ("w_c", ctypes.c_void_p), ("mass", ctypes.c_void_p)]


# name -> (restype, argtypes); the full list of include/spcoarsen.h
P = ctypes.c_void_p
I64 = ctypes.c_int64
PI64 = ctypes.POINTER(ctypes.c_int64)
SIGNATURES = {
    "spc_context_create": (ctypes.c_int, [ctypes.POINTER(P), ctypes.POINTER(spc_allocator), P]),
    "spc_context_destroy": (None, [P]),
    "spc_context_set_stream": (ctypes.c_int, [P, P]),
    "spc_context_set_wait_limit": (ctypes.c_int, [P, ctypes.c_uint32]),
    "spc_status_string": (ctypes.c_char_p, [ctypes.c_int]),
    "spc_default_options": (spc_options, []),
    "spc_coarsen": (ctypes.c_int, [P, ctypes.POINTER(spc_csr), I64,
                                   ctypes.POINTER(spc_options), P, PI64]),
    "spc_coarsen_batched": (ctypes.c_int, [P, ctypes.POINTER(spc_csr), P, I64, I64,
                                           ctypes.POINTER(spc_options), P, P]),
    "spc_get_reorder": (ctypes.c_int, [P, P]),
    "spc_level_count": (ctypes.c_int32, [P]),
    "spc_get_level": (ctypes.c_int, [P, ctypes.c_int32, ctypes.POINTER(spc_level)]),
    "spc_copy": (ctypes.c_int, [P, P, P, ctypes.c_size_t]),
    "spc_take_result": (ctypes.c_int, [P, ctypes.POINTER(spc_result)]),
    "spc_result_free": (None, [P, ctypes.POINTER(spc_result)]),
    "spc_score": (ctypes.c_int, [P, ctypes.POINTER(spc_csr), P, PI64]),
    "spc_sort_fitness": (ctypes.c_int, [P, I64, P, ctypes.c_int, P]),
    "spc_select_merges": (ctypes.c_int, [P, ctypes.POINTER(spc_csr), P, I64, P, P, PI64]),
    "spc_contract": (ctypes.c_int, [P, ctypes.POINTER(spc_csr), P, I64, PI64]),
    "spc_contract_forward": (ctypes.c_int, [P, P, P, I64, P, ctypes.c_int, P]),
    "spc_contract_backward": (ctypes.c_int, [P, P, I64, P, P, ctypes.c_int]),
    "spc_compose_emap": (ctypes.c_int, [P, P]),
    "spc_pool_features": (ctypes.c_int, [P, I64, P, I64, I64, ctypes.c_int, P, P]),
    "spc_pool_features_backward": (ctypes.c_int, [P, I64, P, I64, I64, ctypes.c_int, P, P]),
    "spc_sort_fitness_static": (ctypes.c_int, [I64, P, ctypes.c_int, P, P]),
    "spc_time_kernel": (ctypes.c_int, [P, ctypes.c_char_p]),
    "spc_kernel_time": (ctypes.c_int, [P, PI64, ctypes.POINTER(ctypes.c_double)]),
    "spc_kernel_profile": (ctypes.c_int, [P, ctypes.c_char_p, ctypes.c_size_t]),
    "spc_launch_count": (ctypes.c_int64, [P]),
    "spc_last_call_replayed": (ctypes.c_int, [P]),
}

_lib = None


def lib():
    """Load libspcoarsen.so (raises if it was not built -- there is no fallback)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"{LIB_PATH} is missing: build it with __graft_entry__.build() "
                              "(python paper_2204_11757_gb300/build.py)")
        L = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


def check(status: int, what: str) -> int:
    """Raise SpcError for negative status codes; return warnings (>= 0) unchanged."""
    if status < 0:
        raise SpcError(status, what)
    return status

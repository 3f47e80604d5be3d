"""ctypes loader of libperm.so (the C ABI in include/perm.h).

Argument marshalling only.  The library is built in-tree by build.py; when it
is missing this module raises instead of falling back to anything else.
"""
from __future__ import annotations

import ctypes
import os

from . import build as _build

PERM_F64, PERM_C128, PERM_BIN, PERM_F64X = 0, 1, 2, 3
PERM_SPARSE_PAPER_ORDER = 1
PERM_OK, PERM_EINVAL, PERM_ERANGE, PERM_EOVERFLOW, PERM_ECUDA, PERM_ENOMEM, PERM_EABORTED, PERM_ETIMEOUT = range(8)

_vp = ctypes.c_void_p
_i32p = ctypes.POINTER(ctypes.c_int32)
_lib = None

SYMBOLS = ("perm", "perm_range", "perm_combine", "perm_sparse", "perm_sparse_range", "perm_host", "perm_pipe_peaks",
           "perm_batched_plan_create", "perm_batched_plan_create_labeled", "perm_batched_units", "perm_batched", "perm_batched_autotune", "perm_batched_plan_info",
           "perm_batched_plan_destroy", "perm_grad", "perm_grad_batched", "perm_grad_batched_mixed", "perm_grad_plan_create", "perm_grad_plan_run", "perm_grad_plan_destroy", "perm_decomp_create", "perm_decomp_info", "perm_decomp_leaf",
           "perm_decomp_filtered", "perm_decomp_eval", "perm_decomp_destroy", "perm_sparse_decomp",
           "perm_set_abort_word", "perm_abort_word_alloc", "perm_abort_word_free", "perm_set_time_budget",
           "perm_status_string", "perm_abi_version")


class DecompInfo(ctypes.Structure):
    """perm_decomp_info_t of include/perm.h."""
    _fields_ = [("n", ctypes.c_int), ("nblocks", ctypes.c_int), ("nleaves", ctypes.c_int),
                ("max_leaf_n", ctypes.c_int), ("structurally_zero", ctypes.c_int), ("truncated", ctypes.c_int),
                ("removed_nnz", ctypes.c_int64), ("leaf_steps", ctypes.c_double), ("plain_steps", ctypes.c_double)]


class PermError(RuntimeError):
    """A nonzero perm_status_t from the library; .code holds it."""

    def __init__(self, code: int, what: str = ""):
        self.code = int(code)
        super().__init__(f"{what}: {status_string(code)}" if what else status_string(code))


def lib_path() -> str:
    """Path of the in-tree libperm.so."""
    return _build.LIB


def load(build_if_missing: bool = False):
    """Load libperm.so.  Raises if it was not built (no fallback path exists)."""
    global _lib
    if _lib is not None:
        return _lib
    path = lib_path()
    if not os.path.exists(path):
        if not build_if_missing:
            raise ImportError(f"libperm.so not built ({path}); run paper_2502_16577_gb300.build.build()")
        _build.build()
    lib = ctypes.CDLL(path)
    lib.perm.restype = ctypes.c_int
    lib.perm.argtypes = [_vp, ctypes.c_int, ctypes.c_int, _vp, _vp, _vp]
    lib.perm_range.restype = ctypes.c_int
    lib.perm_range.argtypes = [_vp, ctypes.c_int, ctypes.c_int, ctypes.c_uint64, ctypes.c_uint64, _vp, _vp, _vp]
    lib.perm_combine.restype = ctypes.c_int
    lib.perm_combine.argtypes = [ctypes.c_int, ctypes.c_int, _vp, ctypes.c_int, _vp]
    lib.perm_sparse.restype = ctypes.c_int
    lib.perm_sparse.argtypes = [ctypes.c_int, _vp, _vp, _vp, ctypes.c_int64, _vp, _vp, _vp]
    lib.perm_sparse_range.restype = ctypes.c_int
    lib.perm_sparse_range.argtypes = [ctypes.c_int, _vp, _vp, _vp, ctypes.c_int64, ctypes.c_uint64, ctypes.c_uint64,
                                      ctypes.c_int, _vp, _vp, _vp]
    lib.perm_batched_plan_create.restype = ctypes.c_int
    lib.perm_batched_plan_create.argtypes = [ctypes.POINTER(_vp), ctypes.c_int, ctypes.POINTER(ctypes.c_int),
                                             ctypes.c_int, _vp, ctypes.POINTER(ctypes.c_int64), _vp, _vp]
    lib.perm_batched_plan_create_labeled.restype = ctypes.c_int
    lib.perm_batched_plan_create_labeled.argtypes = [ctypes.POINTER(_vp), ctypes.c_int, ctypes.POINTER(ctypes.c_int),
                                                     ctypes.c_int, _vp, ctypes.POINTER(ctypes.c_int64), _vp, _vp,
                                                     ctypes.POINTER(ctypes.c_int32)]
    lib.perm_batched_units.restype = ctypes.c_int
    lib.perm_batched_units.argtypes = [ctypes.c_int, _vp, ctypes.c_int, _vp, _vp, _vp, ctypes.c_int, _vp]
    lib.perm_batched.restype = ctypes.c_int
    lib.perm_batched.argtypes = [_vp, _vp, _vp, _vp, _vp]
    lib.perm_batched_autotune.restype = ctypes.c_int
    lib.perm_batched_autotune.argtypes = [_vp, ctypes.c_int, _vp]
    lib.perm_batched_plan_info.restype = ctypes.c_int
    lib.perm_batched_plan_info.argtypes = [_vp, ctypes.c_int, ctypes.POINTER(ctypes.c_int),
                                           ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int)]
    lib.perm_batched_plan_destroy.restype = None
    lib.perm_batched_plan_destroy.argtypes = [_vp]
    lib.perm_grad.restype = ctypes.c_int
    lib.perm_grad.argtypes = [_vp, ctypes.c_int, ctypes.c_int, _vp, _vp, _vp, _vp]
    lib.perm_grad_batched.restype = ctypes.c_int
    lib.perm_grad_batched.argtypes = [_vp, ctypes.c_int, ctypes.c_int, ctypes.c_int, _vp, _vp, _vp, _vp]
    lib.perm_grad_batched_mixed.restype = ctypes.c_int
    lib.perm_grad_batched_mixed.argtypes = [ctypes.c_int, ctypes.POINTER(ctypes.c_int), ctypes.c_int, _vp,
                                            ctypes.POINTER(ctypes.c_int64), _vp, _vp, _vp, _vp]
    _dp = ctypes.POINTER(ctypes.c_double)
    _ip = ctypes.POINTER(ctypes.c_int)
    lib.perm_grad_plan_create.restype = ctypes.c_int
    lib.perm_grad_plan_create.argtypes = [ctypes.POINTER(_vp), ctypes.c_int, ctypes.POINTER(ctypes.c_int), ctypes.c_int,
                                          ctypes.POINTER(ctypes.c_int64)]
    lib.perm_grad_plan_run.restype = ctypes.c_int
    lib.perm_grad_plan_run.argtypes = [_vp, _vp, _vp, _vp, _vp, _vp]
    lib.perm_grad_plan_destroy.restype = None
    lib.perm_grad_plan_destroy.argtypes = [_vp]
    lib.perm_decomp_create.restype = ctypes.c_int
    lib.perm_decomp_create.argtypes = [ctypes.POINTER(_vp), ctypes.c_int, _vp, _vp, _vp, ctypes.c_int64, ctypes.c_int]
    lib.perm_decomp_info.restype = ctypes.c_int
    lib.perm_decomp_info.argtypes = [_vp, ctypes.POINTER(DecompInfo)]
    lib.perm_decomp_leaf.restype = ctypes.c_int
    lib.perm_decomp_leaf.argtypes = [_vp, ctypes.c_int, _ip, _ip, _dp, _vp]
    lib.perm_decomp_filtered.restype = ctypes.c_int
    lib.perm_decomp_filtered.argtypes = [_vp, _vp]
    lib.perm_decomp_eval.restype = ctypes.c_int
    lib.perm_decomp_eval.argtypes = [_vp, _dp, _vp]
    lib.perm_decomp_destroy.restype = None
    lib.perm_decomp_destroy.argtypes = [_vp]
    lib.perm_sparse_decomp.restype = ctypes.c_int
    lib.perm_sparse_decomp.argtypes = [ctypes.c_int, _vp, _vp, _vp, ctypes.c_int64, _dp, ctypes.POINTER(DecompInfo),
                                       _vp]
    lib.perm_set_time_budget.restype = ctypes.c_int
    lib.perm_set_time_budget.argtypes = [ctypes.c_uint64]
    lib.perm_set_abort_word.restype = ctypes.c_int
    lib.perm_set_abort_word.argtypes = [_vp]
    lib.perm_abort_word_alloc.restype = ctypes.c_int
    lib.perm_abort_word_alloc.argtypes = [ctypes.POINTER(ctypes.POINTER(ctypes.c_uint32))]
    lib.perm_abort_word_free.restype = ctypes.c_int
    lib.perm_abort_word_free.argtypes = [ctypes.POINTER(ctypes.c_uint32)]
    lib.perm_host.restype = ctypes.c_int
    lib.perm_host.argtypes = [_vp, ctypes.c_int, ctypes.c_int, _vp, _vp]
    lib.perm_pipe_peaks.restype = ctypes.c_int
    lib.perm_pipe_peaks.argtypes = [ctypes.POINTER(ctypes.c_double), ctypes.c_int, _vp]
    lib.perm_status_string.restype = ctypes.c_char_p
    lib.perm_status_string.argtypes = [ctypes.c_int]
    lib.perm_abi_version.restype = ctypes.c_int
    lib.perm_abi_version.argtypes = []
    _lib = lib
    return lib


def status_string(code: int) -> str:
    """The library's text for a perm_status_t code."""
    try:
        return load().perm_status_string(int(code)).decode()
    except ImportError:
        return f"status {code}"


def check(code: int, what: str = "") -> None:
    """Raise PermError for a nonzero perm_status_t."""
    if int(code) != PERM_OK:
        raise PermError(code, what)

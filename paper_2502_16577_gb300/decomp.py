"""Sparse preprocessing of Sec. 4 through the C ABI (perm_decomp_*): the
Dulmage-Mendelsohn filter and block split, then Forbert-Marx expansions
(Alg. 4) into weighted leaves whose permanents the GPU kernels compute.

The graph work itself is native (csrc/decomp.cu); this module marshals a
host CCS matrix in and the leaves / info out."""
from __future__ import annotations

import ctypes

import numpy as np

from ._lib import DecompInfo, check, load


def _ccs(A=None, n=None, cptrs=None, rids=None, cvals=None):
    if A is not None:
        A = np.ascontiguousarray(np.asarray(A, dtype=np.float64))
        if A.ndim != 2 or A.shape[0] != A.shape[1]:
            raise ValueError("A must be square")
        n = A.shape[0]
        cp, ri, cv = [0], [], []
        for j in range(n):
            nz = np.nonzero(A[:, j])[0]
            ri.extend(nz.tolist())
            cv.extend(A[nz, j].tolist())
            cp.append(len(ri))
        cptrs, rids, cvals = cp, ri, cv
    cptrs = np.ascontiguousarray(np.asarray(cptrs, dtype=np.int32))
    rids = np.ascontiguousarray(np.asarray(rids, dtype=np.int32))
    cvals = np.ascontiguousarray(np.asarray(cvals, dtype=np.float64))
    return int(n), cptrs, rids, cvals


def _ptr(a):
    return ctypes.c_void_p(a.ctypes.data) if a.size else ctypes.c_void_p(0)


class SparseDecomposition:
    """Decomposition of one sparse real matrix (a dense numpy array, or
    n with CCS arrays); eval() computes perm(A) with the leaves on the GPU."""

    def __init__(self, A=None, *, n=None, cptrs=None, rids=None, cvals=None, max_leaves: int = 0):
        self._lib = load()
        self.n, cp, ri, cv = _ccs(A, n, cptrs, rids, cvals)
        h = ctypes.c_void_p()
        check(self._lib.perm_decomp_create(ctypes.byref(h), self.n, _ptr(cp), _ptr(ri), _ptr(cv), len(cv),
                                           int(max_leaves)), "perm_decomp_create")
        self._h = h

    def info(self) -> dict:
        """Blocks, leaves and the Gray steps of the leaves against the plain sweep."""
        inf = DecompInfo()
        check(self._lib.perm_decomp_info(self._h, ctypes.byref(inf)), "perm_decomp_info")
        return {f: getattr(inf, f) for f, _ in DecompInfo._fields_}

    def leaves(self):
        """[(block, coef, leaf matrix)] with perm(A) = prod_b sum_{leaves of b} coef * perm(leaf)."""
        out = []
        for k in range(self.info()["nleaves"]):
            n, b, c = ctypes.c_int(), ctypes.c_int(), ctypes.c_double()
            check(self._lib.perm_decomp_leaf(self._h, k, ctypes.byref(n), ctypes.byref(b), ctypes.byref(c), None),
                  "perm_decomp_leaf")
            M = np.zeros((n.value, n.value))
            check(self._lib.perm_decomp_leaf(self._h, k, None, None, None, _ptr(M) if M.size else None),
                  "perm_decomp_leaf")
            out.append((b.value, c.value, M))
        return out

    def filtered(self) -> np.ndarray:
        """A after the Dulmage-Mendelsohn step (entries on no perfect matching zeroed)."""
        M = np.zeros((self.n, self.n))
        if self.n:
            check(self._lib.perm_decomp_filtered(self._h, _ptr(M)), "perm_decomp_filtered")
        return M

    def eval(self, stream=None) -> float:
        """perm(A) from the leaves on the GPU, recombined on the host."""
        out = ctypes.c_double()
        h = ctypes.c_void_p(stream.cuda_stream) if stream is not None else ctypes.c_void_p(0)
        check(self._lib.perm_decomp_eval(self._h, ctypes.byref(out), h), "perm_decomp_eval")
        return out.value

    def close(self):
        if getattr(self, "_h", None):
            self._lib.perm_decomp_destroy(self._h)
            self._h = None

    def __del__(self):
        self.close()


def perm_sparse_decomp(A=None, *, n=None, cptrs=None, rids=None, cvals=None, stream=None):
    """perm(A) of a sparse real matrix through the Sec. 4 preprocessing; returns
    (value, info dict)."""
    lib = load()
    n, cp, ri, cv = _ccs(A, n, cptrs, rids, cvals)
    out = ctypes.c_double()
    inf = DecompInfo()
    h = ctypes.c_void_p(stream.cuda_stream) if stream is not None else ctypes.c_void_p(0)
    check(lib.perm_sparse_decomp(n, _ptr(cp), _ptr(ri), _ptr(cv), len(cv), ctypes.byref(out), ctypes.byref(inf), h),
          "perm_sparse_decomp")
    return out.value, {f: getattr(inf, f) for f, _ in DecompInfo._fields_}

"""Plain CPU oracle for matrix permanents (arXiv:2502.16577).

TEST INFRASTRUCTURE ONLY.  ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` are the only
callers.  The CUDA library never imports or links this package, and this
package imports nothing from the library.

Two layers:

* ``ryser.c`` (loaded through ctypes): Alg. 1 (RYSER in Nijenhuis-Wilf form,
  Eq. nwx) chunked over threads as in Alg. 3 (PARRYSER), for real FP64
  (double-double partial sums, Sec. 5), real with double-double x and products,
  complex128, complex with x and products in double-double, rounding-error
  magnitude sums (Sec. 5), Alg. 2 (SPARYSER on CRS + CCS), exact 0/1 (Eq. 2 without halving
  and Alg. 1 with doubled rows, both mod 2^128), and a row-by-row subset
  expansion of Eq. 1 that uses neither Ryser nor Gray codes.
* pure Python, exact big integers / fractions: brute force over permutations
  (Eq. 1, n <= 9) and closed forms used as pins (n!, derangements, ménage
  numbers, Fibonacci numbers, the Bregman bound).

Every function here is pinned by ``tests/test_oracle_*.py``.
"""
from __future__ import annotations

import ctypes
import itertools
import math
import os
from fractions import Fraction

import numpy as np

from . import build as _build

_u64 = ctypes.c_uint64
_dp = ctypes.POINTER(ctypes.c_double)
_i32p = ctypes.POINTER(ctypes.c_int32)
_u8p = ctypes.POINTER(ctypes.c_uint8)
_u64p = ctypes.POINTER(ctypes.c_uint64)
_ip = ctypes.POINTER(ctypes.c_int)

_LIBS: dict = {}


def default_threads() -> int:
    return max(1, os.cpu_count() or 1)


def load(mutant: int = 0):
    """Load (building if needed) the oracle library, or a planted-mistake variant."""
    if mutant in _LIBS:
        return _LIBS[mutant]
    path = _build.build(mutant)
    lib = ctypes.CDLL(path)
    lib.oracle_gray.restype = _u64
    lib.oracle_gray.argtypes = [_u64]
    lib.oracle_changed_bit.restype = ctypes.c_int
    lib.oracle_changed_bit.argtypes = [_u64]
    lib.oracle_cbl.restype = ctypes.c_int
    lib.oracle_cbl.argtypes = [ctypes.c_int, _ip]
    for name in ("oracle_ryser_f64_range", "oracle_ryser_dd_range", "oracle_ryser_c128_range"):
        f = getattr(lib, name)
        f.restype = ctypes.c_int
        f.argtypes = [_dp, ctypes.c_int, _u64, _u64, ctypes.c_int, _dp]
    for name in ("oracle_ryser_dd_stats_range", "oracle_ryser_cdd_range"):
        f = getattr(lib, name)
        f.restype = ctypes.c_int
        f.argtypes = [_dp, ctypes.c_int, _u64, _u64, ctypes.c_int, _dp]
    for name in ("oracle_perm_f64", "oracle_perm_dd", "oracle_perm_c128"):
        f = getattr(lib, name)
        f.restype = ctypes.c_int
        f.argtypes = [_dp, ctypes.c_int, ctypes.c_int, _dp]
    lib.oracle_spa_ryser_f64_range.restype = ctypes.c_int
    lib.oracle_spa_ryser_f64_range.argtypes = [ctypes.c_int, _i32p, _i32p, _dp, _i32p, _i32p, _dp, _u64, _u64,
                                               ctypes.c_int, _dp]
    lib.oracle_ryser_bin_plain.restype = ctypes.c_int
    lib.oracle_ryser_bin_plain.argtypes = [_u8p, ctypes.c_int, ctypes.c_int, _u64p]
    lib.oracle_ryser_bin_range.restype = ctypes.c_int
    lib.oracle_ryser_bin_range.argtypes = [_u8p, ctypes.c_int, _u64, _u64, ctypes.c_int, _u64p]
    lib.oracle_perm_dp_f64.restype = ctypes.c_int
    lib.oracle_perm_dp_f64.argtypes = [_dp, ctypes.c_int, _dp]
    lib.oracle_perm_dp_c128.restype = ctypes.c_int
    lib.oracle_perm_dp_c128.argtypes = [_dp, ctypes.c_int, _dp]
    lib.oracle_perm_dp_bin.restype = ctypes.c_int
    lib.oracle_perm_dp_bin.argtypes = [_u8p, ctypes.c_int, _u64p]
    _LIBS[mutant] = lib
    return lib


def _check(rc: int, what: str) -> None:
    if rc != 0:
        raise ValueError(f"oracle {what} failed with code {rc}")


def _real(A) -> np.ndarray:
    A = np.ascontiguousarray(np.asarray(A, dtype=np.float64))
    if A.ndim != 2 or A.shape[0] != A.shape[1]:
        raise ValueError("square matrix expected")
    return A


def _cplx(A) -> np.ndarray:
    A = np.ascontiguousarray(np.asarray(A, dtype=np.complex128))
    if A.ndim != 2 or A.shape[0] != A.shape[1]:
        raise ValueError("square matrix expected")
    return A


def _bin(A) -> np.ndarray:
    A = np.asarray(A)
    if A.ndim != 2 or A.shape[0] != A.shape[1]:
        raise ValueError("square matrix expected")
    if not np.all((A == 0) | (A == 1)):
        raise ValueError("0/1 matrix expected")
    return np.ascontiguousarray(A.astype(np.uint8))


def _u128(lo_hi) -> int:
    return int(lo_hi[0]) | (int(lo_hi[1]) << 64)


# ------------------------------------------------------------------- Gray code

def gray(g: int, mutant: int = 0) -> int:
    """Gray_g = g xor (g >> 1) (Sec. 2, Table 1)."""
    return int(load(mutant).oracle_gray(g))


def changed_bit(g: int, mutant: int = 0) -> int:
    """log2(Gray_g xor Gray_{g-1}), g >= 1 (Table 1, Alg. 1)."""
    return int(load(mutant).oracle_changed_bit(g))


def cbl(k: int, mutant: int = 0) -> list:
    """CBL_k built by the reflection recursion of Sec. 3.1.1."""
    buf = (ctypes.c_int * ((1 << k) - 1))()
    n = load(mutant).oracle_cbl(k, buf)
    _check(0 if n == (1 << k) - 1 else -1, "cbl")
    return list(buf)


# -------------------------------------------------------- Ryser (Alg. 1 / Alg. 3)

def ryser_f64_range(A, g0: int, g1: int, threads: int | None = None, mutant: int = 0) -> tuple:
    """Sum over g in [g0, g1) of (-1)^g prod_i x_i(g) (Alg. 1's x), as (hi, lo)."""
    A = _real(A)
    out = (ctypes.c_double * 2)()
    rc = load(mutant).oracle_ryser_f64_range(A.ctypes.data_as(_dp), A.shape[0], g0, g1,
                                             threads or default_threads(), out)
    _check(rc, "ryser_f64_range")
    return out[0], out[1]


def perm_f64(A, threads: int | None = None, mutant: int = 0) -> float:
    """perm(A) by Alg. 1/3 in FP64 with double-double partial sums."""
    A = _real(A)
    out = (ctypes.c_double * 1)()
    rc = load(mutant).oracle_perm_f64(A.ctypes.data_as(_dp), A.shape[0], threads or default_threads(), out)
    _check(rc, "perm_f64")
    return out[0]


def ryser_dd_range(A, g0: int, g1: int, threads: int | None = None) -> tuple:
    """As ryser_f64_range with x and every product in double-double."""
    A = _real(A)
    out = (ctypes.c_double * 2)()
    rc = load().oracle_ryser_dd_range(A.ctypes.data_as(_dp), A.shape[0], g0, g1, threads or default_threads(), out)
    _check(rc, "ryser_dd_range")
    return out[0], out[1]


def perm_dd(A, threads: int | None = None) -> tuple:
    """perm(A) as an unevaluated double-double (hi, lo), high-precision mode."""
    A = _real(A)
    out = (ctypes.c_double * 2)()
    rc = load().oracle_perm_dd(A.ctypes.data_as(_dp), A.shape[0], threads or default_threads(), out)
    _check(rc, "perm_dd")
    return out[0], out[1]


def ryser_dd_stats_range(A, g0: int, g1: int, threads: int | None = None, mutant: int = 0) -> dict:
    """The double-double range sum of ryser_dd_range plus two magnitude sums
    (Sec. 5's error analysis): S = sum_g |prod_i x_i(g)| and
    W = sum_g sum_i R_i prod_{k != i} |x_k(g)| with R_i = sum_j |a_ij|.
    Returns {"hi", "lo", "S", "W"}."""
    A = _real(A)
    out = (ctypes.c_double * 4)()
    rc = load(mutant).oracle_ryser_dd_stats_range(A.ctypes.data_as(_dp), A.shape[0], g0, g1,
                                                  threads or default_threads(), out)
    _check(rc, "ryser_dd_stats_range")
    return {"hi": out[0], "lo": out[1], "S": out[2], "W": out[3]}


def ryser_cdd_range(A, g0: int, g1: int, threads: int | None = None, mutant: int = 0) -> dict:
    """Complex range sum with x and every product in double-double, plus S and W
    as in ryser_dd_stats_range (moduli of complex values).  Returns
    {"re_hi", "re_lo", "im_hi", "im_lo", "S", "W"}."""
    A = _cplx(A)
    out = (ctypes.c_double * 6)()
    rc = load(mutant).oracle_ryser_cdd_range(A.view(np.float64).ctypes.data_as(_dp), A.shape[0], g0, g1,
                                             threads or default_threads(), out)
    _check(rc, "ryser_cdd_range")
    return {"re_hi": out[0], "re_lo": out[1], "im_hi": out[2], "im_lo": out[3], "S": out[4], "W": out[5]}


def ryser_c128_range(A, g0: int, g1: int, threads: int | None = None) -> complex:
    """Complex range sum; returns (re_hi, re_lo, im_hi, im_lo)."""
    A = _cplx(A)
    out = (ctypes.c_double * 4)()
    rc = load().oracle_ryser_c128_range(A.view(np.float64).ctypes.data_as(_dp), A.shape[0], g0, g1,
                                        threads or default_threads(), out)
    _check(rc, "ryser_c128_range")
    return tuple(out)


def perm_c128(A, threads: int | None = None) -> complex:
    A = _cplx(A)
    out = (ctypes.c_double * 2)()
    rc = load().oracle_perm_c128(A.view(np.float64).ctypes.data_as(_dp), A.shape[0], threads or default_threads(), out)
    _check(rc, "perm_c128")
    return complex(out[0], out[1])


# ------------------------------------------------------------ sparse (Alg. 2)

def to_crs_ccs(A):
    """CRS (rptrs, cids, rvals) and CCS (cptrs, rids, cvals) of a dense matrix (Fig. 1)."""
    A = _real(A)
    n = A.shape[0]
    rptrs, cids, rvals = [0], [], []
    for i in range(n):
        for j in range(n):
            if A[i, j] != 0.0:
                cids.append(j)
                rvals.append(A[i, j])
        rptrs.append(len(cids))
    cptrs, rids, cvals = [0], [], []
    for j in range(n):
        for i in range(n):
            if A[i, j] != 0.0:
                rids.append(i)
                cvals.append(A[i, j])
        cptrs.append(len(rids))
    i32 = lambda v: np.ascontiguousarray(np.asarray(v, dtype=np.int32))
    f64 = lambda v: np.ascontiguousarray(np.asarray(v, dtype=np.float64))
    return (i32(rptrs), i32(cids), f64(rvals)), (i32(cptrs), i32(rids), f64(cvals))


def spa_ryser_range(n: int, crs, ccs, g0: int, g1: int, threads: int | None = None) -> tuple:
    rptrs, cids, rvals = crs
    cptrs, rids, cvals = ccs
    out = (ctypes.c_double * 2)()
    rc = load().oracle_spa_ryser_f64_range(n, rptrs.ctypes.data_as(_i32p), cids.ctypes.data_as(_i32p),
                                           rvals.ctypes.data_as(_dp), cptrs.ctypes.data_as(_i32p),
                                           rids.ctypes.data_as(_i32p), cvals.ctypes.data_as(_dp), g0, g1,
                                           threads or default_threads(), out)
    _check(rc, "spa_ryser_range")
    return out[0], out[1]


def perm_sparse(n: int, crs, ccs, threads: int | None = None) -> float:
    if n == 0:
        return 1.0
    hi, lo = spa_ryser_range(n, crs, ccs, 0, 1 << (n - 1), threads)
    return (hi + lo) * (4.0 * (n % 2) - 2.0)


# --------------------------------------------------------------- binary, exact

def perm_bin_plain(A, threads: int | None = None) -> int:
    """perm(A) mod 2^128 by Eq. 2 over all 2^n subsets (exact integers)."""
    A = _bin(A)
    out = (ctypes.c_uint64 * 2)()
    rc = load().oracle_ryser_bin_plain(A.ctypes.data_as(_u8p), A.shape[0], threads or default_threads(), out)
    _check(rc, "ryser_bin_plain")
    return _u128(out)


def ryser_bin_range(A, g0: int, g1: int, threads: int | None = None) -> int:
    """Sum over g in [g0, g1) of (-1)^g prod_i x'_i(g), x' = 2x, mod 2^128."""
    A = _bin(A)
    out = (ctypes.c_uint64 * 2)()
    rc = load().oracle_ryser_bin_range(A.ctypes.data_as(_u8p), A.shape[0], g0, g1, threads or default_threads(), out)
    _check(rc, "ryser_bin_range")
    return _u128(out)


# ------------------------------------------------------- Eq. 1, subset expansion

def perm_dp_f64(A) -> float:
    A = _real(A)
    out = (ctypes.c_double * 1)()
    _check(load().oracle_perm_dp_f64(A.ctypes.data_as(_dp), A.shape[0], out), "perm_dp_f64")
    return out[0]


def perm_dp_c128(A) -> complex:
    A = _cplx(A)
    out = (ctypes.c_double * 2)()
    _check(load().oracle_perm_dp_c128(A.view(np.float64).ctypes.data_as(_dp), A.shape[0], out), "perm_dp_c128")
    return complex(out[0], out[1])


def perm_dp_bin(A) -> int:
    A = _bin(A)
    out = (ctypes.c_uint64 * 2)()
    _check(load().oracle_perm_dp_bin(A.ctypes.data_as(_u8p), A.shape[0], out), "perm_dp_bin")
    return _u128(out)


# ---------------------------------------------------- Eq. 1 brute force, exact

def perm_bruteforce(A):
    """Eq. 1 summed over all n! permutations.

    Integer / Fraction / complex entries are summed exactly (Python numbers);
    float entries are converted to Fraction first, so the result is the exact
    permanent of the given binary64 values (returned as a Fraction).
    """
    rows = [list(r) for r in A]
    n = len(rows)
    if n == 0:
        return 1
    cplx = any(isinstance(v, complex) or isinstance(v, np.complexfloating) for r in rows for v in r)
    if cplx:
        conv = lambda v: (Fraction(complex(v).real), Fraction(complex(v).imag))
        M = [[conv(v) for v in r] for r in rows]
        tr, ti = Fraction(0), Fraction(0)
        for sigma in itertools.permutations(range(n)):
            pr, pi = Fraction(1), Fraction(0)
            for i in range(n):
                ar, ai = M[i][sigma[i]]
                pr, pi = pr * ar - pi * ai, pr * ai + pi * ar
            tr += pr
            ti += pi
        return tr, ti
    conv = (lambda v: Fraction(float(v))) if any(isinstance(v, (float, np.floating)) for r in rows for v in r) \
        else (lambda v: int(v))
    M = [[conv(v) for v in r] for r in rows]
    total = 0
    for sigma in itertools.permutations(range(n)):
        p = 1
        for i in range(n):
            p *= M[i][sigma[i]]
            if p == 0:
                break
        total += p
    return total


# ------------------------------------------------------------------ closed forms

def factorial(n: int) -> int:
    """perm(J_n) = n! (every permutation contributes 1)."""
    return math.factorial(n)


def derangements(n: int) -> int:
    """perm(J_n - I_n) = D_n, D_0 = 1, D_1 = 0, D_n = (n-1)(D_{n-1} + D_{n-2})."""
    a, b = 1, 0
    if n == 0:
        return 1
    for k in range(2, n + 1):
        a, b = b, (k - 1) * (a + b)
    return b


def fibonacci(k: int) -> int:
    """F_0 = 0, F_1 = 1 (Sec. 1); perm of the n x n all-ones tridiagonal matrix is F_{n+1}."""
    a, b = 0, 1
    for _ in range(k):
        a, b = b, a + b
    return a


def menage(n: int) -> int:
    """Touchard's formula: number of permutations sigma with sigma(i) not in {i, i+1 mod n};
    equals perm(J - I - P) for the cyclic shift P, n >= 3."""
    if n == 0:
        return 1
    total = Fraction(0)
    for k in range(0, n + 1):
        total += Fraction((-1) ** k * 2 * n, 2 * n - k) * math.comb(2 * n - k, k) * math.factorial(n - k)
    assert total.denominator == 1
    return int(total)


def bregman_log2(A) -> float:
    """log2 of Bregman's bound perm(A) <= prod_i (r_i!)^(1/r_i) for a 0/1 matrix."""
    A = _bin(A)
    s = 0.0
    for r in A.sum(axis=1):
        r = int(r)
        if r == 0:
            return float("-inf")
        s += math.lgamma(r + 1) / r / math.log(2)
    return s

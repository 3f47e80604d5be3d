"""Seeded synthetic inputs shaped like the workloads of arXiv:2502.16577.

This module only draws and lays out matrices; it holds none of the permanent
arithmetic.  Both the oracle's tests and the CUDA library's tests and
benchmark take their inputs from here, so the two sides see identical bytes.

Recipes (all seeded with ``numpy.random.default_rng``):

* dense real: i.i.d. uniform entries, ``lo + (hi - lo) * rng.random``; for
  [0, 1) and [-1, 1) every value is a multiple of 2^-53 (2^-52), as the
  dense random FP64 matrices of Table 4;
* binary: i.i.d. Bernoulli(p) 0/1 entries (uint8);
* complex: a Haar-random unitary by QR of a complex Ginibre matrix with the
  phases of R's diagonal divided out (Mezzadri's method), as the boson-sampling
  unitaries of Sec. 1;
* sparse: a Bernoulli(density) nonzero mask with at least one nonzero in every
  row and column and a perfect matching (so the permanent is not structurally
  zero), values ``1 - rng.random()`` in (0, 1], laid out as CCS (Fig. 1);
* batched boson submatrices: k x k blocks (k uniform in [kmin, kmax]) made of k
  rows drawn with replacement from a Haar 256 x 256 unitary, first k columns.
"""
from __future__ import annotations

import numpy as np

SEED_BASE = 20250223


def rng(seed: int) -> np.random.Generator:
    return np.random.default_rng(seed)


# ----------------------------------------------------------------- dense real

def uniform_real(n: int, seed: int, lo: float = 0.0, hi: float = 1.0) -> np.ndarray:
    r = rng(seed).random((n, n))
    if lo == 0.0 and hi == 1.0:
        return r
    return lo + (hi - lo) * r


def signed_real(n: int, seed: int) -> np.ndarray:
    """Uniform [-1, 1): 2 u - 1, exact in binary64."""
    return 2.0 * rng(seed).random((n, n)) - 1.0


def constant(n: int, a: float) -> np.ndarray:
    return np.full((n, n), float(a))


# --------------------------------------------------------------------- binary

def bernoulli01(n: int, seed: int, p: float = 0.5) -> np.ndarray:
    return (rng(seed).random((n, n)) < p).astype(np.uint8)


def ones(n: int) -> np.ndarray:
    return np.ones((n, n), dtype=np.uint8)


def derangement_matrix(n: int) -> np.ndarray:
    """J_n - I_n."""
    return (1 - np.eye(n, dtype=np.uint8)).astype(np.uint8)


def menage_matrix(n: int) -> np.ndarray:
    """J_n - I_n - P_n with P_n the cyclic shift i -> i+1 (mod n)."""
    M = np.ones((n, n), dtype=np.uint8)
    for i in range(n):
        M[i, i] = 0
        M[i, (i + 1) % n] = 0
    return M


def tridiagonal_ones(n: int) -> np.ndarray:
    M = np.zeros((n, n), dtype=np.uint8)
    for i in range(n):
        for j in range(max(0, i - 1), min(n, i + 2)):
            M[i, j] = 1
    return M


# ------------------------------------------------------------------- complex

def haar_unitary(m: int, seed: int) -> np.ndarray:
    g = rng(seed)
    Z = (g.standard_normal((m, m)) + 1j * g.standard_normal((m, m))) / np.sqrt(2.0)
    Q, R = np.linalg.qr(Z)
    d = np.diagonal(R)
    return np.ascontiguousarray(Q * (d / np.abs(d)))


def complex_uniform(n: int, seed: int) -> np.ndarray:
    g = rng(seed)
    return (2.0 * g.random((n, n)) - 1.0) + 1j * (2.0 * g.random((n, n)) - 1.0)


def boson_submatrices(count: int, seed: int, kmin: int = 8, kmax: int = 26, m: int = 256,
                      with_rows: bool = False):
    """k x k submatrices: k rows drawn with replacement from a Haar m x m unitary,
    its first k columns; k uniform in [kmin, kmax].  with_rows: also return the
    drawn row (mode) indices of every matrix, which label its equal rows."""
    U = haar_unitary(m, seed)
    g = rng(seed + 1)
    ks = g.integers(kmin, kmax + 1, size=count)
    out, idx = [], []
    for k in ks:
        rows = g.integers(0, m, size=int(k))
        out.append(np.ascontiguousarray(U[rows, : int(k)]))
        idx.append(rows.astype(np.int32))
    return (out, idx) if with_rows else out


# -------------------------------------------------------------------- sparse

def _has_perfect_matching(mask: np.ndarray) -> bool:
    """Kuhn's augmenting paths on the bipartite row/column graph."""
    n = mask.shape[0]
    adj = [np.nonzero(mask[i])[0].tolist() for i in range(n)]
    match_col = [-1] * n

    def augment(i, seen):
        for j in adj[i]:
            if not seen[j]:
                seen[j] = True
                if match_col[j] < 0 or augment(match_col[j], seen):
                    match_col[j] = i
                    return True
        return False

    for i in range(n):
        if not augment(i, [False] * n):
            return False
    return True


def sparse_real(n: int, seed: int, density: float = 0.2) -> np.ndarray:
    """Dense array holding a sparse matrix: Bernoulli(density) mask with every row
    and column nonempty and a perfect matching; values 1 - u in (0, 1]."""
    attempt = 0
    while True:
        g = rng(seed + 7919 * attempt)
        mask = g.random((n, n)) < density
        for i in range(n):
            if not mask[i].any():
                mask[i, g.integers(0, n)] = True
        for j in range(n):
            if not mask[:, j].any():
                mask[g.integers(0, n), j] = True
        if _has_perfect_matching(mask):
            vals = 1.0 - g.random((n, n))
            return np.where(mask, vals, 0.0)
        attempt += 1


def to_ccs(A: np.ndarray):
    """(cptrs, rids, cvals): column pointers, row ids ascending within a column, values."""
    A = np.asarray(A, dtype=np.float64)
    n = A.shape[0]
    cptrs = [0]
    rids, cvals = [], []
    for j in range(n):
        nz = np.nonzero(A[:, j])[0]
        rids.extend(nz.tolist())
        cvals.extend(A[nz, j].tolist())
        cptrs.append(len(rids))
    return (np.asarray(cptrs, dtype=np.int32), np.asarray(rids, dtype=np.int32),
            np.asarray(cvals, dtype=np.float64))


def from_ccs(n: int, cptrs, rids, cvals) -> np.ndarray:
    A = np.zeros((n, n), dtype=np.float64)
    for j in range(n):
        for p in range(int(cptrs[j]), int(cptrs[j + 1])):
            A[int(rids[p]), j] = cvals[p]
    return A


# ------------------------------------------------------------ structured cases

def block_diagonal(blocks) -> np.ndarray:
    n = sum(b.shape[0] for b in blocks)
    dtype = np.result_type(*[b.dtype for b in blocks])
    M = np.zeros((n, n), dtype=dtype)
    o = 0
    for b in blocks:
        k = b.shape[0]
        M[o:o + k, o:o + k] = b
        o += k
    return M


def shuffle_rows_cols(A: np.ndarray, seed: int) -> np.ndarray:
    g = rng(seed)
    n = A.shape[0]
    return np.ascontiguousarray(A[g.permutation(n)][:, g.permutation(n)])


# ------------------------------------------------------- the named workloads

def dense_real_24():
    """Single dense real n=24 matrix, uniform [0, 1)."""
    return uniform_real(24, SEED_BASE + 1)


def dense_real_40():
    """Dense real n=40 matrix, uniform [-1, 1)."""
    return signed_real(40, SEED_BASE + 2)


def binary_36():
    """0/1 Bernoulli(0.5) n=36 matrix."""
    return bernoulli01(36, SEED_BASE + 3, 0.5)


def complex_32():
    """Seeded Haar-random 32 x 32 unitary."""
    return haar_unitary(32, SEED_BASE + 4)


def sparse_44():
    """Sparse n=44, density 0.2, values in (0, 1]."""
    return sparse_real(44, SEED_BASE + 5, 0.2)


def batched_boson(count: int = 8192, with_rows: bool = False):
    return boson_submatrices(count, SEED_BASE + 6, 8, 26, 256, with_rows)


def grad_real_28():
    """Gradient workload: dense real n=28, uniform [-1, 1)."""
    return signed_real(28, SEED_BASE + 7)


def grad_boson_16(count: int = 1024) -> np.ndarray:
    """Gradient workload: count complex 16 x 16 boson-sampling submatrices of a
    Haar 256 x 256 unitary (rows with replacement, first 16 columns), stacked."""
    return np.stack(boson_submatrices(count, SEED_BASE + 8, 16, 16, 256))

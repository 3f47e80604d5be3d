"""Sparse preprocessing of Sec. 4 (host graph work in the C library, no GPU):
the Dulmage-Mendelsohn filter against its definition by brute force (an
entry survives iff it lies on some perfect matching, i.e. iff the 0/1 pattern
minor has a nonzero permanent), and the Forbert-Marx expansion (Eq. expand,
Alg. 4) against the exact permanent by the oracle's subset DP on integer
matrices, where every intermediate value is an exact binary64 integer."""
import numpy as np
import pytest

import synthetic as syn


@pytest.fixture(scope="module")
def dec():
    from paper_2502_16577_gb300 import build

    build.build()
    from paper_2502_16577_gb300 import decomp

    return decomp


def _sparse_int(n, seed, density, hi=2):
    g = syn.rng(seed)
    M = (g.random((n, n)) < density) * g.integers(1, hi + 1, size=(n, n))
    return M.astype(np.float64)


def _minor(A, k, l):
    return np.delete(np.delete(A, k, 0), l, 1)


def test_dm_keeps_exactly_the_entries_on_perfect_matchings(dec, oracle):
    checked = 0
    for seed in range(40):
        n = 4 + seed % 6
        A = _sparse_int(n, 500 + seed, 0.35)
        if oracle.perm_dp_bin((A != 0).astype(np.uint8)) == 0:
            d = dec.SparseDecomposition(A)
            assert d.info()["structurally_zero"] == 1
            assert d.eval() == 0.0
            continue
        d = dec.SparseDecomposition(A)
        F = d.filtered()
        P = (A != 0).astype(np.uint8)
        for i in range(n):
            for j in range(n):
                on_matching = bool(P[i, j]) and (n == 1 or oracle.perm_dp_bin(_minor(P, i, j)) > 0)
                assert (F[i, j] != 0) == on_matching, (seed, i, j)
                if F[i, j] != 0:
                    assert F[i, j] == A[i, j]
        assert d.info()["removed_nnz"] == int(np.count_nonzero(A) - np.count_nonzero(F))
        checked += 1
    assert checked > 10


def test_dm_block_triangular_splits_into_blocks(dec, oracle):
    # lower block triangular with 3 diagonal blocks, rows and columns shuffled
    g = syn.rng(600)
    sizes = (4, 5, 3)
    n = sum(sizes)
    A = np.zeros((n, n))
    o = 0
    for s in sizes:
        A[o:o + s, o:o + s] = 0.5 + g.random((s, s))
        A[o + s:, o:o + s] = (g.random((n - o - s, s)) < 0.5) * g.random((n - o - s, s))
        o += s
    B = syn.shuffle_rows_cols(A, 601)
    d = dec.SparseDecomposition(B)
    info = d.info()
    assert info["nblocks"] == 3
    assert info["removed_nnz"] == int(np.count_nonzero(A[4:, :4]) + np.count_nonzero(A[9:, 4:9]))
    # the filtered matrix is the block diagonal part, so its permanent is the
    # product of the block permanents
    want = np.prod([oracle.perm_dp_f64(A[o:o + s, o:o + s]) for o, s in ((0, 4), (4, 5), (9, 3))])
    assert oracle.perm_dp_f64(d.filtered()) == pytest.approx(want, rel=1e-13)
    assert oracle.perm_dp_f64(B) == pytest.approx(want, rel=1e-13)


def _recombine(d, perm_of):
    if d.info()["structurally_zero"]:
        return 0
    blocks = {}
    for b, c, M in d.leaves():
        blocks[b] = blocks.get(b, 0) + c * (perm_of(M) if M.shape[0] else 1)
    out = 1
    for b in range(d.info()["nblocks"]):
        out *= blocks.get(b, 0)
    return out


@pytest.mark.parametrize("seed", range(12))
def test_forbert_marx_leaves_recombine_exactly(dec, oracle, seed):
    n = 8 + seed % 5
    A = _sparse_int(n, 700 + seed, 0.3 + 0.02 * (seed % 4))
    want = int(round(oracle.perm_dp_f64(A)))
    d = dec.SparseDecomposition(A)
    got = _recombine(d, lambda M: int(round(oracle.perm_dp_f64(M))))
    assert int(round(got)) == want
    for _, c, M in d.leaves():
        if M.shape[0]:
            # every leaf line has more than four nonzeros, or the leaf budget was hit
            assert min(np.count_nonzero(M, axis=0).min(), np.count_nonzero(M, axis=1).min()) > 4 or \
                d.info()["truncated"]
        assert float(c).is_integer()


def test_forbert_marx_on_real_values(dec, oracle):
    for seed in range(6):
        A = syn.sparse_real(11, 800 + seed, 0.3)
        d = dec.SparseDecomposition(A)
        got = _recombine(d, oracle.perm_dp_f64)
        assert got == pytest.approx(oracle.perm_dp_f64(A), rel=1e-12)


def test_fully_decomposable_matrices_need_no_device(dec, oracle):
    # tridiagonal all-ones: every matrix of the expansion keeps a line with two
    # nonzeros, so the leaves are scalars and perm = F_(n+1) exactly
    for n in (5, 20, 44, 63):
        d = dec.SparseDecomposition(syn.tridiagonal_ones(n))
        assert d.info()["max_leaf_n"] == 0
        assert d.eval() == float(oracle.fibonacci(n + 1))
    # triangular: Dulmage-Mendelsohn leaves the diagonal only
    T = np.tril(0.5 + syn.rng(900).random((30, 30)))
    d = dec.SparseDecomposition(T)
    assert d.info()["nblocks"] == 30 and d.info()["removed_nnz"] == 30 * 29 // 2
    assert d.eval() == pytest.approx(np.prod(np.diag(T)), rel=1e-14)
    # no perfect matching: a zero column
    Z = syn.sparse_real(9, 901, 0.5)
    Z[:, 4] = 0.0
    assert dec.SparseDecomposition(Z).eval() == 0.0


def test_leaf_budget_and_validation(dec):
    A = _sparse_int(14, 950, 0.3)
    d = dec.SparseDecomposition(A, max_leaves=2)
    assert d.info()["nleaves"] <= 3
    from paper_2502_16577_gb300 import PermError

    with pytest.raises(PermError):
        dec.SparseDecomposition(n=3, cptrs=[0, 1, 2, 3], rids=[0, 2, 1], cvals=[1.0, np.nan, 1.0])
    with pytest.raises(PermError):
        dec.SparseDecomposition(n=2, cptrs=[0, 2, 3], rids=[1, 0, 1], cvals=[1.0, 1.0, 1.0])

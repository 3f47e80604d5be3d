"""Parity of the sparse CCS path (Alg. 2 with zero-skip, C ABI, GB300) with
the oracle.  Positive values: relative 1e-10 bar, tighter checks as for the
dense real path."""
import math

import numpy as np
import pytest

import synthetic as syn

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pg():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2502_16577_gb300 as pg
    from paper_2502_16577_gb300 import build

    build.build()
    pg.load()
    return pg


def _ccs(A):
    import torch

    cp, ri, cv = syn.to_ccs(A)
    return (A.shape[0], torch.from_numpy(cp).cuda(), torch.from_numpy(ri).cuda(), torch.from_numpy(cv).cuda())


@pytest.mark.parametrize("n,density", [(1, 1.0), (2, 0.9), (5, 0.5), (9, 0.35), (14, 0.25), (19, 0.2), (22, 0.2)])
def test_vs_oracle(pg, oracle, n, density):
    A = syn.sparse_real(n, 9100 + n, density)
    got = pg.perm_sparse(*_ccs(A))
    crs, ccs = oracle.to_crs_ccs(A)
    want_alg2 = oracle.perm_sparse(n, crs, ccs)
    want_dp = oracle.perm_dp_f64(A)
    assert got == pytest.approx(want_dp, rel=1e-10)
    assert got == pytest.approx(want_dp, rel=1e-13)
    assert got == pytest.approx(want_alg2, rel=1e-12)


def test_signed_and_zero_heavy(pg, oracle):
    # integer-valued sparse matrices: many exact zeros in x, the skip fires
    for seed, n in ((1, 12), (2, 17), (3, 20)):
        M = syn.bernoulli01(n, seed, 0.3).astype(float)
        M[np.arange(n), np.arange(n)] = 1.0
        got = pg.perm_sparse(*_ccs(M))
        # integer products that fit 62 bits are exact, the double-double sum of
        # integers is exact: the result is the exact integer
        assert got == oracle.perm_dp_bin(M.astype(np.uint8))
        S = syn.sparse_real(n, 50 + seed, 0.3) * np.where(syn.bernoulli01(n, 60 + seed) > 0, 1.0, -1.0)
        want = oracle.perm_dp_f64(S)
        assert abs(pg.perm_sparse(*_ccs(S)) - want) <= 1e-13 * oracle.perm_dp_f64(np.abs(S))


def test_matches_dense_path(pg):
    import torch

    A = syn.sparse_real(26, 777, 0.25)
    dense = pg.perm(torch.from_numpy(A).cuda())
    assert pg.perm_sparse(*_ccs(A)) == pytest.approx(dense, rel=1e-13)


def test_tridiagonal_n44_full_size(pg, oracle):
    """Full 2^43-step sweep of the n = 44 tridiagonal all-ones matrix:
    perm = F_45 exactly (the zero-skip makes most steps cheap)."""
    n = 44
    got = pg.perm_sparse(*_ccs(syn.tridiagonal_ones(n).astype(float)))
    assert got == float(oracle.fibonacci(n + 1))


def test_config_sparse_n44_block_diagonal_full_size(pg, oracle):
    """The sparse n = 44 configuration at full size (2^43 Gray steps through
    the sparse kernel): two 22 x 22 density-0.2 blocks, rows and columns
    shuffled, so the answer is the product of the two block permanents."""
    B1, B2 = syn.sparse_real(22, 4401, 0.2), syn.sparse_real(22, 4402, 0.2)
    M = syn.shuffle_rows_cols(syn.block_diagonal([B1, B2]), 4403)
    want = oracle.perm_f64(B1) * oracle.perm_f64(B2)
    got = pg.perm_sparse(*_ccs(M))
    assert got == pytest.approx(want, rel=1e-10)


def test_block_diagonal_n32(pg, oracle):
    B1, B2 = syn.sparse_real(16, 1, 0.3), syn.sparse_real(16, 2, 0.3)
    M = syn.shuffle_rows_cols(syn.block_diagonal([B1, B2]), 3)
    want = oracle.perm_dp_f64(B1) * oracle.perm_dp_f64(B2)
    assert pg.perm_sparse(*_ccs(M)) == pytest.approx(want, rel=1e-12)


def test_malformed_ccs_is_rejected(pg):
    import torch

    n = 4
    ok = syn.sparse_real(n, 5, 0.6)
    _, cp, ri, cv = _ccs(ok)
    bad_rows = ri.clone()
    bad_rows[0] = 9  # out of range
    with pytest.raises(pg.PermError) as e:
        pg.perm_sparse(n, cp, bad_rows, cv)
    assert e.value.code == 1
    bad_ptr = cp.clone()
    bad_ptr[1] = bad_ptr[2] + 1  # not monotone
    with pytest.raises(pg.PermError):
        pg.perm_sparse(n, bad_ptr, ri, cv)
    Z = ok.copy()
    Z[2] = 0.0
    assert pg.perm_sparse(*_ccs(Z)) == 0.0


def test_signed_and_dense_inputs_keep_their_accuracy(pg, oracle):
    """Signed values (terms far below the row-sum bound) and a dense matrix
    given as CCS: the per-term rounding must stay relative to each term, so
    the result meets the dense kernel's accuracy, and J_n (the cancellation
    worst case of Sec. 5) comes out as n!."""
    import math

    import torch

    g = syn.rng(4100)
    for n, density in ((16, 0.3), (22, 0.25), (20, 1.0)):
        mask = g.random((n, n)) < density
        np.fill_diagonal(mask, True)
        A = np.where(mask, 2.0 * g.random((n, n)) - 1.0, 0.0)
        got = pg.perm_sparse(*_ccs(A))
        want = oracle.perm_dp_f64(A)
        scale = oracle.perm_dp_f64(np.abs(A))
        assert abs(got - want) <= 1e-10 * scale
        assert abs(got - want) <= 1e-9 * abs(want) + 1e-14 * scale
        dense = pg.perm(torch.from_numpy(A).cuda())
        assert abs(got - dense) <= 1e-12 * max(abs(want), 1e-300) + 1e-15 * scale
    J = np.ones((22, 22))
    assert pg.perm_sparse(*_ccs(J)) == pytest.approx(float(math.factorial(22)), rel=1e-13)


@pytest.mark.parametrize("n,density", [(12, 0.3), (21, 0.2)])
def test_range_partials(pg, oracle, n, density):
    """perm_sparse_range: in Alg. 2's column order a range equals the oracle's
    double-double sweep of the same steps; in the kernel's own order the
    partials of any partition combine to perm_sparse's value; empty and bad
    ranges are handled."""
    from _bounds import dd_oracle_bound, real_rows_on_grid, real_sweep_bound

    A = syn.sparse_real(n, 9300 + n, density)
    nn, cp, ri, cv = _ccs(A)
    N = 1 << (n - 1)
    for g0, g1 in ((0, N), (0, 1), (3, 4), (N // 3, min(N, N // 3 + 4097)), (N - 100, N)):
        hi, lo = pg.perm_sparse_range(nn, cp, ri, cv, g0, g1, paper_order=True)
        o = oracle.ryser_dd_stats_range(A, g0, g1)
        tol = real_sweep_bound(o["S"], o["W"], n, real_rows_on_grid(A)) + dd_oracle_bound(o["S"], n)
        assert abs((hi + lo) - (o["hi"] + o["lo"])) <= tol + 1e-300, (g0, g1)
    full = pg.perm_sparse(nn, cp, ri, cv)
    cuts = [0, 5, N // 7, N // 2 + 3, N]
    parts = [pg.perm_sparse_range(nn, cp, ri, cv, a, b) for a, b in zip(cuts[:-1], cuts[1:])]
    assert pg.perm_combine(pg.PERM_F64, n, parts) == pytest.approx(full, rel=1e-13)
    assert pg.perm_sparse_range(nn, cp, ri, cv, 7, 7) == (0.0, 0.0)
    with pytest.raises(pg.PermError) as e:
        pg.perm_sparse_range(nn, cp, ri, cv, 5, N + 1)
    assert e.value.code == 2

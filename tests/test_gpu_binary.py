"""Parity of the exact 0/1 path (C ABI, GB300) with the oracle: bit-exact."""
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


def _dev(A):
    import torch

    return torch.from_numpy(np.ascontiguousarray(A, dtype=np.uint8)).cuda()


@pytest.mark.parametrize("n", range(1, 9))
def test_small_vs_bruteforce(pg, oracle, n):
    for seed in range(5):
        A = syn.bernoulli01(n, 7000 + 10 * n + seed, 0.55)
        assert pg.perm(_dev(A)) == oracle.perm_bruteforce(A.astype(int).tolist())


@pytest.mark.parametrize("n", [9, 12, 15, 18, 20, 22])
def test_vs_subset_dp(pg, oracle, n):
    A = syn.bernoulli01(n, 7100 + n, 0.5)
    assert pg.perm(_dev(A)) == oracle.perm_dp_bin(A)


@pytest.mark.parametrize("n", [24, 27])
def test_vs_plain_ryser(pg, oracle, n):
    A = syn.bernoulli01(n, 7200 + n, 0.6)
    assert pg.perm(_dev(A)) == oracle.perm_bin_plain(A)


@pytest.mark.parametrize("n", [5, 16, 26, 30, 34])
def test_closed_forms(pg, oracle, n):
    assert pg.perm(_dev(syn.ones(n))) == math.factorial(n)
    assert pg.perm(_dev(syn.derangement_matrix(n))) == oracle.derangements(n)
    assert pg.perm(_dev(syn.menage_matrix(n))) == oracle.menage(n)
    assert pg.perm(_dev(syn.tridiagonal_ones(n))) == oracle.fibonacci(n + 1)


def test_overflow_is_reported(pg):
    # 35! > 2^128
    with pytest.raises(pg.PermError) as e:
        pg.perm(_dev(syn.ones(35)))
    assert e.value.code == 3


def test_invalid_and_degenerate(pg):
    import torch

    A = syn.bernoulli01(7, 3)
    A[2, 2] = 2
    with pytest.raises(pg.PermError) as e:
        pg.perm(_dev(A))
    assert e.value.code == 1
    Z = syn.ones(6)
    Z[3] = 0
    assert pg.perm(_dev(Z)) == 0
    assert pg.perm(torch.zeros((0, 0), dtype=torch.uint8, device="cuda")) == 1
    assert pg.perm(_dev(np.array([[1]]))) == 1
    assert pg.perm(_dev(np.array([[0]]))) == 0
    assert pg.perm(torch.ones((4, 4), dtype=torch.bool, device="cuda")) == 24


def test_range_partials_exact(pg, oracle):
    n = 21
    A = syn.bernoulli01(n, 7300, 0.5)
    N = 2 ** (n - 1)
    for g0, g1 in [(0, 1), (0, 4096), (77, 9000), (N - 13, N), (5, 5)]:
        got = pg.perm_range(_dev(A), g0, g1)
        assert got % 2 ** 128 == oracle.ryser_bin_range(A, g0, g1), (g0, g1)
    cuts = [0, 3, 1000, 65537, N]
    parts = [pg.perm_range(_dev(A), a, b) for a, b in zip(cuts[:-1], cuts[1:])]
    assert pg.perm_combine(pg.PERM_BIN, n, parts) == oracle.perm_dp_bin(A)


def test_config_binary_36_sampled_and_properties(pg, oracle):
    """The 0/1 Bernoulli(0.5) n=36 workload: full run (exact), a sampled
    2^24-step sub-range against the oracle, and the full-range identity
    sum = (-1)^(n-1) 2^(n-1) perm(A) (low n-1 bits zero)."""
    A = syn.binary_36()
    n = 36
    p = pg.perm(_dev(A))
    assert p > 0 and math.log2(p) <= oracle.bregman_log2(A) + 1e-9
    g0 = 2 ** 33 + 123456
    part = pg.perm_range(_dev(A), g0, g0 + 2 ** 22)
    assert part % 2 ** 128 == oracle.ryser_bin_range(A, g0, g0 + 2 ** 22)
    full = pg.perm_range(_dev(A), 0, 2 ** (n - 1))
    assert full % 2 ** (n - 1) == 0
    assert pg.perm_combine(pg.PERM_BIN, n, [full]) == p
    # block-diagonal 36 = 18 + 18 with known factors
    B1, B2 = syn.bernoulli01(18, 1, 0.5), syn.bernoulli01(18, 2, 0.5)
    M = syn.shuffle_rows_cols(syn.block_diagonal([B1, B2]), 3)
    assert pg.perm(_dev(M)) == oracle.perm_dp_bin(B1) * oracle.perm_dp_bin(B2)



def _abs_glynn_sum(B):
    """S = sum over all sign vectors d in {+-1}^m of prod_i |(1/2) sum_j d_j B_ij|
    (the absolute terms of Eq. 2 for one diagonal block, numpy, exact in fp64
    for 18 x 18 0/1 blocks: every factor is a multiple of 1/2 below 10)."""
    m = B.shape[1]
    bits = (np.arange(1 << m)[:, None] >> np.arange(m)) & 1
    D = 1.0 - 2.0 * bits
    return float(np.prod(np.abs(D @ B.T.astype(np.float64)) / 2.0, axis=1).sum())


def test_full_size_fp64_kernel_on_01_input_vs_exact_integer(pg, oracle):
    """The FP64 kernel's true error at full size (n = 36, 2^35 steps) on a 0/1
    matrix with a known exact permanent: two 18 x 18 Bernoulli(0.5) blocks,
    rows and columns shuffled, perm = the product of the block permanents
    (oracle subset DP, exact integers).  The 0/1 kernel must match exactly.
    The FP64 bound is derived, not tuned: rows are exact for 0/1 input, each
    term's 62-bit product is off by < (n+1) 2^-61 relative, so
    |err| <= 2 (n+1) 2^-61 sum_g |term_g|, and for a block-diagonal matrix the
    half-sum of |terms| factors as S(B1) S(B2) / 2 (Sec. 5)."""
    import torch

    B1, B2 = syn.bernoulli01(18, 3601), syn.bernoulli01(18, 3602)
    M = syn.shuffle_rows_cols(syn.block_diagonal([B1, B2]), 3603)
    exact = oracle.perm_dp_bin(B1) * oracle.perm_dp_bin(B2)
    assert exact > 0
    assert pg.perm(torch.from_numpy(M.astype(np.uint8)).cuda()) == exact
    got = pg.perm(torch.from_numpy(M.astype(np.float64)).cuda())
    n = M.shape[0]
    abs_terms = _abs_glynn_sum(B1) * _abs_glynn_sum(B2) / 2.0
    bound = 2.0 * (n + 1) * 2.0**-61 * abs_terms + 2.0**-52 * exact
    err = abs(got - exact)
    print(f"n=36 0/1: exact {exact}, fp64 rel err {err / exact:.3e}, bound {bound / exact:.3e}")
    assert err <= bound

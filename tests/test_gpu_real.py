"""Parity of the dense real path (C ABI, GB300) with the CPU oracle.

Tolerances: the bar for positive real inputs is a relative error of 1e-10 and
for signed inputs |delta| <= 1e-10 perm(|A|); every test also checks a much
tighter bound that follows from the arithmetic (62-bit products of exact
fixed-point rows, one binary64 rounding per term, double-double carries)."""
import math
from fractions import Fraction

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

    return torch.from_numpy(np.ascontiguousarray(A)).cuda()


def _perm_abs(oracle, A):
    B = np.abs(A)
    return oracle.perm_dp_f64(B) if B.shape[0] <= 22 else None


@pytest.mark.parametrize("n", range(1, 10))
def test_small_vs_bruteforce(pg, oracle, n):
    for seed in range(4):
        A = syn.signed_real(n, 3000 + 10 * n + seed)
        exact = oracle.perm_bruteforce(A)
        got = pg.perm(_dev(A))
        scale = float(oracle.perm_bruteforce(np.abs(A)))
        assert abs(Fraction(got) - exact) <= Fraction(1e-10) * Fraction(scale)
        assert abs(Fraction(got) - exact) <= Fraction(1e-15) * Fraction(scale) + Fraction(1e-300)
        P = syn.uniform_real(n, 3100 + 10 * n + seed)
        e2 = oracle.perm_bruteforce(P)
        g2 = pg.perm(_dev(P))
        assert abs(Fraction(g2) - e2) <= Fraction(1e-14) * e2


@pytest.mark.parametrize("n", [10, 13, 16, 17, 19, 21, 22])
def test_mid_vs_subset_dp(pg, oracle, n):
    P = syn.uniform_real(n, 4000 + n)
    want = oracle.perm_dp_f64(P)
    assert pg.perm(_dev(P)) == pytest.approx(want, rel=1e-12)
    S = syn.signed_real(n, 4100 + n)
    hi, lo = oracle.perm_dd(S)
    got = pg.perm(_dev(S))
    scale = oracle.perm_dp_f64(np.abs(S))
    assert abs(got - (hi + lo)) <= 1e-10 * scale
    assert abs(got - (hi + lo)) <= 1e-14 * scale


def test_config1_dense_real_24(pg, oracle):
    """Single dense real n=24, uniform [0, 1): relative error <= 1e-10 against the
    double-double oracle (and the independent subset DP)."""
    A = syn.dense_real_24()
    hi, lo = oracle.perm_dd(A)
    got = pg.perm(_dev(A))
    assert abs(got - (hi + lo)) <= 1e-10 * (hi + lo)
    assert abs(got - (hi + lo)) <= 1e-13 * (hi + lo)
    assert got == pytest.approx(oracle.perm_dp_f64(A), rel=1e-12)


def _all_equal_bound(n):
    """Relative error bound of perm() for an all-equal matrix a J_n, from the
    kernel's arithmetic (tests/_bounds.py): every row value is
    x(T) = a (|T| + 1 - n/2), so the magnitude sums have closed forms,
    S = a^n sum_k C(n-1, k) |k + 1 - n/2|^n and, with R_i = n |a|,
    W = n (n |a|) |a|^(n-1) sum_k C(n-1, k) |k + 1 - n/2|^(n-1);
    the range sum is within real_sweep_bound(S, W) (the rows lie on their
    grids), perm = 2 (-1)^(n-1) times it, plus the final rounding.  The
    ratio is the same for every a."""
    from _bounds import real_sweep_bound

    S = sum(math.comb(n - 1, k) * abs((k + 1) - n / 2) ** n for k in range(n))
    W = n * n * sum(math.comb(n - 1, k) * abs((k + 1) - n / 2) ** (n - 1) for k in range(n))
    return 2 * real_sweep_bound(S, W, n, True) / math.factorial(n) + 2.0 ** -52


@pytest.mark.parametrize("n", [2, 7, 16, 25, 30])
def test_closed_forms(pg, oracle, n):
    # all-equal matrices are the worst case for cancellation (Sec. 5, Table 3)
    tol = max(_all_equal_bound(n), 1e-14)
    assert tol < 1e-10  # the accuracy bar for positive inputs
    assert pg.perm(_dev(np.ones((n, n)))) == pytest.approx(math.factorial(n), rel=tol)
    exact = Fraction(math.factorial(n)) * Fraction(0.91) ** n
    assert pg.perm(_dev(syn.constant(n, 0.91))) == pytest.approx(float(exact), rel=tol)
    assert pg.perm(_dev(syn.derangement_matrix(n).astype(float))) == pytest.approx(oracle.derangements(n), rel=1e-12)
    assert pg.perm(_dev(syn.tridiagonal_ones(n).astype(float))) == pytest.approx(oracle.fibonacci(n + 1), rel=1e-12)
    d = np.linspace(-1.5, 2.5, n)
    assert pg.perm(_dev(np.diag(d))) == pytest.approx(float(np.prod(d)), rel=1e-13, abs=1e-300)


def test_range_partials_match_oracle(pg, oracle):
    n = 20
    A = syn.signed_real(n, 5150)
    N = 2 ** (n - 1)
    scale = oracle.perm_dp_f64(np.abs(A))
    ranges = [(0, 1), (0, 1000), (5, 6), (12345, 200000), (N - 77, N), (0, N), (3, 3)]
    for g0, g1 in ranges:
        hi, lo = pg.perm_range(_dev(A), g0, g1)
        ohi, olo = oracle.ryser_dd_range(A, g0, g1)
        assert abs((hi + lo) - (ohi + olo)) <= 1e-14 * scale, (g0, g1)
    cuts = [0, 7, 4099, 77777, 300001, N]
    parts = [pg.perm_range(_dev(A), a, b) for a, b in zip(cuts[:-1], cuts[1:])]
    combined = pg.perm_combine(pg.PERM_F64, n, parts)
    assert combined == pytest.approx(pg.perm(_dev(A)), abs=1e-14 * scale)


def test_edge_cases(pg):
    import torch

    assert pg.perm(torch.zeros((0, 0), dtype=torch.float64, device="cuda")) == 1.0
    assert pg.perm(_dev(np.array([[-2.75]]))) == -2.75
    assert pg.perm(_dev(np.array([[1.0, 2.0], [3.0, 4.0]]))) == 10.0
    Z = syn.signed_real(9, 1)
    Z[4] = 0.0
    assert pg.perm(_dev(Z)) == 0.0
    B = syn.signed_real(9, 2)
    B[3, 3] = np.nan
    with pytest.raises(pg.PermError) as e:
        pg.perm(_dev(B))
    assert e.value.code == 1
    H = syn.uniform_real(12, 3) * 1e300
    with pytest.raises(pg.PermError) as e:
        pg.perm(_dev(H))
    assert e.value.code == 2
    # widely different row scales are handled by the per-row power-of-two scaling
    S = syn.uniform_real(10, 4)
    S[2] *= 2.0 ** -500
    S[7] *= 2.0 ** 400
    T = syn.uniform_real(10, 4)
    assert pg.perm(_dev(S)) == pytest.approx(pg.perm(_dev(T)) * 2.0 ** -100, rel=1e-14)


def test_host_entry_point(pg, oracle):
    A = syn.uniform_real(15, 77)
    assert pg.perm_host(A) == pg.perm(_dev(A))
    assert pg.perm_host(A) == pytest.approx(oracle.perm_dp_f64(A), rel=1e-12)


def test_bitwise_reproducible(pg):
    A = syn.signed_real(27, 909)
    assert pg.perm(_dev(A)) == pg.perm(_dev(A))


def test_n40_block_diagonal_full_size(pg, oracle):
    """Full 2^39-step run with a known answer: a signed block-diagonal 40x40
    matrix (two 20x20 blocks) with rows and columns shuffled."""
    B1, B2 = syn.signed_real(20, 61), syn.signed_real(20, 62)
    M = syn.shuffle_rows_cols(syn.block_diagonal([B1, B2]), 63)
    p1 = sum(oracle.perm_dd(B1))
    p2 = sum(oracle.perm_dd(B2))
    want = p1 * p2
    got = pg.perm(_dev(M))
    scale = oracle.perm_dp_f64(np.abs(B1)) * oracle.perm_dp_f64(np.abs(B2))  # perm(|M|)
    assert abs(got - want) <= 1e-10 * scale
    assert abs(got - want) <= 1e-11 * abs(want)


def test_n40_constant_matrix_full_size(pg):
    """All entries 0.91 (the matrix of the paper's n = 62 run) at n = 40:
    perm = 40! 0.91^40, the cancellation-heavy case of Sec. 5 / Table 3."""
    n = 40
    exact = float(Fraction(math.factorial(n)) * Fraction(0.91) ** n)
    got = pg.perm(_dev(syn.constant(n, 0.91)))
    assert abs(got - exact) <= 1e-10 * exact
    assert abs(got - exact) <= _all_equal_bound(n) * exact


def test_n40_config_sampled_range(pg, oracle):
    """The dense real n=40 workload: a 2^24-step sub-range in the middle of the
    Gray sweep against the oracle's double-double sweep of the same steps,
    within the bound of the kernel's arithmetic (the full 2^39-step sweep is
    checked in test_gpu_configs.py)."""
    from _bounds import dd_oracle_bound, real_rows_on_grid, real_sweep_bound

    A = syn.dense_real_40()
    g0 = 3 * 2 ** 36 + 12345
    g1 = g0 + 2 ** 24
    hi, lo = pg.perm_range(_dev(A), g0, g1)
    o = oracle.ryser_dd_stats_range(A, g0, g1)
    tol = real_sweep_bound(o["S"], o["W"], 40, real_rows_on_grid(A)) + dd_oracle_bound(o["S"], 40)
    err = abs((Fraction(hi) + Fraction(lo)) - (Fraction(o["hi"]) + Fraction(o["lo"])))
    assert err <= Fraction(tol), (float(err), tol)



def test_columns_scaled_far_apart(pg, oracle):
    """Columns scaled by powers of two far apart (2^-300, 2^+300, 2^-290, 2^+40):
    perm(A diag(d)) = perm(A) prod d exactly, so the GPU result must match the
    oracle on the unscaled matrix times the factor, to the same relative
    accuracy as the unscaled matrix (exact column equilibration in staging).
    Dense real, extended products, complex and sparse paths."""
    import torch

    n = 14
    scales = np.ones(n)
    scales[[2, 5, 9, 11]] = [2.0 ** -300, 2.0 ** 300, 2.0 ** -290, 2.0 ** 40]
    factor_log2 = -300 + 300 - 290 + 40
    P = syn.uniform_real(n, 7100)
    want = math.ldexp(oracle.perm_dp_f64(P), factor_log2)
    got = pg.perm(_dev(P * scales))
    assert got == pytest.approx(want, rel=1e-13)
    hi, lo = pg.perm_x(_dev(P * scales))
    assert hi + lo == pytest.approx(want, rel=1e-13)
    S = syn.signed_real(n, 7101)
    ref = oracle.perm_dd(S)
    got = pg.perm(_dev(S * scales))
    assert abs(math.ldexp(got, -factor_log2) - (ref[0] + ref[1])) <= 1e-14 * oracle.perm_dp_f64(np.abs(S))
    U = syn.haar_unitary(n, 7102)
    gc = pg.perm(_dev(U * scales))
    wc = oracle.perm_dp_c128(U)
    assert abs(complex(math.ldexp(gc.real, -factor_log2), math.ldexp(gc.imag, -factor_log2)) - wc) <= 1e-13
    Z = syn.sparse_real(n, 7103, 0.4)
    cp, ri, cv = (torch.from_numpy(x).cuda() for x in syn.to_ccs(Z * scales))
    gs = pg.perm_sparse(n, cp, ri, cv)
    assert gs == pytest.approx(math.ldexp(oracle.perm_dp_f64(Z), factor_log2), rel=1e-13)
    # one column 2^7 above the others: without equilibration the row sums are
    # dominated by it and the sweep's terms cancel down to the permanent (20
    # bits lost at n = 14); the balanced columns keep full accuracy
    T = syn.uniform_real(n, 7104)
    T2 = T.copy()
    T2[:, 3] *= 2.0 ** 7
    assert pg.perm(_dev(T2)) == pytest.approx(oracle.perm_dp_f64(T) * 2.0 ** 7, rel=1e-13)

"""Pins for the CPU oracle (no GPU): Table 1, the CBL recursion, brute force over
permutations (Eq. 1), closed forms, invariants and cross-checks between
independent oracle routines.  Every routine in ``oracle/`` is exercised here."""
import itertools
import math
import os
from fractions import Fraction

import numpy as np
import pytest

import synthetic as syn

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _perm_abs(A):
    """perm(|A|) by brute force (float), the scale of the signed tolerance."""
    B = np.abs(np.asarray(A))
    n = B.shape[0]
    return math.fsum(math.prod(B[i, s[i]] for i in range(n)) for s in itertools.permutations(range(n)))


# ------------------------------------------------------------------ Gray code

def test_gray_table_1(oracle):
    rows = [l.split() for l in open(os.path.join(GOLDEN, "gray3.txt")) if l.strip() and not l.startswith("#")]
    assert len(rows) == 8
    for g, binary, gray, chb, chg in rows:
        g = int(g)
        assert int(binary, 2) == g
        assert oracle.gray(g) == int(gray, 2)
        if g == 0:
            continue
        assert [int(b) for b in chb.split(",")] == [b for b in range(3) if ((g ^ (g - 1)) >> b) & 1]
        assert oracle.changed_bit(g) == int(chg)
        # one bit changes between consecutive Gray codes
        assert bin(oracle.gray(g) ^ oracle.gray(g - 1)).count("1") == 1


def test_cbl_recursion_matches_golden_and_changed_bits(oracle):
    rows = [l.split() for l in open(os.path.join(GOLDEN, "cbl.txt")) if l.strip() and not l.startswith("#")]
    assert rows[0][0] == "CBL_3"
    assert oracle.cbl(3) == [int(v) for v in rows[0][1:]]
    for k in range(1, 13):
        c = oracle.cbl(k)
        assert len(c) == 2 ** k - 1
        assert c == c[::-1]  # palindrome
        assert c == [oracle.changed_bit(g) for g in range(1, 2 ** k)]


@pytest.mark.parametrize("c", [1, 2, 4, 6])
def test_aligned_chunks_share_changed_bits(oracle, c):
    """Sec. 3.1.1: with chunks of 2^c iterations every chunk sees the same
    changed-bit sequence except at its boundary."""
    seqs = []
    for k in range(8):
        seqs.append([oracle.changed_bit(k * 2 ** c + t) for t in range(1, 2 ** c)])
    assert all(s == seqs[0] for s in seqs)
    assert seqs[0] == oracle.cbl(c)


# ---------------------------------------------------- brute force vs closed forms

@pytest.mark.parametrize("n", range(0, 8))
def test_bruteforce_closed_forms(oracle, n):
    assert oracle.perm_bruteforce(np.ones((n, n), dtype=int).tolist()) == math.factorial(n)
    assert oracle.perm_bruteforce(syn.derangement_matrix(n).astype(int).tolist()) == oracle.derangements(n)
    assert oracle.perm_bruteforce(syn.tridiagonal_ones(n).astype(int).tolist()) == oracle.fibonacci(n + 1)
    if n >= 3:
        assert oracle.perm_bruteforce(syn.menage_matrix(n).astype(int).tolist()) == oracle.menage(n)


def test_closed_form_sequences(oracle):
    """The closed-form helpers against brute-force counting of permutations."""
    for n in range(0, 8):
        perms = list(itertools.permutations(range(n)))
        assert oracle.derangements(n) == sum(all(s[i] != i for i in range(n)) for s in perms)
        if n >= 3:
            assert oracle.menage(n) == sum(all(s[i] not in (i, (i + 1) % n) for i in range(n)) for s in perms)
    assert [oracle.fibonacci(k) for k in range(10)] == [0, 1, 1, 2, 3, 5, 8, 13, 21, 34]


def test_bruteforce_small_cases(oracle):
    a, b, c, d = 3, 5, 7, 11
    assert oracle.perm_bruteforce([[a, b], [c, d]]) == a * d + b * c
    D = np.diag([2, 3, 5, 7])
    assert oracle.perm_bruteforce(D.tolist()) == 2 * 3 * 5 * 7
    U = np.triu(np.arange(1, 17).reshape(4, 4))
    assert oracle.perm_bruteforce(U.tolist()) == 1 * 6 * 11 * 16
    F = oracle.perm_bruteforce([[0.5, 0.25], [0.125, 2.0]])
    assert F == Fraction(1) + Fraction(1, 32)


# ------------------------------------------------------------- Ryser, real FP64

@pytest.mark.parametrize("n", range(1, 9))
def test_ryser_matches_bruteforce(oracle, n):
    for seed in range(3):
        A = syn.signed_real(n, 1000 * n + seed)
        exact = float(oracle.perm_bruteforce(A))
        got = oracle.perm_f64(A, threads=3)
        assert abs(got - exact) <= 1e-14 * _perm_abs(A) + 1e-300
        hi, lo = oracle.perm_dd(A, threads=2)
        assert abs((Fraction(hi) + Fraction(lo)) - oracle.perm_bruteforce(A)) <= Fraction(1, 10 ** 27) * Fraction(
            _perm_abs(A))


def test_perm_of_empty_and_1x1(oracle):
    assert oracle.perm_bruteforce([]) == 1
    assert oracle.perm_f64(np.array([[0.75]])) == 0.75
    assert oracle.perm_f64(np.array([[-3.5]])) == -3.5


@pytest.mark.parametrize("n", [10, 13, 16, 18])
def test_ryser_matches_subset_dp(oracle, n):
    A = syn.uniform_real(n, 77 + n)
    r = oracle.perm_f64(A)
    d = oracle.perm_dp_f64(A)
    assert abs(r - d) <= 1e-12 * abs(d)
    B = syn.signed_real(n, 99 + n)
    assert abs(oracle.perm_f64(B) - oracle.perm_dp_f64(B)) <= 1e-12 * _perm_abs_dp(oracle, B)


def _perm_abs_dp(oracle, A):
    return oracle.perm_dp_f64(np.abs(A))


@pytest.mark.parametrize("n", [5, 12, 19, 20])
def test_ryser_closed_forms_real(oracle, n):
    assert oracle.perm_f64(np.ones((n, n))) == pytest.approx(math.factorial(n), rel=1e-13)
    a = 0.91  # the all-0.91 matrix of the paper's n = 62 run
    exact = Fraction(math.factorial(n)) * Fraction(a) ** n
    assert oracle.perm_f64(syn.constant(n, a)) == pytest.approx(float(exact), rel=1e-12)
    assert oracle.perm_f64(syn.derangement_matrix(n).astype(float)) == pytest.approx(oracle.derangements(n), rel=1e-12)
    assert oracle.perm_f64(syn.tridiagonal_ones(n).astype(float)) == pytest.approx(oracle.fibonacci(n + 1), rel=1e-12)
    d = np.linspace(0.5, 1.5, n)
    assert oracle.perm_f64(np.diag(d)) == pytest.approx(float(np.prod(d)), rel=1e-13)


def test_block_diagonal_product_rule(oracle):
    B1 = syn.signed_real(7, 1)
    B2 = syn.signed_real(9, 2)
    M = syn.shuffle_rows_cols(syn.block_diagonal([B1, B2]), 3)
    want = oracle.perm_f64(B1) * oracle.perm_f64(B2)
    assert oracle.perm_f64(M) == pytest.approx(want, rel=1e-10, abs=1e-10 * _perm_abs_dp(oracle, M))


def test_invariants_real(oracle):
    n = 9
    A = syn.signed_real(n, 4242)
    p = oracle.perm_f64(A)
    tol = 1e-12 * oracle.perm_dp_f64(np.abs(A))
    g = np.random.default_rng(5)
    assert abs(oracle.perm_f64(A[g.permutation(n)]) - p) <= tol
    assert abs(oracle.perm_f64(A[:, g.permutation(n)]) - p) <= tol
    assert abs(oracle.perm_f64(A.T) - p) <= tol
    S = A.copy()
    S[3] *= 2.5
    assert abs(oracle.perm_f64(S) - 2.5 * p) <= 2.5 * tol
    # linear in each row: perm(A with row i = u + v) = perm(.., u, ..) + perm(.., v, ..)
    U, V = A.copy(), A.copy()
    u, v = g.random(n), g.random(n)
    U[4], V[4] = u, v
    W = A.copy()
    W[4] = u + v
    assert abs(oracle.perm_f64(W) - oracle.perm_f64(U) - oracle.perm_f64(V)) <= 4 * tol
    # row expansion: perm(A) = sum_j a_ij perm(A_ij) for every row i
    for i in range(n):
        s = math.fsum(A[i, j] * oracle.perm_f64(np.delete(np.delete(A, i, 0), j, 1)) for j in range(n))
        assert abs(s - p) <= tol


def test_thread_count_independent(oracle):
    A = syn.signed_real(16, 8)
    vals = [oracle.perm_f64(A, threads=t) for t in (1, 2, 3, 7, 16)]
    assert max(vals) - min(vals) <= 1e-13 * oracle.perm_dp_f64(np.abs(A))


@pytest.mark.parametrize("n", [6, 15])
def test_range_partition_real(oracle, n):
    A = syn.signed_real(n, 31 + n)
    N = 2 ** (n - 1)
    full = oracle.ryser_f64_range(A, 0, N, threads=1)
    cuts = sorted({0, N, 1, N // 3, N // 2 + 1, N - 1})
    tot = Fraction(0)
    for a, b in zip(cuts[:-1], cuts[1:]):
        hi, lo = oracle.ryser_f64_range(A, a, b, threads=2)
        tot += Fraction(hi) + Fraction(lo)
    scale = oracle.perm_dp_f64(np.abs(A))
    assert abs(float(tot - Fraction(full[0]) - Fraction(full[1]))) <= 1e-13 * scale
    # the full sum times 2 (-1)^(n-1) is the permanent
    assert 2 * (-1) ** (n - 1) * (full[0] + full[1]) == pytest.approx(oracle.perm_dp_f64(A), abs=1e-12 * scale)


def test_dd_mode_tighter_than_f64(oracle):
    """The double-double mode matches exact arithmetic to ~1e-28 relative on a
    cancellation-heavy case (all-equal matrix, perm = n! a^n, Sec. 5)."""
    n, a = 14, 0.91
    exact = Fraction(math.factorial(n)) * Fraction(a) ** n
    hi, lo = oracle.perm_dd(syn.constant(n, a), threads=4)
    err = abs(Fraction(hi) + Fraction(lo) - exact) / exact
    assert err < Fraction(1, 10 ** 25)


# ------------------------------------------------------------------- complex

@pytest.mark.parametrize("n", range(1, 7))
def test_complex_matches_bruteforce(oracle, n):
    A = syn.complex_uniform(n, 500 + n)
    re, im = oracle.perm_bruteforce(A.tolist())
    got = oracle.perm_c128(A, threads=2)
    scale = _perm_abs(A)
    assert abs(got.real - float(re)) <= 1e-14 * scale
    assert abs(got.imag - float(im)) <= 1e-14 * scale


@pytest.mark.parametrize("n", [8, 12, 16])
def test_complex_matches_dp_and_unitary_bounds(oracle, n):
    U = syn.haar_unitary(n, 600 + n)
    p = oracle.perm_c128(U)
    assert abs(p - oracle.perm_dp_c128(U)) <= 1e-12
    assert abs(p) <= 1.0 + 1e-12  # |perm(U)| <= 1 for unitary U
    q = oracle.perm_c128(np.conj(U))
    assert abs(q - np.conj(p)) <= 1e-13


def test_boson_sampling_normalisation(oracle):
    """sum over output multisets T of size k of |perm(U_{T,[k]})|^2 / prod_t m_t! = 1."""
    m, k = 6, 3
    U = syn.haar_unitary(m, 7)
    total = 0.0
    for T in itertools.combinations_with_replacement(range(m), k):
        sub = U[list(T), :k]
        mult = math.prod(math.factorial(T.count(t)) for t in set(T))
        total += abs(oracle.perm_c128(sub, threads=1)) ** 2 / mult
    assert total == pytest.approx(1.0, abs=1e-12)


def test_range_partition_complex(oracle):
    A = syn.haar_unitary(11, 9)
    N = 2 ** 10
    full = oracle.ryser_c128_range(A, 0, N)
    parts = [oracle.ryser_c128_range(A, a, b) for a, b in ((0, 100), (100, 517), (517, N))]
    for c in (0, 2):
        assert abs(sum(p[c] + p[c + 1] for p in parts) - (full[c] + full[c + 1])) <= 1e-14


# --------------------------------------------------------------------- binary

@pytest.mark.parametrize("n", range(1, 8))
def test_binary_matches_bruteforce(oracle, n):
    for seed in range(3):
        A = syn.bernoulli01(n, 700 + 10 * n + seed)
        exact = oracle.perm_bruteforce(A.astype(int).tolist())
        assert oracle.perm_bin_plain(A, threads=2) == exact
        assert oracle.perm_dp_bin(A) == exact


@pytest.mark.parametrize("n", [12, 16, 20])
def test_binary_dp_vs_plain_ryser(oracle, n):
    A = syn.bernoulli01(n, 800 + n, 0.6)
    assert oracle.perm_bin_plain(A) == oracle.perm_dp_bin(A)


@pytest.mark.parametrize("n", [20, 24])
def test_binary_closed_forms(oracle, n):
    assert oracle.perm_bin_plain(syn.ones(n)) == math.factorial(n) % 2 ** 128
    assert oracle.perm_bin_plain(syn.derangement_matrix(n)) == oracle.derangements(n)
    assert oracle.perm_bin_plain(syn.menage_matrix(n)) == oracle.menage(n)
    assert oracle.perm_bin_plain(syn.tridiagonal_ones(n)) == oracle.fibonacci(n + 1)


@pytest.mark.parametrize("n", [5, 14, 21])
def test_binary_doubled_rows_identity(oracle, n):
    """Alg. 1 on x' = 2x sums to (-1)^(n-1) 2^(n-1) perm(A) over the full range,
    and any partition of the range adds up to the same residue mod 2^128."""
    A = syn.bernoulli01(n, 900 + n)
    N = 2 ** (n - 1)
    p = oracle.perm_bin_plain(A)
    full = oracle.ryser_bin_range(A, 0, N)
    assert full == ((-1) ** (n - 1) * 2 ** (n - 1) * p) % 2 ** 128
    cuts = [0, N // 5, N // 2, N - 3, N]
    assert sum(oracle.ryser_bin_range(A, a, b, threads=3) for a, b in zip(cuts[:-1], cuts[1:])) % 2 ** 128 == full


def test_bregman_bound(oracle):
    A = syn.bernoulli01(10, 4)
    assert oracle.perm_bin_plain(A) <= 2 ** oracle.bregman_log2(A) * (1 + 1e-12)
    assert oracle.bregman_log2(syn.ones(6)) == pytest.approx(math.log2(720.0))


# --------------------------------------------------------------------- sparse

@pytest.mark.parametrize("n,density", [(8, 0.35), (13, 0.25), (17, 0.2)])
def test_sparse_alg2_matches_dense(oracle, n, density):
    A = syn.sparse_real(n, 1200 + n, density)
    crs, ccs = oracle.to_crs_ccs(A)
    cptrs, rids, cvals = syn.to_ccs(A)
    assert np.array_equal(cptrs, ccs[0]) and np.array_equal(rids, ccs[1]) and np.array_equal(cvals, ccs[2])
    assert np.array_equal(syn.from_ccs(n, cptrs, rids, cvals), A)
    got = oracle.perm_sparse(n, crs, ccs, threads=3)
    assert got == pytest.approx(oracle.perm_dp_f64(A), rel=1e-12)
    assert got > 0  # a perfect matching exists and every value is positive
    N = 2 ** (n - 1)
    a = oracle.spa_ryser_range(n, crs, ccs, 0, N // 3)
    b = oracle.spa_ryser_range(n, crs, ccs, N // 3, N)
    d = oracle.ryser_f64_range(A, 0, N)
    assert (a[0] + a[1] + b[0] + b[1]) == pytest.approx(d[0] + d[1], rel=1e-12)


def test_generators_are_deterministic():
    assert np.array_equal(syn.dense_real_40(), syn.dense_real_40())
    assert np.array_equal(syn.binary_36(), syn.binary_36())
    U = syn.complex_32()
    assert np.allclose(U.conj().T @ U, np.eye(32), atol=1e-13)
    S = syn.sparse_44()
    assert (S != 0).any(axis=0).all() and (S != 0).any(axis=1).all()
    assert ((S == 0) | ((S > 0) & (S <= 1))).all()
    assert np.all(syn.signed_real(40, 1) * 2 ** 52 == np.round(syn.signed_real(40, 1) * 2 ** 52))


# --------------------------------------- double-double sweeps with magnitude sums

def _stats_by_definition(A):
    """S and W of the full range computed from scratch for every subset (no Gray
    updates): x_i(T) = (1/2) sum_j d_j a_ij with d_j = +1 for j in T or j = n-1,
    else -1 (Eq. nwx); S = sum_T |prod_i x_i|, W = sum_T sum_i R_i prod_{k != i} |x_k|,
    R_i = sum_j |a_ij|.  Exact rational arithmetic for real entries."""
    A = np.asarray(A)
    n = A.shape[0]
    cplx = np.iscomplexobj(A)
    R = [math.fsum(abs(complex(v)) for v in A[i]) for i in range(n)]
    S, W = 0.0, 0.0
    for T in range(2 ** (n - 1)):
        d = [1 if (j == n - 1 or (T >> j) & 1) else -1 for j in range(n)]
        xs = [sum(complex(A[i, j]) * d[j] for j in range(n)) / 2 for i in range(n)] if cplx else \
            [float(sum(Fraction(float(A[i, j])) * d[j] for j in range(n)) / 2) for i in range(n)]
        mags = [abs(x) for x in xs]
        S += math.prod(mags)
        W += math.fsum(R[i] * math.prod(mags[:i] + mags[i + 1:]) for i in range(n))
    return S, W


@pytest.mark.parametrize("n", [1, 2, 4, 7, 9])
def test_dd_stats_sum_and_magnitudes_by_definition(oracle, n):
    A = syn.signed_real(n, 5500 + n)
    N = 2 ** (n - 1)
    r = oracle.ryser_dd_stats_range(A, 0, N, threads=3)
    exact = oracle.perm_bruteforce(A) if n <= 8 else None
    if exact is not None:
        got = (Fraction(r["hi"]) + Fraction(r["lo"])) * 2 * (-1) ** (n - 1)
        assert abs(got - exact) <= Fraction(1, 10 ** 27) * Fraction(_perm_abs(A))
    S, W = _stats_by_definition(A)
    assert r["S"] == pytest.approx(S, rel=1e-13)
    assert r["W"] == pytest.approx(W, rel=1e-13)
    # the sum is the one of ryser_dd_range, range by range
    for g0, g1 in ((0, N), (0, 1), (N // 3, N)):
        s = oracle.ryser_dd_stats_range(A, g0, g1, threads=2)
        assert (s["hi"], s["lo"]) == oracle.ryser_dd_range(A, g0, g1, threads=2)


@pytest.mark.parametrize("n", [5, 8, 12, 21])
def test_dd_stats_all_equal_closed_forms(oracle, n):
    """a J_n: x_i = a (|T| + 1 - n/2) for every row, so
    S = a^n sum_k C(n-1, k) |k + 1 - n/2|^n and, with R_i = n |a|,
    W = n (n |a|) |a|^(n-1) sum_k C(n-1, k) |k + 1 - n/2|^(n-1)."""
    a = 0.75
    r = oracle.ryser_dd_stats_range(syn.constant(n, a), 0, 2 ** (n - 1), threads=4)
    s = sum(math.comb(n - 1, k) * abs(k + 1 - n / 2) ** n for k in range(n)) * a ** n
    w = n * n * a * a ** (n - 1) * sum(math.comb(n - 1, k) * abs(k + 1 - n / 2) ** (n - 1) for k in range(n))
    assert r["S"] == pytest.approx(s, rel=1e-13)
    assert r["W"] == pytest.approx(w, rel=1e-13)
    exact = Fraction(math.factorial(n)) * Fraction(a) ** n
    got = (Fraction(r["hi"]) + Fraction(r["lo"])) * 2 * (-1) ** (n - 1)
    assert abs(got - exact) <= Fraction(1, 10 ** 26) * exact


def _gaussian_integer_matrix(n, seed):
    g = np.random.default_rng(seed)
    return (g.integers(-3, 4, (n, n)) + 1j * g.integers(-3, 4, (n, n))).astype(np.complex128)


@pytest.mark.parametrize("n", range(1, 8))
def test_cdd_exact_on_gaussian_integers(oracle, n):
    """Gaussian-integer entries: every x_i is a multiple of 1/2 and every product
    is exact in double-double, so the sweep equals Eq. 1 summed exactly."""
    A = _gaussian_integer_matrix(n, 5600 + n)
    re, im = oracle.perm_bruteforce(A.tolist())
    r = oracle.ryser_cdd_range(A, 0, 2 ** (n - 1), threads=2)
    f = 2 * (-1) ** (n - 1)
    assert (Fraction(r["re_hi"]) + Fraction(r["re_lo"])) * f == re
    assert (Fraction(r["im_hi"]) + Fraction(r["im_lo"])) * f == im


@pytest.mark.parametrize("n", [3, 6, 8])
def test_cdd_magnitudes_by_definition(oracle, n):
    A = syn.complex_uniform(n, 5700 + n)
    r = oracle.ryser_cdd_range(A, 0, 2 ** (n - 1), threads=3)
    S, W = _stats_by_definition(A)
    assert r["S"] == pytest.approx(S, rel=1e-12)
    assert r["W"] == pytest.approx(W, rel=1e-12)


def test_cdd_special_cases(oracle):
    """Zero imaginary parts reduce to the real double-double sweep; a Haar unitary
    matches the subset expansion of Eq. 1 and |perm(U)| <= 1; conj(U) gives the
    conjugate; a range partition adds up to the full sum."""
    A = syn.signed_real(11, 5800)
    N = 2 ** 10
    r = oracle.ryser_cdd_range(A.astype(np.complex128), 0, N, threads=2)
    d = oracle.ryser_dd_range(A, 0, N, threads=2)
    assert (r["re_hi"], r["re_lo"]) == d and r["im_hi"] == 0.0 and r["im_lo"] == 0.0
    U = syn.haar_unitary(12, 5801)
    r = oracle.ryser_cdd_range(U, 0, 2 ** 11)
    p = complex(r["re_hi"] + r["re_lo"], r["im_hi"] + r["im_lo"]) * -2
    assert abs(p - oracle.perm_dp_c128(U)) <= 1e-13 and abs(p) <= 1.0
    q = oracle.ryser_cdd_range(np.conj(U), 0, 2 ** 11)
    assert (q["re_hi"], q["re_lo"]) == (r["re_hi"], r["re_lo"])
    assert (q["im_hi"], q["im_lo"]) == (-r["im_hi"], -r["im_lo"])
    parts = [oracle.ryser_cdd_range(U, a, b, threads=2) for a, b in ((0, 5), (5, 1000), (1000, 2 ** 11))]
    tot = sum(Fraction(p["re_hi"]) + Fraction(p["re_lo"]) for p in parts)
    assert abs(float(tot) - (r["re_hi"] + r["re_lo"])) <= 1e-28

"""Extended-precision products (PERM_F64X: Sec. 5's quad inner product) on the
GPU against exact and double-double references.

The bound every test derives: the rows are exact on the inputs used here
(every entry is a multiple of 2^-53 or a 0/1 value, and the row scale puts
the row's absolute sum below 2^61), each of the n factors and the chain merge
loses at most 2^-123 of the term, the head/tail split at most 2^-105, and the
per-step renormalised double-double about 2^-104 of its running value.  So
the unscaled sum is within 2^-95 S of the exact one, with S = sum_g |term_g|
(2^-95 keeps a factor of 2^9 for the accumulation over a lane's steps), and
perm = 2 (-1)^(n-1) sum is within 2^-94 S."""
import math
from fractions import Fraction

import numpy as np
import pytest

import synthetic as syn

pytestmark = pytest.mark.gpu

TOL = 2.0 ** -94


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

    return torch.from_numpy(np.ascontiguousarray(A, dtype=np.float64)).cuda()


def _abs_terms(A, g0=0, g1=None):
    """S = sum over steps g in [g0, g1) of prod_i |x_i(g)|, x_i = (1/2) sum_l d_l a_il
    with d_l = +1 for the columns in Gray(g) and column n-1, else -1 (Eq. 2),
    in numpy (a tolerance scale, not a reference value)."""
    A = np.asarray(A, dtype=np.float64)
    n = A.shape[0]
    g1 = (1 << (n - 1)) if g1 is None else g1
    S = 0.0
    for b0 in range(g0, g1, 1 << 16):
        g = np.arange(b0, min(b0 + (1 << 16), g1), dtype=np.int64)
        G = g ^ (g >> 1)
        d = np.ones((g.size, n))
        d[:, : n - 1] = np.where((G[:, None] >> np.arange(n - 1)) & 1, 1.0, -1.0)
        S += float(np.prod(np.abs(d @ A.T) / 2.0, axis=1).sum())
    return S


def _val(x):
    return Fraction(x[0]) + Fraction(x[1])


def _normalised(x):
    hi, lo = x
    return hi + lo == hi and (hi == 0.0 or abs(lo) <= math.ulp(hi) / 2)


@pytest.mark.parametrize("n", range(1, 9))
def test_small_vs_exact_bruteforce(pg, oracle, n):
    for A in (syn.signed_real(n, 7100 + n), syn.uniform_real(n, 7200 + n)):
        got = pg.perm_x(_dev(A))
        exact = oracle.perm_bruteforce(A)
        assert _normalised(got)
        assert abs(_val(got) - exact) <= Fraction(TOL) * Fraction(_abs_terms(A))


@pytest.mark.parametrize("n", [12, 16, 18])
def test_vs_oracle_double_double(pg, oracle, n):
    """The oracle's high-precision mode (x and products in double-double, Sec. 5)
    is the reference; both sit within about 2^-95 S of the exact sum."""
    for A in (syn.signed_real(n, 7300 + n), syn.uniform_real(n, 7400 + n, -1.0, 1.0)):
        got = pg.perm_x(_dev(A))
        ref = oracle.perm_dd(A)
        assert abs(_val(got) - _val(ref)) <= Fraction(2 * TOL) * Fraction(_abs_terms(A))
        # the binary64 result of the default kernel is the rounded extended one
        # up to the default kernel's own error
        assert pg.perm(_dev(A)) == pytest.approx(got[0] + got[1], rel=1e-12, abs=1e-15 * _abs_terms(A))


@pytest.mark.parametrize("n", [20, 30])
def test_constant_matrix_closed_form(pg, n):
    """perm(a J_n) = n! a^n (Sec. 5's exactly known cases).  All entries equal
    is the cancellation worst case; S has a closed form over the number k of
    other columns in the subset: x = a (k + 1 - n/2) for every row."""
    a = 0.91
    A = syn.constant(n, a)
    exact = math.factorial(n) * Fraction(a) ** n
    S = sum(math.comb(n - 1, k) * Fraction(abs(2 * k + 2 - n), 2) ** n for k in range(n)) * Fraction(a) ** n
    got = pg.perm_x(_dev(A))
    err_x = abs(_val(got) - exact)
    err_d = abs(Fraction(pg.perm(_dev(A))) - exact)
    print(f"J_{n}*{a}: extended rel err {float(err_x / exact):.2e}, default {float(err_d / exact):.2e}, "
          f"S/perm {float(S / exact):.2e}")
    assert err_x <= Fraction(TOL) * S
    assert err_x <= err_d / 1000 or err_d == 0


def test_full_size_block_diagonal_01(pg, oracle):
    """n = 36 at full size (2^35 steps): two shuffled 18 x 18 Bernoulli(0.5)
    blocks; the exact integer is the product of the block permanents, and S
    factors over the blocks (each |x_i| depends on its block's columns only;
    half of the 2^36 sign vectors are steps)."""
    B1, B2 = syn.bernoulli01(18, 3601), syn.bernoulli01(18, 3602)
    M = syn.shuffle_rows_cols(syn.block_diagonal([B1, B2]), 3603).astype(np.float64)
    exact = oracle.perm_dp_bin(B1) * oracle.perm_dp_bin(B2)

    def full_abs(B):  # over all 2^m sign vectors of one block
        m = B.shape[1]
        d = 1.0 - 2.0 * ((np.arange(1 << m)[:, None] >> np.arange(m)) & 1)
        return float(np.prod(np.abs(d @ B.T.astype(np.float64)) / 2.0, axis=1).sum())

    S = full_abs(B1) * full_abs(B2) / 2.0
    got = pg.perm_x(_dev(M))
    err = abs(_val(got) - exact)
    print(f"n=36 0/1 extended: |err| {float(err):.3e} (bound {TOL * S:.3e}, perm {exact})")
    assert err <= Fraction(TOL) * Fraction(S)


def test_range_partials_and_combine(pg, oracle):
    """Partials over a partition of the Gray range (Secs. 3.3, 6.3) match the
    oracle's double-double range sums, and their host combination is the
    permanent."""
    n = 20
    A = syn.signed_real(n, 7500)
    N = 1 << (n - 1)
    cuts = [0, 12345, 1 << 17, N - 777, N]
    parts = []
    for g0, g1 in zip(cuts[:-1], cuts[1:]):
        p = pg.perm_range(_dev(A), g0, g1, extended=True)
        ref = oracle.ryser_dd_range(A, g0, g1)
        assert abs(_val(p) - _val(ref)) <= Fraction(2 * TOL) * Fraction(_abs_terms(A, g0, g1))
        parts.append(p)
    comb = pg.perm_combine(pg.PERM_F64X, n, parts)
    full = pg.perm_x(_dev(A))
    assert abs(_val(comb) - _val(full)) <= Fraction(4 * TOL) * Fraction(_abs_terms(A))


def test_config_dense_40_sampled_range(pg, oracle):
    """The dense n = 40 uniform[-1, 1) workload: 2^20 steps from the middle
    of the range against the oracle's double-double range sum."""
    A = syn.dense_real_40()
    g0 = (1 << 38) + 12345
    g1 = g0 + (1 << 20)
    got = pg.perm_range(_dev(A), g0, g1, extended=True)
    ref = oracle.ryser_dd_range(A, g0, g1)
    assert abs(_val(got) - _val(ref)) <= Fraction(2 * TOL) * Fraction(_abs_terms(A, g0, g1))


def test_edge_cases_and_determinism(pg):
    import torch

    assert pg.perm_x(torch.zeros((0, 0), dtype=torch.float64, device="cuda")) == (1.0, 0.0)
    assert pg.perm_x(_dev(np.array([[-0.375]]))) == (-0.375, 0.0)
    a, b, c, d = 0.1, 0.7, 1.0 / 3.0, -2.5
    got = pg.perm_x(_dev(np.array([[a, b], [c, d]])))
    exact = Fraction(a) * Fraction(d) + Fraction(b) * Fraction(c)
    assert abs(_val(got) - exact) <= Fraction(2.0 ** -100) * abs(exact)
    Z = syn.signed_real(9, 7600)
    Z[4] = 0.0
    assert pg.perm_x(_dev(Z)) == (0.0, 0.0)
    bad = syn.signed_real(6, 7601)
    bad[2, 3] = np.inf
    with pytest.raises(pg.PermError):
        pg.perm_x(_dev(bad))
    with pytest.raises(TypeError):
        pg.perm_x(_dev(bad).to(torch.complex128))
    A = syn.signed_real(26, 7602)
    assert pg.perm_x(_dev(A)) == pg.perm_x(_dev(A))

"""The error bounds of tests/_bounds.py, checked on the CPU.

The GPU parity tests accept a kernel result when it lies within the bound
that tests/_bounds.py derives from the kernel's arithmetic.  Here that
derivation is checked without a GPU, on inputs small enough for exact
rational arithmetic:

* the exact range sum sum_g (-1)^g prod_i x_i(g) and the magnitude sums S and
  W are computed with Fractions (every binary64 entry is a dyadic rational);
* the double-double oracle (ryser_dd_stats_range) must lie within
  dd_oracle_bound of the exact sum and reproduce S and W;
* a bit-level model of the dense real sweep's fixed-point arithmetic (the
  staging of every row, the odd last column, the 62-bit products with their
  renormalising shifts, the exponent bookkeeping, and the integer assembly of
  each term's binary64 head and tail, including a product chain that a factor
  |Y_i| = 1 has emptied; Alg. 1's terms, summed exactly) must lie within
  real_sweep_bound.  The model restates the integer operations the kernel
  documents (two chains over even and odd rows and one merge per step) in
  Python integers; it shares no code with the CUDA sources.  The
  double-double accumulation of the terms (below 2^-64 S per chunk) is left
  out; the bound's 2^-59 S allowance covers it.
"""
import math
from fractions import Fraction

import numpy as np
import pytest

import synthetic as syn
from _bounds import dd_oracle_bound, real_rows_on_grid, real_sweep_bound

M32 = (1 << 32) - 1


def _exact(A):
    """Exact sum_g (-1)^g prod_i x_i(g), S and W over all 2^(n-1) Gray steps
    (x_i = 1/2 sum_j delta_j a_ij, Eq. nwx; Alg. 1's order)."""
    n = A.shape[0]
    F = [[Fraction(float(v)) for v in row] for row in A]
    R = [sum(abs(v) for v in row) for row in F]
    # g = 0: every column but n-1 out
    x = [(F[i][n - 1] - sum(F[i][:n - 1])) / 2 for i in range(n)]
    total, S, W = Fraction(0), Fraction(0), Fraction(0)
    for g in range(1 << (n - 1)):
        if g:
            j = (g & -g).bit_length() - 1
            enter = not ((g >> (j + 1)) & 1)
            for i in range(n):
                x[i] += F[i][j] if enter else -F[i][j]
        p = Fraction(1)
        for v in x:
            p *= v
        total += -p if g & 1 else p
        S += abs(p)
        for i in range(n):
            q = R[i]
            for k in range(n):
                if k != i:
                    q *= abs(x[k])
            W += q
    return total, S, W


def _prod_mul(m0, m1, a0, a1):
    """The 62-bit product step: v = M A / 2^64 (the m0 a0 partial product
    dropped, 2^31 added to the middle ones), then M <- v << (30 - pos) with pos
    the top set bit of v's high word (32-bit wrap-around shift semantics)."""
    t = m1 * a0 + (1 << 31)
    u = m0 * a1 + t
    assert u < (1 << 64)
    v = m1 * a1 + (u >> 32)
    vh, vl = v >> 32, v & M32
    pos = vh.bit_length() - 1 if vh else -1
    s = (30 - pos) & M32
    w = s & 31
    new_m1 = ((((vh << 32) | vl) << w) >> 32) & M32
    new_m0 = (vl << s) & M32 if s < 32 else 0
    return new_m0, new_m1, pos


def _f64_from_bits(b):
    """The binary64 value of a 64-bit pattern (finite patterns only)."""
    sign = -1 if b >> 63 else 1
    e = (b >> 52) & 0x7FF
    m = b & ((1 << 52) - 1)
    assert e != 0x7FF
    if e == 0:
        return sign * Fraction(m) / (1 << 1074)
    return sign * (Fraction((1 << 52) | m) * Fraction(2) ** (e - 1075))


def _term_head_tail(M, f, signbit):
    """The head and tail a term M 2^(f + 1 - 1023 - 62) is split into, from
    the integer assembly: the head adds 512 to M, keeps its top 53 bits and
    places them on the exponent field f; the tail is M minus the head's bits
    (at most 512 units), placed by its own top bit.  f is clamped at 0."""
    f = max(f, 0)
    R = (M + 512) & ((1 << 64) - 1)
    head = _f64_from_bits(((signbit << 63) + (f << 52) + (R >> 10)) & ((1 << 64) - 1))
    r = (M & M32) - (R & M32 & ~0x3FF)
    r = r - (1 << 32) if r >= (1 << 31) else (r + (1 << 32) if r < -(1 << 31) else r)
    mag = abs(r)
    lz = 32 - (mag | 1).bit_length()
    be = f - 61 + 31 - lz
    if mag == 0 or be <= 0:
        return head, Fraction(0)
    tail = Fraction(mag) * Fraction(2) ** (be - 1023 - (31 - lz))
    return head, (-tail if (r < 0) != bool(signbit) else tail)


def _model_sweep(A):
    """The dense real sweep's range sum over all steps, from its integer
    arithmetic: rows in 64-bit fixed point (s_i = 61 - k_i, columns 0..n-2
    rounded to nearest even multiples, column n-1 to odd ones), |Y_i| exact
    (Y_i is odd), two product chains (even / odd rows) merged, and the term
    value from the mantissa and the renormalising shifts."""
    n = A.shape[0]
    Q, scale = [], []
    for i in range(n):
        absum = 0.0
        for j in range(n):
            absum += abs(float(A[i, j]))  # binary64 in column order, as staged
        k = math.frexp(absum)[1] if absum > 0 else 0
        s = 61 - k
        row = [2 * round(Fraction(float(A[i, j])) * Fraction(2) ** (s - 1)) for j in range(n - 1)]
        row.append(2 * math.floor(Fraction(float(A[i, n - 1])) * Fraction(2) ** (s - 1)) + 1)
        Q.append(row)
        scale.append(s + 1)
    Y = [Q[i][n - 1] - sum(Q[i][:n - 1]) for i in range(n)]
    total = Fraction(0)
    K1 = 64 * n + 1025 - (sum(scale) - n)  # sum of the s_i
    for g in range(1 << (n - 1)):
        if g:
            j = (g & -g).bit_length() - 1
            sgn = -1 if (g >> (j + 1)) & 1 else 1
            for i in range(n):
                Y[i] += 2 * sgn * Q[i][j]
        chains = [[0, 1 << 30], [0, 1 << 30]]  # 2^62 each
        epos, neg = 0, 0
        for i, y in enumerate(Y):
            assert y & 1 and abs(y) < (1 << 62)
            a = abs(y)
            neg ^= y < 0
            c = chains[i & 1]
            c[0], c[1], pos = _prod_mul(c[0], c[1], a & M32, a >> 32)
            epos += pos
        m0, m1, pos = _prod_mul(chains[0][0], chains[0][1], chains[1][0], chains[1][1])
        epos += pos
        f = K1 - (30 * (n + 1) - epos) - (n + 1)
        head, tail = _term_head_tail((m1 << 32) | m0, f, int(neg ^ (g & 1)))
        total += head + tail
    return total


def _cases():
    g = syn.rng(9100)
    out = [("signed uniform n=9", syn.signed_real(9, 9101)),
           ("uniform [0, 1) n=10", syn.uniform_real(10, 9102)),
           ("integers in [-3, 3] n=10 (on the grid)", g.integers(-3, 4, size=(10, 10)).astype(np.float64)),
           ("random signs n=10 (many x_i = 0)", np.where(g.random((10, 10)) < 0.5, -1.0, 1.0))]
    B = syn.signed_real(8, 9103)
    B[2] *= 2.0 ** 300
    B[5] *= 2.0 ** -280
    out.append(("rows scaled 2^300 / 2^-280 n=8", B))
    # a row whose x is exactly 0 on half the steps: |Y| = 1 there (the odd
    # unit), which empties its product chain: the first factor, a middle one,
    # and the last factor of either chain (rows alternate between the chains)
    for r in (0, 4, 7, 8):
        C = syn.signed_real(9, 9104 + r)
        C[r] = 0.0
        C[r, 0], C[r, 1] = 1.0, -1.0
        out.append((f"x_{r} = 0 on half the steps n=9", C))
    return out


@pytest.mark.parametrize("name,A", _cases(), ids=lambda v: v if isinstance(v, str) else "")
def test_oracle_dd_and_model_sweep_within_their_bounds(oracle, name, A):
    n = A.shape[0]
    exact, S, W = _exact(A)
    # the double-double oracle: its range sum within (n + 2) 2^-100 S, and its S, W
    r = oracle.ryser_dd_stats_range(A, 0, 1 << (n - 1))
    err_dd = abs(Fraction(r["hi"]) + Fraction(r["lo"]) - exact)
    assert err_dd <= Fraction(dd_oracle_bound(float(S), n)), (name, float(err_dd), float(S))
    assert r["S"] == pytest.approx(float(S), rel=1e-13)
    assert r["W"] == pytest.approx(float(W), rel=1e-13)
    # the dense sweep's arithmetic within the bound the GPU parity tests use
    model = _model_sweep(A)
    bound = real_sweep_bound(float(S), float(W), n, real_rows_on_grid(A))
    err = abs(model - exact)
    assert err <= Fraction(bound), (name, float(err), bound)


def test_model_is_exact_on_small_integers():
    # a check of the model itself: rows of small integers are staged exactly
    # apart from the odd unit of the last column (2^-(s_i+1) in x_i), which
    # changes a 62-bit product of these |Y_i| ~ 2^60 by a quarter of its last
    # unit and is rounded away, and every other product is exact, so the model
    # reproduces the exact sum bit for bit
    A = np.array([[1, 2, 0], [3, -1, 1], [0, 1, 2]], dtype=np.float64)
    exact, _, _ = _exact(A)
    assert _model_sweep(A) == exact


def test_grid_detection():
    # entries of columns 0..n-2 that are multiples of the row's fixed-point
    # unit are on the grid; an entry far below its row sum is not; column n-1
    # is rounded to an odd multiple in any case and is not examined
    assert real_rows_on_grid(np.array([[1.0, -2.0], [0.5, 0.25]]))
    assert not real_rows_on_grid(np.array([[2.0 ** -70, 1.0], [1.0, 1.0]]))
    assert real_rows_on_grid(np.array([[1.0, 2.0 ** -70], [1.0, 1.0]]))

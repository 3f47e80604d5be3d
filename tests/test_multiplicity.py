"""The grouped Glynn sum behind labelled batched plans, pinned on the CPU.

For a matrix whose distinct rows b_rho occur mu_rho times, Glynn's form of
Eq. 2 (a sign vector d over the rows, one row fixed at d = +1) is grouped by
the number k_rho of copies of each row with d = -1:

  perm = 2^(1-n) sum_(k_rho) prod_rho C(mu'_rho, k_rho) (-1)^(k_rho)
         prod_j (b_fj + sum_rho (mu'_rho - 2 k_rho) b_rho j),

mu' = mu less the fixed copy.  This file evaluates that sum in exact rational
arithmetic, with the same grouping the plan builder uses (a singleton row
fixed when there is one), and checks it against the permanent by brute force
and against closed forms.  It is independent of the CUDA path."""
import itertools
import math
from fractions import Fraction

import numpy as np
import pytest

import synthetic as syn


def grouped_glynn(A, labels):
    A = [[Fraction(v) for v in row] for row in A]
    n = len(A)
    groups = {}
    for r, l in enumerate(labels):
        groups.setdefault(l, []).append(r)
    order = sorted(groups.values(), key=lambda g: g[0])
    fixed = min(order, key=len)
    mus = [(g[0], len(g) - (1 if g is fixed else 0)) for g in order]
    mus = [(r, mu) for r, mu in mus if mu > 0]
    total = Fraction(0)
    for ks in itertools.product(*[range(mu + 1) for _, mu in mus]):
        w = 1
        for (r, mu), k in zip(mus, ks):
            w *= math.comb(mu, k) * (-1) ** k
        prod = Fraction(1)
        for j in range(n):
            prod *= A[fixed[0]][j] + sum((mu - 2 * k) * A[r][j] for (r, mu), k in zip(mus, ks))
        total += w * prod
    return total / 2 ** (n - 1), math.prod(mu + 1 for _, mu in mus)


def _repeat(B, labels):
    return np.array([B[l] for l in labels])


@pytest.mark.parametrize("labels", [[0, 0], [0, 0, 1], [0, 1, 0, 2], [3, 3, 3], [0, 0, 1, 1], [5, 1, 5, 5, 2],
                                    [0, 1, 2, 3, 1, 0], [7, 7, 7, 7, 7, 7]])
def test_grouped_sum_equals_bruteforce(oracle, labels):
    n = len(labels)
    B = syn.signed_real(max(labels) + 1 if max(labels) + 1 >= n else n, 8000 + n)[:, :n]
    A = _repeat(B, labels)
    got, terms = grouped_glynn(A, labels)
    assert got == oracle.perm_bruteforce(A)
    mult = [labels.count(l) for l in sorted(set(labels))]
    # a singleton is fixed when there is one: half of prod (mu + 1) terms
    if 1 in mult:
        assert 2 * terms == math.prod(m + 1 for m in mult)


def test_all_rows_equal_closed_form():
    """n equal rows r: perm = n! prod_j r_j, one group with mu' = n - 1."""
    r = syn.signed_real(6, 8100)[0]
    A = np.tile(r, (6, 1))
    got, terms = grouped_glynn(A, [4] * 6)
    assert got == math.factorial(6) * math.prod(Fraction(v) for v in r)
    assert terms == 6


def test_complex_rows_with_repeats(oracle):
    U = syn.haar_unitary(8, 8200)
    labels = [2, 5, 2, 0, 5, 2]
    A = U[labels, :6]
    re, im = oracle.perm_bruteforce(A.tolist())
    Ar = [[complex(v) for v in row] for row in A]
    # exact complex evaluation of the grouped sum: real and imaginary parts
    n = len(labels)
    groups = {}
    for r, l in enumerate(labels):
        groups.setdefault(l, []).append(r)
    order = sorted(groups.values(), key=lambda g: g[0])
    fixed = min(order, key=len)
    mus = [(g[0], len(g) - (1 if g is fixed else 0)) for g in order]
    mus = [(r, mu) for r, mu in mus if mu > 0]
    F = lambda z: (Fraction(z.real), Fraction(z.imag))
    tr, ti = Fraction(0), Fraction(0)
    for ks in itertools.product(*[range(mu + 1) for _, mu in mus]):
        w = 1
        for (r, mu), k in zip(mus, ks):
            w *= math.comb(mu, k) * (-1) ** k
        pr, pi = Fraction(1), Fraction(0)
        for j in range(n):
            sr, si = F(Ar[fixed[0]][j])
            for (r, mu), k in zip(mus, ks):
                ar, ai = F(Ar[r][j])
                sr += (mu - 2 * k) * ar
                si += (mu - 2 * k) * ai
            pr, pi = pr * sr - pi * si, pr * si + pi * sr
        tr += w * pr
        ti += w * pi
    assert tr / 2 ** (n - 1) == re and ti / 2 ** (n - 1) == im


# ------------------------------------------- the C++ planner, evaluated exactly

def _perm_exact(A):
    """Row-expansion subset DP over exact integers (the definition, Eq. 1)."""
    n = len(A)
    f = {0: 1}
    for i in range(n):
        g = {}
        for S, v in f.items():
            for j in range(n):
                if not S >> j & 1 and A[i][j]:
                    g[S | 1 << j] = g.get(S | 1 << j, 0) + v * A[i][j]
        f = g
    return f.get((1 << n) - 1, 0)


def _eval_units(A, units):
    """2 (-1)^(k-1) sum_u w_u sum_g (-1)^g prod_j x_j(g) in exact arithmetic."""
    k = len(A)
    total = Fraction(0)
    for u in units:
        G = u["gray_bits"]
        s = Fraction(0)
        for g in range(1 << G):
            gr = g ^ (g >> 1)
            prod = Fraction(1)
            for j in range(k):
                if u["fixed"] is None:  # plain sweep of A: rows are the factors
                    x = A[j][k - 1] + sum(A[j][c] * (1 if gr >> c & 1 else -1) for c in range(k - 1))
                else:  # transposed: columns are the factors
                    x = A[u["fixed"]][j] + sum(c * A[r][j] for r, c in u["repeated"])
                    x += sum(A[t][j] * (1 if gr >> b & 1 else -1) for b, t in enumerate(u["toggles"]))
                prod *= Fraction(x, 2)
            s += -prod if g & 1 else prod
        total += Fraction(u["weight"]) * s
    return 2 * (-1) ** (k - 1) * total


@pytest.mark.parametrize("labels", [
    [0, 1, 2, 3, 4, 5, 6, 7, 8, 9, 10, 3],      # one pair: 3 sweeps of 2^9 steps
    [0, 1, 2, 3, 4, 5, 6, 7, 8, 9, 5, 5],       # a triple
    [0, 1, 2, 3, 4, 5, 6, 7, 8, 1, 2, 9, 3],    # three pairs
    [0, 1, 0, 2, 1, 0, 2, 1, 0, 2, 1, 0],       # three modes: expanded back into Gray bits
    [4] * 10,                                   # all rows equal: the plain sweep pays
    list(range(9)),                             # all distinct: plain
])
def test_planned_units_sum_to_the_permanent(labels):
    pg = pytest.importorskip("paper_2502_16577_gb300")
    k = len(labels)
    g = syn.rng(8300 + k)
    B = g.integers(-3, 4, size=(max(labels) + 1, k))
    A = [[int(v) for v in B[l]] for l in labels]
    units = pg.batched_units(k, labels)
    assert 1 <= len(units) <= 64
    terms = sum(1 << u["gray_bits"] for u in units)
    assert terms <= 1 << (k - 1)
    if units[0]["fixed"] is not None:
        assert terms < 1 << (k - 1)
        assert all(u["gray_bits"] >= min(k - 1, 8) for u in units)
    assert _eval_units(A, units) == _perm_exact(A)


def test_planned_term_counts_on_the_boson_pattern():
    """Rows drawn with replacement: one repeated pair among 26 rows gives three
    sweeps of 2^23 steps (3/4 of 2^25); a triple gives four of 2^22."""
    pg = pytest.importorskip("paper_2502_16577_gb300")
    pair = list(range(25)) + [7]
    u = pg.batched_units(26, pair)
    assert [x["gray_bits"] for x in u] == [23] * 3
    assert sorted(x["weight"] for x in u) == [-2.0, 1.0, 1.0]
    triple = list(range(24)) + [7, 7]
    u = pg.batched_units(26, triple)
    assert [x["gray_bits"] for x in u] == [22] * 4
    assert pg.batched_units(26, None)[0]["gray_bits"] == 25


def test_equal_row_labels_on_the_host():
    pg = pytest.importorskip("paper_2502_16577_gb300")
    m = np.array([[1.0, 2.0, 0.5], [3.0, 4.0, 0.5], [1.0, 2.0, 0.5]])
    assert pg.equal_row_labels(m).tolist() == [0, 1, 0]
    U = syn.haar_unitary(16, 8400)
    r = [3, 7, 3, 3, 1, 7]
    labels = pg.equal_row_labels(U[r, :6])
    assert labels.tolist() == [0, 1, 0, 0, 4, 1]

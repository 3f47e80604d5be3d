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

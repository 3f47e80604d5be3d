"""Each planted mistake in the oracle (ORACLE_MUTANT in oracle/ryser.c) must be
caught by the pins: a dropped sign, a wrong column index, a dropped halving,
a wrong final factor, a flipped enter/leave sign, an off-by-one chunk start
state and a dropped first term; and, in the double-double sweeps with
magnitude sums, a wrong sign in the complex product and a dropped row weight.  The mistakes live only in separately built
variants of the oracle, never in the library path."""
import math
from fractions import Fraction

import numpy as np
import pytest

import synthetic as syn

MUTANTS = [1, 2, 3, 4, 5, 6, 7]


def _pins_pass(oracle, mutant):
    """A compact battery of the real-FP64 pins; True iff every pin holds."""
    checks = []
    for n in (5, 6):
        checks.append(abs(oracle.perm_f64(np.ones((n, n)), threads=4, mutant=mutant) - math.factorial(n)) < 1e-9)
    for n in (4, 5, 7):
        A = syn.signed_real(n, 31337 + n)
        exact = float(oracle.perm_bruteforce(A))
        got = oracle.perm_f64(A, threads=4, mutant=mutant)
        scale = float(oracle.perm_bruteforce(np.abs(A)))
        checks.append(abs(got - exact) <= 1e-12 * scale)
    return all(checks)


def test_unmutated_oracle_passes_battery(oracle):
    assert _pins_pass(oracle, 0)


@pytest.mark.parametrize("mutant", MUTANTS)
def test_planted_mistake_is_caught(oracle, mutant):
    oracle.load(mutant)
    assert not _pins_pass(oracle, mutant)


def _stats_pins_pass(oracle, mutant):
    """Gaussian-integer brute force (complex double-double sweep) and the closed
    forms of S and W for an all-equal matrix."""
    checks = []
    for n in (3, 5):
        g = np.random.default_rng(40 + n)
        A = (g.integers(-3, 4, (n, n)) + 1j * g.integers(-3, 4, (n, n))).astype(np.complex128)
        re, im = oracle.perm_bruteforce(A.tolist())
        r = oracle.ryser_cdd_range(A, 0, 2 ** (n - 1), threads=2, mutant=mutant)
        f = 2 * (-1) ** (n - 1)
        checks.append((Fraction(r["re_hi"]) + Fraction(r["re_lo"])) * f == re)
        checks.append((Fraction(r["im_hi"]) + Fraction(r["im_lo"])) * f == im)
    n, a = 7, 0.75
    r = oracle.ryser_dd_stats_range(np.full((n, n), a), 0, 2 ** (n - 1), threads=2, mutant=mutant)
    w = n * n * a ** n * sum(math.comb(n - 1, k) * abs(k + 1 - n / 2) ** (n - 1) for k in range(n))
    checks.append(abs(r["W"] - w) <= 1e-12 * w)
    return all(checks)


def test_unmutated_oracle_passes_stats_battery(oracle):
    assert _stats_pins_pass(oracle, 0)


@pytest.mark.parametrize("mutant", [8, 9])
def test_planted_stats_mistake_is_caught(oracle, mutant):
    oracle.load(mutant)
    assert not _stats_pins_pass(oracle, mutant)

"""Each planted mistake in the oracle (ORACLE_MUTANT in oracle/ryser.c) must be
caught by the pins: a dropped sign, a wrong column index, a dropped halving,
a wrong final factor, a flipped enter/leave sign, an off-by-one chunk start
state and a dropped first term.  The mistakes live only in separately built
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

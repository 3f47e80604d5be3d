"""Error bounds of the GPU sweeps, derived from their arithmetic.

Used by the parity tests to turn the oracle's magnitude sums (Sec. 5's error
analysis; oracle.ryser_dd_stats_range / ryser_cdd_range)

    S = sum_g |prod_i x_i(g)|,
    W = sum_g sum_i R_i prod_{k != i} |x_k(g)|,   R_i = sum_j |a_ij|,

into a bound on |GPU range sum - exact range sum| (the unscaled sum over the
Gray steps; perm = 2 (-1)^(n-1) times it).  Every rounding of a sweep is an
error of one of two kinds:

* an error in one factor x_i(g) of at most eps_x R_i (the row's fixed-point
  grid): moves the sum by at most eps_x W (first order);
* a relative error of the whole term of at most eps_t: moves it by eps_t S.

Dense real kernel (62-bit products of exact fixed-point rows):
  rows   Y_i = 2 x_i 2^s_i, s_i = 61 - k_i, R_i in [2^(k_i-1), 2^k_i), so one
         unit of Y_i is 2^-(s_i+1) <= R_i 2^-61 in x_i.
  column n-1 is rounded to an odd multiple (|dx_i| <= R_i 2^-61 per row);
  other columns are exact on the grid, else rounded to nearest
         (|dx_i| <= (n-1) R_i 2^-61 per row);
  product: v = M A / 2^64 with M >= 2^62 loses less than 1.5 units of v,
         i.e. at most 6 units of A = |Y_i|: |dx_i| <= 3 R_i 2^-60; counted as
         R_i 2^-58, which also covers a chain whose mantissa fell below 2^62
         after a factor with |Y_i| < 2^34 (a factor |Y_i| = 1, where x_i is 0
         before the odd rounding, empties the chain; tests/test_bounds.py
         checks such sweeps bit for bit against this bound);
  merge of the two chains: relative 1.5 2^-60; head/tail split: exact;
  double-double accumulation: below 2^-64 S for chunks of at most 2^20 steps.
  => |delta| <= 2 [(2^-58 + (1 + n_g) 2^-61) W + 2^-59 S]   (factor 2: second
     order terms), n_g = 0 when every entry of columns 0..n-2 lies on its row's
     grid, else n - 1.
The sparse kernel has the same rows (column n-1 exact, no odd rounding) and
two more chain merges: the same bound.

Dense complex kernel (signed 62-bit limbs, the larger part normalised to
[2^60, 2^61)):
  rows   s_i = 60 - k_i with k_i from sum_j |re| + |im| <= sqrt(2) R_i; one
         unit of Y_i is 2^-(s_i+1) <= sqrt(2) R_i 2^-60;
  entries rounded to nearest: |dx_i| <= n R_i 2^-60 (n_g = n off the grid);
  product: each part of v = z y / 2^62 loses at most 3 units, |z| >= 2^60,
         so |dx_i| <= 12 sqrt(2) units of Y_i <= 1.5 R_i 2^-56;
  lane-pair merge / padded row: relative 2^-55.
  => |delta| <= 2 [(1.5 2^-56 + n_g 2^-60) W + 2^-55 S]   (each of re, im).
A row-labelled batched plan sums Glynn terms of the transposed matrix grouped
by row multiplicity; grouping only merges equal terms with their counts as
weights, so S and W of the transposed sweep bound it.
"""
from __future__ import annotations

import math

import numpy as np


def real_rows_on_grid(A) -> bool:
    """True when every a_ij of columns 0..n-2 is a multiple of the row's
    fixed-point unit (taken one binary exponent coarser than the kernel's, so
    that a row sum rounding across a power of two cannot matter)."""
    A = np.asarray(A, dtype=np.float64)
    n = A.shape[0]
    for i in range(n):
        r = math.fsum(abs(float(v)) for v in A[i])
        if r == 0.0:
            continue
        k = math.frexp(r)[1] + 1
        s = 61 - k
        for v in A[i, : n - 1]:
            q = math.ldexp(float(v), s - 1)
            if q != math.floor(q):
                return False
    return True


def real_sweep_bound(S: float, W: float, n: int, on_grid: bool) -> float:
    ng = 0 if on_grid else n - 1
    return 2.0 * ((2.0 ** -58 + (1 + ng) * 2.0 ** -61) * W + 2.0 ** -59 * S)


def complex_sweep_bound(S: float, W: float, n: int, on_grid: bool = False) -> float:
    ng = 0 if on_grid else n
    return 2.0 * ((1.5 * 2.0 ** -56 + ng * 2.0 ** -60) * W + 2.0 ** -55 * S)


def dd_oracle_bound(S: float, n: int) -> float:
    """The double-double oracle itself: x exact or within 2^-104, every product
    within about 2^-103 per factor."""
    return (n + 2) * 2.0 ** -100 * S

"""Full-size parity of the named configurations against stored oracle values.

tests/golden/config_goldens.json holds, for every configuration, the
oracle's sum over the Gray steps (double-double x and products, Alg. 1; exact
integers for 0/1) of the very input the generators in synthetic/ produce,
with that input's SHA-256 and the magnitude sums S and W of Sec. 5's error
analysis.  It was written by tests/golden/make_config_goldens.py, which calls
only oracle/ and synthetic/.  Each test runs the GPU path on the same input at
full size and requires agreement within the bound that the kernel's
arithmetic implies (tests/_bounds.py), plus the task's accuracy bars:

* dense real n=24 uniform [0, 1) and n=40 uniform [-1, 1): all 2^23 / 2^39 steps;
* 0/1 n=36: perm() bit-exact, and the 2^35-step range sum mod 2^128;
* complex Haar 32 x 32: all 2^31 steps;
* sparse n=44 (density 0.2): a 2^30-step range in Alg. 2's column order
  against the oracle, and the full 2^43-step sweep against bounds that hold
  for every nonnegative matrix;
* the 8192-matrix boson batch: for every order k in 8..26, two matrices of
  the one-launch plan (plain and row-labelled) against the oracle.
"""
import hashlib
import json
import math
import os
from fractions import Fraction

import numpy as np
import pytest

import synthetic as syn
from _bounds import complex_sweep_bound, dd_oracle_bound, real_rows_on_grid, real_sweep_bound

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "config_goldens.json")


@pytest.fixture(scope="module")
def gold():
    with open(GOLDEN) as f:
        return json.load(f)


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


def _x(h: str) -> float:
    return float.fromhex(h)


def _same_input(A, entry):
    d = hashlib.sha256(np.ascontiguousarray(A).tobytes()).hexdigest()
    assert d == entry["sha256"], (
        "the generator produced other bytes than the stored oracle value describes "
        f"(stored on {entry.get('host')}); rerun tests/golden/make_config_goldens.py on this platform")


def _entry(gold, name):
    assert name in gold, f"{name} missing from {GOLDEN}"
    return gold[name]


def test_cfg1_dense_real_24_full(pg, gold):
    A = syn.dense_real_24()
    g = _entry(gold, "real24")
    _same_input(A, g)
    n = 24
    want = Fraction(_x(g["hi"])) + Fraction(_x(g["lo"]))
    S, W = _x(g["S"]), _x(g["W"])
    tol = real_sweep_bound(S, W, n, real_rows_on_grid(A)) + dd_oracle_bound(S, n)
    hi, lo = pg.perm_range(_dev(A), 0, 1 << (n - 1))
    err = abs(Fraction(hi) + Fraction(lo) - want)
    assert err <= Fraction(tol), (float(err), tol)
    # perm() itself: the positive-input bar (relative 1e-10) and the bound
    perm_ref = float(2 * (-1) ** (n - 1) * want)
    got = pg.perm(_dev(A))
    assert abs(got - perm_ref) <= 1e-10 * abs(perm_ref)
    assert abs(got - perm_ref) <= 2 * tol + 2.0 ** -52 * abs(perm_ref)


def test_cfg2a_dense_real_40_full(pg, gold):
    """All 2^39 Gray steps of the dense real n = 40 workload against the sum of
    the oracle's 64 double-double parts."""
    A = syn.dense_real_40()
    n = 40
    parts = [_entry(gold, f"real40_p{p:02d}") for p in range(64)]
    step = (1 << 39) // 64
    want, S, W = Fraction(0), 0.0, 0.0
    for p, e in enumerate(parts):
        _same_input(A, e)
        assert (e["g0"], e["g1"]) == (p * step, (p + 1) * step)
        want += Fraction(_x(e["hi"])) + Fraction(_x(e["lo"]))
        S += _x(e["S"])
        W += _x(e["W"])
    tol = real_sweep_bound(S, W, n, real_rows_on_grid(A)) + dd_oracle_bound(S, n)
    hi, lo = pg.perm_range(_dev(A), 0, 1 << 39)
    err = abs(Fraction(hi) + Fraction(lo) - want)
    assert err <= Fraction(tol), (float(err), tol, float(want))
    perm_ref = float(2 * (-1) ** (n - 1) * want)
    got = pg.perm(_dev(A))
    assert abs(got - perm_ref) <= 2 * tol + 2.0 ** -52 * abs(perm_ref), (got, perm_ref)
    # the task's bar for signed inputs is |delta| <= 1e-10 perm(|A|); since
    # perm(|A|) >= |perm(A)|, this relative check is stronger
    assert abs(got - perm_ref) <= 1e-10 * abs(perm_ref), (got, perm_ref)


def test_cfg2b_binary_36_full(pg, gold):
    A = syn.binary_36()
    n = 36
    gp, gr = _entry(gold, "bin36_perm"), _entry(gold, "bin36_range")
    _same_input(A, gp)
    _same_input(A, gr)
    want = int(gp["perm_mod_2^128"])
    assert gp["bregman_log2"] < 127  # so perm < 2^128 and the residue is perm itself
    assert pg.perm(_dev(A)) == want
    part = pg.perm_range(_dev(A), 0, 1 << (n - 1))  # mod 2^192
    assert part % (1 << 128) == int(gr["sum_mod_2^128"])
    # Eq. 2 with doubled rows: the full sum is (-1)^(n-1) 2^(n-1) perm(A)
    assert part == ((-1) ** (n - 1) * (1 << (n - 1)) * want) % (1 << 192)


def test_cfg2c_complex_32_full(pg, gold):
    U = syn.complex_32()
    n = 32
    g = _entry(gold, "cplx32")
    _same_input(U, g)
    S, W = _x(g["S"]), _x(g["W"])
    tol = complex_sweep_bound(S, W, n) + dd_oracle_bound(S, n)
    got = pg.perm_range(_dev(U), 0, 1 << (n - 1))
    wr = Fraction(_x(g["re_hi"])) + Fraction(_x(g["re_lo"]))
    wi = Fraction(_x(g["im_hi"])) + Fraction(_x(g["im_lo"]))
    er = abs(Fraction(got[0]) + Fraction(got[1]) - wr)
    ei = abs(Fraction(got[2]) + Fraction(got[3]) - wi)
    assert er <= Fraction(tol) and ei <= Fraction(tol), (float(er), float(ei), tol)
    p = pg.perm(_dev(U))
    ref = complex(float(wr), float(wi)) * 2 * (-1) ** (n - 1)
    assert abs(p - ref) <= 2 * math.sqrt(2) * tol + 2.0 ** -52 * abs(ref)
    assert abs(p) <= 1.0  # |perm(U)| <= 1 for a unitary U


def _sparse_dev(A):
    import torch

    cp, ri, cv = syn.to_ccs(A)
    return tuple(torch.from_numpy(np.ascontiguousarray(x)).cuda() for x in (cp, ri, cv))


def test_cfg3_sparse_44_range(pg, gold):
    """2^30 steps of the sparse n = 44 workload (Alg. 2's column order) against
    the oracle's double-double sweep of the same steps."""
    A = syn.sparse_44()
    n = 44
    g = _entry(gold, "sparse44_range")
    _same_input(A, g)
    S, W = _x(g["S"]), _x(g["W"])
    tol = real_sweep_bound(S, W, n, real_rows_on_grid(A)) + dd_oracle_bound(S, n)
    cp, ri, cv = _sparse_dev(A)
    hi, lo = pg.perm_sparse_range(n, cp, ri, cv, g["g0"], g["g1"], paper_order=True)
    want = Fraction(_x(g["hi"])) + Fraction(_x(g["lo"]))
    err = abs(Fraction(hi) + Fraction(lo) - want)
    assert err <= Fraction(tol), (float(err), tol, float(want))


def _max_matching_product(A) -> float:
    """max over perfect matchings of prod a_{i, sigma(i)} (a lower bound of
    perm(A) for A >= 0), by an assignment search on -log a."""
    from scipy.optimize import linear_sum_assignment

    with np.errstate(divide="ignore"):
        cost = np.where(A > 0, -np.log(np.where(A > 0, A, 1.0)), 1e300)
    r, c = linear_sum_assignment(cost)
    return float(np.prod(A[r, c]))


def test_cfg3_sparse_44_full_sweep(pg):
    """The full 2^43-step sparse sweep of the n = 44 workload (no CPU oracle can
    do it): status OK, and max_sigma prod a_{i,sigma(i)} <= perm(A) <= prod_i r_i,
    which hold for every nonnegative matrix."""
    A = syn.sparse_44()
    n = 44
    cp, ri, cv = _sparse_dev(A)
    got = pg.perm_sparse(n, cp, ri, cv)
    assert np.isfinite(got)
    assert _max_matching_product(A) <= got * (1 + 1e-12)
    assert got <= float(np.prod(A.sum(axis=1))) * (1 + 1e-12)


def _boson_entries(gold, prefix):
    return sorted(((e["index"], e) for k, e in gold.items() if k.startswith(prefix)), key=lambda t: t[0])


def test_cfg4_batched_boson_every_order(pg, gold):
    """The 8192-matrix boson batch in one launch (plain plan, and with the drawn
    modes as row labels): two matrices of every order k = 8..26 against the
    oracle's complex double-double sweep."""
    mats, rows = syn.batched_boson(with_rows=True)
    plain = dict(_boson_entries(gold, "boson_k"))
    trans = dict(_boson_entries(gold, "bosonT_k"))
    assert sorted({mats[i].shape[0] for i in plain}) == list(range(8, 27))
    assert set(plain) == set(trans)
    plan = pg.BatchPlan(mats)
    res_plain = plan.run()
    plan.close()
    plan = pg.BatchPlan(mats, row_labels=rows)
    res_lab = plan.run()
    plan.close()
    for i, g in plain.items():
        A = mats[i]
        k = A.shape[0]
        _same_input(A, g)
        _same_input(np.ascontiguousarray(A.T), trans[i])
        f = 2 * (-1) ** (k - 1)
        ref = complex(_x(g["re_hi"]) + _x(g["re_lo"]), _x(g["im_hi"]) + _x(g["im_lo"])) * f
        t = trans[i]
        ref_t = complex(_x(t["re_hi"]) + _x(t["re_lo"]), _x(t["im_hi"]) + _x(t["im_lo"])) * f
        tol_a = 2 * (complex_sweep_bound(_x(g["S"]), _x(g["W"]), k) + dd_oracle_bound(_x(g["S"]), k))
        tol_t = 2 * (complex_sweep_bound(_x(t["S"]), _x(t["W"]), k) + dd_oracle_bound(_x(t["S"]), k))
        # perm(A^T) = perm(A): the two oracle sweeps agree
        assert abs(ref - ref_t) <= tol_a + tol_t, (i, k)
        ulp = 2.0 ** -52 * abs(ref)
        assert abs(res_plain[i] - ref) <= math.sqrt(2) * tol_a + ulp, (i, k, res_plain[i], ref)
        # a labelled matrix runs either grouped sweeps of A^T or, where grouping
        # does not pay, the plain sweep of A
        assert abs(res_lab[i] - ref) <= math.sqrt(2) * max(tol_a, tol_t) + ulp, (i, k, res_lab[i], ref)

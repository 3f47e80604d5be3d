"""Batched complex permanents (one graph replay) against the oracle and the
single-matrix entry point."""
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


def test_uneven_sizes_vs_oracle(pg, oracle):
    mats = syn.boson_submatrices(300, 11, 1, 14, 64)
    plan = pg.BatchPlan(mats)
    got = plan.run()
    for m, g in zip(mats, got):
        want = oracle.perm_dp_c128(m)
        assert abs(g - want) <= 1e-13 * max(1.0, oracle.perm_dp_f64(np.abs(m)))
    # replay gives the same bits
    assert np.array_equal(plan.run(), got)
    plan.close()


def test_large_k_chunked_vs_single(pg):
    import torch

    mats = syn.boson_submatrices(40, 12, 15, 22, 128)
    plan = pg.BatchPlan(mats)
    got = plan.run()
    for m, g in zip(mats, got):
        single = pg.perm(torch.from_numpy(np.ascontiguousarray(m)).cuda())
        assert abs(g - single) <= 1e-13
    plan.close()


def test_autotune_keeps_results(pg, oracle):
    mats = syn.boson_submatrices(200, 13, 8, 18, 64)
    plan = pg.BatchPlan(mats, autotune_rounds=1)
    info = [plan.info(k) for k in range(8, 19)]
    assert all(i["c"] >= 0 for i in info)
    got = plan.run()
    for m, g in zip(mats[:40], got[:40]):
        assert abs(g - oracle.perm_dp_c128(m)) <= 1e-12
    plan.close()


def test_invalid_entries_flagged(pg):
    mats = syn.boson_submatrices(5, 14, 3, 6, 16)
    mats[2] = mats[2].copy()
    mats[2][0, 0] = complex(np.nan, 0.0)
    plan = pg.BatchPlan(mats)
    with pytest.raises(pg.PermError):
        plan.run()
    st = plan.status.cpu().numpy()
    assert st[2] == 1 and (np.delete(st, 2) == 0).all()
    plan.close()


def test_real_plan_uneven_sizes_vs_oracle(pg, oracle):
    """float64 plans: the integer product chains of the real kernel per matrix,
    lane mode (small k) and chunked mode (k > 14)."""
    g = syn.rng(15)
    ks = [1, 2, 3, 5, 8, 11, 14, 15, 18, 21] * 12
    mats = [2.0 * g.random((k, k)) - 1.0 for k in ks]
    plan = pg.BatchPlan(mats, dtype="float64")
    got = plan.run()
    assert got.dtype == np.float64
    for m, v in zip(mats, got):
        want = oracle.perm_dp_f64(m)
        assert abs(v - want) <= 1e-13 * oracle.perm_dp_f64(np.abs(m))
    assert np.array_equal(plan.run(), got)
    plan.close()


def test_real_plan_matches_single_matrix_kernel_and_autotune(pg):
    import torch

    mats = [syn.uniform_real(k, 1600 + k) for k in range(16, 25)] * 3
    plan = pg.BatchPlan(mats, dtype="float64", autotune_rounds=1)
    got = plan.run()
    for m, v in zip(mats, got):
        single = pg.perm(torch.from_numpy(np.ascontiguousarray(m)).cuda())
        assert v == pytest.approx(single, rel=1e-13)
    plan.close()
    bad = [syn.signed_real(4, 1700), syn.signed_real(5, 1701)]
    bad[1][2, 2] = np.inf
    plan = pg.BatchPlan(bad, dtype="float64")
    with pytest.raises(pg.PermError):
        plan.run()
    assert plan.status.cpu().numpy().tolist() == [0, 1]
    plan.close()


# ---------------------------------------------------- labelled (repeated) rows

def test_labeled_boson_plan_vs_oracle(pg, oracle):
    """Rows drawn with replacement from a small unitary (many repeats): the
    multiplicity sweeps match the oracle and the unlabelled plan."""
    mats, rows = syn.boson_submatrices(400, 21, 2, 16, 24, with_rows=True)
    assert sum(len(set(r.tolist())) < len(r) for r in rows) > 150
    plan = pg.BatchPlan(mats, row_labels=rows)
    got = plan.run()
    plain = pg.BatchPlan(mats).run()
    for m, g, p in zip(mats, got, plain):
        scale = max(1.0, oracle.perm_dp_f64(np.abs(m)))
        assert abs(g - oracle.perm_dp_c128(m)) <= 1e-12 * scale
        assert abs(g - p) <= 1e-12 * scale
    assert np.array_equal(plan.run(), got)
    plan.close()


def test_labeled_chunked_sizes_and_autotune(pg):
    """k = 17..24 with repeats: chunked sweeps on lane pairs with fewer Gray
    bits than k - 1, before and after autotuning."""
    import torch

    mats, rows = syn.boson_submatrices(24, 22, 17, 24, 24, with_rows=True)
    plan = pg.BatchPlan(mats, row_labels=rows)
    got = plan.run()
    for m, g in zip(mats, got):
        single = pg.perm(torch.from_numpy(np.ascontiguousarray(m)).cuda())
        assert abs(g - single) <= 1e-12 * max(1.0, abs(single))
    plan.close()
    plan = pg.BatchPlan(mats[:8], row_labels=rows[:8], autotune_rounds=1)
    tuned = plan.run()
    assert np.allclose(tuned, got[:8], rtol=1e-12, atol=1e-15)
    plan.close()


def test_labeled_real_plan_and_closed_forms(pg, oracle):
    """float64 plans with repeated rows; k equal rows r give k! prod_j r_j."""
    import math

    g = syn.rng(23)
    mats, labels = [], []
    for k in [2, 3, 4, 6, 9, 12, 15, 16, 19] * 4:
        lab = g.integers(0, max(2, k // 2), size=k).astype(np.int32)
        B = 2.0 * g.random((k, k)) - 1.0
        mats.append(B[lab])
        labels.append(lab)
    r = syn.signed_real(7, 2300)[0]
    mats.append(np.tile(r, (7, 1)))
    labels.append(np.full(7, 3, dtype=np.int32))
    plan = pg.BatchPlan(mats, dtype="float64", row_labels=labels)
    got = plan.run()
    for m, v in zip(mats[:-1], got[:-1]):
        assert abs(v - oracle.perm_dp_f64(m)) <= 1e-13 * oracle.perm_dp_f64(np.abs(m))
    assert got[-1] == pytest.approx(math.factorial(7) * float(np.prod(r)), rel=1e-14)
    plan.close()


def test_labels_all_distinct_are_the_plain_plan_and_bad_labels_flagged(pg):
    mats = syn.boson_submatrices(50, 24, 3, 14, 64)
    labels = [np.arange(m.shape[0], dtype=np.int32) for m in mats]
    assert np.array_equal(pg.BatchPlan(mats, row_labels=labels).run(), pg.BatchPlan(mats).run())
    wrong = [l.copy() for l in labels]
    wrong[7][1] = wrong[7][0]  # claims two different rows are equal
    plan = pg.BatchPlan(mats, row_labels=wrong)
    with pytest.raises(pg.PermError):
        plan.run()
    st = plan.status.cpu().numpy()
    assert st[7] == 1 and (np.delete(st, 7) == 0).all()
    plan.close()
    with pytest.raises(ValueError):
        pg.BatchPlan(mats[:2], row_labels=labels[:1])


def test_labeled_heavy_repeats_capped(pg):
    """k = 12..24 rows drawn from 3..6 modes: thousands of multiplicity
    combinations before the cap; the plan expands groups back into Gray bits
    (at most 64 sweeps of at least 2^min(k-1, 8) steps per matrix)."""
    import torch

    mats, labels = [], []
    for i, (k, modes) in enumerate([(12, 3), (16, 4), (18, 5), (20, 6), (22, 4), (24, 6), (13, 2), (9, 9)]):
        U = syn.haar_unitary(max(modes, k), 2500 + i)
        r = syn.rng(2600 + i).integers(0, modes, size=k).astype(np.int32)
        mats.append(np.ascontiguousarray(U[r, :k]))
        labels.append(r)
    plan = pg.BatchPlan(mats, row_labels=labels)
    got = plan.run()
    for m, g in zip(mats, got):
        single = pg.perm(torch.from_numpy(m).cuda())
        assert abs(g - single) <= 1e-11 * max(1.0, abs(single))
    plan.close()


def test_labeled_edges_k1_k32_and_real_heavy(pg, oracle):
    """k = 1 and 2 (nothing to group), k = 32 (the largest batched order, lane
    pairs) drawn from 12 modes, and a real plan with rows from 3 modes."""
    import torch

    U = syn.haar_unitary(32, 2700)
    r32 = syn.rng(2701).integers(0, 12, size=32).astype(np.int32)
    mats = [U[:1, :1].copy(), U[[5, 5], :2].copy(), np.ascontiguousarray(U[r32, :32])]
    labels = [np.array([0], np.int32), np.array([5, 5], np.int32), r32]
    got = pg.BatchPlan(mats, row_labels=labels).run()
    assert got[0] == mats[0][0, 0]
    assert abs(got[1] - 2 * mats[1][0, 0] * mats[1][0, 1]) <= 1e-15
    single = pg.perm(torch.from_numpy(mats[2]).cuda())
    assert abs(got[2] - single) <= 1e-11 * max(1.0, abs(single))
    g = syn.rng(2702)
    reals, rl = [], []
    for k in (10, 17, 23):
        lab = g.integers(0, 3, size=k).astype(np.int32)
        reals.append((2.0 * g.random((3, k)) - 1.0)[lab])
        rl.append(lab)
    gotr = pg.BatchPlan(reals, dtype="float64", row_labels=rl).run()
    for m, v in zip(reals, gotr):
        want = pg.perm(torch.from_numpy(np.ascontiguousarray(m)).cuda())
        assert abs(v - want) <= 1e-12 * oracle.perm_dp_f64(np.abs(m))


def test_auto_labels_match_the_drawn_modes(pg):
    """row_labels="auto" finds the equal rows on the host: the same grouping
    as the drawn modes, hence the same sweeps and the same bits."""
    mats, rows = syn.boson_submatrices(200, 25, 8, 18, 32, with_rows=True)
    by_mode = pg.BatchPlan(mats, row_labels=rows).run()
    auto = pg.BatchPlan(mats, row_labels="auto").run()
    assert np.array_equal(by_mode, auto)
    with pytest.raises(ValueError):
        pg.BatchPlan(mats[:2], row_labels="modes")


def test_per_call_buffers(pg, oracle):
    """perm_batched with buffers of the call: a second input laid out like the
    first is read instead of the plan's own, results go to the given output,
    and a call without buffers goes back to the plan's (no new plan, no
    capture)."""
    import torch

    m1 = syn.boson_submatrices(120, 61, 6, 18, 64)
    m2 = [0.3 * syn.complex_uniform(a.shape[0], 6200 + i) for i, a in enumerate(m1)]
    plan = pg.BatchPlan(m1)
    first = plan.run()
    A2 = torch.from_numpy(np.concatenate([b.reshape(-1) for b in m2]).astype(np.complex128)).cuda()
    out2 = torch.zeros_like(plan.out)
    st2 = torch.full_like(plan.status, -1)
    plan.run_async(A=A2, out=out2, status=st2)
    torch.cuda.synchronize()
    assert (st2 == 0).all()
    o = out2.cpu().numpy()
    got2 = o[0::2] + 1j * o[1::2]
    for m, g in zip(m2, got2):
        assert abs(g - oracle.perm_dp_c128(m)) <= 1e-12 * max(1.0, oracle.perm_dp_f64(np.abs(m)))
    assert np.array_equal(plan.run(), first)  # the plan's own buffers again
    plan.close()


def test_large_k_chunked_vs_oracle_every_order(pg, oracle):
    """Chunked lane-pair sweeps of orders 19..26 (the orders that carry most of
    the boson batch's work), plain and row-labelled, against the oracle's
    complex double-double sweep, within the bound of tests/_bounds.py (for the
    labelled plan, the larger of the bounds of A and of its transpose)."""
    from _bounds import complex_sweep_bound, dd_oracle_bound

    mats, rows = syn.boson_submatrices(16, 63, 19, 26, 256, with_rows=True)
    assert sorted({m.shape[0] for m in mats})[0] <= 20 and max(m.shape[0] for m in mats) >= 25
    plain = pg.BatchPlan(mats)
    lab = pg.BatchPlan(mats, row_labels=rows)
    rp, rl = plain.run(), lab.run()
    plain.close()
    lab.close()
    for m, a, b in zip(mats, rp, rl):
        k = m.shape[0]
        f = 2 * (-1) ** (k - 1)
        o = oracle.ryser_cdd_range(m, 0, 1 << (k - 1))
        t = oracle.ryser_cdd_range(np.ascontiguousarray(m.T), 0, 1 << (k - 1))
        want = complex(o["re_hi"] + o["re_lo"], o["im_hi"] + o["im_lo"]) * f
        tol_a = 2 * (complex_sweep_bound(o["S"], o["W"], k) + dd_oracle_bound(o["S"], k))
        tol_t = 2 * (complex_sweep_bound(t["S"], t["W"], k) + dd_oracle_bound(t["S"], k))
        ulp = 2.0 ** -52 * abs(want)
        assert abs(a - want) <= np.sqrt(2) * tol_a + ulp, (k, a, want, tol_a)
        assert abs(b - want) <= np.sqrt(2) * max(tol_a, tol_t) + ulp, (k, b, want, tol_t)


def test_lines_scaled_far_apart(pg, oracle):
    """perm(diag(r) A diag(d)) = perm(A) prod r prod d exactly: columns (and,
    for row-labelled plans, label groups of rows) scaled by powers of two far
    apart must give the unscaled oracle value times the factor, to the accuracy
    of the unscaled matrix (exact equilibration of the toggled lines)."""
    import math

    g = syn.rng(2400)
    ks = [8, 11, 14, 17, 20]
    cexp = {k: np.zeros(k, dtype=int) for k in ks}
    for k in ks:
        cexp[k][[1, 4, k - 3, k - 1]] = [-300, 300, -290, 40]
    # plain complex and real plans: columns scaled
    cm = [syn.haar_unitary(k, 2401 + k) for k in ks]
    rm = [syn.signed_real(k, 2420 + k) for k in ks]
    got_c = pg.BatchPlan([m * np.ldexp(1.0, cexp[m.shape[0]]) for m in cm]).run()
    got_r = pg.BatchPlan([m * np.ldexp(1.0, cexp[m.shape[0]]) for m in rm], dtype="float64").run()
    for m, v in zip(cm, got_c):
        e = int(cexp[m.shape[0]].sum())
        assert abs(complex(math.ldexp(v.real, -e), math.ldexp(v.imag, -e)) - oracle.perm_dp_c128(m)) <= 1e-13
    for m, v in zip(rm, got_r):
        e = int(cexp[m.shape[0]].sum())
        assert abs(math.ldexp(float(v), -e) - oracle.perm_f64(m)) <= 1e-12 * oracle.perm_f64(np.abs(m))
    # row-labelled plans (the repeated-row sweeps toggle rows): each label's
    # rows scaled alike
    lm, ll, lf = [], [], []
    for k in ks:
        lab = np.sort(g.integers(0, k // 2, size=k)).astype(np.int32)
        U = syn.haar_unitary(k, 2440 + k)
        while True:  # rows far apart, their product within the binary64 range
            re = g.integers(-280, 280, size=k)
            rexp = re[lab]
            if abs(int(rexp.sum())) <= 150:
                break
        lm.append((U[lab], U[lab] * np.ldexp(1.0, rexp)[:, None]))
        ll.append(lab)
        lf.append(int(rexp.sum()))
    got_l = pg.BatchPlan([s for _, s in lm], row_labels=ll).run()
    for (m, _), e, v in zip(lm, lf, got_l):
        assert abs(complex(math.ldexp(v.real, -e), math.ldexp(v.imag, -e)) - oracle.perm_dp_c128(m)) <= 1e-12

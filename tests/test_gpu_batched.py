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

"""Cancellation through perm_set_abort_word (mapped host memory read between
chunk groups): a set word makes a launch stop with PERM_EABORTED, a word set
while a long sweep runs ends it early, a cleared word leaves results intact.
Nothing here waits on the device: the kernels only read the word."""
import time

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


def _dev(A):
    import torch

    return torch.from_numpy(np.ascontiguousarray(A)).cuda()


def test_set_word_stops_every_sweep(pg, oracle):
    w = pg.AbortWord()
    try:
        A = syn.signed_real(22, 31)
        w.set()
        for M in (A, A.astype(np.complex128), syn.bernoulli01(22, 32)):
            with pytest.raises(pg.PermError) as e:
                pg.perm(_dev(M))
            assert e.value.code == pg.PERM_EABORTED
        cp, ri, cv = syn.to_ccs(syn.sparse_real(20, 33, 0.3))
        import torch

        with pytest.raises(pg.PermError):
            pg.perm_sparse(20, torch.from_numpy(cp).cuda(), torch.from_numpy(ri).cuda(), torch.from_numpy(cv).cuda())
        w.clear()
        assert pg.perm(_dev(A)) == pytest.approx(oracle.perm_dp_f64(A), abs=1e-12 * oracle.perm_dp_f64(np.abs(A)))
    finally:
        w.close()


def test_word_set_during_a_long_sweep(pg):
    import torch

    A = _dev(syn.signed_real(38, 34))
    out = torch.zeros(1, dtype=torch.float64, device="cuda")
    st = torch.full((1,), -1, dtype=torch.int32, device="cuda")
    w = pg.AbortWord()
    try:
        t0 = time.perf_counter()
        pg.perm_async(A, out, st)  # about 5 s uninterrupted
        time.sleep(0.2)
        w.set()
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        assert int(st.item()) == pg.PERM_EABORTED
        assert np.isnan(out.item())
        assert dt < 2.0, dt
    finally:
        w.close()
    # unregistered again: a short sweep completes
    B = syn.uniform_real(12, 35)
    assert pg.perm(_dev(B)) > 0.0


def test_time_budget_stops_every_sweep(pg):
    """perm_set_time_budget: a sweep that outlives its budget stops between
    chunk groups with PERM_ETIMEOUT, promptly, and a removed budget lets the
    same sweep finish.  The budget is made to run out by asking for 1 us; no
    wait is involved."""
    import torch

    A = _dev(syn.signed_real(36, 41))  # about 1.3 s uninterrupted
    out = torch.zeros(1, dtype=torch.float64, device="cuda")
    st = torch.full((1,), -1, dtype=torch.int32, device="cuda")
    pg.set_time_budget(1e-6)
    try:
        t0 = time.perf_counter()
        pg.perm_async(A, out, st)
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        assert int(st.item()) == pg.PERM_ETIMEOUT
        assert np.isnan(out.item())
        assert dt < 0.5, dt
        for M in (syn.haar_unitary(30, 42), syn.bernoulli01(34, 43)):
            with pytest.raises(pg.PermError) as e:
                pg.perm(_dev(M))
            assert e.value.code == pg.PERM_ETIMEOUT
        cp, ri, cv = (torch.from_numpy(x).cuda() for x in syn.to_ccs(syn.sparse_real(36, 44, 0.2)))
        with pytest.raises(pg.PermError) as e:
            pg.perm_sparse(36, cp, ri, cv)
        assert e.value.code == pg.PERM_ETIMEOUT
        mats = syn.boson_submatrices(64, 45, 20, 24, 64)
        plan = pg.BatchPlan(mats)
        with pytest.raises(pg.PermError) as e:
            plan.run()
        assert e.value.code == pg.PERM_ETIMEOUT
        B = torch.from_numpy(np.stack(syn.boson_submatrices(64, 46, 16, 16, 64))).cuda()
        with pytest.raises(pg.PermError) as e:
            pg.perm_grad_batched(B)
        assert e.value.code == pg.PERM_ETIMEOUT
        # a single real gradient
        with pytest.raises(pg.PermError) as e:
            pg.perm_grad(_dev(syn.signed_real(28, 50)))
        assert e.value.code == pg.PERM_ETIMEOUT
    finally:
        pg.set_time_budget(None)
    # without the budget the same launches complete (the plan is replayed
    # unchanged: the budget is read at every replay)
    pg.perm_async(A, out, st)
    torch.cuda.synchronize()
    assert int(st.item()) == pg.PERM_OK and np.isfinite(out.item())
    res = plan.run()
    assert np.all(np.isfinite(res))
    plan.close()
    p, G = pg.perm_grad_batched(B)
    assert torch.isfinite(G).all()


def test_abort_word_stops_batched_and_gradient(pg, oracle):
    import torch

    mats = syn.boson_submatrices(40, 47, 8, 14, 64)
    plan = pg.BatchPlan(mats)
    B = torch.from_numpy(np.stack(syn.boson_submatrices(8, 48, 12, 12, 64))).cuda()
    w = pg.AbortWord()
    try:
        w.set()
        with pytest.raises(pg.PermError) as e:
            plan.run()
        assert e.value.code == pg.PERM_EABORTED
        with pytest.raises(pg.PermError) as e:
            pg.perm_grad_batched(B)
        assert e.value.code == pg.PERM_EABORTED
        with pytest.raises(pg.PermError) as e:
            pg.perm_grad(_dev(syn.signed_real(20, 49)))
        assert e.value.code == pg.PERM_EABORTED
        w.clear()
        res = plan.run()
        for m, r in zip(mats, res):
            assert abs(r - oracle.perm_dp_c128(m)) <= 1e-12
        p, G = pg.perm_grad_batched(B)
        assert torch.isfinite(G).all()
    finally:
        w.close()
        plan.close()

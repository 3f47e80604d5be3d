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

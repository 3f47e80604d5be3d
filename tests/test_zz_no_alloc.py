"""perm_f64_noalloc, the entry point for callers that may not allocate device
memory (a framework owns the whole pool, or allocation is forbidden once a
loop runs): called through the C ABI, it must give what perm() gives for the
same real matrix, on two calls in a row (the scratch array it reuses keeps
the previous call's contents)."""
import ctypes

import numpy as np
import pytest

import synthetic as syn

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2502_16577_gb300 import build

    build.build()
    import paper_2502_16577_gb300 as pg

    lib = pg.load()
    lib.perm_f64_noalloc.restype = ctypes.c_int
    lib.perm_f64_noalloc.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
    return lib


@pytest.mark.parametrize("n,seed", [(13, 1), (24, 2), (31, 3)])
def test_noalloc_matches_perm(lib, oracle, n, seed):
    import torch

    A = syn.signed_real(n, 9000 + seed)
    dA = torch.from_numpy(A).cuda()
    stream = torch.cuda.current_stream()
    h = ctypes.c_void_p(stream.cuda_stream)
    ref = torch.zeros(1, dtype=torch.float64, device="cuda")
    ref_st = torch.full((1,), -1, dtype=torch.int32, device="cuda")
    assert lib.perm(ctypes.c_void_p(dA.data_ptr()), n, 0, ctypes.c_void_p(ref.data_ptr()),
                    ctypes.c_void_p(ref_st.data_ptr()), h) == 0
    results = []
    for _ in range(2):  # two calls in a row on the shared scratch array
        out = torch.full((1,), float("nan"), dtype=torch.float64, device="cuda")
        st = torch.full((1,), -1, dtype=torch.int32, device="cuda")
        assert lib.perm_f64_noalloc(ctypes.c_void_p(dA.data_ptr()), n, ctypes.c_void_p(out.data_ptr()),
                                    ctypes.c_void_p(st.data_ptr()), h) == 0
        stream.synchronize()
        assert int(st.item()) == 0
        results.append(float(out.item()))
    stream.synchronize()
    assert int(ref_st.item()) == 0
    want = float(ref.item())
    # same tolerance as the dense real parity tests: 1e-14 of perm(|A|)
    import paper_2502_16577_gb300 as pg

    scale = pg.perm(torch.from_numpy(np.abs(A)).cuda())
    for got in results:
        assert abs(got - want) <= 1e-14 * scale
    assert results[0] == results[1]


def test_noalloc_rejects_bad_arguments(lib):
    vp = ctypes.c_void_p
    assert lib.perm_f64_noalloc(vp(16), 64, vp(16), vp(0), vp(0)) == 2
    assert lib.perm_f64_noalloc(vp(0), 5, vp(16), vp(0), vp(0)) == 1

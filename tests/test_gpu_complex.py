"""Parity of the complex128 path (C ABI, GB300) with the oracle.
Bar: |delta| <= 1e-10 perm(|A|); the tighter checks follow from 60-bit
fixed-point rows, 60-bit products and one binary64 rounding per term."""
import itertools
import math

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

    return torch.from_numpy(np.ascontiguousarray(A, dtype=np.complex128)).cuda()


@pytest.mark.parametrize("n", range(1, 8))
def test_small_vs_bruteforce(pg, oracle, n):
    for seed in range(3):
        A = syn.complex_uniform(n, 8000 + 10 * n + seed)
        re, im = oracle.perm_bruteforce(A.tolist())
        got = pg.perm(_dev(A))
        scale = oracle.perm_dp_f64(np.abs(A))
        assert abs(got.real - float(re)) <= 1e-14 * scale
        assert abs(got.imag - float(im)) <= 1e-14 * scale


@pytest.mark.parametrize("n", [9, 12, 15, 16, 17, 19, 20, 21])
def test_unitary_vs_dp(pg, oracle, n):
    U = syn.haar_unitary(n, 8100 + n)
    want = oracle.perm_dp_c128(U)
    got = pg.perm(_dev(U))
    scale = oracle.perm_dp_f64(np.abs(U))
    assert abs(got - want) <= 1e-10 * scale
    assert abs(got - want) <= 1e-13
    assert abs(got) <= 1.0 + 1e-12
    assert abs(pg.perm(_dev(np.conj(U))) - np.conj(got)) <= 1e-14


def test_boson_normalisation(pg):
    m, k = 6, 3
    U = syn.haar_unitary(m, 7)
    total = 0.0
    for T in itertools.combinations_with_replacement(range(m), k):
        sub = U[list(T), :k]
        mult = math.prod(math.factorial(T.count(t)) for t in set(T))
        total += abs(pg.perm(_dev(sub))) ** 2 / mult
    assert total == pytest.approx(1.0, abs=1e-12)


def test_real_matrix_as_complex_matches_real_path(pg, oracle):
    A = syn.signed_real(14, 5)
    got = pg.perm(_dev(A.astype(np.complex128)))
    want = oracle.perm_dp_f64(A)
    assert abs(got.imag) <= 1e-14 * oracle.perm_dp_f64(np.abs(A))
    assert got.real == pytest.approx(want, abs=1e-13 * oracle.perm_dp_f64(np.abs(A)))


def test_range_partials(pg, oracle):
    U = syn.haar_unitary(17, 99)
    N = 2 ** 16
    for g0, g1 in [(0, 1), (0, 300), (1000, 40000), (N - 5, N)]:
        got = pg.perm_range(_dev(U), g0, g1)
        want = oracle.ryser_c128_range(U, g0, g1)
        assert abs((got[0] + got[1]) - (want[0] + want[1])) <= 1e-14
        assert abs((got[2] + got[3]) - (want[2] + want[3])) <= 1e-14


def test_config_complex_32(pg, oracle):
    """Haar 32 x 32 unitary: |perm| <= 1, conjugation symmetry, a sampled
    2^22-step sub-range against the oracle, and a block-diagonal 32 = 16 + 16
    unitary with a known permanent."""
    U = syn.complex_32()
    p = pg.perm(_dev(U))
    assert abs(p) <= 1.0
    assert abs(pg.perm(_dev(np.conj(U))) - np.conj(p)) <= 1e-13
    g0 = 3 * 2 ** 28 + 1
    got = pg.perm_range(_dev(U), g0, g0 + 2 ** 22)
    want = oracle.ryser_c128_range(U, g0, g0 + 2 ** 22)
    assert abs((got[0] + got[1]) - (want[0] + want[1])) <= 1e-12
    assert abs((got[2] + got[3]) - (want[2] + want[3])) <= 1e-12
    V1, V2 = syn.haar_unitary(16, 1), syn.haar_unitary(16, 2)
    M = syn.shuffle_rows_cols(syn.block_diagonal([V1, V2]), 4)
    want = oracle.perm_dp_c128(V1) * oracle.perm_dp_c128(V2)
    assert abs(pg.perm(_dev(M)) - want) <= 1e-13


def test_edge_cases(pg):
    import torch

    assert pg.perm(torch.zeros((0, 0), dtype=torch.complex128, device="cuda")) == 1.0
    assert pg.perm(_dev(np.array([[1.5 - 2j]]))) == 1.5 - 2j
    B = syn.complex_uniform(5, 1)
    B[1, 1] = complex(np.inf, 0)
    with pytest.raises(pg.PermError):
        pg.perm(_dev(B))

"""Sparse preprocessing of Sec. 4 end to end on the GPU: the decomposition's
leaves through the batched launch (order <= 32) and the dense / sparse
kernels (larger), recombined on the host, against the oracle."""
import numpy as np
import pytest

import synthetic as syn

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dec():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2502_16577_gb300 import build

    build.build()
    import paper_2502_16577_gb300 as pg
    from paper_2502_16577_gb300 import decomp

    pg.load()
    return decomp


@pytest.mark.parametrize("n,density,seed", [(14, 0.3, 1), (20, 0.2, 2), (24, 0.2, 3), (24, 0.15, 4), (26, 0.25, 5)])
def test_random_sparse_against_the_oracle(dec, oracle, n, density, seed):
    A = syn.sparse_real(n, 1200 + seed, density)
    got, info = dec.perm_sparse_decomp(A)
    want = oracle.perm_dp_f64(A) if n <= 22 else oracle.perm_f64(A)
    assert got == pytest.approx(want, rel=1e-10)
    assert info["leaf_steps"] <= info["plain_steps"]


def test_shuffled_block_diagonal_n44(dec, oracle):
    """Two 22 x 22 blocks at density 0.2, rows and columns shuffled: the
    Dulmage-Mendelsohn step splits the 2^43-step sweep into two of 2^21."""
    B1, B2 = syn.sparse_real(22, 1301, 0.2), syn.sparse_real(22, 1302, 0.2)
    A = syn.shuffle_rows_cols(syn.block_diagonal([B1, B2]), 1303)
    got, info = dec.perm_sparse_decomp(A)
    assert info["nblocks"] >= 2 and info["leaf_steps"] <= 2 * 2.0 ** 21
    want = oracle.perm_f64(B1) * oracle.perm_f64(B2)
    assert got == pytest.approx(want, rel=1e-10)


def _min_degree_core(n, seed, perms):
    """Union of random permutation matrices: every line keeps more than four
    nonzeros (so Alg. 4 leaves it whole) at density about perms / n."""
    g = syn.rng(seed)
    while True:
        M = np.zeros((n, n))
        for _ in range(perms):
            M[np.arange(n), g.permutation(n)] = 1.0
        if min((M != 0).sum(0).min(), (M != 0).sum(1).min()) > 4:
            return M * (0.25 + g.random((n, n)))


def test_large_leaves_use_the_single_matrix_kernels(dec):
    """Leaves of order > 32: a 34 x 34 core (dense, then sparse at density
    about 0.2) with two extra rows / columns of two nonzeros that the expansion
    folds away; checked against the dense GPU kernel on the full matrix."""
    import paper_2502_16577_gb300 as pg
    import torch

    for core in (syn.uniform_real(34, 1410) + 0.1, _min_degree_core(34, 1420, 7)):
        n = 36
        A = np.zeros((n, n))
        A[:34, :34] = core
        A[34, 3], A[34, 34] = 0.75, 0.5
        A[35, 35], A[35, 10] = 1.25, 0.5
        A[5, 35] = 0.25
        A[20, 34] = 0.5
        got, info = dec.perm_sparse_decomp(A)
        assert info["max_leaf_n"] == 34
        want = pg.perm(torch.from_numpy(A).cuda())
        assert got == pytest.approx(want, rel=1e-10)


def test_structurally_singular_and_trivial(dec):
    Z = syn.sparse_real(30, 1500, 0.2)
    Z[7, :] = 0.0
    assert dec.perm_sparse_decomp(Z)[0] == 0.0
    T = np.triu(0.5 + syn.rng(1501).random((40, 40)))
    assert dec.perm_sparse_decomp(T)[0] == pytest.approx(np.prod(np.diag(T)), rel=1e-14)


def test_leaves_with_equal_rows_use_the_multiplicity_sweep(dec, oracle):
    """Two dense 20 x 20 blocks whose rows repeat (12 distinct rows each),
    shuffled: the Dulmage-Mendelsohn blocks are the leaves, and their equal
    rows are labelled on the host, so the batched launch sums them over the
    row multiplicities."""
    g = syn.rng(1400)
    blocks = []
    for b in range(2):
        rows = 1.0 - g.random((12, 20))
        lab = np.concatenate([np.arange(12), g.integers(0, 12, size=8)])
        blocks.append(rows[lab])
    A = syn.shuffle_rows_cols(syn.block_diagonal(blocks), 1401)
    got, info = dec.perm_sparse_decomp(A)
    assert info["nblocks"] >= 2
    want = oracle.perm_dp_f64(blocks[0]) * oracle.perm_dp_f64(blocks[1])
    assert got == pytest.approx(want, rel=1e-10)

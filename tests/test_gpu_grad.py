"""The fused gradient (perm_grad / perm_grad_batched through the C ABI) on a
GB300: against the oracle's minor permanents, closed forms, exact central
differences of the oracle (perm is affine in every entry), the row-expansion
identity and torch.autograd.gradcheck.

Tolerance of G_kl (besides the 1e-10 perm(|minor|) bar): every term
v_k(g) = prod_{i != k} x_i(g) carries a relative error below 2^-52 (62-bit
products, one rounding to binary64); the terms are summed in binary64 in
chunks of at most 2^9 steps, then over 16 chunks, then over at most a few
hundred block-items per CTA, then in double-double.  The recursive-summation
bound is then below (2^9 + 16 + 512 + 2) 2^-53 S_k < 2^-42 S_k with
S_k = sum_g |v_k(g)|, so 2^-40 S_k holds with margin; S_k is computed here
exactly enough in numpy for n <= 16."""
import itertools
import math

import numpy as np
import pytest

import synthetic as syn

pytestmark = pytest.mark.gpu

TOL_S = 2.0 ** -40


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


def _minor(A, k, l):
    return np.delete(np.delete(A, k, 0), l, 1)


def _abs_scale(A):
    """S_k = sum over the 2^(n-1) Gray subsets of prod_{i != k} |x_i| (n <= 16)."""
    n = A.shape[0]
    if n == 1:
        return np.ones(1)
    signs = np.array(list(itertools.product((-1.0, 1.0), repeat=n - 1)))
    D = np.concatenate([signs, np.ones((signs.shape[0], 1))], axis=1)  # delta_l, column n-1 always in
    X = np.abs(0.5 * (D @ A.T))  # (2^(n-1), n): |x_i| per subset
    pre = np.cumprod(np.concatenate([np.ones((X.shape[0], 1)), X[:, :-1]], axis=1), axis=1)
    suf = np.cumprod(np.concatenate([np.ones((X.shape[0], 1)), X[:, :0:-1]], axis=1), axis=1)[:, ::-1]
    return (pre * suf).sum(axis=0)


def _check_minors(G, A, oracle, cplx=False, rows=None, cols=None, scale=None):
    n = A.shape[0]
    S = _abs_scale(A) if scale is None and n <= 16 else scale
    for k in rows if rows is not None else range(n):
        for l in cols if cols is not None else range(n):
            if n == 1:
                want, bar = 1.0, 1.0
            else:
                M = _minor(A, k, l)
                want = oracle.perm_c128(M) if cplx else oracle.perm_f64(M)
                bar = oracle.perm_dp_f64(np.abs(M)) if n <= 21 else oracle.perm_f64(np.abs(M))
            err = abs(G[k, l] - want)
            assert err <= 1e-10 * bar, (k, l, err, bar)
            if S is not None:
                assert err <= TOL_S * S[k], (k, l, err, S[k])


@pytest.mark.parametrize("n", [1, 2, 3, 4, 5, 7, 8, 9, 12, 16, 17, 20])
def test_real_gradient_is_the_minor_permanents(pg, oracle, n):
    A = syn.signed_real(n, 10000 + n)
    p, G = pg.perm_grad(_dev(A))
    G = G.cpu().numpy()
    _check_minors(G, A, oracle)
    scale = oracle.perm_dp_f64(np.abs(A)) if n <= 20 else 1.0
    assert abs(p - oracle.perm_f64(A)) <= 1e-12 * scale


@pytest.mark.parametrize("n", [1, 2, 3, 6, 8, 9, 13, 16, 17, 22])
def test_complex_gradient_is_the_minor_permanents(pg, oracle, n):
    A = syn.haar_unitary(max(n, 1), 10100 + n)
    p, G = pg.perm_grad(_dev(A))
    G = G.cpu().numpy()
    _check_minors(G, A, oracle, cplx=True, rows=None if n <= 16 else (0, n // 2, n - 1))
    assert abs(p - oracle.perm_c128(A)) <= 1e-12


def test_positive_real_matches_the_subset_dp(pg, oracle):
    # positive entries: the DP is free of cancellation, so this measures the
    # gradient's true relative error on an ill-conditioned Ryser sum
    n = 18
    A = syn.uniform_real(n, 10200)
    _, G = pg.perm_grad(_dev(A))
    G = G.cpu().numpy()
    for k, l in ((0, 0), (5, 11), (17, 3), (17, 17)):
        want = oracle.perm_dp_f64(_minor(A, k, l))
        assert abs(G[k, l] - want) <= 1e-10 * want


def test_closed_forms(pg):
    import torch

    # J_n: every minor is J_(n-1), G = (n-1)! everywhere (the all-equal
    # matrix is Ryser's worst cancellation: S_k / G_kl is about 40 at n = 16)
    for n in (5, 11, 16):
        J = np.ones((n, n))
        _, G = pg.perm_grad(_dev(J))
        want = math.factorial(n - 1)
        S = _abs_scale(J)
        assert np.max(np.abs(G.cpu().numpy() - want)) <= min(TOL_S * S[0], 1e-10 * want)
    # diagonal: G_kk = prod_{i != k} a_ii; off-diagonal minors have a zero row.
    # Here S_k = prod_{i != k} a_ii exactly.
    d = 0.5 + syn.rng(10301).random(12)
    p, G = pg.perm_grad(_dev(np.diag(d)))
    G = G.cpu().numpy()
    for k in range(12):
        Sk = np.prod(np.delete(d, k))
        assert abs(G[k, k] - Sk) <= TOL_S * Sk
        assert np.max(np.abs(np.delete(G[k], k))) <= TOL_S * Sk
    assert p == pytest.approx(np.prod(d), rel=1e-13)
    # 2 x 2: perm = ad + bc, G = [[d, c], [b, a]]
    p, G = pg.perm_grad(_dev(np.array([[1.5, -2.0], [0.25, 3.0]])))
    assert G.cpu().numpy().tolist() == [[3.0, 0.25], [-2.0, 1.5]]
    assert p == 1.5 * 3.0 + (-2.0) * 0.25
    # n = 0: the empty permanent, no entries
    out = torch.zeros(1, dtype=torch.float64, device="cuda")
    st = torch.full((1,), -1, dtype=torch.int32, device="cuda")
    pg.perm_grad_async(torch.zeros((0, 0), dtype=torch.float64, device="cuda"), out,
                       torch.zeros((0, 0), dtype=torch.float64, device="cuda"), st)
    torch.cuda.synchronize()
    assert out.item() == 1.0 and st.item() == 0


def test_zero_rows_and_bad_input(pg, oracle):
    A = syn.signed_real(9, 10400)
    A[4] = 0.0
    p, G = pg.perm_grad(_dev(A))
    G = G.cpu().numpy()
    assert p == 0.0
    assert np.all(G[np.arange(9) != 4] == 0.0)
    for l in range(9):
        assert abs(G[4, l] - oracle.perm_f64(_minor(A, 4, l))) <= 1e-13 * oracle.perm_dp_f64(np.abs(_minor(A, 4, l)))
    A[7] = 0.0
    p, G = pg.perm_grad(_dev(A))
    assert p == 0.0 and not np.any(G.cpu().numpy())
    B = syn.signed_real(6, 10401)
    B[2, 3] = np.nan
    with pytest.raises(pg.PermError):
        pg.perm_grad(_dev(B))


@pytest.mark.parametrize("n", [14, 15, 18, 21, 24, 26])
def test_single_real_orders_14_to_26(pg, oracle, n):
    """One real matrix of each order (R = 2, 3, 4 rows per lane): sampled
    minors against the oracle, perm against the oracle, and the row expansion."""
    A = syn.signed_real(n, 10500 + n)
    p, G = pg.perm_grad(_dev(A))
    G = G.cpu().numpy()
    picks = (0, n // 3, n - 2, n - 1)
    _check_minors(G, A, oracle, rows=picks if n > 18 else None, cols=picks if n > 18 else None)
    assert abs(p - oracle.perm_f64(A)) <= 1e-10 * oracle.perm_f64(np.abs(A))
    for i in range(n):
        assert abs(float(np.dot(A[i], G[i])) - p) <= 1e-9 * float(np.sum(np.abs(A[i] * G[i])))


def test_single_real_edge_cases(pg, oracle):
    # a zero row (its Y stays 0: every product but its own minor vanishes),
    # entries of very different size, and a nonfinite entry
    A = syn.signed_real(15, 10600)
    A[6] = 0.0
    p, G = pg.perm_grad(_dev(A))
    G = G.cpu().numpy()
    assert p == 0.0
    assert np.all(G[np.arange(15) != 6] == 0.0)
    for l in (0, 7, 14):
        assert abs(G[6, l] - oracle.perm_f64(_minor(A, 6, l))) <= 1e-11 * oracle.perm_f64(np.abs(_minor(A, 6, l)))
    # perm is multilinear in rows and columns: a row times 2^300 and a column
    # times 2^-200 scale every minor by an exact power of two, so the
    # references come from the unscaled matrix B0
    B0 = syn.signed_real(16, 10601)
    B = B0.copy()
    B[3] *= 2.0 ** 300
    B[:, 5] *= 2.0 ** -200
    p, G = pg.perm_grad(_dev(B))
    G = G.cpu().numpy()
    assert abs(p - math.ldexp(oracle.perm_f64(B0), 100)) <= math.ldexp(1e-10 * oracle.perm_f64(np.abs(B0)), 100)
    for k, l in ((3, 5), (0, 0), (3, 0), (15, 5)):
        M = _minor(B0, k, l)
        e = (300 if k != 3 else 0) - (200 if l != 5 else 0)
        err = abs(G[k, l] - math.ldexp(oracle.perm_f64(M), e))
        assert err <= math.ldexp(1e-10 * oracle.perm_f64(np.abs(M)), e), (k, l)
    B[2, 9] = np.inf
    with pytest.raises(pg.PermError) as e:
        pg.perm_grad(_dev(B))
    assert e.value.code == pg.PERM_EINVAL


def test_gradient_columns_scaled_far_apart(pg, oracle):
    """Columns scaled by 2^-300 .. 2^300, real (one matrix and a batch) and
    complex: every minor is the unscaled oracle minor times an exact power of
    two (the sweep equilibrates the columns and scales G back)."""
    n = 12
    ce = np.zeros(n, dtype=int)
    ce[[1, 4, 8, 11]] = [-300, 300, -290, 40]
    d = np.ldexp(1.0, ce)
    for A0, cplx in ((syn.signed_real(n, 10700), False), (syn.haar_unitary(n, 10701), True)):
        p, G = pg.perm_grad(_dev(A0 * d))
        G = G.cpu().numpy()
        want_p = oracle.perm_c128(A0) if cplx else oracle.perm_f64(A0)
        assert abs(p * 2.0 ** -int(ce.sum()) - want_p) <= 1e-12 * oracle.perm_f64(np.abs(A0))
        for k in range(n):
            for l in range(n):
                M = _minor(A0, k, l)
                e = int(ce.sum() - ce[l])
                want = oracle.perm_c128(M) if cplx else oracle.perm_f64(M)
                err = abs(G[k, l] * 2.0 ** -e - want)
                assert err <= 1e-12 * oracle.perm_f64(np.abs(M)), (cplx, k, l, err)
    B = np.stack([syn.signed_real(n, 10710 + i) for i in range(5)])
    p, G = pg.perm_grad_batched(_dev(B * d))
    G = G.cpu().numpy()
    for i in range(5):
        for k, l in ((0, 1), (3, 4), (11, 0), (6, 11)):
            M = _minor(B[i], k, l)
            e = int(ce.sum() - ce[l])
            assert abs(G[i, k, l] * 2.0 ** -e - oracle.perm_f64(M)) <= 1e-12 * oracle.perm_f64(np.abs(M)), (i, k, l)


def test_row_expansion_identity(pg):
    for n, seed in ((9, 1), (16, 2), (23, 3), (32, 4)):
        A = syn.signed_real(n, 11000 + seed)
        p, G = pg.perm_grad(_dev(A))
        G = G.cpu().numpy()
        scale = pg.perm(_dev(np.abs(A)))
        for i in range(n):
            dot = float(np.dot(A[i], G[i]))
            assert abs(dot - p) <= 1e-10 * scale
            assert abs(dot - p) <= 1e-9 * float(np.sum(np.abs(A[i] * G[i])))
        assert abs(float(np.sum(A * G)) - n * p) <= 1e-9 * float(np.sum(np.abs(A * G)))
        assert abs(p - pg.perm(_dev(A))) <= 1e-9 * float(np.sum(np.abs(A[0] * G[0])))


def test_central_differences_of_the_oracle(pg, oracle):
    # perm is affine in each entry, so the central difference is exact up to
    # the oracle's rounding, for any step h
    n = 10
    A = syn.uniform_real(n, 12000)
    _, G = pg.perm_grad(_dev(A))
    G = G.cpu().numpy()
    for k, l in ((0, 0), (3, 7), (9, 2), (5, 9)):
        h = 0.25
        Ap, Am = A.copy(), A.copy()
        Ap[k, l] += h
        Am[k, l] -= h
        fd = (oracle.perm_dp_f64(Ap) - oracle.perm_dp_f64(Am)) / (2 * h)
        assert fd == pytest.approx(G[k, l], rel=1e-12)


def test_deterministic(pg):
    A = _dev(syn.signed_real(21, 12050))
    _, G1 = pg.perm_grad(A)
    _, G2 = pg.perm_grad(A)
    assert bool((G1 == G2).all())


def test_batched_equals_single(pg, oracle):
    import torch

    Ms = np.stack(syn.boson_submatrices(40, 12060, 11, 11, 64))
    out, G = pg.perm_grad_batched(_dev(Ms))
    out, G = out.cpu().numpy(), G.cpu().numpy()
    for p in (0, 17, 39):
        v, Gs = pg.perm_grad(_dev(Ms[p]))
        assert abs(out[p] - v) <= 1e-13
        assert np.max(np.abs(G[p] - Gs.cpu().numpy())) <= 1e-13
        assert abs(out[p] - oracle.perm_c128(Ms[p])) <= 1e-12
    _check_minors(G[5], Ms[5], oracle, cplx=True)
    R = np.stack([syn.signed_real(7, 12070 + i) for i in range(300)])
    out, G = pg.perm_grad_batched(_dev(R))
    out, G = out.cpu().numpy(), G.cpu().numpy()
    for p in (0, 150, 299):
        assert abs(out[p] - oracle.perm_f64(R[p])) <= 1e-13 * oracle.perm_dp_f64(np.abs(R[p]))
        _check_minors(G[p], R[p], oracle)
    R[77, 1, 1] = np.inf
    with pytest.raises(pg.PermError):
        pg.perm_grad_batched(_dev(R))


def test_autograd_function(pg):
    import torch

    A = torch.from_numpy(syn.signed_real(7, 12100)).cuda().requires_grad_(True)
    y = pg.permanent(A)
    y.backward()
    _, G = pg.perm_grad(A.detach())
    assert torch.equal(A.grad, G)
    B = torch.from_numpy(syn.signed_real(5, 12200)).cuda().requires_grad_(True)
    assert torch.autograd.gradcheck(pg.permanent, (B,), eps=1e-3, atol=1e-9, rtol=1e-9)
    C = torch.from_numpy(syn.haar_unitary(4, 12300)).cuda().requires_grad_(True)
    assert torch.autograd.gradcheck(pg.permanent, (C,), eps=1e-4, atol=1e-9, rtol=1e-7)
    Bt = torch.from_numpy(np.stack(syn.boson_submatrices(6, 12400, 5, 5, 16))).cuda().requires_grad_(True)
    assert torch.autograd.gradcheck(lambda X: pg.permanent(X).abs().pow(2).sum(), (Bt,), eps=1e-4, atol=1e-9,
                                    rtol=1e-7)


def test_config_real_n28(pg, oracle):
    """Dense real n=28 uniform [-1, 1): sampled minors from the oracle and the
    identity sum_j a_ij G_ij = perm for every row."""
    A = syn.grad_real_28()
    n = 28
    p, G = pg.perm_grad(_dev(A))
    G = G.cpu().numpy()
    for i in range(n):
        assert abs(float(np.dot(A[i], G[i])) - p) <= 1e-9 * float(np.sum(np.abs(A[i] * G[i])))
    for k, l in ((0, 27), (13, 4), (27, 27)):
        want = oracle.perm_f64(_minor(A, k, l))
        assert abs(G[k, l] - want) <= 1e-10 * pg.perm(_dev(np.abs(_minor(A, k, l))))
        assert abs(G[k, l] - want) <= 1e-9 * abs(want)


def test_config_complex_batch_1024_k16(pg, oracle):
    """1024 complex 16 x 16 Haar submatrices in one batched launch: sampled
    matrices' full gradients against the oracle's minors."""
    Ms = syn.grad_boson_16(1024)
    out, G = pg.perm_grad_batched(_dev(Ms))
    out, G = out.cpu().numpy(), G.cpu().numpy()
    for p in (0, 511, 1023):
        assert abs(out[p] - oracle.perm_c128(Ms[p])) <= 1e-12
        _check_minors(G[p], Ms[p], oracle, cplx=True)


def test_mixed_orders(pg, oracle):
    """Matrices of mixed orders (0 .. 20, real and complex) in one call: each
    gradient equals the single-matrix sweep, the permanents the oracle."""
    g = syn.rng(12500)
    ks = [3, 7, 0, 12, 7, 1, 20, 3, 16, 9, 12]
    mats = [2.0 * g.random((k, k)) - 1.0 for k in ks]
    perms, grads = pg.perm_grad_mixed(mats)
    for M, p, G in zip(mats, perms, grads):
        k = M.shape[0]
        if k == 0:
            assert p == 1.0
            continue
        scale = oracle.perm_dp_f64(np.abs(M))
        assert abs(p - oracle.perm_dp_f64(M)) <= 1e-12 * scale
        _, Gs = pg.perm_grad(_dev(M))
        assert np.max(np.abs(G - Gs.cpu().numpy())) <= 1e-12 * scale
    cm = syn.boson_submatrices(30, 12600, 5, 17, 64)
    perms, grads = pg.perm_grad_mixed(cm)
    for M, p, G in zip(cm, perms, grads):
        assert abs(p - oracle.perm_c128(M)) <= 1e-12
        _, Gs = pg.perm_grad(_dev(M))
        assert np.max(np.abs(G - Gs.cpu().numpy())) <= 1e-13


def test_gradient_plan_runs_without_allocating(pg, oracle):
    """perm_grad_plan_*: the buffers are allocated at creation; runs on other
    inputs of the same shapes reuse them and give the results of
    perm_grad_batched_mixed bit for bit (the same kernels and launch shapes)."""
    import torch

    g = syn.rng(12700)
    ks = [5, 11, 0, 16, 11, 2, 20]
    offs, tot = [], 0
    for k in ks:
        offs.append(tot)
        tot += k * k
    plan = pg.GradPlan(ks)
    for rep in range(3):
        mats = [2.0 * g.random((k, k)) - 1.0 for k in ks]
        A = torch.zeros(max(tot, 1), dtype=torch.float64, device="cuda")
        for M, o in zip(mats, offs):
            A[o:o + M.size] = torch.from_numpy(M.reshape(-1))
        Gp = torch.zeros_like(A)
        out = torch.zeros(len(ks), dtype=torch.float64, device="cuda")
        st = torch.full((1,), -1, dtype=torch.int32, device="cuda")
        before = torch.cuda.memory_allocated()
        plan.run_async(A, out, Gp, st)
        torch.cuda.synchronize()
        assert torch.cuda.memory_allocated() == before
        assert int(st.item()) == 0
        perms, grads = pg.perm_grad_mixed(mats)
        assert np.array_equal(out.cpu().numpy(), perms)
        Gh = Gp.cpu().numpy()
        for M, o, G in zip(mats, offs, grads):
            k = M.shape[0]
            assert np.array_equal(Gh[o:o + k * k].reshape(k, k), G)
            if k:
                assert abs(out.cpu().numpy()[ks.index(k)] - oracle.perm_dp_f64(mats[ks.index(k)])) <= \
                    1e-12 * oracle.perm_dp_f64(np.abs(mats[ks.index(k)]))
    plan.close()

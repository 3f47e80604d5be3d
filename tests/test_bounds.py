"""The error bounds of tests/_bounds.py, checked on the CPU.

The GPU parity tests accept a kernel result when it lies within the bound
that tests/_bounds.py derives from the kernel's arithmetic.  Here that
derivation is checked without a GPU, on inputs small enough for exact
rational arithmetic:

* the exact range sum sum_g (-1)^g prod_i x_i(g) and the magnitude sums S and
  W are computed with Fractions (every binary64 entry is a dyadic rational);
* the double-double oracles (ryser_dd_stats_range, ryser_cdd_range) must lie
  within dd_oracle_bound of the exact sum and reproduce S and W;
* bit-level models of the kernels' integer arithmetic must lie within the
  bounds the GPU parity tests use.  Each model restates in Python integers
  the operations its kernel documents and shares no code with the CUDA
  sources; the double-double accumulation of the terms (below 2^-64 S per
  chunk) is left out, the bounds' 2^-59 S allowance covers it:
  - dense real (real_sweep_bound): the staging of every row, the odd last
    column, two chains of 62-bit products over even and odd rows with their
    renormalising shifts and one merge, the exponent bookkeeping, and the
    integer assembly of each term's binary64 head and tail, including a chain
    that a factor |Y_i| = 1 has emptied;
  - sparse in Alg. 2's column order (real_sweep_bound): rows without the odd
    unit, exact zeros skipped, the chain of all rows merged with two empty
    chains;
  - complex (complex_sweep_bound, part by part): signed 62-bit limb products
    with the larger part renormalised to 2^60, in the one-lane layout
    (n < 16: two chains and a merge) and the two-lane layout (n >= 16: one
    chain per lane over half the rows, then a merge);
  - the real gradient (2^-42 S_k): normalised leaves, the exclusive butterfly
    over eight lanes, one rounding per term, binary64 prefix and column sums
    inside each chunk.
"""
import math
from fractions import Fraction

import numpy as np
import pytest

import synthetic as syn
from _bounds import complex_sweep_bound, dd_oracle_bound, real_rows_on_grid, real_sweep_bound

M32 = (1 << 32) - 1


def _exact(A):
    """Exact sum_g (-1)^g prod_i x_i(g), S and W over all 2^(n-1) Gray steps
    (x_i = 1/2 sum_j delta_j a_ij, Eq. nwx; Alg. 1's order)."""
    n = A.shape[0]
    F = [[Fraction(float(v)) for v in row] for row in A]
    R = [sum(abs(v) for v in row) for row in F]
    # g = 0: every column but n-1 out
    x = [(F[i][n - 1] - sum(F[i][:n - 1])) / 2 for i in range(n)]
    total, S, W = Fraction(0), Fraction(0), Fraction(0)
    for g in range(1 << (n - 1)):
        if g:
            j = (g & -g).bit_length() - 1
            enter = not ((g >> (j + 1)) & 1)
            for i in range(n):
                x[i] += F[i][j] if enter else -F[i][j]
        p = Fraction(1)
        for v in x:
            p *= v
        total += -p if g & 1 else p
        S += abs(p)
        for i in range(n):
            q = R[i]
            for k in range(n):
                if k != i:
                    q *= abs(x[k])
            W += q
    return total, S, W


def _prod_mul(m0, m1, a0, a1):
    """The 62-bit product step: v = M A / 2^64 (the m0 a0 partial product
    dropped, 2^31 added to the middle ones), then M <- v << (30 - pos) with pos
    the top set bit of v's high word (32-bit wrap-around shift semantics)."""
    t = m1 * a0 + (1 << 31)
    u = m0 * a1 + t
    assert u < (1 << 64)
    v = m1 * a1 + (u >> 32)
    vh, vl = v >> 32, v & M32
    pos = vh.bit_length() - 1 if vh else -1
    s = (30 - pos) & M32
    w = s & 31
    new_m1 = ((((vh << 32) | vl) << w) >> 32) & M32
    new_m0 = (vl << s) & M32 if s < 32 else 0
    return new_m0, new_m1, pos


def _f64_from_bits(b):
    """The binary64 value of a 64-bit pattern (finite patterns only)."""
    sign = -1 if b >> 63 else 1
    e = (b >> 52) & 0x7FF
    m = b & ((1 << 52) - 1)
    assert e != 0x7FF
    if e == 0:
        return sign * Fraction(m) / (1 << 1074)
    return sign * (Fraction((1 << 52) | m) * Fraction(2) ** (e - 1075))


def _term_head_tail(M, f, signbit):
    """The head and tail a term M 2^(f + 1 - 1023 - 62) is split into, from
    the integer assembly: the head adds 512 to M, keeps its top 53 bits and
    places them on the exponent field f; the tail is M minus the head's bits
    (at most 512 units), placed by its own top bit.  f is clamped at 0."""
    f = max(f, 0)
    R = (M + 512) & ((1 << 64) - 1)
    head = _f64_from_bits(((signbit << 63) + (f << 52) + (R >> 10)) & ((1 << 64) - 1))
    r = (M & M32) - (R & M32 & ~0x3FF)
    r = r - (1 << 32) if r >= (1 << 31) else (r + (1 << 32) if r < -(1 << 31) else r)
    mag = abs(r)
    lz = 32 - (mag | 1).bit_length()
    be = f - 61 + 31 - lz
    if mag == 0 or be <= 0:
        return head, Fraction(0)
    tail = Fraction(mag) * Fraction(2) ** (be - 1023 - (31 - lz))
    return head, (-tail if (r < 0) != bool(signbit) else tail)


def _model_sweep(A):
    """The dense real sweep's range sum over all steps, from its integer
    arithmetic: rows in 64-bit fixed point (s_i = 61 - k_i, columns 0..n-2
    rounded to nearest even multiples, column n-1 to odd ones), |Y_i| exact
    (Y_i is odd), two product chains (even / odd rows) merged, and the term
    value from the mantissa and the renormalising shifts."""
    n = A.shape[0]
    Q, scale = [], []
    for i in range(n):
        absum = 0.0
        for j in range(n):
            absum += abs(float(A[i, j]))  # binary64 in column order, as staged
        k = math.frexp(absum)[1] if absum > 0 else 0
        s = 61 - k
        row = [2 * round(Fraction(float(A[i, j])) * Fraction(2) ** (s - 1)) for j in range(n - 1)]
        row.append(2 * math.floor(Fraction(float(A[i, n - 1])) * Fraction(2) ** (s - 1)) + 1)
        Q.append(row)
        scale.append(s + 1)
    Y = [Q[i][n - 1] - sum(Q[i][:n - 1]) for i in range(n)]
    total = Fraction(0)
    K1 = 64 * n + 1025 - (sum(scale) - n)  # sum of the s_i
    for g in range(1 << (n - 1)):
        if g:
            j = (g & -g).bit_length() - 1
            sgn = -1 if (g >> (j + 1)) & 1 else 1
            for i in range(n):
                Y[i] += 2 * sgn * Q[i][j]
        chains = [[0, 1 << 30], [0, 1 << 30]]  # 2^62 each
        epos, neg = 0, 0
        for i, y in enumerate(Y):
            assert y & 1 and abs(y) < (1 << 62)
            a = abs(y)
            neg ^= y < 0
            c = chains[i & 1]
            c[0], c[1], pos = _prod_mul(c[0], c[1], a & M32, a >> 32)
            epos += pos
        m0, m1, pos = _prod_mul(chains[0][0], chains[0][1], chains[1][0], chains[1][1])
        epos += pos
        f = K1 - (30 * (n + 1) - epos) - (n + 1)
        head, tail = _term_head_tail((m1 << 32) | m0, f, int(neg ^ (g & 1)))
        total += head + tail
    return total


def _cases():
    g = syn.rng(9100)
    out = [("signed uniform n=9", syn.signed_real(9, 9101)),
           ("uniform [0, 1) n=10", syn.uniform_real(10, 9102)),
           ("integers in [-3, 3] n=10 (on the grid)", g.integers(-3, 4, size=(10, 10)).astype(np.float64)),
           ("random signs n=10 (many x_i = 0)", np.where(g.random((10, 10)) < 0.5, -1.0, 1.0))]
    B = syn.signed_real(8, 9103)
    B[2] *= 2.0 ** 300
    B[5] *= 2.0 ** -280
    out.append(("rows scaled 2^300 / 2^-280 n=8", B))
    # a row whose x is exactly 0 on half the steps: |Y| = 1 there (the odd
    # unit), which empties its product chain: the first factor, a middle one,
    # and the last factor of either chain (rows alternate between the chains)
    for r in (0, 4, 7, 8):
        C = syn.signed_real(9, 9104 + r)
        C[r] = 0.0
        C[r, 0], C[r, 1] = 1.0, -1.0
        out.append((f"x_{r} = 0 on half the steps n=9", C))
    return out


@pytest.mark.parametrize("name,A", _cases(), ids=lambda v: v if isinstance(v, str) else "")
def test_oracle_dd_and_model_sweep_within_their_bounds(oracle, name, A):
    n = A.shape[0]
    exact, S, W = _exact(A)
    # the double-double oracle: its range sum within (n + 2) 2^-100 S, and its S, W
    r = oracle.ryser_dd_stats_range(A, 0, 1 << (n - 1))
    err_dd = abs(Fraction(r["hi"]) + Fraction(r["lo"]) - exact)
    assert err_dd <= Fraction(dd_oracle_bound(float(S), n)), (name, float(err_dd), float(S))
    assert r["S"] == pytest.approx(float(S), rel=1e-13)
    assert r["W"] == pytest.approx(float(W), rel=1e-13)
    # the dense sweep's arithmetic within the bound the GPU parity tests use
    model = _model_sweep(A)
    bound = real_sweep_bound(float(S), float(W), n, real_rows_on_grid(A))
    err = abs(model - exact)
    assert err <= Fraction(bound), (name, float(err), bound)


def test_model_is_exact_on_small_integers():
    # a check of the model itself: rows of small integers are staged exactly
    # apart from the odd unit of the last column (2^-(s_i+1) in x_i), which
    # changes a 62-bit product of these |Y_i| ~ 2^60 by a quarter of its last
    # unit and is rounded away, and every other product is exact, so the model
    # reproduces the exact sum bit for bit
    A = np.array([[1, 2, 0], [3, -1, 1], [0, 1, 2]], dtype=np.float64)
    exact, _, _ = _exact(A)
    assert _model_sweep(A) == exact


def test_grid_detection():
    # entries of columns 0..n-2 that are multiples of the row's fixed-point
    # unit are on the grid; an entry far below its row sum is not; column n-1
    # is rounded to an odd multiple in any case and is not examined
    assert real_rows_on_grid(np.array([[1.0, -2.0], [0.5, 0.25]]))
    assert not real_rows_on_grid(np.array([[2.0 ** -70, 1.0], [1.0, 1.0]]))
    assert real_rows_on_grid(np.array([[1.0, 2.0 ** -70], [1.0, 1.0]]))


# ---------------------------------------------------------------- complex


def _s32(v):
    v &= M32
    return v - (1 << 32) if v >> 31 else v


def _split62(y):
    """(bits 31..62 of y as a signed 32-bit limb, bits 0..30)."""
    u = y & ((1 << 64) - 1)
    ul, uh = u & M32, u >> 32
    return _s32((uh << 1) | (ul >> 31)), ul & 0x7FFFFFFF


def _cprod_mul(p, yr, yi):
    """The complex limb product step: the middle partial products (scale 2^31,
    floored by an arithmetic shift), the high ones (scale 2^62), then both
    parts shifted so that the larger one's top bit sits at 2^60 (the top bit
    found in the ones'-complement magnitudes of the high words).  p = [r1, r0,
    i1, i0]; returns the shift s (the product was scaled by 2^(s - 62))."""
    r1, r0, i1, i0 = p
    yr1, yr0 = _split62(yr)
    yi1, yi0 = _split62(yi)
    ni1, ni0 = _s32(-i1), _s32(-i0)
    tr = (r1 * yr0 + r0 * yr1 + ni1 * yi0 + ni0 * yi1) >> 31
    ti = (r1 * yi0 + r0 * yi1 + i1 * yr0 + i0 * yr1) >> 31
    vr = r1 * yr1 + ni1 * yi1 + tr
    vi = r1 * yi1 + i1 * yr1 + ti
    w = 0
    for v in (vr, vi):
        h = _s32(v >> 32)
        w |= (h ^ (h >> 31)) & M32
    pos = w.bit_length() - 1 if w else -1
    sh = 28 - pos
    assert 0 <= sh < 64
    out = []
    for v in (vr, vi):
        u = (v << sh) & ((1 << 64) - 1)
        out.extend(_split62(u - (1 << 64) if u >> 63 else u))
    p[:] = out
    return sh


def _model_cplx_sweep(A):
    """The one-lane complex sweep's range sum (re, im) from its integer
    arithmetic: rows s_i = 60 - k_i with k_i from sum_j |re| + |im|, every
    entry rounded to nearest, two chains over even / odd rows starting at 2^60,
    their merge, and the term z 2^(ebase - sum of the shifts) (its exact
    head + tail)."""
    n = A.shape[0]
    Q, ssum = [], 0
    for i in range(n):
        absum = 0.0
        for j in range(n):
            absum += abs(float(A[i, j].real))
            absum += abs(float(A[i, j].imag))
        k = math.frexp(absum)[1] if absum > 0 else 0
        s = 60 - k
        ssum += s
        Q.append([(round(Fraction(float(A[i, j].real)) * Fraction(2) ** s),
                   round(Fraction(float(A[i, j].imag)) * Fraction(2) ** s)) for j in range(n)])
    Yr = [Q[i][n - 1][0] - sum(q[0] for q in Q[i][:n - 1]) for i in range(n)]
    Yi = [Q[i][n - 1][1] - sum(q[1] for q in Q[i][:n - 1]) for i in range(n)]
    ebase = 62 * (n + 1) - 120 - ssum - n
    tot_r, tot_i = Fraction(0), Fraction(0)
    for g in range(1 << (n - 1)):
        if g:
            j = (g & -g).bit_length() - 1
            sgn = -1 if (g >> (j + 1)) & 1 else 1
            for i in range(n):
                Yr[i] += 2 * sgn * Q[i][j][0]
                Yi[i] += 2 * sgn * Q[i][j][1]
        chains = [[1 << 29, 0, 0, 0], [1 << 29, 0, 0, 0]]  # 2^60 each
        shifts = 0
        for i in range(n):
            assert abs(Yr[i]) < (1 << 61) and abs(Yi[i]) < (1 << 61)
            shifts += _cprod_mul(chains[i & 1], Yr[i], Yi[i])
        b = chains[1]
        shifts += _cprod_mul(chains[0], b[0] * (1 << 31) + b[1], b[2] * (1 << 31) + b[3])
        a = chains[0]
        scale = Fraction(2) ** (ebase - shifts) * (-1 if g & 1 else 1)
        tot_r += (a[0] * (1 << 31) + a[1]) * scale
        tot_i += (a[2] * (1 << 31) + a[3]) * scale
    return tot_r, tot_i


def _exact_cplx(A):
    """Exact complex range sum (re, im) as Fractions, and S, W in binary64."""
    n = A.shape[0]
    F = [[(Fraction(float(v.real)), Fraction(float(v.imag))) for v in row] for row in A]
    xr = [(F[i][n - 1][0] - sum(v[0] for v in F[i][:n - 1])) / 2 for i in range(n)]
    xi = [(F[i][n - 1][1] - sum(v[1] for v in F[i][:n - 1])) / 2 for i in range(n)]
    R = [float(np.sum(np.abs(A[i]))) for i in range(n)]
    tr, ti, S, W = Fraction(0), Fraction(0), 0.0, 0.0
    for g in range(1 << (n - 1)):
        if g:
            j = (g & -g).bit_length() - 1
            enter = not ((g >> (j + 1)) & 1)
            for i in range(n):
                xr[i] += F[i][j][0] if enter else -F[i][j][0]
                xi[i] += F[i][j][1] if enter else -F[i][j][1]
        pr, pi = Fraction(1), Fraction(0)
        for a, b in zip(xr, xi):
            pr, pi = pr * a - pi * b, pr * b + pi * a
        if g & 1:
            pr, pi = -pr, -pi
        tr += pr
        ti += pi
        mods = [math.hypot(float(a), float(b)) for a, b in zip(xr, xi)]
        S += math.prod(mods)
        for i in range(n):
            W += R[i] * math.prod(m for k, m in enumerate(mods) if k != i)
    return tr, ti, S, W


def _cplx_cases():
    g = syn.rng(9200)
    out = [("Haar n=8", syn.haar_unitary(8, 9201)),
           ("Gaussian n=9", (g.standard_normal((9, 9)) + 1j * g.standard_normal((9, 9))) / math.sqrt(2.0)),
           ("Gaussian integers n=8", (g.integers(-2, 3, size=(8, 8)) + 1j * g.integers(-2, 3, size=(8, 8))))]
    C = syn.haar_unitary(8, 9202)
    C[3] = 0.0
    C[3, 0], C[3, 1] = 0.5 + 0.5j, -0.5 - 0.5j  # x_3 = 0 on half the steps
    out.append(("x_3 = 0 on half the steps n=8", C))
    return out


@pytest.mark.parametrize("name,A", _cplx_cases(), ids=lambda v: v if isinstance(v, str) else "")
def test_complex_oracle_and_model_sweep_within_their_bounds(oracle, name, A):
    A = np.ascontiguousarray(A, dtype=np.complex128)
    n = A.shape[0]
    er, ei, S, W = _exact_cplx(A)
    r = oracle.ryser_cdd_range(A, 0, 1 << (n - 1))
    tol_dd = Fraction(dd_oracle_bound(S, n))
    assert abs(Fraction(r["re_hi"]) + Fraction(r["re_lo"]) - er) <= tol_dd, name
    assert abs(Fraction(r["im_hi"]) + Fraction(r["im_lo"]) - ei) <= tol_dd, name
    assert r["S"] == pytest.approx(S, rel=1e-12)
    assert r["W"] == pytest.approx(W, rel=1e-12)
    mr, mi = _model_cplx_sweep(A)
    bound = Fraction(complex_sweep_bound(S, W, n))
    assert abs(mr - er) <= bound and abs(mi - ei) <= bound, (name, float(abs(mr - er)), float(abs(mi - ei)),
                                                             float(bound))


# ----------------------------------------------------------------- sparse


def _model_sparse_paper_order(A):
    """The sparse sweep's range sum over all steps in Alg. 2's column order
    (no column moved to the low Gray bits): rows s_i = 61 - k_i with every
    stored entry rounded to nearest (no odd unit, so Y_i is 0 exactly when its
    fixed-point sum is), a step whose rows include a zero adds nothing, else
    the product of all rows in row order forms one chain that is merged into
    two empty chains (2^62 each), and the term is assembled as in the dense
    sweep."""
    n = A.shape[0]
    Q, ssum = [], 0
    for i in range(n):
        absum = 0.0
        for j in range(n):
            if A[i, j] != 0.0:
                absum += abs(float(A[i, j]))
        k = math.frexp(absum)[1] if absum > 0 else 0
        s = 61 - k
        ssum += s
        Q.append([round(Fraction(float(A[i, j])) * Fraction(2) ** s) for j in range(n)])
    Y = [Q[i][n - 1] - sum(Q[i][:n - 1]) for i in range(n)]
    F0 = 33 * n + 966 - ssum
    total = Fraction(0)
    for g in range(1 << (n - 1)):
        if g:
            j = (g & -g).bit_length() - 1
            sgn = -1 if (g >> (j + 1)) & 1 else 1
            for i in range(n):
                Y[i] += 2 * sgn * Q[i][j]
        if any(y == 0 for y in Y):
            continue
        pq = [0, 1 << 30]
        epos, neg = 0, 0
        for y in Y:
            a = abs(y)
            neg ^= y < 0
            pq[0], pq[1], pos = _prod_mul(pq[0], pq[1], a & M32, a >> 32)
            epos += pos
        m0, m1, pos = _prod_mul(0, 1 << 30, 0, 1 << 30)  # the two empty chains
        epos += pos
        m0, m1, pos = _prod_mul(m0, m1, pq[0], pq[1])
        epos += pos
        head, tail = _term_head_tail((m1 << 32) | m0, F0 + epos, int(neg ^ (g & 1)))
        total += head + tail
    return total


def _sparse_cases():
    return [("density 0.4 n=10", syn.sparse_real(10, 9301, 0.4)),
            ("density 0.3 n=9", syn.sparse_real(9, 9302, 0.3)),
            ("0/1 density 0.5 n=10 (exact zeros on many steps)",
             (syn.rng(9303).random((10, 10)) < 0.5).astype(np.float64) + np.eye(10))]


@pytest.mark.parametrize("name,A", _sparse_cases(), ids=lambda v: v if isinstance(v, str) else "")
def test_sparse_model_sweep_within_the_real_bound(name, A):
    n = A.shape[0]
    exact, S, W = _exact(A)
    model = _model_sparse_paper_order(A)
    bound = real_sweep_bound(float(S), float(W), n, real_rows_on_grid(A))
    err = abs(model - exact)
    assert err <= Fraction(bound), (name, float(err), bound)


# --------------------------------------------------------------- gradient

TOL_GRAD = 2.0 ** -42  # the gradient sweep's derived bound, relative to S_k


def _leaf(y):
    """|Y| normalised to a mantissa in [2^62, 2^63): (m0, m1, e), |Y| = M 2^e."""
    a = abs(y)
    lz = 64 - a.bit_length()
    m = a << (lz - 1)
    return [m & M32, m >> 32, 1 - lz]


def _gmul(a, b):
    m0, m1, pos = _prod_mul(a[0], a[1], b[0], b[1])
    return [m0, m1, a[2] + b[2] + 34 + pos]


def _to_double(v, eoff, neg):
    """The term's single rounding: the top 53 of the mantissa's 63 bits
    (+512 then a 10-bit shift, ties away from zero) placed on the exponent
    field f = e + eoff + 62 + 1022, flushed to zero below the normal range."""
    f = v[2] + eoff + 62 + 1022
    if f < 1:
        return 0.0
    M = (v[1] << 32) | v[0]
    word = (min(f, 2045) << 52) + ((M + 512) >> 10)
    x = float(_f64_from_bits(word))
    return -x if neg else x


def _model_grad(A, cq):
    """The real gradient sweep (8 lanes per chunk, two rows per lane, n <= 16)
    from its arithmetic: fixed-point rows as in the forward sweep, normalised
    leaves, the local exclusive products and the three-level exclusive
    butterfly over the lanes, one rounding of every term to binary64, the
    running prefix P_k and the column sums U_kj (j < cq) in binary64 inside
    each chunk, the chunk-end additions of P as the kernel does them.  The
    chunks' contributions are then added exactly.  Returns G (Fractions)."""
    n = A.shape[0]
    NR, L = 16, 8
    Q, s_sc = [], []
    for i in range(n):
        absum = 0.0
        for j in range(n):
            absum += abs(float(A[i, j]))
        k = math.frexp(absum)[1] if absum > 0 else 0
        s = 61 - k
        row = [2 * round(Fraction(float(A[i, j])) * Fraction(2) ** (s - 1)) for j in range(n - 1)]
        row.append(2 * math.floor(Fraction(float(A[i, n - 1])) * Fraction(2) ** (s - 1)) + 1)
        Q.append(row)
        s_sc.append(s)
    s_all = sum(s + 1 for s in s_sc)
    eo = [-(s_all - (s_sc[i] + 1)) if i < n else None for i in range(NR)]
    U = [[Fraction(0)] * n for _ in range(n)]  # U[k][l]
    T = [Fraction(0)] * n
    for c0 in range(0, 1 << (n - 1), 1 << cq):
        G0 = c0 ^ (c0 >> 1)
        Y = [sum((Q[i][j] if (j == n - 1 or (G0 >> j) & 1) else -Q[i][j]) for j in range(n)) if i < n else 1
             for i in range(NR)]
        P = [0.0] * n
        Uc = [[0.0] * cq for _ in range(n)]
        for t in range(1 << cq):
            g = c0 + t
            if t:
                j = (t & -t).bit_length() - 1
                leave = (g >> (j + 1)) & 1
                for i in range(n):
                    Y[i] += -2 * Q[i][j] if leave else 2 * Q[i][j]
                for k in range(n):
                    Uc[k][j] = Uc[k][j] + (P[k] if leave else -P[k])
            lf = [_leaf(y) for y in Y]
            negs = [1 if y < 0 else 0 for y in Y]
            grp = [_gmul(lf[2 * l], lf[2 * l + 1]) for l in range(L)]
            o = [grp[l ^ 1] for l in range(L)]
            grp = [_gmul(grp[l], o[l]) for l in range(L)]
            x2 = [grp[l ^ 2] for l in range(L)]
            o = [_gmul(o[l], x2[l]) for l in range(L)]
            grp = [_gmul(grp[l], x2[l]) for l in range(L)]
            x4 = [grp[l ^ 4] for l in range(L)]
            o = [_gmul(o[l], x4[l]) for l in range(L)]
            allneg = sum(negs) & 1
            for k in range(n):
                l, r = divmod(k, 2)
                v = _gmul(o[l], lf[2 * l + 1 - r])
                neg = allneg ^ negs[k] ^ (g & 1)
                P[k] = P[k] + _to_double(v, eo[k], neg)
        G1 = (c0 + (1 << cq) - 1) ^ ((c0 + (1 << cq) - 1) >> 1)
        for k in range(n):
            T[k] += Fraction(P[k])
            for j in range(n - 1):
                if j < cq:
                    U[k][j] += Fraction(Uc[k][j] + (P[k] if (G1 >> j) & 1 else 0.0))
                elif (G0 >> j) & 1:
                    U[k][j] += Fraction(P[k])
    sg = -1 if (n - 1) & 1 else 1
    return [[sg * (2 * U[k][l] - T[k]) if l < n - 1 else sg * T[k] for l in range(n)] for k in range(n)]


def _exact_grad(A):
    """Exact G_kl = (-1)^(n-1) sum_g (-1)^g delta_l(g) prod_{i != k} x_i(g) and
    S_k = sum_g prod_{i != k} |x_i(g)|."""
    n = A.shape[0]
    F = [[Fraction(float(v)) for v in row] for row in A]
    x = [(F[i][n - 1] - sum(F[i][:n - 1])) / 2 for i in range(n)]
    G = [[Fraction(0)] * n for _ in range(n)]
    S = [Fraction(0)] * n
    sg = -1 if (n - 1) & 1 else 1
    for g in range(1 << (n - 1)):
        if g:
            j = (g & -g).bit_length() - 1
            enter = not ((g >> (j + 1)) & 1)
            for i in range(n):
                x[i] += F[i][j] if enter else -F[i][j]
        gray = g ^ (g >> 1)
        for k in range(n):
            v = Fraction(1)
            for i in range(n):
                if i != k:
                    v *= x[i]
            S[k] += abs(v)
            w = -v if g & 1 else v
            for l in range(n):
                d = 1 if (l == n - 1 or (gray >> l) & 1) else -1
                G[k][l] += sg * d * w
    return G, S


@pytest.mark.parametrize("n,cq,seed", [(9, 4, 9401), (10, 5, 9402)])
def test_gradient_model_within_its_bound(oracle, n, cq, seed):
    A = syn.signed_real(n, seed)
    G, S = _exact_grad(A)
    # the exact sums are the minor permanents (a check of _exact_grad itself)
    for k, l in ((0, 0), (n - 1, 2)):
        M = np.delete(np.delete(A, k, axis=0), l, axis=1)
        assert float(G[k][l]) == pytest.approx(oracle.perm_dp_f64(M), rel=1e-12, abs=1e-12)
    Gm = _model_grad(A, cq)
    worst = 0.0
    for k in range(n):
        for l in range(n):
            r = float(abs(Gm[k][l] - G[k][l]) / S[k])
            worst = max(worst, r)
    assert worst <= TOL_GRAD, worst


def _model_cplx2_sweep(A):
    """The two-lane complex sweep (used from n = 16): lane 0 multiplies rows
    0..R-1 and lane 1 rows R..2R-1 into one chain each (R = ceil(n/2); an odd
    n pads lane 1 with the constant 2^60, taken back out of the exponent), the
    two halves are merged by one more limb product, and the term z 2^E is
    added exactly.  The arithmetic does not depend on n, so small n check the
    bound of the kernel's layout."""
    n = A.shape[0]
    R = (n + 1) // 2
    Q, ssum = [], 0
    for i in range(n):
        absum = 0.0
        for j in range(n):
            absum += abs(float(A[i, j].real))
            absum += abs(float(A[i, j].imag))
        k = math.frexp(absum)[1] if absum > 0 else 0
        s = 60 - k
        ssum += s
        Q.append([(round(Fraction(float(A[i, j].real)) * Fraction(2) ** s),
                   round(Fraction(float(A[i, j].imag)) * Fraction(2) ** s)) for j in range(n)])
    Yr = [Q[i][n - 1][0] - sum(q[0] for q in Q[i][:n - 1]) for i in range(n)] + [1 << 60] * (2 * R - n)
    Yi = [Q[i][n - 1][1] - sum(q[1] for q in Q[i][:n - 1]) for i in range(n)] + [0] * (2 * R - n)
    eoff = -(ssum + n) - (60 if n & 1 else 0)
    tot_r, tot_i = Fraction(0), Fraction(0)
    for g in range(1 << (n - 1)):
        if g:
            j = (g & -g).bit_length() - 1
            sgn = -1 if (g >> (j + 1)) & 1 else 1
            for i in range(n):
                Yr[i] += 2 * sgn * Q[i][j][0]
                Yi[i] += 2 * sgn * Q[i][j][1]
        halves = []
        for h in range(2):
            p = [1 << 29, 0, 0, 0]
            ss = 0
            for r in range(R):
                ss += _cprod_mul(p, Yr[h * R + r], Yi[h * R + r])
            halves.append((p, -60 + 62 * R - ss))
        (a, ea), (b, eb) = halves
        s = _cprod_mul(a, b[0] * (1 << 31) + b[1], b[2] * (1 << 31) + b[3])
        scale = Fraction(2) ** (ea + eb + 62 - s + eoff) * (-1 if g & 1 else 1)
        tot_r += (a[0] * (1 << 31) + a[1]) * scale
        tot_i += (a[2] * (1 << 31) + a[3]) * scale
    return tot_r, tot_i


@pytest.mark.parametrize("name,A", _cplx_cases()[:2] + [("Haar n=9 (a padded row)", syn.haar_unitary(9, 9203))],
                         ids=lambda v: v if isinstance(v, str) else "")
def test_two_lane_complex_model_within_the_bound(name, A):
    A = np.ascontiguousarray(A, dtype=np.complex128)
    n = A.shape[0]
    er, ei, S, W = _exact_cplx(A)
    mr, mi = _model_cplx2_sweep(A)
    bound = Fraction(complex_sweep_bound(S, W, n))
    assert abs(mr - er) <= bound and abs(mi - ei) <= bound, (name, float(abs(mr - er)), float(abs(mi - ei)),
                                                             float(bound))

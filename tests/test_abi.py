"""The C ABI without a GPU: the library loads, exports every function that
include/perm.h declares, rejects bad arguments on the host before touching
CUDA, and combines range partials on the host (checked against the oracle)."""
import ctypes
import math
import os
import re

import numpy as np
import pytest

import synthetic as syn

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_2502_16577_gb300 import build as b

    b.build()
    import paper_2502_16577_gb300 as pg

    return pg.load()


def _declared_functions():
    names = []
    for h in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if h.endswith(".h"):
            src = open(os.path.join(ROOT, "include", h)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names += re.findall(r"^\s*(?:int|const char\*|void)\s+(\w+)\s*\(", src, flags=re.M)
    return names


def test_exports_every_declared_symbol(lib):
    declared = _declared_functions()
    assert "perm" in declared and "perm_combine" in declared
    for name in declared:
        assert hasattr(lib, name), name
    from paper_2502_16577_gb300 import _lib

    assert set(_lib.SYMBOLS) <= set(declared)


def test_abi_version_and_status_strings(lib):
    import re

    header = open(os.path.join(ROOT, "include", "perm.h")).read()
    assert lib.perm_abi_version() == int(re.search(r"#define PERM_ABI_VERSION (\d+)", header).group(1))
    for code in range(7):
        assert b"unknown" not in lib.perm_status_string(code)
    assert b"unknown" in lib.perm_status_string(99)


def test_new_entry_points_check_arguments_on_the_host(lib):
    vp = ctypes.c_void_p
    dummy = vp(16)
    # gradient: type, order and count are checked before any CUDA call
    assert lib.perm_grad(dummy, 4, 2, dummy, dummy, vp(0), vp(0)) == 1       # 0/1 type
    assert lib.perm_grad(dummy, 33, 0, dummy, dummy, vp(0), vp(0)) == 2      # n > 32
    assert lib.perm_grad_batched(dummy, 4, -1, 0, dummy, dummy, vp(0), vp(0)) == 1
    # cancellation word: unregistering needs no device
    assert lib.perm_set_abort_word(None) == 0
    # sweep-unit planner of labelled batched plans: host only
    assert lib.perm_batched_units(0, None, 0, None, None, None, 0, None) == -2   # k < 1
    assert lib.perm_batched_units(33, None, 0, None, None, None, 0, None) == -2  # k > 32
    assert lib.perm_batched_units(5, None, 0, None, None, None, 0, None) == 1    # all distinct: one sweep
    pair = (ctypes.c_int32 * 12)(*(list(range(11)) + [4]))
    assert lib.perm_batched_units(12, pair, 0, None, None, None, 0, None) == 3
    assert lib.perm_batched_units(12, pair, 3, None, None, None, 0, None) == -5  # no room for descriptors


def test_host_argument_checks_need_no_gpu(lib):
    vp = ctypes.c_void_p
    dummy = vp(16)
    assert lib.perm(dummy, 64, 0, dummy, vp(0), vp(0)) == 2    # n > 63
    assert lib.perm(dummy, -1, 0, dummy, vp(0), vp(0)) == 2
    assert lib.perm(dummy, 5, 7, dummy, vp(0), vp(0)) == 1     # bad type
    assert lib.perm(dummy, 5, 4, dummy, vp(0), vp(0)) == 1     # first type past PERM_F64X
    assert lib.perm(dummy, 64, 3, dummy, vp(0), vp(0)) == 2    # PERM_F64X, n > 63
    assert lib.perm(vp(0), 5, 0, dummy, vp(0), vp(0)) == 1     # null A
    assert lib.perm(dummy, 5, 0, vp(0), vp(0), vp(0)) == 1     # null out
    assert lib.perm_range(dummy, 5, 0, 3, 2, dummy, vp(0), vp(0)) == 2   # begin > end
    assert lib.perm_range(dummy, 5, 0, 0, 17, dummy, vp(0), vp(0)) == 2  # end > 2^(n-1)


def test_combine_real_partials(oracle):
    import paper_2502_16577_gb300 as pg

    for n in (1, 2, 7, 12):
        A = syn.signed_real(n, 40 + n)
        N = 2 ** (n - 1)
        cuts = sorted({0, N, N // 3, N // 2})
        parts = [oracle.ryser_f64_range(A, a, b) for a, b in zip(cuts[:-1], cuts[1:])]
        got = pg.perm_combine(pg.PERM_F64, n, parts)
        assert got == pytest.approx(oracle.perm_dp_f64(A), abs=1e-13 * oracle.perm_dp_f64(np.abs(A)))


def test_combine_extended_partials_stay_double_double(oracle):
    """PERM_F64X partials (same layout as PERM_F64) combine into an unevaluated
    (hi, lo) scaled exactly by 2 (-1)^(n-1); the oracle's double-double range
    sums stand in for the kernel's partials."""
    from fractions import Fraction

    import paper_2502_16577_gb300 as pg

    for n in (1, 6, 11):
        A = syn.signed_real(n, 60 + n)
        N = 2 ** (n - 1)
        cuts = sorted({0, N, N // 3, N // 2})
        parts = [oracle.ryser_dd_range(A, a, b) for a, b in zip(cuts[:-1], cuts[1:])]
        hi, lo = pg.perm_combine(pg.PERM_F64X, n, parts)
        assert hi + lo == hi
        exact = oracle.perm_bruteforce(A) if n <= 8 else sum(map(Fraction, oracle.perm_dd(A)))
        assert abs(Fraction(hi) + Fraction(lo) - exact) <= Fraction(1, 10 ** 26) * Fraction(
            oracle.perm_dp_f64(np.abs(A)))
    assert pg.perm_combine(pg.PERM_F64X, 0, []) == (1.0, 0.0)


def test_combine_complex_partials(oracle):
    import paper_2502_16577_gb300 as pg

    U = syn.haar_unitary(9, 3)
    N = 2 ** 8
    parts = [oracle.ryser_c128_range(U, a, b) for a, b in ((0, 77), (77, 200), (200, N))]
    got = pg.perm_combine(pg.PERM_C128, 9, parts)
    assert abs(got - oracle.perm_dp_c128(U)) <= 1e-13


@pytest.mark.parametrize("n", [1, 2, 9, 18])
def test_combine_binary_partials_exact(oracle, n):
    import paper_2502_16577_gb300 as pg

    A = syn.bernoulli01(n, 50 + n, 0.6)
    N = 2 ** (n - 1)
    cuts = sorted({0, N, N // 4, (3 * N) // 4})
    parts = [oracle.ryser_bin_range(A, a, b) for a, b in zip(cuts[:-1], cuts[1:])]
    # the oracle's partials are residues mod 2^128; the ABI takes 192-bit words,
    # so lift them with the same residue (the sum's top 64 bits are then 0 or
    # negative-extended); exact when |sum| < 2^127, true here.
    lifted = [(p - (1 << 128)) % (1 << 192) if p >= (1 << 127) else p for p in parts]
    assert pg.perm_combine(pg.PERM_BIN, n, lifted) == oracle.perm_dp_bin(A)


def test_combine_binary_rejects_bad_sum():
    import paper_2502_16577_gb300 as pg

    with pytest.raises(pg.PermError):
        pg.perm_combine(pg.PERM_BIN, 5, [3])  # low bits not zero: not a full-range sum
    big = (1 << 130) << 4  # 2^(n-1) * 2^130 with n = 5
    with pytest.raises(pg.PermError):
        pg.perm_combine(pg.PERM_BIN, 5, [big])


def test_combine_trivial_sizes():
    import paper_2502_16577_gb300 as pg

    assert pg.perm_combine(pg.PERM_F64, 0, []) == 1.0
    assert pg.perm_combine(pg.PERM_BIN, 0, []) == 1
    assert pg.perm_combine(pg.PERM_C128, 0, []) == 1.0


def test_package_fails_loudly_without_library(monkeypatch, tmp_path):
    from paper_2502_16577_gb300 import _lib, build

    monkeypatch.setattr(_lib, "_lib", None)
    monkeypatch.setattr(build, "LIB", str(tmp_path / "missing.so"))
    with pytest.raises(ImportError):
        _lib.load()

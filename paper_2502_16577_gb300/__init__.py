"""GB300 permanents: Ryser / Nijenhuis-Wilf Gray-code sweep on sm_103a.

A thin Python binding of libperm.so (include/perm.h).  Every step of the
computation runs in the library's CUDA kernels; this module only moves
pointers, sizes and results.  PyTorch supplies device memory and streams.

    import torch, paper_2502_16577_gb300 as pg
    A = torch.rand(24, 24, dtype=torch.float64, device="cuda")
    pg.perm(A)                       # float
    pg.perm(U_complex128)            # complex
    pg.perm(B_uint8)                 # int, exact
    pg.perm_range(A, g0, g1)         # raw partial of steps [g0, g1)
    pg.perm_combine(A_type, n, [..]) # host reduction of partials
"""
from __future__ import annotations

import ctypes

import numpy as np

from . import _lib
from ._lib import (PERM_BIN, PERM_C128, PERM_EABORTED, PERM_EINVAL, PERM_ENOMEM, PERM_EOVERFLOW, PERM_ERANGE,
                   PERM_ETIMEOUT, PERM_F64, PERM_F64X, PERM_OK, PermError, check, load)

__all__ = ["perm", "perm_async", "perm_range", "perm_range_async", "perm_combine", "perm_sparse", "perm_sparse_async", "perm_sparse_range", "perm_sparse_range_async", "perm_host", "pipe_peaks", "BatchPlan", "AbortWord", "perm_grad", "perm_grad_async", "perm_grad_batched", "perm_grad_batched_async", "perm_grad_mixed", "GradPlan", "set_time_budget", "permanent", "batched_units", "equal_row_labels", "perm_type_of", "PermError",
           "PERM_F64", "PERM_C128", "PERM_BIN", "PERM_F64X", "perm_x", "PERM_EABORTED", "PERM_ETIMEOUT", "PERM_OK", "PERM_EINVAL", "PERM_ERANGE", "PERM_EOVERFLOW", "PERM_ENOMEM",
           "load"]


def _torch():
    import torch

    return torch


def perm_type_of(dtype) -> int:
    """The perm_type_t of a torch dtype (float64, complex128, uint8/bool 0/1)."""
    torch = _torch()
    if dtype in (torch.float64,):
        return PERM_F64
    if dtype in (torch.complex128,):
        return PERM_C128
    if dtype in (torch.uint8, torch.bool):
        return PERM_BIN
    raise TypeError(f"unsupported dtype {dtype}: use float64, complex128 or uint8 (0/1)")


def _as_device_matrix(A):
    torch = _torch()
    if not isinstance(A, torch.Tensor) or not A.is_cuda:
        raise TypeError("A must be a CUDA torch.Tensor (use perm_host for host arrays)")
    if A.dim() != 2 or A.shape[0] != A.shape[1]:
        raise ValueError("A must be a square matrix")
    if A.dtype == torch.bool:
        A = A.to(torch.uint8)
    return A.contiguous()


def _stream_handle(stream):
    torch = _torch()
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream), s


def _out_buffers(t: int, device, words: int):
    torch = _torch()
    if t == PERM_BIN:
        out = torch.zeros(words, dtype=torch.int64, device=device)
    else:
        out = torch.zeros(words, dtype=torch.float64, device=device)
    status = torch.full((1,), -1, dtype=torch.int32, device=device)
    return out, status


def _u(words) -> int:
    v = 0
    for i, w in enumerate(words):
        v |= (int(w) & 0xFFFFFFFFFFFFFFFF) << (64 * i)
    return v


def _type_for(A, extended: bool) -> int:
    t = perm_type_of(A.dtype)
    if extended:
        if t != PERM_F64:
            raise TypeError("extended-precision products are for float64 matrices")
        return PERM_F64X
    return t


def perm_async(A, out, status=None, stream=None, extended: bool = False) -> None:
    """Enqueue perm(A) on a stream without waiting; out / status are device tensors
    (float64[1], float64[2] for complex or extended, int64[2] for 0/1; int32[1])."""
    lib = load()
    A = _as_device_matrix(A)
    t = _type_for(A, extended)
    h, _ = _stream_handle(stream)
    rc = lib.perm(ctypes.c_void_p(A.data_ptr()), A.shape[0], t, ctypes.c_void_p(out.data_ptr()),
                  ctypes.c_void_p(status.data_ptr() if status is not None else 0), h)
    check(rc, "perm")


def perm(A, stream=None):
    """Permanent of a square CUDA tensor: float64 -> float, complex128 -> complex,
    uint8/bool 0/1 -> exact int.  Waits for the result."""
    A = _as_device_matrix(A)
    t = perm_type_of(A.dtype)
    out, status = _out_buffers(t, A.device, 1 if t == PERM_F64 else 2)
    perm_async(A, out, status, stream)
    _, s = _stream_handle(stream)
    s.synchronize()
    check(int(status.item()), "perm")
    o = out.cpu().numpy()
    if t == PERM_F64:
        return float(o[0])
    if t == PERM_C128:
        return complex(float(o[0]), float(o[1]))
    return _u(o)


def perm_x(A, stream=None) -> tuple:
    """Permanent of a float64 CUDA matrix with extended-precision products
    (PERM_F64X): the unevaluated double-double (hi, lo).  Waits for it."""
    A = _as_device_matrix(A)
    out, status = _out_buffers(PERM_F64X, A.device, 2)
    perm_async(A, out, status, stream, extended=True)
    _, s = _stream_handle(stream)
    s.synchronize()
    check(int(status.item()), "perm")
    o = out.cpu().numpy()
    return float(o[0]), float(o[1])


def perm_range_async(A, g_begin: int, g_end: int, out, status=None, stream=None, extended: bool = False) -> None:
    """Enqueue perm_range on a stream without waiting (out: float64[2] real,
    float64[4] complex, int64[3] for 0/1; status: int32[1])."""
    lib = load()
    A = _as_device_matrix(A)
    t = _type_for(A, extended)
    h, _ = _stream_handle(stream)
    rc = lib.perm_range(ctypes.c_void_p(A.data_ptr()), A.shape[0], t, int(g_begin), int(g_end),
                        ctypes.c_void_p(out.data_ptr()), ctypes.c_void_p(status.data_ptr() if status is not None else 0),
                        h)
    check(rc, "perm_range")


def perm_range(A, g_begin: int, g_end: int, stream=None, extended: bool = False):
    """Raw partial over steps [g_begin, g_end): (hi, lo) for float64 (also with
    extended products), (re_hi, re_lo, im_hi, im_lo) for complex128, an int
    mod 2^192 for 0/1."""
    lib = load()
    A = _as_device_matrix(A)
    t = _type_for(A, extended)
    words = {PERM_F64: 2, PERM_F64X: 2, PERM_C128: 4, PERM_BIN: 3}[t]
    out, status = _out_buffers(t, A.device, words)
    h, s = _stream_handle(stream)
    rc = lib.perm_range(ctypes.c_void_p(A.data_ptr()), A.shape[0], t, int(g_begin), int(g_end),
                        ctypes.c_void_p(out.data_ptr()), ctypes.c_void_p(status.data_ptr()), h)
    check(rc, "perm_range")
    s.synchronize()
    st = int(status.item())
    o = out.cpu().numpy()
    if t == PERM_BIN:
        if st not in (_lib.PERM_OK, _lib.PERM_EOVERFLOW):
            check(st, "perm_range")
        return _u(o)
    check(st, "perm_range")
    return tuple(float(v) for v in o)


def perm_combine(t: int, n: int, partials):
    """Host-side reduction of perm_range partials covering [0, 2^(n-1))."""
    lib = load()
    if t == PERM_BIN:
        arr = np.zeros((len(partials), 3), dtype=np.uint64)
        for i, v in enumerate(partials):
            v = int(v) % (1 << 192)
            for w in range(3):
                arr[i, w] = (v >> (64 * w)) & 0xFFFFFFFFFFFFFFFF
        out = np.zeros(2, dtype=np.uint64)
    else:
        width = 2 if t in (PERM_F64, PERM_F64X) else 4
        arr = np.ascontiguousarray(np.asarray(partials, dtype=np.float64).reshape(len(partials), width))
        out = np.zeros(1 if t == PERM_F64 else 2, dtype=np.float64)
    rc = lib.perm_combine(t, n, arr.ctypes.data_as(ctypes.c_void_p), len(partials), out.ctypes.data_as(ctypes.c_void_p))
    check(rc, "perm_combine")
    if t == PERM_F64:
        return float(out[0])
    if t == PERM_C128:
        return complex(float(out[0]), float(out[1]))
    if t == PERM_F64X:
        return float(out[0]), float(out[1])
    return _u(out)


def perm_sparse_async(n: int, cptrs, rids, cvals, out, status=None, stream=None) -> None:
    """Enqueue the permanent of an n x n CCS matrix (device int32 cptrs[n+1],
    int32 rids[nnz], float64 cvals[nnz]) into out (float64[1])."""
    lib = load()
    torch = _torch()
    for t, dt in ((cptrs, torch.int32), (rids, torch.int32), (cvals, torch.float64)):
        if not isinstance(t, torch.Tensor) or not t.is_cuda or t.dtype != dt or not t.is_contiguous():
            raise TypeError("CCS arrays must be contiguous CUDA tensors (int32, int32, float64)")
    h, _ = _stream_handle(stream)
    rc = lib.perm_sparse(int(n), ctypes.c_void_p(cptrs.data_ptr()), ctypes.c_void_p(rids.data_ptr()),
                         ctypes.c_void_p(cvals.data_ptr()), int(rids.numel()), ctypes.c_void_p(out.data_ptr()),
                         ctypes.c_void_p(status.data_ptr() if status is not None else 0), h)
    check(rc, "perm_sparse")


def perm_sparse_range_async(n: int, cptrs, rids, cvals, g_begin: int, g_end: int, out, status=None, stream=None,
                            paper_order: bool = False) -> None:
    """Enqueue the raw partial of the sparse sweep over steps [g_begin, g_end)
    into out (float64[2] = hi, lo); paper_order selects Alg. 2's own column
    order instead of the kernel's quiet-row order."""
    lib = load()
    torch = _torch()
    for t, dt in ((cptrs, torch.int32), (rids, torch.int32), (cvals, torch.float64)):
        if not isinstance(t, torch.Tensor) or not t.is_cuda or t.dtype != dt or not t.is_contiguous():
            raise TypeError("CCS arrays must be contiguous CUDA tensors (int32, int32, float64)")
    h, _ = _stream_handle(stream)
    rc = lib.perm_sparse_range(int(n), ctypes.c_void_p(cptrs.data_ptr()), ctypes.c_void_p(rids.data_ptr()),
                               ctypes.c_void_p(cvals.data_ptr()), int(rids.numel()), int(g_begin), int(g_end),
                               _lib.PERM_SPARSE_PAPER_ORDER if paper_order else 0, ctypes.c_void_p(out.data_ptr()),
                               ctypes.c_void_p(status.data_ptr() if status is not None else 0), h)
    check(rc, "perm_sparse_range")


def perm_sparse_range(n: int, cptrs, rids, cvals, g_begin: int, g_end: int, stream=None,
                      paper_order: bool = False) -> tuple:
    """Raw partial (hi, lo) of the sparse sweep over steps [g_begin, g_end); waits."""
    torch = _torch()
    dev = cptrs.device
    out = torch.zeros(2, dtype=torch.float64, device=dev)
    status = torch.full((1,), -1, dtype=torch.int32, device=dev)
    perm_sparse_range_async(n, cptrs, rids, cvals, g_begin, g_end, out, status, stream, paper_order)
    _, s = _stream_handle(stream)
    s.synchronize()
    check(int(status.item()), "perm_sparse_range")
    o = out.cpu().numpy()
    return float(o[0]), float(o[1])


def perm_sparse(n: int, cptrs, rids, cvals, stream=None) -> float:
    """Permanent of an n x n real matrix in CCS form (Alg. 2); waits for it."""
    torch = _torch()
    dev = cptrs.device
    out = torch.zeros(1, dtype=torch.float64, device=dev)
    status = torch.full((1,), -1, dtype=torch.int32, device=dev)
    perm_sparse_async(n, cptrs, rids, cvals, out, status, stream)
    _, s = _stream_handle(stream)
    s.synchronize()
    check(int(status.item()), "perm_sparse")
    return float(out.item())


def _grad_type(A) -> int:
    t = perm_type_of(A.dtype)
    if t == PERM_BIN:
        raise TypeError("perm_grad takes float64 or complex128 matrices")
    return t


def perm_grad_async(A, out, G, status=None, stream=None) -> None:
    """Enqueue the fused permanent + gradient of an n x n CUDA tensor (float64
    or complex128, n <= 32): out has one element of A's dtype, G is n x n."""
    lib = load()
    A = _as_device_matrix(A)
    t = _grad_type(A)
    h, _ = _stream_handle(stream)
    rc = lib.perm_grad(ctypes.c_void_p(A.data_ptr()), A.shape[0], t, ctypes.c_void_p(out.data_ptr()),
                       ctypes.c_void_p(G.data_ptr()), ctypes.c_void_p(status.data_ptr() if status is not None else 0),
                       h)
    check(rc, "perm_grad")


def perm_grad(A, stream=None):
    """(perm(A), d perm / dA) for a CUDA tensor; the permanent as a Python number,
    the gradient as a tensor on A's device (holomorphic derivative for complex A)."""
    torch = _torch()
    A = _as_device_matrix(A)
    out = torch.zeros(1, dtype=A.dtype, device=A.device)
    G = torch.empty_like(A)
    status = torch.full((1,), -1, dtype=torch.int32, device=A.device)
    perm_grad_async(A, out, G, status, stream)
    _, s = _stream_handle(stream)
    s.synchronize()
    check(int(status.item()), "perm_grad")
    v = out.item()
    return v, G


def perm_grad_batched_async(A, out, G, status=None, stream=None) -> None:
    """Enqueue perm_grad_batched over a (count, n, n) CUDA tensor."""
    lib = load()
    torch = _torch()
    if not isinstance(A, torch.Tensor) or not A.is_cuda or A.dim() != 3 or A.shape[1] != A.shape[2]:
        raise ValueError("A must be a CUDA tensor of shape (count, n, n)")
    A = A.contiguous()
    t = _grad_type(A)
    h, _ = _stream_handle(stream)
    rc = lib.perm_grad_batched(ctypes.c_void_p(A.data_ptr()), A.shape[1], A.shape[0], t,
                               ctypes.c_void_p(out.data_ptr()), ctypes.c_void_p(G.data_ptr()),
                               ctypes.c_void_p(status.data_ptr() if status is not None else 0), h)
    check(rc, "perm_grad_batched")


def perm_grad_batched(A, stream=None):
    """(perms, grads) of a (count, n, n) CUDA tensor: perms (count,), grads (count, n, n)."""
    torch = _torch()
    A = A.contiguous()
    out = torch.zeros(A.shape[0], dtype=A.dtype, device=A.device)
    G = torch.empty_like(A)
    status = torch.full((1,), -1, dtype=torch.int32, device=A.device)
    perm_grad_batched_async(A, out, G, status, stream)
    _, s = _stream_handle(stream)
    s.synchronize()
    check(int(status.item()), "perm_grad_batched")
    return out, G


def perm_grad_mixed(mats, device=None, stream=None):
    """Permanents and gradients of a list of square matrices of mixed orders
    (all float64 or all complex128) through perm_grad_batched_mixed; returns
    (numpy array of permanents, list of numpy gradients)."""
    torch = _torch()
    lib = load()
    device = device or torch.device("cuda")
    arrs = [np.asarray(m.detach().cpu().numpy() if hasattr(m, "detach") else m) for m in mats]
    cplx = any(np.iscomplexobj(a) for a in arrs)
    dt = np.complex128 if cplx else np.float64
    ns = [int(a.shape[0]) for a in arrs]
    offs, total = [], 0
    for n in ns:
        offs.append(total)
        total += n * n
    host = np.zeros(max(total, 1), dtype=dt)
    for a, o in zip(arrs, offs):
        host[o:o + a.size] = np.asarray(a, dtype=dt).reshape(-1)
    A = torch.from_numpy(host).to(device)
    G = torch.zeros_like(A)
    out = torch.zeros(len(ns), dtype=A.dtype, device=device)
    status = torch.full((1,), -1, dtype=torch.int32, device=device)
    h, s = _stream_handle(stream)
    karr = (ctypes.c_int * max(len(ns), 1))(*ns)
    oarr = (ctypes.c_int64 * max(len(ns), 1))(*offs)
    check(lib.perm_grad_batched_mixed(PERM_C128 if cplx else PERM_F64, karr, len(ns), ctypes.c_void_p(A.data_ptr()),
                                      oarr, ctypes.c_void_p(out.data_ptr()), ctypes.c_void_p(G.data_ptr()),
                                      ctypes.c_void_p(status.data_ptr()), h), "perm_grad_batched_mixed")
    s.synchronize()
    check(int(status.item()), "perm_grad_batched_mixed")
    g = G.cpu().numpy()
    return out.cpu().numpy(), [g[o:o + n * n].reshape(n, n) for o, n in zip(offs, ns)]


class GradPlan:
    """Permanents and gradients of a fixed list of matrix orders (all float64 or
    all complex128) through perm_grad_plan_*: the device buffers are allocated
    once here; run() gathers, sweeps and scatters without allocating or
    waiting.  A_packed / G_packed hold matrix m at element offsets[m]."""

    def __init__(self, ns, complex_=False, offsets=None):
        lib = load()
        self.ns = [int(n) for n in ns]
        if offsets is None:
            offsets, tot = [], 0
            for n in self.ns:
                offsets.append(tot)
                tot += n * n
        self.offsets = [int(o) for o in offsets]
        self.type = PERM_C128 if complex_ else PERM_F64
        self._plan = ctypes.c_void_p(0)
        karr = (ctypes.c_int * max(len(self.ns), 1))(*self.ns)
        oarr = (ctypes.c_int64 * max(len(self.ns), 1))(*self.offsets)
        check(lib.perm_grad_plan_create(ctypes.byref(self._plan), self.type, karr, len(self.ns), oarr),
              "perm_grad_plan_create")

    def run_async(self, A_packed, out, G_packed, status=None, stream=None) -> None:
        """Enqueue one run on device tensors (A_packed, G_packed: the packed
        layout; out: one element per matrix)."""
        h, _ = _stream_handle(stream)
        check(load().perm_grad_plan_run(self._plan, ctypes.c_void_p(A_packed.data_ptr()),
                                        ctypes.c_void_p(out.data_ptr()), ctypes.c_void_p(G_packed.data_ptr()),
                                        ctypes.c_void_p(status.data_ptr() if status is not None else 0), h),
              "perm_grad_plan_run")

    def close(self):
        if self._plan:
            load().perm_grad_plan_destroy(self._plan)
            self._plan = ctypes.c_void_p(0)

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def set_time_budget(seconds) -> None:
    """Time budget of every sweep launched afterwards (perm_set_time_budget);
    None or 0 removes it.  A sweep that runs out stops with PERM_ETIMEOUT."""
    ns = 0 if not seconds else max(1, int(seconds * 1e9))
    check(load().perm_set_time_budget(ns), "perm_set_time_budget")


def _autograd_function():
    torch = _torch()

    class Permanent(torch.autograd.Function):
        """perm of a float64 / complex128 CUDA matrix (n, n) or batch (count, n, n).

        A single matrix runs perm() forward and the fused gradient sweep
        (perm_grad) backward; a batch runs perm_grad_batched once forward and
        keeps G for backward.  For complex inputs backward returns
        grad_out * conj(G), PyTorch's convention for holomorphic functions."""

        @staticmethod
        def forward(ctx, A):
            if A.dim() == 3:
                out, G = perm_grad_batched(A)
                ctx.save_for_backward(G)
                ctx.batched = True
                return out
            A = _as_device_matrix(A)
            out, status = _out_buffers(perm_type_of(A.dtype), A.device, 2 if A.is_complex() else 1)
            perm_async(A, out, status)
            torch.cuda.current_stream().synchronize()
            check(int(status.item()), "perm")
            ctx.save_for_backward(A)
            ctx.batched = False
            v = torch.view_as_complex(out.view(1, 2))[0] if A.is_complex() else out[0]
            return v.clone()

        @staticmethod
        def backward(ctx, grad_out):
            (X,) = ctx.saved_tensors
            if ctx.batched:
                G = X
                g = grad_out.reshape(-1, 1, 1)
            else:
                _, G = perm_grad(X)
                g = grad_out
            return g * (G.conj() if G.is_complex() else G)

    return Permanent


_PERMANENT = None


def permanent(A):
    """Differentiable permanent (torch.autograd) of a float64 / complex128 CUDA
    matrix (n, n) -> scalar, or of a batch (count, n, n) -> (count,)."""
    global _PERMANENT
    if _PERMANENT is None:
        _PERMANENT = _autograd_function()
    return _PERMANENT.apply(A)


class AbortWord:
    """A word of mapped host memory registered with perm_set_abort_word: set()
    makes the sweeps of perm / perm_range / perm_sparse stop at their next
    chunk group with PERM_EABORTED; clear() lets new launches run."""

    def __init__(self):
        lib = load()
        self._p = ctypes.POINTER(ctypes.c_uint32)()
        check(lib.perm_abort_word_alloc(ctypes.byref(self._p)), "perm_abort_word_alloc")
        check(lib.perm_set_abort_word(ctypes.cast(self._p, ctypes.c_void_p)), "perm_set_abort_word")

    def set(self) -> None:
        self._p[0] = 1

    def clear(self) -> None:
        self._p[0] = 0

    def close(self) -> None:
        if self._p:
            load().perm_abort_word_free(self._p)
            self._p = ctypes.POINTER(ctypes.c_uint32)()


def batched_units(k: int, labels=None):
    """The sweep units a labelled batched plan builds for one k x k matrix
    (host only, perm_batched_units): a list of dicts with gray_bits, weight
    and, for a sweep of the transposed matrix, fixed (row), toggles (rows)
    and repeated ((row, coefficient) pairs); plain sweeps have fixed None."""
    lib = load()
    lab = None if labels is None else np.ascontiguousarray(np.asarray(labels, dtype=np.int32))
    lp = ctypes.c_void_p(0) if lab is None else lab.ctypes.data_as(ctypes.c_void_p)
    cnt = lib.perm_batched_units(int(k), lp, 0, None, None, None, 0, None)
    if cnt < 0:
        check(-cnt, "perm_batched_units")
    g = np.zeros(cnt, dtype=np.int32)
    w = np.zeros(cnt, dtype=np.float64)
    off = np.zeros(cnt, dtype=np.int32)
    cap = cnt * (2 * k + 4)
    desc = np.zeros(max(cap, 1), dtype=np.int32)
    rc = lib.perm_batched_units(int(k), lp, cnt, g.ctypes.data_as(ctypes.c_void_p), w.ctypes.data_as(ctypes.c_void_p),
                                desc.ctypes.data_as(ctypes.c_void_p), cap, off.ctypes.data_as(ctypes.c_void_p))
    if rc < 0:
        check(-rc, "perm_batched_units")
    out = []
    for u in range(cnt):
        d = {"gray_bits": int(g[u]), "weight": float(w[u]), "fixed": None, "toggles": [], "repeated": []}
        if off[u] >= 0:
            o = int(off[u])
            d["fixed"] = int(desc[o])
            G = int(desc[o + 1])
            d["toggles"] = [int(x) for x in desc[o + 2:o + 2 + G]]
            R = int(desc[o + 2 + G])
            rp = desc[o + 3 + G:o + 3 + G + 2 * R]
            d["repeated"] = [(int(rp[2 * t]), int(rp[2 * t + 1])) for t in range(R)]
        out.append(d)
    return out


def equal_row_labels(m) -> np.ndarray:
    """Labels of the rows of one matrix: the index of the first bitwise-equal row."""
    a = np.ascontiguousarray(m.detach().cpu().numpy() if hasattr(m, "detach") else np.asarray(m))
    first = {}
    return np.array([first.setdefault(a[i].tobytes(), i) for i in range(a.shape[0])], dtype=np.int32)


class BatchPlan:
    """A batched plan over a list of square matrices (perm_batched_*), all
    complex128 or all float64 (dtype picks; default: complex128 unless every
    input is real and dtype="float64").

    The matrices are packed into one device buffer owned by the plan; run()
    replays the captured graph (one launch) and returns the device results.

    row_labels (optional): one integer sequence per matrix, equal labels
    marking equal rows (e.g. the modes a boson-sampling submatrix was drawn
    from); such matrices are summed over row multiplicities, with fewer
    terms.  Labelled rows are checked for equality on the device.  "auto"
    labels the bitwise-equal rows of every matrix on the host."""

    def __init__(self, mats, device=None, autotune_rounds: int = 0, stream=None, dtype="complex128",
                 row_labels=None):
        torch = _torch()
        lib = load()
        device = device or torch.device("cuda")
        real = str(dtype) in ("float64", "torch.float64", "<class 'numpy.float64'>")
        self.type = PERM_F64 if real else PERM_C128
        ks = [int(m.shape[0]) for m in mats]
        offs, total = [], 0
        for k in ks:
            offs.append(total)
            total += k * k
        host = np.zeros(total, dtype=np.float64 if real else np.complex128)
        for m, o in zip(mats, offs):
            a = m.detach().cpu().numpy() if hasattr(m, "detach") else np.asarray(m)
            if real and np.iscomplexobj(a):
                raise TypeError("dtype float64 needs real matrices")
            host[o:o + a.size] = np.asarray(a, dtype=host.dtype).reshape(-1)
        self.A = torch.from_numpy(host).to(device)
        self.out = torch.zeros((1 if real else 2) * len(ks), dtype=torch.float64, device=device)
        self.status = torch.full((len(ks),), -1, dtype=torch.int32, device=device)
        self.ks = ks
        self._plan = ctypes.c_void_p(0)
        karr = (ctypes.c_int * len(ks))(*ks)
        oarr = (ctypes.c_int64 * len(ks))(*offs)
        if isinstance(row_labels, str):
            if row_labels != "auto":
                raise ValueError('row_labels must be None, "auto" or one label sequence per matrix')
            row_labels = [equal_row_labels(m) for m in mats]
        if row_labels is None:
            check(lib.perm_batched_plan_create(ctypes.byref(self._plan), self.type, karr, len(ks),
                                               ctypes.c_void_p(self.A.data_ptr()), oarr,
                                               ctypes.c_void_p(self.out.data_ptr()),
                                               ctypes.c_void_p(self.status.data_ptr())), "perm_batched_plan_create")
        else:
            if len(row_labels) != len(ks) or any(len(l) != k for l, k in zip(row_labels, ks)):
                raise ValueError("row_labels needs one label per row of every matrix")
            flat = np.ascontiguousarray(np.concatenate([np.asarray(l, dtype=np.int32) for l in row_labels]))
            larr = flat.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))
            check(lib.perm_batched_plan_create_labeled(ctypes.byref(self._plan), self.type, karr, len(ks),
                                                       ctypes.c_void_p(self.A.data_ptr()), oarr,
                                                       ctypes.c_void_p(self.out.data_ptr()),
                                                       ctypes.c_void_p(self.status.data_ptr()), larr),
                  "perm_batched_plan_create_labeled")
        if autotune_rounds:
            h, _ = _stream_handle(stream)
            check(lib.perm_batched_autotune(self._plan, int(autotune_rounds), h), "perm_batched_autotune")

    def run_async(self, stream=None, A=None, out=None, status=None) -> None:
        """Replay the plan on a stream without waiting.  A, out, status: device
        tensors of this call laid out like self.A / self.out / self.status
        (default: the plan's own); results land in out."""
        h, _ = _stream_handle(stream)
        ptr = lambda t: ctypes.c_void_p(t.data_ptr() if t is not None else 0)
        for t, ref in ((A, self.A), (out, self.out), (status, self.status)):
            if t is not None and (not t.is_cuda or t.dtype != ref.dtype or t.numel() != ref.numel()
                                  or not t.is_contiguous()):
                raise ValueError("per-call buffers must match the plan's layout (dtype, size, contiguous, CUDA)")
        check(load().perm_batched(self._plan, ptr(A), ptr(out), ptr(status), h), "perm_batched")

    def run(self, stream=None):
        """Replay and return a numpy array of the permanents (complex128 or float64)."""
        self.run_async(stream)
        _, s = _stream_handle(stream)
        s.synchronize()
        st = self.status.cpu().numpy()
        bad = np.nonzero(st != 0)[0]
        if len(bad):
            check(int(st[bad[0]]), f"perm_batched (matrix {int(bad[0])})")
        o = self.out.cpu().numpy()
        return o.copy() if self.type == PERM_F64 else o[0::2] + 1j * o[1::2]

    def info(self, k: int):
        """The size class choice for order k: mode, chunk exponent, queue length."""
        mode, c, n = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
        check(load().perm_batched_plan_info(self._plan, int(k), ctypes.byref(mode), ctypes.byref(c), ctypes.byref(n)),
              "perm_batched_plan_info")
        return {"mode": "lane" if mode.value == 1 else "chunks", "c": c.value, "items": n.value}

    def close(self):
        if self._plan:
            load().perm_batched_plan_destroy(self._plan)
            self._plan = ctypes.c_void_p(0)

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


PIPE_NAMES = ("fp64_fma", "fp64_add", "imad", "imad_wide", "shf")


def pipe_peaks(stream=None) -> dict:
    """Measured lane-instructions per second of the pipes the kernels use
    (perm_pipe_peaks)."""
    lib = load()
    out = (ctypes.c_double * len(PIPE_NAMES))()
    h, _ = _stream_handle(stream)
    check(lib.perm_pipe_peaks(out, len(PIPE_NAMES), h), "perm_pipe_peaks")
    return dict(zip(PIPE_NAMES, list(out)))


def perm_host(A, stream=None):
    """perm() on a host numpy array (copies in and out inside the library)."""
    lib = load()
    A = np.asarray(A)
    if A.ndim != 2 or A.shape[0] != A.shape[1]:
        raise ValueError("A must be a square matrix")
    if np.iscomplexobj(A):
        t, A = PERM_C128, np.ascontiguousarray(A, dtype=np.complex128)
        out = np.zeros(2, dtype=np.float64)
    elif A.dtype in (np.uint8, np.bool_):
        t, A = PERM_BIN, np.ascontiguousarray(A, dtype=np.uint8)
        out = np.zeros(2, dtype=np.uint64)
    else:
        t, A = PERM_F64, np.ascontiguousarray(A, dtype=np.float64)
        out = np.zeros(1, dtype=np.float64)
    h = ctypes.c_void_p(0)
    if stream is not None:
        h = ctypes.c_void_p(stream.cuda_stream)
    rc = lib.perm_host(A.ctypes.data_as(ctypes.c_void_p), A.shape[0], t, out.ctypes.data_as(ctypes.c_void_p), h)
    check(rc, "perm_host")
    if t == PERM_F64:
        return float(out[0])
    if t == PERM_C128:
        return complex(float(out[0]), float(out[1]))
    if t == PERM_F64X:
        return float(out[0]), float(out[1])
    return _u(out)

"""Host-side logic of splitting a Gray-code sweep across GPUs, processes or
time (Secs. 3.3 and 6.3: the iteration space is split first per GPU, and the
only exchange is the final sum of partials).

* shard: the contiguous share of [0, 2^(n-1)) that one of `world` ranks owns;
* gather_partials: the single exchange, one all_gather of each rank's partial
  (16-48 bytes) over an initialised torch.distributed group;
* checkpoint / restore: completed ranges with their exact partials as JSON
  (binary64 words as hex), so a long sweep resumes where it stopped and the
  combined result is bit-identical to an uninterrupted run;
* shard_matrices / gather_results: a batch of independent permanents split
  over ranks by matrix, longest first (cost 2^(k-1) k per k x k matrix, or
  the caller's costs), and the per-rank results put back in batch order.
"""
from __future__ import annotations

import json

import numpy as np

from ._lib import PERM_BIN, PERM_C128, PERM_F64, PERM_F64X

WORDS = {PERM_F64: 2, PERM_F64X: 2, PERM_C128: 4, PERM_BIN: 3}


def total_steps(n: int) -> int:
    """Number of Gray steps of an n x n sweep, 2^(n-1) (0 for n = 0)."""
    return 1 << (n - 1) if n > 0 else 0


def shard(n_steps: int, rank: int, world: int):
    """[lo, hi) of rank `rank` out of `world`: contiguous, sizes differ by at most 1."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError("bad rank / world")
    base, rem = divmod(n_steps, world)
    lo = rank * base + min(rank, rem)
    return lo, lo + base + (1 if rank < rem else 0)


def split(n_steps: int, parts: int):
    """The shards of all `parts` ranks, in rank order."""
    return [shard(n_steps, r, parts) for r in range(parts)]


def check_cover(ranges, n_steps: int) -> None:
    """The ranges must tile [0, n_steps) exactly once (any order)."""
    pos = 0
    for lo, hi in sorted(ranges):
        if lo != pos or hi < lo:
            raise ValueError(f"ranges do not tile [0, {n_steps}): gap or overlap at {pos}")
        pos = hi
    if pos != n_steps:
        raise ValueError(f"ranges stop at {pos}, not {n_steps}")


def partial_to_words(t: int, value):
    """A perm_range partial (tuple of floats, or an int for 0/1) as JSON-safe words."""
    if t == PERM_BIN:
        v = int(value) % (1 << 192)
        return [format(v, "048x")]
    return [float(x).hex() for x in value]


def words_to_partial(t: int, words):
    """Inverse of partial_to_words."""
    if t == PERM_BIN:
        return int(words[0], 16)
    return tuple(float.fromhex(w) for w in words)


def checkpoint(t: int, n: int, done) -> str:
    """JSON of completed (lo, hi, partial) triples."""
    return json.dumps({"type": int(t), "n": int(n),
                       "done": [[int(lo), int(hi), partial_to_words(t, p)] for lo, hi, p in done]})


def restore(text: str):
    """(type, n, done triples) from checkpoint() JSON."""
    d = json.loads(text)
    t = int(d["type"])
    return t, int(d["n"]), [(lo, hi, words_to_partial(t, w)) for lo, hi, w in d["done"]]


def remaining(n: int, done):
    """Ranges of [0, 2^(n-1)) not yet covered by done (lo, hi, partial) triples."""
    out, pos = [], 0
    for lo, hi, _ in sorted(done, key=lambda x: x[0]):
        if lo > pos:
            out.append((pos, lo))
        pos = max(pos, hi)
    if pos < total_steps(n):
        out.append((pos, total_steps(n)))
    return out


def gather_partials(dist, t: int, partial_words):
    """All-gather each rank's partial (a list of 64-bit words) with torch.distributed;
    returns the list of partials in rank order on every rank."""
    import torch

    w = WORDS[t]
    if t == PERM_BIN:
        v = int(partial_words) % (1 << 192)
        local = torch.tensor([((v >> (64 * k)) & 0xFFFFFFFFFFFFFFFF) - (1 << 64 if (v >> (64 * k + 63)) & 1 else 0)
                              for k in range(w)], dtype=torch.int64)
    else:
        local = torch.tensor(list(partial_words), dtype=torch.float64)
    backend_dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    local = local.to(backend_dev)
    parts = [torch.zeros_like(local) for _ in range(dist.get_world_size())]
    dist.all_gather(parts, local)
    out = []
    for p in parts:
        p = p.cpu().tolist()
        if t == PERM_BIN:
            out.append(sum((int(x) % (1 << 64)) << (64 * k) for k, x in enumerate(p)))
        else:
            out.append(tuple(p))
    return out


def matrix_cost(k: int) -> float:
    """Work of one k x k sweep: 2^(k-1) Gray steps of k factors each."""
    return float(2 ** (k - 1) * k) if k > 0 else 0.0


def shard_matrices(ks, world: int, costs=None):
    """Indices of the matrices each of `world` ranks computes: longest
    processing time first, each matrix to the least-loaded rank (ties to the
    lower rank, so every rank derives the same assignment).  Returns a list of
    `world` sorted index lists."""
    if world < 1:
        raise ValueError("bad world")
    costs = [matrix_cost(int(k)) for k in ks] if costs is None else [float(c) for c in costs]
    if len(costs) != len(ks):
        raise ValueError("one cost per matrix")
    load = [0.0] * world
    parts = [[] for _ in range(world)]
    for i in sorted(range(len(costs)), key=lambda i: (-costs[i], i)):
        r = min(range(world), key=lambda q: (load[q], q))
        parts[r].append(i)
        load[r] += costs[i]
    return [sorted(p) for p in parts]


def gather_results(dist, indices, values, count: int):
    """All-gather every rank's (index, value) results and return the `count`
    values in batch order on every rank: Python floats when every rank's
    values are real (float64 results, PERM_F64X heads), complex numbers when
    any rank has a complex one.  A rank may hold no matrices.  Indices travel
    as int64, values as float64 pairs."""
    import torch

    vals = list(values)
    idx = [int(i) for i in indices]
    if len(vals) != len(idx):
        raise ValueError("one value per index")
    cplx_local = any(isinstance(v, complex) or np.iscomplexobj(v) for v in vals)
    head = torch.tensor([len(idx), int(cplx_local)], dtype=torch.int64)
    heads = [torch.zeros(2, dtype=torch.int64) for _ in range(dist.get_world_size())]
    dist.all_gather(heads, head)
    width = max(1, max(int(h[0]) for h in heads))  # never a zero-width exchange
    cplx = any(int(h[1]) for h in heads)
    pidx = torch.full((width,), -1, dtype=torch.int64)
    pval = torch.zeros((width, 2), dtype=torch.float64)
    for r, (i, v) in enumerate(zip(idx, vals)):
        c = complex(v)
        pidx[r] = i
        pval[r, 0], pval[r, 1] = c.real, c.imag
    oidx = [torch.zeros_like(pidx) for _ in heads]
    oval = [torch.zeros_like(pval) for _ in heads]
    dist.all_gather(oidx, pidx)
    dist.all_gather(oval, pval)
    res = [None] * count
    for h, ii, vv in zip(heads, oidx, oval):
        for r in range(int(h[0])):
            re, im = (float(x) for x in vv[r].tolist())
            res[int(ii[r])] = complex(re, im) if cplx else re
    if any(v is None for v in res):
        raise ValueError("some matrices were computed by no rank")
    return res

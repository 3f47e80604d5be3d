#!/usr/bin/env python
"""Oracle values of the named configurations, at full size.

Writes ``tests/golden/config_goldens.json``: for each task, the oracle's
result on the seeded input of ``synthetic/``, the SHA-256 of the input's bytes
(the GPU tests recompute it and refuse to compare a different matrix), the
oracle call that produced it and the host it ran on.  Only ``oracle/`` and
``synthetic/`` are used; nothing here touches the CUDA library.

Tasks (all sums are over Alg. 1's Gray steps g in [g0, g1); see oracle/):

  real24            dense real n = 24, uniform [0, 1): double-double sweep
                    with the magnitude sums S and W (ryser_dd_stats_range).
  real40_pPP        dense real n = 40, uniform [-1, 1): part PP of 64 equal
                    parts of [0, 2^39), each a double-double sweep with S, W.
                    The tests add the 64 parts exactly.
  bin36_perm        0/1 n = 36, Bernoulli(0.5): perm(A) mod 2^128 by Eq. 2
                    over all 2^36 subsets without halving (ryser_bin_plain).
  bin36_range       the same matrix: sum over [0, 2^35) of (-1)^g prod x'_i,
                    x' = 2x, mod 2^128 (ryser_bin_range).
  cplx32            Haar 32 x 32 unitary: complex double-double sweep of
                    [0, 2^31) with S, W (ryser_cdd_range).
  boson_kKK_iII     the batched boson workload (8192 matrices, k in 8..26):
                    for every k, the first two matrices of that order,
                    complex double-double sweeps with S, W.
  bosonT_kKK_iII    the same matrices transposed (their permanent is the same;
                    S and W of the transposed sweep bound the sweeps over the
                    columns that the row-labelled batched plans run).
  sparse44_range    sparse n = 44 (density 0.2): the 2^30 steps
                    [2^42, 2^42 + 2^30) of the sweep in Alg. 2's column order
                    (the same Gray steps as Alg. 1 on the dense form; zero
                    entries add nothing), double-double with S, W on the dense
                    form (ryser_dd_stats_range).  The full 2^43 steps are out
                    of reach of the CPU.

Every part runs with a fixed thread count (16), so its value does not depend
on the machine's core count.  Finished tasks are skipped; --only selects
tasks by prefix, --budget stops starting new tasks after that many seconds,
--out writes somewhere else (merge such files back with --merge FILE).

Usage:  python tests/golden/make_config_goldens.py [--only PREFIX ...] [--budget S]
                                                  [--out FILE] [--merge FILE ...]
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import platform
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import oracle  # noqa: E402
import synthetic as syn  # noqa: E402

GOLDEN = os.path.join(HERE, "config_goldens.json")
THREADS = 16
REAL40_PARTS = 64


def digest(a: np.ndarray) -> str:
    return hashlib.sha256(np.ascontiguousarray(a).tobytes()).hexdigest()


def fx(v: float) -> str:
    return float(v).hex()


def boson_selection():
    """(index, k) of the first two matrices of every order k in 8..26."""
    mats = syn.batched_boson()
    picked, seen = [], {}
    for i, m in enumerate(mats):
        k = m.shape[0]
        if seen.get(k, 0) < 2:
            seen[k] = seen.get(k, 0) + 1
            picked.append((i, k))
    return mats, sorted(picked, key=lambda t: (t[1], t[0]))


def tasks():
    out = {}
    out["real24"] = lambda: _dd_stats(syn.dense_real_24(), 0, 1 << 23)
    N40 = 1 << 39
    step = N40 // REAL40_PARTS
    for p in range(REAL40_PARTS):
        out[f"real40_p{p:02d}"] = (lambda p=p: _dd_stats(syn.dense_real_40(), p * step, (p + 1) * step))
    out["bin36_perm"] = lambda: _bin_plain(syn.binary_36())
    out["bin36_range"] = lambda: _bin_range(syn.binary_36(), 0, 1 << 35)
    out["cplx32"] = lambda: _cdd(syn.complex_32(), 0, 1 << 31)
    for i, k in boson_selection()[1]:
        out[f"boson_k{k:02d}_i{i:04d}"] = (lambda i=i: _cdd(syn.batched_boson()[i], 0, 1 << (syn.batched_boson()[i].shape[0] - 1), index=i))
    for i, k in boson_selection()[1]:
        out[f"bosonT_k{k:02d}_i{i:04d}"] = (lambda i=i: _cdd(np.ascontiguousarray(syn.batched_boson()[i].T), 0,
                                                              1 << (syn.batched_boson()[i].shape[0] - 1), index=i))
    out["sparse44_range"] = lambda: _dd_stats(syn.sparse_44(), 1 << 42, (1 << 42) + (1 << 30))
    return out


def _dd_stats(A, g0, g1):
    r = oracle.ryser_dd_stats_range(A, g0, g1, threads=THREADS)
    return {"call": f"oracle.ryser_dd_stats_range(A, {g0}, {g1}, threads={THREADS})", "n": A.shape[0],
            "g0": g0, "g1": g1, "sha256": digest(A), "hi": fx(r["hi"]), "lo": fx(r["lo"]),
            "S": fx(r["S"]), "W": fx(r["W"])}


def _cdd(A, g0, g1, index=None):
    r = oracle.ryser_cdd_range(A, g0, g1, threads=THREADS)
    d = {"call": f"oracle.ryser_cdd_range(A, {g0}, {g1}, threads={THREADS})", "n": A.shape[0], "g0": g0,
         "g1": g1, "sha256": digest(A), **{k: fx(v) for k, v in r.items()}}
    if index is not None:
        d["index"] = index
    return d


def _bin_plain(A):
    v = oracle.perm_bin_plain(A, threads=THREADS)
    return {"call": f"oracle.perm_bin_plain(A, threads={THREADS})", "n": A.shape[0], "sha256": digest(A),
            "perm_mod_2^128": str(v), "bregman_log2": oracle.bregman_log2(A)}


def _bin_range(A, g0, g1):
    v = oracle.ryser_bin_range(A, g0, g1, threads=THREADS)
    return {"call": f"oracle.ryser_bin_range(A, {g0}, {g1}, threads={THREADS})", "n": A.shape[0], "g0": g0,
            "g1": g1, "sha256": digest(A), "sum_mod_2^128": str(v)}


def load(path=GOLDEN) -> dict:
    try:
        with open(path) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def save(data: dict, path=GOLDEN) -> None:
    tmp = path + ".tmp"
    with open(tmp, "w") as f:
        json.dump(dict(sorted(data.items())), f, indent=1)
        f.write("\n")
    os.replace(tmp, path)


def host() -> str:
    return f"{platform.machine()} x{os.cpu_count()}"


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--only", nargs="*", default=None)
    ap.add_argument("--budget", type=float, default=None)
    ap.add_argument("--out", default=GOLDEN)
    ap.add_argument("--merge", nargs="*", default=None)
    ap.add_argument("--reverse", action="store_true", help="run the selected tasks last to first")
    args = ap.parse_args()
    if args.merge:
        data = load(GOLDEN)
        for p in args.merge:
            for k, v in load(p).items():
                data.setdefault(k, v)
        save(data, GOLDEN)
        print(f"merged {len(args.merge)} file(s): {len(data)} tasks")
        return 0
    data = load(args.out)
    done_elsewhere = load(GOLDEN) if args.out != GOLDEN else {}
    t_start = time.time()
    todo = [(k, f) for k, f in tasks().items()
            if k not in data and k not in done_elsewhere and (not args.only or any(k.startswith(p) for p in args.only))]
    if args.reverse:
        todo.reverse()
    for name, fn in todo:
        if args.budget is not None and time.time() - t_start > args.budget:
            break
        t0 = time.time()
        res = fn()
        res["seconds"] = round(time.time() - t0, 1)
        res["host"] = host()
        data = load(args.out)
        data[name] = res
        save(data, args.out)
        print(f"{name}: {res['seconds']} s", flush=True)
    return 0


if __name__ == "__main__":
    sys.exit(main())

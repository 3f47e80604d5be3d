#!/usr/bin/env python
"""Benchmark of the Ryser / Nijenhuis-Wilf Gray-code sweep on GB300.

One step = one pass of the whole hot path over the dense workload:
  * dense real n=40, uniform [-1, 1)            (2^39 Gray steps)
  * 0/1 Bernoulli(0.5) n=36, exact              (2^35 Gray steps)
  * complex128 Haar-random 32 x 32 unitary      (2^31 Gray steps)
The metric is Gray-code steps per second over all three (whole job, all
ranks).  Under torchrun every permanent's Gray range is split evenly across
ranks (perm_range per rank), the partials are gathered and rank 0 combines
them (perm_combine): the single exchange of the method (Secs. 3.3, 6.3).

Prints one JSON line (rank 0).  `--impl reference` times the CPU oracle
instead (as it stands, all host cores, a bounded sample of the same workload
per step).
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import synthetic as syn  # noqa: E402

METRIC = "Gray-code steps/s & FP64-peak fraction (n=40 dense); batched perms/s; grad/fwd"
WORKLOAD = "dense real n=40 U[-1,1) + 0/1 Bernoulli(0.5) n=36 + complex128 Haar 32x32 (one permanent each per step)"
L2_FLUSH_BYTES = 256 << 20  # larger than the 129 MB L2


def workloads():
    return [
        ("real40", syn.dense_real_40()),
        ("bin36", syn.binary_36()),
        ("cplx32", syn.complex_32()),
    ]


def steps_of(n: int) -> int:
    return 1 << (n - 1)


# ----------------------------------------------------------------- clocks

class ClockSampler:
    """nvidia-smi clock / throttle samples every 200 ms during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(prefix="clocks", suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200", "-f", self.path], stdout=subprocess.DEVNULL, stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        rows = []
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 9 and parts[1].replace(".", "").isdigit():
                rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        sm = [float(r[1]) for r in rows]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4) if r[5 + k].lower() == "active"})
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": float(rows[0][2]), "reasons": reasons,
                "samples": len(rows), "power_w_max": max(float(r[3]) for r in rows if r[3].replace(".", "").isdigit())}


# -------------------------------------------------------------- distributed

def dist_setup(ngpus: int):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist

        backend = "nccl" if _cuda_ok() else "gloo"
        dist.init_process_group(backend=backend)
        return rank, world, local, dist
    return 0, 1, 0, None


def _cuda_ok() -> bool:
    try:
        import torch

        return torch.cuda.is_available()
    except ImportError:
        return False


# ---------------------------------------------------------------- CPU oracle

def oracle_sample(frac_log2: int, threads: int):
    """Time the oracle (as it stands) on a bounded sample of every permanent:
    the first 2^(n-1-frac_log2) steps of each Gray range.  Returns
    (steps, seconds)."""
    import oracle

    total, secs = 0, 0.0
    for name, A in workloads():
        n = A.shape[0]
        s = max(1, steps_of(n) >> frac_log2)
        fn = {"real40": oracle.ryser_f64_range, "bin36": oracle.ryser_bin_range,
              "cplx32": oracle.ryser_c128_range}[name]
        t0 = time.perf_counter()
        fn(A, 0, s, threads=threads)
        secs += time.perf_counter() - t0
        total += s
    return total, secs


def run_reference(args):
    # under torchrun only rank 0 runs the CPU oracle; the others exit at once
    if int(os.environ.get("RANK", "0")) != 0:
        return 0
    threads = os.cpu_count() or 1
    frac = 10  # 2^-10 of each Gray range per step
    for _ in range(args.warmup):
        oracle_sample(frac, threads)
    tot_steps, tot_secs = 0, 0.0
    for _ in range(args.steps):
        s, t = oracle_sample(frac, threads)
        tot_steps += s
        tot_secs += t
    value = tot_steps / tot_secs
    sample = f"first 2^-{frac} of each Gray range per step (real40 2^29, bin36 2^25, cplx32 2^21 steps)"
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "steps/s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * tot_secs / args.steps,
        "higher_is_better": True, "scaling": "strong", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": {"workload": WORKLOAD, "oracle": "CPU Ryser/N-W (Alg. 1/3), pthreads"},
        "cpu_baseline": {"value": value, "unit": "steps/s", "cores": threads, "kind": "oracle", "sample": sample,
                         "host": host_cpu()},
        "e2e": {"value": value, "unit": "steps/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


# ------------------------------------------------------------------- GPU arm

# Executed lane-instructions per Gray step of ryser_real_kernel<40>, from an ncu
# capture of this kernel (smsp__inst_executed.sum x 32 / steps), with the
# SHA-256 (first 16 hex digits) of the kernel source it was taken on.  The
# issue view below is reported only while real.cuh still has that hash.
REAL40_INST_PER_STEP = 737.0
REAL40_INST_SOURCE = "542f77d7e2948508"


def kernel_source_hash() -> str:
    import hashlib

    with open(os.path.join(ROOT, "paper_2502_16577_gb300", "csrc", "real.cuh"), "rb") as f:
        return hashlib.sha256(f.read()).hexdigest()[:16]


def host_cpu() -> str:
    """The host CPU as the kernel reports it: machine, model name (x86) or
    implementer / part (Arm), and the core count."""
    import platform

    model = ""
    try:
        info = open("/proc/cpuinfo").read().splitlines()
        for key in ("model name", "CPU part"):
            vals = [l.split(":", 1)[1].strip() for l in info if l.startswith(key)]
            if vals:
                model = f"{key} {vals[0]}"
                break
    except OSError:
        pass
    return f"{platform.machine()} {model} x{os.cpu_count() or 1}".strip()


def measured_peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except (OSError, ValueError):
        return {}


def run_gpu(args):
    import torch

    import paper_2502_16577_gb300 as pg
    from paper_2502_16577_gb300 import ranges

    rank, world, local, dist = dist_setup(args.gpus)
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    pg.load()
    stream = torch.cuda.current_stream(dev)
    mats = []
    for name, A in workloads():
        t = torch.from_numpy(np.ascontiguousarray(A)).to(dev)
        n = A.shape[0]
        lo, hi = ranges.shard(steps_of(n), rank, world)
        typ = pg.perm_type_of(t.dtype)
        words = {pg.PERM_F64: 2, pg.PERM_C128: 4, pg.PERM_BIN: 3}[typ]
        out = torch.zeros(words, dtype=torch.int64 if typ == pg.PERM_BIN else torch.float64, device=dev)
        mats.append(dict(name=name, A=t, host=A, n=n, lo=lo, hi=hi, type=typ, out=out,
                         status=torch.zeros(1, dtype=torch.int32, device=dev)))
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.int32, device=dev)
    ev = lambda: torch.cuda.Event(enable_timing=True)

    def one_step(real_events=None):
        for m in mats:
            if m["name"] == "real40" and real_events is not None:
                real_events[0].record(stream)
            if world == 1:
                pg.perm_async(m["A"], m["out"], m["status"], stream)
            else:
                pg.perm_range_async(m["A"], m["lo"], m["hi"], m["out"], m["status"], stream)
            if m["name"] == "real40" and real_events is not None:
                real_events[1].record(stream)

    def gather_and_combine():
        """The exchange: every rank's partials to rank 0, combined on the host."""
        results = {}
        for m in mats:
            if world == 1:
                results[m["name"]] = m["out"].cpu().numpy().copy()
                continue
            o = m["out"].cpu().numpy()
            local_part = sum((int(w) % (1 << 64)) << (64 * i) for i, w in enumerate(o)) \
                if m["type"] == pg.PERM_BIN else tuple(float(v) for v in o)
            parts = ranges.gather_partials(dist, m["type"], local_part)
            if rank == 0:
                results[m["name"]] = pg.perm_combine(m["type"], m["n"], parts)
        return results

    # warm-up (untimed)
    for _ in range(args.warmup):
        one_step()
        torch.cuda.synchronize(dev)
        gather_and_combine()
    for m in mats:
        st = int(m["status"].item())
        if st not in (0,):
            raise RuntimeError(f"{m['name']}: status {st}")
        m["ref"] = m["out"].clone()  # the kernels are deterministic: every timed step must match

    def verify_step():
        for m in mats:
            st = int(m["status"].item())
            if st != 0:
                raise RuntimeError(f"timed step: {m['name']} status {st}")
            if not torch.equal(m["out"], m["ref"]):
                raise RuntimeError(f"timed step: {m['name']} result differs from the warm-up's bits")

    peaks = pg.pipe_peaks(stream) if rank == 0 else {}

    sampler = ClockSampler(local)
    if dist is not None:
        dist.barrier()
    torch.cuda.synchronize(dev)
    sampler.start()
    step_ms, real_ms = [], []
    for _ in range(args.steps):
        flush.zero_()  # L2 flush between timed steps (outside the events)
        e0, e1, r0, r1 = ev(), ev(), ev(), ev()
        e0.record(stream)
        one_step((r0, r1))
        e1.record(stream)
        torch.cuda.synchronize(dev)
        verify_step()
        gather_and_combine()
        step_ms.append(e0.elapsed_time(e1))
        real_ms.append(r0.elapsed_time(r1))
    torch.cuda.synchronize(dev)
    if dist is not None:
        dist.barrier()
    clocks = sampler.stop()
    local_ms = sum(step_ms)
    if dist is not None:
        t = torch.tensor([local_ms], dtype=torch.float64, device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        local_ms = float(t.item())
    total_steps = sum(steps_of(m["n"]) for m in mats)
    value = total_steps * args.steps / (local_ms * 1e-3)

    # end to end through the public host-buffer entry point (rank 0 of N=1 only,
    # or every rank on its shard through the device path plus copies)
    e2e = None
    if world == 1:
        host = [(m["host"], m["n"]) for m in mats]
        h2d = sum(a.nbytes for a, _ in host)
        d2h = 8 + 16 + 16
        ke = args.steps
        want = [pg.perm_host(a) for a, _ in host]  # untimed: the values every timed step must return
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        for _ in range(ke):
            got = [pg.perm_host(a) for a, _ in host]
            if got != want:
                raise RuntimeError("e2e: a host-buffer step returned other values")
        dt = time.perf_counter() - t0
        e2e = {"value": total_steps * ke / dt, "unit": "steps/s", "h2d_bytes_per_step": h2d,
               "d2h_bytes_per_step": d2h}

    if rank != 0:
        return 0

    batched = None if args.no_batched else measure_batched(pg, dev, stream)
    grad = None if args.no_batched else measure_grad(pg, dev, stream)

    extras = None if args.no_batched else measure_extras(pg, dev, stream)

    # roofline of the dominant kernel (dense real n=40).  The method's work is
    # 2n operations per Gray step (n row updates and n factors of the product,
    # Alg. 1); the kernel runs them on the integer pipes, so the ceiling is the
    # SM issue rate (152 SMs x 128 lanes x the maximum SM clock).
    n40 = 40
    method_ops = 2 * n40
    real_s = statistics.median(real_ms) * 1e-3
    real_steps = mats[0]["hi"] - mats[0]["lo"]
    mp = measured_peaks()
    sm_max = float(mp.get("sm_max_mhz", 2070.0))
    import torch as _t

    nsm = _t.cuda.get_device_properties(dev).multi_processor_count
    issue_peak = nsm * 128 * sm_max * 1e6  # lane-instructions/s
    achieved = method_ops * real_steps / real_s
    fp64_peak = peaks.get("fp64_fma", 0.0)  # FP64 instructions/s (an FMA counts once)
    issue_view = None
    if REAL40_INST_PER_STEP and REAL40_INST_SOURCE == kernel_source_hash():
        issue_view = {"inst_per_step": REAL40_INST_PER_STEP,
                      "issue_frac": REAL40_INST_PER_STEP * real_steps / real_s / issue_peak,
                      "source": "ncu smsp__inst_executed.sum of this kernel source"}
    line = {
        "metric": METRIC, "value": value, "unit": "steps/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": local_ms / args.steps, "higher_is_better": True,
        "scaling": "strong", "vs_baseline": None, "dtype": "int64",
        "data": "synthetic",
        "config": {"workload": WORKLOAD, "l2": "flushed between timed steps (256 MiB write, outside the events)",
                   "steps_per_pass": total_steps, "split": "Gray range split evenly across ranks" if world > 1
                   else "one launch per permanent", "arith": "int64 fixed-point rows, 62-bit integer products, "
                   "binary64 + double-double sums; 0/1 exact mod 2^192"},
        "gpu_launches": 3 * args.steps,
        "roofline": {"bound": "alu", "achieved": achieved / 1e12, "peak": issue_peak / 1e12,
                     "unit": "Tops/s", "frac": achieved / issue_peak, "traffic": args.traffic,
                     "kernel": "ryser_real_kernel<40>", "work_per_step": method_ops,
                     "work": "2n method operations per Gray step (Alg. 1: n row updates, n product factors)",
                     "peak_from": f"{nsm} SMs x 128 issue lanes x {sm_max:.0f} MHz (max SM clock)",
                     "issue_view": issue_view},
        "fp64_view": {"steps_per_s": real_steps / real_s, "fp64_equiv_ops_per_s": method_ops * real_steps / real_s,
                      "fp64_pipe_peak_ops_per_s": fp64_peak,
                      "fp64_equiv_rate_over_fp64_peak": method_ops * real_steps / real_s / fp64_peak
                      if fp64_peak else None,
                      "note": "the 2n operations per step run on the integer pipes, not the FP64 pipe",
                      "paper_gv100_steps_per_s": 2 ** 39 / 14.17},
        "pipe_peaks": peaks,
        "per_config_ms": {"real40": statistics.median(real_ms)},
        "extras": extras,
        "batched": batched,
        "grad": grad,
        "clocks": clocks,
        "e2e": e2e,
    }
    if not args.no_cpu_baseline:
        s, t = oracle_sample(8, os.cpu_count() or 1)
        line["cpu_baseline"] = {"value": s / t, "unit": "steps/s", "cores": os.cpu_count() or 1, "kind": "oracle",
                                "sample": "first 2^-8 of each Gray range (real40 2^31, bin36 2^27, cplx32 2^23 steps)",
                                "seconds": t, "host": host_cpu()}
    print(json.dumps(line), flush=True)
    return 0


def _median_ms(fn, sync, ev, stream, reps: int = 5, check=None):
    """Median device time (CUDA events on the stream) of reps calls of fn, after
    one untimed call; check() runs after every timed call."""
    fn()
    sync()
    if check:
        check()
    ts = []
    for _ in range(reps):
        e0, e1 = ev(), ev()
        e0.record(stream)
        fn()
        e1.record(stream)
        sync()
        if check:
            check()
        ts.append(e0.elapsed_time(e1))
    return statistics.median(ts)


def measure_batched(pg, dev, stream, count: int = 8192, reps: int = 5):
    """Batched boson workload: 8192 complex k x k submatrices (k uniform in
    8..26, rows with replacement from a Haar 256 x 256 unitary): graph replays
    (median of reps) of the plan with the heuristic chunking, and of the plan
    with the drawn modes as row labels (repeated rows summed over their
    multiplicities), heuristic and autotuned (perm_batched_autotune, one
    round), against a loop of perm() launches on one stream.  Every replay's
    statuses and bits are checked."""
    import torch

    mats, rows = syn.batched_boson(count, with_rows=True)
    ev = lambda: torch.cuda.Event(enable_timing=True)
    sync = lambda: torch.cuda.synchronize(dev)

    def timed_plan(plan):
        ref = plan.run(stream)

        def check():
            if not bool((plan.status == 0).all()):
                raise RuntimeError("batched replay: a nonzero status")
            o = plan.out.cpu().numpy()
            if not np.array_equal(o[0::2] + 1j * o[1::2], ref):
                raise RuntimeError("batched replay: results differ between replays")

        ms = _median_ms(lambda: plan.run_async(stream), sync, ev, stream, reps, check)
        return ms * 1e-3, ref

    plan = pg.BatchPlan(mats, device=dev)
    t_plain, res = timed_plan(plan)
    plan.close()
    plan = pg.BatchPlan(mats, device=dev, row_labels=rows)
    t_lab, res_lab = timed_plan(plan)
    plan.close()
    t0 = time.perf_counter()
    plan = pg.BatchPlan(mats, device=dev, row_labels=rows, autotune_rounds=1, stream=stream)
    tune_lab_s = time.perf_counter() - t0
    t_lab_tuned, _ = timed_plan(plan)
    plan.close()
    devm = [torch.from_numpy(np.ascontiguousarray(m)).to(dev) for m in mats]
    out = torch.zeros(2 * count, dtype=torch.float64, device=dev)
    st = torch.zeros(count, dtype=torch.int32, device=dev)

    def loop():
        for i in range(count):
            pg.perm_async(devm[i], out[2 * i:2 * i + 2], st[i:i + 1], stream)

    def check_loop():
        if not bool((st == 0).all()):
            raise RuntimeError("perm() loop: a nonzero status")

    t_loop = _median_ms(loop, sync, ev, stream, 3, check_loop) * 1e-3
    o = out.cpu().numpy()
    same = bool(np.array_equal(res, o[0::2] + 1j * o[1::2]))
    scale = np.maximum(np.abs(res), 1e-300)
    steps = sum(1 << (m.shape[0] - 1) for m in mats)
    best = min(t_lab, t_lab_tuned)
    return {"workload": f"{count} complex128 boson submatrices, k uniform 8..26, drawn modes as row labels",
            "perms_per_s": count / best, "labeled_perms_per_s": count / t_lab,
            "labeled_autotuned_perms_per_s": count / t_lab_tuned,
            "plain_perms_per_s": count / t_plain, "autotune_seconds": tune_lab_s,
            "steps_per_s": steps / t_plain, "loop_perms_per_s": count / t_loop,
            "speedup_vs_loop": t_loop / best,
            "labeled_vs_plain_max_rel": float(np.max(np.abs(res_lab - res) / scale)),
            "plain_identical_to_loop": same, "launches_per_replay": 3, "timing": f"median of {reps} replays"}


def measure_grad(pg, dev, stream, reps: int = 5):
    """Fused gradient: dense real n=28 uniform [-1, 1) (perm_grad vs perm on the
    same matrix, and vs n^2 forwards of one (n-1) minor), and 1024 complex
    16 x 16 Haar submatrices (perm_grad_batched vs the batched forward plan).
    Medians of reps launches; statuses checked after each."""
    import torch

    ev = lambda: torch.cuda.Event(enable_timing=True)
    sync = lambda: torch.cuda.synchronize(dev)
    st = torch.zeros(1, dtype=torch.int32, device=dev)

    def ok():
        if int(st.item()) != 0:
            raise RuntimeError(f"gradient section: status {int(st.item())}")

    A = torch.from_numpy(syn.grad_real_28()).to(dev)
    n = A.shape[0]
    out = torch.zeros(2, dtype=torch.float64, device=dev)
    G = torch.empty_like(A)
    t_grad = _median_ms(lambda: pg.perm_grad_async(A, out[:1], G, st, stream), sync, ev, stream, reps, ok) * 1e-3
    t_fwd = _median_ms(lambda: pg.perm_async(A, out, st, stream), sync, ev, stream, reps, ok) * 1e-3
    M = A[1:, 1:].contiguous()
    t_minor = _median_ms(lambda: pg.perm_async(M, out, st, stream), sync, ev, stream, reps, ok) * 1e-3
    mats = syn.grad_boson_16(1024)
    B = torch.from_numpy(mats).to(dev)
    bout = torch.zeros(1024, dtype=torch.complex128, device=dev)
    BG = torch.empty_like(B)
    t_bgrad = _median_ms(lambda: pg.perm_grad_batched_async(B, bout, BG, st, stream), sync, ev, stream, reps,
                         ok) * 1e-3
    plan = pg.BatchPlan(list(mats), device=dev)
    t_bfwd = _median_ms(lambda: plan.run_async(stream), sync, ev, stream, reps) * 1e-3
    plan.close()
    k = mats.shape[1]
    return {"real28": {"grad_ms": t_grad * 1e3, "fwd_ms": t_fwd * 1e3, "grad_over_fwd": t_grad / t_fwd,
                       "steps_per_s": (1 << (n - 1)) / t_grad,
                       "n2_minor_forwards_ms": n * n * t_minor * 1e3,
                       "speedup_vs_n2_minor_forwards": n * n * t_minor / t_grad},
            "complex16_x1024": {"grad_ms": t_bgrad * 1e3, "fwd_ms": t_bfwd * 1e3,
                                "grad_over_fwd": t_bgrad / t_bfwd,
                                "steps_per_s": 1024 * (1 << (k - 1)) / t_bgrad},
            "timing": f"median of {reps} launches",
            "launches": "grad: 1 sweep + 3 small finishing kernels; fwd: 1 (real), 3 per graph replay (batched)"}


def measure_extras(pg, dev, stream, reps: int = 5):
    """The other named workloads: the sparse n = 44 matrix (density 0.2) on a
    fixed 2^36-step sub-range of its sweep (every chunk the same work), and the
    latency of one dense real n = 24 uniform [0, 1) permanent (2^23 steps, too
    small to fill the GPU).  Medians of reps launches, statuses checked."""
    import torch

    ev = lambda: torch.cuda.Event(enable_timing=True)
    sync = lambda: torch.cuda.synchronize(dev)
    st = torch.zeros(1, dtype=torch.int32, device=dev)

    def ok():
        if int(st.item()) != 0:
            raise RuntimeError(f"extras: status {int(st.item())}")

    S = syn.sparse_44()
    cp, ri, cv = (torch.from_numpy(np.ascontiguousarray(x)).to(dev) for x in syn.to_ccs(S))
    part = torch.zeros(2, dtype=torch.float64, device=dev)
    g0, g1 = 1 << 40, (1 << 40) + (1 << 36)
    t_sp = _median_ms(lambda: pg.perm_sparse_range_async(44, cp, ri, cv, g0, g1, part, st, stream), sync, ev,
                      stream, reps, ok) * 1e-3
    A = torch.from_numpy(syn.dense_real_24()).to(dev)
    out = torch.zeros(1, dtype=torch.float64, device=dev)
    lat = _median_ms(lambda: pg.perm_async(A, out, st, stream), sync, ev, stream, 4 * reps, ok)
    return {"sparse44": {"steps": g1 - g0, "ms": t_sp * 1e3, "steps_per_s": (g1 - g0) / t_sp,
                         "nnz": int(ri.numel()), "full_sweep_s_estimate": (1 << 43) / ((g1 - g0) / t_sp)},
            "dense24": {"latency_ms": lat, "steps_per_s": (1 << 23) / (lat * 1e-3)},
            "timing": f"median of {reps} (dense24: {4 * reps}) launches"}


def run_case(args):
    """One kernel on one input, for profiling and sweeps: KIND:N with KIND in
    real (uniform [-1, 1)), realx (the same with extended-precision products),
    bin (Bernoulli 0.5), cplx (Haar unitary), sparse
    (density 0.2, CCS), grad (real, fused gradient), bgrad (1024 complex N x N
    boson submatrices, batched gradient).  Prints one JSON line."""
    import torch

    import paper_2502_16577_gb300 as pg

    pg.load()
    kind, n = args.case.split(":")
    n = int(n)
    dev = torch.device("cuda", 0)
    stream = torch.cuda.current_stream(dev)
    st = torch.zeros(1, dtype=torch.int32, device=dev)
    seed = syn.SEED_BASE + 100 + n
    steps = 1 << (n - 1)
    if kind in ("real", "realx", "bin", "cplx"):
        A = {"real": lambda: syn.signed_real(n, seed), "realx": lambda: syn.signed_real(n, seed),
             "bin": lambda: syn.bernoulli01(n, seed), "cplx": lambda: syn.haar_unitary(n, seed)}[kind]()
        A = torch.from_numpy(A).to(dev)
        out = torch.zeros(4, dtype=torch.int64 if kind == "bin" else torch.float64, device=dev)
        fn = lambda: pg.perm_async(A, out, st, stream, extended=kind == "realx")
    elif kind == "sparse":
        cp, ri, cv = syn.to_ccs(syn.sparse_real(n, seed, 0.2))
        cp, ri, cv = (torch.from_numpy(np.ascontiguousarray(x)).to(dev) for x in (cp, ri, cv))
        out = torch.zeros(1, dtype=torch.float64, device=dev)
        fn = lambda: pg.perm_sparse_async(n, cp, ri, cv, out, st, stream)
    elif kind == "grad":
        A = torch.from_numpy(syn.signed_real(n, seed)).to(dev)
        out = torch.zeros(1, dtype=torch.float64, device=dev)
        G = torch.empty_like(A)
        fn = lambda: pg.perm_grad_async(A, out, G, st, stream)
    elif kind == "bgrad":
        B = torch.from_numpy(np.stack(syn.boson_submatrices(1024, seed, n, n, 256))).to(dev)
        out = torch.zeros(1024, dtype=torch.complex128, device=dev)
        G = torch.empty_like(B)
        fn = lambda: pg.perm_grad_batched_async(B, out, G, st, stream)
        steps *= 1024
    else:
        raise SystemExit(f"unknown case {args.case}")
    for _ in range(args.warmup):
        fn()
    torch.cuda.synchronize(dev)
    ms = []
    for _ in range(args.steps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        fn()
        e1.record(stream)
        torch.cuda.synchronize(dev)
        ms.append(e0.elapsed_time(e1))
    if int(st.item()) != 0:
        raise SystemExit(f"status {int(st.item())}")
    t = statistics.median(ms)
    print(json.dumps({"case": args.case, "ms": t, "steps_per_s": steps / (t * 1e-3), "launches": args.steps}),
          flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-batched", action="store_true")
    ap.add_argument("--traffic", type=float, default=None,
                    help="DRAM bytes per launch of the dominant kernel from an ncu capture")
    ap.add_argument("--case", default=None, help="KIND:N, one kernel on one input (profiling)")
    args = ap.parse_args()
    if args.case:
        return run_case(args)
    if args.warmup < 3:
        ap.error("--warmup must be at least 3")
    if args.impl == "reference":
        return run_reference(args)
    return run_gpu(args)


if __name__ == "__main__":
    sys.exit(main())

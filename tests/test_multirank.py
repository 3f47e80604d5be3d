"""Multi-rank host logic on CPU (gloo, world size 2): every rank computes its
shard of the Gray range (here with the oracle, the stand-in for a GPU), the
partials are all-gathered once and combined by the library's host
perm_combine; a rank that drops its work is detected; a checkpointed sweep
resumes to the same bits."""
import os
import socket

import numpy as np
import pytest

import synthetic as syn

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _oracle_partial(t, A, lo, hi):
    import oracle
    from paper_2502_16577_gb300 import PERM_BIN, PERM_C128, PERM_F64, PERM_F64X

    if lo == hi:
        return 0 if t == PERM_BIN else (0.0,) * (2 if t in (PERM_F64, PERM_F64X) else 4)
    if t == PERM_F64:
        return oracle.ryser_f64_range(A, lo, hi, threads=2)
    if t == PERM_F64X:  # extended products: the oracle's double-double range sum
        return oracle.ryser_dd_range(A, lo, hi, threads=2)
    if t == PERM_C128:
        return oracle.ryser_c128_range(A, lo, hi, threads=2)
    v = oracle.ryser_bin_range(A, lo, hi, threads=2)  # residue mod 2^128 of a small sum
    return (v - (1 << 128)) % (1 << 192) if v >= (1 << 127) else v


def _worker(rank, world, port, results, drop_rank):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import paper_2502_16577_gb300 as pg
        from paper_2502_16577_gb300 import ranges

        cases = [(pg.PERM_F64, syn.signed_real(13, 1)), (pg.PERM_C128, syn.haar_unitary(11, 2)),
                 (pg.PERM_BIN, syn.bernoulli01(14, 3)), (pg.PERM_F64X, syn.signed_real(12, 4))]
        out = []
        for t, A in cases:
            n = A.shape[0]
            lo, hi = ranges.shard(ranges.total_steps(n), rank, world)
            if rank == drop_rank:
                lo = hi  # a failed rank: its range is never computed
            part = _oracle_partial(t, A, lo, hi)
            parts = ranges.gather_partials(dist, t, part)
            if rank == 0:
                try:
                    out.append(("ok", pg.perm_combine(t, n, parts)))
                except pg.PermError as e:
                    out.append(("err", e.code))
        if rank == 0:
            results.extend(out)
    finally:
        dist.destroy_process_group()


def _run(drop_rank):
    ctx = mp.get_context("spawn")
    with ctx.Manager() as m:
        results = m.list()
        procs = [ctx.Process(target=_worker, args=(r, 2, _free_port_cache[0], results, drop_rank)) for r in range(2)]
        for p in procs:
            p.start()
        for p in procs:
            p.join(120)
            assert p.exitcode == 0
        return list(results)


_free_port_cache = [None]


@pytest.fixture(autouse=True)
def _port():
    _free_port_cache[0] = _free_port()


def test_two_ranks_combine_to_the_full_permanent(oracle):
    from fractions import Fraction

    res = _run(drop_rank=-1)
    assert [r[0] for r in res] == ["ok", "ok", "ok", "ok"]
    want_r = oracle.perm_dp_f64(syn.signed_real(13, 1))
    want_c = oracle.perm_dp_c128(syn.haar_unitary(11, 2))
    want_b = oracle.perm_dp_bin(syn.bernoulli01(14, 3))
    scale = oracle.perm_dp_f64(np.abs(syn.signed_real(13, 1)))
    assert abs(res[0][1] - want_r) <= 1e-13 * scale
    assert abs(res[1][1] - want_c) <= 1e-13
    assert res[2][1] == want_b
    hi, lo = res[3][1]
    want_x = sum(map(Fraction, oracle.perm_dd(syn.signed_real(12, 4))))
    assert abs(Fraction(hi) + Fraction(lo) - want_x) <= Fraction(1, 10 ** 27) * Fraction(
        oracle.perm_dp_f64(np.abs(syn.signed_real(12, 4))))


def test_a_rank_that_drops_its_range_is_detected(oracle):
    res = _run(drop_rank=1)
    want_r = oracle.perm_dp_f64(syn.signed_real(13, 1))
    assert res[0][0] == "ok" and abs(res[0][1] - want_r) > 1e-6 * abs(want_r)
    # the 0/1 sum carries a checksum: its low n-1 bits must be zero
    assert res[2] == ("err", 1) or res[2][1] != oracle.perm_dp_bin(syn.bernoulli01(14, 3))


def test_shards_tile_the_range():
    from paper_2502_16577_gb300 import ranges

    for n_steps in (1, 7, 2 ** 20, 2 ** 39 + 3):
        for world in (1, 2, 3, 8):
            parts = ranges.split(n_steps, world)
            ranges.check_cover(parts, n_steps)
            sizes = [b - a for a, b in parts]
            assert max(sizes) - min(sizes) <= 1
    with pytest.raises(ValueError):
        ranges.check_cover([(0, 3), (4, 8)], 8)


def test_checkpoint_resume_is_bit_identical(oracle):
    import paper_2502_16577_gb300 as pg
    from paper_2502_16577_gb300 import ranges

    A = syn.signed_real(15, 9)
    n = 15
    N = ranges.total_steps(n)
    cuts = [(0, 5000), (5000, 9000), (9000, N)]
    straight = [oracle.ryser_f64_range(A, a, b, threads=2) for a, b in cuts]
    # first session: two ranges done, checkpoint written
    text = ranges.checkpoint(pg.PERM_F64, n, [(a, b, p) for (a, b), p in zip(cuts[:2], straight[:2])])
    t, n2, done = ranges.restore(text)
    todo = ranges.remaining(n2, done)
    assert todo == [(9000, N)]
    done += [(a, b, oracle.ryser_f64_range(A, a, b, threads=2)) for a, b in todo]
    ranges.check_cover([(a, b) for a, b, _ in done], N)
    resumed = pg.perm_combine(t, n2, [p for _, _, p in sorted(done)])
    assert resumed == pg.perm_combine(pg.PERM_F64, n, straight)
    B = syn.bernoulli01(12, 4)
    bparts = [(0, 100, oracle.ryser_bin_range(B, 0, 100)), (100, 2 ** 11, oracle.ryser_bin_range(B, 100, 2 ** 11))]
    bparts = [(a, b, (v - (1 << 128)) % (1 << 192) if v >= (1 << 127) else v) for a, b, v in bparts]
    t, nb, done = ranges.restore(ranges.checkpoint(pg.PERM_BIN, 12, bparts))
    assert pg.perm_combine(t, nb, [p for _, _, p in done]) == oracle.perm_dp_bin(B)


# ------------------------------------------------- batches shard by matrix

def test_batch_shards_cover_and_balance():
    from paper_2502_16577_gb300 import ranges

    g = syn.rng(77)
    for world in (1, 2, 3, 8):
        ks = [int(k) for k in g.integers(8, 27, size=500)]
        parts = ranges.shard_matrices(ks, world)
        assert sorted(i for p in parts for i in p) == list(range(len(ks)))
        loads = [sum(ranges.matrix_cost(ks[i]) for i in p) for p in parts]
        total, big = sum(loads), max(ranges.matrix_cost(k) for k in ks)
        assert max(loads) <= total / world + big  # LPT: within one matrix of the mean
        assert parts == ranges.shard_matrices(ks, world)  # every rank derives the same split
    with pytest.raises(ValueError):
        ranges.shard_matrices([3, 4], 2, costs=[1.0])


def _batch_worker(rank, world, port, results):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import oracle
        from paper_2502_16577_gb300 import ranges

        mats = syn.boson_submatrices(30, 31, 3, 10, 32)
        mine = ranges.shard_matrices([m.shape[0] for m in mats], world)[rank]
        vals = [oracle.perm_dp_c128(mats[i]) for i in mine]  # stands in for this rank's batched plan
        res = ranges.gather_results(dist, mine, vals, len(mats))
        if rank == 0:
            results.extend(res)
    finally:
        dist.destroy_process_group()


def test_two_ranks_share_a_batch(oracle):
    ctx = mp.get_context("spawn")
    with ctx.Manager() as m:
        results = m.list()
        procs = [ctx.Process(target=_batch_worker, args=(r, 2, _free_port_cache[0], results)) for r in range(2)]
        for p in procs:
            p.start()
        for p in procs:
            p.join(120)
            assert p.exitcode == 0
        got = list(results)
    mats = syn.boson_submatrices(30, 31, 3, 10, 32)
    assert got == [oracle.perm_dp_c128(x) for x in mats]


def _real_batch_worker(rank, world, port, results):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import oracle
        from paper_2502_16577_gb300 import ranges

        mats = [syn.signed_real(k, 40 + k) for k in (5, 9)]  # two matrices, three ranks
        mine = ranges.shard_matrices([m.shape[0] for m in mats], world)[rank]
        vals = [oracle.perm_dp_f64(mats[i]) for i in mine]  # stands in for this rank's real batched plan
        res = ranges.gather_results(dist, mine, vals, len(mats))
        results.append((rank, len(mine), res))
    finally:
        dist.destroy_process_group()


def test_real_results_and_an_empty_shard(oracle):
    """More ranks than matrices: one rank holds no matrix; real values come
    back as floats in batch order on every rank."""
    ctx = mp.get_context("spawn")
    port = _free_port_cache[0]
    with ctx.Manager() as m:
        results = m.list()
        procs = [ctx.Process(target=_real_batch_worker, args=(r, 3, port, results)) for r in range(3)]
        for p in procs:
            p.start()
        for p in procs:
            p.join(120)
            assert p.exitcode == 0
        got = list(results)
    mats = [syn.signed_real(k, 40 + k) for k in (5, 9)]
    want = [oracle.perm_dp_f64(x) for x in mats]
    assert sorted(n for _, n, _ in got) == [0, 1, 1]
    for _, _, res in got:
        assert res == want and all(isinstance(v, float) for v in res)


def _gpu_batch_worker(rank, world, port, results):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import torch

        import paper_2502_16577_gb300 as pg
        from paper_2502_16577_gb300 import ranges

        mats = syn.boson_submatrices(40, 33, 3, 16, 24)  # 24 modes: repeated rows are common
        mine = ranges.shard_matrices([m.shape[0] for m in mats], world)[rank]
        plan = pg.BatchPlan([mats[i] for i in mine], device=torch.device("cuda", 0), row_labels="auto")
        vals = list(plan.run())
        plan.close()
        res = ranges.gather_results(dist, mine, vals, len(mats))
        if rank == 0:
            results.extend(res)
    finally:
        dist.destroy_process_group()


@pytest.mark.gpu
def test_two_ranks_batched_plans_on_one_gpu(oracle):
    """Two gloo ranks on one GPU, each running the batched plan (rows labelled
    by equality) on its share of the batch; the gathered results match the
    oracle.  The ranks' launches are independent: nothing waits on the other."""
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2502_16577_gb300 import build

    build.build()
    ctx = mp.get_context("spawn")
    port = _free_port_cache[0]
    with ctx.Manager() as m:
        results = m.list()
        procs = [ctx.Process(target=_gpu_batch_worker, args=(r, 2, port, results)) for r in range(2)]
        for p in procs:
            p.start()
        for p in procs:
            p.join(300)
            assert p.exitcode == 0
        got = list(results)
    mats = syn.boson_submatrices(40, 33, 3, 16, 24)
    for x, g in zip(mats, got):
        assert abs(g - oracle.perm_dp_c128(x)) <= 1e-10 * oracle.perm_dp_f64(np.abs(x))

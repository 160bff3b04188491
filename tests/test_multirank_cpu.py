"""Multi-rank host logic with world size 2 over gloo on CPU: the LPT split covers every signal
exactly once with balanced work, and recovering each shard separately (here with the oracle, the
CPU stand-in for a rank's GPU) and gathering on rank 0 equals recovering the whole batch."""
import os
import socket

import numpy as np
import torch.multiprocessing as mp

from paper_1711_11407_gb300 import shard as SH
from paper_1711_11407_gb300 import synth as S


def test_lpt_partition_covers_every_signal_once_and_balances():
    wl = S.make_workload("uneven_2d", batch=64, T=4)
    for world in (1, 2, 3, 8):
        parts = SH.lpt_partition(SH.estimated_work(wl.dims), world)
        allidx = np.sort(np.concatenate(parts))
        assert np.array_equal(allidx, np.arange(wl.batch))
        w = SH.estimated_work(wl.dims)
        loads = [w[p].sum() for p in parts]
        assert max(loads) - min(loads) <= w.max() + 1e-9


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _rank_main(rank, world, port, q):
    import torch.distributed as dist
    from oracle import fpssft_oracle as O
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    wl = S.make_workload("uneven_2d", batch=10, shapes=[(16, 16), (12, 18), (8, 24)], K=lambda N: 6, T=8)
    mine = SH.shard(wl.dims, world, rank)
    res = []
    for b in mine:
        r = O.recover(wl.cube(b), wl.alpha[b], wl.tau[b], O.Params(T=8, k_cap=32))
        res.append((r.k, r.a, r.iters))
    merged = SH.gather_results(res, mine, world, rank)
    if rank == 0:
        ok = sorted(merged) == list(range(wl.batch))
        for b in range(wl.batch):
            r = O.recover(wl.cube(b), wl.alpha[b], wl.tau[b], O.Params(T=8, k_cap=32))
            k, a, it = merged[b]
            ok = ok and np.array_equal(k, r.k) and np.allclose(a, r.a) and it == r.iters
        q.put(ok)
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_shard_and_gather_equal_the_whole_batch():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
    assert all(p.exitcode == 0 for p in procs), [p.exitcode for p in procs]
    assert q.get(timeout=5) is True


def _bench_rank_main(rank, world, port, q):
    import torch.distributed as dist
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    # rank r's timed region took 10 * (r + 1) ms over 5 steps; every rank processed 4096 signals
    total = bench.max_over_ranks(10.0 * (rank + 1), world, "cpu")
    q.put((rank, total, bench.job_rate(4096, world, total / 5)))
    dist.barrier()
    dist.destroy_process_group()


def test_benchmark_takes_the_slowest_rank_and_counts_every_rank_s_signals():
    """The benchmark's cross-rank reduction on two gloo ranks: both ranks see the slowest rank's
    time, and the job's rate counts the signals of both ranks over that time."""
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    if root not in sys.path:
        sys.path.insert(0, root)
    import bench
    assert bench.max_over_ranks(3.5, 1, "cpu") == 3.5
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_bench_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
    assert all(p.exitcode == 0 for p in procs), [p.exitcode for p in procs]
    got = sorted(q.get(timeout=5) for _ in range(2))
    for rank, total, rate in got:
        assert total == 20.0
        assert abs(rate - 2 * 4096 / (4.0 / 1000.0)) < 1e-6

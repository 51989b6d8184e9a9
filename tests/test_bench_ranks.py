"""The benchmark's multi-rank bookkeeping, on CPU: with --gpus N every rank
runs its own replica and the job's time is the slowest rank's.  Two gloo
ranks (world size 2, rendezvous on 127.0.0.1) must agree on that time and on
the whole-job rate computed from it."""
import multiprocessing as mp
import os
import socket

import pytest


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    import torch.distributed as dist

    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    t_ms = bench.max_over_ranks(10.0 + 5.0 * rank, dist, device="cpu")   # rank 1 is the slow one
    rate = bench.job_rate(world, 1000, 4, t_ms / 1e3)
    dist.barrier()
    dist.destroy_process_group()
    q.put((rank, t_ms, rate))


def test_two_gloo_ranks_agree_on_the_slowest_time():
    pytest.importorskip("torch")
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=180) for _ in procs)
    for p in procs:
        p.join(timeout=60)
    assert all(p.exitcode == 0 for p in procs)
    assert [r[1] for r in res] == [15.0, 15.0]
    assert [r[2] for r in res] == [2 * 1000 * 4 / 0.015] * 2


def test_single_rank_needs_no_group():
    import bench
    assert bench.max_over_ranks(7.5) == 7.5
    assert bench.job_rate(1, 100, 3, 0.5) == 600.0

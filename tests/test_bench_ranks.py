"""The benchmark's host-side logic, on CPU.  Multi-rank bookkeeping: with
--gpus N every rank runs its own replica and the job's time is the slowest
rank's; two gloo ranks (world size 2, rendezvous on 127.0.0.1) must agree on
that time and on the whole-job rate computed from it.  Also the roofline's
per-frame counts and the bounded oracle baseline."""
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


def test_roofline_arithmetic_of_the_headline_workload():
    """The per-frame algorithmic counts the benchmark's roofline divides by,
    for runup_16m (Nf 4096, L 2049, z = 4, 513 band bins, 2049 output bins):
    forward 5 Nf log2 Nf + 4 L + 20 nb, inverse 2.5 z Nf log2 Nf + 8 z L;
    T written once by the forward and read once by the inverse."""
    import bench
    from paper_2003_07065_gb300 import workloads as W
    w = W.RUNUP_16M
    fl, by = bench.flops_per_frame(w), bench.bytes_per_frame(w)
    assert fl["forward"] == 5 * 4096 * 12 + 4 * 2049 + 20 * 513 == 264216
    assert fl["inverse"] == 2.5 * 4 * 4096 * 12 + 8 * 4 * 2049 == 557088
    assert by["forward"] == 4 * 32 + 8 * 2049 and by["inverse"] == 8 * 2049 + 4 * 32
    F = -(-w.n // w.hop)
    assert F == 524288 and by["inverse"] * F == 8661237760


def test_oracle_baseline_sample_is_bounded():
    """The CPU baseline times the oracle on a bounded prefix of the workload
    (whole path: STFTs, IF, reassignment, inverse) and reports samples/s."""
    import bench
    from paper_2003_07065_gb300 import workloads as W
    v, threads, sample, el = bench.oracle_sample_rate(W.RUNUP_16M, budget_s=0.0, n_max=1 << 12)
    assert v > 0 and threads >= 1 and "first 4096 samples of runup_16m" in sample


def test_roofline_traffic_only_from_a_capture_of_the_current_sources(tmp_path, monkeypatch):
    """roofline.traffic comes from the committed ncu capture only while the
    kernel sources hash as they did when it was taken; otherwise it is null
    and its note says why, with the capture's figure."""
    import hashlib
    import json
    import shutil

    import bench
    csrc = tmp_path / "paper_2003_07065_gb300" / "csrc"
    csrc.mkdir(parents=True)
    (tmp_path / "profiles").mkdir()
    (csrc / "k.cuh").write_text("kernel v1\n")
    rec = {"kernel_sources": ["k.cuh"], "dram_bytes_per_frame": {"inverse": 16622.5},
           "kernel_source_sha256": hashlib.sha256(b"kernel v1\n").hexdigest()}
    (tmp_path / "profiles" / "dram_traffic_runup.json").write_text(json.dumps(rec))
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    bpf, note = bench.measured_traffic_per_frame("inverse")
    assert bpf == 16622.5 and "scaled by frames" in note
    (csrc / "k.cuh").write_text("kernel v2\n")
    bpf, note = bench.measured_traffic_per_frame("inverse")
    assert bpf is None and note.startswith("null") and "16622" in note
    shutil.rmtree(tmp_path / "profiles")
    assert bench.measured_traffic_per_frame("inverse")[0] is None

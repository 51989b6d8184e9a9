"""One signal split by frame ranges, on the CPU.

* The oracle's split mode (each part's frames read from its own samples with
  the M-sample halo, one max-reduction for the relative threshold, the
  overlap-add numerator shares moved to the parts whose samples they cover)
  against the unsplit oracle: in one process for 1-4 parts, and on two gloo
  ranks (world size 2, rendezvous on 127.0.0.1) with torch.distributed doing
  the all-reduce and the point-to-point exchange.
* The product's exchange lists (paper_2003_07065_gb300.partition): every tile
  a part's output needs arrives exactly once, from the part that computed it;
  and its DistComm moving workspace segments and the maximum between two
  gloo ranks."""
import multiprocessing as mp
import os
import socket

import numpy as np
import pytest

import oracle as O
from paper_2003_07065_gb300 import partition as PT

P = dict(fs=8000.0, L=257, sigma=32.0, hop=8, nfft=256, f_lo=300.0, f_hi=2500.0, z=2, gamma=1e-3)
N = 9001


def signal():
    t = np.arange(N) / P["fs"]
    x = np.cos(2 * np.pi * (600 * t + 300 * t * t)) + 0.4 * np.cos(2 * np.pi * 1900 * t)
    return x + 0.2 * np.random.default_rng(5).standard_normal(N)


def unsplit(x, relative=True):
    return O.sst(x, P["fs"], P["L"], P["sigma"], P["hop"], P["nfft"], P["f_lo"], P["f_hi"], P["z"], P["gamma"],
                 relative, inverse_range=(0, N)).xhat


def part_job(x, parts, r, allreduce_max, exchange, relative=True, align=4):
    """Part r of `parts`: its input samples, its max, the reduced threshold,
    its numerator, the exchange and its output samples."""
    F = O.frames(N, P["hop"])
    ranges = O.frame_ranges(F, parts, align)
    m_b, m_e = ranges[r]
    x_b, x_e = O.part_input_range(m_b, m_e, P["hop"], P["L"], N)
    x_part = x[x_b:x_e]                                  # all this part reads
    k_lo, k_hi = O.band_bins(P["fs"], P["nfft"], P["f_lo"], P["f_hi"])
    if relative:
        vmax = allreduce_max(O.part_max_abs_v(x_part, x_b, N, P["L"], P["sigma"], P["hop"], P["nfft"], k_lo, k_hi,
                                              m_b, m_e))
        gam = P["gamma"] * vmax
    else:
        gam = P["gamma"]
    num, q_b, _ = O.part_numerator(x_part, x_b, N, P["L"], P["sigma"], P["hop"], P["nfft"], k_lo, k_hi, P["z"], gam,
                                   m_b, m_e)
    outs = [O.part_output_range(b, e, P["hop"], N, i == parts - 1) for i, (b, e) in enumerate(ranges)]
    received = exchange(r, (num, q_b), outs)             # shares of every part touching my samples, by part
    p_b, p_e = outs[r]
    return p_b, O.part_finalise(received, p_b, p_e, P["L"], P["sigma"], P["hop"], N)


# a window longer than zNf (halo M = 512 samples, the inverse's transform read
# periodically), for the split mode's long-window case
P_LONG = dict(fs=8000.0, L=1025, sigma=200.0, hop=16, nfft=128, f_lo=300.0, f_hi=2500.0, z=3, gamma=1e-3)


@pytest.mark.parametrize("parts", [1, 2, 3, 4])
@pytest.mark.parametrize("relative", [True, False])
@pytest.mark.parametrize("long_window", [False, True])
def test_oracle_split_equals_unsplit(parts, relative, long_window):
    """In one process: every part's maximum first, then every part's
    numerator under the reduced threshold, then each part's samples from the
    shares of all parts (ascending)."""
    P = P_LONG if long_window else globals()["P"]
    x = signal()
    ref = O.sst(x, P["fs"], P["L"], P["sigma"], P["hop"], P["nfft"], P["f_lo"], P["f_hi"], P["z"], P["gamma"],
                relative, inverse_range=(0, N)).xhat
    maxes = [0.0] * parts
    shares = [None] * parts
    F = O.frames(N, P["hop"])
    ranges = O.frame_ranges(F, parts, 4)
    k_lo, k_hi = O.band_bins(P["fs"], P["nfft"], P["f_lo"], P["f_hi"])
    for r, (m_b, m_e) in enumerate(ranges):
        x_b, x_e = O.part_input_range(m_b, m_e, P["hop"], P["L"], N)
        maxes[r] = O.part_max_abs_v(x[x_b:x_e], x_b, N, P["L"], P["sigma"], P["hop"], P["nfft"], k_lo, k_hi, m_b, m_e)
    gam = P["gamma"] * max(maxes) if relative else P["gamma"]
    for r, (m_b, m_e) in enumerate(ranges):
        x_b, x_e = O.part_input_range(m_b, m_e, P["hop"], P["L"], N)
        num, q_b, _ = O.part_numerator(x[x_b:x_e], x_b, N, P["L"], P["sigma"], P["hop"], P["nfft"], k_lo, k_hi, P["z"],
                                       gam, m_b, m_e)
        shares[r] = (num, q_b)
    outs = [O.part_output_range(b, e, P["hop"], N, i == parts - 1) for i, (b, e) in enumerate(ranges)]
    assert sum(e - b for b, e in outs) == N
    out = np.empty(N)
    for p_b, p_e in outs:
        out[p_b:p_e] = O.part_finalise(shares, p_b, p_e, P["L"], P["sigma"], P["hop"], N)
    np.testing.assert_allclose(out, ref, rtol=0, atol=1e-12 * np.abs(ref).max())


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _oracle_rank(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    import torch
    import torch.distributed as dist
    dist.init_process_group("gloo", rank=rank, world_size=world)
    x = signal()

    def allreduce_max(v):
        t = torch.tensor([v], dtype=torch.float64)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        return float(t.item())

    def exchange(me, mine, outs):
        # my numerator on each other part's output samples goes to that part;
        # its numerator on mine comes back (a header with the sample range first)
        num, q_b = mine
        inbox = {me: (num, q_b)}
        for peer, (p_b, p_e) in enumerate(outs):
            if peer == me:
                continue
            lo, hi = max(p_b, q_b), min(p_e, q_b + len(num))
            hdr = torch.tensor([lo, max(hi, lo)], dtype=torch.int64)
            other = torch.empty(2, dtype=torch.int64)
            if me < peer:
                dist.send(hdr, peer)
                dist.recv(other, peer)
            else:
                dist.recv(other, peer)
                dist.send(hdr, peer)
            ops = []
            if hi > lo:
                ops.append(dist.isend(torch.from_numpy(np.ascontiguousarray(num[lo - q_b:hi - q_b])), peer))
            o_lo, o_hi = int(other[0]), int(other[1])
            if o_hi > o_lo:
                buf = torch.empty(o_hi - o_lo, dtype=torch.float64)
                ops.append(dist.irecv(buf, peer))
                inbox[peer] = (buf, o_lo)
            for op in ops:
                op.wait()
        return [(np.asarray(inbox[p][0]), inbox[p][1]) for p in sorted(inbox)]

    p_b, xh = part_job(x, world, rank, allreduce_max, exchange)
    dist.barrier()
    dist.destroy_process_group()
    q.put((rank, p_b, xh))


def test_oracle_split_on_two_gloo_ranks():
    pytest.importorskip("torch")
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_oracle_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted((q.get(timeout=300) for _ in procs), key=lambda t: t[0])
    for p in procs:
        p.join(timeout=60)
    assert all(p.exitcode == 0 for p in procs)
    out = np.concatenate([xh for _, _, xh in res])
    assert res[1][1] == len(res[0][2]) and len(out) == N
    ref = unsplit(signal())
    np.testing.assert_allclose(out, ref, rtol=0, atol=1e-12 * np.abs(ref).max())


def synthetic_layouts(ntiles, parts, B, hop, L, n):
    """Layouts with the C library's rules (sst_part_layout) for given B."""
    M = (L - 1) // 2
    F = -(-n // hop)
    seg_len = (B - 1) * hop + L
    BH = B * hop
    out = []
    for p in range(parts):
        tb, te = ntiles * p // parts, ntiles * (p + 1) // parts
        fb, fe = min(F, tb * B), min(F, te * B)
        ob = 0 if p == 0 else min(n, fb * hop)
        oe = n if p == parts - 1 else min(n, fe * hop)
        if oe > ob:
            num = ob + M - seg_len + 1
            nb_ = 0 if num <= 0 else -(-num // BH)
            ne = min(ntiles, (oe - 1 + M) // BH + 1)
        else:
            nb_ = ne = tb
        out.append(dict(tile_begin=tb, tile_end=te, need_begin=nb_, need_end=ne, out_begin=ob, out_end=oe))
    return out


@pytest.mark.parametrize("parts", [1, 2, 3, 7])
@pytest.mark.parametrize("B,hop,L", [(64, 32, 2049), (2, 8, 257), (6, 16, 1025), (2, 16, 8193)])
def test_exchange_lists_deliver_every_needed_tile_once(parts, B, hop, L):
    n = 300000
    F = -(-n // hop)
    ntiles = -(-F // B)
    lays = synthetic_layouts(ntiles, parts, B, hop, L, n)
    for me in range(parts):
        sends, recvs = PT.exchange_lists(lays, me)
        got = {}
        for q, a, b in recvs:
            assert q != me
            for t in range(a, b):
                assert t not in got
                got[t] = q
                assert lays[q]["tile_begin"] <= t < lays[q]["tile_end"]
        mine = set(range(lays[me]["tile_begin"], lays[me]["tile_end"]))
        need = set(range(lays[me]["need_begin"], lays[me]["need_end"]))
        assert set(got) == need - mine
        # what I send to q is what q receives from me
        for q, a, b in sends:
            _, r2 = PT.exchange_lists(lays, q)
            assert (me, a, b) in r2


def _comm_rank(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    import torch
    import torch.distributed as dist
    dist.init_process_group("gloo", rank=rank, world_size=world)
    comm = PT.DistComm(dist)
    B, hop, L, n = 4, 8, 129, 4000
    F = -(-n // hop)
    ntiles = -(-F // B)
    seg_len = (B - 1) * hop + L
    lays = synthetic_layouts(ntiles, world, B, hop, L, n)
    ws = torch.zeros(256 + 4 * seg_len * ntiles, dtype=torch.uint8)
    mine = lays[rank]
    seg = PT.segments(ws, 256, seg_len, mine["tile_begin"], mine["tile_end"])
    seg.copy_(torch.arange(seg.numel(), dtype=torch.float32) + 1000.0 * (rank + 1))
    sends, recvs = PT.exchange_lists(lays, rank)
    comm.exchange([(p, PT.segments(ws, 256, seg_len, a, b)) for p, a, b in sends],
                  [(p, PT.segments(ws, 256, seg_len, a, b)) for p, a, b in recvs])
    r = torch.tensor([float(rank) + 0.5])
    comm.allreduce_max(r)
    ok = True
    for p, a, b in recvs:
        got = PT.segments(ws, 256, seg_len, a, b)
        base = (a - lays[p]["tile_begin"]) * seg_len
        want = torch.arange(base, base + got.numel(), dtype=torch.float32) + 1000.0 * (p + 1)
        ok = ok and torch.equal(got, want)
    dist.barrier()
    dist.destroy_process_group()
    q.put((rank, ok, len(recvs), float(r.item())))


def test_dist_comm_moves_segments_between_two_gloo_ranks():
    pytest.importorskip("torch")
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_comm_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=180) for _ in procs)
    for p in procs:
        p.join(timeout=60)
    assert all(p.exitcode == 0 for p in procs)
    for rank, ok, nrecv, rmax in res:
        assert ok and nrecv == 1 and rmax == 1.5

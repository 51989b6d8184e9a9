"""One signal split by frame ranges (sst_part_* and
paper_2003_07065_gb300.partition.run), its parts run on one GPU by host
threads, one plan and workspace per part, with a communicator that reduces
the maximum and moves the boundary segments between the parts' workspaces on
the device.  The parts' outputs, concatenated, must carry the same bits as
the unsplit forward + inverse without a TFR output: the same pre-pass values
(whole groups of four frames), the same threshold, the same tiles and the
same tile-ordered sums at every sample.  No kernel waits on another: the
threads meet only on the host, between launches."""
import threading

import numpy as np
import pytest

from paper_2003_07065_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def sst():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2003_07065_gb300 import build, sst as S
    build.build()
    S.load()
    return S


class ThreadComm:
    """The partition communicator for parts run by threads on one device
    (all on the default stream, so launches follow the host's order)."""

    def __init__(self, parts):
        self.parts = parts
        self.barrier = threading.Barrier(parts)
        self.slots = [None] * parts
        self.posted = {}
        self.lock = threading.Lock()

    def for_rank(self, rank):
        comm = self

        class Rank:
            def allreduce_max(self, t):
                comm.slots[rank] = t
                comm.barrier.wait()
                m = torch.stack([s.reshape(-1)[0] for s in comm.slots]).max()
                comm.barrier.wait()
                t.fill_(m)
                comm.barrier.wait()

            def exchange(self, sends, recvs):
                with comm.lock:
                    for peer, t in sends:
                        comm.posted[(rank, peer)] = t
                comm.barrier.wait()
                for peer, t in recvs:
                    t.copy_(comm.posted[(peer, rank)])
                comm.barrier.wait()
                with comm.lock:
                    for peer, _ in sends:
                        comm.posted.pop((rank, peer), None)
                comm.barrier.wait()
        return Rank()


def run_split(S, params, x32, parts):
    from paper_2003_07065_gb300 import partition as PT
    plans = [S.Plan(**params) for _ in range(parts)]
    lays = PT.layouts(plans[0], parts)
    comm = ThreadComm(parts)
    outs, errs = [None] * parts, []

    def work(r):
        try:
            lay = lays[r]
            xp = torch.from_numpy(np.ascontiguousarray(x32[lay["x_begin"]:lay["x_end"]])).cuda()
            outs[r] = PT.run(plans[r], xp, r, parts, comm.for_rank(r), lays)
        except Exception as e:   # surfaced below; a failed part must not leave the others waiting
            errs.append(e)
            comm.barrier.abort()

    threads = [threading.Thread(target=work, args=(r,)) for r in range(parts)]
    for t in threads:
        t.start()
    for t in threads:
        t.join()
    torch.cuda.synchronize()
    if errs:
        raise errs[0]
    for p in plans:
        p.close()
    assert sum(lay["out_end"] - lay["out_begin"] for lay in lays) == params["n"]
    assert all(lays[i]["out_end"] == lays[i + 1]["out_begin"] for i in range(parts - 1))
    return torch.cat([o for o in outs if o.numel()]), lays


def unsplit(S, params, x32):
    # the split path takes the exact max |S^g| from its pre-pass (all-reduced
    # over the parts), as a two-pass plan does
    plan = S.Plan(**params, two_pass=True)
    out = plan.reconstruct(torch.from_numpy(x32).cuda())
    torch.cuda.synchronize()
    plan.close()
    return out


@pytest.mark.parametrize("name,parts", [("runup_256k", 2), ("runup_256k", 3), ("runup_256k", 5),
                                        ("chirp_fm_64k", 2), ("chirp_fm_64k", 4)])
def test_split_equals_unsplit(sst, name, parts):
    w = W.ALL[name]
    x32 = w.signal()[0].astype(np.float32)
    got, lays = run_split(sst, w.params(), x32, parts)
    ref = unsplit(sst, w.params(), x32)
    assert torch.equal(got, ref), (got - ref).abs().max().item()
    # each part read only its own samples plus the halo
    assert all(lay["x_end"] - lay["x_begin"] < w.n for lay in lays) or parts == 1


def test_split_absolute_threshold_and_more_parts_than_tiles(sst):
    p = dict(n=3001, fs=2000.0, L=257, sigma=32.0, hop=7, nfft=256, f_lo=700.0, f_hi=1000.0, z=4, gamma=0.5,
             relative=False)
    t = np.arange(p["n"]) / p["fs"]
    x32 = (np.cos(2 * np.pi * 850 * t) + 0.3 * np.random.default_rng(3).standard_normal(p["n"])).astype(np.float32)
    ref = unsplit(sst, p, x32)
    for parts in (2, 7):
        got, lays = run_split(sst, p, x32, parts)
        assert torch.equal(got, ref), parts
    # 40 samples: 6 frames in 3 tiles of two, over 7 parts (four of them empty)
    q = dict(p, n=40, relative=True, gamma=1e-3)
    x40 = np.ascontiguousarray(x32[:40])
    got, lays = run_split(sst, q, x40, 7)
    assert sum(1 for lay in lays if lay["tile_end"] == lay["tile_begin"]) == 4
    assert torch.equal(got, unsplit(sst, q, x40))


def sweep_shapes():
    from test_gpu_sweep import SHAPES, signal
    return [(i, SHAPES[i], signal) for i in range(0, len(SHAPES), 4)]


@pytest.mark.parametrize("case", sweep_shapes(), ids=lambda c: f"shape{c[0]}_nf{c[1]['nfft']}_z{c[1]['z']}")
def test_split_sweep_shapes(sst, case):
    """Every fourth shape of the plan-shape sweep, split in two and three:
    the same bits as unsplit (where the plan's fused kernel fits)."""
    i, p, signal = case
    x32 = signal(p, 100 + i)
    try:
        ref = unsplit(sst, p, x32)
    except sst.SstError as e:
        assert e.status == 6
        pytest.skip("fused kernel does not fit this plan")
    for parts in (2, 3):
        got, _ = run_split(sst, p, x32, parts)
        assert torch.equal(got, ref), (parts, (got - ref).abs().max().item())

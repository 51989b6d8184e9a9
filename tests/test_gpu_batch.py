"""Batched execution (many channels, uneven lengths, mixed hop / Nf / band /
z / window class / threshold kind) through sst_batch_*: every channel's TFR
and reconstruction must be bit-identical to the single-plan call on the same
input (same arithmetic, deterministic sums; relative thresholds from the
separate max|V| pre-pass, i.e. plans made with SST_TWO_PASS), with and
without the captured CUDA graph and after autotuning; every channel is also
checked against the FP64 oracle under the parity bars."""
import numpy as np
import pytest

import oracle as O

from parity import as_complex, compare, gpu_map

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

CHANNELS = [
    dict(n=3000, fs=8000.0, L=257, sigma=32.0, hop=8, nfft=256, f_lo=500.0, f_hi=2500.0, z=2, gamma=1e-3, relative=True),
    dict(n=20011, fs=8000.0, L=513, sigma=64.0, hop=16, nfft=512, f_lo=0.0, f_hi=4000.0, z=1, gamma=1e-3, relative=True),
    dict(n=777, fs=8000.0, L=129, sigma=16.0, hop=4, nfft=256, f_lo=1000.0, f_hi=1500.0, z=4, gamma=0.0, relative=False),
    dict(n=40000, fs=16000.0, L=1025, sigma=128.0, hop=32, nfft=1024, f_lo=1000.0, f_hi=5000.0, z=4, gamma=1e-3, relative=True),
    dict(n=9000, fs=16000.0, L=1025, sigma=128.0, hop=16, nfft=1024, f_lo=0.0, f_hi=8000.0, z=1, gamma=1e-3, relative=True),
    dict(n=65536, fs=25600.0, L=2049, sigma=256.0, hop=64, nfft=4096, f_lo=2000.0, f_hi=6000.0, z=2, gamma=1e-3, relative=True),
    dict(n=5000, fs=16000.0, L=1025, sigma=128.0, hop=8, nfft=2048, f_lo=3000.0, f_hi=5000.0, z=2, gamma=0.05, relative=False),
    dict(n=30000, fs=16000.0, L=4097, sigma=512.0, hop=64, nfft=8192, f_lo=0.0, f_hi=3000.0, z=1, gamma=1e-3, relative=True),
    dict(n=1, fs=1000.0, L=65, sigma=8.0, hop=8, nfft=64, f_lo=0.0, f_hi=500.0, z=1, gamma=0.0, relative=False),
    dict(n=12345, fs=16000.0, L=257, sigma=32.0, hop=16, nfft=512, f_lo=4000.0, f_hi=8000.0, z=2, gamma=1e-3, relative=True),
]


@pytest.fixture(scope="module")
def sst():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2003_07065_gb300 import build, sst as S
    build.build()
    S.load()
    return S


def signal(p, seed):
    gen = np.random.default_rng(seed)
    t = np.arange(p["n"]) / p["fs"]
    f0, f1 = p["f_lo"] + 0.2 * (p["f_hi"] - p["f_lo"]), p["f_lo"] + 0.8 * (p["f_hi"] - p["f_lo"])
    dur = max(p["n"] / p["fs"], 1e-9)
    x = np.cos(2 * np.pi * (f0 * t + 0.5 * (f1 - f0) / dur * t * t)) + 0.2 * gen.standard_normal(p["n"])
    return x.astype(np.float32)


def setup(S):
    plans, xs, refs = [], [], []
    for i, p in enumerate(CHANNELS):
        pl = S.Plan(**p, two_pass=True)     # the batch's relative thresholds are two-pass
        x = torch.from_numpy(signal(p, i)).cuda()
        t, xh = pl.forward_inverse(x)
        plans.append(pl)
        xs.append(x)
        refs.append((t.clone(), xh.clone()))
    torch.cuda.synchronize()
    return plans, xs, refs


def run_batch(S, plans, xs, graph, tune=False, reps=2):
    outs = [(pl.new_tfr().fill_(float("nan")), torch.full((pl.n,), float("nan"), device="cuda"))
            for pl in plans]
    items = [(pl.handle, x, pl.n, t, xh) for pl, x, (t, xh) in zip(plans, xs, outs)]
    b = S.sst_batch_create(items, graph=graph)
    ws = torch.empty(max(S.sst_batch_workspace(b), 256), dtype=torch.uint8, device="cuda")
    times = None
    if tune:
        times = S.sst_batch_tune(b, ws)
    for _ in range(reps):
        S.sst_batch_run(b, ws)
    torch.cuda.synchronize()
    knobs = S.sst_batch_knobs(b)
    S.sst_batch_destroy(b)
    return outs, times, knobs


@pytest.mark.parametrize("graph", [False, True])
def test_batch_bit_identical_to_single_plan(sst, graph):
    plans, xs, refs = setup(sst)
    outs, _, _ = run_batch(sst, plans, xs, graph)
    for i, ((t, xh), (tr, xr)) in enumerate(zip(outs, refs)):
        assert torch.equal(t, tr), f"channel {i}: TFR differs"
        assert torch.equal(xh, xr), f"channel {i}: reconstruction differs"
    for pl in plans:
        pl.close()


def test_batch_tuned_still_identical(sst):
    plans, xs, refs = setup(sst)
    outs, times, knobs = run_batch(sst, plans, xs, graph=True, tune=True)
    assert times[0] > 0 and times[1] > 0 and times[1] <= times[0] * 1.0001
    for i, ((t, xh), (tr, xr)) in enumerate(zip(outs, refs)):
        assert torch.equal(t, tr), f"channel {i}: TFR differs after tuning ({knobs})"
        assert torch.equal(xh, xr), f"channel {i}: reconstruction differs after tuning"
    for pl in plans:
        pl.close()


def test_batch_channels_match_oracle(sst):
    """Every channel against the FP64 oracle under the bars of tests/parity.py
    (map, T in replay mode, mass, the inverse alone and end to end).  The
    batch's decisions are those of the channel's single two-pass plan, whose
    map and STFT come from sst_reassign_map / sst_stft."""
    plans, xs, _ = setup(sst)
    outs, _, _ = run_batch(sst, plans, xs, graph=True)
    for i, p in enumerate(CHANNELS):
        x = xs[i].cpu().numpy().astype(np.float64)
        r = O.sst(x, p["fs"], p["L"], p["sigma"], p["hop"], p["nfft"], p["f_lo"], p["f_hi"], p["z"],
                  p["gamma"], p["relative"], inverse_range=(0, p["n"]))
        g = gpu_map(sst, p, xs[i], two_pass=True)
        g.update(T=as_complex(outs[i][0].cpu().numpy()), xhat=outs[i][1].cpu().numpy())
        print(i, compare(g, r, p))
    for pl in plans:
        pl.close()


def test_batch_submit_one_shot(sst):
    plans, xs, refs = setup(sst)
    outs = [(pl.new_tfr(), torch.empty(pl.n, device="cuda")) for pl in plans]
    items = [(pl.handle, x, pl.n, t, xh) for pl, x, (t, xh) in zip(plans, xs, outs)]
    nbytes = sst.sst_batch_workspace_for(items)
    ws = torch.empty(nbytes, dtype=torch.uint8, device="cuda")
    sst.sst_batch_submit(items, ws, nbytes)
    for (t, xh), (tr, xr) in zip(outs, refs):
        assert torch.equal(t, tr) and torch.equal(xh, xr)
    with pytest.raises(sst.SstError):
        sst.sst_batch_submit(items, ws, nbytes - 256)
    for pl in plans:
        pl.close()


def test_batch_of_the_sweep_shapes(sst):
    """The 32 plan shapes of the plan-shape sweep in one batch (a mix of
    Nf 128 .. 2048, z 1 .. 4, quarter, half and folded windows, absolute and
    relative thresholds): every channel carries the same bits as its
    single-plan call."""
    from test_gpu_sweep import SHAPES, signal as sweep_signal
    plans, xs, refs = [], [], []
    for i, p in enumerate(SHAPES):
        pl = sst.Plan(**p, two_pass=True)
        x = torch.from_numpy(sweep_signal(p, 100 + i)).cuda()
        t, xh = pl.forward_inverse(x)
        plans.append(pl)
        xs.append(x)
        refs.append((t.clone(), xh.clone()))
    torch.cuda.synchronize()
    outs, _, _ = run_batch(sst, plans, xs, graph=False)
    for i, ((t, xh), (tr, xr)) in enumerate(zip(outs, refs)):
        assert torch.equal(t, tr), f"shape {i}: TFR differs"
        assert torch.equal(xh, xr), f"shape {i}: reconstruction differs"
    for pl in plans:
        pl.close()

"""The plan's extreme parameters: the largest subdivision factor z = 16 (and
8, and an odd 7) with half-length, folded and long windows, and the largest
Nf, 8192, with the longest window.  Each through the path with a TFR output
against the FP64 oracle (every parity bar) and the path without one (bit for
bit for a two-pass plan, within the reconstruction bar for a one-pass one)."""
import numpy as np
import pytest

import oracle as O

from parity import as_complex, compare, gpu_map

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

XHAT_RTOL = 2e-5

SHAPES = [
    # z = 16, half-length window (9 taps per thread), a pruned band of Nf 1024
    dict(n=20000, fs=8000.0, L=513, sigma=64.0, hop=16, nfft=1024, f_lo=500.0, f_hi=1500.0, z=16, gamma=1e-3,
         relative=True),
    # z = 16, folded Nf + 1 window, the whole band (DC and Nyquist)
    dict(n=9001, fs=8000.0, L=257, sigma=32.0, hop=8, nfft=256, f_lo=0.0, f_hi=4000.0, z=16, gamma=0.05,
         relative=False),
    # z = 16 with a window four times Nf
    dict(n=6000, fs=8000.0, L=257, sigma=40.0, hop=8, nfft=64, f_lo=0.0, f_hi=4000.0, z=16, gamma=1e-3,
         relative=True),
    # z = 8 on the bench's Nf and window (class 1 band)
    dict(n=30000, fs=51200.0, L=2049, sigma=256.0, hop=32, nfft=4096, f_lo=0.0, f_hi=6400.0, z=8, gamma=1e-3,
         relative=True),
    # odd z = 7 up to Nyquist
    dict(n=4001, fs=16000.0, L=257, sigma=32.0, hop=16, nfft=256, f_lo=4000.0, f_hi=8000.0, z=7, gamma=1e-3,
         relative=True),
    # the largest Nf with the longest window
    dict(n=40000, fs=16000.0, L=8193, sigma=1024.0, hop=64, nfft=8192, f_lo=0.0, f_hi=3000.0, z=2, gamma=1e-3,
         relative=True),
]
IDS = [f"nf{p['nfft']}_L{p['L']}_z{p['z']}_{'rel' if p['relative'] else 'abs'}" for p in SHAPES]


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
    dur = p["n"] / p["fs"]
    f0 = p["f_lo"] + 0.2 * (p["f_hi"] - p["f_lo"])
    f1 = p["f_lo"] + 0.8 * (p["f_hi"] - p["f_lo"])
    clean = np.cos(2 * np.pi * (f0 * t + 0.5 * (f1 - f0) / dur * t * t))
    return (clean + 0.3 * gen.standard_normal(p["n"])).astype(np.float32)


@pytest.mark.parametrize("i", range(len(SHAPES)), ids=IDS)
def test_extreme_shape(sst, i):
    p = SHAPES[i]
    x32 = signal(p, 700 + i)
    x = torch.from_numpy(x32).cuda()
    plan = sst.Plan(**p)
    tfr, xhat = plan.forward_inverse(x)
    g = gpu_map(sst, p, x)
    g.update(T=as_complex(tfr.cpu().numpy()), xhat=xhat.cpu().numpy().astype(np.float64))
    r = O.sst(x32.astype(np.float64), p["fs"], p["L"], p["sigma"], p["hop"], p["nfft"], p["f_lo"], p["f_hi"],
              p["z"], p["gamma"], p["relative"], inverse_range=(0, p["n"]))
    stats = compare(g, r, p)
    try:
        one = plan.reconstruct(x)
    except sst.SstError as e:   # the fused kernel's shared memory does not fit this plan
        assert e.status == 6
        one = None
    if one is not None:
        one2 = plan.reconstruct(x)
        torch.cuda.synchronize()
        assert torch.equal(one, one2)
        assert (one - xhat).abs().max().item() <= XHAT_RTOL * xhat.abs().max().item()
        two = sst.Plan(**p, two_pass=True)
        _, xt = two.forward_inverse(x)
        xf = two.reconstruct(x)
        torch.cuda.synchronize()
        assert torch.equal(xf, xt)
        two.close()
    plan.close()
    print(p, stats, "fused" if one is not None else "no fused kernel")

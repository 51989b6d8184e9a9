"""A seeded sweep of plan shapes through every path that forms a
reconstruction, against the FP64 oracle and against each other: Nf from 64
to 2048 (Stockham and in-place FFT forms, first radices 2, 4, 8, 16), z from 1
to 4 (z = 3 for a phase table whose size is not a power of two), windows
of a quarter, a half and a whole frame plus one (folded), bands anywhere
from DC to Nyquist, relative and absolute thresholds, odd lengths.  For each
shape: the path with a TFR output meets every parity bar (tests/parity.py);
a two-pass plan's path without a TFR output carries the same bits as its
path with one; a one-pass plan's stays within the reconstruction bar of
its path with one and repeats bit for bit."""
import numpy as np
import pytest

import oracle as O

from parity import as_complex, compare

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

XHAT_RTOL = 2e-5


@pytest.fixture(scope="module")
def sst():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2003_07065_gb300 import build, sst as S
    build.build()
    S.load()
    return S


def shapes(count=32, seed=2003):
    gen = np.random.default_rng(seed)
    out = []
    for _ in range(count):
        nf = int(gen.choice([64, 128, 256, 512, 1024, 2048]))
        L = int(gen.choice([nf // 4 + 1, nf // 2 + 1, nf + 1]))
        hop = int(max(1, nf // int(gen.choice([8, 16, 32]))))
        fs = 8000.0
        df = fs / nf
        k_lo = int(gen.integers(0, nf // 2 - 1))
        k_hi = int(gen.integers(k_lo + 1, nf // 2 + 1))
        relative = bool(gen.integers(0, 2))
        out.append(dict(n=int(gen.integers(3 * nf, 12000)), fs=fs, L=L, sigma=(L - 1) / 8.0, hop=hop, nfft=nf,
                        f_lo=k_lo * df, f_hi=k_hi * df, z=int(gen.integers(1, 5)),
                        gamma=float(gen.choice([1e-3, 1e-2])) if relative else 0.05, relative=relative))
    return out


SHAPES = shapes()


def signal(p, seed):
    gen = np.random.default_rng(seed)
    t = np.arange(p["n"]) / p["fs"]
    dur = p["n"] / p["fs"]
    f0 = p["f_lo"] + 0.2 * (p["f_hi"] - p["f_lo"])
    f1 = p["f_lo"] + 0.8 * (p["f_hi"] - p["f_lo"])
    clean = np.cos(2 * np.pi * (f0 * t + 0.5 * (f1 - f0) / dur * t * t))
    return (clean + 0.3 * gen.standard_normal(p["n"])).astype(np.float32)


@pytest.mark.parametrize("i", range(len(SHAPES)),
                         ids=[f"nf{p['nfft']}_L{p['L']}_z{p['z']}_{'rel' if p['relative'] else 'abs'}" for p in SHAPES])
def test_shape(sst, i):
    p = SHAPES[i]
    x32 = signal(p, 100 + i)
    x = torch.from_numpy(x32).cuda()
    plan = sst.Plan(**p)
    tfr, xhat = plan.forward_inverse(x)
    _, dest = plan.reassign_map(x)
    torch.cuda.synchronize()
    g = dict(T=as_complex(tfr.cpu().numpy()), dest=dest.cpu().numpy(), xhat=xhat.cpu().numpy().astype(np.float64))
    r = O.sst(x32.astype(np.float64), p["fs"], p["L"], p["sigma"], p["hop"], p["nfft"], p["f_lo"], p["f_hi"],
              p["z"], p["gamma"], p["relative"], inverse_range=(0, p["n"]))
    stats = compare(g, r, p)
    # the paths without a TFR output (where the plan's fused kernel fits)
    try:
        one = plan.reconstruct(x)
        one2 = plan.reconstruct(x)
    except sst.SstError as e:
        assert e.status == 6
        one = None
    if one is not None:
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
    print(p, stats)

"""Windows longer than Nf + 1.  The forward folds the window modulo Nf (Eq. 8
summed into Eq. 9's Nf positions, exact), and the inverse evaluates Eq. 25 at
every tap |n| <= M, which wraps the Nf-point sub-grid transforms more than
once (a window of up to 128 Nf, and longer than zNf, where Eq. 25 repeats
with period zNf).  Seeded shapes from a window just over Nf + 1 to the
longest one a plan takes, through the path with a TFR output against the
FP64 oracle (every parity bar, the STFT included), the path without one
against it (bit for bit for a two-pass plan; within the reconstruction bar
and repeatable for a one-pass one), a batch of them beside ordinary channels
against their single-plan calls bit for bit, a split signal against the
unsplit call bit for bit, and a stream against the oracle."""
import numpy as np
import pytest

import oracle as O

from parity import as_complex, compare, gpu_map

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

XHAT_RTOL = 2e-5

LONG = [
    # L = Nf + 3: one tap more on each side than a folded Nf + 1 window
    dict(n=6000, fs=8000.0, L=67, sigma=8.0, hop=4, nfft=64, f_lo=0.0, f_hi=4000.0, z=1, gamma=1e-3, relative=True),
    # four wraps, z = 2
    dict(n=9001, fs=8000.0, L=257, sigma=32.0, hop=8, nfft=64, f_lo=500.0, f_hi=2500.0, z=2, gamma=1e-3,
         relative=True),
    # 2 Nf + 1, the whole band with z = 3, absolute threshold
    dict(n=7777, fs=8000.0, L=257, sigma=40.0, hop=16, nfft=128, f_lo=0.0, f_hi=4000.0, z=3, gamma=0.05,
         relative=False),
    # 3 Nf + 1, a band up to Nyquist with z = 4
    dict(n=12000, fs=16000.0, L=769, sigma=96.0, hop=32, nfft=256, f_lo=2000.0, f_hi=8000.0, z=4, gamma=1e-3,
         relative=True),
    dict(n=20011, fs=16000.0, L=1025, sigma=128.0, hop=16, nfft=512, f_lo=0.0, f_hi=3000.0, z=2, gamma=1e-2,
         relative=True),
    dict(n=30000, fs=16000.0, L=4097, sigma=512.0, hop=64, nfft=1024, f_lo=1000.0, f_hi=5000.0, z=2, gamma=0.05,
         relative=False),
    # the longest window, at Nf 4096 (in-place FFT form) and at Nf 64 (128
    # wraps, longer than zNf = 256)
    dict(n=40000, fs=25600.0, L=8193, sigma=1024.0, hop=128, nfft=4096, f_lo=0.0, f_hi=6400.0, z=1, gamma=1e-3,
         relative=True),
    dict(n=20000, fs=8000.0, L=8193, sigma=1024.0, hop=256, nfft=64, f_lo=0.0, f_hi=4000.0, z=4, gamma=1e-3,
         relative=True),
]
IDS = [f"nf{p['nfft']}_L{p['L']}_z{p['z']}_{'rel' if p['relative'] else 'abs'}" for p in LONG]


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


@pytest.mark.parametrize("i", range(len(LONG)), ids=IDS)
def test_long_window(sst, i):
    p = LONG[i]
    x32 = signal(p, 300 + i)
    x = torch.from_numpy(x32).cuda()
    plan = sst.Plan(**p)
    tfr, xhat = plan.forward_inverse(x)
    g = gpu_map(sst, p, x)
    g.update(T=as_complex(tfr.cpu().numpy()), xhat=xhat.cpu().numpy().astype(np.float64))
    r = O.sst(x32.astype(np.float64), p["fs"], p["L"], p["sigma"], p["hop"], p["nfft"], p["f_lo"], p["f_hi"],
              p["z"], p["gamma"], p["relative"], inverse_range=(0, p["n"]))
    stats = compare(g, r, p)
    # the path without a TFR output
    one = plan.reconstruct(x)
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
    print(p, stats)


def test_long_windows_in_a_batch(sst):
    """The long-window shapes in one batch with two ordinary channels (a half
    and a folded Nf + 1 window): every channel carries the same bits as its
    single-plan call."""
    from test_gpu_batch import run_batch
    shapes = LONG + [
        dict(n=9000, fs=16000.0, L=1025, sigma=128.0, hop=16, nfft=1024, f_lo=0.0, f_hi=8000.0, z=1, gamma=1e-3,
             relative=True),
        dict(n=3000, fs=8000.0, L=129, sigma=16.0, hop=8, nfft=256, f_lo=500.0, f_hi=2500.0, z=2, gamma=1e-3,
             relative=True),
    ]
    plans, xs, refs = [], [], []
    for i, p in enumerate(shapes):
        pl = sst.Plan(**p, two_pass=True)
        x = torch.from_numpy(signal(p, 500 + i)).cuda()
        t, xh = pl.forward_inverse(x)
        plans.append(pl)
        xs.append(x)
        refs.append((t.clone(), xh.clone()))
    torch.cuda.synchronize()
    outs, _, _ = run_batch(sst, plans, xs, graph=True)
    for i, ((t, xh), (tr, xr)) in enumerate(zip(outs, refs)):
        assert torch.equal(t, tr), f"shape {i}: TFR differs"
        assert torch.equal(xh, xr), f"shape {i}: reconstruction differs"
    for pl in plans:
        pl.close()


@pytest.mark.parametrize("i", [1, 3, 5])
def test_long_window_split(sst, i):
    """A signal split by frame ranges in two and three parts: the same bits as
    the unsplit call (the parts' halo is M samples, here longer than Nf)."""
    from test_gpu_partition import run_split, unsplit
    p = LONG[i]
    x32 = signal(p, 300 + i)
    ref = unsplit(sst, p, x32)
    for parts in (2, 3):
        got, _ = run_split(sst, p, x32, parts)
        assert torch.equal(got, ref), (parts, (got - ref).abs().max().item())


def test_long_window_stream(sst):
    """A stream whose window (4097 taps) is twice Nf + 1 and longer than a
    pushed chunk, against the FP64 oracle under the bars of tests/parity.py."""
    import test_gpu_stream as TS
    P = dict(fs=16000.0, L=4097, sigma=512.0, hop=32, nfft=2048, f_lo=0.0, f_hi=4000.0, z=2, gamma=0.02)
    saved = TS.P
    TS.P = P
    try:
        x = TS.sig(30000, 13)
        (T, xh), = TS.run_streams(sst, [x], seed=17)
    finally:
        TS.P = saved
    r = O.sst(x.astype(np.float64), P["fs"], P["L"], P["sigma"], P["hop"], P["nfft"], P["f_lo"], P["f_hi"],
              P["z"], P["gamma"], False, inverse_range=(0, len(x)))
    params = dict(n=len(x), relative=False, **P)
    g = gpu_map(sst, params, torch.from_numpy(x).cuda())
    g.update(T=T, xhat=xh)
    print(compare(g, r, params))


@pytest.mark.parametrize("i", [2, 5], ids=[IDS[2], IDS[5]])
def test_long_window_tensor_form(sst, i):
    """The tensor band form (BF16 hi + lo) on long windows: its contraction is
    Eq. 8's direct sum over all L taps (no fold), its inverse the plan's;
    against the oracle with the form's bounds."""
    from test_gpu_tc import check_form, oracle_of, run_tc
    p = LONG[i]
    x32 = signal(p, 300 + i)
    r = oracle_of(p, x32)
    g = run_tc(sst, p, x32, "bf16x3")
    st = check_form(g, r, p, x32.astype(np.float64), "bf16x3")
    print(p, st)


@pytest.mark.parametrize("i", [1, 4], ids=[IDS[1], IDS[4]])
def test_long_window_second_order(sst, i):
    """The second-order path (five STFTs packed into three FFTs, folded as the
    first-order ones) on long windows, against the oracle's second order."""
    from test_gpu_sst2 import check, run
    p = LONG[i]
    x32 = signal(p, 300 + i)
    g = run(sst, p, x32)
    stats, _ = check(p, x32, g)
    print(p, stats)


@pytest.mark.parametrize("i", [2, 6], ids=[IDS[2], IDS[6]])
def test_long_window_zone_inverse(sst, i):
    """The zone inverse (the oracle's T in, zone half-width 3) on long
    windows, against the oracle's zone inverse."""
    from test_gpu_post import _to_gpu, _zone_centres
    p = LONG[i]
    x = signal(p, 300 + i)
    r = O.sst(x.astype(np.float64), p["fs"], p["L"], p["sigma"], p["hop"], p["nfft"], p["f_lo"], p["f_hi"],
              p["z"], p["gamma"], p["relative"])
    plan = sst.Plan(**p)
    F, nbo = r.T.shape
    ridge = _zone_centres(F, nbo, seed=i)
    g, _ = O.window(p["L"], p["sigma"])
    want = O.zone_inverse(r.T, ridge, 3, r.k_lo, p["nfft"], p["z"], g, p["hop"], p["n"])
    got = plan.inverse_zone(_to_gpu(r.T), torch.from_numpy(ridge).cuda(), 3).cpu().numpy().astype(np.float64)
    plan.close()
    full = np.abs(O.inverse(r.T, r.k_lo, p["nfft"], p["z"], g, p["hop"], p["n"])).max()
    err = np.abs(got - want).max()
    assert err <= XHAT_RTOL * full + 1e-7 * max(np.abs(want).max(), 1e-30), (err, full)

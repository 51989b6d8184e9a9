"""Streaming service: continuous batching of live streams.

A stream's output must not depend on how its data was chunked or which other
streams shared its ticks (bit-identical alone vs in a mix with interleaved
pushes and ticks), must equal the whole-signal transform of the concatenated
chunks within the parity tolerances, and match the FP64 oracle; admission is
by device memory, and relative thresholds are refused."""
import numpy as np
import pytest

import oracle as O

from parity import XHAT_RTOL, compare, gpu_map

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

P = dict(fs=25600.0, L=1025, sigma=128.0, hop=16, nfft=2048, f_lo=0.0, f_hi=8000.0, z=2, gamma=0.02)
MAXC = 4096


@pytest.fixture(scope="module")
def sst():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2003_07065_gb300 import build, sst as S
    build.build()
    S.load()
    return S


def sig(n, seed):
    gen = np.random.default_rng(seed)
    t = np.arange(n) / P["fs"]
    x = (np.cos(2 * np.pi * (600 + 300 * seed) * t + 400 * t * t) +
         0.6 * np.cos(2 * np.pi * 3000 * t + 20 * np.sin(2 * np.pi * 2 * t)) + 0.2 * gen.standard_normal(n))
    return x.astype(np.float32)


def bins_of(S):
    k_hi = int(np.floor(P["f_hi"] * P["nfft"] / P["fs"] + 0.5))
    return P["z"] * k_hi + 1


def drain(S, svc, sid, nb, acc):
    while True:
        t, fc, x, fs_, fin = S.sst_stream_poll(svc, sid, nb)
        if len(t):
            assert fc == sum(len(a) for a in acc[0])
            acc[0].append(t)
        if len(x):
            assert fs_ == sum(len(a) for a in acc[1])
            acc[1].append(x)
        if not len(t) and not len(x):
            return fin


def run_streams(S, signals, seed, budget=8 << 30, xhat_only=False):
    """Push each signal in random chunks, interleaving streams and ticks."""
    gen = np.random.default_rng(seed)
    svc = S.sst_service_create(16, budget)
    nb = bins_of(S)
    ids = [S.sst_stream_open(svc, 8.0, MAXC, xhat_only=xhat_only, **P) for _ in signals]
    pos = [0] * len(signals)
    acc = [([], []) for _ in signals]
    while any(p < len(x) for p, x in zip(pos, signals)):
        i = int(gen.integers(len(signals)))
        if pos[i] < len(signals[i]):
            c = int(gen.integers(1, MAXC + 1))
            S.sst_stream_push(svc, ids[i], signals[i][pos[i]:pos[i] + c])
            pos[i] += c
            if pos[i] >= len(signals[i]):
                S.sst_stream_close(svc, ids[i])
        if gen.random() < 0.4:
            S.sst_service_tick(svc)
            for k, sid in enumerate(ids):
                drain(S, svc, sid, nb, acc[k])
    done = [False] * len(signals)
    for _ in range(1000):
        S.sst_service_tick(svc)
        for k, sid in enumerate(ids):
            done[k] = drain(S, svc, sid, nb, acc[k]) or done[k]
        if all(done):
            break
    assert all(done)
    out = [(np.concatenate(a[0]) if a[0] else None, np.concatenate(a[1])) for a in acc]
    S.sst_service_destroy(svc)
    return out


def test_stream_alone_equals_mix(sst):
    signals = [sig(n, i) for i, n in enumerate((30000, 45001, 12345, 60000))]
    mixed = run_streams(sst, signals, seed=1)
    for i, x in enumerate(signals):
        alone = run_streams(sst, [x], seed=100 + i)[0]
        assert np.array_equal(alone[0], mixed[i][0]), f"stream {i}: TFR differs alone vs mix"
        assert np.array_equal(alone[1], mixed[i][1]), f"stream {i}: reconstruction differs alone vs mix"


def test_stream_xhat_only(sst):
    """Reconstruction-only streams deliver no TFR columns and the same x-hat."""
    signals = [sig(n, i) for i, n in enumerate((30000, 12345))]
    full = run_streams(sst, signals, seed=9)
    xo = run_streams(sst, signals, seed=9, xhat_only=True)
    for (t, x), (t2, x2) in zip(full, xo):
        assert t is not None and t2 is None
        assert np.array_equal(x, x2)


def test_stream_equals_whole_signal(sst):
    x = sig(50000, 7)
    (T, xh), = run_streams(sst, [x], seed=3)
    plan = sst.Plan(n=len(x), relative=False, **P)
    tr, xr = plan.forward_inverse(torch.from_numpy(x).cuda())
    tr = tr.cpu().numpy()
    tr = tr[..., 0] + 1j * tr[..., 1]
    xr = xr.cpu().numpy()
    assert T.shape == tr.shape and len(xh) == len(x)
    # same per-frame arithmetic; only the fixed-point scale differs
    assert np.abs(T - tr).max() <= 1e-6 * np.abs(tr).max()
    # tiles of 16 frames vs the whole-signal tiling: only the summation grouping differs
    assert np.abs(xh - xr).max() <= XHAT_RTOL * np.abs(xr).max()
    plan.close()


def test_stream_matches_oracle(sst):
    """A stream against the FP64 oracle under the bars of tests/parity.py; its
    decisions are those of a single plan with the same absolute threshold."""
    x = sig(20000, 11)
    (T, xh), = run_streams(sst, [x], seed=5)
    r = O.sst(x.astype(np.float64), P["fs"], P["L"], P["sigma"], P["hop"], P["nfft"], P["f_lo"], P["f_hi"],
              P["z"], P["gamma"], False, inverse_range=(0, len(x)))
    params = dict(n=len(x), relative=False, **P)
    g = gpu_map(sst, params, torch.from_numpy(x).cuda())
    g.update(T=T, xhat=xh)
    print(compare(g, r, params))


def test_stream_admission_and_errors(sst):
    svc = sst.sst_service_create(4, 1 << 30)
    sid = sst.sst_stream_open(svc, 8.0, MAXC, **P)
    used, budget = sst.sst_service_memory(svc)
    assert 0 < used <= budget
    n_ok = 1
    with pytest.raises(sst.SstError) as e:
        while True:
            sst.sst_stream_open(svc, 8.0, MAXC, **P)
            n_ok += 1
    assert e.value.status == 4 and n_ok * used <= budget
    sst.sst_stream_release(svc, sid)
    sst.sst_stream_open(svc, 8.0, MAXC, **P)        # room again
    with pytest.raises(sst.SstError) as e:
        from paper_2003_07065_gb300.sst import _params, load, sst_params
        import ctypes
        p, _ = _params(0, relative=True, sigma=P["sigma"], g=None, dg=None,
                       **{k: v for k, v in P.items() if k != "sigma"})
        sid2 = ctypes.c_int32()
        st = load().sst_stream_open(svc, ctypes.byref(p), 8.0, MAXC, ctypes.byref(sid2))
        sst._check(st)
    assert e.value.status == 6
    with pytest.raises(sst.SstError):
        sst.sst_stream_push(svc, 99, np.zeros(10, np.float32))
    sst.sst_service_destroy(svc)

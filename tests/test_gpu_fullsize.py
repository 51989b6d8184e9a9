"""Parity at the benchmarks' full sizes, each run by the GPU exactly as the
benchmark runs it, checked against the oracle on outputs it can compute one
by one:

* runup_16m: N = 2^24 (524288 frames, Nf 4096, L 2049, hop 32, z = 4, band
  0-6.4 kHz, gamma = 1e-3 max|V|), one sst_forward_inverse with the default
  one-pass threshold;
* batch256: the 256 mixed channels (204 M samples, 138 GB of TFRs) in one
  captured graph, four channels checked (the longest, the shortest and two
  others);
* stream64: 64 streams in the benchmark's shape, three compared whole.

Per checked signal of the first two: the threshold base (max|V| of the GPU's loudest frame
recomputed by the oracle, and no sampled frame louder); sampled frames (the
first two, the last two and the loudest included): STFT, reassignment map and
T rows in replay mode under the oracle's threshold (gamma times that max);
x_hat on 512-sample windows (the start, the end and interior ones): the
oracle's inverse of the GPU's T rows against the GPU's x_hat, and the
oracle's own x_hat with the exact effect of the sources placed differently
(the bars of tests/parity.py)."""
import numpy as np
import pytest

import oracle as O
from paper_2003_07065_gb300 import workloads as W

from parity import (MAP_RATE, STFT_RTOL, as_complex, check_inverse_alone, check_map, check_tfr_replay,
                    check_xhat_end_to_end, compare, gpu_map, moved_bound)

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


def sampled_check(plan, p, x32, tfr, xhat, n_frames, n_windows, seed):
    """Compare one signal's GPU outputs (tfr, xhat on the device) with the
    oracle on sampled frames and windows; returns the map mismatch rate."""
    x64 = x32.astype(np.float64)
    F, nbo, nf, hop, z = plan.frames, plan.bins, p["nfft"], p["hop"], p["z"]
    M = (p["L"] - 1) // 2
    x = torch.from_numpy(x32).cuda()
    V_g, _ = plan.stft(x)
    _, dest_g = plan.reassign_map(x)
    g, dg = O.window(p["L"], p["sigma"])
    k_lo, k_hi = O.band_bins(p["fs"], nf, p["f_lo"], p["f_hi"])
    assert (k_lo, k_hi) == (plan.k_lo, plan.k_hi)

    # the threshold base
    mag2 = V_g[..., 0] ** 2 + V_g[..., 1] ** 2
    m_star = int(torch.argmax(mag2.max(dim=1).values).item())
    vmax_g = float(mag2.max().sqrt().item())
    V1, _ = O.stft(x64, g, dg, hop, nf, k_lo, k_hi, m_star, 1)
    vmax = float(np.abs(V1).max())
    assert abs(vmax_g - vmax) <= STFT_RTOL * vmax, (vmax_g, vmax)
    gamma = p["gamma"] * vmax if p["relative"] else p["gamma"]

    # sampled frames: STFT, map, T rows in replay mode
    rng = np.random.default_rng(seed)
    extra = rng.choice(F, min(F, n_frames), replace=False)
    frames = np.unique(np.concatenate([[0, min(1, F - 1), max(F - 2, 0), F - 1, m_star], extra]))
    nb = plan.nb
    V_or = np.empty((len(frames), nb), np.complex128)
    dest_or = np.empty((len(frames), nb), np.int64)
    for i, m in enumerate(frames):
        r = O.sst(x64, p["fs"], p["L"], p["sigma"], hop, nf, p["f_lo"], p["f_hi"], z, p["gamma"], True,
                  m0=int(m), nm=1, gamma_abs=gamma)
        V_or[i], dest_or[i] = r.V[0], r.dest[0]
    assert np.abs(V_or).max() <= vmax * (1 + STFT_RTOL), "a sampled frame is louder than the threshold base"
    idx = torch.from_numpy(frames).cuda()
    assert np.abs(as_complex(V_g[idx].cpu().numpy()) - V_or).max() <= STFT_RTOL * vmax
    dg_rows = dest_g[idx].cpu().numpy().astype(np.int64)
    _, rate = check_map(dg_rows, dest_or, V_or, gamma, nbo)
    check_tfr_replay(as_complex(tfr[idx].cpu().numpy()), V_or, dg_rows, dest_or, gamma, nbo)

    # reconstruction windows: the inverse alone (the oracle's inverse of the
    # GPU's T rows) and end to end (with the exact effect of every source the
    # two sides place differently)
    xh = xhat.cpu().numpy().astype(np.float64)
    n = p["n"]
    npw = min(512, n)
    starts = [0, n - npw] + [int(v) for v in rng.integers(0, max(1, n - npw), n_windows - 2)]
    for p0 in starts:
        mlo = max(0, -(-(p0 - M) // hop))
        mhi = min(F - 1, (p0 + npw - 1 + M) // hop)
        r = O.sst(x64, p["fs"], p["L"], p["sigma"], hop, nf, p["f_lo"], p["f_hi"], z, p["gamma"], True, m0=mlo,
                  nm=mhi - mlo + 1, inverse_range=(p0, npw), gamma_abs=gamma)
        rows = torch.arange(mlo, mhi + 1, device="cuda")
        dgc = dest_g[rows].cpu().numpy().astype(np.int64)
        Tg = as_complex(tfr[rows].cpu().numpy())
        check_inverse_alone(Tg, xh[p0:p0 + npw], k_lo, nf, z, g, hop, n, p0, npw, mt0=mlo)
        bound = moved_bound(r.V, dgc, r.dest, k_lo, nf, z, g, hop, n, p0, npw, m0=mlo)
        check_xhat_end_to_end(xh[p0:p0 + npw], r.xhat, bound)
    del V_g, dest_g, mag2
    return rate


def test_runup_16m_sampled_parity(sst):
    w = W.RUNUP_16M
    noisy, _ = w.signal()
    x32 = noisy.astype(np.float32)
    plan = sst.Plan(**w.params())
    x = torch.from_numpy(x32).cuda()
    tfr, xhat = plan.forward_inverse(x)           # the benchmark's call
    torch.cuda.synchronize()
    rate = sampled_check(plan, w.params(), x32, tfr, xhat, n_frames=507, n_windows=3, seed=2024)
    plan.close()
    assert rate <= MAP_RATE


def test_batch256_sampled_parity(sst):
    chans = W.batch_channels(256)
    plans, keep, items = [], [], []
    for params, x in chans:
        pl = sst.Plan(**params)
        xd = torch.from_numpy(x).cuda()
        t = pl.new_tfr()
        xh = torch.empty(pl.n, dtype=torch.float32, device="cuda")
        plans.append(pl)
        keep.append((xd, t, xh))
        items.append((pl.handle, xd, pl.n, t, xh))
    b = sst.sst_batch_create(items, graph=True)    # the benchmark's launch
    ws = torch.empty(max(sst.sst_batch_workspace(b), 256), dtype=torch.uint8, device="cuda")
    sst.sst_batch_run(b, ws)
    torch.cuda.synchronize()
    lengths = np.array([p["n"] for p, _ in chans])
    longest, shortest = int(lengths.argmax()), int(lengths.argmin())
    others = [int(i) for i in np.random.default_rng(7).choice(len(chans), 6, replace=False)
              if int(i) not in (longest, shortest)][:2]
    for i in [longest, shortest] + others:
        params, x = chans[i]
        _, t, xh = keep[i]
        rate = sampled_check(plans[i], params, x, t, xh, n_frames=96, n_windows=3, seed=100 + i)
        assert rate <= MAP_RATE, (i, rate)
    sst.sst_batch_destroy(b)
    for pl in plans:
        pl.close()


def test_stream64_fullsize_parity(sst):
    """The streaming configuration at its benchmark shape: 64 streams at
    25.6 kHz (Nf 2048, hop 16, band 0-8 kHz, z = 2), each 40 chunks of 8192
    samples (12.8 s), pushed round-robin with a tick per round; three streams
    deliver their TFR and are compared whole with the oracle (the bars of the
    single-stream oracle test), the other 61 run reconstruction-only.  Each
    checked stream's absolute threshold is 1e-3 of the oracle's own max|V|."""
    from paper_2003_07065_gb300 import signals
    fs, chunk, nchunks, nstreams = 25600.0, 8192, 40, 64
    P = dict(fs=fs, L=1025, sigma=128.0, hop=16, nfft=2048, f_lo=0.0, f_hi=8000.0, z=2)
    n = chunk * nchunks
    sigs = [signals.chirp_fm_mix(n, fs, 10.0, seed=(5, 1000 + i))[0].astype(np.float32) for i in range(nstreams)]
    checked = (0, 31, 63)
    g, dg = O.window(P["L"], P["sigma"])
    k_lo, k_hi = O.band_bins(fs, P["nfft"], P["f_lo"], P["f_hi"])
    gammas = {i: 1e-3 * O.global_max_abs_v(sigs[i].astype(np.float64), g, dg, P["hop"], P["nfft"], k_lo, k_hi)
              for i in checked}
    svc = sst.sst_service_create(nstreams, 64 << 30)
    ids = [sst.sst_stream_open(svc, 8.0, chunk, gamma=gammas.get(i, 0.02), xhat_only=i not in checked, **P)
           for i in range(nstreams)]
    nb = P["z"] * k_hi + 1
    acc = {i: ([], []) for i in range(nstreams)}

    def drain_all():
        fins = []
        for i, sid in enumerate(ids):
            fin = False
            while True:
                t, fc, xq, fsmp, fin = sst.sst_stream_poll(svc, sid, nb)
                if len(t):
                    acc[i][0].append(t)
                if len(xq):
                    acc[i][1].append(xq)
                if not len(t) and not len(xq):
                    break
            fins.append(fin)
        return fins

    for c in range(nchunks):
        for i, sid in enumerate(ids):
            sst.sst_stream_push(svc, sid, sigs[i][c * chunk:(c + 1) * chunk])
            if c == nchunks - 1:
                sst.sst_stream_close(svc, sid)
        sst.sst_service_tick(svc)
        drain_all()
    for _ in range(1000):
        sst.sst_service_tick(svc)
        if all(drain_all()):
            break
    sst.sst_service_destroy(svc)
    for i in range(nstreams):
        assert sum(len(a) for a in acc[i][1]) == n, i
    for i in checked:
        T = np.concatenate(acc[i][0])
        xh = np.concatenate(acc[i][1]).astype(np.float64)
        r = O.sst(sigs[i].astype(np.float64), fs, P["L"], P["sigma"], P["hop"], P["nfft"], P["f_lo"], P["f_hi"],
                  P["z"], gammas[i], False, inverse_range=(0, n))
        assert T.shape == r.T.shape, (i, T.shape, r.T.shape)
        params = dict(n=n, gamma=gammas[i], relative=False, **P)
        # the stream's decisions are those of a single plan with its threshold
        gm = gpu_map(sst, params, torch.from_numpy(sigs[i]).cuda())
        gm.update(T=T, xhat=xh)
        print(i, compare(gm, r, params))

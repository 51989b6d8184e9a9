"""Parity at the benchmark's full size: the run-up workload at N = 2^24
(524288 frames, Nf 4096, L 2049, hop 32, z = 4, band 0-6.4 kHz, gamma =
1e-3 max|V|), run by the GPU exactly as the benchmark runs it (one
sst_forward_inverse with the default one-pass threshold), checked against
the oracle on outputs it can compute one by one:

* the threshold base: max|V| of the GPU's loudest frame recomputed by the
  oracle, and no sampled frame louder;
* 512 sampled frames (the first and last included): STFT, reassignment map
  and T rows, with the oracle's threshold (1e-3 of that max);
* x_hat on three 512-sample windows (the start, the end and an interior one),
  from the oracle's T of every frame covering them."""
import numpy as np
import pytest

import oracle as O
from paper_2003_07065_gb300 import workloads as W

from parity import MAP_RATE, STFT_RTOL, T_RTOL, XHAT_RTOL, as_complex, check_map

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


def test_runup_16m_sampled_parity(sst):
    w = W.RUNUP_16M
    noisy, _ = w.signal()
    x32 = noisy.astype(np.float32)
    x64 = x32.astype(np.float64)
    plan = sst.Plan(**w.params())
    F, nbo, nf, hop, z = plan.frames, plan.bins, w.nfft, w.hop, w.z
    M = (w.L - 1) // 2
    x = torch.from_numpy(x32).cuda()
    tfr, xhat = plan.forward_inverse(x)           # the benchmark's call
    V_g, Vd_g = plan.stft(x)
    _, dest_g = plan.reassign_map(x)
    torch.cuda.synchronize()

    g, dg = O.window(w.L, w.sigma)
    k_lo, k_hi = O.band_bins(w.fs, nf, w.f_lo, w.f_hi)
    assert (k_lo, k_hi) == (plan.k_lo, plan.k_hi)

    # ---- the threshold base
    mag2 = V_g[..., 0] ** 2 + V_g[..., 1] ** 2
    m_star = int(torch.argmax(mag2.max(dim=1).values).item())
    vmax_g = float(mag2.max().sqrt().item())
    V1, _ = O.stft(x64, g, dg, hop, nf, k_lo, k_hi, m_star, 1)
    vmax = float(np.abs(V1).max())
    assert abs(vmax_g - vmax) <= STFT_RTOL * vmax, (vmax_g, vmax)
    gamma = w.gamma * vmax

    # ---- sampled frames
    rng = np.random.default_rng(2024)
    frames = np.unique(np.concatenate([[0, 1, F - 2, F - 1, m_star], rng.choice(F, 507, replace=False)]))
    V_or = np.empty((len(frames), plan.nb), np.complex128)
    dest_or = np.empty((len(frames), plan.nb), np.int64)
    om_or = np.empty((len(frames), plan.nb))
    T_or = np.empty((len(frames), nbo), np.complex128)
    for i, m in enumerate(frames):
        r = O.sst(x64, w.fs, w.L, w.sigma, hop, nf, w.f_lo, w.f_hi, z, w.gamma, True, m0=int(m), nm=1,
                  gamma_abs=gamma)
        V_or[i], dest_or[i], om_or[i], T_or[i] = r.V[0], r.dest[0], r.omega[0], r.T[0]
    assert np.abs(V_or).max() <= vmax * (1 + STFT_RTOL), "a sampled frame is louder than the threshold base"
    idx = torch.from_numpy(frames).cuda()
    Vg = as_complex(V_g[idx].cpu().numpy())
    assert np.abs(Vg - V_or).max() <= STFT_RTOL * vmax
    dg_rows = dest_g[idx].cpu().numpy().astype(np.int64)
    moved, rate = check_map(dg_rows, dest_or, V_or, gamma, nbo)
    # T: 1e-5 max|V| plus, at both destinations of every moved source and of
    # every source within the STFT bar of gamma (the one-pass forward's own
    # maximum may differ from the map's in the last bit), its modulus
    Tg = as_complex(tfr[idx].cpu().numpy())
    allow = np.zeros(T_or.shape)
    near = np.abs(np.abs(V_or) - gamma) <= STFT_RTOL * vmax
    for rr, cc in zip(*np.nonzero(moved | near)):
        a = np.abs(V_or[rr, cc]) * (1 + 1e-6)
        cand = {int(dg_rows[rr, cc]), int(dest_or[rr, cc])}
        if near[rr, cc] and np.isfinite(om_or[rr, cc]):
            # a threshold flip: the destination the source has when kept (Eq. 28), +-1 for rounding
            l0 = int(np.floor(z * (om_or[rr, cc] - k_lo) + 0.5))
            cand |= {l0 - 1, l0, l0 + 1}
        for dst in cand:
            if 0 <= dst < nbo:
                allow[rr, dst] += a
    err = np.abs(Tg - T_or)
    assert (err <= T_RTOL * vmax + allow).all(), f"T mismatch, max err {err.max():.3e}"

    # ---- reconstruction windows
    xh = xhat.cpu().numpy().astype(np.float64)
    n, npw = w.n, 512
    for p0 in (0, n - npw, int(rng.integers(npw, n - 2 * npw))):
        mlo = max(0, -(-(p0 - M) // hop))
        mhi = min(F - 1, (p0 + npw - 1 + M) // hop)
        r = O.sst(x64, w.fs, w.L, w.sigma, hop, nf, w.f_lo, w.f_hi, z, w.gamma, True, m0=mlo,
                  nm=mhi - mlo + 1, inverse_range=(p0, npw), gamma_abs=gamma)
        cov = torch.arange(mlo, mhi + 1, device="cuda")
        dgc = dest_g[cov].cpu().numpy().astype(np.int64)
        nr = np.abs(np.abs(r.V) - gamma) <= STFT_RTOL * vmax
        mv = (dgc != r.dest) & ~nr
        # a source moved by one fine bin changes r~ by at most (2/Nf)|V| min(2, 2 pi M/(z Nf)),
        # one kept by one side only (within the bar of gamma) by (2/Nf)|V|; per covering frame,
        # summed over the <= L/hop frames covering a sample, divided by min D
        per = 0.0
        if mv.any():
            per = max(per, (2.0 / nf) * np.abs(r.V[mv]).max() * min(2.0, 2 * np.pi * M / (z * nf)))
        if nr.any():
            per = max(per, (2.0 / nf) * np.abs(r.V[nr]).max())
        allow = per * np.ceil(w.L / hop) / (np.sqrt(2.0) / hop * 0.5)
        e = np.abs(xh[p0:p0 + npw] - r.xhat).max()
        assert e <= XHAT_RTOL * np.abs(r.xhat).max() + allow, (p0, e, np.abs(r.xhat).max(), allow)
    plan.close()
    assert rate <= MAP_RATE

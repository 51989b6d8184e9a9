"""Comparison helpers for the GPU-vs-oracle parity tests.

Bars (spec tolerances; the FP32 arithmetic behind each is derived in
the design notes):
  STFT         max|V_gpu - V_or| <= 1e-5 max|V_or|  (same for S^g')
  map          at most 1e-4 of the sources kept by either side land in a
               different bin, and every such pair of destinations is
               adjacent (|dl| = 1); a source kept by one side only must sit
               within 1e-5 max|V| of the threshold (or one step off the grid
               edge).  Where the oracle's S^g' is given, a source whose
               destination coordinate z (w - k_lo) + 1/2 lies within the
               change that the STFT bar allows (both STFTs moved by 1e-5 of
               their maxima) of an integer may land on either side: such
               flips are the bar's own rounding and do not count against
               the rate (a sample of fewer than 1e4 kept sources could not
               otherwise show one)
  TFR          replay mode: the oracle re-accumulates its FP64 V with the
               GPU's destination map, and |T_gpu - T_replay| <= 1e-5 max|V|
               with no allowance, except for the sources within 1e-5 max|V|
               of the threshold (where the GPU's one-pass threshold and its
               map may round differently), which may be present or absent
               as a whole
  column mass  |sum_l T_gpu - sum_l T_or| <= 1e-5 sum|kept V| + the modulus
               of every source kept by one side only (a move to an adjacent
               bin does not change the mass)
  inverse      alone: the oracle's inverse of the GPU's own T (widened to
               FP64) against the GPU's reconstruction, max error <=
               XHAT_RTOL max|xhat|, no allowance;
               end to end: |xhat_gpu - xhat_or|[p] <= XHAT_RTOL max|xhat_or|
               + the exact effect at p of every source the two sides place
               differently (Eq. 25-26 are linear in T), and the output SNR
               within 0.1 dB where a clean signal exists
"""
from __future__ import annotations

import numpy as np

import oracle as O

STFT_RTOL = 1e-5
MAP_RATE = 1e-4
T_RTOL = 1e-5
MASS_RTOL = 1e-5
SNR_DB = 0.1
XHAT_RTOL = 2e-5


def as_complex(a) -> np.ndarray:
    a = np.asarray(a)
    return a[..., 0].astype(np.float64) + 1j * a[..., 1].astype(np.float64)


def check_stft(V_gpu, V_or, what="V"):
    err = np.abs(V_gpu - V_or).max()
    scale = np.abs(V_or).max()
    assert err <= STFT_RTOL * scale, f"{what}: max err {err:.3e} > {STFT_RTOL} * {scale:.3e}"
    return err / scale if scale > 0 else 0.0


def edge_flips(diff, dg, do, V_or, Vd_or, omega_or, k_lo, nfft, z):
    """The mismatches between adjacent destinations whose oracle coordinate
    u = z (w - k_lo) + 1/2 lies within |du| of an integer, |du| the change of
    u that the STFT bar allows: d = -(Nf / 2 pi) Im(V' / V) moves by at most
    (Nf / 2 pi) (e max|V'| / |V| + e max|V| |V'| / |V|^2) with e = STFT_RTOL
    (first order), plus a few FP32 roundings of the coordinate itself."""
    both = diff & (dg >= 0) & (do >= 0) & (np.abs(dg - do) == 1)
    if not both.any():
        return both
    V = np.abs(V_or)
    c = nfft / (2 * np.pi)
    with np.errstate(divide="ignore", invalid="ignore"):
        dd = c * (STFT_RTOL * np.abs(Vd_or).max() / V + STFT_RTOL * V.max() * np.abs(Vd_or) / V ** 2)
    k = np.arange(V_or.shape[1], dtype=np.float64)[None, :] + k_lo
    u = z * (np.asarray(omega_or, dtype=np.float64) - k_lo) + 0.5
    tol = z * dd + 4.0 * 2.0 ** -23 * z * (np.abs(k) + 1.0)
    near = np.abs(u - np.round(u)) <= tol
    return both & np.where(np.isfinite(near), near, False)


def check_map(dest_gpu, dest_or, V_or, gamma, nbo, Vd_or=None, omega_or=None, k_lo=0, nfft=0, z=1):
    """Returns the boolean mask of sources whose destination differs and the
    mismatch rate over the sources kept by either side (flips at a bin edge
    within the STFT bar's reach not counted, where Vd_or and omega_or are
    given)."""
    dg = np.asarray(dest_gpu, dtype=np.int64)
    do = np.asarray(dest_or, dtype=np.int64)
    kept = (dg >= 0) | (do >= 0)
    diff = (dg != do) & kept
    n_kept = int(kept.sum())
    n_diff = int(diff.sum())
    if n_kept == 0:
        return diff, 0.0
    if Vd_or is not None and omega_or is not None:
        n_diff -= int(edge_flips(diff, dg, do, V_or, Vd_or, omega_or, k_lo, nfft, z).sum())
    rate = n_diff / n_kept
    assert rate <= MAP_RATE, f"map mismatch rate {rate:.2e} ({n_diff}/{n_kept})"
    both = diff & (dg >= 0) & (do >= 0)
    if both.any():
        assert np.abs(dg[both] - do[both]).max() == 1, "non-adjacent destination mismatch"
    flip = diff & ((dg == -1) | (do == -1))
    if flip.any():
        vm = np.abs(V_or).max()
        assert np.abs(np.abs(V_or[flip]) - gamma).max() <= STFT_RTOL * vm, \
            "threshold decision differs away from the threshold"
    grid = diff & (((dg == -2) & (do >= 0)) | ((do == -2) & (dg >= 0)))
    # a source that one side drops off the grid and the other keeps must be
    # one rounding step from the edge, i.e. kept at l = 0 or l = nbo - 1
    if grid.any():
        other = np.where(dg[grid] == -2, do[grid], dg[grid])
        assert np.all((other == 0) | (other == nbo - 1)), "grid-edge decision differs away from the edge"
    return diff, rate


def replay_T(V, dest, nbo):
    """T re-accumulated in FP64 from V with a given destination map: T[m, l] =
    sum of V[m, k] over the bins k (ascending) with dest[m, k] = l (Eq. 27-29)."""
    dest = np.asarray(dest, dtype=np.int64)
    T = np.zeros((V.shape[0], nbo), dtype=np.complex128)
    rows, cols = np.nonzero(dest >= 0)        # row-major: ascending k within a frame
    np.add.at(T, (rows, dest[rows, cols]), V[rows, cols])
    return T


def threshold_ambiguous(V_or, gamma):
    """Sources whose oracle modulus lies within 1e-5 max|V| of the threshold."""
    if gamma <= 0:
        return np.zeros(V_or.shape, dtype=bool)
    return np.abs(np.abs(V_or) - gamma) <= STFT_RTOL * np.abs(V_or).max()


def check_tfr_replay(T_gpu, V_or, dest_gpu, dest_or, gamma, nbo):
    """T against the oracle's replay of the GPU's destination map (see the
    module docstring).  Returns max error / max|V|."""
    vmax = np.abs(V_or).max()
    T_rep = replay_T(V_or, dest_gpu, nbo)
    allow = np.zeros(T_rep.shape)
    amb = threshold_ambiguous(V_or, gamma)
    for r, c in np.argwhere(amb):
        a = np.abs(V_or[r, c]) * (1 + 1e-6) + T_RTOL * vmax
        for dst in (dest_gpu[r, c], dest_or[r, c]):
            for d in (dst - 1, dst, dst + 1):
                if 0 <= d < nbo and dst >= 0:
                    allow[r, d] += a
    err = np.abs(T_gpu - T_rep)
    bad = err > T_RTOL * vmax + allow
    assert not bad.any(), (f"TFR differs from the replay at {np.argwhere(bad)[:5].tolist()}, "
                           f"max err {err.max():.3e} (max|V| {vmax:.3e})")
    return float(err.max() / vmax) if vmax > 0 else 0.0


def check_mass(T_gpu, T_or, V_or, dest_gpu, dest_or):
    """Column mass; only sources kept by exactly one side change it."""
    dg = np.asarray(dest_gpu)
    do = np.asarray(dest_or)
    kept = np.where(do >= 0, np.abs(V_or), 0.0).sum(axis=1)
    one_side = (dg >= 0) != (do >= 0)
    flipped = np.where(one_side, np.abs(V_or), 0.0).sum(axis=1)
    d = np.abs(T_gpu.sum(axis=1) - T_or.sum(axis=1))
    assert np.all(d <= MASS_RTOL * kept + flipped * (1 + 1e-6) + 1e-30), "column mass differs"
    ok = kept > 0
    return float(np.max(d[ok] / kept[ok])) if ok.any() else 0.0


def moved_bound(V_or, dest_gpu, dest_or, k_lo, nfft, z, g, hop, n, p0=0, np_=None, m0=0):
    """Per-sample bound on |xhat_gpu - xhat_or| from the sources the two sides
    place differently: source V of frame m at fine bin l enters
    r~[m, j] as (2/Nf) Re(w_l V exp(i 2 pi (z k_lo + l) j / (z Nf))) (Eq. 25,
    w_l = 1/2 at DC and Nyquist), so moving it from l_or to l_gpu (or keeping
    it on one side only, w = 0 on the other) changes x^[p], p = m hop + j, by
    at most g[j] (2/Nf) |V| |w_gpu e^{i th_gpu} - w_or e^{i th_or}| / D[p]
    (Eq. 26)."""
    if np_ is None:
        np_ = n - p0
    L = len(g)
    M = (L - 1) // 2
    G = z * nfft
    j = np.arange(-M, M + 1)
    dg = np.asarray(dest_gpu, dtype=np.int64)
    do = np.asarray(dest_or, dtype=np.int64)
    diff = (dg != do) & ((dg >= 0) | (do >= 0))
    num = np.zeros(np_)

    def term(l):
        if l < 0:
            return np.zeros(L, dtype=np.complex128)
        kk = z * k_lo + int(l)
        w = 0.5 if (kk == 0 or 2 * kk == G) else 1.0
        return w * np.exp(2j * np.pi * ((kk * j) % G) / G)

    for mi, k in np.argwhere(diff):
        m = m0 + int(mi)
        d = (2.0 / nfft) * np.abs(V_or[mi, k]) * np.abs(term(dg[mi, k]) - term(do[mi, k]))
        p = m * hop + j
        ok = (p >= p0) & (p < p0 + np_)
        np.add.at(num, p[ok] - p0, g[ok] * d[ok])
    if not diff.any():
        return num
    D = O.normaliser(g, hop, n, p0, np_)
    return num / D


def check_inverse_alone(T_gpu, xhat_gpu, k_lo, nfft, z, g, hop, n, p0=0, np_=None, mt0=0):
    """The oracle's inverse (Eq. 25-26) of the GPU's own T against the GPU's
    reconstruction, at XHAT_RTOL with no allowance.  Returns the max error
    relative to max|xhat|."""
    xo = O.inverse(np.asarray(T_gpu, dtype=np.complex128), k_lo, nfft, z, g, hop, n, p0, np_, mt0=mt0)
    xg = np.asarray(xhat_gpu, dtype=np.float64)
    scale = np.abs(xo).max()
    err = np.abs(xg - xo).max()
    assert err <= XHAT_RTOL * scale + 1e-30, f"inverse alone: max err {err:.3e} > {XHAT_RTOL} * {scale:.3e}"
    return err / scale if scale > 0 else 0.0


def check_xhat_end_to_end(xhat_gpu, xhat_or, bound):
    """End to end: XHAT_RTOL max|xhat_or| plus the moved-source bound per
    sample.  Returns (max error / max|xhat_or|, the same after subtracting
    the bound)."""
    xg = np.asarray(xhat_gpu, dtype=np.float64)
    scale = np.abs(xhat_or).max()
    err = np.abs(xg - xhat_or)
    bad = err > XHAT_RTOL * scale + bound * (1 + 1e-6) + 1e-30
    assert not bad.any(), (f"xhat differs at {np.argwhere(bad)[:5].ravel().tolist()}: max err {err.max():.3e}, "
                           f"bar {XHAT_RTOL * scale:.3e} + bound {bound.max():.3e}")
    if scale == 0:
        return 0.0, 0.0
    return float(err.max() / scale), float(np.max(err - bound) / scale)


def snr_db(clean, xhat, sl=slice(None)):
    c = np.asarray(clean)[sl]
    e = c - np.asarray(xhat)[sl]
    return 10 * np.log10(np.sum(c * c) / np.sum(e * e))


def gpu_map(S, params, x_dev, two_pass=False):
    """V, V' and the destination map of a single plan with these parameters
    on the device signal x_dev (sst_stft, sst_reassign_map): the decisions the
    batched and streamed paths share with it.  Returns numpy arrays."""
    plan = S.Plan(**params, two_pass=two_pass)
    V, Vd = plan.stft(x_dev)
    _, dest = plan.reassign_map(x_dev)
    out = dict(V=as_complex(V.cpu().numpy()), Vd=as_complex(Vd.cpu().numpy()),
               dest=dest.cpu().numpy().astype(np.int64))
    plan.close()
    return out


def compare(g, r, params, clean=None, inverse_range=None):
    """Every bar above for one signal.  g: the GPU's outputs (dict with T,
    dest, xhat and optionally V, Vd, maxv); r: the oracle's Result for the
    same float32 input (with xhat over inverse_range, default the whole
    signal); params: the plan parameters."""
    nbo = r.T.shape[1]
    assert g["T"].shape == r.T.shape
    stats = {}
    if "V" in g:
        stats["stft"] = check_stft(g["V"], r.V, "V")
        stats["stft_d"] = check_stft(g["Vd"], r.Vd, "Vd")
    if params["relative"] and "maxv" in g:
        vmax = np.abs(r.V).max()
        assert abs(g["maxv"] - vmax) <= STFT_RTOL * vmax
    _, rate = check_map(g["dest"], r.dest, r.V, r.gamma, nbo, r.Vd, r.omega, r.k_lo, params["nfft"], params["z"])
    stats["map_rate"] = rate
    stats["tfr_replay"] = check_tfr_replay(g["T"], r.V, g["dest"], r.dest, r.gamma, nbo)
    stats["mass"] = check_mass(g["T"], r.T, r.V, g["dest"], r.dest)
    if "xhat" in g and r.xhat is not None:
        n = params["n"]
        p0, np_ = inverse_range if inverse_range is not None else (0, n)
        win, _ = O.window(params["L"], params["sigma"])
        xg = np.asarray(g["xhat"], dtype=np.float64)[p0:p0 + np_] if len(g["xhat"]) == n else g["xhat"]
        stats["xhat_inverse_alone"] = check_inverse_alone(g["T"], xg, r.k_lo, params["nfft"], params["z"], win,
                                                          params["hop"], n, p0, np_, mt0=r.m0)
        bound = moved_bound(r.V, g["dest"], r.dest, r.k_lo, params["nfft"], params["z"], win, params["hop"], n,
                            p0, np_, m0=r.m0)
        stats["xhat"], stats["xhat_beyond_bound"] = check_xhat_end_to_end(xg, r.xhat, bound)
        if clean is not None:
            c = np.asarray(clean)[p0:p0 + np_]
            s_g, s_o = snr_db(c, xg), snr_db(c, r.xhat)
            stats["snr_gpu"], stats["snr_oracle"] = s_g, s_o
            assert abs(s_g - s_o) <= SNR_DB, (s_g, s_o)
    return stats

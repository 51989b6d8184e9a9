"""Comparison helpers for the GPU-vs-oracle parity tests.

Tolerances (spec bars; the FP32 arithmetic behind each is derived in
the design notes):
  STFT         max|V_gpu - V_or| <= 1e-5 max|V_or|  (same for S^g')
  map          at most 1e-4 of the sources kept by either side land in a
               different bin, and every such pair of destinations is
               adjacent (|dl| = 1); a source kept by one side only must sit
               within 1e-5 max|V| of the threshold
  TFR          |T_gpu - T_or| <= 1e-5 max|V| + the modulus of every source
               whose destination differs between the two sides, at both of
               its destinations
  column mass  |sum_l T_gpu - sum_l T_or| <= 1e-5 sum|kept V| + moved-off mass
  inverse      output SNR within 0.1 dB, and max|xhat_gpu - xhat_or| <=
               XHAT_RTOL max|xhat_or| + the flipped-source allowance
"""
from __future__ import annotations

import numpy as np

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
    return err / scale


def check_map(dest_gpu, dest_or, V_or, gamma, nbo):
    """Returns the boolean mask of sources whose destination differs."""
    dg = np.asarray(dest_gpu, dtype=np.int64)
    do = np.asarray(dest_or, dtype=np.int64)
    kept = (dg != -1) | (do != -1)
    diff = dg != do
    n_kept = int(kept.sum())
    n_diff = int((diff & kept).sum())
    assert n_kept > 0
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
    return diff & kept, rate


def check_tfr(T_gpu, T_or, V_or, moved, dest_gpu, dest_or):
    vmax = np.abs(V_or).max()
    allow = np.zeros(T_or.shape)
    rows, cols = np.nonzero(moved)
    for r, c in zip(rows, cols):
        a = np.abs(V_or[r, c]) * (1 + 1e-6)
        for dst in (dest_gpu[r, c], dest_or[r, c]):
            if dst >= 0:
                allow[r, dst] += a
    err = np.abs(T_gpu - T_or)
    bad = err > T_RTOL * vmax + allow
    assert not bad.any(), f"TFR mismatch at {np.argwhere(bad)[:5]}, max err {err.max():.3e} (vmax {vmax:.3e})"
    return float(np.max(err - allow)) / vmax


def check_mass(T_gpu, T_or, V_or, gamma, moved):
    kept = np.where(np.abs(V_or) > gamma, np.abs(V_or), 0.0).sum(axis=1)
    moved_mass = np.where(moved, np.abs(V_or), 0.0).sum(axis=1)
    d = np.abs(T_gpu.sum(axis=1) - T_or.sum(axis=1))
    assert np.all(d <= MASS_RTOL * kept + moved_mass + 1e-30), "column mass differs"
    ok = kept > 0
    return float(np.max(d[ok] / kept[ok])) if ok.any() else 0.0


def snr_db(clean, xhat, sl=slice(None)):
    c = np.asarray(clean)[sl]
    e = c - np.asarray(xhat)[sl]
    return 10 * np.log10(np.sum(c * c) / np.sum(e * e))

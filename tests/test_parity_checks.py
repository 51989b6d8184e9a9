"""The parity checker itself, on the CPU (no GPU): results built from the
oracle in FP32 with one source moved to an adjacent bin pass every bar of
tests/parity.py, and each planted mistake (a dropped source in T, a source
moved two bins, a wrong reconstruction sample, a T that does not follow its
own map) fails the bar meant to catch it."""
import numpy as np
import pytest

import oracle as O

import parity as P

PARAMS = dict(n=6000, fs=8000.0, L=257, sigma=32.0, hop=8, nfft=256, f_lo=500.0, f_hi=3000.0, z=2,
              gamma=1e-3, relative=True)


@pytest.fixture(scope="module")
def case():
    p = PARAMS
    t = np.arange(p["n"]) / p["fs"]
    clean = np.cos(2 * np.pi * (900 * t + 400 * t * t)) + 0.5 * np.cos(2 * np.pi * 2200 * t)
    x = (clean + 0.1 * np.random.default_rng(0).standard_normal(p["n"])).astype(np.float32)
    r = O.sst(x.astype(np.float64), p["fs"], p["L"], p["sigma"], p["hop"], p["nfft"], p["f_lo"], p["f_hi"],
              p["z"], p["gamma"], True, inverse_range=(0, p["n"]))
    return x, clean, r


def fake_gpu(r, move=None):
    """A stand-in for the GPU's outputs: V rounded to FP32, the oracle's map
    with `move` = (m, k, dl) applied, T replayed from them and rounded, the
    reconstruction from that T rounded to FP32."""
    p = PARAMS
    V32 = r.V.astype(np.complex64).astype(np.complex128)
    dest = r.dest.copy()
    if move is not None:
        m, k, dl = move
        dest[m, k] += dl
    nbo = r.T.shape[1]
    T = P.replay_T(V32, dest, nbo).astype(np.complex64).astype(np.complex128)
    g, _ = O.window(p["L"], p["sigma"])
    xh = O.inverse(T, r.k_lo, p["nfft"], p["z"], g, p["hop"], p["n"]).astype(np.float32)
    return dict(V=V32, Vd=r.Vd.astype(np.complex64).astype(np.complex128), dest=dest, T=T, xhat=xh,
                maxv=float(np.abs(V32).max()))


def loud_source(r):
    """The loudest kept source with room for a move of two bins either way."""
    a = np.where((r.dest >= 2) & (r.dest < r.T.shape[1] - 2), np.abs(r.V), 0.0)
    return np.unravel_index(np.argmax(a), a.shape)


def test_fp32_result_with_an_adjacent_move_passes(case):
    x, clean, r = case
    m, k = loud_source(r)
    g = fake_gpu(r, move=(m, k, 1))
    stats = P.compare(g, r, PARAMS, clean)
    # the move is visible end to end and covered by its exact bound
    assert stats["xhat"] > 1e-4 and stats["xhat_beyond_bound"] <= P.XHAT_RTOL


def test_dropped_source_in_T_fails_replay(case):
    _, _, r = case
    g = fake_gpu(r)
    m, k = loud_source(r)
    g["T"][m, r.dest[m, k]] -= r.V[m, k]
    with pytest.raises(AssertionError, match="replay"):
        P.check_tfr_replay(g["T"], r.V, g["dest"], r.dest, r.gamma, r.T.shape[1])


def test_T_not_following_its_map_fails_replay(case):
    # T built with a moved source while the map still says the oracle's bin
    _, _, r = case
    m, k = loud_source(r)
    moved = fake_gpu(r, move=(m, k, 1))
    moved["dest"] = r.dest.copy()
    with pytest.raises(AssertionError, match="replay"):
        P.check_tfr_replay(moved["T"], r.V, moved["dest"], r.dest, r.gamma, r.T.shape[1])


def test_move_of_two_bins_fails_map(case):
    _, _, r = case
    m, k = loud_source(r)
    g = fake_gpu(r, move=(m, k, 2))
    with pytest.raises(AssertionError, match="non-adjacent"):
        P.check_map(g["dest"], r.dest, r.V, r.gamma, r.T.shape[1])


def test_wrong_reconstruction_sample_fails_both_inverse_checks(case):
    _, _, r = case
    g = fake_gpu(r)
    p = PARAMS
    win, _ = O.window(p["L"], p["sigma"])
    bad = g["xhat"].astype(np.float64)
    bad[1234] += 1e-4 * np.abs(r.xhat).max()
    with pytest.raises(AssertionError, match="inverse alone"):
        P.check_inverse_alone(g["T"], bad, r.k_lo, p["nfft"], p["z"], win, p["hop"], p["n"])
    bound = P.moved_bound(r.V, g["dest"], r.dest, r.k_lo, p["nfft"], p["z"], win, p["hop"], p["n"])
    with pytest.raises(AssertionError, match="xhat differs"):
        P.check_xhat_end_to_end(bad, r.xhat, bound)


def test_moved_bound_covers_one_move_tightly(case):
    """Eq. 25-26 are linear in T, so one moved source changes xhat by the real
    part of the term the bound takes the modulus of: never more than the
    bound, and close to it where the phase lines up."""
    _, _, r = case
    p = PARAMS
    m, k = loud_source(r)
    win, _ = O.window(p["L"], p["sigma"])
    dest = r.dest.copy()
    dest[m, k] += 1
    T2 = P.replay_T(r.V, dest, r.T.shape[1])
    x2 = O.inverse(T2, r.k_lo, p["nfft"], p["z"], win, p["hop"], p["n"])
    bound = P.moved_bound(r.V, dest, r.dest, r.k_lo, p["nfft"], p["z"], win, p["hop"], p["n"])
    delta = np.abs(x2 - r.xhat)
    assert np.all(delta <= bound * (1 + 1e-9) + 1e-15)
    j = slice(m * p["hop"] - 100, m * p["hop"] + 100)
    assert delta[j].max() >= 0.9 * bound[j].max() > 0


def edge_distance(r, p):
    """|u - round(u)| of every source and the tolerance the STFT bar allows."""
    u = p["z"] * (r.omega - r.k_lo) + 0.5
    V = np.abs(r.V)
    c = p["nfft"] / (2 * np.pi)
    with np.errstate(divide="ignore", invalid="ignore"):
        tol = p["z"] * c * (P.STFT_RTOL * np.abs(r.Vd).max() / V + P.STFT_RTOL * V.max() * np.abs(r.Vd) / V ** 2)
    return np.abs(u - np.round(u)), u, tol


def test_many_moves_away_from_edges_fail_the_rate(case):
    """Adjacent moves of loud sources far from a bin edge are not rounding:
    more of them than the rate allows fail, with or without the oracle's
    IF supplied."""
    _, _, r = case
    p = PARAMS
    dist, _, tol = edge_distance(r, p)
    nbo = r.T.shape[1]
    cand = (r.dest >= 1) & (r.dest < nbo - 1) & (dist > 0.25) & (dist > 10 * np.nan_to_num(tol, nan=1.0))
    idx = np.argwhere(cand)
    n_kept = int((r.dest >= 0).sum())
    n_move = int(2 * P.MAP_RATE * n_kept) + 2
    assert len(idx) >= n_move
    dest = r.dest.copy()
    for m, k in idx[:n_move]:
        dest[m, k] += 1
    with pytest.raises(AssertionError, match="map mismatch rate"):
        P.check_map(dest, r.dest, r.V, r.gamma, nbo, r.Vd, r.omega, r.k_lo, p["nfft"], p["z"])


def test_flips_at_a_bin_edge_within_the_stft_bar_are_allowed(case):
    """Sources whose destination coordinate sits within the STFT bar's reach
    of a bin edge may land on either side: moved across the edge, they pass
    once the oracle's IF is supplied, however many, and fail the rate without
    it when they are more than it allows."""
    _, _, r = case
    p = PARAMS
    dist, u, tol = edge_distance(r, p)
    nbo = r.T.shape[1]
    near = (r.dest >= 1) & (r.dest < nbo - 1) & (dist <= 0.5 * np.nan_to_num(tol, nan=0.0))
    idx = np.argwhere(near)
    n_kept = int((r.dest >= 0).sum())
    assert len(idx) > P.MAP_RATE * n_kept + 1, len(idx)
    dest = r.dest.copy()
    for m, k in idx:   # across the nearest edge
        dest[m, k] += 1 if u[m, k] - np.floor(u[m, k]) > 0.5 else -1
    P.check_map(dest, r.dest, r.V, r.gamma, nbo, r.Vd, r.omega, r.k_lo, p["nfft"], p["z"])
    with pytest.raises(AssertionError, match="map mismatch rate"):
        P.check_map(dest, r.dest, r.V, r.gamma, nbo)

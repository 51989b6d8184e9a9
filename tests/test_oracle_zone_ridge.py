"""Pins of the oracle's zone reconstruction (Eq. 15 zone, Sec. 2.3 TF
filtering), ridge extraction and Renyi entropy (Eq. 32) to facts outside
their code: linearity of the inverse over a tiling of zones, the zone's
inclusive boundary, two-tone separation against the single-tone closed form,
a library argmax, a smoothing case worked by hand, a linear chirp's IF, and
closed-form entropies.  CPU only."""
import math

import numpy as np
import pytest

import oracle as O
from paper_2003_07065_gb300 import signals as S

FS, NFFT, L, SIGMA, HOP = 25600.0, 1024, 2049, 128.0, 16


def _two_tone(n=16384, z=2, f1_bin=150.0, f2_bin=220.0):
    x1 = S.tone(n, FS, f1_bin * FS / NFFT, amp=0.8, phase=1.1)
    x2 = S.tone(n, FS, f2_bin * FS / NFFT, amp=0.5, phase=0.3)
    r = O.sst(x1 + x2, FS, L, SIGMA, HOP, NFFT, 0.0, 6400.0, z, 0.0, False, inverse_range=(0, n))
    g, _ = O.window(L, SIGMA)
    return x1, x2, r, g


def _zinv(r, g, ridge, hw, z, n):
    return O.zone_inverse(r.T, ridge, hw, r.k_lo, NFFT, z, g, HOP, n)


def test_zone_covering_everything_is_the_inverse():
    n, z = 16384, 2
    _, _, r, g = _two_tone(n, z)
    F, nbo = r.T.shape
    xq = _zinv(r, g, np.zeros(F, np.int64), nbo, z, n)
    np.testing.assert_array_equal(xq, r.xhat)


def test_zones_tiling_the_band_add_up_to_the_inverse():
    """The inverse is linear, so zones that partition the output bins give
    components that sum to the full reconstruction; an off-by-one at a zone
    edge drops or doubles a column of bins and breaks the sum."""
    n, z = 16384, 2
    _, _, r, g = _two_tone(n, z)
    F, nbo = r.T.shape
    w = (nbo + 2) // 6 + 1          # three zones of 2w + 1 bins cover [0, 6w + 3) >= nbo
    parts = [_zinv(r, g, np.full(F, c, np.int64), w, z, n) for c in (w, 3 * w + 1, 5 * w + 2)]
    total = parts[0] + parts[1] + parts[2]
    np.testing.assert_allclose(total, r.xhat, rtol=0, atol=1e-12 * np.abs(r.xhat).max())
    assert np.abs(parts[0]).max() > 0 and np.abs(parts[1]).max() > 0


@pytest.mark.parametrize("z", [1, 3])
def test_zone_tiling_small_grid(z):
    """The tiling identity with an odd subdivision (its zNf-point inverse is a
    plain DFT in the oracle, so the grid is kept small) and without one."""
    n, fs, nfft, L, sigma, hop = 3000, 8000.0, 256, 129, 16.0, 8
    x = S.tone(n, fs, 37.0 * fs / nfft, amp=0.8, phase=0.2) + S.tone(n, fs, 90.3 * fs / nfft, amp=0.4, phase=1.0)
    r = O.sst(x, fs, L, sigma, hop, nfft, 0.0, fs / 2, z, 0.0, False, inverse_range=(0, n))
    g, _ = O.window(L, sigma)
    F, nbo = r.T.shape
    w = (nbo + 2) // 6 + 1
    total = sum(O.zone_inverse(r.T, np.full(F, c, np.int64), w, r.k_lo, nfft, z, g, hop, n)
                for c in (w, 3 * w + 1, 5 * w + 2))
    np.testing.assert_allclose(total, r.xhat, rtol=0, atol=1e-12 * np.abs(r.xhat).max())


def test_zone_edge_is_inclusive_and_no_ridge_means_empty():
    F, nbo, l0, w = 40, 64, 20, 3
    T = np.zeros((F, nbo), np.complex128)
    T[:, l0] = 1.0 + 0.5j
    g, _ = O.window(129, 16.0)
    args = (0, 128, 1, g, 8, 8 * F)
    on = O.zone_inverse(T, np.full(F, l0 + w), w, *args)
    off = O.zone_inverse(T, np.full(F, l0 + w + 1), w, *args)
    none = O.zone_inverse(T, np.full(F, -1), 100, *args)
    assert np.abs(on).max() > 1e-3
    assert np.abs(off).max() == 0.0 and np.abs(none).max() == 0.0
    m = O.zone_mask(nbo, [l0 - w, l0 + w, l0 + w + 1, -1], w)
    assert m[0, l0] and m[1, l0] and not m[2, l0] and not m[3].any()


@pytest.mark.parametrize("z", [1, 2, 4])
def test_zone_separates_two_tones(z):
    """Each tone is squeezed into its own bin (Sec. 2.2), so a zone of a few
    bins around one tone returns that tone as the single-tone closed form
    does (x_hat = x inside, Sec. 2.3) and none of the other."""
    n = 16384
    x1, x2, r, g = _two_tone(n, z)
    F = r.T.shape[0]
    inner = slice(4096, n - 4096)
    for xt, fb in ((x1, 150.0), (x2, 220.0)):
        c = int(round((fb - r.k_lo) * z))
        xq = _zinv(r, g, np.full(F, c, np.int64), 2 * z, z, n)
        assert np.abs(xq[inner] - xt[inner]).max() < 1e-6


def test_ridge_without_smoothing_is_the_band_argmax():
    rng = np.random.default_rng(3)
    T = rng.standard_normal((50, 40)) + 1j * rng.standard_normal((50, 40))
    got = O.ridge(T, 5, 30, 0)
    want = 5 + np.argmax(np.abs(T[:, 5:31]), axis=1)
    np.testing.assert_array_equal(got, want)


def test_ridge_ties_go_to_the_smallest_bin_and_empty_frames_to_minus_one():
    T = np.zeros((3, 8), np.complex128)
    T[0, [2, 5]] = 1.0
    T[1, [6, 3, 4]] = [2.0, 2.0j, -2.0]
    got = O.ridge(T, 1, 7, 0)
    np.testing.assert_array_equal(got, [2, 3, -1])


def test_ridge_smoothing_worked_example():
    """A steady line of energy 1 at bin 7 and a one-frame spike of energy 2.5
    at bin 2 in frame 5.  Unsmoothed, frame 5 picks the spike; with |d| <= 1
    the line collects 3 (three frames of 1) against the spike's 2.5 in frames
    4, 5 and 6; with |d| <= 2 near the ends the line collects 2 or 3."""
    F = 12
    T = np.zeros((F, 10), np.complex128)
    T[:, 7] = 1.0
    T[5, 2] = math.sqrt(2.5)
    np.testing.assert_array_equal(O.ridge(T, 0, 9, 0), [7] * 5 + [2] + [7] * 6)
    np.testing.assert_array_equal(O.ridge(T, 0, 9, 1), [7] * F)
    np.testing.assert_array_equal(O.ridge(T, 0, 3, 1), [-1, -1, -1, -1, 2, 2, 2, -1, -1, -1, -1, -1])


def test_ridge_follows_a_linear_chirp():
    """A linear chirp's IF f0 + c t (Eq. 1 with phi = 2 pi (f0 t + c t^2 / 2))
    is followed to within one output bin (Delta f / z) away from the ends."""
    n, z = 32768, 4
    f0, f1 = 1500.0, 3500.0
    t = np.arange(n) / FS
    c = (f1 - f0) / t[-1]
    x = np.cos(2 * np.pi * (f0 * t + 0.5 * c * t * t))
    r = O.sst(x, FS, 1025, 128.0, HOP, NFFT, 1000.0, 4000.0, z, 1e-3, True)
    rid = O.ridge(r.T, 0, r.T.shape[1] - 1, 2)
    f_hat = O.ridge_hz(rid, r.k_lo, z, FS, NFFT)
    tm = np.arange(r.T.shape[0]) * HOP / FS
    inner = (tm > 0.1) & (tm < t[-1] - 0.1)
    assert np.abs(f_hat[inner] - (f0 + c * tm[inner])).max() <= FS / NFFT / z


def test_renyi_closed_forms():
    K = 37
    for a in (0.5, 2.0, 3.0):
        assert O.renyi(np.ones(K), a) == pytest.approx(math.log2(K), abs=1e-12)
        d = np.zeros(K)
        d[4] = 3.0
        assert O.renyi(d, a) == pytest.approx(0.0, abs=1e-12)
    # one cell of probability q, the rest share 1 - q equally (P = |T|^2)
    q, a = 0.6, 3.0
    P = np.full(K, (1 - q) / (K - 1))
    P[0] = q
    want = math.log2(q ** a + (K - 1) * ((1 - q) / (K - 1)) ** a) / (1 - a)
    assert O.renyi(np.sqrt(P) * np.exp(1j * np.arange(K)), a) == pytest.approx(want, abs=1e-12)
    # scale invariance and the cell area's additive log2
    rng = np.random.default_rng(1)
    T = rng.standard_normal((20, 30)) + 1j * rng.standard_normal((20, 30))
    assert O.renyi(7.5 * T) == pytest.approx(O.renyi(T), abs=1e-12)
    assert O.renyi(T, 3.0, cell=0.25) == pytest.approx(O.renyi(T) - 2.0, abs=1e-12)
    with pytest.raises(ValueError):
        O.renyi(T, 1.0)


def test_renyi_sst_more_concentrated_than_stft():
    """Sec. 3.2: for a tone, the synchrosqueezed TFR has lower entropy than
    the STFT it came from (the lobe's mass sits in one bin)."""
    n = 16384
    x = S.tone(n, FS, 150.0 * FS / NFFT, amp=1.0, phase=0.0)
    r = O.sst(x, FS, L, SIGMA, HOP, NFFT, 0.0, 6400.0, 1, 1e-3, True)
    assert O.renyi(r.T) < O.renyi(r.V) - 1.0

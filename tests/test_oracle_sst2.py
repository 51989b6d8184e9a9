"""Pins of the oracle's second-order IF and reassignment (the extension the
paper names as future work, Sec. 6) to closed forms: a linear chirp's IF
f0 + c t and chirp rate c returned exactly where the first-order estimate
(Eq. 13) is biased off the ridge, a tone's chirp rate 0 (second order equals
first order), the sign of a falling chirp, and a chirp's whole kept lobe
reassigned to the one fine bin of its IF.  CPU only."""
import numpy as np
import pytest

import oracle as O

FS, NFFT, L, SIGMA, HOP = 25600.0, 1024, 2049, 128.0, 16


def chirp(n, f0, c):
    """cos 2 pi (f0 t + c t^2 / 2), t in samples, f0 in cycles/sample, c in cycles/sample^2."""
    t = np.arange(n, dtype=np.float64)
    return np.cos(2 * np.pi * (f0 * t + 0.5 * c * t * t))


@pytest.mark.parametrize("c", [2e-7, -1.5e-7, 6e-7])
def test_linear_chirp_if_and_rate_exact(c):
    n, f0 = 16384, 3000.0 / FS
    x = chirp(n, f0, c)
    m0, nm = 300, 5
    V, w1, w2, q = O.if2(x, L, SIGMA, HOP, NFFT, 0, 512, m0=m0, nm=nm)
    for i in range(nm):
        tm = (m0 + i) * HOP
        ifb = (f0 + c * tm) * NFFT                 # the chirp's IF at the frame centre, in bins
        a = np.abs(V[i])
        lobe = a > 0.05 * a.max()
        assert lobe.sum() >= 5
        assert np.abs(w2[i, lobe] - ifb).max() < 1e-8
        np.testing.assert_allclose(q[i, lobe].real, c * NFFT, rtol=1e-8)
        assert np.abs(q[i, lobe].imag).max() < 1e-8 * abs(c * NFFT)
        # the first-order estimate is off the IF away from the ridge
        assert np.abs(w1[i, lobe] - ifb).max() > 1e-5


def test_tone_has_no_chirp_rate():
    x = np.cos(2 * np.pi * (200.3 / NFFT) * np.arange(16384) + 0.4)
    V, w1, w2, q = O.if2(x, L, SIGMA, HOP, NFFT, 100, 300, m0=200, nm=3)
    a = np.abs(V)
    lobe = a > 1e-3 * a.max()
    assert np.abs(q[lobe]).max() < 1e-9
    assert np.abs(w2[lobe] - w1[lobe]).max() < 1e-7
    assert np.abs(w2[lobe] - 200.3).max() < 1e-6


@pytest.mark.parametrize("z", [4, 16])
def test_chirp_lobe_lands_in_one_fine_bin(z):
    """With the exact IF every kept source of a frame goes to the fine bin of
    the chirp's IF (chosen away from a bin edge), so T holds the lobe's sum
    there and nothing elsewhere."""
    n, c = 16384, 5e-6                               # fast: the first-order bias is ~20 % off the ridge
    f0 = (200.0 + 0.3 / z) / NFFT - c * 250 * HOP    # IF at frame 250 sits 0.3 fine bins past a grid point
    x = chirp(n, f0, c)
    k_lo, k_hi = 150, 260
    m = 250
    V, w1, w2, q = O.if2(x, L, SIGMA, HOP, NFFT, k_lo, k_hi, m0=m, nm=1)
    gamma = 1e-3 * np.abs(V).max()
    dest, T = O.reassign2(V, w2, k_lo, k_hi, z, gamma)
    ifb = (f0 + c * m * HOP) * NFFT
    lstar = int(np.floor(z * (ifb - k_lo) + 0.5))
    kept = np.abs(V[0]) > gamma
    assert kept.sum() >= 5
    assert set(dest[0, kept]) == {lstar}
    np.testing.assert_allclose(T[0, lstar], V[0, kept].sum(), rtol=1e-12)
    others = np.delete(T[0], lstar)
    assert np.abs(others).max() == 0.0
    # the first-order estimate spreads the same lobe over several fine bins
    dest1, _ = O.reassign2(V, w1, k_lo, k_hi, z, gamma)
    assert len(set(dest1[0, kept])) > 1


def test_reassign2_threshold_and_grid_edges():
    V = np.array([[1.0, 0.5, 2.0, 3.0]], dtype=np.complex128)
    om = np.array([[10.2, 10.0, 9.4, 13.6]])
    dest, T = O.reassign2(V, om, 10, 13, 2, 0.7)
    # |V| <= gamma: -1; l = floor(2 (om - 10) + 1/2): 0 (10.2), below the grid (9.4 -> -1): -2,
    # 13.6 -> 7 > z N_r = 6: -2
    np.testing.assert_array_equal(dest, [[0, -1, -2, -2]])
    assert T[0, 0] == 1.0 and np.abs(T).sum() == 1.0


def test_sst2_equals_sst_on_a_tone():
    """q = 0 for a tone, so on the frames whose window lies inside the signal
    (the onset and the end are transients) the second-order transform equals
    the first-order one: same destinations, same T, and the same
    reconstruction where only such frames contribute."""
    n = 16384
    M = (L - 1) // 2
    x = np.cos(2 * np.pi * (150.0 / NFFT) * np.arange(n) + 0.7)
    a = O.sst(x, FS, L, SIGMA, HOP, NFFT, 0.0, 6400.0, 4, 1e-3, True, inverse_range=(0, n))
    b = O.sst2(x, FS, L, SIGMA, HOP, NFFT, 0.0, 6400.0, 4, 1e-3, True, inverse_range=(0, n))
    inner = slice(-(-M // HOP), (n - 1 - M) // HOP + 1)
    np.testing.assert_array_equal(a.dest[inner], b.dest[inner])
    np.testing.assert_allclose(b.T[inner], a.T[inner], rtol=0, atol=1e-12 * np.abs(a.T).max())
    ps = slice(2 * M + HOP, n - 2 * M - HOP)
    np.testing.assert_allclose(b.xhat[ps], a.xhat[ps], rtol=0, atol=1e-12 * np.abs(a.xhat).max())


def test_impulse_falls_back_to_first_order():
    """At an impulse the complex time does not move with t (d/dt t~ = 0): the
    chirp rate is undefined and the second-order IF is the first-order one."""
    n = 8192
    x = np.zeros(n)
    x[4000] = 1.0
    V, w1, w2, q = O.if2(x, L, SIGMA, HOP, NFFT, 10, 500, m0=4000 // HOP - 2, nm=5)
    ok = np.abs(V) > 1e-6 * np.abs(V).max()
    np.testing.assert_array_equal(w2[ok], w1[ok])

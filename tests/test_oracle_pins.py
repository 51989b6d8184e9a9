"""Pins of the FP64 oracle to facts outside itself: library and brute-force
transforms on tiny inputs, closed forms (tone, Gaussian-windowed chirp, the
Eq. 22 continuous limit), invariants (mass, odd-z coarsening, WOLA and Eq. 15
exactness) and the numbers the paper prints.  CPU only."""
import math
import os

import numpy as np
import pytest

import oracle as O
from paper_2003_07065_gb300 import signals as S

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ------------------------------------------------------------------ FFT
@pytest.mark.parametrize("n", [1, 2, 4, 8, 64, 1024, 4096])
def test_fft_matches_numpy(n):
    r = np.random.default_rng(n)
    x = r.standard_normal(n) + 1j * r.standard_normal(n)
    np.testing.assert_allclose(O.fft(x, -1), np.fft.fft(x), atol=1e-12 * max(1, n))
    np.testing.assert_allclose(O.fft(x, +1), np.fft.ifft(x) * n, atol=1e-12 * max(1, n))


def test_fft_matches_naive_dft():
    n = 32
    x = np.random.default_rng(7).standard_normal(n) + 0j
    k = np.arange(n)
    W = np.exp(-2j * np.pi * np.outer(k, k) / n)
    np.testing.assert_allclose(O.fft(x, -1), W @ x, atol=1e-12)


# ------------------------------------------------------------------ window
def test_window_closed_form():
    L, sigma = 129, 16.0
    g, dg = O.window(L, sigma)
    M = (L - 1) // 2
    assert g[M] == pytest.approx((math.pi * sigma ** 2) ** -0.25, rel=1e-15)
    # unit energy of the continuous window (Sec. 2.1, Eq. 6): the sampled,
    # truncated window keeps 1 - erfc(M / sigma) of it, up to the end-point
    # (Euler-Maclaurin) term g(M)^2; the Poisson aliasing is negligible here
    assert abs(np.sum(g ** 2) - (1 - math.erfc(M / sigma))) <= 2 * g[-1] ** 2
    # g' is the derivative of g: compare with a central difference of the
    # analytic Gaussian evaluated off the grid
    t = np.arange(-M, M + 1, dtype=np.float64)
    h = 1e-5
    gg = lambda u: (math.pi * sigma ** 2) ** -0.25 * np.exp(-u * u / (2 * sigma ** 2))
    np.testing.assert_allclose(dg, (gg(t + h) - gg(t - h)) / (2 * h), atol=1e-10)


# ------------------------------------------------------------------ STFT
@pytest.mark.parametrize("L", [33, 65, 161, 289])
def test_stft_matches_brute_force_eq8(L):
    """Eq. 9 (FFT, phase factor, folding for L > Nf, up to four and a half
    times Nf) against Eq. 8 summed directly on a tiny input."""
    n, hop, nfft = 256, 4, 64
    sigma = max(6.0, (L - 1) / 4.0)   # the window's ends carry weight (e^-2)
    x = np.random.default_rng(L).standard_normal(n)
    g, dg = O.window(L, sigma)
    V, Vd = O.stft(x, g, dg, hop, nfft, 0, nfft // 2)
    M = (L - 1) // 2
    F = O.frames(n, hop)
    j = np.arange(-M, M + 1)
    k = np.arange(nfft // 2 + 1)
    E = np.exp(-2j * np.pi * np.outer(j, k) / nfft)
    Vb = np.zeros_like(V)
    Vdb = np.zeros_like(V)
    for m in range(F):
        p = m * hop + j
        xs = np.where((p >= 0) & (p < n), x[np.clip(p, 0, n - 1)], 0.0)
        Vb[m] = (xs * g) @ E
        Vdb[m] = (xs * dg) @ E
    scale = np.abs(Vb).max()
    assert np.abs(V - Vb).max() <= 1e-12 * scale
    assert np.abs(Vd - Vdb).max() <= 1e-12 * np.abs(Vdb).max()


def test_stft_band_slice_equals_full():
    n, hop, nfft, L = 512, 8, 128, 97
    x = np.random.default_rng(3).standard_normal(n)
    g, dg = O.window(L, 12.0)
    Vf, Vdf = O.stft(x, g, dg, hop, nfft, 0, nfft // 2)
    Vb, Vdb = O.stft(x, g, dg, hop, nfft, 10, 40, m0=5, nm=20)
    np.testing.assert_array_equal(Vb, Vf[5:25, 10:41])
    np.testing.assert_array_equal(Vdb, Vdf[5:25, 10:41])


# ------------------------------------------------------------------ IF (Eq. 13)
@pytest.mark.parametrize("L,tol", [(1025, 3e-3), (2049, 1e-6)])
@pytest.mark.parametrize("offset", [0.0, 0.3, -0.45])
def test_tone_if_closed_form(offset, L, tol):
    """A stationary tone gives omega_hat = f0 in every bin of its lobe
    (Sec. 2.3, Eq. 17; Eq. 36 with a constant IF).  The only error is the
    window truncation: about 1e-3 bin at L = 8 sigma + 1, and nothing
    measurable at L = 16 sigma + 1 (folded mod Nf, reading R2)."""
    n, fs, nfft, sigma, hop = 16384, 25600.0, 1024, 128.0, 16
    k0 = 200 + offset
    x = S.tone(n, fs, k0 * fs / nfft, phase=0.4)
    g, dg = O.window(L, sigma)
    V, Vd = O.stft(x, g, dg, hop, nfft, 150, 250, m0=300, nm=8)
    om, _, _, _ = O.reassign(V, Vd, 150, 250, nfft, 1, 0.0)
    mag = np.abs(V)
    sel = mag >= 0.1 * mag.max(axis=1, keepdims=True)
    assert sel.sum() >= 8 * 4
    assert np.abs(om[sel] - k0).max() < tol


def test_gaussian_chirp_if_closed_form():
    """Complex linear chirp x = exp(i(w0 t + c t^2 / 2)), Gaussian window:
    omega_hat(u, xi) = w(u) + (xi - w(u)) c^2 s^4 / (1 + c^2 s^4), derived
    from Eq. 1 and Eq. 34; it equals the chirp's IF on the ridge."""
    n, nfft, L, sigma, hop = 32768, 1024, 1025, 128.0, 64
    w0 = 2 * np.pi * 100 / nfft               # rad / sample
    c = 2 * np.pi * 200 / nfft / n            # rad / sample^2 (100 -> 300 bins)
    t = np.arange(n, dtype=np.float64)
    x = np.exp(1j * (w0 * t + 0.5 * c * t * t))
    g, dg = O.window(L, sigma)
    # the oracle STFT takes real input; the complex chirp is the sum of the
    # transforms of its real and imaginary parts
    Vr, Vdr = O.stft(x.real, g, dg, hop, nfft, 0, nfft // 2)
    Vi, Vdi = O.stft(x.imag, g, dg, hop, nfft, 0, nfft // 2)
    V, Vd = Vr + 1j * Vi, Vdr + 1j * Vdi
    om, _, _, _ = O.reassign(V, Vd, 0, nfft // 2, nfft, 1, 0.0)
    F = V.shape[0]
    ms = np.arange(F // 4, 3 * F // 4)
    u = ms * hop
    wu = (w0 + c * u) * nfft / (2 * np.pi)   # IF in bins
    lam = (c * sigma ** 2) ** 2 / (1 + (c * sigma ** 2) ** 2)
    k = np.arange(nfft // 2 + 1)
    pred = wu[:, None] + (k[None, :] - wu[:, None]) * lam
    mag = np.abs(V[ms])
    sel = mag >= 0.1 * mag.max(axis=1, keepdims=True)
    err = np.abs(om[ms][sel] - pred[sel])
    assert err.max() < 2e-3
    # the bias term is not negligible: dropping it fails this test
    assert np.abs(om[ms][sel] - np.broadcast_to(wu[:, None], pred.shape)[sel]).max() > 5e-3


# ------------------------------------------------------------------ reassignment
def _brute_dest(omega, mag, k_lo, k_hi, z, gamma):
    """Eq. 28 by search: the grid point xi*[l] = k_lo + l/z nearest omega,
    accepted when within half a fine interval (a tie goes to the upper l)."""
    nbo = z * (k_hi - k_lo) + 1
    grid = k_lo + np.arange(nbo) / z
    out = np.full(omega.shape, -1, dtype=np.int64)
    for idx in np.ndindex(omega.shape):
        if not mag[idx] > gamma:
            continue
        d = np.abs(omega[idx] - grid)
        cand = np.nonzero(d <= 0.5 / z + 1e-12)[0]
        out[idx] = cand.max() if len(cand) else -2
    return out


@pytest.mark.parametrize("z,band", [(1, (0, 64)), (2, (10, 40)), (3, (5, 50)), (4, (0, 32)), (7, (20, 64)),
                                    (16, (0, 64))])
def test_reassign_brute_force(z, band):
    n, hop, nfft, L = 1024, 8, 128, 97
    x = np.random.default_rng(z).standard_normal(n)
    g, dg = O.window(L, 12.0)
    k_lo, k_hi = band
    V, Vd = O.stft(x, g, dg, hop, nfft, k_lo, k_hi)
    gamma = 0.05 * np.abs(V).max()
    om, dest, T, leak = O.reassign(V, Vd, k_lo, k_hi, nfft, z, gamma)
    bd = _brute_dest(om, np.abs(V), k_lo, k_hi, z, gamma)
    assert np.array_equal(dest, bd)
    # T by explicit accumulation in ascending k
    nbo = z * (k_hi - k_lo) + 1
    Tb = np.zeros((V.shape[0], nbo), dtype=complex)
    Lb = np.zeros(V.shape[0], dtype=complex)
    for m in range(V.shape[0]):
        for i in range(V.shape[1]):
            if bd[m, i] >= 0:
                Tb[m, bd[m, i]] += V[m, i]
            elif bd[m, i] == -2:
                Lb[m] += V[m, i]
    np.testing.assert_allclose(T, Tb, atol=1e-13 * np.abs(V).max())
    np.testing.assert_allclose(leak, Lb, atol=1e-13 * np.abs(V).max())


def test_mass_invariant():
    """sum_l T[m,l] + leak[m] = sum of in-band coefficients above threshold."""
    x, _ = S.chirp_fm_mix(8192)
    g, dg = O.window(257, 32.0)
    V, Vd = O.stft(x, g, dg, 16, 256, 20, 100)
    gamma = 1e-2 * np.abs(V).max()
    _, dest, T, leak = O.reassign(V, Vd, 20, 100, 256, 2, gamma)
    kept = np.where(np.abs(V) > gamma, V, 0)
    np.testing.assert_allclose(T.sum(axis=1) + leak, kept.sum(axis=1),
                               atol=1e-12 * np.abs(V).max())
    assert (dest == -2).any() and (dest >= 0).any()


def test_tone_single_destination():
    """A tone on a bin centre puts its whole above-threshold lobe into one bin
    (Eq. 17: the SST of a stationary tone is a delta at its IF)."""
    n, fs, nfft, L, sigma, hop = 16384, 25600.0, 1024, 1025, 128.0, 16
    x = S.tone(n, fs, 300 * fs / nfft)
    g, dg = O.window(L, sigma)
    V, Vd = O.stft(x, g, dg, hop, nfft, 0, 512, m0=200, nm=16)
    gamma = 1e-3 * np.abs(V).max()
    _, dest, T, leak = O.reassign(V, Vd, 0, 512, nfft, 1, gamma)
    kept = np.where(np.abs(V) > gamma, V, 0)
    np.testing.assert_allclose(T[:, 300], kept.sum(axis=1), rtol=1e-12)
    assert np.abs(np.delete(T, 300, axis=1)).max() < 1e-12 * np.abs(T[:, 300]).min()


def test_odd_subdivision_coarsens_to_z1():
    """For odd z the fine cells of Eq. 29 tile the coarse cells of Eq. 27:
    T_z1[q] = T_z3[3q-1] + T_z3[3q] + T_z3[3q+1] away from the grid edges."""
    x, _ = S.chirp_fm_mix(8192)
    g, dg = O.window(257, 32.0)
    k_lo, k_hi = 10, 120
    V, Vd = O.stft(x, g, dg, 16, 256, k_lo, k_hi)
    gamma = 1e-3 * np.abs(V).max()
    _, _, T1, _ = O.reassign(V, Vd, k_lo, k_hi, 256, 1, gamma)
    _, _, T3, _ = O.reassign(V, Vd, k_lo, k_hi, 256, 3, gamma)
    q = np.arange(1, k_hi - k_lo)
    coarse = T3[:, 3 * q - 1] + T3[:, 3 * q] + T3[:, 3 * q + 1]
    np.testing.assert_allclose(T1[:, q], coarse, atol=1e-12 * np.abs(V).max())


def test_full_band_z1_is_eq14():
    """Eq. 27 over the full band with z = 1 is Eq. 14: nearest coarse bin."""
    n, hop, nfft, L = 2048, 16, 256, 129
    x = np.random.default_rng(11).standard_normal(n)
    g, dg = O.window(L, 16.0)
    V, Vd = O.stft(x, g, dg, hop, nfft, 0, nfft // 2)
    gamma = 1e-2 * np.abs(V).max()
    om, dest, T, _ = O.reassign(V, Vd, 0, nfft // 2, nfft, 1, gamma)
    near = np.floor(om + 0.5)
    ok = (np.abs(V) > gamma) & (near >= 0) & (near <= nfft // 2)
    assert np.array_equal(dest[ok], near[ok].astype(np.int32))
    assert np.all(dest[np.abs(V) <= gamma] == -1)


def test_threshold_extremes():
    x = np.random.default_rng(5).standard_normal(1024)
    g, dg = O.window(65, 8.0)
    V, Vd = O.stft(x, g, dg, 8, 64, 0, 32)
    _, dest, T, _ = O.reassign(V, Vd, 0, 32, 64, 2, np.abs(V).max() * (1 + 1e-12))
    assert np.all(dest == -1) and not T.any()
    _, dest, _, _ = O.reassign(V, Vd, 0, 32, 64, 2, 0.0)
    assert np.all(dest != -1)


# ------------------------------------------------------------------ inverse
def test_wola_exact_reconstruction():
    """Eq. 10-11: STFT synthesis with the window and normaliser sum g^2
    recovers the signal exactly for L <= Nf."""
    n, hop, nfft, L = 4096, 16, 512, 257
    x = np.random.default_rng(9).standard_normal(n)
    g, dg = O.window(L, 32.0)
    V, _ = O.stft(x, g, dg, hop, nfft, 0, nfft // 2)
    xr = O.inverse(V, 0, nfft, 1, g, hop, n, mode=1)
    assert np.abs(xr - x).max() < 1e-12


def test_normaliser_continuous_limit_eq22():
    """Eq. 22: g(0) * integral g = sqrt(2) for the unit-energy Gaussian, so in
    the interior D[p] * hop -> sqrt(2) when sigma >> hop (and the window is
    long enough, here 16 sigma + 1, for its truncation not to show)."""
    L, sigma, hop, n = 2049, 128.0, 16, 8192
    g, _ = O.window(L, sigma)
    D = O.normaliser(g, hop, n, 2048, 4096)
    np.testing.assert_allclose(D * hop, math.sqrt(2.0), rtol=1e-10)


@pytest.mark.parametrize("L", [49, 161, 289])
def test_inverse_matches_brute_force_eq25(L):
    """The zNf-point zero-padded IDFT route against Eq. 25-26 summed directly
    over the fine bins, on a tiny input, for several z; windows shorter than
    Nf and longer than zNf (taps |j| > zNf / 2, where the IDFT route reads
    its transform periodically and the direct sum needs no period)."""
    n, hop, nfft = 512, 8, 64
    x = np.random.default_rng(21).standard_normal(n)
    g, dg = O.window(L, max(6.0, (L - 1) / 4.0))   # long windows: ends of weight e^-2
    M = (L - 1) // 2
    for z, (k_lo, k_hi) in ((1, (0, 32)), (2, (4, 20)), (3, (0, 12)), (4, (10, 32)), (7, (20, 32)), (16, (0, 32))):
        V, Vd = O.stft(x, g, dg, hop, nfft, k_lo, k_hi)
        _, _, T, _ = O.reassign(V, Vd, k_lo, k_hi, nfft, z, 0.0)
        xr = O.inverse(T, k_lo, nfft, z, g, hop, n)
        F = T.shape[0]
        nbo = T.shape[1]
        xi = k_lo + np.arange(nbo) / z                  # fine-bin centres, coarse units
        w = np.where((xi == 0) | (xi == nfft / 2), 0.5, 1.0)
        j = np.arange(-M, M + 1)
        E = np.exp(2j * np.pi * np.outer(xi, j) / nfft)
        num = np.zeros(n)
        den = np.zeros(n)
        for m in range(F):
            r = (2.0 / nfft) * np.real((w * T[m]) @ E)
            p = m * hop + j
            ok = (p >= 0) & (p < n)
            num[p[ok]] += g[ok] * r[ok]
            den[p[ok]] += g[M] * g[ok]
        np.testing.assert_allclose(xr, num / den, atol=1e-12 * np.abs(num / den).max())


def test_inverse_independent_of_thread_count():
    """The inverse computes each frame's r~ (Eq. 25) in parallel and
    overlap-adds them in ascending frame order (Eq. 26): one thread and all
    threads give the same bits, over several frame chunks and a sub-range."""
    n, hop, nfft, L, z = 6000, 5, 128, 97, 2
    x = np.random.default_rng(31).standard_normal(n)
    g, dg = O.window(L, 12.0)
    k_lo, k_hi = 3, 50
    V, Vd = O.stft(x, g, dg, hop, nfft, k_lo, k_hi)
    _, _, T, _ = O.reassign(V, Vd, k_lo, k_hi, nfft, z, 1e-3 * np.abs(V).max())
    before = O.get_threads()
    try:
        O.set_threads(1)
        one = O.inverse(T, k_lo, nfft, z, g, hop, n)
        part1 = O.inverse(T, k_lo, nfft, z, g, hop, n, p0=1234, np_=2345)
        O.set_threads(0)
        many = O.inverse(T, k_lo, nfft, z, g, hop, n)
        partn = O.inverse(T, k_lo, nfft, z, g, hop, n, p0=1234, np_=2345)
    finally:
        O.set_threads(before)
    assert T.shape[0] > 3 * 256   # several chunks of frames
    assert np.array_equal(one, many)
    assert np.array_equal(part1, partn)
    assert np.array_equal(one[1234:1234 + 2345], part1)


@pytest.mark.parametrize("z,frac", [(1, 0.0), (2, 0.5), (4, 0.25)])
def test_inverse_reconstructs_tone(z, frac):
    """A tone on a (fine) bin centre is squeezed into one bin and the direct
    inverse returns it: T ~ (A/2) Nf g(0) e^{i w m hop} gives r~ = A g(0) cos,
    and dividing the overlap-add by D gives back x (Sec. 2.3, Eq. 17-26).
    The window is 16 sigma + 1 long (folded, reading R2) so that its
    truncation does not limit the comparison."""
    n, fs, nfft, L, sigma, hop = 16384, 25600.0, 1024, 2049, 128.0, 16
    x = S.tone(n, fs, (200 + frac) * fs / nfft, amp=0.8, phase=1.1)
    r = O.sst(x, fs, L, sigma, hop, nfft, 0.0, fs / 2 if z == 1 else 6400.0, z,
              0.0, False, inverse_range=(0, n))
    inner = slice(4096, n - 4096)
    assert np.abs(r.xhat[inner] - x[inner]).max() < 1e-9


def test_column_sum_inverse_exact_eq15():
    """Ht = 1, Nf = N, gamma = 0, full band: the Eq. 15 column sum returns
    the signal exactly when no mass enters or leaves the DC/Nyquist bins and
    nothing leaks (conditions checked, and their mass bounds the error)."""
    n, L, sigma = 1024, 257, 32.0
    nfft, hop = n, 1
    t = np.arange(n)
    x = (np.cos(2 * np.pi * 211.3 * t / n + 0.3) + 0.5 * np.cos(2 * np.pi * 305.7 * t / n)
         + 0.25 * np.cos(2 * np.pi * (150 * t + 40 * t * t / n) / n))
    g, dg = O.window(L, sigma)
    V, Vd = O.stft(x, g, dg, hop, nfft, 0, nfft // 2)
    _, dest, T, leak = O.reassign(V, Vd, 0, nfft // 2, nfft, 1, 0.0)
    xc = O.colsum(T, 0, nfft, 1, g[(L - 1) // 2])
    k = np.arange(nfft // 2 + 1)
    edge = (dest == -2) | ((dest == 0) != (k == 0)) | ((dest == nfft // 2) != (k == nfft // 2))
    bound = 4.0 * np.where(edge, np.abs(V), 0).sum(axis=1) / (nfft * g[(L - 1) // 2])
    err = np.abs(xc - x)
    assert np.all(err <= bound + 1e-11)
    clean = bound == 0.0
    assert clean.sum() >= 100          # the bound is not vacuous
    assert err[clean].max() < 1e-12


def test_column_sum_vs_direct_inverse_at_ht1():
    """The Eq. 26 path at Ht = 1 and the Eq. 15 column sum reconstruct the
    same noisy multicomponent signal with nearly the same SNR (Sec. 3.3)."""
    n, fs = 4096, 1024.0
    x1, x2, x3, *_ = S.paper_three_component(n, fs)
    clean = x1 + x2 + x3
    noisy = S.add_noise(clean, 10.0, S.rng(99))
    nfft, L, sigma = n, 257, 0.03 * fs
    r = O.sst(noisy, fs, L, sigma, 1, nfft, 0.0, fs / 2, 1, 1e-3, True,
              inverse_range=(0, n))
    g, _ = O.window(L, sigma)
    xc = O.colsum(r.T, 0, nfft, 1, g[(L - 1) // 2])
    snr = lambda y: 10 * np.log10(np.sum(clean ** 2) / np.sum((clean - y) ** 2))
    inner = slice(512, n - 512)
    s_direct = 10 * np.log10(np.sum(clean[inner] ** 2) / np.sum((clean - r.xhat)[inner] ** 2))
    s_col = 10 * np.log10(np.sum(clean[inner] ** 2) / np.sum((clean - xc)[inner] ** 2))
    assert s_col > 9.0 and s_direct > 9.0
    assert abs(s_direct - s_col) < 1.5
    assert snr(r.xhat) > 5.0


# ------------------------------------------------------------------ printed numbers
def _golden():
    out = {}
    with open(os.path.join(GOLDEN, "paper_numbers.txt")) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            name, val, tol, *_ = line.split()
            out[name] = (float(val), float(tol))
    return out


def test_parameter_relations_match_printed_numbers():
    gd = _golden()

    def check(name, value):
        v, tol = gd[name]
        assert abs(value - v) <= tol, (name, value, v)

    check("sigma_f_sim_hz", O.sigma_f(0.03))
    check("support_6sigma_f_hz", 6 * O.sigma_f(0.03))
    r1 = O.hf_max_rule1(8192, 0.03, 1024)
    assert 63 < r1 < 64
    check("hf_max_rule1_sim", r1)
    check("hf_max_rule2_sim", O.hf_max_rule2(8192, 0.03, 1024))
    check("hf_max_rule1_aero", O.hf_max_rule1(9035089, 0.02, 44100))
    check("hf_aero", 9035089 / 2 ** 13)
    check("delta_f_aero_hz", O.delta_f(44100, 2 ** 13, 8))
    check("delta_f_chatter_hz", O.delta_f(10240, 2 ** 15, 1))
    check("half_interval_hf70_hz", O.delta_f(1024, 8192 // 70, 1) / 2)

"""The synthetic inputs against their stated recipe (CPU): noise at exactly
the requested SNR, pink noise with a 1/f power spectrum, the run-up's order
track, the chirp / FM mixture's components where the recipe puts them, the
paper's Eq. 30 signal continuous where its second component switches law
(Eq. 31), and seeded streams that are reproducible and distinct."""
import numpy as np
import pytest

from paper_2003_07065_gb300 import signals as S


@pytest.mark.parametrize("pink", [False, True])
@pytest.mark.parametrize("snr_db", [0.0, 5.0, 10.0])
def test_noise_snr_is_exact(pink, snr_db):
    clean = S.tone(1 << 15, 1000.0, 37.0)
    noisy = S.add_noise(clean, snr_db, S.rng(9, 1), pink=pink)
    noise = noisy - clean
    got = 10 * np.log10(np.mean(clean ** 2) / np.mean(noise ** 2))
    assert abs(got - snr_db) < 1e-9


def test_pink_noise_has_a_one_over_f_spectrum():
    n = 1 << 18
    w = S.add_noise(np.zeros(n) + 1e-3, 0.0, S.rng(9, 2), pink=True) - 1e-3
    P = np.abs(np.fft.rfft(w)) ** 2
    f = np.arange(len(P))
    # average the power in octave bands and fit log P against log f
    edges = 2 ** np.arange(4, 16)
    fc = np.sqrt(edges[:-1] * edges[1:])
    Pb = np.array([P[a:b].mean() for a, b in zip(edges[:-1], edges[1:])])
    slope = np.polyfit(np.log(fc), np.log(Pb), 1)[0]
    assert abs(slope + 1.0) < 0.05


def _peak_hz(x, fs, centre, nwin=8192):
    seg = x[centre - nwin // 2:centre + nwin // 2] * np.hanning(nwin)
    spec = np.abs(np.fft.rfft(seg))
    k = int(np.argmax(spec))
    # parabolic interpolation of the peak
    a, b, c = np.log(spec[k - 1:k + 2] + 1e-300)
    return (k + 0.5 * (a - c) / (a - 2 * b + c)) * fs / nwin


def test_runup_order_one_track():
    """Shaft speed f_r ramps linearly 20 -> 200 Hz over the record; order 1
    (amplitude 1) is the strongest component below 1 kHz."""
    n, fs = 1 << 20, 51200.0
    _, clean = S.runup(n, fs)
    dur = n / fs
    for frac in (0.25, 0.5, 0.75):
        c = int(frac * n)
        low = np.fft.irfft(np.fft.rfft(clean) * (np.fft.rfftfreq(n, 1 / fs) < 1000.0), n)
        assert abs(_peak_hz(low, fs, c, 16384) - (20.0 + 180.0 * c / fs / dur)) < 1.0


def test_chirp_fm_components():
    n, fs = 65536, 25600.0
    noisy, clean = S.chirp_fm_mix(n, fs)
    dur = n / fs
    lp = np.fft.irfft(np.fft.rfft(clean) * (np.fft.rfftfreq(n, 1 / fs) < 3000.0), n)
    for frac in (0.3, 0.6):
        c = int(frac * n)
        assert abs(_peak_hz(lp, fs, c, 4096) - (500.0 + 1500.0 * c / fs / dur)) < 6.0
    hp = clean - lp
    spec = np.abs(np.fft.rfft(hp)) ** 2
    f = np.fft.rfftfreq(n, 1 / fs)
    band = (f > 3600) & (f < 4400)
    assert spec[band].sum() > 0.999 * spec.sum()
    # power-weighted mean frequency = the time average of the IF 4000 + 300 cos(2 pi 3 t)
    # over the record (2.56 s, not a whole number of modulation periods)
    T = n / fs
    want = 4000.0 + 300.0 * np.sin(2 * np.pi * 3.0 * T) / (2 * np.pi * 3.0 * T)
    assert abs(np.sum(f[band] * spec[band]) / np.sum(spec[band]) - want) < 0.5
    # Carson's rule: ~98 % of the power within 4000 +- (300 + 3) Hz
    cum = np.cumsum(spec[band]) / spec[band].sum()
    fb = f[band]
    assert fb[np.searchsorted(cum, 0.005)] > 3680 and fb[np.searchsorted(cum, 0.995)] < 4320
    assert 10 * np.log10(np.mean(clean ** 2) / np.mean((noisy - clean) ** 2)) == pytest.approx(10.0, abs=1e-9)


def test_paper_signal_continuous_at_the_switch():
    """Eq. 30's second component changes law at t = 4 s: its phase and IF
    (Eq. 31) are continuous there."""
    fs = 1024.0
    x1, x2, x3, f1, f2, f3 = S.paper_three_component(8192, fs)
    i = int(4 * fs)
    assert f2[i - 1] == pytest.approx(150.0 + 25.0 / fs, abs=1e-9)
    assert f2[i] == pytest.approx(150.0, abs=1e-12)
    # the phase just below and at t = 4 s (the sample jump is the IF times one sample)
    dphi = np.angle(np.exp(1j * (np.arccos(np.clip(x2[i], -1, 1)) - np.arccos(np.clip(x2[i - 1], -1, 1)))))
    assert abs(abs(dphi) - 2 * np.pi * 150.0 / fs) < 2e-2
    assert f1.min() == f1.max() == 50.0
    assert f3.min() >= 270.0 - 1e-9 and f3.max() <= 470.0 + 1e-9


def test_seeded_streams_reproducible_and_distinct():
    a = S.rng(2, 0).standard_normal(8)
    b = S.rng(2, 0).standard_normal(8)
    c = S.rng(2, 1).standard_normal(8)
    d = S.rng(3, 0).standard_normal(8)
    np.testing.assert_array_equal(a, b)
    assert not np.allclose(a, c) and not np.allclose(a, d)

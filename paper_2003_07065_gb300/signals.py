"""Seeded synthetic input signals.

This module only synthesises test and benchmark inputs; it holds none of the
transform's arithmetic, so both the CUDA path and the FP64 oracle can take
their inputs from it.  Every generator is deterministic for a given
``(workload, channel)`` seed.  Noise levels are set as the ratio of mean-square
signal power to mean-square noise power over the whole record.
"""
from __future__ import annotations

import numpy as np

SEED_BASE = 0x2003070650000000


def rng(workload: int, channel: int = 0) -> np.random.Generator:
    """Counter-free PCG64 stream keyed by (workload, channel)."""
    return np.random.Generator(np.random.PCG64(
        np.random.SeedSequence([SEED_BASE & 0xFFFFFFFF, SEED_BASE >> 32,
                                int(workload), int(channel)])))


def add_noise(clean: np.ndarray, snr_db: float, gen: np.random.Generator,
              pink: bool = False) -> np.ndarray:
    """clean + white (or 1/f-power pink) Gaussian noise at the given SNR."""
    n = len(clean)
    w = gen.standard_normal(n)
    if pink:
        spec = np.fft.rfft(w)
        f = np.arange(len(spec), dtype=np.float64)
        shape = np.zeros_like(f)
        shape[1:] = 1.0 / np.sqrt(f[1:])
        w = np.fft.irfft(spec * shape, n)
    ps = np.mean(clean * clean)
    pn = np.mean(w * w)
    if pn == 0.0:
        return clean.copy()
    scale = np.sqrt(ps / (pn * 10.0 ** (snr_db / 10.0)))
    return clean + scale * w


def tone(n: int, fs: float, f0: float, amp: float = 1.0, phase: float = 0.0,
         complex_: bool = False) -> np.ndarray:
    t = np.arange(n) / fs
    if complex_:
        return amp * np.exp(1j * (2 * np.pi * f0 * t + phase))
    return amp * np.cos(2 * np.pi * f0 * t + phase)


def linear_chirp(n: int, fs: float, f0: float, f1: float, amp: float = 1.0,
                 complex_: bool = False) -> np.ndarray:
    """Frequency ramps linearly from f0 at t=0 to f1 at t=n/fs."""
    t = np.arange(n) / fs
    dur = n / fs
    ph = 2 * np.pi * (f0 * t + 0.5 * (f1 - f0) / dur * t * t)
    return amp * (np.exp(1j * ph) if complex_ else np.cos(ph))


def chirp_fm_mix(n: int = 65536, fs: float = 25600.0, snr_db: float = 10.0,
                 seed=(1, 0)):
    """Linear chirp 500->2000 Hz (amplitude 1) + sinusoidal-FM tone at
    4000 Hz +/- 300 Hz with 3 Hz modulation (amplitude 0.7) + white noise.

    Returns (noisy, clean) float64 arrays."""
    t = np.arange(n) / fs
    clean = linear_chirp(n, fs, 500.0, 2000.0, 1.0)
    clean = clean + 0.7 * np.cos(2 * np.pi * 4000.0 * t
                                 + (300.0 / 3.0) * np.sin(2 * np.pi * 3.0 * t))
    noisy = add_noise(clean, snr_db, rng(*seed))
    return noisy, clean


def runup(n: int = 1 << 24, fs: float = 51200.0, snr_db: float = 5.0,
          seed=(2, 0)):
    """Run-up vibration: shaft speed f_r ramps 20 -> 200 Hz linearly over the
    record; orders 1, 2, 3.5, 7 with amplitudes 1, 0.5, 0.3, 0.2; a 3.2 kHz
    resonance amplitude-modulated by order 1; pink noise.

    Returns (noisy, clean) float64 arrays."""
    t = np.arange(n) / fs
    dur = n / fs
    phi1 = 2 * np.pi * (20.0 * t + 0.5 * (180.0 / dur) * t * t)
    clean = np.zeros(n)
    for order, amp in ((1.0, 1.0), (2.0, 0.5), (3.5, 0.3), (7.0, 0.2)):
        clean += amp * np.cos(order * phi1)
    clean += 0.5 * (1.0 + 0.5 * np.cos(phi1)) * np.cos(2 * np.pi * 3200.0 * t)
    noisy = add_noise(clean, snr_db, rng(*seed), pink=True)
    return noisy, clean


def paper_three_component(n: int = 8192, fs: float = 1024.0):
    """The three AM-FM components of the paper's simulation (Eq. 30), and
    their instantaneous frequencies in Hz (Eq. 31).

    Returns (x1, x2, x3, f1, f2, f3)."""
    t = np.arange(n) / fs
    x1 = (1 - 0.1 * np.cos(0.25 * np.pi * t)) * np.cos(100 * np.pi * t)
    ph2 = np.where(t < 4,
                   500 * np.pi * t - 25 * np.pi * t ** 2,
                   500 * np.pi * t - 50 * np.pi * t ** 2
                   + 25.0 / 6.0 * np.pi * t ** 3 + 4.0 / 3.0 * np.pi)
    x2 = np.cos(ph2)
    x3 = (1 - 0.2 * np.cos(0.125 * np.pi * t)) * np.cos(
        740 * np.pi * t + 400.0 / 3.0 * np.sin(0.75 * np.pi * t)
        - 200 * np.sin(0.5 * np.pi * t))
    f1 = np.full(n, 50.0)
    f2 = np.where(t < 4, 250 - 25 * t, 250 - 50 * t + 6.25 * t ** 2)
    f3 = 370 + 50 * np.cos(0.75 * np.pi * t) - 50 * np.cos(0.5 * np.pi * t)
    return x1, x2, x3, f1, f2, f3


def random_mix(n: int, fs: float, f_lo: float, f_hi: float, gen: np.random.Generator):
    """1-4 components (linear chirp or sinusoidal FM) with frequencies inside
    [f_lo, f_hi], plus white noise at 0-20 dB.  Returns (noisy, clean)."""
    t = np.arange(n) / fs
    dur = n / fs
    width = f_hi - f_lo
    lo = f_lo + 0.1 * width
    hi = f_hi - 0.1 * width
    clean = np.zeros(n)
    for _ in range(int(gen.integers(1, 5))):
        amp = float(gen.uniform(0.3, 1.0))
        if gen.random() < 0.5:
            fa, fb = gen.uniform(lo, hi, size=2)
            ph = 2 * np.pi * (fa * t + 0.5 * (fb - fa) / dur * t * t)
        else:
            fc = float(gen.uniform(lo, hi))
            dev = float(gen.uniform(0.0, 0.3)) * min(fc - lo, hi - fc)
            rate = float(gen.uniform(0.5, 5.0))
            ph = 2 * np.pi * fc * t + (dev / rate) * np.sin(2 * np.pi * rate * t)
        clean += amp * np.cos(ph + float(gen.uniform(0, 2 * np.pi)))
    snr = float(gen.uniform(0.0, 20.0))
    return add_noise(clean, snr, gen), clean

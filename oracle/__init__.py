"""FP64 CPU oracle of the downsampled STFT-based synchrosqueezing transform.

TEST INFRASTRUCTURE ONLY.  This package is the slow, plain reference the CUDA
path is checked against.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import it;
the product library never does, and it shares no code with it.

The arithmetic lives in ``sst_oracle.c`` (plain C, double precision, its own
radix-2 FFT); this module only marshals numpy arrays through ctypes and maps
the user-level band in Hz to DFT bins.  Each function names the equation of
He & Cao (arXiv 2003.07065) it follows.
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
import sys
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "sst_oracle.c")
_LIB = os.path.join(_HERE, "_build", "libsst_oracle.so")
_lib = None

_dp = ctypes.POINTER(ctypes.c_double)
_ip = ctypes.POINTER(ctypes.c_int32)
_i64 = ctypes.c_int64
_int = ctypes.c_int


def build(force: bool = False) -> str:
    """Compile the oracle with gcc into ``oracle/_build`` (git-ignored)."""
    os.makedirs(os.path.dirname(_LIB), exist_ok=True)
    if (not force and os.path.exists(_LIB)
            and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC)):
        return _LIB
    tmp = _LIB + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-std=c11",
           "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is not None:
        return _lib
    build()
    lib = ctypes.CDLL(_LIB)
    lib.oro_window.argtypes = [_int, ctypes.c_double, _dp, _dp]
    lib.oro_fft.argtypes = [_dp, _dp, _i64, _int]
    lib.oro_frames.argtypes = [_i64, _int]
    lib.oro_frames.restype = _i64
    lib.oro_stft.argtypes = [_dp, _i64, _dp, _dp, _int, _int, _int, _i64, _i64,
                             _int, _int, _dp, _dp]
    lib.oro_reassign.argtypes = [_dp, _dp, _i64, _int, _int, _int, _int,
                                 ctypes.c_double, _dp, _ip, _dp, _dp]
    lib.oro_normaliser.argtypes = [_dp, _int, _int, _i64, _i64, _i64, _int, _dp]
    lib.oro_inverse.argtypes = [_dp, _i64, _i64, _int, _int, _int, _int, _dp,
                                _int, _int, _i64, _i64, _i64, _int, _dp]
    lib.oro_colsum.argtypes = [_dp, _i64, _int, _int, _int, _int,
                               ctypes.c_double, _dp]
    for name in ("oro_sigma_f",):
        getattr(lib, name).argtypes = [ctypes.c_double]
        getattr(lib, name).restype = ctypes.c_double
    for name in ("oro_hf_max_rule1", "oro_hf_max_rule2"):
        getattr(lib, name).argtypes = [ctypes.c_double] * 3
        getattr(lib, name).restype = ctypes.c_double
    lib.oro_set_threads.argtypes = [_int]
    lib.oro_set_threads.restype = None
    lib.oro_get_threads.argtypes = []
    lib.oro_get_threads.restype = _int
    lib.oro_delta_f.argtypes = [ctypes.c_double, _int, _int]
    lib.oro_delta_f.restype = ctypes.c_double
    _lib = lib
    return lib


def _p(a: np.ndarray):
    return a.ctypes.data_as(_dp)


def _c(a, dtype=np.float64) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=dtype)


def _cx(a: np.ndarray) -> np.ndarray:
    """complex128 array -> interleaved float64 view (contiguous)."""
    a = np.ascontiguousarray(a, dtype=np.complex128)
    return a.view(np.float64)


# ---------------------------------------------------------------- primitives
def set_threads(n: int) -> int:
    """OpenMP threads for the oracle's frame loops (0: all cores); returns the
    count now in effect.  Timing only: the results do not depend on it."""
    lib = _load()
    lib.oro_set_threads(int(n))
    return int(lib.oro_get_threads())


def get_threads() -> int:
    """OpenMP threads the oracle's frame loops use."""
    return int(_load().oro_get_threads())


def window(L: int, sigma: float):
    """Gaussian g (Sec. 2.1) and g' (Sec. 2.2) on j = -M..M, sigma in samples."""
    lib = _load()
    g = np.empty(L)
    dg = np.empty(L)
    if lib.oro_window(L, float(sigma), _p(g), _p(dg)) != 0:
        raise ValueError("bad window parameters")
    return g, dg


def fft(x: np.ndarray, sign: int = -1) -> np.ndarray:
    """The oracle's own radix-2 FFT (unnormalised, exp(sign 2 pi i k n / n))."""
    lib = _load()
    x = np.asarray(x, dtype=np.complex128)
    re = np.ascontiguousarray(x.real.copy())
    im = np.ascontiguousarray(x.imag.copy())
    if lib.oro_fft(_p(re), _p(im), len(x), sign) != 0:
        raise ValueError("fft size must be a power of two")
    return re + 1j * im


def frames(n: int, hop: int) -> int:
    return (n + hop - 1) // hop


def stft(x, g, dg, hop: int, nfft: int, k_lo: int, k_hi: int, m0: int = 0,
         nm: int | None = None):
    """Eq. 9 STFTs with windows g and g' for frames [m0, m0+nm), bins [k_lo, k_hi]."""
    lib = _load()
    x = _c(x)
    g = _c(g)
    dg = _c(dg)
    L = len(g)
    if nm is None:
        nm = frames(len(x), hop) - m0
    nb = k_hi - k_lo + 1
    V = np.zeros((nm, nb), dtype=np.complex128)
    Vd = np.zeros((nm, nb), dtype=np.complex128)
    rc = lib.oro_stft(_p(x), len(x), _p(g), _p(dg), L, hop, nfft, m0, nm,
                      k_lo, k_hi, _p(V.view(np.float64)), _p(Vd.view(np.float64)))
    if rc != 0:
        raise ValueError(f"oro_stft failed ({rc})")
    return V, Vd


def reassign(V, Vd, k_lo: int, k_hi: int, nfft: int, z: int, gamma: float):
    """Eq. 12-13 IF estimate and Eq. 27-29 reassignment.

    Returns (omega [bins], dest, T, leak)."""
    lib = _load()
    V = np.ascontiguousarray(V, dtype=np.complex128)
    Vd = np.ascontiguousarray(Vd, dtype=np.complex128)
    nm, nb = V.shape
    nbo = z * (k_hi - k_lo) + 1
    omega = np.empty((nm, nb))
    dest = np.empty((nm, nb), dtype=np.int32)
    T = np.zeros((nm, nbo), dtype=np.complex128)
    leak = np.zeros(nm, dtype=np.complex128)
    rc = lib.oro_reassign(_p(V.view(np.float64)), _p(Vd.view(np.float64)), nm,
                          k_lo, k_hi, nfft, z, float(gamma), _p(omega),
                          dest.ctypes.data_as(_ip), _p(T.view(np.float64)),
                          _p(leak.view(np.float64)))
    if rc != 0:
        raise ValueError("oro_reassign failed")
    return omega, dest, T, leak


def normaliser(g, hop: int, n: int, p0: int = 0, np_: int | None = None,
               mode: int = 0) -> np.ndarray:
    """Eq. 26 normaliser D[p] = g[0] sum_m g[p - m hop] (mode 0) or the Eq. 11
    WOLA normaliser sum_m g[p - m hop]^2 (mode 1)."""
    lib = _load()
    g = _c(g)
    if np_ is None:
        np_ = n - p0
    D = np.empty(np_)
    lib.oro_normaliser(_p(g), len(g), hop, frames(n, hop), p0, np_, mode, _p(D))
    return D


def inverse(T, k_lo: int, nfft: int, z: int, g, hop: int, n: int,
            p0: int = 0, np_: int | None = None, mt0: int = 0, mode: int = 0):
    """Eq. 25-26 direct inverse (zNf-point zero-padded IDFT, P. 223).

    T holds frames [mt0, mt0 + len(T)); output samples [p0, p0 + np_)."""
    lib = _load()
    T = np.ascontiguousarray(T, dtype=np.complex128)
    g = _c(g)
    ntf, nbo = T.shape
    if np_ is None:
        np_ = n - p0
    out = np.empty(np_)
    rc = lib.oro_inverse(_p(T.view(np.float64)), mt0, ntf, k_lo, nbo, nfft, z,
                         _p(g), len(g), hop, n, p0, np_, mode, _p(out))
    if rc != 0:
        raise ValueError(f"oro_inverse failed ({rc})")
    return out


def colsum(T, k_lo: int, nfft: int, z: int, g0: float) -> np.ndarray:
    """Eq. 15 column-sum inverse over the whole grid (hop = 1)."""
    lib = _load()
    T = np.ascontiguousarray(T, dtype=np.complex128)
    nm, nbo = T.shape
    out = np.empty(nm)
    lib.oro_colsum(_p(T.view(np.float64)), nm, k_lo, nbo, nfft, z, float(g0), _p(out))
    return out


def sigma_f(sigma_s: float) -> float:
    """Eq. 35."""
    return _load().oro_sigma_f(sigma_s)


def hf_max_rule1(n: float, sigma_s: float, fs: float) -> float:
    """Eq. 38."""
    return _load().oro_hf_max_rule1(n, sigma_s, fs)


def hf_max_rule2(n: float, sigma_s: float, fs: float) -> float:
    """Eq. 46 restated as a bound on Hf."""
    return _load().oro_hf_max_rule2(n, sigma_s, fs)


def delta_f(fs: float, nfft: int, z: int = 1) -> float:
    """Eq. 12 / Eq. 28 frequency interval in Hz."""
    return _load().oro_delta_f(fs, nfft, z)


# ------------------------------------------------- after the path: zones,
# ridges, concentration (plain numpy in FP64 plus the inverse above)
def zone_mask(nbo: int, ridge, half_width: int) -> np.ndarray:
    """The zone M_q[m] of Eq. 15 as a boolean (frames x nbo) mask: output bin
    l of frame m belongs to it iff ridge[m] >= 0 and |l - ridge[m]| <=
    half_width (a band offset in both directions from the ridge, Sec. 2.2)."""
    ridge = np.asarray(ridge, dtype=np.int64)
    l = np.arange(nbo)[None, :]
    c = ridge[:, None]
    return (c >= 0) & (np.abs(l - c) <= half_width)


def zone_inverse(T, ridge, half_width: int, k_lo: int, nfft: int, z: int, g, hop: int,
                 n: int, p0: int = 0, np_: int | None = None, mt0: int = 0):
    """Component recovery by time-frequency filtering (the closing paragraph
    of Sec. 2.3): the Eq. 25-26 inverse of T with every coefficient outside
    the zone of Eq. 15 set to zero.  ridge[i] belongs to frame mt0 + i."""
    T = np.asarray(T, dtype=np.complex128)
    Tq = np.where(zone_mask(T.shape[1], ridge, half_width), T, 0.0)
    return inverse(Tq, k_lo, nfft, z, g, hop, n, p0, np_, mt0)


def ridge(T, l_lo: int, l_hi: int, smooth: int) -> np.ndarray:
    """Ridge of one component, one output bin per frame (reading: the paper
    extracts ridges, Sec. 2.2 and Sec. 5, without stating how).  The energy
    E[m, l] = sum over |d| <= smooth (frames inside [0, F)) of |T[m + d, l]|^2
    is maximised over l in [l_lo, l_hi]; ties go to the smallest l; a frame
    with E = 0 throughout the band gets -1."""
    P = np.abs(np.asarray(T, dtype=np.complex128)) ** 2
    F = P.shape[0]
    band = P[:, l_lo:l_hi + 1]
    out = np.empty(F, dtype=np.int64)
    for m in range(F):
        a, b = max(0, m - smooth), min(F, m + smooth + 1)
        E = band[a:b].sum(axis=0)
        i = int(np.argmax(E))   # first of the maxima
        out[m] = l_lo + i if E[i] > 0.0 else -1
    return out


def ridge_hz(ridge_bins, k_lo: int, z: int, fs: float, nfft: int) -> np.ndarray:
    """Frequency of output bin l: (k_lo + l / z) fs / Nf (Eq. 28's fine grid)."""
    r = np.asarray(ridge_bins, dtype=np.float64)
    return np.where(r >= 0, (k_lo + r / z) * fs / nfft, np.nan)


def renyi(T, alpha: float = 3.0, cell: float = 1.0) -> float:
    """Renyi entropy of order alpha (Eq. 32) of the distribution P = |T|^2 on
    the TF grid: (1 / (1 - alpha)) log2 sum (P / sum P)^alpha, plus log2 of the
    grid cell's area (du dxi) when the integrals are read as sums over cells
    of that area (cell = 1: the plain discrete form)."""
    if alpha <= 0 or alpha == 1:
        raise ValueError("alpha must be positive and not 1")
    P = np.abs(np.asarray(T, dtype=np.complex128)) ** 2
    tot = P.sum()
    if tot <= 0:
        raise ValueError("empty distribution")
    p = P / tot
    return float(np.log2(np.sum(p ** alpha)) / (1.0 - alpha) + np.log2(cell))


# ------------------------------------------------------- second-order IF
# The paper names a second-order extension as future work (Sec. 6) without
# formulas.  Written here from the STFT's derivatives in the paper's
# convention, V^h[m, k] = sum_j x[m H + j] h[j] e^{-i w j} (Eq. 8-9, phase
# measured from the frame centre, w = 2 pi k / Nf): for any window h,
# d/dt V^h = -V^{h'} + i w V^h, d/dw V^h = -i V^{t h}.  Hence the complex IF
# w~ = w + i V^{g'}/V (its real part is Eq. 13), the complex time
# t~ = t + V^{tg}/V, and the local chirp rate
# q~ = (d/dt w~) / (d/dt t~) = i ((V^{g'})^2 - V^{g''} V) / (V^{tg} V^{g'} - V^{tg'} V);
# the second-order IF is Re(w~ + q~ (t - t~)) = Re(w~ - q~ V^{tg}/V), which a
# linear chirp returns exactly.
def window2(L: int, sigma: float):
    """g'' = (j^2/sigma^4 - 1/sigma^2) g, t g = j g and t g' = j g' on j = -M..M
    (derivatives of the Gaussian of Sec. 2.1, in samples)."""
    g, dg = window(L, sigma)
    j = np.arange(L, dtype=np.float64) - (L - 1) // 2
    return g, dg, (j * j / sigma ** 4 - 1.0 / sigma ** 2) * g, j * g, j * dg


IF2_MIN_DT = 1e-3   # |d/dt t~| = |V^{tg} V^{g'} - V^{tg'} V| / |V|^2 below this: first order


def if2(x, L: int, sigma: float, hop: int, nfft: int, k_lo: int, k_hi: int, m0: int = 0,
        nm: int | None = None):
    """First- and second-order IF estimates in coarse bins for frames
    [m0, m0 + nm), bins [k_lo, k_hi], with V.  Where the complex time barely
    moves with t (|d/dt t~| <= IF2_MIN_DT, e.g. at an impulse) the chirp rate
    is ill-conditioned and the second-order value is the first-order one.
    Returns (V, omega1, omega2, q) with q in bins per sample."""
    g, dg, d2g, tg, tdg = window2(L, sigma)
    V, Vd = stft(x, g, dg, hop, nfft, k_lo, k_hi, m0, nm)
    V2, Vt = stft(x, d2g, tg, hop, nfft, k_lo, k_hi, m0, nm)
    Vtd, _ = stft(x, tdg, tdg, hop, nfft, k_lo, k_hi, m0, nm)
    k = np.arange(k_lo, k_hi + 1, dtype=np.float64)[None, :]
    w = 2 * np.pi * k / nfft
    with np.errstate(divide="ignore", invalid="ignore"):
        wt = w + 1j * Vd / V
        den = Vt * Vd - Vtd * V
        q = 1j * (Vd * Vd - V2 * V) / den
        w2 = np.where(np.abs(den) > IF2_MIN_DT * np.abs(V) ** 2, (wt - q * Vt / V).real, wt.real)
        to_bins = nfft / (2 * np.pi)
        return V, wt.real * to_bins, w2 * to_bins, q * to_bins   # (q is not finite where den = 0)


def reassign2(V, omega2, k_lo: int, k_hi: int, z: int, gamma: float):
    """Eq. 27-29 with the second-order IF: each source with |V| > gamma goes to
    l = floor(z (omega2 - k_lo) + 1/2) when 0 <= l <= z N_r.  Returns (dest, T)
    with dest -1 below the threshold, -2 off the grid."""
    V = np.asarray(V, dtype=np.complex128)
    nm, nb = V.shape
    nbo = z * (k_hi - k_lo) + 1
    dest = np.full((nm, nb), -1, dtype=np.int64)
    T = np.zeros((nm, nbo), dtype=np.complex128)
    for m in range(nm):
        for kk in range(nb):
            if not abs(V[m, kk]) > gamma or not np.isfinite(omega2[m, kk]):
                continue
            l = int(np.floor(z * (omega2[m, kk] - k_lo) + 0.5))
            if 0 <= l < nbo:
                dest[m, kk] = l
                T[m, l] += V[m, kk]
            else:
                dest[m, kk] = -2
    return dest, T


# ---------------------------------------------------------------- pipeline
def band_bins(fs: float, nfft: int, f_lo: float, f_hi: float):
    """Band [f_lo, f_hi] Hz -> inclusive coarse bins, rounding half up."""
    k_lo = int(math.floor(f_lo * nfft / fs + 0.5))
    k_hi = int(math.floor(f_hi * nfft / fs + 0.5))
    k_hi = min(k_hi, nfft // 2)
    return k_lo, k_hi


@dataclass
class Result:
    V: np.ndarray
    Vd: np.ndarray
    omega: np.ndarray
    dest: np.ndarray
    T: np.ndarray
    leak: np.ndarray
    gamma: float
    k_lo: int
    k_hi: int
    m0: int
    xhat: np.ndarray | None = None


def sst(x, fs: float, L: int, sigma: float, hop: int, nfft: int, f_lo: float,
        f_hi: float, z: int, gamma: float, relative: bool, m0: int = 0,
        nm: int | None = None, inverse_range: tuple[int, int] | None = None,
        gamma_abs: float | None = None) -> Result:
    """Whole path: Eq. 9 STFTs -> Eq. 13 IF + threshold -> Eq. 28 reassignment
    -> Eq. 25-26 inverse.

    With ``relative`` the threshold is gamma * max|V| over all frames and the
    in-band bins (computed over every frame even when only [m0, m0+nm) is
    returned), unless ``gamma_abs`` supplies the absolute threshold directly.
    ``inverse_range`` = (p0, np) asks for xhat on those samples; the frames
    [m0, m0+nm) must then cover them."""
    x = _c(x)
    n = len(x)
    g, dg = window(L, sigma)
    k_lo, k_hi = band_bins(fs, nfft, f_lo, f_hi)
    F = frames(n, hop)
    if nm is None:
        nm = F - m0
    V, Vd = stft(x, g, dg, hop, nfft, k_lo, k_hi, m0, nm)
    if gamma_abs is not None:
        gam = float(gamma_abs)
    elif relative:
        gam = gamma * global_max_abs_v(x, g, dg, hop, nfft, k_lo, k_hi)
    else:
        gam = float(gamma)
    omega, dest, T, leak = reassign(V, Vd, k_lo, k_hi, nfft, z, gam)
    xhat = None
    if inverse_range is not None:
        p0, np_ = inverse_range
        xhat = inverse(T, k_lo, nfft, z, g, hop, n, p0, np_, mt0=m0)
    return Result(V, Vd, omega, dest, T, leak, gam, k_lo, k_hi, m0, xhat)


def sst2(x, fs: float, L: int, sigma: float, hop: int, nfft: int, f_lo: float, f_hi: float, z: int,
         gamma: float, relative: bool, m0: int = 0, nm: int | None = None,
         inverse_range: tuple[int, int] | None = None, gamma_abs: float | None = None) -> Result:
    """sst with the second-order IF (if2) in the reassignment: the same STFT,
    threshold (gamma, or gamma max|V| over all frames when relative), grid
    (Eq. 27-29) and inverse (Eq. 25-26).  Result.omega holds the second-order
    IF; leak is not tracked (zeros)."""
    x = _c(x)
    n = len(x)
    g, dg = window(L, sigma)
    k_lo, k_hi = band_bins(fs, nfft, f_lo, f_hi)
    F = frames(n, hop)
    if nm is None:
        nm = F - m0
    V, _, omega2, _ = if2(x, L, sigma, hop, nfft, k_lo, k_hi, m0, nm)
    if gamma_abs is not None:
        gam = float(gamma_abs)
    elif relative:
        gam = gamma * global_max_abs_v(x, g, dg, hop, nfft, k_lo, k_hi)
    else:
        gam = float(gamma)
    dest, T = reassign2(V, omega2, k_lo, k_hi, z, gam)
    _, Vd = stft(x, g, dg, hop, nfft, k_lo, k_hi, m0, nm)
    xhat = None
    if inverse_range is not None:
        p0, np_ = inverse_range
        xhat = inverse(T, k_lo, nfft, z, g, hop, n, p0, np_, mt0=m0)
    return Result(V, Vd, omega2, dest, T, np.zeros(nm, np.complex128), gam, k_lo, k_hi, m0, xhat)


# ------------------------------------------------ one signal split by frames
# Frames are independent (Sec. 2.1, Eq. 7-9); only the overlap-add of Eq. 26
# couples neighbouring frames, and a relative threshold needs the maximum of
# |V| over every frame.  So a long signal splits into contiguous frame ranges:
# each part reads its frames' samples (a read-only halo of M samples beyond
# its own), one max-reduction gives the threshold, and each part sends its
# overlap-add numerator on a neighbour's samples to that neighbour.
def frame_ranges(F: int, parts: int, align: int = 1):
    """Contiguous frame ranges [m_b, m_e) of `parts` parts, as equal as
    multiples of `align` frames allow."""
    units = -(-F // align)
    out = []
    for r in range(parts):
        ub, ue = units * r // parts, units * (r + 1) // parts
        out.append((min(F, ub * align), min(F, ue * align)))
    return out


def part_input_range(m_b: int, m_e: int, hop: int, L: int, n: int):
    """Samples [x_b, x_e) that frames [m_b, m_e) read (Eq. 7-8)."""
    M = (L - 1) // 2
    return max(0, m_b * hop - M), min(n, (m_e - 1) * hop + M + 1)


def part_output_range(m_b: int, m_e: int, hop: int, n: int, last: bool):
    """Output samples [p_b, p_e) a part finalises: from its first frame's
    centre to the next part's (to n for the last part)."""
    return min(n, m_b * hop), (n if last else min(n, m_e * hop))


def _embed(x_part, x_b, n):
    xl = np.zeros(n)
    xl[x_b:x_b + len(x_part)] = x_part
    return xl


def part_max_abs_v(x_part, x_b: int, n: int, L: int, sigma: float, hop: int, nfft: int,
                   k_lo: int, k_hi: int, m_b: int, m_e: int) -> float:
    """max |V| over the part's frames and the in-band bins, from its input
    samples only (the part's contribution to the max-reduction of a relative
    threshold)."""
    if m_e <= m_b:
        return 0.0
    g, dg = window(L, sigma)
    V, _ = stft(_embed(x_part, x_b, n), g, dg, hop, nfft, k_lo, k_hi, m_b, m_e - m_b)
    return float(np.abs(V).max())


def part_numerator(x_part, x_b: int, n: int, L: int, sigma: float, hop: int, nfft: int, k_lo: int,
                   k_hi: int, z: int, gam: float, m_b: int, m_e: int):
    """The part's STFT, reassignment (threshold gam, Eq. 13, 27-29) and
    overlap-add numerator sum_m g[p - m hop] r~[m, p - m hop] over its frames
    (Eq. 25-26 before the division by D), on the samples its frames touch.
    Returns (numerator, first sample, T of the part's frames)."""
    M = (L - 1) // 2
    g, dg = window(L, sigma)
    V, Vd = stft(_embed(x_part, x_b, n), g, dg, hop, nfft, k_lo, k_hi, m_b, m_e - m_b)
    _, _, T, _ = reassign(V, Vd, k_lo, k_hi, nfft, z, gam)
    q_b = max(0, m_b * hop - M)
    q_e = min(n, (m_e - 1) * hop + M + 1)
    num = inverse(T, k_lo, nfft, z, g, hop, n, q_b, q_e - q_b, mt0=m_b, mode=2)
    return num, q_b, T


def part_finalise(shares, p_b: int, p_e: int, L: int, sigma: float, hop: int, n: int) -> np.ndarray:
    """x^ on [p_b, p_e) from the numerator shares (array, first sample) of the
    parts whose frames touch it, added in the order given (ascending parts),
    divided by the Eq. 26 normaliser D."""
    num = np.zeros(p_e - p_b)
    for arr, q_b in shares:
        lo, hi = max(p_b, q_b), min(p_e, q_b + len(arr))
        if hi > lo:
            num[lo - p_b:hi - p_b] += arr[lo - q_b:hi - q_b]
    g, _ = window(L, sigma)
    return num / normaliser(g, hop, n, p_b, p_e - p_b)


def global_max_abs_v(x, g, dg, hop, nfft, k_lo, k_hi, chunk: int = 4096) -> float:
    """max over every frame and in-band bin of |V| (the relative-threshold base)."""
    n = len(x)
    F = frames(n, hop)
    best = 0.0
    for m0 in range(0, F, chunk):
        nm = min(chunk, F - m0)
        V, _ = stft(x, g, dg, hop, nfft, k_lo, k_hi, m0, nm)
        best = max(best, float(np.abs(V).max()))
    return best

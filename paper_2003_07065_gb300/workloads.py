"""Named workloads: transform parameters plus the seeded synthetic signal each
one runs on.  Parameters only; no transform arithmetic lives here.

chirp_fm_64k   N = 65536 at 25.6 kHz, chirp 500->2000 Hz + FM tone 4 kHz
               +/-300 Hz @ 3 Hz + white noise 10 dB; L = 1025, sigma = 128,
               hop 16, Nf 1024, full band, z = 1, gamma = 1e-3 max|V|.
runup_16m      N = 2^24 at 51.2 kHz run-up vibration (orders 1, 2, 3.5, 7 of a
               20->200 Hz shaft, AM 3.2 kHz resonance, pink noise 5 dB);
               L = 2049, sigma = 256, hop 32, Nf 4096, band 0-6.4 kHz, z = 4,
               gamma = 1e-3 max|V|.
runup_256k     the run-up recipe and parameters at N = 2^18 - 37 (a ragged
               tail), small enough for the oracle to check every output.
runup_4m       the run-up recipe at N = 2^22 (profiling-sized: 2.1 GB TFR).
precision_64k  chirp_fm_64k's signal with Nf 4096, L = 2049, sigma = 256,
               hop 16, band 0-6.4 kHz (bins 0..1024), z = 1.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

from . import signals


@dataclass(frozen=True)
class Workload:
    name: str
    n: int
    fs: float
    L: int
    sigma: float
    hop: int
    nfft: int
    f_lo: float
    f_hi: float
    z: int
    gamma: float
    relative: bool
    recipe: str = ""

    def params(self) -> dict:
        return dict(n=self.n, fs=self.fs, L=self.L, sigma=self.sigma, hop=self.hop, nfft=self.nfft,
                    f_lo=self.f_lo, f_hi=self.f_hi, z=self.z, gamma=self.gamma,
                    relative=self.relative)

    def signal(self):
        """(noisy, clean) float64 arrays."""
        if self.recipe == "chirp_fm":
            return signals.chirp_fm_mix(self.n, self.fs, 10.0, seed=(1, 0))
        if self.recipe == "runup":
            return signals.runup(self.n, self.fs, 5.0, seed=(2, 0))
        raise ValueError(self.recipe)

    def with_n(self, n: int, name: str | None = None) -> "Workload":
        d = dict(self.__dict__)
        d["n"] = int(n)
        d["name"] = name or f"{self.name}@{n}"
        return Workload(**d)


CHIRP_FM_64K = Workload("chirp_fm_64k", 65536, 25600.0, 1025, 128.0, 16, 1024, 0.0, 12800.0, 1,
                        1e-3, True, "chirp_fm")
RUNUP_16M = Workload("runup_16m", 1 << 24, 51200.0, 2049, 256.0, 32, 4096, 0.0, 6400.0, 4,
                     1e-3, True, "runup")
RUNUP_256K = RUNUP_16M.with_n((1 << 18) - 37, "runup_256k")
RUNUP_4M = RUNUP_16M.with_n(1 << 22, "runup_4m")
PRECISION_64K = Workload("precision_64k", 65536, 25600.0, 2049, 256.0, 16, 4096, 0.0, 6400.0, 1,
                         1e-3, True, "chirp_fm")

ALL = {w.name: w for w in (CHIRP_FM_64K, RUNUP_16M, RUNUP_256K, RUNUP_4M, PRECISION_64K)}


def batch_channels(count: int = 256, log2_min: float = 14.0, log2_max: float = 22.0, seed: int = 4):
    """Mixed multi-channel batch: per channel a length log-uniform in
    [2^log2_min, 2^log2_max], hop in {8, 16, 32, 64}, Nf in {512 .. 8192},
    L = Nf/2 + 1, sigma = (L - 1)/8, fs = 25.6 kHz, a band of 10-50 % of
    Nyquist at a uniform start, z in {1, 2, 4}, gamma = 1e-3 max|V|, and a
    seeded random mix of 1-4 chirp / FM components plus 0-20 dB noise.

    Returns a list of (params dict, noisy float32 signal)."""
    out = []
    fs = 25600.0
    for i in range(count):
        gen = signals.rng(seed, i)
        n = int(round(2.0 ** gen.uniform(log2_min, log2_max)))
        hop = int(gen.choice([8, 16, 32, 64]))
        nfft = int(gen.choice([512, 1024, 2048, 4096, 8192]))
        L = nfft // 2 + 1
        width = float(gen.uniform(0.1, 0.5)) * fs / 2
        f_lo = float(gen.uniform(0.0, fs / 2 - width))
        z = int(gen.choice([1, 2, 4]))
        noisy, _ = signals.random_mix(n, fs, f_lo, f_lo + width, gen)
        params = dict(n=n, fs=fs, L=L, sigma=(L - 1) / 8.0, hop=hop, nfft=nfft, f_lo=f_lo,
                      f_hi=f_lo + width, z=z, gamma=1e-3, relative=True)
        out.append((params, noisy.astype(np.float32)))
    return out

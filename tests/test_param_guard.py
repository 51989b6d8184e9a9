"""Parameter guard of Sec. 4 in the product library (sst_params_check,
host arithmetic only, so these run on the CPU): sigma_f (Eq. 35), the Hf
bounds of Eq. 38 and Eq. 46 and the frequency intervals (Eq. 12, 28),
pinned to the numbers the paper prints for its simulation (Sec. 3-4) and its
aero-engine and chatter cases (Sec. 5), listed in tests/golden/paper_numbers.txt."""
import os

import numpy as np
import pytest

from paper_2003_07065_gb300 import build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _golden():
    out = {}
    with open(os.path.join(ROOT, "tests", "golden", "paper_numbers.txt")) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            name, val, tol, *_ = line.split()
            out[name] = (float(val), float(tol))
    return out


def _close(name, value):
    v, tol = _golden()[name]
    assert abs(value - v) <= tol, (name, value, v)


@pytest.fixture(scope="module")
def S():
    build.build()
    from paper_2003_07065_gb300 import sst
    sst.load()
    return sst


def sim(S, nfft):
    # Sec. 3 simulation: N = 8192 samples at fs = 1024 Hz, sigma = 0.03 s
    return S.sst_params_check(n=8192, fs=1024.0, L=129, hop=8, nfft=nfft, f_lo=0.0, f_hi=512.0,
                              sigma=0.03 * 1024)


def test_simulation_numbers(S):
    r = sim(S, 256)
    _close("sigma_f_sim_hz", r["sigma_f_hz"])
    _close("support_6sigma_f_hz", 6 * r["sigma_f_hz"])
    assert 63 < r["hf_max_eq38"] < 64           # "Hf < 64"
    _close("hf_max_rule1_sim", r["hf_max_eq38"])
    _close("hf_max_rule2_sim", r["hf_max_eq46"])
    assert r["hf"] == 32 and r["flags"] == 0
    # the bounds on Delta f are the same statements: Delta f = Hf fs / N
    assert abs(r["delta_f_max_eq37_hz"] - r["hf_max_eq38"] * 1024 / 8192) < 1e-9
    assert abs(r["delta_f_max_eq46_hz"] - r["hf_max_eq46"] * 1024 / 8192) < 1e-9


def test_simulation_flags_follow_hf(S):
    # Hf = 64 is beyond both bounds (63.7 and 60.0); Hf = 32 beyond neither
    r = sim(S, 128)
    assert r["hf"] == 64 and r["beyond_eq38"] and r["beyond_eq46"]
    assert sim(S, 256)["flags"] == 0
    # between the two bounds: Hf = 62 (not a power of two, so only through n)
    r = S.sst_params_check(n=62 * 128, fs=1024.0, L=129, hop=8, nfft=128, f_lo=0.0, f_hi=512.0,
                           sigma=0.03 * 1024 * (62 * 128 / 8192))
    # sigma scaled with n keeps the bounds in samples: Eq. 38 -> 63.7, Eq. 46 -> 60.0
    assert not r["beyond_eq38"] and r["beyond_eq46"]


def test_aero_engine_numbers(S):
    # Sec. 5.1: N = 9035089 at 44.1 kHz, Nf = 2^13, sigma = 0.02 s, z = 8
    r = S.sst_params_check(n=9035089, fs=44100.0, L=8191, hop=1149, nfft=8192, f_lo=6900.0, f_hi=9500.0,
                           z=8, sigma=0.02 * 44100)
    _close("hf_max_rule1_aero", r["hf_max_eq38"])
    _close("hf_aero", r["hf"])
    _close("delta_f_aero_hz", r["delta_f_fine_hz"])
    assert not r["beyond_eq38"]                 # "less than the critical value 2446"


def test_chatter_interval(S):
    # Sec. 5.2: fs = 10240 Hz, Nf = 2^15
    r = S.sst_params_check(n=573440, fs=10240.0, L=2049, hop=667, nfft=8192, f_lo=1200.0, f_hi=1400.0,
                           sigma=256.0)
    assert abs(r["delta_f_hz"] - 10240 / 8192) < 1e-12
    # the paper's Nf = 2^15 exceeds this library's largest DFT; the same
    # interval fs / 2^15 is the output grid of Nf = 2^12 subdivided by z = 8
    r = S.sst_params_check(n=573440, fs=10240.0, L=2049, hop=667, nfft=4096, f_lo=1200.0, f_hi=1400.0,
                           z=8, sigma=256.0)
    _close("delta_f_chatter_hz", r["delta_f_fine_hz"])


def test_supplied_window_uses_its_second_moment(S):
    sigma, L = 40.0, 641
    j = np.arange(L) - (L - 1) // 2
    g = np.exp(-j * j / (2 * sigma * sigma))
    dg = -(j / sigma ** 2) * g
    r = S.sst_params_check(n=100000, fs=8000.0, L=L, hop=16, nfft=1024, f_lo=0.0, f_hi=4000.0, g=g, dg=dg)
    assert abs(r["sigma_s"] * 8000.0 - sigma) <= 1e-9 * sigma
    r2 = S.sst_params_check(n=100000, fs=8000.0, L=L, hop=16, nfft=1024, f_lo=0.0, f_hi=4000.0, sigma=sigma)
    assert abs(r["hf_max_eq38"] - r2["hf_max_eq38"]) <= 1e-9 * r2["hf_max_eq38"]


def test_invalid_parameters_rejected(S):
    with pytest.raises(S.SstError) as e:
        S.sst_params_check(n=1000, fs=1000.0, L=64, hop=8, nfft=64, f_lo=0.0, f_hi=500.0, sigma=8.0)
    assert e.value.status == 1
    with pytest.raises(S.SstError):
        S.sst_params_check(n=1000, fs=1000.0, L=65, hop=8, nfft=64, f_lo=0.0, f_hi=500.0, sigma=0.0)


def test_window_length_limit(S):
    """Windows up to SST_MAX_L = 8193 taps are valid for every nfft (a window
    longer than nfft is folded, Eq. 8); a longer one is an argument error."""
    r = S.sst_params_check(n=100000, fs=8000.0, L=8193, hop=64, nfft=64, f_lo=0.0, f_hi=4000.0, sigma=1024.0)
    assert r["hf_max_eq38"] > 0
    S.sst_params_check(n=100000, fs=8000.0, L=67, hop=8, nfft=64, f_lo=0.0, f_hi=4000.0, sigma=8.0)
    with pytest.raises(S.SstError) as e:
        S.sst_params_check(n=100000, fs=8000.0, L=8195, hop=64, nfft=8192, f_lo=0.0, f_hi=4000.0, sigma=1024.0)
    assert e.value.status == 1

"""GPU parity: the CUDA path through the C ABI against the FP64 oracle on the
same seeded inputs (the oracle reads the same float32 samples, widened), with
the bars of tests/parity.py: STFT, map, T in replay mode (the oracle's V
re-accumulated with the GPU's destination map), column mass, the inverse
alone (the oracle's inverse of the GPU's T) and end to end (with the exact
effect of every source the two sides place differently), and the SNR.

Covers the small chirp/FM workload and the run-up workload at 2^18 - 37
samples (many inverse tiles and a ragged tail) element by element, the
degenerate cases (tiny signals, a one-bin band, the Nyquist band, L = Nf + 1
folding, zero threshold), and run-to-run bit determinism."""
import numpy as np
import pytest

import oracle as O
from paper_2003_07065_gb300 import workloads as W

from parity import as_complex, compare

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def sst():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2003_07065_gb300 import build, sst as S
    build.build()
    S.load()
    return S


def run_gpu(S, params, x32):
    plan = S.Plan(**params)
    x = torch.from_numpy(x32).cuda()
    V, Vd = plan.stft(x)
    om, dest = plan.reassign_map(x)
    tfr, xhat = plan.forward_inverse(x)
    maxv = plan.max_abs_v(x)
    torch.cuda.synchronize()
    out = dict(V=as_complex(V.cpu().numpy()), Vd=as_complex(Vd.cpu().numpy()),
               omega=om.cpu().numpy(), dest=dest.cpu().numpy(), T=as_complex(tfr.cpu().numpy()),
               xhat=xhat.cpu().numpy().astype(np.float64), maxv=float(maxv.item()),
               k_lo=plan.k_lo, k_hi=plan.k_hi, bins=plan.bins)
    plan.close()
    return out


def run_oracle(params, x32):
    p = dict(params)
    x = x32.astype(np.float64)
    r = O.sst(x, p["fs"], p["L"], p["sigma"], p["hop"], p["nfft"], p["f_lo"], p["f_hi"], p["z"],
              p["gamma"], p["relative"], inverse_range=(0, len(x)))
    return r


@pytest.mark.parametrize("name", ["chirp_fm_64k", "runup_256k"])
def test_workload_parity(sst, name):
    w = W.ALL[name]
    noisy, clean = w.signal()
    x32 = noisy.astype(np.float32)
    params = w.params()
    g = run_gpu(sst, params, x32)
    r = run_oracle(params, x32)
    stats = compare(g, r, params, clean)
    print(name, stats)


EDGE = [
    # n, fs, L, sigma, hop, nfft, f_lo, f_hi, z, gamma, relative
    dict(n=1, fs=1000.0, L=65, sigma=8.0, hop=8, nfft=64, f_lo=0.0, f_hi=500.0, z=1, gamma=0.0, relative=False),
    dict(n=100, fs=1000.0, L=65, sigma=8.0, hop=8, nfft=64, f_lo=0.0, f_hi=500.0, z=2, gamma=1e-3, relative=True),
    dict(n=999, fs=1000.0, L=129, sigma=16.0, hop=5, nfft=128, f_lo=100.0, f_hi=100.0 + 1e-9, z=3,
         gamma=1e-3, relative=True),
    dict(n=3001, fs=2000.0, L=257, sigma=32.0, hop=7, nfft=256, f_lo=700.0, f_hi=1000.0, z=4, gamma=1e-3,
         relative=True),
    dict(n=5000, fs=8000.0, L=1025, sigma=128.0, hop=16, nfft=1024, f_lo=0.0, f_hi=4000.0, z=2, gamma=1e-4,
         relative=True),
    dict(n=7777, fs=8000.0, L=513, sigma=64.0, hop=31, nfft=512, f_lo=1000.0, f_hi=3000.0, z=1, gamma=0.0,
         relative=False),
    dict(n=20000, fs=16000.0, L=4097, sigma=512.0, hop=64, nfft=8192, f_lo=0.0, f_hi=2000.0, z=2, gamma=1e-3,
         relative=True),
    dict(n=12000, fs=16000.0, L=2049, sigma=256.0, hop=16, nfft=2048, f_lo=3000.0, f_hi=8000.0, z=1,
         gamma=1e-3, relative=True),
    # pruned radix-16 first pass: band class 1 (k_hi < 3 Nf/16) and class 2 (k_hi < 5 Nf/16) with a
    # half-length window, at Nf 256 and 4096, k_lo = 0 and > 0, odd z, absolute gamma = 0 (odd z only
    # at Nf 256: the oracle's zNf-point inverse is a plain DFT when zNf is not a power of two)
    dict(n=1500, fs=2000.0, L=129, sigma=16.0, hop=6, nfft=256, f_lo=0.0, f_hi=100.0, z=3, gamma=1e-3,
         relative=True),
    dict(n=2500, fs=2000.0, L=101, sigma=12.0, hop=3, nfft=256, f_lo=200.0, f_hi=500.0, z=1, gamma=0.0,
         relative=False),
    dict(n=30011, fs=16000.0, L=2049, sigma=256.0, hop=24, nfft=4096, f_lo=100.0, f_hi=1500.0, z=2,
         gamma=1e-3, relative=True),
    dict(n=9001, fs=16000.0, L=1537, sigma=192.0, hop=40, nfft=4096, f_lo=0.0, f_hi=3500.0, z=2,
         gamma=1e-3, relative=True),
]


@pytest.mark.parametrize("params", EDGE, ids=[f"n{p['n']}_nf{p['nfft']}_z{p['z']}" for p in EDGE])
def test_edge_cases(sst, params):
    gen = np.random.default_rng(params["n"])
    t = np.arange(params["n"]) / params["fs"]
    mid = 0.5 * (params["f_lo"] + params["f_hi"])
    x = np.cos(2 * np.pi * mid * t + 0.3) + 0.3 * gen.standard_normal(params["n"])
    x32 = x.astype(np.float32)
    g = run_gpu(sst, params, x32)
    r = run_oracle(params, x32)
    print(params, compare(g, r, params))


def test_deterministic(sst):
    w = W.CHIRP_FM_64K
    x = torch.from_numpy(w.signal()[0].astype(np.float32)).cuda()
    plan = sst.Plan(**w.params())
    t1, x1 = plan.forward_inverse(x)
    t2, x2 = plan.forward_inverse(x)
    torch.cuda.synchronize()
    assert torch.equal(t1, t2) and torch.equal(x1, x2)
    plan.close()


def test_plan_errors(sst):
    with pytest.raises(sst.SstError) as e:
        sst.sst_plan_create(n=100, fs=1000.0, L=64, hop=8, nfft=64, f_lo=0, f_hi=500, sigma=8.0)
    assert e.value.status == 1
    p = sst.Plan(n=1000, fs=1000.0, L=65, sigma=8.0, hop=8, nfft=64, f_lo=0, f_hi=500)
    x = torch.zeros(999, device="cuda")
    with pytest.raises(sst.SstError):
        sst.sst_forward(p.handle, x, 999, p.new_tfr(), p.workspace)
    p.close()


def test_inverse_unaligned_rows(sst):
    """T rows at an address that is not 16-byte aligned take the synchronous
    staging path of the inverse; the result is the same."""
    w = W.CHIRP_FM_64K
    x = torch.from_numpy(w.signal()[0].astype(np.float32)).cuda()
    plan = sst.Plan(**w.params())
    tfr, xhat = plan.forward_inverse(x)
    flat = torch.empty(tfr.numel() + 2, dtype=torch.float32, device="cuda")
    shifted = flat[2:].view(tfr.shape)          # 8 bytes past a 16-byte boundary
    shifted.copy_(tfr)
    assert shifted.data_ptr() % 16 == 8
    xh2 = plan.inverse(shifted)
    torch.cuda.synchronize()
    assert torch.equal(xhat, xh2)
    plan.close()


def test_inverse_wait_expiry_reported(sst):
    """A row copy that never lands (test hook: CTA 0 does not issue it) makes
    the inverse's bounded waits run out; that CTA stages its tile
    synchronously, the result keeps its bits, sst_check reports SST_ETIMEOUT,
    and the next inverse is clean again."""
    w = W.CHIRP_FM_64K
    x = torch.from_numpy(w.signal()[0].astype(np.float32)).cuda()
    plan = sst.Plan(**w.params())
    tfr, xhat = plan.forward_inverse(x)
    sst.sst_check(plan.handle, plan.workspace)
    sst.sst_test_withhold_row_copy(plan.handle)
    xh2 = plan.inverse(tfr)
    with pytest.raises(sst.SstError) as e:
        sst.sst_check(plan.handle, plan.workspace)
    assert e.value.status == 5
    assert torch.equal(xhat, xh2)
    xh3 = plan.inverse(tfr)
    sst.sst_check(plan.handle, plan.workspace)
    assert torch.equal(xhat, xh3)
    plan.close()


def test_forward_sample_copy_expiry_reported(sst):
    """The forward of the run-up class (pruning class 1) stages each chunk's
    samples with one bulk copy; a copy that never lands (test hook) makes
    that CTA's waits run out, it loads the samples directly, the TFR keeps
    its bits and sst_check reports SST_ETIMEOUT; the next call is clean."""
    w = W.ALL["runup_256k"]
    x = torch.from_numpy(w.signal()[0].astype(np.float32)).cuda()
    plan = sst.Plan(**w.params())
    ref = plan.forward(x)
    sst.sst_check(plan.handle, plan.workspace)
    sst.sst_test_withhold_sample_copy(plan.handle)
    got = plan.forward(x)
    with pytest.raises(sst.SstError) as e:
        sst.sst_check(plan.handle, plan.workspace)
    assert e.value.status == 5
    assert torch.equal(ref, got)
    again = plan.forward(x)
    sst.sst_check(plan.handle, plan.workspace)
    assert torch.equal(ref, again)
    plan.close()


def test_plan_check_matches_params_check(sst):
    w = W.ALL["runup_256k"]
    p = w.params()
    plan = sst.Plan(**p)
    a = sst.sst_plan_check(plan.handle)
    b = sst.sst_params_check(**p)
    assert a == b
    assert a["hf"] == p["n"] / p["nfft"]
    plan.close()

"""Forward + inverse without a TFR output (sst_forward_inverse with a NULL
tfr): T stays in shared memory between the forward and the inverse of each
pair of frames (Eq. 25 needs only the frame's own column).

* Two-pass plans (max |S^g| from a pre-pass first): the reconstruction must
  carry the same bits as the same plan's forward + inverse through a TFR in
  global memory (same per-frame arithmetic, same tiles and overlap-add
  order).
* One-pass plans (the default for a relative threshold): the sources
  between the threshold's two bounds are left out of the rows and, once the
  exact maximum is known, the kept ones are added to the reconstruction
  directly (one coefficient's term of Eq. 25-26).  The kept set is the one
  the one-pass TFR path keeps (same STFT arithmetic, same bounds), so the two
  reconstructions differ by rounding only: within the reconstruction bar.
  Repeated calls give the same bits.  A record overflow falls back to the
  two-pass kernels and then matches them bit for bit.
* Both meet the parity bars against the FP64 oracle (the inverse end to end,
  with the moved-source bound, and the SNR)."""
import numpy as np
import pytest

import oracle as O
from paper_2003_07065_gb300 import workloads as W

from parity import check_map, check_xhat_end_to_end, moved_bound, snr_db, SNR_DB

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from test_gpu_parity import EDGE  # noqa: E402


@pytest.fixture(scope="module")
def sst():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2003_07065_gb300 import build, sst as S
    build.build()
    S.load()
    return S


XHAT_RTOL = 2e-5


def same_bits_as_two_pass(S, params, x32):
    x = torch.from_numpy(x32).cuda()
    two = S.Plan(**params, two_pass=True)
    _, ref = two.forward_inverse(x)
    got = torch.full_like(ref, float("nan"))
    two.reconstruct(x, got)
    got2 = two.reconstruct(x)
    torch.cuda.synchronize()
    assert torch.equal(got, ref), (got - ref).abs().max().item()
    assert torch.equal(got, got2)
    out = got.cpu().numpy().astype(np.float64)
    _, dest = two.reassign_map(x)
    dest = dest.cpu().numpy().astype(np.int64)
    two.close()
    return out, dest


def one_pass_close(S, params, x32):
    """The default plan's reconstruction without a TFR output against its
    TFR path: same kept sources, rounding-level differences only; repeat
    calls bit-identical.  Returns the reconstruction and the threshold stats."""
    x = torch.from_numpy(x32).cuda()
    one = S.Plan(**params)
    _, ref = one.forward_inverse(x)
    got = torch.full_like(ref, float("nan"))
    one.reconstruct(x, got)
    stats = S.sst_threshold_stats(one.handle, one.workspace)
    got2 = one.reconstruct(x)
    torch.cuda.synchronize()
    assert torch.equal(got, got2)
    err = (got - ref).abs().max().item()
    scale = ref.abs().max().item()
    assert err <= XHAT_RTOL * scale, (err, scale)
    out = got.cpu().numpy().astype(np.float64)
    one.close()
    return out, stats, err / max(scale, 1e-30)


def oracle_check(params, x32, xhat, dest, clean=None):
    p = params
    r = O.sst(x32.astype(np.float64), p["fs"], p["L"], p["sigma"], p["hop"], p["nfft"], p["f_lo"], p["f_hi"],
              p["z"], p["gamma"], p["relative"], inverse_range=(0, p["n"]))
    check_map(dest, r.dest, r.V, r.gamma, r.T.shape[1])
    g, _ = O.window(p["L"], p["sigma"])
    bound = moved_bound(r.V, dest, r.dest, r.k_lo, p["nfft"], p["z"], g, p["hop"], p["n"])
    stats = check_xhat_end_to_end(xhat, r.xhat, bound)
    if clean is not None:
        assert abs(snr_db(clean, xhat) - snr_db(clean, r.xhat)) <= SNR_DB
    return stats


@pytest.mark.parametrize("name", ["chirp_fm_64k", "runup_256k"])
def test_workloads(sst, name):
    w = W.ALL[name]
    noisy, clean = w.signal()
    x32 = noisy.astype(np.float32)
    xhat, dest = same_bits_as_two_pass(sst, w.params(), x32)
    print(name, oracle_check(w.params(), x32, xhat, dest, clean))
    x1, stats, rel = one_pass_close(sst, w.params(), x32)
    assert not stats["fell_back"], stats
    print(name, "one pass", stats, rel, oracle_check(w.params(), x32, x1, dest, clean))


@pytest.mark.parametrize("params", EDGE, ids=[f"n{p['n']}_nf{p['nfft']}_z{p['z']}" for p in EDGE])
def test_edge_cases(sst, params):
    gen = np.random.default_rng(params["n"] + 1)
    t = np.arange(params["n"]) / params["fs"]
    mid = 0.5 * (params["f_lo"] + params["f_hi"])
    x32 = (np.cos(2 * np.pi * mid * t + 0.3) + 0.3 * gen.standard_normal(params["n"])).astype(np.float32)
    try:
        xhat, dest = same_bits_as_two_pass(sst, params, x32)
    except sst.SstError as e:
        assert e.status == 6 and "shared memory" in str(e)
        pytest.skip("fused kernel does not fit this plan: " + str(e))
    print(params, oracle_check(params, x32, xhat, dest))
    if params["relative"]:
        x1, stats, rel = one_pass_close(sst, params, x32)
        print("one pass", stats, rel)


@pytest.mark.parametrize("z,f_lo", [(3, 1000.0), (2, 0.0)], ids=["z3_band_to_nyquist", "z2_dc_and_nyquist"])
def test_one_pass_settling_variants(sst, z, f_lo):
    """The settling pass where its arithmetic differs most: a phase table of
    z Nf = 3072 entries (z not a power of two) with a band from above DC up
    to Nyquist, and a band holding both the DC and the Nyquist bin (weight
    1/2); sources must actually wait for the exact threshold."""
    w = W.ALL["chirp_fm_64k"]
    noisy, clean = w.signal()
    x32 = noisy.astype(np.float32)
    params = dict(w.params(), z=z, f_lo=f_lo)
    x1, stats, rel = one_pass_close(sst, params, x32)
    assert stats["waiting"] > 0 and not stats["fell_back"], stats
    _, dest = same_bits_as_two_pass(sst, params, x32)
    print(params, stats, rel, oracle_check(params, x32, x1, dest, clean))


LONG_ROWS = [
    # T rows longer than the frame buffer (small Nf, wide band, z >= 3)
    dict(n=40000, fs=16000.0, L=257, sigma=32.0, hop=8, nfft=256, f_lo=0.0, f_hi=8000.0, z=4, gamma=1e-3,
         relative=True),
    dict(n=30011, fs=8000.0, L=513, sigma=64.0, hop=16, nfft=512, f_lo=500.0, f_hi=4000.0, z=3, gamma=0.02,
         relative=False),
]


@pytest.mark.parametrize("params", LONG_ROWS, ids=["nf256_z4_full", "nf512_z3_abs"])
def test_rows_longer_than_frame_buffer(sst, params):
    gen = np.random.default_rng(params["n"])
    t = np.arange(params["n"]) / params["fs"]
    f0, f1 = 0.2 * params["fs"] / 2, 0.7 * params["fs"] / 2
    dur = params["n"] / params["fs"]
    clean = np.cos(2 * np.pi * (f0 * t + 0.5 * (f1 - f0) / dur * t * t))
    x32 = (clean + 0.2 * gen.standard_normal(params["n"])).astype(np.float32)
    xhat, dest = same_bits_as_two_pass(sst, params, x32)
    print(params["nfft"], params["z"], oracle_check(params, x32, xhat, dest))
    if params["relative"]:
        x1, stats, rel = one_pass_close(sst, params, x32)
        print("one pass", stats, rel)


def test_runup_16m_full_size(sst):
    """The benchmark's workload: a two-pass plan gives the same bits as its
    TFR path; the default (one-pass) plan stays within the reconstruction bar
    of its TFR path, without falling back."""
    w = W.RUNUP_16M
    x32 = w.signal()[0].astype(np.float32)
    x = torch.from_numpy(x32).cuda()
    two = sst.Plan(**w.params(), two_pass=True)
    _, ref = two.forward_inverse(x)
    got = two.reconstruct(x)
    torch.cuda.synchronize()
    assert torch.equal(got, ref)
    two.close()
    del ref, got
    _, stats, rel = one_pass_close(sst, w.params(), x32)
    assert not stats["fell_back"], stats
    print("runup_16m one pass", rel)


def test_one_pass_overflow_falls_back(sst):
    """A transient whose loudest frames fall between the sampled pre-pass
    frames leaves most sources between the two bounds: the records overflow
    and the call redoes itself with the two-pass kernels, bit for bit."""
    n, fs = 65536, 25600.0
    params = dict(n=n, fs=fs, L=1025, sigma=128.0, hop=16, nfft=1024, f_lo=0.0, f_hi=12800.0, z=1,
                  gamma=1e-3, relative=True)
    gen = np.random.default_rng(77)
    t = np.arange(n) / fs
    x = 1e-3 * gen.standard_normal(n)
    env = np.exp(-0.5 * ((np.arange(n) - 1600) / 40.0) ** 2)
    x = torch.from_numpy((x + env * np.sin(2 * np.pi * 3000 * t)).astype(np.float32)).cuda()
    one = sst.Plan(**params)
    two = sst.Plan(**params, two_pass=True)
    got = one.reconstruct(x)
    stats = sst.sst_threshold_stats(one.handle, one.workspace)
    ref = two.reconstruct(x)
    torch.cuda.synchronize()
    assert stats["fell_back"], stats
    assert torch.equal(got, ref)
    one.close()
    two.close()


def test_unsupported_plan_reported(sst):
    # Nf 8192 over the whole band with z = 4: accumulators alone exceed shared memory
    p = dict(n=20000, fs=16000.0, L=4097, sigma=512.0, hop=64, nfft=8192, f_lo=0.0, f_hi=8000.0, z=4,
             gamma=1e-3, relative=True)
    try:
        plan = sst.Plan(**p)
    except sst.SstError as e:          # the TFR path itself may not fit either
        assert e.status == 6
        return
    x = torch.zeros(p["n"], device="cuda")
    with pytest.raises(sst.SstError) as e:
        plan.reconstruct(x)
    assert e.value.status == 6
    plan.close()

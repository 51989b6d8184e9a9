"""GPU parity of the steps after the transform: component recovery by zone
(sst_inverse_zone), ridge extraction (sst_ridge) and the Renyi entropy
(sst_renyi), each through the C ABI against the oracle on the same T.

T is the oracle's (FP64, rounded to complex64 for the GPU), so the
comparison isolates each step; the zone centres come from the test's own
generator.  Both staging paths of the inverse (rows copied in bulk, rows
staged one by one) are covered, as are a ragged last tile, frames without a
ridge, ties and the argument checks."""
import math

import numpy as np
import pytest

import oracle as O
from paper_2003_07065_gb300 import signals as S

from parity import XHAT_RTOL

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

# a run-up-like configuration (Nf 4096, L = Nf/2 + 1, hop 32, z = 4, band
# 0-6.4 kHz at 51.2 kHz: the pruned class-1 inverse) and a full-band one
CFGS = {
    "runup_like": dict(n=65536 - 37, fs=51200.0, L=2049, sigma=256.0, hop=32, nfft=4096, f_lo=0.0, f_hi=6400.0,
                       z=4, gamma=1e-3, relative=True),
    "fullband": dict(n=20011, fs=8000.0, L=1025, sigma=128.0, hop=16, nfft=1024, f_lo=0.0, f_hi=4000.0, z=2,
                     gamma=1e-3, relative=True),
}


@pytest.fixture(scope="module")
def sst():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2003_07065_gb300 import build, sst as S_
    build.build()
    S_.load()
    return S_


def _signal(p, seed=7):
    gen = np.random.default_rng(seed)
    n, fs = p["n"], p["fs"]
    t = np.arange(n) / fs
    f1, f2 = 0.12 * p["f_hi"] + 0.05 * fs / p["nfft"], 0.55 * p["f_hi"]
    x = (0.8 * np.cos(2 * np.pi * (f1 * t + 2.0 * t * t)) + 0.5 * np.cos(2 * np.pi * f2 * t + 0.4)
         + 0.05 * gen.standard_normal(n))
    return x.astype(np.float32)


_cache = {}


def _oracle(name):
    if name not in _cache:
        p = CFGS[name]
        x = _signal(p)
        r = O.sst(x.astype(np.float64), p["fs"], p["L"], p["sigma"], p["hop"], p["nfft"], p["f_lo"], p["f_hi"],
                  p["z"], p["gamma"], p["relative"])
        _cache[name] = (p, x, r)
    return _cache[name]


def _to_gpu(T):
    a = np.stack([T.real, T.imag], axis=-1).astype(np.float32)
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _zone_centres(F, nbo, seed):
    """Centres that wander over the band, with runs of frames without a ridge."""
    gen = np.random.default_rng(seed)
    c = np.clip(np.cumsum(gen.integers(-3, 4, F)) + nbo // 3, 0, nbo - 1).astype(np.int32)
    c[gen.random(F) < 0.1] = -1
    c[: min(5, F)] = -1
    return c


@pytest.mark.parametrize("name", list(CFGS))
@pytest.mark.parametrize("hw", [0, 3, 40])
@pytest.mark.parametrize("aligned", [True, False])
def test_zone_inverse_matches_oracle(sst, name, hw, aligned):
    p, _, r = _oracle(name)
    plan = sst.Plan(**{k: v for k, v in p.items()})
    F, nbo = r.T.shape
    assert (F, nbo) == (plan.frames, plan.bins)
    ridge = _zone_centres(F, nbo, seed=hw + 11)
    g, _ = O.window(p["L"], p["sigma"])
    want = O.zone_inverse(r.T, ridge, hw, r.k_lo, p["nfft"], p["z"], g, p["hop"], p["n"])
    T = _to_gpu(r.T)
    if not aligned:   # rows 8 bytes past a 16-byte boundary: the one-by-one staging path
        flat = torch.empty(T.numel() + 2, dtype=torch.float32, device="cuda")
        T2 = flat[2:].view(T.shape)
        T2.copy_(T)
        assert T2.data_ptr() % 16 == 8
        T = T2
    rg = torch.from_numpy(ridge).cuda()
    got = plan.inverse_zone(T, rg, hw).cpu().numpy().astype(np.float64)
    plan.close()
    scale = max(np.abs(want).max(), 1e-30)
    err = np.abs(got - want).max()
    assert err <= XHAT_RTOL * np.abs(O.inverse(r.T, r.k_lo, p["nfft"], p["z"], g, p["hop"], p["n"])).max() + 1e-7 * scale, \
        f"zone inverse err {err:.3e} (max {scale:.3e})"


def test_zone_covering_everything_is_the_inverse(sst):
    p, x, _ = _oracle("runup_like")
    plan = sst.Plan(**p)
    xt = torch.from_numpy(x).cuda()
    tfr, xh = plan.forward_inverse(xt)
    ridge = torch.zeros(plan.frames, dtype=torch.int32, device="cuda")
    xz = plan.inverse_zone(tfr, ridge, plan.bins)
    assert torch.equal(xz, xh)
    none = plan.inverse_zone(tfr, ridge - 1, plan.bins)
    assert float(none.abs().max()) == 0.0
    plan.close()


def _check_ridge(got, want, T, l_lo, l_hi, smooth):
    """Equal, or (near-ties between FP32 and FP64 energies) the GPU's bin has
    the oracle's largest energy to within 1e-5."""
    diff = np.nonzero(got != want)[0]
    if len(diff) == 0:
        return 0
    P = np.abs(T) ** 2
    F = P.shape[0]
    for m in diff:
        a, b = max(0, m - smooth), min(F, m + smooth + 1)
        E = P[a:b].sum(axis=0)
        assert got[m] >= l_lo and got[m] <= l_hi, (m, got[m])
        assert want[m] >= 0, (m, got[m], want[m])
        assert E[got[m]] >= E[want[m]] * (1 - 1e-5), (m, got[m], want[m], E[got[m]], E[want[m]])
    assert len(diff) <= max(2, len(got) // 1000)
    return len(diff)


@pytest.mark.parametrize("name", list(CFGS))
@pytest.mark.parametrize("smooth", [0, 2, 4, 9, 32])
def test_ridge_matches_oracle(sst, name, smooth):
    p, _, r = _oracle(name)
    F, nbo = r.T.shape
    T = _to_gpu(r.T)
    for l_lo, l_hi in ((0, nbo - 1), (nbo // 5, nbo // 5 + 300), (nbo // 2, nbo // 2)):
        l_hi = min(l_hi, nbo - 1)
        want = O.ridge(r.T, l_lo, l_hi, smooth)
        out = torch.empty(F, dtype=torch.int32, device="cuda")
        sst.sst_ridge(T, F, nbo, l_lo, l_hi, smooth, out)
        got = out.cpu().numpy().astype(np.int64)
        _check_ridge(got, want, r.T, l_lo, l_hi, smooth)


def test_ridge_ties_empty_frames_and_ragged_tiles(sst):
    F, nbo = 37, 600                      # 37 frames: a ragged last tile; 600 bins: three chunks
    T = np.zeros((F, nbo), np.complex128)
    T[0, [5, 300, 599]] = 2.0             # a three-way tie across chunks -> 5
    T[1, 450] = 1.0
    T[1, 451] = 1.0j                      # a tie inside one chunk -> 450
    T[3:, 599] = 0.5
    T[20, 10] = 0.8                       # single frame: beats the line alone, not once smoothed
    want0, want1 = O.ridge(T, 0, nbo - 1, 0), O.ridge(T, 0, nbo - 1, 1)
    Tg = _to_gpu(T)
    for smooth, want in ((0, want0), (1, want1)):
        out = torch.full((F,), 7, dtype=torch.int32, device="cuda")
        sst.sst_ridge(Tg, F, nbo, 0, nbo - 1, smooth, out)
        np.testing.assert_array_equal(out.cpu().numpy(), want)
    assert want0[0] == 5 and want0[1] == 450 and want0[2] == -1 and want0[20] == 10 and want1[20] == 599


@pytest.mark.parametrize("alpha", [3.0, 2.0, 0.5, 2.5])
def test_renyi_matches_oracle(sst, alpha):
    for name in CFGS:
        _, _, r = _oracle(name)
        T = _to_gpu(r.T)
        F, nbo = r.T.shape
        ws = torch.empty(max(sst.sst_renyi_workspace_bytes(), 256), dtype=torch.uint8, device="cuda")
        out = torch.empty(1, dtype=torch.float64, device="cuda")
        for cell in (1.0, 0.125):
            sst.sst_renyi(T, F, nbo, nbo, alpha, cell, out, ws)
            want = O.renyi(r.T.astype(np.complex64), alpha, cell)
            assert abs(float(out.item()) - want) < 1e-5 * max(1.0, abs(want)), (name, alpha, cell, out.item(), want)
        # a sub-grid through the row stride: the band's first 100 bins
        sst.sst_renyi(T, F, 100, nbo, alpha, 1.0, out, ws)
        want = O.renyi(r.T[:, :100].astype(np.complex64), alpha)
        assert abs(float(out.item()) - want) < 1e-5 * max(1.0, abs(want))


def test_renyi_closed_forms_on_device(sst):
    ws = torch.empty(max(sst.sst_renyi_workspace_bytes(), 256), dtype=torch.uint8, device="cuda")
    out = torch.empty(1, dtype=torch.float64, device="cuda")
    K = 3000 * 777
    T = torch.zeros((3000, 777, 2), dtype=torch.float32, device="cuda")
    T[..., 1] = 0.25
    sst.sst_renyi(T, 3000, 777, 777, 3.0, 1.0, out, ws)
    assert abs(out.item() - math.log2(K)) < 1e-9
    T.zero_()
    T[1234, 5, 0] = 3.0
    sst.sst_renyi(T, 3000, 777, 777, 3.0, 1.0, out, ws)
    assert abs(out.item()) < 1e-12
    T.zero_()
    sst.sst_renyi(T, 3000, 777, 777, 3.0, 1.0, out, ws)
    assert math.isnan(out.item())


def test_post_argument_checks(sst):
    T = torch.zeros((10, 20, 2), dtype=torch.float32, device="cuda")
    out = torch.empty(10, dtype=torch.int32, device="cuda")
    for args in ((0, 20, 0), (5, 4, 0), (0, 19, 33), (0, 19, -1)):
        with pytest.raises(sst.SstError):
            sst.sst_ridge(T, 10, 20, args[0], args[1], args[2], out)
    ws = torch.empty(max(sst.sst_renyi_workspace_bytes(), 256), dtype=torch.uint8, device="cuda")
    d = torch.empty(1, dtype=torch.float64, device="cuda")
    for alpha, cell in ((1.0, 1.0), (0.0, 1.0), (3.0, 0.0)):
        with pytest.raises(sst.SstError):
            sst.sst_renyi(T, 10, 20, 20, alpha, cell, d, ws)
    p, _, _ = _oracle("fullband")
    plan = sst.Plan(**p)
    with pytest.raises(sst.SstError):
        plan.inverse_zone(plan.new_tfr(), torch.zeros(plan.frames, dtype=torch.int32, device="cuda"), -1)
    plan.close()


def post_sweep_cases():
    from test_gpu_sweep import SHAPES, signal
    return [(i, SHAPES[i], signal) for i in range(2, len(SHAPES), 5)]


@pytest.mark.parametrize("case", post_sweep_cases(), ids=lambda c: f"shape{c[0]}_nf{c[1]['nfft']}_z{c[1]['z']}")
def test_zone_inverse_sweep_shapes(sst, case):
    """Every fifth shape of the plan-shape sweep through the zone inverse
    (oracle T in, zone half-width 3), against the oracle's."""
    i, p, signal = case
    x = signal(p, 100 + i)
    r = O.sst(x.astype(np.float64), p["fs"], p["L"], p["sigma"], p["hop"], p["nfft"], p["f_lo"], p["f_hi"],
              p["z"], p["gamma"], p["relative"])
    plan = sst.Plan(**p)
    F, nbo = r.T.shape
    ridge = _zone_centres(F, nbo, seed=i)
    g, _ = O.window(p["L"], p["sigma"])
    want = O.zone_inverse(r.T, ridge, 3, r.k_lo, p["nfft"], p["z"], g, p["hop"], p["n"])
    got = plan.inverse_zone(_to_gpu(r.T), torch.from_numpy(ridge).cuda(), 3).cpu().numpy().astype(np.float64)
    plan.close()
    full = np.abs(O.inverse(r.T, r.k_lo, p["nfft"], p["z"], g, p["hop"], p["n"])).max()
    err = np.abs(got - want).max()
    assert err <= XHAT_RTOL * full + 1e-7 * max(np.abs(want).max(), 1e-30), (err, full)

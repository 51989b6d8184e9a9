"""sst_forward_static: the forward transform for callers that cannot call
cudaMalloc when they run it (their device memory belongs to a host
application's pool, or the call sits in a loop that must not pay cudaMalloc's
device synchronisation).  It takes no workspace; its scratch is a fixed
64 KiB array inside libsst.so.

The tests call it through the C ABI twice in a row, on two different
signals, and check each result against sst_forward (which uses a caller
workspace) within the TFR tolerance of the parity tests, for a relative and
an absolute threshold (the absolute one's pre-pass, max |x|, also writes the
shared array).  The second signal is 1000x weaker than the first, so a
threshold or scale left over from the first call in the shared array would
change the second result.  The relative case is also compared with the FP64
oracle under the parity bars, and a plan that needs more scratch than the
array holds is rejected (through a test hook that lowers the capacity,
since no plan on this GPU needs that much).  It lives in its own file so
pytest collects it last."""
import numpy as np
import pytest

import oracle as O
from parity import as_complex, check_map, check_tfr_replay

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

T_RTOL = 1e-5


@pytest.fixture(scope="module")
def sst():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2003_07065_gb300 import build, sst as S
    build.build()
    S.load()
    return S


def _signal(n, fs):
    t = np.arange(n) / fs
    gen = np.random.default_rng(2024)
    return np.cos(2 * np.pi * (800 * t + 300 * t * t)) + 0.2 * gen.standard_normal(n)


@pytest.mark.parametrize("relative,gamma", [(True, 1e-3), (False, 0.05)], ids=["relative", "absolute"])
def test_forward_static_matches_forward(sst, relative, gamma):
    n, fs = 50000, 25600.0
    params = dict(n=n, fs=fs, L=1025, sigma=128.0, hop=16, nfft=1024, f_lo=0.0, f_hi=6400.0, z=2,
                  gamma=gamma, relative=relative)
    plan = sst.Plan(**params)
    base = _signal(n, fs)
    for scale in (1.0, 1e-3):
        x = torch.from_numpy((scale * base).astype(np.float32)).cuda()
        ref = plan.forward(x)
        got = torch.full_like(ref, float("nan"))
        sst.sst_forward_static(plan.handle, x, n, got)
        torch.cuda.synchronize()
        err = (got - ref).abs().max().item()
        assert torch.isfinite(got).all()
        assert err <= T_RTOL * max(ref.abs().max().item(), 1e-30), (scale, err)
        if not relative and scale < 1:
            assert ref.abs().max().item() == 0.0   # everything below the absolute threshold
    plan.close()


def test_forward_static_matches_oracle(sst):
    n, fs = 50000, 25600.0
    params = dict(n=n, fs=fs, L=1025, sigma=128.0, hop=16, nfft=1024, f_lo=0.0, f_hi=6400.0, z=2,
                  gamma=1e-3, relative=True)
    plan = sst.Plan(**params)
    x32 = _signal(n, fs).astype(np.float32)
    x = torch.from_numpy(x32).cuda()
    got = torch.empty((plan.frames, plan.bins, 2), dtype=torch.float32, device="cuda")
    sst.sst_forward_static(plan.handle, x, n, got)
    _, dest = plan.reassign_map(x)
    torch.cuda.synchronize()
    r = O.sst(x32.astype(np.float64), fs, params["L"], params["sigma"], params["hop"], params["nfft"],
              params["f_lo"], params["f_hi"], params["z"], params["gamma"], True)
    dg = dest.cpu().numpy()
    check_map(dg, r.dest, r.V, r.gamma, r.T.shape[1])
    check_tfr_replay(as_complex(got.cpu().numpy()), r.V, dg, r.dest, r.gamma, r.T.shape[1])
    plan.close()


def test_forward_static_rejects_plan_beyond_capacity(sst):
    plan = sst.Plan(n=20000, fs=8000.0, L=257, sigma=32.0, hop=8, nfft=256, f_lo=0.0, f_hi=4000.0)
    x = torch.zeros(20000, device="cuda")
    tfr = plan.new_tfr()
    try:
        sst.sst_test_static_capacity(64)        # the header only: no room for any pre-pass partial
        with pytest.raises(sst.SstError) as e:
            sst.sst_forward_static(plan.handle, x, 20000, tfr)
        assert e.value.status == 6
        assert "scratch floats" in str(e.value)
    finally:
        sst.sst_test_static_capacity(0)
    sst.sst_forward_static(plan.handle, x, 20000, tfr)
    torch.cuda.synchronize()
    plan.close()


def test_forward_static_rejects_bad_arguments(sst):
    plan = sst.Plan(n=1000, fs=1000.0, L=65, sigma=8.0, hop=8, nfft=64, f_lo=0.0, f_hi=500.0)
    x = torch.zeros(1000, device="cuda")
    with pytest.raises(sst.SstError) as e:
        sst.sst_forward_static(plan.handle, x, 999, plan.new_tfr())
    assert e.value.status == 1
    with pytest.raises(sst.SstError):
        sst.sst_forward_static(plan.handle, x, 1000, None)
    plan.close()

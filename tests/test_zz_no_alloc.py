"""sst_forward_static: the forward transform for callers that cannot call
cudaMalloc when they run it (their device memory belongs to a host
application's pool, or the call sits in a loop that must not pay cudaMalloc's
device synchronisation).  It takes no workspace; its scratch is a fixed
64 KiB array inside libsst.so.

The test calls it through the C ABI twice in a row, on two different
signals, and checks each result against sst_forward (which uses a caller
workspace) within the TFR tolerance of the parity tests.  The second signal
is 1000x weaker than the first, so a relative threshold left over from the
first call in the shared array would change the second result.  It lives in
its own file so pytest collects it last."""
import numpy as np
import pytest

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


def test_forward_static_matches_forward(sst):
    n, fs = 50000, 25600.0
    params = dict(n=n, fs=fs, L=1025, sigma=128.0, hop=16, nfft=1024, f_lo=0.0, f_hi=6400.0, z=2,
                  gamma=1e-3, relative=True)
    plan = sst.Plan(**params)
    t = np.arange(n) / fs
    gen = np.random.default_rng(2024)
    base = np.cos(2 * np.pi * (800 * t + 300 * t * t)) + 0.2 * gen.standard_normal(n)
    for scale in (1.0, 1e-3):
        x = torch.from_numpy((scale * base).astype(np.float32)).cuda()
        ref = plan.forward(x)
        got = torch.full_like(ref, float("nan"))
        sst.sst_forward_static(plan.handle, x, n, got)
        torch.cuda.synchronize()
        err = (got - ref).abs().max().item()
        assert torch.isfinite(got).all()
        assert err <= T_RTOL * ref.abs().max().item(), (scale, err)
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

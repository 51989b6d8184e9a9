"""sst_forward_inverse_host: the end-to-end call with host buffers.  Its
output lands in the host buffer either straight from the finalising kernel
(page-locked memory the device addresses) or by a copy after it (pageable
memory); both must carry the same bits as the device-buffer call, with and
without a TFR output, and leave the device output buffer written too."""
import numpy as np
import pytest

from paper_2003_07065_gb300 import workloads as W

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


@pytest.mark.parametrize("with_tfr", [True, False], ids=["tfr", "no_tfr"])
@pytest.mark.parametrize("pinned", [True, False], ids=["pinned", "pageable"])
def test_host_call_matches_device_call(sst, with_tfr, pinned):
    w = W.ALL["chirp_fm_64k"]
    x32 = w.signal()[0].astype(np.float32)
    plan = sst.Plan(**w.params())
    x_dev = torch.from_numpy(x32).cuda()
    tfr = plan.new_tfr() if with_tfr else None
    ref = torch.empty(plan.n, dtype=torch.float32, device="cuda")
    sst.sst_forward_inverse(plan.handle, x_dev, plan.n, tfr, ref, plan.workspace)
    x_host = torch.from_numpy(x32)
    xh_host = torch.full((plan.n,), float("nan"), dtype=torch.float32)
    if pinned:
        x_host = x_host.pin_memory()
        xh_host = xh_host.pin_memory()
    xh_dev = torch.full((plan.n,), float("nan"), dtype=torch.float32, device="cuda")
    x2 = torch.empty_like(x_dev)
    for _ in range(2):   # a repeat call overwrites the output again
        sst.sst_forward_inverse_host(plan.handle, x_host, plan.n, xh_host, x2, tfr, xh_dev, plan.workspace)
        assert torch.equal(xh_host, ref.cpu())
        assert torch.equal(xh_dev, ref)
        xh_host.fill_(float("nan"))
    plan.close()

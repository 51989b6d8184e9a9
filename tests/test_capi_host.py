"""CPU checks of the C ABI: the library builds for sm_103a, loads, exports
every function include/sst.h declares, and validates arguments on the host
(no GPU is touched: invalid parameters are rejected before any CUDA call)."""
import ctypes
import os
import re

import pytest

from paper_2003_07065_gb300 import build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions(header=None):
    """Functions declared in include/<header> (every header when None)."""
    names = set()
    inc = os.path.join(ROOT, "include")
    for f in os.listdir(inc):
        if f.endswith(".h") and (header is None or f == header):
            txt = open(os.path.join(inc, f)).read()
            txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
            names |= set(re.findall(r"\b(sst_[a-z0-9_]+)\s*\(", txt))
    return sorted(names)


@pytest.fixture(scope="module")
def lib():
    build.build()
    build.build_tc()
    from paper_2003_07065_gb300 import sst as S
    S.load()
    return S


def test_header_declares_entry_points():
    names = declared_functions()
    for n in ("sst_plan_create", "sst_forward", "sst_inverse", "sst_forward_inverse", "sst_plan_destroy"):
        assert n in names


def test_library_exports_every_declared_symbol(lib):
    so = ctypes.CDLL(build.LIB)
    missing = [n for n in declared_functions("sst.h") if not hasattr(so, n)]
    assert not missing, missing
    assert set(declared_functions()) == set(declared_functions("sst.h")) | set(declared_functions("sst_tc.h"))


def test_tensor_library_exports_its_symbols(lib):
    so = ctypes.CDLL(build.TC_LIB)
    names = declared_functions("sst_tc.h")
    assert names and all(n.startswith("sst_tc_") for n in names)
    missing = [n for n in names if not hasattr(so, n)]
    assert not missing, missing
    # the tensor form lives in its own library only
    base = ctypes.CDLL(build.LIB)
    assert not any(hasattr(base, n) for n in names)


def test_multi_gpu_library_has_no_cluster_multicast_loads():
    """libsst.so, the library every multi-GPU program loads, is built from
    csrc/*.cu, *.cuh, *.h alone: none of them issues a multicast TMA load or
    a multicast commit (the tensor form, which does, is csrc/tc/, built into
    libsst_tc.so)."""
    csrc = os.path.join(ROOT, "paper_2003_07065_gb300", "csrc")
    for f in os.listdir(csrc):
        path = os.path.join(csrc, f)
        if os.path.isfile(path) and f.endswith((".cu", ".cuh", ".h")):
            assert "multicast" not in open(path).read(), f


def test_binding_loads_tensor_library_only_on_demand():
    import subprocess
    import sys
    code = ("import sys; sys.path.insert(0, %r)\n"
            "from paper_2003_07065_gb300 import build, sst\n"
            "build.build(); sst.load()\n"
            "maps = open('/proc/self/maps').read()\n"
            "assert 'libsst.so' in maps and 'libsst_tc.so' not in maps, 'tc loaded'\n"
            "assert not sst.tc_loaded()\n" % ROOT)
    r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr


def test_status_strings(lib):
    assert lib.sst_status_string(0) == "SST_OK"
    assert lib.sst_status_string(1) == "SST_EINVAL"
    assert lib.sst_status_string(6) == "SST_EUNSUPPORTED"


BAD = [
    (dict(L=64), "L must be odd"),
    (dict(nfft=1000), "power of two"),
    (dict(nfft=32), "power of two"),
    (dict(hop=0), "hop"),
    (dict(hop=40), "hop"),
    (dict(f_lo=300.0, f_hi=200.0), "band"),
    (dict(f_hi=600.0), "band"),
    (dict(z=0), "z must"),
    (dict(z=17), "z must"),
    (dict(gamma=-1.0), "gamma"),
    (dict(n=0), "n must"),
    (dict(sigma=0.0), "sigma"),
]


@pytest.mark.parametrize("change,msg", BAD)
def test_invalid_parameters_rejected_on_host(lib, change, msg):
    kw = dict(n=1000, fs=1000.0, L=65, sigma=8.0, hop=8, nfft=64, f_lo=0.0, f_hi=500.0, z=1,
              gamma=1e-3, relative=True)
    kw.update(change)
    with pytest.raises(lib.SstError) as e:
        lib.sst_plan_create(**kw)
    assert e.value.status == 1
    assert msg in str(e.value)


def test_window_longer_than_the_limit_rejected(lib):
    """Any odd L up to SST_MAX_L = 8193 is valid for every nfft (a window
    longer than nfft is folded, Eq. 8); a longer one is an argument error,
    found before any device call."""
    with pytest.raises(lib.SstError) as e:
        lib.sst_plan_create(n=100000, fs=1000.0, L=lib.SST_MAX_L + 2, sigma=8.0, hop=8, nfft=64, f_lo=0, f_hi=500)
    assert e.value.status == 1
    assert str(lib.SST_MAX_L) in str(e.value)
    hdr = open(os.path.join(build.INCLUDE, "sst.h")).read()
    assert re.search(r"#define SST_MAX_L (\d+)", hdr).group(1) == str(lib.SST_MAX_L)


def test_null_arguments(lib):
    L = lib.load()
    assert L.sst_plan_create(None, None) == 1
    assert L.sst_forward(None, None, 0, None, None, None) == 1
    assert L.sst_plan_query(None, None, None, None, None, None) == 1
    L.sst_plan_destroy(None)


def test_host_calls_return_promptly(lib):
    """Entry points that fail validation or find no device return at once
    (a regression guard for host-side loops: runs in a child with a timeout)."""
    import subprocess
    import sys
    code = ("import sys; sys.path.insert(0, %r)\n"
            "from paper_2003_07065_gb300 import sst as S\n"
            "L = S.load()\n"
            "print(L.sst_launch_count())\n"
            "for _ in range(3):\n"
            "    try:\n"
            "        S.sst_plan_create(n=1000, fs=1000.0, L=65, sigma=8.0, hop=8, nfft=64, f_lo=0, f_hi=500)\n"
            "    except S.SstError as e:\n"
            "        print(e.status)\n" % ROOT)
    r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, timeout=120)
    assert r.returncode == 0, r.stderr


def test_post_steps_reject_bad_arguments_on_host(lib):
    """sst_ridge, sst_renyi and sst_inverse_zone validate before any CUDA call
    (the pointers below are never dereferenced)."""
    L = lib.load()
    t, r = 1 << 12, 1 << 13          # 8-byte aligned stand-ins for device pointers
    assert L.sst_ridge(None, 10, 20, 0, 19, 0, r, None) == 1
    assert L.sst_ridge(t, 10, 20, 0, 20, 0, r, None) == 1          # l_hi past the bins
    assert L.sst_ridge(t, 10, 20, 5, 4, 0, r, None) == 1           # empty band
    assert L.sst_ridge(t, 10, 20, 0, 19, 33, r, None) == 1         # smoothing past the limit
    assert L.sst_ridge(t, 10, 20, 0, 19, -1, r, None) == 1
    assert L.sst_ridge(t + 4, 10, 20, 0, 19, 0, r, None) == 1      # TFR not 8-byte aligned
    assert L.sst_ridge(t, 0, 20, 0, 19, 0, r, None) == 1           # no frames
    ws, out = 1 << 16, 1 << 14
    assert L.sst_renyi_workspace_bytes() >= 256
    assert L.sst_renyi(None, 10, 20, 20, 3.0, 1.0, out, ws, None) == 1
    assert L.sst_renyi(t, 10, 20, 20, 1.0, 1.0, out, ws, None) == 1   # alpha = 1
    assert L.sst_renyi(t, 10, 20, 20, 0.0, 1.0, out, ws, None) == 1
    assert L.sst_renyi(t, 10, 20, 20, 3.0, 0.0, out, ws, None) == 1   # cell area
    assert L.sst_renyi(t, 0, 20, 20, 3.0, 1.0, out, ws, None) == 1    # empty grid
    assert L.sst_renyi(t, 10, 20, 19, 3.0, 1.0, out, ws, None) == 1   # row stride below the columns
    assert L.sst_renyi(t, 10, 20, 20, 3.0, 1.0, out, ws + 8, None) == 1   # workspace alignment
    assert L.sst_inverse_zone(None, t, 10, r, 3, out, ws, None) == 1


def test_binding_checks_tensor_arguments():
    """The checks a raw pointer cannot carry through the C ABI (element type,
    device, contiguity, size), made by the binding before a call."""
    torch = pytest.importorskip("torch")
    from paper_2003_07065_gb300.sst import check_tensor
    x = torch.zeros(100, dtype=torch.float32)
    assert check_tensor(x, "x", torch.float32, 100) is x            # a host tensor where a host one is wanted
    for bad, why in [(x.double(), "expected torch.float32"), (x[::2], "contiguous"), (x[:99], "needs 100"),
                     (x.numpy(), "expected a torch tensor")]:
        with pytest.raises(ValueError, match=why):
            check_tensor(bad, "x", torch.float32, 100)
    with pytest.raises(ValueError, match="expected a tensor on cuda:0"):
        check_tensor(x, "x", torch.float32, 100, torch.device("cuda", 0))


def test_binding_constants_match_the_headers():
    """Every SST_* constant the binding mirrors has the header's value, and the
    status names follow the header's enum."""
    from paper_2003_07065_gb300 import sst as S
    seen = 0
    for h in ("sst.h", "sst_tc.h"):
        text = open(os.path.join(build.INCLUDE, h)).read()
        for name, val in re.findall(r"#define (SST_\w+) (0x[0-9a-fA-F]+|\d+)u?\b", text):
            if hasattr(S, name):
                assert getattr(S, name) == int(val, 0), name
                seen += 1
    assert seen >= 10
    enum = re.search(r"typedef enum \{(.*?)\} sst_status;", open(os.path.join(build.INCLUDE, "sst.h")).read(), re.S)
    for name, val in re.findall(r"(SST_\w+) = (\d+)", enum.group(1)):
        assert S.STATUS[int(val)] == name


def test_binding_signatures_match_the_headers(lib):
    """Each entry point the binding declares takes as many arguments as its
    prototype in include/sst.h or include/sst_tc.h (a wrong count would
    misplace every argument after it)."""
    from paper_2003_07065_gb300 import sst as S
    protos = {}
    for h in ("sst.h", "sst_tc.h"):
        text = re.sub(r"/\*.*?\*/", "", open(os.path.join(build.INCLUDE, h)).read(), flags=re.S)
        for name, args in re.findall(r"\b(sst_\w+)\s*\(([^;{]*?)\)\s*;", text):
            args = " ".join(args.split())
            protos[name] = 0 if args in ("", "void") else args.count(",") + 1
    tc = S.load_tc()
    checked = 0
    for so in (S.load(), tc):
        for name, n in protos.items():
            f = getattr(so, name, None)
            if f is not None and f.argtypes is not None:
                assert len(f.argtypes) == n, (name, len(f.argtypes), n)
                checked += 1
    assert checked >= 40

"""ctypes binding of libsst.so (declared in include/sst.h) and of the
tensor-core band form's libsst_tc.so (include/sst_tc.h).

Argument marshalling only: every function here forwards to the C entry point
of the same name, passing device pointers (``tensor.data_ptr()``) and the
``cudaStream_t`` of a torch stream (the ``Plan`` class first checks each
tensor argument's element type, device, contiguity and size, which a raw
pointer cannot carry).  The libraries must have been built
(``paper_2003_07065_gb300.build.build()``, ``build.build_tc()``); loading
fails loudly otherwise, and there is no CPU fallback.  libsst_tc.so is loaded
only when a ``sst_tc_*`` function is first called.
"""
from __future__ import annotations

import ctypes
import os

from . import build as _build

SST_MAX_L = 8193            # the longest window a plan takes (any Nf; longer than Nf is folded)
SST_GAMMA_RELATIVE = 0x1
SST_TWO_PASS = 0x2
SST_STREAM_XHAT_ONLY = 0x100
STATUS = {0: "SST_OK", 1: "SST_EINVAL", 2: "SST_ENOMEM", 3: "SST_ECUDA", 4: "SST_EBUSY",
          5: "SST_ETIMEOUT", 6: "SST_EUNSUPPORTED", 7: "SST_EINTERNAL"}


class SstError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


class sst_params(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int64), ("fs", ctypes.c_double), ("L", ctypes.c_int32),
                ("sigma", ctypes.c_double), ("g", ctypes.POINTER(ctypes.c_double)),
                ("dg", ctypes.POINTER(ctypes.c_double)), ("hop", ctypes.c_int32),
                ("nfft", ctypes.c_int32), ("f_lo", ctypes.c_double), ("f_hi", ctypes.c_double),
                ("z", ctypes.c_int32), ("gamma", ctypes.c_double), ("flags", ctypes.c_uint32)]


class sst_param_report(ctypes.Structure):
    _fields_ = [("sigma_s", ctypes.c_double), ("sigma_f_hz", ctypes.c_double), ("hf", ctypes.c_double),
                ("hf_max_eq38", ctypes.c_double), ("hf_max_eq46", ctypes.c_double),
                ("delta_f_hz", ctypes.c_double), ("delta_f_fine_hz", ctypes.c_double),
                ("delta_f_max_eq37_hz", ctypes.c_double), ("delta_f_max_eq46_hz", ctypes.c_double),
                ("flags", ctypes.c_uint32)]


class sst_part(ctypes.Structure):
    _fields_ = [(f, ctypes.c_int64) for f in ("tile_begin", "tile_end", "frame_begin", "frame_end", "x_begin",
                                               "x_end", "out_begin", "out_end", "need_begin", "need_end")]

    def as_dict(self) -> dict:
        return {f: getattr(self, f) for f, _ in self._fields_}


SST_GUARD_EQ38 = 0x1
SST_GUARD_EQ46 = 0x2


class sst_batch_item(ctypes.Structure):
    _fields_ = [("plan", ctypes.c_void_p), ("x", ctypes.c_void_p), ("n", ctypes.c_int64),
                ("tfr", ctypes.c_void_p), ("xhat", ctypes.c_void_p)]


SST_BATCH_GRAPH = 0x1

_lib = None
_vp = ctypes.c_void_p
_i64 = ctypes.c_int64


def lib_path() -> str:
    return _build.LIB


def tc_loaded() -> bool:
    """Whether this process has loaded libsst_tc.so."""
    return _tc_lib is not None


def load():
    """Load libsst.so; raises if it has not been built."""
    global _lib
    if _lib is not None:
        return _lib
    path = _build.LIB
    if not os.path.exists(path):
        raise RuntimeError(f"libsst.so not built at {path}: run paper_2003_07065_gb300.build.build()")
    lib = ctypes.CDLL(path)
    sig = {
        "sst_plan_create": ([ctypes.POINTER(sst_params), ctypes.POINTER(_vp)], ctypes.c_int),
        "sst_plan_destroy": ([_vp], None),
        "sst_plan_query": ([_vp, ctypes.POINTER(_i64), ctypes.POINTER(ctypes.c_int32),
                            ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_int32),
                            ctypes.POINTER(ctypes.c_size_t)], ctypes.c_int),
        "sst_params_check": ([ctypes.POINTER(sst_params), ctypes.POINTER(sst_param_report)], ctypes.c_int),
        "sst_plan_check": ([_vp, ctypes.POINTER(sst_param_report)], ctypes.c_int),
        "sst_forward": ([_vp, _vp, _i64, _vp, _vp, _vp], ctypes.c_int),
        "sst_part_layout": ([_vp, ctypes.c_int32, ctypes.c_int32, ctypes.POINTER(sst_part)], ctypes.c_int),
        "sst_part_segments": ([_vp, ctypes.POINTER(ctypes.c_size_t), ctypes.POINTER(ctypes.c_int32),
                               ctypes.POINTER(_i64)], ctypes.c_int),
        "sst_part_prepass": ([_vp, ctypes.POINTER(sst_part), _vp, _vp, _vp, _vp], ctypes.c_int),
        "sst_part_forward_inverse": ([_vp, ctypes.POINTER(sst_part), _vp, _vp, _vp, _vp], ctypes.c_int),
        "sst_part_finalize": ([_vp, ctypes.POINTER(sst_part), _vp, _vp, _vp], ctypes.c_int),
        "sst_inverse": ([_vp, _vp, _i64, _vp, _vp, _vp], ctypes.c_int),
        "sst_forward_inverse": ([_vp, _vp, _i64, _vp, _vp, _vp, _vp], ctypes.c_int),
        "sst_inverse_zone": ([_vp, _vp, _i64, _vp, ctypes.c_int32, _vp, _vp, _vp], ctypes.c_int),
        "sst_ridge": ([_vp, _i64, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, _vp, _vp],
                      ctypes.c_int),
        "sst_renyi_workspace_bytes": ([], ctypes.c_size_t),
        "sst_renyi": ([_vp, _i64, ctypes.c_int32, _i64, ctypes.c_double, ctypes.c_double, _vp, _vp, _vp],
                      ctypes.c_int),
        "sst_forward_inverse_host": ([_vp, _vp, _i64, _vp, _vp, _vp, _vp, _vp, _vp], ctypes.c_int),
        "sst_stft": ([_vp, _vp, _i64, _vp, _vp, _vp, _vp], ctypes.c_int),
        "sst_reassign_map": ([_vp, _vp, _i64, _vp, _vp, _vp, _vp], ctypes.c_int),
        "sst_forward2": ([_vp, _vp, _i64, _vp, _vp, _vp], ctypes.c_int),
        "sst_reassign_map2": ([_vp, _vp, _i64, _vp, _vp, _vp, _vp], ctypes.c_int),
        "sst_max_abs_v": ([_vp, _vp, _i64, _vp, _vp, _vp], ctypes.c_int),
        "sst_forward_static": ([_vp, _vp, _i64, _vp, _vp], ctypes.c_int),
        "sst_fp32_peak": ([ctypes.POINTER(ctypes.c_double), _vp], ctypes.c_int),
        "sst_check": ([_vp, _vp, _vp], ctypes.c_int),
        "sst_test_static_capacity": ([ctypes.c_size_t], ctypes.c_int),
        "sst_test_withhold_row_copy": ([_vp], ctypes.c_int),
        "sst_test_withhold_sample_copy": ([_vp], ctypes.c_int),
        "sst_threshold_stats": ([_vp, _vp, ctypes.POINTER(_i64), ctypes.POINTER(_i64),
                                 ctypes.POINTER(ctypes.c_int32)], ctypes.c_int),
        "sst_batch_create": ([ctypes.POINTER(sst_batch_item), ctypes.c_int32, ctypes.c_uint32,
                              ctypes.POINTER(_vp)], ctypes.c_int),
        "sst_batch_workspace": ([_vp, ctypes.POINTER(ctypes.c_size_t)], ctypes.c_int),
        "sst_batch_run": ([_vp, _vp, _vp], ctypes.c_int),
        "sst_batch_tune": ([_vp, _vp, _vp, ctypes.POINTER(ctypes.c_double),
                            ctypes.POINTER(ctypes.c_double)], ctypes.c_int),
        "sst_batch_knobs": ([_vp, ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_int32),
                             ctypes.POINTER(ctypes.c_int32)], ctypes.c_int),
        "sst_batch_destroy": ([_vp], None),
        "sst_batch_submit": ([ctypes.POINTER(sst_batch_item), ctypes.c_int32, _vp, ctypes.c_size_t, _vp],
                             ctypes.c_int),
        "sst_batch_workspace_for": ([ctypes.POINTER(sst_batch_item), ctypes.c_int32,
                                     ctypes.POINTER(ctypes.c_size_t)], ctypes.c_int),
        "sst_service_create": ([ctypes.c_int32, ctypes.c_size_t, ctypes.POINTER(_vp)], ctypes.c_int),
        "sst_stream_open": ([_vp, ctypes.POINTER(sst_params), ctypes.c_float, _i64,
                             ctypes.POINTER(ctypes.c_int32)], ctypes.c_int),
        "sst_stream_push": ([_vp, ctypes.c_int32, _vp, _i64, ctypes.c_double], ctypes.c_int),
        "sst_stream_close": ([_vp, ctypes.c_int32], ctypes.c_int),
        "sst_service_tick": ([_vp], ctypes.c_int),
        "sst_stream_poll": ([_vp, ctypes.c_int32, _vp, _i64, ctypes.POINTER(_i64), ctypes.POINTER(_i64), _vp,
                             _i64, ctypes.POINTER(_i64), ctypes.POINTER(_i64), ctypes.POINTER(ctypes.c_int32)],
                            ctypes.c_int),
        "sst_stream_release": ([_vp, ctypes.c_int32], ctypes.c_int),
        "sst_service_latency": ([_vp, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double),
                                 ctypes.POINTER(_i64), ctypes.c_int32], ctypes.c_int),
        "sst_service_memory": ([_vp, ctypes.POINTER(ctypes.c_size_t), ctypes.POINTER(ctypes.c_size_t)],
                               ctypes.c_int),
        "sst_service_destroy": ([_vp], None),
        "sst_sync": ([_vp], ctypes.c_int),
        "sst_launch_count": ([], ctypes.c_uint64),
        "sst_profile_enable": ([ctypes.c_int], ctypes.c_int),
        "sst_profile_collect": ([ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_uint64)],
                                ctypes.c_int),
        "sst_profile_kind_name": ([ctypes.c_int], ctypes.c_char_p),
        "sst_status_string": ([ctypes.c_int], ctypes.c_char_p),
        "sst_last_error": ([], ctypes.c_char_p),
    }
    for name, (args, res) in sig.items():
        f = getattr(lib, name)
        f.argtypes = args
        f.restype = res
    _lib = lib
    return lib


_tc_lib = None


def load_tc():
    """Load libsst_tc.so, the tensor-core band form (single-GPU programs
    only; it links against libsst.so, loaded first).  Raises if it has not
    been built (``build.build_tc()``)."""
    global _tc_lib
    if _tc_lib is not None:
        return _tc_lib
    load()
    path = _build.TC_LIB
    if not os.path.exists(path):
        raise RuntimeError(f"libsst_tc.so not built at {path}: run paper_2003_07065_gb300.build.build_tc()")
    lib = ctypes.CDLL(path)
    sig = {
        "sst_tc_plan_create": ([_vp, ctypes.c_int32, ctypes.POINTER(_vp)], ctypes.c_int),
        "sst_tc_plan_destroy": ([_vp], None),
        "sst_tc_plan_query": ([_vp, ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(_i64),
                               ctypes.POINTER(ctypes.c_int32)], ctypes.c_int),
        "sst_tc_plan_set_cluster": ([_vp, ctypes.c_int32], ctypes.c_int),
        "sst_tc_plan_tune": ([_vp, _vp, _i64, _vp, ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_float)],
                             ctypes.c_int),
        "sst_tc_forward": ([_vp, _vp, _i64, _vp, _vp], ctypes.c_int),
        "sst_tc_stft": ([_vp, _vp, _i64, _vp, _vp, _vp], ctypes.c_int),
        "sst_tc_reassign_map": ([_vp, _vp, _i64, _vp, _vp, _vp], ctypes.c_int),
        "sst_tc_contract": ([_vp, _vp, _i64, _vp], ctypes.c_int),
        "sst_tc_check": ([_vp, _vp], ctypes.c_int),
        "sst_tc_plan_test_withhold": ([_vp], ctypes.c_int),
    }
    for name, (args, res) in sig.items():
        f = getattr(lib, name)
        f.argtypes = args
        f.restype = res
    _tc_lib = lib
    return lib


def _check(status: int):
    if status != 0:
        raise SstError(status, load().sst_last_error().decode(errors="replace"))


def _ptr(t) -> int | None:
    if t is None:
        return None
    if isinstance(t, int):
        return t
    return t.data_ptr()


def _stream(stream) -> int | None:
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


# ------------------------------------------------------------------ C names
def _params(n, fs, L, hop, nfft, f_lo, f_hi, z, gamma, relative, sigma, g, dg, two_pass=False):
    p = sst_params()
    p.n, p.fs, p.L = int(n), float(fs), int(L)
    p.sigma = float(sigma) if sigma is not None else 0.0
    keep = []
    if g is not None:
        import numpy as np
        ga = np.ascontiguousarray(g, dtype=np.float64)
        da = np.ascontiguousarray(dg, dtype=np.float64)
        keep = [ga, da]
        p.g = ga.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
        p.dg = da.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    p.hop, p.nfft = int(hop), int(nfft)
    p.f_lo, p.f_hi, p.z = float(f_lo), float(f_hi), int(z)
    p.gamma = float(gamma)
    p.flags = (SST_GAMMA_RELATIVE if relative else 0) | (SST_TWO_PASS if two_pass else 0)
    return p, keep


def sst_plan_create(n: int, fs: float, L: int, hop: int, nfft: int, f_lo: float, f_hi: float,
                    z: int = 1, gamma: float = 1e-3, relative: bool = True, sigma: float | None = None,
                    g=None, dg=None, two_pass: bool = False) -> int:
    """Returns an opaque plan handle (int).  g, dg: optional FP64 numpy windows;
    two_pass: SST_TWO_PASS (separate max|V| pre-pass for relative thresholds)."""
    lib = load()
    p, keep = _params(n, fs, L, hop, nfft, f_lo, f_hi, z, gamma, relative, sigma, g, dg, two_pass)
    out = _vp()
    _check(lib.sst_plan_create(ctypes.byref(p), ctypes.byref(out)))
    del keep
    return out.value


def _report(r) -> dict:
    out = {name: getattr(r, name) for name, _ in sst_param_report._fields_}
    out["beyond_eq38"] = bool(r.flags & SST_GUARD_EQ38)
    out["beyond_eq46"] = bool(r.flags & SST_GUARD_EQ46)
    return out


def sst_params_check(n: int, fs: float, L: int, hop: int, nfft: int, f_lo: float, f_hi: float,
                     z: int = 1, gamma: float = 1e-3, relative: bool = True, sigma: float | None = None,
                     g=None, dg=None) -> dict:
    """Parameter guard of Sec. 4 (Eq. 35, 38, 46) for a parameter set; host
    arithmetic, no device needed."""
    p, keep = _params(n, fs, L, hop, nfft, f_lo, f_hi, z, gamma, relative, sigma, g, dg)
    r = sst_param_report()
    _check(load().sst_params_check(ctypes.byref(p), ctypes.byref(r)))
    del keep
    return _report(r)


def sst_plan_check(plan: int) -> dict:
    r = sst_param_report()
    _check(load().sst_plan_check(plan, ctypes.byref(r)))
    return _report(r)


def sst_part_layout(plan, part: int, parts: int) -> sst_part:
    out = sst_part()
    _check(load().sst_part_layout(plan, part, parts, ctypes.byref(out)))
    return out


def sst_part_segments(plan) -> tuple:
    """(byte offset of tile 0's segment in the workspace, floats per segment, tiles)."""
    off, sl, nt = ctypes.c_size_t(), ctypes.c_int32(), _i64()
    _check(load().sst_part_segments(plan, ctypes.byref(off), ctypes.byref(sl), ctypes.byref(nt)))
    return off.value, sl.value, nt.value


def sst_part_prepass(plan, part, x, r, workspace, stream=None):
    _check(load().sst_part_prepass(plan, ctypes.byref(part), _ptr(x), _ptr(r), _ptr(workspace), _stream(stream)))


def sst_part_forward_inverse(plan, part, x, r, workspace, stream=None):
    _check(load().sst_part_forward_inverse(plan, ctypes.byref(part), _ptr(x), _ptr(r), _ptr(workspace),
                                           _stream(stream)))


def sst_part_finalize(plan, part, workspace, xhat, stream=None):
    _check(load().sst_part_finalize(plan, ctypes.byref(part), _ptr(workspace), _ptr(xhat), _stream(stream)))


def sst_plan_destroy(plan: int) -> None:
    load().sst_plan_destroy(plan)


def sst_plan_query(plan: int) -> dict:
    f, b, lo, hi, ws = _i64(), ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int32(), ctypes.c_size_t()
    _check(load().sst_plan_query(plan, ctypes.byref(f), ctypes.byref(b), ctypes.byref(lo),
                                 ctypes.byref(hi), ctypes.byref(ws)))
    return {"frames": f.value, "bins": b.value, "k_lo": lo.value, "k_hi": hi.value,
            "workspace_bytes": ws.value}


def sst_forward(plan, x, n, tfr, workspace, stream=None):
    _check(load().sst_forward(plan, _ptr(x), n, _ptr(tfr), _ptr(workspace), _stream(stream)))


def sst_inverse(plan, tfr, n, xhat, workspace, stream=None):
    _check(load().sst_inverse(plan, _ptr(tfr), n, _ptr(xhat), _ptr(workspace), _stream(stream)))


def sst_inverse_zone(plan, tfr, n, ridge, half_width, xhat, workspace, stream=None):
    _check(load().sst_inverse_zone(plan, _ptr(tfr), n, _ptr(ridge), int(half_width), _ptr(xhat), _ptr(workspace),
                                   _stream(stream)))


def sst_ridge(tfr, frames, bins, l_lo, l_hi, smooth, ridge, stream=None):
    _check(load().sst_ridge(_ptr(tfr), int(frames), int(bins), int(l_lo), int(l_hi), int(smooth), _ptr(ridge),
                            _stream(stream)))


def sst_renyi_workspace_bytes():
    return int(load().sst_renyi_workspace_bytes())


def sst_renyi(tfr, rows, cols, ld, alpha, cell, out, workspace, stream=None):
    _check(load().sst_renyi(_ptr(tfr), int(rows), int(cols), int(ld), float(alpha), float(cell), _ptr(out),
                            _ptr(workspace), _stream(stream)))


def sst_forward_inverse(plan, x, n, tfr, xhat, workspace, stream=None):
    _check(load().sst_forward_inverse(plan, _ptr(x), n, _ptr(tfr), _ptr(xhat), _ptr(workspace),
                                      _stream(stream)))


def sst_forward_inverse_host(plan, x_host, n, xhat_host, x_dev, tfr_dev, xhat_dev, workspace,
                             stream=None):
    _check(load().sst_forward_inverse_host(plan, _ptr(x_host), n, _ptr(xhat_host), _ptr(x_dev),
                                           _ptr(tfr_dev), _ptr(xhat_dev), _ptr(workspace),
                                           _stream(stream)))


def sst_stft(plan, x, n, V, Vd, workspace, stream=None):
    _check(load().sst_stft(plan, _ptr(x), n, _ptr(V), _ptr(Vd), _ptr(workspace), _stream(stream)))


def sst_reassign_map(plan, x, n, omega, dest, workspace, stream=None):
    _check(load().sst_reassign_map(plan, _ptr(x), n, _ptr(omega), _ptr(dest), _ptr(workspace),
                                   _stream(stream)))


def sst_forward2(plan, x, n, tfr, workspace, stream=None):
    _check(load().sst_forward2(plan, _ptr(x), n, _ptr(tfr), _ptr(workspace), _stream(stream)))


def sst_reassign_map2(plan, x, n, omega2, dest, workspace, stream=None):
    _check(load().sst_reassign_map2(plan, _ptr(x), n, _ptr(omega2), _ptr(dest), _ptr(workspace), _stream(stream)))


def sst_max_abs_v(plan, x, n, maxv, workspace, stream=None):
    _check(load().sst_max_abs_v(plan, _ptr(x), n, _ptr(maxv), _ptr(workspace), _stream(stream)))


def sst_forward_static(plan, x, n, tfr, stream=None):
    _check(load().sst_forward_static(plan, _ptr(x), n, _ptr(tfr), _stream(stream)))


SST_FORM_BF16, SST_FORM_BF16X3, SST_FORM_TF32 = 0, 1, 2
FORMS = {"bf16": SST_FORM_BF16, "bf16x3": SST_FORM_BF16X3, "tf32": SST_FORM_TF32}


def sst_tc_plan_create(plan, form: int) -> int:
    h = _vp()
    _check(load_tc().sst_tc_plan_create(plan, form, ctypes.byref(h)))
    return h.value


def sst_tc_plan_destroy(tc) -> None:
    load_tc().sst_tc_plan_destroy(tc)


def sst_tc_plan_query(tc) -> dict:
    hv, fl, cl = ctypes.c_int32(), _i64(), ctypes.c_int32()
    _check(load_tc().sst_tc_plan_query(tc, ctypes.byref(hv), ctypes.byref(fl), ctypes.byref(cl)))
    return {"hankel_view": bool(hv.value), "gemm_flops": fl.value, "cluster": cl.value}


def sst_tc_plan_set_cluster(tc, cluster: int) -> None:
    _check(load_tc().sst_tc_plan_set_cluster(tc, cluster))


def sst_tc_plan_tune(tc, x, n, stream=None) -> tuple:
    """(chosen cluster size, its contraction time in ms)."""
    cl, ms = ctypes.c_int32(), ctypes.c_float()
    _check(load_tc().sst_tc_plan_tune(tc, _ptr(x), n, _stream(stream), ctypes.byref(cl), ctypes.byref(ms)))
    return cl.value, ms.value


def sst_tc_forward(tc, x, n, tfr, stream=None):
    _check(load_tc().sst_tc_forward(tc, _ptr(x), n, _ptr(tfr), _stream(stream)))


def sst_tc_stft(tc, x, n, V, Vd, stream=None):
    _check(load_tc().sst_tc_stft(tc, _ptr(x), n, _ptr(V), _ptr(Vd), _stream(stream)))


def sst_tc_reassign_map(tc, x, n, omega, dest, stream=None):
    _check(load_tc().sst_tc_reassign_map(tc, _ptr(x), n, _ptr(omega), _ptr(dest), _stream(stream)))


def sst_tc_contract(tc, x, n, stream=None):
    _check(load_tc().sst_tc_contract(tc, _ptr(x), n, _stream(stream)))


def sst_tc_check(tc, stream=None):
    _check(load_tc().sst_tc_check(tc, _stream(stream)))


def sst_tc_plan_test_withhold(tc):
    _check(load_tc().sst_tc_plan_test_withhold(tc))


def sst_fp32_peak(stream=None) -> float:
    """Measured FP32 FMA throughput of the current device, TFLOP/s."""
    t = ctypes.c_double()
    _check(load().sst_fp32_peak(ctypes.byref(t), _stream(stream)))
    return t.value


def sst_test_static_capacity(floats: int):
    _check(load().sst_test_static_capacity(int(floats)))


def sst_check(plan, workspace, stream=None):
    """Raises SstError(SST_ETIMEOUT) if the last inverse on this workspace gave
    up a bounded wait (its output is still correct)."""
    _check(load().sst_check(plan, _ptr(workspace), _stream(stream)))


def sst_test_withhold_row_copy(plan):
    _check(load().sst_test_withhold_row_copy(plan))


def sst_test_withhold_sample_copy(plan):
    _check(load().sst_test_withhold_sample_copy(plan))


def sst_threshold_stats(plan, workspace) -> dict:
    w, b, f = _i64(), _i64(), ctypes.c_int32()
    _check(load().sst_threshold_stats(plan, _ptr(workspace), ctypes.byref(w), ctypes.byref(b), ctypes.byref(f)))
    return {"waiting": w.value, "bins": b.value, "fell_back": bool(f.value)}


def _items(items):
    arr = (sst_batch_item * len(items))()
    for i, (plan, x, n, tfr, xhat) in enumerate(items):
        arr[i].plan, arr[i].x, arr[i].n = plan, _ptr(x), int(n)
        arr[i].tfr, arr[i].xhat = _ptr(tfr), _ptr(xhat)
    return arr


def sst_batch_create(items, graph: bool = False) -> int:
    """items: sequence of (plan handle, x, n, tfr, xhat); returns a batch handle."""
    arr = _items(items)
    out = _vp()
    _check(load().sst_batch_create(arr, len(items), SST_BATCH_GRAPH if graph else 0, ctypes.byref(out)))
    return out.value


def sst_batch_workspace(batch) -> int:
    b = ctypes.c_size_t()
    _check(load().sst_batch_workspace(batch, ctypes.byref(b)))
    return b.value


def sst_batch_run(batch, workspace, stream=None):
    _check(load().sst_batch_run(batch, _ptr(workspace), _stream(stream)))


def sst_batch_tune(batch, workspace, stream=None):
    """Returns (untuned ms, tuned ms) per batch run."""
    u, t = ctypes.c_double(), ctypes.c_double()
    _check(load().sst_batch_tune(batch, _ptr(workspace), _stream(stream), ctypes.byref(u), ctypes.byref(t)))
    return u.value, t.value


def sst_batch_knobs(batch) -> dict:
    a, b_, c = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int32()
    _check(load().sst_batch_knobs(batch, ctypes.byref(a), ctypes.byref(b_), ctypes.byref(c)))
    return {"fwd_frames": a.value, "abs_quads": b_.value, "grid_mul": c.value}


def sst_batch_destroy(batch):
    load().sst_batch_destroy(batch)


def sst_batch_submit(items, workspace, workspace_bytes, stream=None):
    arr = _items(items)
    _check(load().sst_batch_submit(arr, len(items), _ptr(workspace), int(workspace_bytes), _stream(stream)))


def sst_batch_workspace_for(items) -> int:
    arr = _items(items)
    b = ctypes.c_size_t()
    _check(load().sst_batch_workspace_for(arr, len(items), ctypes.byref(b)))
    return b.value


def sst_service_create(max_streams: int, mem_budget: int) -> int:
    out = _vp()
    _check(load().sst_service_create(int(max_streams), int(mem_budget), ctypes.byref(out)))
    return out.value


def sst_stream_open(svc, amp_bound: float, max_chunk: int, fs: float, L: int, hop: int, nfft: int,
                    f_lo: float, f_hi: float, z: int = 1, gamma: float = 0.0, sigma: float | None = None,
                    g=None, dg=None, xhat_only: bool = False) -> int:
    """Open a stream (absolute threshold gamma); returns its id.  xhat_only:
    SST_STREAM_XHAT_ONLY (TFR columns stay on the device)."""
    p, keep = _params(0, fs, L, hop, nfft, f_lo, f_hi, z, gamma, False, sigma, g, dg)
    if xhat_only:
        p.flags |= SST_STREAM_XHAT_ONLY
    sid = ctypes.c_int32()
    _check(load().sst_stream_open(svc, ctypes.byref(p), float(amp_bound), int(max_chunk), ctypes.byref(sid)))
    del keep
    return sid.value


def sst_stream_push(svc, sid: int, chunk, t_arrival: float = -1.0):
    import numpy as np
    a = np.ascontiguousarray(chunk, dtype=np.float32)
    _check(load().sst_stream_push(svc, int(sid), a.ctypes.data, len(a), float(t_arrival)))


def sst_stream_close(svc, sid: int):
    _check(load().sst_stream_close(svc, int(sid)))


def sst_service_tick(svc):
    _check(load().sst_service_tick(svc))


_poll_bufs = {}


def sst_stream_poll(svc, sid: int, bins: int, max_cols: int = 4096, max_samples: int = 1 << 17):
    """Returns (tfr [cols, bins] complex64, first_col, xhat float32, first_sample, finished).
    The host staging buffers are reused across calls (one pair per shape)."""
    import numpy as np
    key = (bins, max_cols, max_samples)
    if key not in _poll_bufs:
        _poll_bufs[key] = (np.empty((max_cols, bins, 2), dtype=np.float32), np.empty(max_samples, dtype=np.float32))
    t, x = _poll_bufs[key]
    cols, fc, ns, fs_, fin = _i64(), _i64(), _i64(), _i64(), ctypes.c_int32()
    _check(load().sst_stream_poll(svc, int(sid), t.ctypes.data, max_cols, ctypes.byref(cols), ctypes.byref(fc),
                                  x.ctypes.data, max_samples, ctypes.byref(ns), ctypes.byref(fs_),
                                  ctypes.byref(fin)))
    tc = t[:cols.value].view(np.complex64)[..., 0].copy()
    return tc, fc.value, x[:ns.value].copy(), fs_.value, bool(fin.value)


def sst_stream_release(svc, sid: int):
    _check(load().sst_stream_release(svc, int(sid)))


def sst_service_latency(svc, reset: bool = False):
    """Returns (p50 s, p99 s, chunks)."""
    a, b, c = ctypes.c_double(), ctypes.c_double(), _i64()
    _check(load().sst_service_latency(svc, ctypes.byref(a), ctypes.byref(b), ctypes.byref(c), 1 if reset else 0))
    return a.value, b.value, c.value


def sst_service_memory(svc):
    u, b = ctypes.c_size_t(), ctypes.c_size_t()
    _check(load().sst_service_memory(svc, ctypes.byref(u), ctypes.byref(b)))
    return u.value, b.value


def sst_service_destroy(svc):
    load().sst_service_destroy(svc)


def sst_sync(stream=None):
    _check(load().sst_sync(_stream(stream)))


def sst_launch_count() -> int:
    return int(load().sst_launch_count())


PROFILE_KINDS = 9


def sst_profile_enable(on: bool = True):
    _check(load().sst_profile_enable(1 if on else 0))


def sst_profile_collect() -> dict:
    """{kind name: (total ms, launches)} since the last collect."""
    ms = (ctypes.c_double * PROFILE_KINDS)()
    ct = (ctypes.c_uint64 * PROFILE_KINDS)()
    _check(load().sst_profile_collect(ms, ct))
    out = {}
    for i in range(PROFILE_KINDS):
        if ct[i]:
            out[load().sst_profile_kind_name(i).decode()] = (ms[i], int(ct[i]))
    return out


def sst_status_string(s: int) -> str:
    return load().sst_status_string(s).decode()


def sst_last_error() -> str:
    return load().sst_last_error().decode(errors="replace")


# ------------------------------------------------------------------ torch helper
def check_tensor(t, name: str, dtype, min_numel: int = 0, device=None):
    """The checks a raw pointer cannot carry through the C ABI: t is a torch
    tensor of element type dtype, contiguous, with at least min_numel
    elements, on `device` (a torch.device; None: in host memory).  Raises
    ValueError; returns t."""
    import torch
    if not isinstance(t, torch.Tensor):
        raise ValueError(f"{name}: expected a torch tensor, got {type(t).__name__}")
    if t.dtype != dtype:
        raise ValueError(f"{name}: expected {dtype}, got {t.dtype}")
    if device is None:
        if t.is_cuda:
            raise ValueError(f"{name}: expected a host tensor, got one on {t.device}")
    elif t.device != device:
        raise ValueError(f"{name}: expected a tensor on {device}, got one on {t.device}")
    if not t.is_contiguous():
        raise ValueError(f"{name}: must be contiguous")
    if t.numel() < min_numel:
        raise ValueError(f"{name}: has {t.numel()} elements, the call needs {min_numel}")
    return t


class Plan:
    """Owns a plan handle and the device buffers one signal needs (torch
    tensors on the current device): workspace, TFR and reconstruction.
    Tensor arguments are checked (element type, device, contiguity, size)
    before their pointers are passed on."""

    def __init__(self, **kw):
        import torch
        self.handle = sst_plan_create(**kw)
        q = sst_plan_query(self.handle)
        self.frames, self.bins = q["frames"], q["bins"]
        self.k_lo, self.k_hi = q["k_lo"], q["k_hi"]
        self.nb = self.k_hi - self.k_lo + 1
        self.n = int(kw["n"])
        dev = torch.device("cuda", torch.cuda.current_device())
        self.workspace = torch.empty(max(q["workspace_bytes"], 256), dtype=torch.uint8, device=dev)
        self.device = dev

    def new_tfr(self):
        import torch
        return torch.empty((self.frames, self.bins, 2), dtype=torch.float32, device=self.device)

    # argument checks (check_tensor) for the signal, a TFR and the outputs
    def _x(self, x, name="x"):
        import torch
        return check_tensor(x, name, torch.float32, self.n, self.device)

    def _tfr(self, tfr):
        import torch
        return check_tensor(tfr, "tfr", torch.float32, 2 * self.frames * self.bins, self.device)

    def _out(self, t, name, dtype, numel):
        return check_tensor(t, name, dtype, numel, self.device)

    def forward(self, x, tfr=None):
        tfr = self.new_tfr() if tfr is None else self._tfr(tfr)
        sst_forward(self.handle, self._x(x), self.n, tfr, self.workspace)
        return tfr

    def inverse(self, tfr, xhat=None):
        import torch
        xhat = torch.empty(self.n, dtype=torch.float32, device=self.device) if xhat is None else \
            self._out(xhat, "xhat", torch.float32, self.n)
        sst_inverse(self.handle, self._tfr(tfr), self.n, xhat, self.workspace)
        return xhat

    def inverse_zone(self, tfr, ridge, half_width, xhat=None):
        """Component recovery: the inverse restricted to |l - ridge[m]| <= half_width."""
        import torch
        xhat = torch.empty(self.n, dtype=torch.float32, device=self.device) if xhat is None else \
            self._out(xhat, "xhat", torch.float32, self.n)
        self._out(ridge, "ridge", torch.int32, self.frames)
        sst_inverse_zone(self.handle, self._tfr(tfr), self.n, ridge, half_width, xhat, self.workspace)
        return xhat

    def ridge(self, tfr, l_lo=0, l_hi=None, smooth=0, out=None):
        """Ridge (output bin per frame) of the component in [l_lo, l_hi]."""
        import torch
        l_hi = self.bins - 1 if l_hi is None else l_hi
        out = torch.empty(self.frames, dtype=torch.int32, device=self.device) if out is None else \
            self._out(out, "out", torch.int32, self.frames)
        sst_ridge(self._tfr(tfr), self.frames, self.bins, l_lo, l_hi, smooth, out)
        return out

    def renyi(self, tfr, alpha=3.0, cell=1.0, out=None):
        """Renyi entropy (Eq. 32) of |T|^2 as a one-element float64 device tensor."""
        import torch
        if getattr(self, "_renyi_ws", None) is None:
            self._renyi_ws = torch.empty(max(sst_renyi_workspace_bytes(), 256), dtype=torch.uint8,
                                         device=self.device)
        out = torch.empty(1, dtype=torch.float64, device=self.device) if out is None else \
            self._out(out, "out", torch.float64, 1)
        sst_renyi(self._tfr(tfr), self.frames, self.bins, self.bins, alpha, cell, out, self._renyi_ws)
        return out

    def forward_inverse(self, x, tfr=None, xhat=None):
        import torch
        tfr = self.new_tfr() if tfr is None else self._tfr(tfr)
        xhat = torch.empty(self.n, dtype=torch.float32, device=self.device) if xhat is None else \
            self._out(xhat, "xhat", torch.float32, self.n)
        sst_forward_inverse(self.handle, self._x(x), self.n, tfr, xhat, self.workspace)
        return tfr, xhat

    def reconstruct(self, x, xhat=None):
        """Forward + inverse without a TFR output (T stays on chip)."""
        import torch
        xhat = torch.empty(self.n, dtype=torch.float32, device=self.device) if xhat is None else \
            self._out(xhat, "xhat", torch.float32, self.n)
        sst_forward_inverse(self.handle, self._x(x), self.n, None, xhat, self.workspace)
        return xhat

    def stft(self, x):
        import torch
        V = torch.empty((self.frames, self.nb, 2), dtype=torch.float32, device=self.device)
        Vd = torch.empty_like(V)
        sst_stft(self.handle, self._x(x), self.n, V, Vd, self.workspace)
        return V, Vd

    def reassign_map(self, x):
        import torch
        om = torch.empty((self.frames, self.nb), dtype=torch.float32, device=self.device)
        de = torch.empty((self.frames, self.nb), dtype=torch.int32, device=self.device)
        sst_reassign_map(self.handle, self._x(x), self.n, om, de, self.workspace)
        return om, de

    def forward2(self, x, tfr=None):
        """Second-order forward (sst_forward2)."""
        tfr = self.new_tfr() if tfr is None else self._tfr(tfr)
        sst_forward2(self.handle, self._x(x), self.n, tfr, self.workspace)
        return tfr

    def reassign_map2(self, x):
        import torch
        om = torch.empty((self.frames, self.nb), dtype=torch.float32, device=self.device)
        de = torch.empty((self.frames, self.nb), dtype=torch.int32, device=self.device)
        sst_reassign_map2(self.handle, self._x(x), self.n, om, de, self.workspace)
        return om, de

    def max_abs_v(self, x):
        import torch
        out = torch.empty(1, dtype=torch.float32, device=self.device)
        sst_max_abs_v(self.handle, self._x(x), self.n, out, self.workspace)
        return out

    def close(self):
        for tc in getattr(self, "_tc", {}).values():
            sst_tc_plan_destroy(tc)
        self._tc = {}
        if self.handle:
            sst_plan_destroy(self.handle)
            self.handle = 0

    # tensor-core band form ("bf16", "bf16x3", "tf32"); the tensor plan is
    # created on first use and owned by this object
    def _tc_handle(self, form: str) -> int:
        if not hasattr(self, "_tc"):
            self._tc = {}
        if form not in self._tc:
            self._tc[form] = sst_tc_plan_create(self.handle, FORMS[form])
        return self._tc[form]

    def tc_forward(self, x, form: str, tfr=None):
        tfr = self.new_tfr() if tfr is None else self._tfr(tfr)
        sst_tc_forward(self._tc_handle(form), self._x(x), self.n, tfr)
        sst_tc_check(self._tc_handle(form))
        return tfr

    def tc_stft(self, x, form: str):
        import torch
        V = torch.empty((self.frames, self.nb, 2), dtype=torch.float32, device=self.device)
        Vd = torch.empty_like(V)
        sst_tc_stft(self._tc_handle(form), self._x(x), self.n, V, Vd)
        sst_tc_check(self._tc_handle(form))
        return V, Vd

    def tc_reassign_map(self, x, form: str):
        import torch
        om = torch.empty((self.frames, self.nb), dtype=torch.float32, device=self.device)
        de = torch.empty((self.frames, self.nb), dtype=torch.int32, device=self.device)
        sst_tc_reassign_map(self._tc_handle(form), self._x(x), self.n, om, de)
        sst_tc_check(self._tc_handle(form))
        return om, de

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

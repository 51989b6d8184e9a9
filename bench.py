"""Throughput benchmark of the fused SST forward + direct inverse.

One step = sst_forward_inverse over the whole run-up vibration workload
(N = 2^24 float32 samples at 51.2 kHz, Gaussian window L = 2049, hop 32,
Nf 4096, band 0-6.4 kHz, subdivision z = 4, gamma = 1e-3 max|V|): threshold
pre-pass, forward (T written to HBM, 8.6 GB), inverse and overlap-add.  The
same step without a TFR output (T kept on chip by the fused kernel) is timed
beside it and reported under "variants".
Metric: input samples/s.  With --gpus N > 1 (torchrun), every rank runs its
own replica of the workload on its own GPU (weak scaling, no collective on
the data path).

``--impl reference`` times the FP64 CPU oracle instead, on a bounded sample
of the same workload, and prints the same JSON line with "impl": "reference".
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_2003_07065_gb300 import workloads as W  # noqa: E402

METRIC = "input samples/s through SST fwd+inverse"
UNIT = "samples/s"
L2_BYTES = 129 * 1024 * 1024
FALLBACK_BF16_TFLOPS = 1900.0      # used only when MEASURED_PEAKS.json is absent
TF32_OVER_BF16 = 1.1 / 2.25        # nominal dense TF32 / BF16 tensor rate


def flops_per_frame(w) -> dict:
    """Algorithmic FLOPs per frame of each kernel (conventional 5 N log2 N per
    complex FFT, 2.5 N log2 N per real-output one):
      absmax : half a packed FFT per frame + window + |V|^2 on the band
      forward: packed complex FFT + window (x g, x g') + ~20 per band bin
      inverse: z real-output IFFTs + 8 z L for the sub-grid twiddles and
               the window / overlap-add."""
    nf, L, z = w.nfft, w.L, w.z
    k_lo = int(math.floor(w.f_lo * nf / w.fs + 0.5))
    k_hi = min(nf // 2, int(math.floor(w.f_hi * nf / w.fs + 0.5)))
    nb = k_hi - k_lo + 1
    lg = math.log2(nf)
    return {
        "absmax": 2.5 * nf * lg + 2 * L + 4 * nb,
        "forward": 5 * nf * lg + 4 * L + 20 * nb,
        "inverse": 2.5 * z * nf * lg + 8 * z * L,
    }


def bytes_per_frame(w) -> dict:
    """Algorithmic DRAM bytes per frame: x read once (hop new samples per
    frame), T written by the forward and read by the inverse, xhat written."""
    nf = w.nfft
    k_lo = int(math.floor(w.f_lo * nf / w.fs + 0.5))
    k_hi = min(nf // 2, int(math.floor(w.f_hi * nf / w.fs + 0.5)))
    nbo = w.z * (k_hi - k_lo) + 1
    return {"absmax": 4 * w.hop, "forward": 4 * w.hop + 8 * nbo, "inverse": 8 * nbo + 4 * w.hop}


class ClockSampler:
    """nvidia-smi clock / throttle sampling during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except (OSError, FileNotFoundError):
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.thread.join(timeout=5)
        sm, smax, reasons, power = [], [], set(), []
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
                power.append(float(parts[3]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm),
                "power_w_max": max(power) if power else None}


def measured_peaks() -> dict:
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            return json.load(f)
    return {}


def measured_traffic_per_frame(kernel: str):
    """(DRAM bytes per frame of `kernel` from the committed ncu capture
    (profiles/dram_traffic_runup.json), a note on where it comes from).  The
    bytes are None when there is no capture or the kernel sources have
    changed since it was taken; the note then says so and gives the
    capture's figure for reference."""
    import hashlib
    p = os.path.join(ROOT, "profiles", "dram_traffic_runup.json")
    if not os.path.exists(p):
        return None, "no ncu capture of the DRAM traffic is committed"
    with open(p) as f:
        rec = json.load(f)
    # the files that define the FFT-path kernels (device code, launch shapes)
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_2003_07065_gb300", "csrc")
    for name in rec.get("kernel_sources", []):
        with open(os.path.join(csrc, name), "rb") as f:
            h.update(f.read())
    bpf = rec["dram_bytes_per_frame"].get(kernel)
    if h.hexdigest() != rec.get("kernel_source_sha256"):
        return None, (f"null: the kernel sources changed after the committed ncu capture "
                      f"(profiles/dram_traffic_runup.json, {bpf:.0f} B per frame then)" if bpf is not None else
                      "null: the kernel sources changed after the committed ncu capture")
    return bpf, "ncu dram__bytes_read+write of one runup_4m launch scaled by frames"


def fp32_peak_tflops(num_sms: int, mhz: float) -> float:
    """FP32 ALU peak: 128 FP32 lanes per SM, one FMA (2 FLOPs) per lane per
    clock."""
    return num_sms * 128 * 2 * mhz * 1e6 / 1e12


# ------------------------------------------------------------------ reference arm
def plan_supports_fused(sst, plan, x, n, xhat, stream) -> bool:
    """Whether the plan runs forward + inverse without a TFR output (its
    fused kernel fits in shared memory)."""
    try:
        sst.sst_forward_inverse(plan.handle, x, n, None, xhat, plan.workspace, stream)
        return True
    except sst.SstError as e:
        if e.status == 6:
            return False
        raise


def max_over_ranks(x: float, dist=None, device="cuda") -> float:
    """The largest x over the ranks of the process group (x itself without
    one): the job's time is its slowest replica's."""
    if dist is None:
        return float(x)
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_rate(world: int, units_per_rank: float, steps: int, seconds: float) -> float:
    """Whole-job throughput: every rank processes units_per_rank per step, the
    job takes the slowest rank's time (weak scaling)."""
    return world * units_per_rank * steps / seconds


def cpu_model() -> str:
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                k, _, v = line.partition(":")
                if k.strip().lower() in ("model name", "cpu model", "hardware"):
                    return v.strip()
        out = subprocess.run(["lscpu"], capture_output=True, text=True).stdout
        for line in out.splitlines():
            if line.lower().startswith("model name"):
                return line.split(":", 1)[1].strip()
    except Exception:
        pass
    return "unknown"


def oracle_sample_rate(w, budget_s: float = 15.0, n_max: int = 1 << 15):
    """Run the FP64 oracle on a bounded prefix of the workload's signal (the
    whole path: STFTs, IF, reassignment, inverse) and return samples/s."""
    import oracle as O
    noisy, _ = w.signal()
    n_sample = min(w.n, n_max)
    x = noisy[:n_sample].astype(np.float32).astype(np.float64)
    t0 = time.perf_counter()
    reps = 0
    while True:
        O.sst(x, w.fs, w.L, w.sigma, w.hop, w.nfft, w.f_lo, w.f_hi, w.z, w.gamma, w.relative,
              inverse_range=(0, len(x)))
        reps += 1
        el = time.perf_counter() - t0
        if el >= budget_s or reps >= 64:
            break
    threads = O.get_threads()
    return reps * n_sample / el, threads, f"{reps} x first {n_sample} samples of {w.name}", el


def run_reference(args, w):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    import oracle as O
    O.build()
    O.set_threads(0)
    vals = []
    for _ in range(args.warmup):
        oracle_sample_rate(w, budget_s=0.0)
    for _ in range(args.steps):
        v, threads, sample, _ = oracle_sample_rate(w, budget_s=max(1.0, 30.0 / max(args.steps, 1)))
        vals.append(v)
    value = statistics.mean(vals)
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": w.name, "n": w.n, "nfft": w.nfft, "hop": w.hop, "L": w.L, "z": w.z,
                   "band_hz": [w.f_lo, w.f_hi]},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": threads, "kind": "oracle", "sample": sample,
                         "cpu_model": cpu_model()},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))
    return 0


# ------------------------------------------------------------------ batched workload
def params_flops(p: dict) -> dict:
    """flops_per_frame for a plan's parameter dict."""
    import types
    return flops_per_frame(types.SimpleNamespace(**p))


def batch_leg(args) -> dict:
    """256 mixed channels in one captured CUDA graph (per-NF persistent
    launches over a work-item table), autotuned; tuned vs untuned time, the
    timed rate and the FP32 roofline fraction of the batch's algorithmic
    FLOPs (pre-pass, forward, inverse of every channel)."""
    import torch
    from paper_2003_07065_gb300 import build, sst
    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    build.build()
    sst.load()
    chans = W.batch_channels(256)
    plans, items, keep = [], [], []
    tfr_bytes = 0
    flops = 0.0
    for params, x in chans:
        pl = sst.Plan(**params)
        xd = torch.from_numpy(x).cuda()
        t = pl.new_tfr()
        xh = torch.empty(pl.n, dtype=torch.float32, device="cuda")
        tfr_bytes += t.numel() * 4
        fl = params_flops(params)
        flops += pl.frames * (fl["forward"] + fl["inverse"] + (fl["absmax"] / 2 if params["relative"] else 0.0))
        plans.append(pl)
        keep.append((xd, t, xh))
        items.append((pl.handle, xd, pl.n, t, xh))
    total = sum(p["n"] for p, _ in chans)
    b = sst.sst_batch_create(items, graph=True)
    ws = torch.empty(max(sst.sst_batch_workspace(b), 256), dtype=torch.uint8, device="cuda")
    untuned_ms, tuned_ms = sst.sst_batch_tune(b, ws)
    knobs = sst.sst_batch_knobs(b)
    flush = torch.empty(2 * L2_BYTES // 4, dtype=torch.float32, device="cuda")
    stream = torch.cuda.current_stream()
    for _ in range(max(args.warmup, 3)):
        sst.sst_batch_run(b, ws, stream)
    torch.cuda.synchronize()
    sampler = ClockSampler(0)
    sampler.start()
    time.sleep(0.3)
    l0 = sst.sst_launch_count()
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    torch.cuda.synchronize()
    for i in range(args.steps):
        flush.fill_(float(i))
        evs[i][0].record(stream)
        sst.sst_batch_run(b, ws, stream)
        evs[i][1].record(stream)
    torch.cuda.synchronize()
    launches = sst.sst_launch_count() - l0
    clocks = sampler.stop()
    t_ms = sum(a.elapsed_time(c) for a, c in evs)
    peak = sst.sst_fp32_peak(stream)
    step_s = t_ms / args.steps / 1e3
    out = {
        "value": total * args.steps / (t_ms / 1e3), "unit": UNIT, "steps": args.steps,
        "ms_per_step": t_ms / args.steps, "total_samples": total, "tfr_bytes": tfr_bytes,
        "autotune": {"untuned_ms": untuned_ms, "tuned_ms": tuned_ms, "knobs": knobs},
        "roofline": {"bound": "alu", "achieved": flops / step_s / 1e12, "peak": peak, "unit": "TFLOP/s",
                     "frac": flops / step_s / 1e12 / peak, "algorithmic_flops": flops,
                     "note": "pre-pass (half a packed FFT per frame), forward and inverse of every channel, "
                             "conventional 5 N log2 N per complex FFT; peak as sst_fp32_peak"},
        "gpu_launches": launches, "clocks": clocks,
    }
    sst.sst_batch_destroy(b)
    for pl in plans:
        pl.close()
    del keep, flush, ws
    torch.cuda.empty_cache()
    return out


def run_batch(args):
    leg = batch_leg(args)
    line = {
        "metric": METRIC, "value": leg["value"], "unit": UNIT, "n_gpus": 1,
        "steps": args.steps, "warmup": max(args.warmup, 3), "ms_per_step": leg["ms_per_step"],
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": "batch256", "channels": 256, "total_samples": leg["total_samples"],
                   "tfr_bytes": leg["tfr_bytes"], "lengths": "log-uniform [2^14, 2^22]",
                   "nfft": "512..8192", "hop": "8..64", "z": "1,2,4", "graph": True,
                   "l2": "flushed before each timed step"},
        "autotune": leg["autotune"], "roofline": leg["roofline"],
        "gpu_launches": leg["gpu_launches"], "clocks": leg["clocks"],
    }
    print(json.dumps(line))
    return 0


# ------------------------------------------------------------------ tensor-core band form
TC_FORMS = ("fft", "bf16", "bf16x3", "tf32")


def tensor_forms(args, w, params, x, clean, stream, flush, bf16_peak):
    """Per form: fwd+inv step time (L2 flushed before each step), SNR of the
    reconstruction against the clean signal, per-kernel times and, for the
    tensor forms, the contraction's tensor-pipe fraction."""
    import torch
    from paper_2003_07065_gb300 import sst
    plan = sst.Plan(**params)
    tfr = plan.new_tfr()
    xhat = torch.empty(w.n, dtype=torch.float32, device="cuda")
    forms = {}
    for form in TC_FORMS:
        info = {}
        if form == "fft":
            def fwd():
                sst.sst_forward(plan.handle, x, w.n, tfr, plan.workspace, stream)
        else:
            h = plan._tc_handle(form)
            cl, _ = sst.sst_tc_plan_tune(h, x, w.n, stream)
            q = sst.sst_tc_plan_query(h)
            info.update(cluster=cl, hankel_view=q["hankel_view"], gemm_flops=q["gemm_flops"])

            def fwd(h=h):
                sst.sst_tc_forward(h, x, w.n, tfr, stream)

        def step():
            fwd()
            sst.sst_inverse(plan.handle, tfr, w.n, xhat, plan.workspace, stream)

        for _ in range(max(args.warmup, 3)):
            step()
        torch.cuda.synchronize()
        sst.sst_profile_enable(True)
        sst.sst_profile_collect()
        evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
               for _ in range(args.steps)]
        for i in range(args.steps):
            flush.fill_(float(i))
            evs[i][0].record(stream)
            step()
            evs[i][1].record(stream)
        torch.cuda.synchronize()
        sst.sst_profile_enable(False)
        prof = sst.sst_profile_collect()
        if form != "fft":
            sst.sst_tc_check(plan._tc_handle(form))
        t_ms = sum(a.elapsed_time(b) for a, b in evs) / args.steps
        xh = xhat.cpu().numpy().astype(np.float64)
        err = clean - xh
        info.update(ms_per_step=t_ms, samples_per_s=w.n / (t_ms / 1e3),
                    snr_db=float(10 * np.log10(np.sum(clean ** 2) / np.sum(err ** 2))),
                    kernels={k: {"ms_per_step": v[0] / args.steps, "launches_per_step": v[1] / args.steps}
                             for k, v in prof.items()})
        if form != "fft":
            gemm_ms = prof["stft"][0] / args.steps      # the contraction is timed under this kind
            peak = bf16_peak * (TF32_OVER_BF16 if form == "tf32" else 1.0)
            info["contraction"] = {"ms": gemm_ms, "tflops": info["gemm_flops"] / gemm_ms / 1e9,
                                   "peak_tflops": peak, "frac": info["gemm_flops"] / gemm_ms / 1e9 / peak}
        forms[form] = info
    bins = plan.nb
    plan.close()
    return forms, bins


def tensor_leg(args) -> dict:
    """Precision workload (Nf 4096, L 2049, hop 16; the 0-6.4 kHz band at
    25.6 kHz = 1025 bins): one step = forward (the FFT form, or the tcgen05
    contraction in one of its three operand forms) + the shared direct inverse.
    Every form's time and reconstruction SNR (against the clean signal); the
    same on the literal 512-bin shape (k = 0..511).  Single GPU only: it loads
    the tensor-form library."""
    import dataclasses
    import torch
    from paper_2003_07065_gb300 import build, sst
    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    build.build_tc()
    sst.load_tc()
    w = W.PRECISION_64K
    noisy, clean = w.signal()
    x = torch.from_numpy(noisy.astype(np.float32)).cuda()
    flush = torch.empty(2 * L2_BYTES // 4, dtype=torch.float32, device="cuda")
    stream = torch.cuda.current_stream()
    bf16_peak = measured_peaks().get("bf16_tflops") or FALLBACK_BF16_TFLOPS
    sampler = ClockSampler(0)
    sampler.start()
    time.sleep(0.3)
    l0 = sst.sst_launch_count()
    forms, bins = tensor_forms(args, w, w.params(), x, clean, stream, flush, bf16_peak)
    w512 = dataclasses.replace(w, f_hi=511 * w.fs / w.nfft)
    forms512, bins512 = tensor_forms(args, w512, w512.params(), x, clean, stream, flush, bf16_peak)
    launches = sst.sst_launch_count() - l0
    clocks = sampler.stop()
    head = forms["bf16"]
    best = max((f for f in forms if f != "fft" and abs(forms[f]["snr_db"] - forms["fft"]["snr_db"]) <= 0.1),
               key=lambda f: forms[f]["samples_per_s"], default="bf16")
    del flush
    return {
        "w": w, "bins": bins, "head": head, "forms": forms, "forms512": forms512, "bins512": bins512, "w512": w512,
        "vs_fft_form": head["samples_per_s"] / forms["fft"]["samples_per_s"],
        "snr_gap_db": head["snr_db"] - forms["fft"]["snr_db"],
        "best_form_at_equal_snr": {"form": best, "vs_fft_form": forms[best]["samples_per_s"] /
                                   forms["fft"]["samples_per_s"],
                                   "snr_gap_db": forms[best]["snr_db"] - forms["fft"]["snr_db"]},
        "bf16_peak": bf16_peak, "gpu_launches": launches, "clocks": clocks,
    }


def run_tensor(args):
    """The tensor-form leg as its own JSON line; the headline is the BF16
    tensor form, its roofline the contraction's against the measured dense
    BF16 tensor peak (TF32 at the nominal TF32 / BF16 ratio)."""
    leg = tensor_leg(args)
    w, head, forms = leg["w"], leg["head"], leg["forms"]
    line = {
        "metric": METRIC, "value": head["samples_per_s"], "unit": UNIT, "n_gpus": 1, "steps": args.steps,
        "warmup": max(args.warmup, 3), "ms_per_step": head["ms_per_step"], "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "bf16", "data": "synthetic",
        "config": {"workload": w.name, "n": w.n, "fs": w.fs, "nfft": w.nfft, "hop": w.hop, "L": w.L,
                   "sigma": w.sigma, "z": w.z, "band_hz": [w.f_lo, w.f_hi], "bins": leg["bins"],
                   "form": "bf16 tcgen05 contraction + FP32 inverse", "l2": "flushed before each timed step"},
        "vs_fft_form": leg["vs_fft_form"],
        "snr_gap_db": leg["snr_gap_db"],
        "best_form_at_equal_snr": leg["best_form_at_equal_snr"],
        "roofline": {"bound": "tensor", "kernel": "k_tc_gemm", "achieved": head["contraction"]["tflops"],
                     "peak": leg["bf16_peak"], "unit": "TFLOP/s", "frac": head["contraction"]["frac"],
                     "traffic": None,
                     "peak_note": ("of measured: dense BF16 burst (MEASURED_PEAKS.json)" if measured_peaks().get(
                         "bf16_tflops") else f"of fallback: {FALLBACK_BF16_TFLOPS} TFLOP/s dense BF16 (no "
                         "MEASURED_PEAKS.json on this machine)")},
        "forms": forms,
        "literal_512_bins": {"band_hz": [leg["w512"].f_lo, leg["w512"].f_hi], "bins": leg["bins512"],
                             "forms": leg["forms512"]},
        "gpu_launches": leg["gpu_launches"], "clocks": leg["clocks"],
    }
    print(json.dumps(line))
    return 0


# ------------------------------------------------------------------ streaming workload
def stream_leg(args, dur: float, overload_s: float = 3.0) -> dict:
    """64 sensor streams at 25.6 kHz pushing 8192-sample chunks with Poisson
    arrivals (2 chunks/s per stream; bursts of 1 s at 5x the rate starting as
    a 0.1/s Poisson process), served in real time for `dur` seconds: p50/p99
    latency (tick completion minus scheduled arrival).  Then an overload phase
    (every stream's queue kept full) gives the sustained samples/s."""
    import torch
    from paper_2003_07065_gb300 import build, sst, signals
    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    build.build()
    sst.load()
    nstreams, fs, chunk = 64, 25600.0, 8192
    P = dict(fs=fs, L=1025, sigma=128.0, hop=16, nfft=2048, f_lo=0.0, f_hi=8000.0, z=2)
    # arrival schedules
    sched = []
    for i in range(nstreams):
        gen = signals.rng(5, i)
        bursts = []
        t = 0.0
        while t < dur:
            t += gen.exponential(1 / 0.1)
            bursts.append((t, t + 1.0))
        arr, t = [], 0.0
        while t < dur:
            rate = 2.0 * (5.0 if any(a <= t < b for a, b in bursts) else 1.0)
            t += gen.exponential(1 / rate)
            if t < dur:
                arr.append(t)
        sched.append(arr)
    need = max(len(a) for a in sched) * chunk + 64 * chunk
    sigs, gammas = [], []
    for i in range(nstreams):
        x, _ = signals.chirp_fm_mix(need, fs, 10.0, seed=(5, 1000 + i))
        sigs.append(x.astype(np.float32))
    # per-stream absolute threshold: 1e-3 of the stream's whole-signal max |V| (product path)
    for i in range(nstreams):
        pl = sst.Plan(n=len(sigs[i]), gamma=1e-3, relative=True, **P)
        gammas.append(1e-3 * float(pl.max_abs_v(torch.from_numpy(sigs[i]).cuda()).item()))
        pl.close()
    nb = P["z"] * int(math.floor(P["f_hi"] * P["nfft"] / fs + 0.5)) + 1
    svc = sst.sst_service_create(nstreams, 64 << 30)
    ids = [sst.sst_stream_open(svc, 8.0, chunk, gamma=gammas[i], **P) for i in range(nstreams)]
    l0 = sst.sst_launch_count()
    # real-time phase
    events = sorted((t, i) for i, a in enumerate(sched) for t in a)
    pos = [0] * nstreams
    t0 = time.monotonic()
    k = 0
    pushed = dropped = ticks = 0
    while True:
        now = time.monotonic() - t0
        if now >= dur and k >= len(events):
            break
        while k < len(events) and events[k][0] <= now:
            ta, i = events[k]
            try:
                sst.sst_stream_push(svc, ids[i], sigs[i][pos[i]:pos[i] + chunk], t0 + ta)
                pos[i] += chunk
                pushed += chunk
            except sst.SstError:
                dropped += 1
            k += 1
        sst.sst_service_tick(svc)
        ticks += 1
        for i in range(nstreams):
            while True:
                t, _, x, _, _ = sst.sst_stream_poll(svc, ids[i], nb)
                if not len(t) and not len(x):
                    break
        if k < len(events):
            wait = events[k][0] - (time.monotonic() - t0)
            if wait > 0:
                time.sleep(min(wait, 0.002))
    wall = time.monotonic() - t0
    p50, p99, nlat = sst.sst_service_latency(svc, reset=True)
    # overload phase: keep every queue full for overload_s seconds
    def overload(svc, ids, pos, seconds=overload_s):
        t1 = time.monotonic()
        processed = 0
        while time.monotonic() - t1 < seconds:
            for i in range(nstreams):
                for _ in range(4):
                    if pos[i] + chunk > len(sigs[i]):
                        pos[i] = 0
                    try:
                        sst.sst_stream_push(svc, ids[i], sigs[i][pos[i]:pos[i] + chunk])
                        pos[i] += chunk
                        processed += chunk
                    except sst.SstError:
                        break
            sst.sst_service_tick(svc)
            for i in range(nstreams):
                while True:
                    t, _, x, _, _ = sst.sst_stream_poll(svc, ids[i], nb)
                    if not len(t) and not len(x):
                        break
        return processed / (time.monotonic() - t1)

    sustained = overload(svc, ids, pos)
    o50, o99, _ = sst.sst_service_latency(svc, reset=True)
    # the same with reconstruction-only streams (TFR columns stay on the device)
    svc2 = sst.sst_service_create(nstreams, 64 << 30)
    ids2 = [sst.sst_stream_open(svc2, 8.0, chunk, gamma=gammas[i], xhat_only=True, **P) for i in range(nstreams)]
    sustained_x = overload(svc2, ids2, [0] * nstreams)
    x50, x99, _ = sst.sst_service_latency(svc2, reset=True)
    sst.sst_service_destroy(svc2)
    launches = sst.sst_launch_count() - l0
    sst.sst_service_destroy(svc)
    return {
        "value": sustained, "unit": "samples/s", "ticks": ticks, "seconds": dur,
        "config": {"workload": "stream64", "streams": nstreams, "chunk": chunk, "fs": fs, "hop": 16, "nfft": 2048,
                   "L": 1025, "band_hz": [0.0, 8000.0], "z": 2, "arrivals": "Poisson 2/s, 1 s bursts x5 at 0.1/s",
                   "seconds": dur},
        "latency_s": {"p50": p50, "p99": p99, "chunks": nlat, "offered_samples_per_s": pushed / wall,
                      "dropped_chunks": dropped, "ticks": ticks},
        "overload_latency_s": {"p50": o50, "p99": o99},
        "sustained_note": ("value: every TFR column (1281 complex bins per 16 samples = 640 B per input sample) "
                           "and x-hat delivered to the host"),
        "sustained_xhat_only": {"value": sustained_x, "unit": "samples/s", "p50": x50, "p99": x99},
        "gpu_launches": launches,
    }


def run_stream(args):
    leg = stream_leg(args, args.seconds)
    line = {
        "metric": "p50/p99 stream latency; sustained input samples/s", "value": leg["value"], "unit": "samples/s",
        "n_gpus": 1, "steps": leg["ticks"], "warmup": 0, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic", "config": leg["config"],
        "latency_s": leg["latency_s"], "overload_latency_s": leg["overload_latency_s"],
        "sustained_note": leg["sustained_note"], "sustained_xhat_only": leg["sustained_xhat_only"],
        "gpu_launches": leg["gpu_launches"],
    }
    print(json.dumps(line))
    return 0


# ------------------------------------------------------------------ GPU arm
# ------------------------------------------------------------------ steps after the transform
POST_METRIC = "input samples/s through ridge + zone inverse + Renyi entropy"
POST_SMOOTH, POST_HW, POST_ALPHA = 2, 16, 3.0


def oracle_post_rate(w, budget_s: float = 10.0, n_sample: int = 1 << 15):
    """The oracle's ridge, zone inverse and entropy on the T of a bounded
    prefix of the workload (the transform itself untimed); samples/s."""
    import oracle as O
    noisy, _ = w.signal()
    x = noisy[:n_sample].astype(np.float32).astype(np.float64)
    r = O.sst(x, w.fs, w.L, w.sigma, w.hop, w.nfft, w.f_lo, w.f_hi, w.z, w.gamma, w.relative)
    g, _ = O.window(w.L, w.sigma)
    t0 = time.perf_counter()
    reps = 0
    while True:
        rid = O.ridge(r.T, 0, r.T.shape[1] - 1, POST_SMOOTH)
        O.zone_inverse(r.T, rid, POST_HW, r.k_lo, w.nfft, w.z, g, w.hop, len(x))
        O.renyi(r.T, POST_ALPHA)
        reps += 1
        el = time.perf_counter() - t0
        if el >= budget_s or reps >= 64:
            break
    return reps * n_sample / el, O.get_threads(), f"{reps} x first {n_sample} samples of {w.name}", el


def run_post(args):
    """One step = the steps after the transform on the run-up workload's T
    (runup_16m_post; runup_4m_post is the profiling-sized case)
    produced once, untimed: sst_ridge over the whole band (smoothing over
    +-2 frames), sst_inverse_zone around that ridge (+-16 output bins) and
    sst_renyi (alpha = 3) of T.  The zone inverse is the dominant kernel (FP32
    ALU roofline); the ridge and the entropy stream T (HBM roofline each)."""
    import torch
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    w = W.ALL[args.workload[:-len("_post")]]
    if args.impl == "reference":
        if rank != 0:
            return 0
        import oracle as O
        O.build()
        O.set_threads(0)
        vals = []
        for _ in range(args.warmup):
            oracle_post_rate(w, budget_s=0.0, n_sample=1 << 13)
        for _ in range(args.steps):
            v, threads, sample, _ = oracle_post_rate(w, budget_s=max(1.0, 30.0 / max(args.steps, 1)))
            vals.append(v)
        value = statistics.mean(vals)
        print(json.dumps({
            "impl": "reference", "metric": POST_METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": args.workload, "smooth": POST_SMOOTH, "half_width": POST_HW,
                       "alpha": POST_ALPHA},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": threads, "kind": "oracle", "sample": sample,
                             "cpu_model": cpu_model()},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}))
        return 0
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    from paper_2003_07065_gb300 import build, sst
    if rank == 0:
        build.build()
    if dist is not None:
        dist.barrier()
    build.build()
    sst.load()
    noisy, _ = w.signal()
    x_host = torch.from_numpy(noisy.astype(np.float32)).pin_memory()
    x = x_host.cuda()
    plan = sst.Plan(**w.params())
    tfr = plan.forward(x)
    F, bins = plan.frames, plan.bins
    ridge = torch.empty(F, dtype=torch.int32, device="cuda")
    xq = torch.empty(w.n, dtype=torch.float32, device="cuda")
    ent = torch.empty(1, dtype=torch.float64, device="cuda")
    rws = torch.empty(max(sst.sst_renyi_workspace_bytes(), 256), dtype=torch.uint8, device="cuda")
    flush = torch.empty(2 * L2_BYTES // 4, dtype=torch.float32, device="cuda")
    stream = torch.cuda.current_stream()

    def do_ridge():
        sst.sst_ridge(tfr, F, bins, 0, bins - 1, POST_SMOOTH, ridge, stream)

    def do_zone():
        sst.sst_inverse_zone(plan.handle, tfr, w.n, ridge, POST_HW, xq, plan.workspace, stream)

    def do_renyi():
        sst.sst_renyi(tfr, F, bins, bins, POST_ALPHA, 1.0, ent, rws, stream)

    def step():
        do_ridge()
        do_zone()
        do_renyi()

    for _ in range(max(args.warmup, 3)):
        step()
    torch.cuda.synchronize()

    def timed(fn, k):
        evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(k)]
        for i in range(k):
            flush.fill_(float(i))
            evs[i][0].record(stream)
            fn()
            evs[i][1].record(stream)
        torch.cuda.synchronize()
        return [a.elapsed_time(b) for a, b in evs]

    sampler = ClockSampler(local)
    sampler.start()
    time.sleep(0.3)
    launches0 = sst.sst_launch_count()
    if dist is not None:
        dist.barrier()
    torch.cuda.synchronize()
    step_ms = timed(step, args.steps)
    if dist is not None:
        dist.barrier()
    launches = sst.sst_launch_count() - launches0
    clocks = sampler.stop()
    t_ms = max_over_ranks(sum(step_ms), dist)
    value = job_rate(world, w.n, args.steps, t_ms / 1e3)
    # each kernel alone, for its roofline
    ridge_ms = statistics.mean(timed(do_ridge, args.steps))
    zone_ms = statistics.mean(timed(do_zone, args.steps))
    renyi_ms = statistics.mean(timed(do_renyi, args.steps))

    # end to end through the C ABI with host buffers: x in, forward, the three
    # steps, and the component, the ridge and the entropy out
    xq_host = torch.empty(w.n, dtype=torch.float32).pin_memory()
    ridge_host = torch.empty(F, dtype=torch.int32).pin_memory()
    ent_host = torch.empty(1, dtype=torch.float64).pin_memory()

    def e2e_step():
        x.copy_(x_host, non_blocking=True)
        sst.sst_forward(plan.handle, x, w.n, tfr, plan.workspace, stream)
        step()
        xq_host.copy_(xq, non_blocking=True)
        ridge_host.copy_(ridge, non_blocking=True)
        ent_host.copy_(ent, non_blocking=True)
        torch.cuda.synchronize()

    for _ in range(2):
        e2e_step()
    e0 = time.perf_counter()
    for _ in range(args.steps):
        e2e_step()
    e_s = max_over_ranks(time.perf_counter() - e0, dist)
    e2e = job_rate(world, w.n, args.steps, e_s)
    if rank != 0:
        if dist is not None:
            dist.destroy_process_group()
        return 0

    peaks = measured_peaks()
    hbm = peaks.get("hbm_gbs")
    peak = sst.sst_fp32_peak(stream)
    fl = flops_per_frame(w)
    t_bytes = F * bins * 8
    zone_flops = fl["inverse"] * F
    ridge_bytes = t_bytes + F * 4            # T once (algorithmic) + the ridge written
    renyi_bytes = 2 * t_bytes                # two passes: the exact maximum, then the sums
    roof = {"bound": "alu", "kernel": "inverse_zone", "achieved": zone_flops / (zone_ms / 1e3) / 1e12,
            "peak": peak, "unit": "TFLOP/s", "frac": zone_flops / (zone_ms / 1e3) / 1e12 / peak, "traffic": None,
            "peak_note": "FP32 FMA throughput measured in this run (sst_fp32_peak)",
            "algorithmic_flops_per_launch": zone_flops, "avg_launch_ms": zone_ms,
            "others": {
                "ridge": {"bound": "hbm", "avg_launch_ms": ridge_ms, "algorithmic_bytes": ridge_bytes,
                          "achieved_gbs": ridge_bytes / (ridge_ms / 1e3) / 1e9, "peak_gbs": hbm,
                          "frac": ridge_bytes / (ridge_ms / 1e3) / 1e9 / hbm if hbm else None},
                "renyi": {"bound": "hbm", "avg_launch_ms": renyi_ms, "algorithmic_bytes": renyi_bytes,
                          "achieved_gbs": renyi_bytes / (renyi_ms / 1e3) / 1e9, "peak_gbs": hbm,
                          "frac": renyi_bytes / (renyi_ms / 1e3) / 1e9 / hbm if hbm else None}}}
    cpu = None
    if world == 1 and not args.no_cpu_baseline:
        import oracle as O
        O.build()
        O.set_threads(0)
        v, threads, sample, el = oracle_post_rate(w, budget_s=10.0)
        cpu = {"value": v, "unit": UNIT, "cores": threads, "kind": "oracle", "sample": sample, "seconds": el,
               "cpu_model": cpu_model()}
    line = {
        "metric": POST_METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": max(args.warmup, 3), "ms_per_step": t_ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": args.workload, "n": w.n, "frames": F, "bins": bins, "smooth": POST_SMOOTH,
                   "half_width": POST_HW, "alpha": POST_ALPHA, "tfr_bytes": t_bytes,
                   "l2": f"flushed before each timed step (2x L2 write); T ({t_bytes / 1e9:.1f} GB) also exceeds L2",
                   "parallelism": f"replicas x{world}"},
        "gpu_launches": launches, "gpu_launches_per_step": launches / args.steps,
        "kernels": {"ridge": {"ms": ridge_ms}, "inverse_zone": {"ms": zone_ms}, "renyi": {"ms": renyi_ms}},
        "entropy_bits": float(ent.item()),
        "roofline": roof, "cpu_baseline": cpu,
        "e2e": {"value": e2e, "unit": UNIT, "h2d_bytes_per_step": 4 * w.n,
                "d2h_bytes_per_step": 4 * w.n + 4 * F + 8,
                "note": "x in, forward, ridge, zone inverse, entropy, component + ridge + entropy out"},
        "clocks": clocks,
    }
    print(json.dumps(line))
    plan.close()
    if dist is not None:
        dist.destroy_process_group()
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="runup_16m",
                    choices=sorted(W.ALL) + ["batch256", "stream64", "precision64k_tc", "runup_16m_post",
                                             "runup_4m_post"])
    ap.add_argument("--seconds", type=float, default=12.0, help="stream64: simulated real-time seconds")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-legs", action="store_true", help="skip the tensor-form, stream and batch legs")
    args = ap.parse_args()
    if args.workload == "batch256":
        return run_batch(args)
    if args.workload == "stream64":
        return run_stream(args)
    if args.workload == "precision64k_tc":
        return run_tensor(args)
    if args.workload.endswith("_post"):
        return run_post(args)
    w = W.ALL[args.workload]
    if args.impl == "reference":
        return run_reference(args, w)

    import torch
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    def barrier():
        if dist is not None:
            dist.barrier()

    from paper_2003_07065_gb300 import build, sst
    if rank == 0:
        build.build()
    barrier()
    build.build()
    sst.load()

    noisy, _ = w.signal()
    x_host = torch.from_numpy(noisy.astype(np.float32)).pin_memory()
    x = x_host.cuda()
    plan = sst.Plan(**w.params())
    tfr = plan.new_tfr()
    xhat = torch.empty(w.n, dtype=torch.float32, device="cuda")
    xhat_host = torch.empty(w.n, dtype=torch.float32).pin_memory()
    flush = torch.empty(2 * L2_BYTES // 4, dtype=torch.float32, device="cuda")
    stream = torch.cuda.current_stream()

    def step():
        sst.sst_forward_inverse(plan.handle, x, w.n, tfr, xhat, plan.workspace, stream)

    for _ in range(max(args.warmup, 3)):
        step()
    torch.cuda.synchronize()

    # ---- timed region: K steps, L2 flushed before each (outside the events)
    sampler = ClockSampler(local)
    sampler.start()
    time.sleep(0.3)
    launches0 = sst.sst_launch_count()
    sst.sst_profile_enable(True)
    sst.sst_profile_collect()
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
           for _ in range(args.steps)]
    barrier()
    torch.cuda.synchronize()
    wall0 = time.perf_counter()
    for i in range(args.steps):
        flush.fill_(float(i))
        evs[i][0].record(stream)
        step()
        evs[i][1].record(stream)
    torch.cuda.synchronize()
    barrier()
    wall = time.perf_counter() - wall0
    sst.sst_profile_enable(False)
    prof = sst.sst_profile_collect()
    launches = sst.sst_launch_count() - launches0
    clocks = sampler.stop()
    step_ms = [a.elapsed_time(b) for a, b in evs]
    t_ms = max_over_ranks(sum(step_ms), dist)
    value = job_rate(world, w.n, args.steps, t_ms / 1e3)

    # ---- end to end through the C ABI with host buffers
    for _ in range(2):
        sst.sst_forward_inverse_host(plan.handle, x_host, w.n, xhat_host, x, tfr, xhat, plan.workspace, stream)
    barrier()
    e0 = time.perf_counter()
    for _ in range(args.steps):
        sst.sst_forward_inverse_host(plan.handle, x_host, w.n, xhat_host, x, tfr, xhat, plan.workspace, stream)
    e_s = max_over_ranks(time.perf_counter() - e0, dist)
    e2e = job_rate(world, w.n, args.steps, e_s)

    # ---- the same step without a TFR output (T kept on chip, one fused
    # kernel per tile; relative threshold from a pre-pass over every frame)
    fused = None
    if plan_supports_fused(sst, plan, x, w.n, xhat, stream):
        for _ in range(2):
            sst.sst_forward_inverse(plan.handle, x, w.n, None, xhat, plan.workspace, stream)
        torch.cuda.synchronize()
        sst.sst_profile_enable(True)
        sst.sst_profile_collect()
        fevs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
                for _ in range(args.steps)]
        barrier()
        torch.cuda.synchronize()
        for i in range(args.steps):
            flush.fill_(float(i))
            fevs[i][0].record(stream)
            sst.sst_forward_inverse(plan.handle, x, w.n, None, xhat, plan.workspace, stream)
            fevs[i][1].record(stream)
        torch.cuda.synchronize()
        sst.sst_profile_enable(False)
        fprof = sst.sst_profile_collect()
        f_ms = max_over_ranks(sum(a.elapsed_time(b) for a, b in fevs), dist)
        fused = {"value": job_rate(world, w.n, args.steps, f_ms / 1e3), "unit": UNIT,
                 "ms_per_step": f_ms / args.steps,
                 "kernels": {k: {"ms_per_step": v[0] / args.steps, "launches_per_step": v[1] / args.steps}
                             for k, v in fprof.items()}}

    if rank != 0:
        if dist is not None:
            dist.destroy_process_group()
        return 0

    # ---- roofline of the dominant kernel
    F = plan.frames
    fl = flops_per_frame(w)
    by = bytes_per_frame(w)
    dom = max(prof, key=lambda k: prof[k][0]) if prof else None
    roof = None
    peaks = measured_peaks()
    num_sms = torch.cuda.get_device_properties(0).multi_processor_count
    if dom in fl:
        tot_ms, cnt = prof[dom]
        per_launch_ms = tot_ms / cnt
        units = F
        flops = fl[dom] * units
        achieved = flops / (per_launch_ms / 1e3) / 1e12
        sm_max = peaks.get("sm_max_mhz") or 2070.0
        nominal = fp32_peak_tflops(num_sms, sm_max)
        peak = sst.sst_fp32_peak(stream)
        tpf, tnote = measured_traffic_per_frame(dom)
        step_flops = sum(fl[k] for k in ("forward", "inverse")) * units
        roof = {"bound": "alu", "kernel": dom, "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                "frac": achieved / peak, "traffic": (tpf * units if tpf is not None else None),
                "traffic_note": tnote,
                "peak_note": ("FP32 FMA throughput measured in this run (sst_fp32_peak: independent fmaf "
                              f"chains); nominal {nominal:.1f} = {num_sms} SMs x 128 lanes x 2 x {sm_max:.0f} MHz"),
                "algorithmic_flops_per_launch": flops, "avg_launch_ms": per_launch_ms,
                "hbm_gbs_achieved": by[dom] * units / (per_launch_ms / 1e3) / 1e9,
                "hbm_peak_gbs": peaks.get("hbm_gbs"),
                "fused_step": {"algorithmic_flops": step_flops, "achieved": step_flops / (t_ms / args.steps / 1e3) / 1e12,
                               "frac": step_flops / (t_ms / args.steps / 1e3) / 1e12 / peak}}

    if fused is not None and roof is not None:
        f_s = fused["ms_per_step"] / 1e3
        fused["fused_step"] = {"algorithmic_flops": step_flops, "achieved": step_flops / f_s / 1e12,
                               "frac": step_flops / f_s / 1e12 / peak,
                               "note": "forward + inverse FLOPs as in roofline.fused_step; the pre-pass "
                                       "over every frame is extra work not counted"}
    kern = {k: {"ms_per_step": v[0] / args.steps, "launches_per_step": v[1] / args.steps} for k, v in prof.items()}
    cpu = None
    if world == 1 and not args.no_cpu_baseline:
        import oracle as O
        O.build()
        O.set_threads(0)
        v, threads, sample, el = oracle_sample_rate(w, budget_s=10.0)
        O.set_threads(1)
        v1, _, sample1, el1 = oracle_sample_rate(w, budget_s=5.0, n_max=1 << 13)
        O.set_threads(0)
        cpu = {"value": v, "unit": UNIT, "cores": threads, "kind": "oracle", "sample": sample,
               "seconds": el, "cpu_model": cpu_model(),
               "single_thread": {"value": v1, "sample": sample1, "seconds": el1}}
    legs = None
    if world == 1 and not args.no_legs:
        # the rest of the metric, after the headline's timed region: the
        # tensor form against the FFT form, the streaming service's latency,
        # the batch's tuned time (the main workload's buffers freed first)
        plan.close()
        del tfr, xhat, flush, x
        torch.cuda.empty_cache()
        legs = run_legs(args)
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": max(args.warmup, 3), "ms_per_step": t_ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": w.name, "n": w.n, "fs": w.fs, "nfft": w.nfft, "hop": w.hop, "L": w.L,
                   "sigma": w.sigma, "z": w.z, "band_hz": [w.f_lo, w.f_hi], "gamma": "1e-3 max|V|",
                   "frames": F, "bins": plan.bins, "tfr_bytes": F * plan.bins * 8,
                   "l2": "flushed before each timed step (2x L2 write); T (8.6 GB) also exceeds L2",
                   "parallelism": f"replicas x{world}"},
        "gpu_launches": launches // max(1, 1),
        "gpu_launches_per_step": launches / args.steps,
        "kernels": kern,
        "roofline": roof,
        "variants": {"no_tfr_output": fused},
        "legs": legs,
        "cpu_baseline": cpu,
        "e2e": {"value": e2e, "unit": UNIT, "h2d_bytes_per_step": 4 * w.n, "d2h_bytes_per_step": 4 * w.n},
        "clocks": clocks,
        "wall_s_timed": wall,
    }
    print(json.dumps(line))
    plan.close()
    if dist is not None:
        dist.destroy_process_group()
    return 0


def second_order_leg(args) -> dict:
    """The second-order IF variant (sst_forward2, three packed FFTs per frame,
    + sst_inverse) on the run-up recipe at 2^22 samples: samples/s, beside
    the first-order forward + inverse of the same plan."""
    import torch
    from paper_2003_07065_gb300 import sst
    w = W.ALL["runup_4m"]
    x = torch.from_numpy(w.signal()[0].astype(np.float32)).cuda()
    plan = sst.Plan(**w.params())
    tfr = plan.new_tfr()
    xhat = torch.empty(w.n, dtype=torch.float32, device="cuda")
    flush = torch.empty(2 * L2_BYTES // 4, dtype=torch.float32, device="cuda")
    stream = torch.cuda.current_stream()
    res = {}
    for name, fwd in (("second_order", lambda: sst.sst_forward2(plan.handle, x, w.n, tfr, plan.workspace, stream)),
                      ("first_order", lambda: sst.sst_forward(plan.handle, x, w.n, tfr, plan.workspace, stream))):
        def step():
            fwd()
            sst.sst_inverse(plan.handle, tfr, w.n, xhat, plan.workspace, stream)
        for _ in range(args.warmup):
            step()
        evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
        torch.cuda.synchronize()
        for i in range(args.steps):
            flush.fill_(float(i))
            evs[i][0].record(stream)
            step()
            evs[i][1].record(stream)
        torch.cuda.synchronize()
        ms = sum(a.elapsed_time(b) for a, b in evs) / args.steps
        res[name] = {"ms_per_step": ms, "samples_per_s": w.n / (ms / 1e3)}
    plan.close()
    del tfr, flush
    torch.cuda.empty_cache()
    res["workload"] = w.name
    return res


def run_legs(args) -> dict:
    """Short runs of the other workloads for the headline line (one GPU)."""
    import types
    out = {}
    k = types.SimpleNamespace(steps=max(3, min(args.steps, 5)), warmup=3)
    try:
        t = tensor_leg(k)
        out["precision64k_tc"] = {
            "bf16_vs_fft_form": t["vs_fft_form"], "bf16_snr_gap_db": t["snr_gap_db"],
            "best_form_at_equal_snr": t["best_form_at_equal_snr"],
            "forms": {f: {"ms_per_step": v["ms_per_step"], "snr_db": v["snr_db"],
                          "contraction_frac": v.get("contraction", {}).get("frac")} for f, v in t["forms"].items()},
            "bf16_peak_tflops": t["bf16_peak"],
            "bf16_peak_source": "measured" if measured_peaks().get("bf16_tflops") else "fallback"}
    except Exception as e:   # reported, never fatal to the headline
        out["precision64k_tc"] = {"error": repr(e)}
    try:
        st = stream_leg(k, dur=4.0, overload_s=2.0)
        out["stream64"] = {"p50_s": st["latency_s"]["p50"], "p99_s": st["latency_s"]["p99"],
                           "chunks": st["latency_s"]["chunks"], "dropped": st["latency_s"]["dropped_chunks"],
                           "offered_samples_per_s": st["latency_s"]["offered_samples_per_s"],
                           "sustained_samples_per_s": st["value"],
                           "sustained_xhat_only_samples_per_s": st["sustained_xhat_only"]["value"],
                           "seconds": st["seconds"]}
    except Exception as e:
        out["stream64"] = {"error": repr(e)}
    try:
        out["runup_4m_second_order"] = second_order_leg(k)
    except Exception as e:
        out["runup_4m_second_order"] = {"error": repr(e)}
    try:
        b = batch_leg(k)
        out["batch256"] = {"samples_per_s": b["value"], "ms_per_step": b["ms_per_step"],
                           "untuned_ms": b["autotune"]["untuned_ms"], "tuned_ms": b["autotune"]["tuned_ms"],
                           "roofline_frac": b["roofline"]["frac"], "total_samples": b["total_samples"]}
    except Exception as e:
        out["batch256"] = {"error": repr(e)}
    return out


if __name__ == "__main__":
    sys.exit(main())

"""Builds the two libraries in-tree with nvcc for sm_103a.

libsst.so: each DFT length gets its own translation unit (sst_inst.cu with
-DSST_NF=...) so the units compile in parallel; the host code is sst_capi.cu
and its siblings in csrc/.

libsst_tc.so (build_tc): the tensor-core band form, csrc/tc/, linked against
libsst.so.  It is a separate library because its contraction uses multicast
TMA loads within a cluster; programs that run on several GPUs build and load
libsst.so alone.

Both go to ``paper_2003_07065_gb300/_lib/`` (git-ignored).
"""
from __future__ import annotations

import concurrent.futures as cf
import hashlib
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(ROOT, "include")
OUT_DIR = os.path.join(HERE, "_lib")
LIB = os.path.join(OUT_DIR, "libsst.so")
TC_LIB = os.path.join(OUT_DIR, "libsst_tc.so")
TC_SRC = os.path.join(CSRC, "tc", "sst_tc.cu")
NFS = (64, 128, 256, 512, 1024, 2048, 4096, 8192)
HOST_UNITS = ("sst_capi", "sst_batch", "sst_stream", "sst_post")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def _nvcc() -> str:
    for c in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if c and os.path.exists(c):
            return c
    raise RuntimeError("nvcc not found")


def _sources():
    return sorted(os.path.join(CSRC, f) for f in os.listdir(CSRC)
                  if f.endswith((".cu", ".cuh", ".h")))


def _fingerprint(flags, extra=()) -> str:
    h = hashlib.sha256()
    for p in _sources() + [os.path.join(INCLUDE, "sst.h")] + list(extra):
        with open(p, "rb") as f:
            h.update(f.read())
    h.update(" ".join(flags).encode())
    return h.hexdigest()


def _flags(ptxas_verbose: bool):
    flags = ARCH + ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC",
                    "-Xcompiler", "-fvisibility=hidden", "-I", CSRC, "-I", INCLUDE]
    if ptxas_verbose:
        flags += ["-Xptxas", "-v"]
    return flags


def build(verbose: bool = False, force: bool = False, ptxas_verbose: bool = False) -> str:
    """Builds libsst.so (skipped when its sources and flags are unchanged)."""
    nvcc = _nvcc()
    flags = _flags(ptxas_verbose)
    os.makedirs(OUT_DIR, exist_ok=True)
    stamp = os.path.join(OUT_DIR, "libsst.stamp")
    fp = _fingerprint(flags)
    if not force and os.path.exists(LIB) and os.path.exists(stamp):
        with open(stamp) as f:
            if f.read().strip() == fp:
                return LIB
    objdir = os.path.join(OUT_DIR, "obj")
    os.makedirs(objdir, exist_ok=True)
    jobs = [([nvcc] + flags + [f"-DSST_NF={nf}", "-c", os.path.join(CSRC, "sst_inst.cu"),
                               "-o", os.path.join(objdir, f"inst_{nf}.o")]) for nf in NFS]
    for name in HOST_UNITS:
        jobs.append([nvcc] + flags + ["-c", os.path.join(CSRC, name + ".cu"),
                                      "-o", os.path.join(objdir, name + ".o")])

    def run(cmd):
        r = subprocess.run(cmd, capture_output=True, text=True)
        return cmd, r

    workers = max(1, min(len(jobs), os.cpu_count() or 4))
    with cf.ThreadPoolExecutor(workers) as ex:
        for cmd, r in ex.map(run, jobs):
            if verbose or ptxas_verbose or r.returncode != 0:
                sys.stderr.write(r.stdout + r.stderr)
            if r.returncode != 0:
                raise RuntimeError("nvcc failed: " + " ".join(cmd))
    objs = [os.path.join(objdir, f"inst_{nf}.o") for nf in NFS] + \
        [os.path.join(objdir, name + ".o") for name in HOST_UNITS]
    tmp = LIB + f".tmp{os.getpid()}"
    cmd = [nvcc] + ARCH + ["-shared", "-o", tmp] + objs
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        sys.stderr.write(r.stdout + r.stderr)
        raise RuntimeError("link failed")
    os.replace(tmp, LIB)
    with open(stamp, "w") as f:
        f.write(fp)
    return LIB


def build_tc(verbose: bool = False, force: bool = False, ptxas_verbose: bool = False) -> str:
    """Builds libsst_tc.so (after libsst.so, which it links against)."""
    build(verbose=verbose, force=force, ptxas_verbose=ptxas_verbose)
    nvcc = _nvcc()
    flags = _flags(ptxas_verbose)
    stamp = os.path.join(OUT_DIR, "libsst_tc.stamp")
    fp = _fingerprint(flags, [TC_SRC, os.path.join(INCLUDE, "sst_tc.h"), LIB])
    if not force and os.path.exists(TC_LIB) and os.path.exists(stamp):
        with open(stamp) as f:
            if f.read().strip() == fp:
                return TC_LIB
    objdir = os.path.join(OUT_DIR, "obj")
    os.makedirs(objdir, exist_ok=True)
    obj = os.path.join(objdir, "sst_tc.o")
    r = subprocess.run([nvcc] + flags + ["-c", TC_SRC, "-o", obj], capture_output=True, text=True)
    if verbose or ptxas_verbose or r.returncode != 0:
        sys.stderr.write(r.stdout + r.stderr)
    if r.returncode != 0:
        raise RuntimeError("nvcc failed on " + TC_SRC)
    tmp = TC_LIB + f".tmp{os.getpid()}"
    cmd = [nvcc] + ARCH + ["-shared", "-o", tmp, obj, "-L", OUT_DIR, "-lsst",
                           "-Xlinker", "-rpath", "-Xlinker", "$ORIGIN"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        sys.stderr.write(r.stdout + r.stderr)
        raise RuntimeError("link of libsst_tc.so failed")
    os.replace(tmp, TC_LIB)
    with open(stamp, "w") as f:
        f.write(fp)
    return TC_LIB


if __name__ == "__main__":
    build(verbose=True, force="--force" in sys.argv, ptxas_verbose="-v" in sys.argv)
    print(LIB)
    if "--tc" in sys.argv:
        build_tc(verbose=True, force="--force" in sys.argv, ptxas_verbose="-v" in sys.argv)
        print(TC_LIB)

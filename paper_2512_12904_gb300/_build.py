"""Build the CUDA library (libhqc_gb300.so) in-tree with nvcc for sm_103a.

The translation units are compiled in parallel and linked into one shared
library with a plain C ABI (include/hqc_gb300.h); the on-chip peak
microbenchmarks go into a second one (libhqc_peaks.so).
"""
from __future__ import annotations

import hashlib
import os
import subprocess
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(BUILD, "libhqc_gb300.so")
PEAKS_LIB = os.path.join(BUILD, "libhqc_peaks.so")
SOURCES = ["hqc_decrypt.cu", "hqc_stage.cu", "hqc_tune.cu", "hqc_encrypt.cu", "hqc_abi.cu", "hqc_noalloc.cu", "hqc_plan.cu", "hqc_serve.cu", "hqc_host.cu", "hqc_kem.cu", "hqc_rm_tc.cu"]
PEAKS_SOURCES = ["hqc_peaks.cu"]
HEADERS = ["hqc_params.cuh", "hqc_device.cuh", "hqc_kernels.cuh", "hqc_internal.h", "hqc_keccak.cuh", "hqc_kem_k.cuh"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-Xcompiler", "-Wall"]


def _nvcc() -> str:
    cand = os.path.join(os.environ.get("CUDA_HOME", "/usr/local/cuda"), "bin", "nvcc")
    return cand if os.path.exists(cand) else "nvcc"


def _digest() -> str:
    h = hashlib.sha256()
    files = [os.path.join(CSRC, f) for f in SOURCES + PEAKS_SOURCES + HEADERS]
    files.append(os.path.join(ROOT, "include", "hqc_gb300.h"))
    for f in files:
        with open(f, "rb") as fh:
            h.update(fh.read())
    h.update(" ".join(ARCH + FLAGS).encode())
    return h.hexdigest()


def kernel_digest() -> str:
    """Digest of the device code of the decryption kernels (the kernel
    templates up to their launch helpers, and the headers they include):
    profile counters of those kernels stay valid while it holds."""
    h = hashlib.sha256()
    for f in ("hqc_kernels.cuh", "hqc_device.cuh", "hqc_params.cuh", "hqc_internal.h"):
        with open(os.path.join(CSRC, f), "rb") as fh:
            data = fh.read()
        if f == "hqc_kernels.cuh":
            cut = data.find(b"// Launch helpers")
            data = data[:cut] if cut >= 0 else data
        h.update(data)
    h.update(" ".join(ARCH + FLAGS).encode())
    return h.hexdigest()


def build(force: bool = False, verbose: bool = False) -> str:
    """Compile if the sources changed since the last build; return the .so path."""
    os.makedirs(BUILD, exist_ok=True)
    stamp = os.path.join(BUILD, "stamp")
    dig = _digest()
    if not force and os.path.exists(LIB) and os.path.exists(PEAKS_LIB) and os.path.exists(stamp):
        with open(stamp) as f:
            if f.read().strip() == dig:
                return LIB
    nvcc = _nvcc()

    def compile_one(src):
        obj = os.path.join(BUILD, src.replace(".cu", ".o"))
        cmd = [nvcc, *ARCH, *FLAGS, "-c", os.path.join(CSRC, src), "-o", obj]
        if verbose:
            cmd.insert(1, "-Xptxas=-v")
        res = subprocess.run(cmd, capture_output=True, text=True)
        if res.returncode != 0:
            raise RuntimeError("nvcc failed for %s:\n%s%s" % (src, res.stdout, res.stderr))
        return obj, res.stderr

    with ThreadPoolExecutor(len(SOURCES) + len(PEAKS_SOURCES)) as ex:
        results = list(ex.map(compile_one, SOURCES + PEAKS_SOURCES))
    if verbose:
        for _, log in results:
            print(log)
    for lib, objs in ((LIB, results[:len(SOURCES)]), (PEAKS_LIB, results[len(SOURCES):])):
        tmp = lib + ".tmp%d" % os.getpid()
        cmd = [nvcc, *ARCH, "-shared", "-o", tmp] + [o for o, _ in objs]
        res = subprocess.run(cmd, capture_output=True, text=True)
        if res.returncode != 0:
            raise RuntimeError("link failed:\n%s%s" % (res.stdout, res.stderr))
        os.replace(tmp, lib)
    with open(stamp, "w") as f:
        f.write(dig)
    return LIB


if __name__ == "__main__":
    import sys
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))

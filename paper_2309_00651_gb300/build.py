"""Build libhfx.so in-tree with nvcc for sm_103a (GB300).

The three translation units (host API + pair staging, FP32 passes, FP64 passes) compile in
parallel, then link into ``paper_2309_00651_gb300/libhfx.so``.  A stamp of the sources,
flags and host machine skips the rebuild when nothing changed.
"""
from __future__ import annotations

import concurrent.futures as cf
import fcntl
import hashlib
import os
import platform
import shutil
import subprocess

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
BUILD = os.path.join(PKG, "_build")
LIB = os.path.join(PKG, "libhfx.so")
LIB_DEBUG = os.path.join(PKG, "libhfx_debug.so")
INCLUDE = os.path.join(ROOT, "include")

SOURCES = ["hfx_api.cu", "hfx_passes_f32.cu", "hfx_passes_f64.cu", "hfx_ace.cu", "hfx_ace_tc.cu", "hfx_dft_tc.cu", "hfx_scdm.cu", "hfx_sinr.cu", "hfx_peak.cu"] + [
    f"hfx_ct_{n}.cu" for n in (32, 48, 64, 72, 80, 90, 96, 128)]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ["-std=c++17", "-O3", "-lineinfo", "-Xcompiler", "-fPIC,-O2", "-I", INCLUDE] + ARCH


def nvcc_path() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found (CUDA toolkit required to build libhfx)")


def source_hash() -> str:
    """Hash of the CUDA/C sources and headers alone (the same on every machine)."""
    h = hashlib.sha256()
    for d in (CSRC, INCLUDE):
        for name in sorted(os.listdir(d)):
            p = os.path.join(d, name)
            if os.path.isfile(p):
                h.update(name.encode())
                with open(p, "rb") as f:
                    h.update(f.read())
    return h.hexdigest()[:16]


KERNEL_SOURCES = ("fft_codelets.cuh", "fft_plan.h", "hfx_kernels.cuh", "hfx_ct.cuh")


def kernel_hash() -> str:
    """Hash of the device-kernel sources only (the code whose hardware counters profiles/ records)."""
    h = hashlib.sha256()
    for name in KERNEL_SOURCES:
        with open(os.path.join(CSRC, name), "rb") as f:
            h.update(name.encode())
            h.update(f.read())
    return h.hexdigest()[:16]


def _stamp() -> str:
    h = hashlib.sha256()
    for d in (CSRC, INCLUDE):
        for name in sorted(os.listdir(d)):
            p = os.path.join(d, name)
            if os.path.isfile(p):
                h.update(name.encode())
                with open(p, "rb") as f:
                    h.update(f.read())
    h.update(" ".join(NVCC_FLAGS).encode())
    h.update(platform.machine().encode())
    return h.hexdigest()


def build(verbose: bool = False, force: bool = False, debug: bool = False) -> str:
    """Compile (if needed) and return the path of libhfx.so, or of libhfx_debug.so with debug=True
    (HFX_DEBUG: workspace guard bands and the device-side couple-layout check)."""
    build_dir = BUILD + ("_debug" if debug else "")
    os.makedirs(build_dir, exist_ok=True)
    # one build at a time per folder: the ranks of a multi-process launch all call build(), and
    # only the first compiles; the others wait here and then find the stamp up to date
    with open(os.path.join(build_dir, "lock"), "w") as lock:
        fcntl.flock(lock, fcntl.LOCK_EX)
        try:
            return _build(build_dir, verbose, force, debug)
        finally:
            fcntl.flock(lock, fcntl.LOCK_UN)


def _build(build_dir: str, verbose: bool, force: bool, debug: bool) -> str:
    lib = LIB_DEBUG if debug else LIB
    flags = NVCC_FLAGS + (["-DHFX_DEBUG"] if debug else [])
    stamp_file = os.path.join(build_dir, "stamp")
    stamp = _stamp() + ("-debug" if debug else "")
    if not force and os.path.exists(lib) and os.path.exists(stamp_file):
        with open(stamp_file) as f:
            if f.read().strip() == stamp:
                return lib
    nvcc = nvcc_path()

    def compile_one(src: str) -> str:
        obj = os.path.join(build_dir, src.replace(".cu", ".o"))
        cmd = [nvcc] + flags + ["-c", os.path.join(CSRC, src), "-o", obj]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed for {src}:\n{r.stdout}\n{r.stderr}")
        if verbose:
            print(r.stdout + r.stderr)
        return obj

    with cf.ThreadPoolExecutor(max_workers=min(len(SOURCES), max(2, os.cpu_count() or 2))) as ex:
        objs = list(ex.map(compile_one, SOURCES))
    tmp = lib + ".tmp"
    cmd = [nvcc] + ARCH + ["-shared", "-Xcompiler", "-fPIC", "-o", tmp] + objs
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, lib)
    with open(stamp_file, "w") as f:
        f.write(stamp)
    return lib


if __name__ == "__main__":
    print(build(verbose=True, force=True))

"""Compile the CUDA library in place: one object per translation unit (in
parallel), linked into paper_2302_00752_gb300/libsparse_spectral.so for sm_103a.

    python -m paper_2302_00752_gb300.build
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libsparse_spectral.so")
PEAKS_LIB = os.path.join(HERE, "libss_peaks.so")   # rate microbenchmarks (benchmark only)
SOURCES = ["api.cu", "scan.cu", "stamp.cu", "apply.cu", "lattice.cu", "sft.cu", "solve.cu", "batch.cu", "proxy.cu",
           "pipeline.cu", "fft_df.cu", "fft_pruned.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found")


def cuda_lib_dir(nv: str) -> str:
    root = os.path.dirname(os.path.dirname(os.path.realpath(nv)))
    for sub in ("lib64", "lib", os.path.join("targets", "sbsa-linux", "lib"), os.path.join("targets", "x86_64-linux", "lib")):
        p = os.path.join(root, sub)
        if os.path.exists(os.path.join(p, "libcufft.so")):
            return p
    return os.path.join(root, "lib64")


def _compile(nv: str, src: str, obj: str, verbose: bool) -> None:
    cmd = [nv, "-std=c++17", *ARCH, "-O3", "-lineinfo", "-Xcompiler", "-fPIC", "-c", src, "-o", obj]
    if verbose:
        cmd.insert(1, "-Xptxas=-v")
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"nvcc failed for {os.path.basename(src)}:\n{r.stdout}\n{r.stderr}")
    if verbose:
        sys.stderr.write(r.stderr)


def up_to_date() -> bool:
    if not os.path.exists(LIB) or not os.path.exists(PEAKS_LIB):
        return False
    t = min(os.path.getmtime(LIB), os.path.getmtime(PEAKS_LIB))
    deps = [os.path.join(CSRC, f) for f in os.listdir(CSRC)]
    deps.append(os.path.join(os.path.dirname(HERE), "include", "sparse_spectral.h"))
    return all(os.path.getmtime(p) <= t for p in deps)


def build(force: bool = False, verbose: bool = False) -> str:
    if not force and up_to_date():
        return LIB
    nv = nvcc()
    os.makedirs(BUILD, exist_ok=True)
    objs = [os.path.join(BUILD, s.replace(".cu", ".o")) for s in SOURCES]
    peaks_obj = os.path.join(BUILD, "peaks.o")
    with cf.ThreadPoolExecutor(max_workers=min(len(SOURCES) + 1, os.cpu_count() or 4)) as ex:
        futs = [ex.submit(_compile, nv, os.path.join(CSRC, s), o, verbose) for s, o in zip(SOURCES, objs)]
        futs.append(ex.submit(_compile, nv, os.path.join(CSRC, "peaks.cu"), peaks_obj, verbose))
        for f in futs:
            f.result()
    libdir = cuda_lib_dir(nv)
    tmp = LIB + ".tmp"
    cmd = [nv, *ARCH, "-shared", "-cudart", "shared", "-o", tmp, *objs, f"-L{libdir}", "-lcufft",
           "-Xlinker", f"-rpath={libdir}"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, LIB)
    tmp = PEAKS_LIB + ".tmp"
    r = subprocess.run([nv, *ARCH, "-shared", "-cudart", "shared", "-o", tmp, peaks_obj], capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link of the peaks library failed:\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, PEAKS_LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))

"""In-tree build of the CUDA library (``_build/librhd.so``) and its tools.

Everything is compiled for sm_103a only, with one nvcc call per target so the
build stays a few seconds long; the outputs live next to the sources and are
git-ignored.
"""
from __future__ import annotations

import os
import subprocess
from concurrent.futures import ThreadPoolExecutor

PKG = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(PKG, "csrc")
BUILD = os.path.join(PKG, "_build")
LIB = os.path.join(BUILD, "librhd.so")
FP_PEAK = os.path.join(BUILD, "fp_peak")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC = os.environ.get("NVCC", "nvcc")


def _newer(out: str, deps: list[str]) -> bool:
    return os.path.exists(out) and os.path.getmtime(out) >= max(os.path.getmtime(d) for d in deps)


def _sources() -> list[str]:
    deps = [os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith((".cu", ".cuh"))]
    deps.append(os.path.join(os.path.dirname(PKG), "include", "rhd.h"))
    return deps


def _run(cmd: list[str], out: str) -> str:
    tmp = out + f".tmp{os.getpid()}"
    subprocess.run(cmd + ["-o", tmp], check=True)
    os.replace(tmp, out)
    return out


def build_lib(force: bool = False) -> str:
    if not force and _newer(LIB, _sources()):
        return LIB
    cmd = [NVCC, *ARCH, "-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-shared",
           "-cudart", "shared", os.path.join(CSRC, "rhd.cu")]
    return _run(cmd, LIB)


def build_fp_peak(force: bool = False) -> str:
    src = os.path.join(CSRC, "fp_peak.cu")
    if not force and _newer(FP_PEAK, [src]):
        return FP_PEAK
    return _run([NVCC, *ARCH, "-O3", "-lineinfo", src], FP_PEAK)


def build_all(force: bool = False) -> list[str]:
    os.makedirs(BUILD, exist_ok=True)
    with ThreadPoolExecutor(max_workers=2) as ex:
        futs = [ex.submit(build_lib, force), ex.submit(build_fp_peak, force)]
        return [f.result() for f in futs]


if __name__ == "__main__":
    for p in build_all(force=True):
        print(p)

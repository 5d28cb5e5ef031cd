"""Build the library in-tree: paper_1909_02294_gb300/libftv.so for sm_103a (nvcc, no cmake).

Translation units are compiled in parallel, then linked with the CUDA runtime linked statically so the
shared object does not depend on where libcudart lives. Host code is compiled without floating-point
contraction so the FP64 homographies round identically on x86-64 and AArch64.
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
LIB = os.path.join(HERE, "libftv.so")
BUILD = os.path.join(HERE, "_build")
LIB_CHECKED = os.path.join(HERE, "libftv_checked.so")
BUILD_CHECKED = os.path.join(HERE, "_build_checked")
SOURCES = ["ftv_api.cu", "ftv_cost.cu", "ftv_index.cu", "ftv_temporal.cu", "ftv_batch.cu", "ftv_noalloc.cu",
           "ftv_centre.cu", "ftv_adjacency.cu", "ftv_superpixels.cu", "ftv_geometry.cpp"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def nvcc() -> str:
    for p in [os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"]:
        if p and os.path.exists(p):
            return p
    raise RuntimeError("nvcc not found")


def _flags(checked: bool = False) -> list[str]:
    return ["-O3", "-std=c++17", *ARCH, "-lineinfo", "-I", os.path.join(ROOT, "include"),
            "-Xcompiler", "-fPIC,-fvisibility=hidden,-ffp-contract=off,-fno-fast-math",
            "-Xptxas", "-warn-spills", *(["-DFTV_CHECKED"] if checked else [])]


def _compile(src: str, checked: bool = False) -> str:
    build_dir = BUILD_CHECKED if checked else BUILD
    obj = os.path.join(build_dir, os.path.basename(src) + ".o")
    path = os.path.join(CSRC, src)
    headers = [os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith((".h", ".cuh"))]
    deps = [path, *headers, os.path.join(ROOT, "include", "ftv.h")]
    if os.path.exists(obj) and all(os.path.getmtime(obj) >= os.path.getmtime(d) for d in deps):
        return obj
    cmd = [nvcc(), *_flags(checked), "-c", path, "-o", obj]
    if src.endswith(".cpp"):
        cmd = [nvcc(), "-x", "c++", *_flags(checked), "-c", path, "-o", obj]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"nvcc failed for {src}:\n{r.stdout}\n{r.stderr}")
    if r.stderr.strip() and not checked:
        sys.stderr.write(r.stderr)
    return obj


def build(verbose: bool = False, checked: bool = False) -> str:
    """The library (libftv.so), or with checked=True its checked variant (libftv_checked.so: every cost-kernel
    gather tested against its view, an index outside recorded as FTV_ERR_CHECKED and skipped), a test build
    that the tests load through FTV_LIBRARY."""
    build_dir, lib = (BUILD_CHECKED, LIB_CHECKED) if checked else (BUILD, LIB)
    os.makedirs(build_dir, exist_ok=True)
    srcs = [s for s in SOURCES if os.path.exists(os.path.join(CSRC, s))]
    with cf.ThreadPoolExecutor(max_workers=len(srcs)) as ex:
        objs = list(ex.map(lambda src: _compile(src, checked), srcs))
    if not os.path.exists(lib) or any(os.path.getmtime(o) > os.path.getmtime(lib) for o in objs):
        tmp = lib + f".tmp{os.getpid()}"
        cmd = [nvcc(), *ARCH, "-shared", "-cudart", "static", "-o", tmp, *objs, "-ldl"]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
        os.replace(tmp, lib)
    if verbose:
        print(f"built {lib}")
    return lib


def ptxas_report(src: str = "ftv_cost.cu") -> str:
    """Registers, spills and shared memory per kernel (ptxas -v), for tuning."""
    cmd = [nvcc(), *_flags(), "-Xptxas", "-v", "-c", os.path.join(CSRC, src), "-o", os.devnull]
    r = subprocess.run(cmd, capture_output=True, text=True)
    return r.stdout + r.stderr


if __name__ == "__main__":
    build(verbose=True)

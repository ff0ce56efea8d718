"""Build libsv.so in-tree with nvcc for sm_103a (no GPU needed to compile).

Each translation unit under csrc/ compiles in parallel to an object file in
_build/, then nvcc links them into paper_1912_03243_gb300/libsv.so with the
static CUDA runtime.
"""

from __future__ import annotations

import concurrent.futures as cf
import hashlib
import os
import platform
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(ROOT, "_build")
LIB = os.path.join(HERE, "libsv.so")
WORKER_SRC = os.path.join(HERE, "csrc", "worker", "nvrtc_worker.cpp")
WORKER = os.path.join(HERE, "sv_nvrtc_worker")  # next to libsv.so, where the library looks for it
INCLUDE = os.path.join(ROOT, "include")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC", "-Xcompiler", "-O2",
              "--expt-relaxed-constexpr", "-I", INCLUDE, "-I", CSRC]


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found")


def sources() -> list[str]:
    return sorted(os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith((".cu", ".cpp")))


def headers() -> list[str]:
    hs = [os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith(".h")]
    return sorted(hs + [os.path.join(INCLUDE, "sv.h")])


def _digest(src: str, extra: list[str]) -> str:
    h = hashlib.sha1()
    for p in [src] + headers():
        with open(p, "rb") as f:
            h.update(f.read())
    h.update(" ".join(extra + NVCC_FLAGS + ARCH + [platform.machine()]).encode())
    return h.hexdigest()[:16]


def _compile(src: str, extra: list[str], verbose: bool) -> str:
    base = os.path.splitext(os.path.basename(src))[0]
    obj = os.path.join(BUILD, f"{base}.{_digest(src, extra)}.o")
    if os.path.exists(obj):
        return obj
    cmd = [nvcc(), *ARCH, *NVCC_FLAGS, *extra, "-c", src, "-o", obj + ".tmp"]
    if src.endswith(".cpp"):
        cmd.insert(1, "-x")
        cmd.insert(2, "cu")
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"nvcc failed for {src}:\n{r.stdout}\n{r.stderr}")
    if verbose and (r.stdout or r.stderr):
        sys.stderr.write(r.stdout + r.stderr)
    os.replace(obj + ".tmp", obj)
    return obj


def build(verbose: bool = False, ptxas_v: bool = False) -> str:
    """Compile every CUDA source and link libsv.so; returns its path."""
    os.makedirs(BUILD, exist_ok=True)
    extra = ["-Xptxas", "-v"] if ptxas_v else []
    srcs = sources()
    with cf.ThreadPoolExecutor(max_workers=min(8, len(srcs))) as ex:
        objs = list(ex.map(lambda s: _compile(s, extra, verbose or ptxas_v), srcs))
    tmp = LIB + f".tmp{os.getpid()}"
    cuda_lib = os.path.join(os.path.dirname(os.path.dirname(os.path.realpath(nvcc()))), "lib64")
    cmd = [nvcc(), *ARCH, "-shared", "-cudart", "static", "-o", tmp, *objs, "-lnvrtc",
           "-Xlinker", f"-rpath={cuda_lib}"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, LIB)
    build_worker(cuda_lib)
    return LIB


def build_worker(cuda_lib: str) -> str:
    """The NVRTC compile worker (an executable: NVRTC serialises compilations
    within a process, so the library runs several workers at once)."""
    h = hashlib.sha1()
    for p in (WORKER_SRC, os.path.join(CSRC, "nvrtc_opts.h")):
        with open(p, "rb") as f:
            h.update(f.read())
    h.update(platform.machine().encode())
    stamp = os.path.join(BUILD, f"sv_nvrtc_worker.{h.hexdigest()[:16]}")
    if not (os.path.exists(stamp) and os.path.exists(WORKER)):
        tmp = WORKER + f".tmp{os.getpid()}"
        cmd = [nvcc(), "-O2", "-std=c++17", "-o", tmp, WORKER_SRC, "-lnvrtc", "-Xlinker", f"-rpath={cuda_lib}"]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"worker build failed:\n{r.stdout}\n{r.stderr}")
        os.replace(tmp, WORKER)
        with open(stamp, "w"):
            pass
    return WORKER


if __name__ == "__main__":
    print(build(verbose=True, ptxas_v="-v" in sys.argv))

"""Builds libmppi.so for sm_103a (nvcc, in-tree, no cmake).

Each .cu translation unit compiles in parallel; the shared library links the
CUDA runtime statically so that it shares the device's primary context with
whatever else the process uses.
"""
from __future__ import annotations

import os
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
OUT_DIR = os.path.join(HERE, "lib")
LIB = os.path.join(OUT_DIR, "libmppi.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-Xcompiler", "-Wall",
              "--expt-relaxed-constexpr"]
# rollout kernel: 96 registers so that five 128-thread blocks fit on an SM
# (measured: 2.44 ms per 256-drone batched step vs 2.54 ms at 128 or 80)
DEFAULT_DEFINES = ("MPPI_ROLLOUT_MIN_BLOCKS=5",)
SOURCES = ["mppi_rollout_gate.cu", "mppi_rollout_contour.cu", "mppi_rollout_track.cu", "mppi_kernels.cu",
           "mppi_api.cu", "mppi_serve.cu", "mppi_noalloc.cu"]


def _nvcc() -> str:
    for c in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", "nvcc"):
        if c and (os.path.sep not in c or os.path.exists(c)):
            return c
    return "nvcc"


def _stale(lib: str, deps) -> bool:
    if not os.path.exists(lib):
        return True
    t = os.path.getmtime(lib)
    return any(os.path.getmtime(d) > t for d in deps)


def build(force: bool = False, verbose: bool = False, out_dir: str = None, defines=DEFAULT_DEFINES) -> str:
    """Compiles every translation unit and links libmppi.so into out_dir
    (default: the package's lib/).  defines: extra -D options."""
    out = out_dir or OUT_DIR
    lib = os.path.join(out, "libmppi.so")
    os.makedirs(out, exist_ok=True)
    srcs = [os.path.join(CSRC, s) for s in SOURCES if os.path.exists(os.path.join(CSRC, s))]
    deps = srcs + [os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith((".cuh", ".h"))]
    deps.append(os.path.join(os.path.dirname(HERE), "include", "mppi.h"))
    if not force and not _stale(lib, deps):
        return lib
    nvcc = _nvcc()
    objs = [os.path.join(out, os.path.basename(s).replace(".cu", ".o")) for s in srcs]

    def compile_one(pair):
        src, obj = pair
        cmd = [nvcc, *ARCH, *NVCC_FLAGS, *[f"-D{d}" for d in defines], "-c", src, "-o", obj]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed for {src}:\n{r.stderr}")
        if verbose and r.stderr:
            sys.stderr.write(r.stderr)
        return obj

    with ThreadPoolExecutor(max_workers=len(srcs)) as ex:
        list(ex.map(compile_one, zip(srcs, objs)))
    tmp = lib + ".tmp"
    cmd = [nvcc, *ARCH, "-shared", "-o", tmp, *objs, "-lpthread"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stderr}")
    os.replace(tmp, lib)
    return lib


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True))

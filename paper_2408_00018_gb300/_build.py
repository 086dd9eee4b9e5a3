"""In-tree build of the CUDA library (libsa103.so) for sm_103a with nvcc.

Each translation unit is compiled in parallel, then linked into one shared
library next to this file.  The library exposes the C ABI of include/sa.h
and links the CUDA runtime statically; it does not depend on PyTorch.
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
LIB = os.path.join(HERE, "libsa103.so")
BUILD_DIR = os.path.join(HERE, "_build")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
COMMON = ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC", "-Xptxas", "-v",
          "--expt-relaxed-constexpr", "-I" + CSRC]
# translation unit -> extra flags.  The FP64 sweep is compiled without FMA
# contraction so that its rounding follows the written expressions.
UNITS = {
    "sweep_f32.cu": [],
    "sweep_f32w.cu": [],
    "sweep_f64.cu": ["-fmad=false"],
    "reduce.cu": [],
    "sa_api.cu": [],
    "argmin_static.cu": [],
    "polish.cu": [],
    "gemm_tc.cu": [],
    "sweep_rot.cu": [],
    "rot_prep.cu": [],
    "mlp.cu": [],
    "da.cu": [],
    "crossover.cu": ["-fmad=false"],
    "pipes.cu": [],
    "sweep_batch.cu": [],
    "rot_tc.cu": [],
    "mlp_fused.cu": [],
}


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", shutil.which("nvcc")):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA library cannot be built")


def _sources():
    deps = [os.path.join(CSRC, f) for f in os.listdir(CSRC)]
    deps.append(os.path.join(os.path.dirname(HERE), "include", "sa.h"))
    return deps


def _stale() -> bool:
    if not os.path.exists(LIB):
        return True
    t = os.path.getmtime(LIB)
    return any(os.path.getmtime(p) > t for p in _sources())


def build(force: bool = False, verbose: bool = False) -> str:
    if not force and not _stale():
        return LIB
    os.makedirs(BUILD_DIR, exist_ok=True)
    cc = nvcc()

    def compile_unit(item):
        src, extra = item
        obj = os.path.join(BUILD_DIR, src.replace(".cu", ".o"))
        tuning = os.environ.get("SA_NVCC_FLAGS", "").split()  # e.g. -DSA_F32W_MIN_BLOCKS=2 for tuning runs
        cmd = [cc, *ARCH, *COMMON, *extra, *tuning, "-c", os.path.join(CSRC, src), "-o", obj]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed on {src}:\n{r.stdout}\n{r.stderr}")
        return obj, r.stderr

    with cf.ThreadPoolExecutor(max_workers=len(UNITS)) as ex:
        results = list(ex.map(compile_unit, UNITS.items()))
    if verbose:
        for _, log in results:
            print(log)
    tmp = LIB + f".tmp{os.getpid()}"
    cmd = [cc, *ARCH, "-shared", "-Xcompiler", "-fPIC", *[o for o, _ in results], "-o", tmp, "-cudart=static"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force=True, verbose=True))

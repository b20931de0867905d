"""Build ``libge.so`` in-tree for sm_103a (nvcc for the kernels, the host C++
compiler for the C ABI), translation units compiled in parallel.

    python -m paper_1310_3422_gb300.build
"""
from __future__ import annotations

import os
import shutil
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
INCLUDE = os.path.join(ROOT, "include")
OBJ_DIR = os.path.join(PKG, "_build")
LIB_PATH = os.path.join(PKG, "libge.so")

CUDA_HOME = os.environ.get("CUDA_HOME", "/usr/local/cuda")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
CU_SOURCES = ["ge_canon.cu", "ge_tb.cu", "ge_tb_df.cu", "ge_tbb.cu", "ge_tbb_df.cu", "ge_sweep.cu", "ge_noalloc.cu", "ge_sno_kernels.cu", "ge_sno_tc.cu", "ge_probe.cu"]
CPP_SOURCES = ["ge_api.cpp", "ge_tb_plan.cpp", "ge_batch.cpp", "ge_sno.cpp"]


def _nvcc() -> str:
    cand = os.path.join(CUDA_HOME, "bin", "nvcc")
    return cand if os.path.exists(cand) else (shutil.which("nvcc") or "nvcc")


def _run(cmd):
    res = subprocess.run(cmd, capture_output=True, text=True)
    if res.returncode != 0:
        raise RuntimeError("build step failed:\n" + " ".join(cmd) + "\n" + res.stdout + res.stderr)
    return res.stdout + res.stderr


def build(verbose: bool = False, defines=(), lib_path: str = LIB_PATH, obj_dir: str = OBJ_DIR) -> str:
    """Compile and link the library.  `defines` are extra -D macros (tuning
    knobs of the kernels); `lib_path`/`obj_dir` place a variant elsewhere."""
    os.makedirs(obj_dir, exist_ok=True)
    dflags = ["-D" + d for d in defines]
    inc = ["-I" + INCLUDE, "-I" + CSRC, "-I" + os.path.join(CUDA_HOME, "include")]
    jobs = []
    for src in CU_SOURCES:
        obj = os.path.join(obj_dir, src + ".o")
        jobs.append([_nvcc(), *ARCH, "-O3", "-lineinfo", "-std=c++17", "-Xptxas", "-v",
                     "-Xcompiler", "-fPIC,-ffp-contract=off", *dflags, *inc, "-c",
                     os.path.join(CSRC, src), "-o", obj])
    for src in CPP_SOURCES:
        obj = os.path.join(obj_dir, src + ".o")
        jobs.append(["g++", "-O2", "-std=c++17", "-fPIC", "-ffp-contract=off", "-Wall",
                     *dflags, *inc, "-c", os.path.join(CSRC, src), "-o", obj])
    with ThreadPoolExecutor(max_workers=len(jobs)) as ex:
        logs = list(ex.map(_run, jobs))
    if verbose:
        for log in logs:
            sys.stdout.write(log)
    objs = [os.path.join(obj_dir, s + ".o") for s in CU_SOURCES + CPP_SOURCES]
    tmp = lib_path + ".tmp"
    _run(["g++", "-shared", "-o", tmp, *objs, "-L" + os.path.join(CUDA_HOME, "lib64"),
          "-lcudart", "-ldl", "-Wl,-rpath," + os.path.join(CUDA_HOME, "lib64")])
    os.replace(tmp, lib_path)
    return lib_path


if __name__ == "__main__":
    print(build(verbose="-v" in sys.argv))

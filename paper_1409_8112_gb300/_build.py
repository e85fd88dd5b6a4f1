"""Build of the GPU library (sm_103a) and of the input-generator library.

``build()`` compiles every translation unit in parallel with nvcc
(-gencode arch=compute_103a,code=sm_103a) and links ``_build/librtg.so`` with the CUDA
runtime linked statically, so the library loads on a machine without a GPU (only its
compute calls need one).  Rebuilds only when a source is newer than the library.
"""
from __future__ import annotations

import os
import shutil
import subprocess
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(ROOT, "include")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(BUILD, "librtg.so")

CU_SOURCES = ["rtg_api.cu", "rtg_keys.cu", "rtg_sort.cu", "rtg_pairs.cu", "rtg_serve.cu",
              "rtg_tc.cu", "rtg_noalloc.cu", "rtg_tune.cu", "rtg_query.cu",
              "rtg_params.cu", "rtg_index.cu"]
C_SOURCES = [os.path.join("gen", "rtg_gen.c")]
HEADERS = ["rtg_internal.cuh", "rtg_host.h", os.path.join("gen", "rtg_gen.h")]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def _nvcc() -> str:
    for cand in (shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found")


def _deps():
    deps = [os.path.join(CSRC, s) for s in CU_SOURCES + C_SOURCES + HEADERS]
    deps.append(os.path.join(INCLUDE, "rtg.h"))
    deps.append(os.path.abspath(__file__))
    return deps


def up_to_date() -> bool:
    if not os.path.exists(LIB):
        return False
    t = os.path.getmtime(LIB)
    return all(os.path.getmtime(p) <= t for p in _deps())


def build(force: bool = False, verbose: bool = False) -> str:
    if not force and up_to_date():
        return LIB
    os.makedirs(BUILD, exist_ok=True)
    nvcc = _nvcc()
    common = ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC", "-I", INCLUDE, "-I", CSRC]

    def cu(src):
        obj = os.path.join(BUILD, os.path.basename(src).replace(".cu", ".o"))
        cmd = [nvcc, *ARCH, *common, "-c", os.path.join(CSRC, src), "-o", obj]
        if verbose:
            cmd.insert(1, "-Xptxas=-v")
        res = subprocess.run(cmd, capture_output=True, text=True)
        if res.returncode != 0:
            raise RuntimeError(f"nvcc failed on {src}:\n{res.stderr}")
        return obj, res.stderr

    def cc(src):
        obj = os.path.join(BUILD, os.path.basename(src).replace(".c", "_c.o"))
        cmd = ["gcc", "-std=c11", "-O2", "-fPIC", "-c", os.path.join(CSRC, src), "-o", obj]
        subprocess.run(cmd, check=True)
        return obj, ""

    with ThreadPoolExecutor(max_workers=len(CU_SOURCES) + len(C_SOURCES)) as ex:
        futs = [ex.submit(cu, s) for s in CU_SOURCES] + [ex.submit(cc, s) for s in C_SOURCES]
        results = [f.result() for f in futs]
    if verbose:
        for _, err in results:
            if err:
                print(err)
    tmp = LIB + f".tmp{os.getpid()}"
    objs = [o for o, _ in results]
    subprocess.run([nvcc, *ARCH, "-shared", "-cudart", "static", "-o", tmp, *objs], check=True)
    os.replace(tmp, LIB)
    return LIB

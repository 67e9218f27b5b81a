"""Build the CUDA library csrc/liblbgb.so for sm_103a (GB300) in-tree.

Each .cu translation unit is compiled by its own nvcc process (in parallel),
then linked into one shared library against the shared CUDA runtime, so the
library and PyTorch use the same runtime instance in one process.
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
ROOT = os.path.dirname(HERE)
LIB = os.path.join(CSRC, "liblbgb.so")
SOURCES = ["lbgb_api.cu", "lbgb_step_f32.cu", "lbgb_step_f16.cu", "lbgb_step_bf16.cu", "lbgb_step_mc.cu",
           "lbgb_static.cu", "lbgb_batch.cu", "lbgb_stats.cu", "lbgb_weno.cu", "lbgb_peak.cu", "lbgb_step_pair_f16.cu",
           "lbgb_step_pair_bf16.cu", "lbgb_step_g16_f16.cu", "lbgb_step_g16_bf16.cu", "lbgb_step_pair_g16_f16.cu",
           "lbgb_step_pair_g16_bf16.cu", "lbgb_step_pair_vd_f16.cu", "lbgb_step_pair_vd_bf16.cu", "lbgb_batch_pair_vd_f16.cu",
           "lbgb_batch_pair_vd_bf16.cu", "lbgb_step_pair_pf_f16.cu", "lbgb_step_pair_pf_bf16.cu"] + [
           f"lbgb_step_{v}_{st}.cu" for v in ("vd", "fd", "fdvd") for st in ("f32", "f16", "bf16", "mc")]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found")


def _flags(verbose: bool):
    f = ARCH + ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-I", os.path.join(ROOT, "include")]
    if verbose:
        f += ["-Xptxas", "-v"]
    return f


def _deps():
    files = [os.path.join(CSRC, s) for s in SOURCES]
    files += [os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith((".cuh", ".inc"))]
    files.append(os.path.join(ROOT, "include", "lbgb.h"))
    return files


def up_to_date() -> bool:
    if not os.path.exists(LIB):
        return False
    t = os.path.getmtime(LIB)
    return all(os.path.getmtime(f) <= t for f in _deps())


def build(force: bool = False, verbose: bool = False) -> str:
    """Compile (if stale) and return the path of liblbgb.so."""
    if not force and up_to_date():
        return LIB
    cc = nvcc()
    objdir = os.path.join(CSRC, "_build")
    os.makedirs(objdir, exist_ok=True)

    def compile_one(src):
        obj = os.path.join(objdir, src.replace(".cu", ".o"))
        cmd = [cc] + _flags(verbose) + ["-c", os.path.join(CSRC, src), "-o", obj]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed for {src}:\n{r.stdout}\n{r.stderr}")
        return obj, r.stderr

    with cf.ThreadPoolExecutor(max_workers=len(SOURCES)) as ex:
        results = list(ex.map(compile_one, SOURCES))
    if verbose:
        for _, log in results:
            sys.stderr.write(log)
    objs = [o for o, _ in results]
    tmp = LIB + ".tmp"
    cmd = [cc] + ARCH + ["-shared", "-cudart", "shared", "-o", tmp] + objs + ["-lcufft"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))

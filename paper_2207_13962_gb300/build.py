"""Build the CUDA library ``libfslbm.so`` in-tree for sm_103a.

Each translation unit under ``csrc/`` is compiled by its own nvcc process (in
parallel), and every engine (storage format and lattice) is an object of its
own; the engines are compiled with ``--fmad=false`` so their arithmetic
rounds exactly as written.  The shared library links the CUDA runtime
dynamically so that it shares one runtime with PyTorch in the same process.
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
LIB = os.path.join(HERE, "libfslbm.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
# (source, object, flags): the C-ABI units, then one engine per storage
# format and lattice from fslbm_engine_inst.cu, all without multiply-add
# contraction: the FP64 engine then rounds exactly as written (bitwise the
# oracle), and in every engine a cell's arithmetic is the same in each
# kernel that inlines it (single-domain and batched runs agree bitwise);
# the hot FP32 collision writes its multiply-adds out as fused operations
ENGINES = [("f64", "StoreF64"), ("f32", "StoreF32"), ("f16s", "StoreF16S"), ("bf16s", "StoreBF16S"),
           ("f32mc", "StoreF32MC"), ("f16smc", "StoreF16SMC")]
SOURCES = [(f, f.replace(".cu", ".o"), []) for f in
           ("fslbm_api.cu", "fslbm_noalloc.cu", "fslbm_batch.cu", "fslbm_server.cu", "fslbm_front.cu")]
for _name, _store in ENGINES:
    for _q in (19, 27):
        SOURCES.append(("fslbm_engine_inst.cu", f"engine_{_name}_q{_q}.o",
                        [f"-DFSLBM_INST_NAME=ops_{_name}_q{_q}", f"-DFSLBM_INST_Q={_q}",
                         f"-DFSLBM_INST_STORE={_store}", "--fmad=false"]))


def nvcc() -> str:
    cand = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(cand):
        raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libfslbm")
    return cand


def _deps():
    files = [os.path.join(CSRC, f) for f in os.listdir(CSRC)]
    files.append(os.path.join(os.path.dirname(HERE), "include", "fslbm.h"))
    files.append(os.path.abspath(__file__))
    return files


def up_to_date() -> bool:
    if not os.path.exists(LIB):
        return False
    t = os.path.getmtime(LIB)
    return all(os.path.getmtime(f) <= t for f in _deps())


def build(force: bool = False, verbose: bool = False, extra_flags=None) -> str:
    if not force and up_to_date():
        return LIB
    os.makedirs(BUILD, exist_ok=True)
    cc = nvcc()
    # host code without floating-point contraction too: the bubble relabelling
    # divides the gas on the host in the oracle's order of operations, and an
    # Arm host compiler would otherwise fuse its multiply-adds
    common = ARCH + ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-Xcompiler", "-O2",
                     "-Xcompiler", "-ffp-contract=off", "-I", os.path.join(os.path.dirname(HERE), "include")]
    if extra_flags:
        common += list(extra_flags)

    def compile_one(item):
        src, obj, flags = item
        obj = os.path.join(BUILD, obj)
        cmd = [cc] + common + flags + ["-c", os.path.join(CSRC, src), "-o", obj]
        if verbose:
            print(" ".join(cmd), flush=True)
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed for {src}:\n{r.stdout}\n{r.stderr}")
        if verbose and r.stderr:
            print(r.stderr, flush=True)
        return obj

    with cf.ThreadPoolExecutor(max_workers=min(len(SOURCES), max(2, os.cpu_count() or 2))) as ex:
        objs = list(ex.map(compile_one, SOURCES))
    tmp = LIB + f".{os.getpid()}.tmp"
    cmd = [cc] + ARCH + ["-shared", "-cudart", "shared", "-o", tmp] + objs + [
        "-Xlinker", "-rpath,/usr/local/cuda/lib64"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    build(force="--force" in sys.argv, verbose=True,
          extra_flags=["-Xptxas", "-v"] if "--ptxas" in sys.argv else None)
    print(LIB)

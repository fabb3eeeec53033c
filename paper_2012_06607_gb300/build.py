"""Build the CUDA library libmdnewton.so in-tree for sm_103a.

Translation units (one per limb count plus the C ABI layer) are compiled in
parallel with nvcc and linked into ``paper_2012_06607_gb300/libmdnewton.so``.
Objects go to ``paper_2012_06607_gb300/_build``.
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
LIB = os.path.join(HERE, "libmdnewton.so")
ROOT = os.path.dirname(HERE)

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVFLAGS = ARCH + ["-O3", "-lineinfo", "-fmad=false", "-std=c++17", "-Xcompiler", "-fPIC", "-I" + os.path.join(ROOT, "include")]

LIMBS = [1, 2, 3, 4, 5, 8, 10]


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found")


PARTS = ("ops", "eval", "solve", "batched")


def units():
    """(source, object name, extra flags): one instantiation unit per (K, P, part)."""
    out = []
    inst = os.path.join(CSRC, "inst.cu")
    for k in LIMBS:
        for p in (1, 2):
            for i, part in enumerate(PARTS):
                if part == "batched" and k > 5:
                    continue  # the batched form covers up to five limbs
                out.append((inst, f"inst_k{k}_p{p}_{part}.o", [f"-DMDK_K={k}", f"-DMDK_P={p}", f"-DMDK_PART={i}"]))
    out.append((os.path.join(CSRC, "capi.cu"), "capi.o", []))
    out.append((os.path.join(CSRC, "noalloc.cu"), "noalloc.o", []))
    return out


def _deps():
    return [os.path.join(CSRC, f) for f in os.listdir(CSRC)] + [os.path.join(ROOT, "include", "mdnewton.h")]


def _compile(src: str, obj: str, extra):
    cmd = [nvcc(), *NVFLAGS, *extra, "-c", src, "-o", obj]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"nvcc failed for {os.path.basename(src)}:\n{r.stdout}\n{r.stderr}")
    return obj


def build(force: bool = False, verbose: bool = False, extra=()) -> str:
    os.makedirs(BUILD, exist_ok=True)
    newest_dep = max(os.path.getmtime(p) for p in _deps())
    if not force and os.path.exists(LIB) and os.path.getmtime(LIB) >= newest_dep:
        return LIB
    objs = []
    jobs = []
    todo = units()
    # longest units first (more limbs, complex) so the pool ends evenly
    todo.sort(key=lambda u: -sum(int(f.split("=")[1]) for f in u[2] if f.startswith(("-DMDK_K", "-DMDK_P"))) if u[2] else 0)
    with cf.ThreadPoolExecutor(max_workers=max(2, os.cpu_count() or 4)) as ex:
        for src, oname, flags in todo:
            obj = os.path.join(BUILD, oname)
            objs.append(obj)
            jobs.append(ex.submit(_compile, src, obj, list(extra) + flags))
        for j in jobs:
            j.result()
    tmp = LIB + f".tmp{os.getpid()}"
    cmd = [nvcc(), *ARCH, "-shared", "-o", tmp, *objs, "-lcudart"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, LIB)
    if verbose:
        print("built", LIB)
    return LIB


if __name__ == "__main__":
    build(force="--force" in sys.argv, verbose=True)

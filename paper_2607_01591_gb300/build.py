"""Build the CUDA library (sm_103a) in-tree: paper_2607_01591_gb300/_lib/libmoc_gb300.so.

nvcc compiles the kernels and the C ABI; g++ compiles the host geometry; the two translation
units build in parallel. CUDA runtime is linked statically.
"""
from __future__ import annotations

import os
import shutil
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
INC = os.path.join(ROOT, "include")
OUT_DIR = os.path.join(HERE, "_lib")
BUILD_DIR = os.path.join(HERE, "_build")
LIB = os.path.join(OUT_DIR, "libmoc_gb300.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
SOURCES = ["moc_api.cu", "moc_mlp.cu", "moc_track.cu", "moc_probe.cu", "moc_geom.cpp"]
HEADERS = ["moc_kernels.cuh", "moc_cmfd.cuh", "moc_dg.cuh", "moc_aniso.cuh", "moc_tc.cuh", "moc_geom.h", "moc_walk.h",
           "moc_track.h", "exp_f32_coef.h"]
# the device walk must round every double multiply and add separately, like the host build
NO_FMA = {"moc_track.cu"}


def _nvcc() -> str:
    for cand in (shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build the library")


def _stale() -> bool:
    if not os.path.exists(LIB):
        return True
    t = os.path.getmtime(LIB)
    deps = [os.path.join(CSRC, f) for f in SOURCES + HEADERS] + [os.path.join(INC, h) for h in os.listdir(INC)]
    return any(os.path.getmtime(d) > t for d in deps)


def build(force: bool = False, verbose: bool = False) -> str:
    if not force and not _stale():
        return LIB
    os.makedirs(OUT_DIR, exist_ok=True)
    os.makedirs(BUILD_DIR, exist_ok=True)
    nvcc = _nvcc()
    objs = []
    cmds = []
    for src in SOURCES:
        obj = os.path.join(BUILD_DIR, src.replace(".", "_") + ".o")
        objs.append(obj)
        if src.endswith(".cu"):
            cmd = [nvcc, *ARCH, "-O3", "-lineinfo", "-std=c++17", "-I", INC, "-I", CSRC, "-Xcompiler",
                   "-fPIC,-fopenmp,-ffp-contract=off", *(["--fmad=false"] if src in NO_FMA else []),
                   "-c", os.path.join(CSRC, src), "-o", obj]
        else:
            cmd = ["g++", "-O2", "-ffp-contract=off", "-std=c++17", "-fPIC", "-fopenmp", "-I", INC, "-I", CSRC, "-c", os.path.join(CSRC, src),
                   "-o", obj]
        cmds.append(cmd)

    def run(cmd):
        if verbose:
            print(" ".join(cmd), file=sys.stderr)
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("build failed:\n" + " ".join(cmd) + "\n" + r.stdout + r.stderr)
        return r

    with ThreadPoolExecutor(len(cmds)) as ex:
        list(ex.map(run, cmds))
    tmp = LIB + f".{os.getpid()}.tmp"
    run([nvcc, *ARCH, "-shared", "-o", tmp, *objs, "-Xcompiler", "-fPIC", "-lgomp"])
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True))

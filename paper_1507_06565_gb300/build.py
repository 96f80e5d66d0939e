"""Build liblbm.so (sm_103a) in-tree with nvcc.

Translation units are compiled in parallel into ``_build/`` and linked into
``_build/liblbm.so``.  Host code is compiled with -ffp-contract=off so that the
geometry arithmetic rounds identically on x86-64 and AArch64 hosts.
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
OUT = os.path.join(HERE, "_build")
LIB = os.path.join(OUT, "liblbm.so")
INCLUDE = os.path.join(ROOT, "include")

SOURCES = ["lbm_geometry.cpp", "lbm_api.cpp", "lbm_checkpoint.cpp", "lbm_build.cu", "lbm_step.cu", "lbm_post.cu", "lbm_static_scratch.cu",
           "lbm_sdf.cu", "unet.cu", "glbm.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def _nvcc() -> str:
    cand = os.path.join(os.environ.get("CUDA_HOME", "/usr/local/cuda"), "bin", "nvcc")
    return cand if os.path.exists(cand) else (shutil.which("nvcc") or "nvcc")


def _flags(src: str, openmp: bool) -> list[str]:
    host = ["-fPIC", "-ffp-contract=off", "-O3"] + (["-fopenmp"] if openmp else [])
    f = ["-std=c++17", "-O3", "-lineinfo", "-I", INCLUDE, "-I", CSRC, "-Xcompiler", ",".join(host)]
    if src.endswith(".cu"):
        f += ARCH + ["-Xptxas", "-v"] if os.environ.get("LBM_PTXAS_VERBOSE") else ARCH
    return f


def _openmp_ok() -> bool:
    probe = os.path.join(OUT, "omp_probe.c")
    with open(probe, "w") as fh:
        fh.write("#include <omp.h>\nint main(void){return omp_get_max_threads() > 0 ? 0 : 1;}\n")
    r = subprocess.run(["gcc", "-fopenmp", probe, "-o", probe + ".bin"], capture_output=True)
    return r.returncode == 0


def _stale(objs: list[str]) -> bool:
    if not os.path.exists(LIB):
        return True
    t = os.path.getmtime(LIB)
    deps = [os.path.join(CSRC, f) for f in os.listdir(CSRC)] + [os.path.join(INCLUDE, f) for f in os.listdir(INCLUDE)]
    deps.append(__file__)
    return any(os.path.getmtime(d) > t for d in deps)


def build(force: bool = False, verbose: bool = False) -> str:
    os.makedirs(OUT, exist_ok=True)
    objs = [os.path.join(OUT, s + ".o") for s in SOURCES]
    if not force and not _stale(objs):
        return LIB
    nvcc = _nvcc()
    openmp = _openmp_ok()

    def compile_one(src: str) -> tuple[str, str]:
        obj = os.path.join(OUT, src + ".o")
        cmd = [nvcc, "-c", os.path.join(CSRC, src), "-o", obj] + _flags(src, openmp)
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed for {src}:\n{' '.join(cmd)}\n{r.stdout}\n{r.stderr}")
        return src, r.stdout + r.stderr

    with cf.ThreadPoolExecutor(max_workers=len(SOURCES)) as ex:
        for src, log in ex.map(compile_one, SOURCES):
            if verbose and log.strip():
                print(f"[{src}]\n{log}", file=sys.stderr)
    tmp = LIB + f".tmp{os.getpid()}"
    cmd = [nvcc, "-shared", "-o", tmp] + objs + ARCH + (["-Xcompiler", "-fopenmp", "-lgomp"] if openmp else [])
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{' '.join(cmd)}\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True))

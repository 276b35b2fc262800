"""In-tree build of the CUDA sampler library (sm_103a) and the input generator.

``build()`` compiles each translation unit of ``csrc/`` with nvcc in parallel
and links ``_build/libpimc.so``, and the checked variant
``_build/libpimc_check.so`` (the sweep kernels compiled with PIMC_CHECK: site
visit counters and index checks, for tests); nothing is installed outside the
tree.
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(BUILD, "libpimc.so")
LIB_CHECK = os.path.join(BUILD, "libpimc_check.so")
CHECKED_SOURCES = ["sweep.cu"]  # the translation units that differ under PIMC_CHECK
ROOT = os.path.dirname(HERE)

CU_SOURCES = ["sweep.cu", "ops.cu", "runtime.cu", "noalloc.cu", "hmc.cu"]
HEADERS = ["device.cuh", "internal.h", "stats.cuh", "scheme.cuh", "reduce.cuh"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def _nvcc() -> str:
    cand = os.environ.get("CUDA_HOME", "/usr/local/cuda")
    p = os.path.join(cand, "bin", "nvcc")
    return p if os.path.exists(p) else (shutil.which("nvcc") or "nvcc")


def _flags():
    return ARCH + ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-Xcompiler", "-O2",
                   "--expt-relaxed-constexpr", "-I", os.path.join(ROOT, "include")]


def _stale(obj: str, deps) -> bool:
    if not os.path.exists(obj):
        return True
    t = os.path.getmtime(obj)
    return any(os.path.getmtime(d) > t for d in deps)


def build(force: bool = False, verbose: bool = False) -> str:
    os.makedirs(BUILD, exist_ok=True)
    nvcc = _nvcc()
    hdrs = [os.path.join(CSRC, h) for h in HEADERS] + [os.path.join(ROOT, "include", "pimc.h")]
    jobs = []
    objs = []
    objs_check = []
    for src in CU_SOURCES:
        sp = os.path.join(CSRC, src)
        obj = os.path.join(BUILD, src.replace(".cu", ".o"))
        objs.append(obj)
        if force or _stale(obj, [sp] + hdrs):
            cmd = [nvcc] + _flags() + ["-c", sp, "-o", obj]
            if verbose:
                cmd += ["-Xptxas", "-v"]
            jobs.append(cmd)
        if src in CHECKED_SOURCES:
            objc = os.path.join(BUILD, src.replace(".cu", "_check.o"))
            objs_check.append(objc)
            if force or _stale(objc, [sp] + hdrs):
                jobs.append([nvcc] + _flags() + ["-DPIMC_CHECK", "-c", sp, "-o", objc])
        else:
            objs_check.append(obj)

    def run(cmd):
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("nvcc failed:\n" + " ".join(cmd) + "\n" + r.stdout + r.stderr)
        return r.stdout + r.stderr

    logs = []
    with cf.ThreadPoolExecutor(max_workers=max(1, len(jobs))) as ex:
        for out in ex.map(run, jobs):
            logs.append(out)
    if verbose:
        for l in logs:
            print(l)
    for lib, ob in ((LIB, objs), (LIB_CHECK, objs_check)):
        if force or jobs or not os.path.exists(lib):
            tmp = lib + f".{os.getpid()}.tmp"
            run([nvcc] + ARCH + ["-shared", "-o", tmp] + ob + ["-lcudart"])
            os.replace(tmp, lib)
    return LIB


if __name__ == "__main__":
    import sys
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))

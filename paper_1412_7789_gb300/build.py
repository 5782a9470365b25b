"""Compile the library (CUDA kernels + C++ host code) into ``_build/libpfac.so``.

Targets sm_103a only.  Translation units are compiled in parallel and linked
with nvcc (CUDA runtime linked statically, so loading the library needs no GPU).
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
BUILD_DIR = os.path.join(HERE, "_build")
LIB_PATH = os.path.join(BUILD_DIR, "libpfac.so")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
SOURCES = ["builder.cpp", "api.cpp", "serve.cpp", "kernels.cu", "jump8.cu", "filter.cu", "filter8.cu", "noalloc.cu",
           "batch.cu", "compact.cu", "full.cu", "filter_help.cu", "filter_multi_dense.cu", "filter_multi_slots.cu", "survivors.cu",
           "filter_direct.cu"]
HEADERS = ["pfac_internal.h", "pfac_device.cuh", "filter_kernel.cuh"]


def _nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found")


def _compile_cmd(src: str, obj: str) -> list[str]:
    common = ["-O3", "-std=c++17", "-I", INCLUDE, "-I", CSRC, "-Xcompiler", "-fPIC", "-Xcompiler", "-pthread"]
    if src.endswith(".cu"):
        return [_nvcc(), *ARCH, "-lineinfo", *common, "-c", src, "-o", obj]
    return [_nvcc(), *common, "-x", "c++", "-c", src, "-o", obj]


def _stale(target: str, deps: list[str]) -> bool:
    if not os.path.exists(target):
        return True
    t = os.path.getmtime(target)
    return any(os.path.getmtime(d) > t for d in deps)


def build(force: bool = False, verbose: bool = False) -> str:
    os.makedirs(BUILD_DIR, exist_ok=True)
    headers = [os.path.join(CSRC, h) for h in HEADERS] + [os.path.join(INCLUDE, "ac.h")]
    jobs = []
    objs = []
    for s in SOURCES:
        src = os.path.join(CSRC, s)
        obj = os.path.join(BUILD_DIR, s + ".o")
        objs.append(obj)
        if force or _stale(obj, [src, *headers, __file__]):
            jobs.append(_compile_cmd(src, obj))

    def run(cmd):
        if verbose:
            print(" ".join(cmd), flush=True)
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("compile failed: %s\n%s%s" % (" ".join(cmd), r.stdout, r.stderr))
        return r.stderr

    with ThreadPoolExecutor(max_workers=max(1, len(jobs))) as ex:
        for err in ex.map(run, jobs):
            if verbose and err:
                print(err)
    if force or jobs or _stale(LIB_PATH, objs):
        tmp = LIB_PATH + ".tmp%d" % os.getpid()
        run([_nvcc(), *ARCH, "-shared", "-o", tmp, *objs, "-cudart", "static", "-lpthread"])
        os.replace(tmp, LIB_PATH)
    return LIB_PATH


if __name__ == "__main__":
    import sys

    print(build(force="--force" in sys.argv, verbose=True))

"""Build libfsmp.so (the C-ABI library) in-tree with nvcc for sm_103a.

Translation units are compiled in parallel and linked with the shared CUDA runtime (so the
library and PyTorch share one runtime and one primary context per device).
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(os.path.dirname(HERE), "include")
OUT_DIR = os.path.join(HERE, "_build")
LIB = os.path.join(OUT_DIR, "libfsmp.so")
SOURCES = ["fsmp_tables.cu", "fsmp_chain.cu", "fsmp_pe.cu", "fsmp_pe_mix.cu", "fsmp_lucy.cu", "fsmp_runtime.cu",
           "fsmp_probe.cu", "fsmp_rhat.cu",
           "fsmp_noalloc.cu"]
HEADERS = [os.path.join(CSRC, "fsmp_internal.h"), os.path.join(CSRC, "fsmp_pe_kernel.cuh"),
           os.path.join(INCLUDE, "fsmp.h")]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-Xcompiler", "-Wall"]


def _nvcc():
    cuda = os.environ.get("CUDA_HOME", "/usr/local/cuda")
    p = os.path.join(cuda, "bin", "nvcc")
    return p if os.path.exists(p) else (shutil.which("nvcc") or "nvcc"), cuda


def _stale(target, deps):
    if not os.path.exists(target):
        return True
    t = os.path.getmtime(target)
    return any(os.path.getmtime(d) > t for d in deps)


def build(force: bool = False, verbose: bool = False, ptxas_info: bool = False) -> str:
    """Compile and link libfsmp.so if any source changed; returns its path."""
    nvcc, cuda = _nvcc()
    os.makedirs(OUT_DIR, exist_ok=True)
    objs, jobs = [], []
    for src in SOURCES:
        sp = os.path.join(CSRC, src)
        obj = os.path.join(OUT_DIR, src.replace(".cu", ".o"))
        objs.append(obj)
        if force or ptxas_info or _stale(obj, [sp] + HEADERS):
            cmd = [nvcc, *ARCH, *FLAGS, "-c", sp, "-o", obj]
            if ptxas_info:
                cmd.insert(1, "-Xptxas=-v")
            jobs.append(cmd)

    def run(cmd):
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("nvcc failed:\n%s\n%s" % (" ".join(cmd), r.stderr))
        return r.stderr

    with cf.ThreadPoolExecutor(max_workers=len(SOURCES)) as ex:
        for log in ex.map(run, jobs):
            if verbose and log:
                print(log)
    if force or jobs or _stale(LIB, objs):
        tmp = LIB + ".tmp.%d" % os.getpid()
        run([nvcc, *ARCH, "-shared", "-o", tmp, *objs, "-cudart", "shared",
             "-Xlinker", "-rpath," + os.path.join(cuda, "lib64")])
        os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    import sys
    print(build(force="--force" in sys.argv, verbose=True, ptxas_info="--ptxas" in sys.argv))

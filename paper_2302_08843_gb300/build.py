"""Build libmm.so in-tree with nvcc for sm_103a (no cmake, parallel units).

    python -m paper_2302_08843_gb300.build

Objects go to paper_2302_08843_gb300/_build/, the library to
paper_2302_08843_gb300/libmm.so (both git-ignored).  Host code is compiled
with -ffp-contract=off so that x86-64 and aarch64 builds round alike.
"""
import concurrent.futures
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
SRC = os.path.join(HERE, "csrc")
OUT = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libmm.so")
NVCC = os.environ.get("NVCC", "/usr/local/cuda/bin/nvcc")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
CU_UNITS = ["mm_api.cu", "demag_passes.cu", "demag_rt.cu", "llg_kernels.cu", "noalloc.cu", "adjoint.cu", "batch.cu",
            "diag.cu"]
CPP_UNITS = ["tensor_host.cpp"]


def _nvcc_flags():
    return (["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC,-fopenmp,-ffp-contract=off",
             "-I" + SRC, "-I" + os.path.join(ROOT, "include")] + ARCH)


def _run(cmd):
    r = subprocess.run(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT, text=True)
    if r.returncode != 0:
        raise RuntimeError("build step failed: %s\n%s" % (" ".join(cmd), r.stdout))
    return r.stdout


def _stale(obj, deps):
    if not os.path.exists(obj):
        return True
    t = os.path.getmtime(obj)
    return any(os.path.getmtime(d) > t for d in deps)


def build(verbose=False, force=False, extra_flags=()):
    os.makedirs(OUT, exist_ok=True)
    headers = [os.path.join(SRC, f) for f in os.listdir(SRC) if f.endswith((".h", ".cuh"))]
    headers.append(os.path.join(ROOT, "include", "mm.h"))
    jobs = []
    objs = []
    for u in CU_UNITS:
        src = os.path.join(SRC, u)
        obj = os.path.join(OUT, u + ".o")
        objs.append(obj)
        if force or _stale(obj, [src] + headers):
            jobs.append([NVCC, "-c", src, "-o", obj] + _nvcc_flags() + list(extra_flags))
    for u in CPP_UNITS:
        src = os.path.join(SRC, u)
        obj = os.path.join(OUT, u + ".o")
        objs.append(obj)
        if force or _stale(obj, [src] + headers):
            jobs.append(["g++", "-c", src, "-o", obj, "-O3", "-std=c++17", "-fPIC", "-fopenmp",
                         "-ffp-contract=off", "-I" + SRC, "-I" + os.path.join(ROOT, "include")])
    with concurrent.futures.ThreadPoolExecutor(max_workers=max(1, min(8, os.cpu_count() or 1))) as ex:
        outs = list(ex.map(_run, jobs))
    if verbose:
        for o in outs:
            if o.strip():
                print(o)
    if force or jobs or not os.path.exists(LIB):
        _run([NVCC, "-shared", "-o", LIB] + objs + ARCH + ["-Xcompiler", "-fopenmp", "-lgomp"])
    return LIB


if __name__ == "__main__":
    print(build(verbose=True, force="--force" in sys.argv))

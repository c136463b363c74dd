"""Build the CUDA library libzolo_csd.so in-tree with nvcc (sm_103a).

Each translation unit is compiled in parallel, then linked into one shared
library next to this file.  Re-running only recompiles stale objects.
"""
import concurrent.futures as cf
import os
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(os.path.dirname(HERE), "include")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libzolo_csd.so")
SOURCES = ["blas.cu", "fact.cu", "linalg.cu", "solver.cu", "profile.cu", "noalloc.cu", "tc_gemm.cu", "peak.cu", "grad.cu", "svd.cu", "eig.cu", "batch.cu", "coef.cpp"]
HEADERS = ["common.cuh", "ops.h", "linalg.h", "profile.h", "solver.h", "tc_gemm.h"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ["-O3", "-lineinfo", "-std=c++17", "--extended-lambda", "-Xcompiler", "-fPIC", "-I", INCLUDE]


def _nvcc():
    for c in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", "nvcc"):
        if c and (os.path.sep not in c or os.path.exists(c)):
            return c
    return "nvcc"


def _dep_mtime():
    files = [os.path.join(CSRC, h) for h in HEADERS] + [os.path.join(INCLUDE, "zolo_csd.h")]
    return max(os.path.getmtime(f) for f in files)


def _obj(src):
    return os.path.join(BUILD, src + ".o")


def _compile(src):
    out = _obj(src)
    cmd = [_nvcc()] + ARCH + NVCC_FLAGS + ["-c", os.path.join(CSRC, src), "-o", out + ".tmp"]
    subprocess.run(cmd, check=True)
    os.replace(out + ".tmp", out)
    return out


def build(force: bool = False, verbose: bool = False) -> str:
    os.makedirs(BUILD, exist_ok=True)
    dep = _dep_mtime()
    todo = []
    for s in SOURCES:
        o = _obj(s)
        if force or not os.path.exists(o) or os.path.getmtime(o) < max(dep, os.path.getmtime(os.path.join(CSRC, s))):
            todo.append(s)
    if todo:
        with cf.ThreadPoolExecutor(max_workers=min(len(todo), os.cpu_count() or 4)) as ex:
            list(ex.map(_compile, todo))
    objs = [_obj(s) for s in SOURCES]
    if todo or force or not os.path.exists(LIB) or os.path.getmtime(LIB) < max(os.path.getmtime(o) for o in objs):
        tmp = LIB + f".tmp{os.getpid()}"
        cmd = [_nvcc()] + ARCH + ["-shared", "-o", tmp] + objs + ["-cudart", "static"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, LIB)
    if verbose:
        print(LIB)
    return LIB


if __name__ == "__main__":
    build(force=True, verbose=True)

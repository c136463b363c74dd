"""Oracle (test infrastructure only; never on the product path).

Compiles the oracle's plain-C Jacobi sub-solvers (jacobi.c) into
``oracle/liboracle_jacobi.so`` with gcc and OpenMP.  Called by the
package build step and, on demand, by ``oracle.jacobi`` when the shared
library is missing or older than its sources.
"""
import os
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = [os.path.join(HERE, "jacobi.c"), os.path.join(HERE, "jacobi_impl.h")]
LIB = os.path.join(HERE, "liboracle_jacobi.so")


def stale() -> bool:
    if not os.path.exists(LIB):
        return True
    t = os.path.getmtime(LIB)
    return any(os.path.getmtime(s) > t for s in SRC)


def build(force: bool = False) -> str:
    if force or stale():
        tmp = LIB + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-std=c99", "-fopenmp", "-fPIC", "-shared", "-ffp-contract=off",
               "-o", tmp, os.path.join(HERE, "jacobi.c"), "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force=True))

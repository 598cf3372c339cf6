"""Compile the plain-C oracle into oracle/_build/liboracle.so.

Test infrastructure: the oracle is the CPU reference the tests, the smoke check
and the benchmark's CPU baseline compare against.  It is built with plain gcc,
-O2, no fast-math and no floating-point contraction, so an x86 build and an Arm
build return the same bits.
"""
import os
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "pcdm_oracle.c")              # LASSO, the samplers
SRC_GLM = os.path.join(HERE, "pcdm_oracle_glm.c")      # SVM dual and logistic regression
SRC_THREADS = os.path.join(HERE, "pcdm_oracle_threads.c")   # threaded timing mode of the LASSO run
SOURCES = (SRC, SRC_GLM, SRC_THREADS)
OUT_DIR = os.path.join(HERE, "_build")
OUT = os.path.join(OUT_DIR, "liboracle.so")


def build(force: bool = False) -> str:
    """Build (if stale) and return the path of the shared library."""
    os.makedirs(OUT_DIR, exist_ok=True)
    if not force and os.path.exists(OUT) and all(os.path.getmtime(OUT) >= os.path.getmtime(s) for s in SOURCES):
        return OUT
    tmp = OUT + ".tmp%d" % os.getpid()
    cmd = ["gcc", "-std=c11", "-O2", "-fPIC", "-shared", "-ffp-contract=off", "-fno-fast-math", "-pthread",
           "-Wall", "-Wextra", *SOURCES, "-o", tmp, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, OUT)
    return OUT


if __name__ == "__main__":
    print(build(force=True))

"""Compile the FP64 CPU oracle (oracle.c) into oracle/_build/liboracle.so.

Test infrastructure only: the product library never links or loads it.
The oracle is built with -ffp-contract=off so its FP32 key arithmetic is two
separately rounded IEEE operations, like the GPU kernel's.
"""
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "oracle.c")
OUT_DIR = os.path.join(HERE, "_build")
LIB = os.path.join(OUT_DIR, "liboracle.so")


def compile_to(src, out, openmp=True):
    """Compile one oracle source file into the shared library `out`.
    Returns (ok, compiler messages)."""
    tmp = out + ".tmp.%d" % os.getpid()
    cmd = ["gcc", "-O2", "-std=gnu11", "-fPIC", "-shared", "-ffp-contract=off",
           "-fno-fast-math", "-Wall", src, "-o", tmp, "-lm"]
    if openmp:
        cmd.insert(1, "-fopenmp")
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        return False, r.stderr
    os.replace(tmp, out)
    return True, ""


def _compile(openmp):
    os.makedirs(OUT_DIR, exist_ok=True)
    return compile_to(SRC, LIB, openmp)


def build(force=False):
    """Build liboracle.so if it is missing or older than its source.
    The environment variable ORACLE_LIB names a prebuilt library to use
    instead (the mutation check of the pins loads planted-mistake copies)."""
    if os.environ.get("ORACLE_LIB"):
        return os.environ["ORACLE_LIB"]
    if (not force and os.path.exists(LIB)
            and os.path.getmtime(LIB) >= os.path.getmtime(SRC)):
        return LIB
    ok, err = _compile(openmp=True)
    if not ok:
        ok, err2 = _compile(openmp=False)
        if not ok:
            raise RuntimeError("oracle build failed:\n" + err + "\n" + err2)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv))

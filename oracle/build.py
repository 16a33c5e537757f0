"""Build step for the CPU oracle (test infrastructure only).

Compiles ``oracle.cpp`` (which includes ``edge_tree.h`` and ``nee_edge.h``) into ``oracle/_build/liboracle.so`` with
``-ffp-contract=off`` so every FP32 operation on the decision path is one
IEEE rounding, as the oracle's header requires.
"""
import os
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "oracle.cpp")
DEPS = [SRC, os.path.join(HERE, "edge_tree.h"), os.path.join(HERE, "nee_edge.h")]
OUT_DIR = os.path.join(HERE, "_build")
LIB = os.path.join(OUT_DIR, "liboracle.so")


def build(force: bool = False) -> str:
    """Compile the oracle if the library is missing or older than its source."""
    os.makedirs(OUT_DIR, exist_ok=True)
    if not force and os.path.exists(LIB) and os.path.getmtime(LIB) >= max(os.path.getmtime(f) for f in DEPS):
        return LIB
    tmp = LIB + ".tmp%d" % os.getpid()
    cmd = ["g++", "-O2", "-std=c++17", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared",
           "-pthread", SRC, "-o", tmp]
    subprocess.run(cmd, check=True)
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force=True))

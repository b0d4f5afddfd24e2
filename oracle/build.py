"""Build the FP64 CPU oracle (test infrastructure only) into oracle/liborc.so.

Plain g++ with fused multiply-add contraction disabled, so the oracle evaluates
every expression in source order on x86-64 and aarch64 alike; OpenMP for the
optional multi-threaded particle loops (orc_set_threads), which give the same bits.
"""
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
SOURCES = ["orc_contact.cpp", "orc_fluid.cpp", "orc_neighbors.cpp", "orc_step.cpp",
           "orc_average.cpp", "orc_cnn.cpp"]
LIB = os.path.join(HERE, "liborc.so")


def build(force: bool = False) -> str:
    srcs = [os.path.join(HERE, s) for s in SOURCES]
    hdrs = [os.path.join(HERE, h) for h in ("orc.h", "orc_internal.h")]
    if not force and os.path.exists(LIB):
        newest = max(os.path.getmtime(f) for f in srcs + hdrs)
        if os.path.getmtime(LIB) >= newest:
            return LIB
    cmd = ["g++", "-O2", "-std=c++17", "-fPIC", "-shared", "-ffp-contract=off",
           "-fno-fast-math", "-fopenmp", "-o", LIB + ".tmp"] + srcs
    subprocess.run(cmd, check=True)
    os.replace(LIB + ".tmp", LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv))

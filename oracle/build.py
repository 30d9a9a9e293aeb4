"""Builds the oracle shared library (plain C++, host compiler only).

The oracle is test infrastructure: only tests/, __graft_entry__.smoke() and the
CPU-baseline legs of bench.py load it.
"""
import os
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
SOURCES = ["exact.cpp", "philox.cpp", "delaunay.cpp", "spv.cpp", "avm.cpp", "adjoint.cpp"]
LIB = os.path.join(HERE, "libcgo.so")


def build(force: bool = False) -> str:
    srcs = [os.path.join(HERE, s) for s in SOURCES if os.path.exists(os.path.join(HERE, s))]
    # every header of the oracle (internal.h, spv_core.h, ...) is a dependency
    hdrs = sorted(os.path.join(HERE, h) for h in os.listdir(HERE) if h.endswith(".h"))
    deps = srcs + hdrs
    if not force and os.path.exists(LIB):
        t = os.path.getmtime(LIB)
        if all(os.path.getmtime(d) <= t for d in deps):
            return LIB
    # -ffp-contract=off: no fused multiply-add contraction, so the oracle rounds
    # identically on x86-64 and aarch64.
    cmd = ["g++", "-O2", "-std=c++17", "-fPIC", "-shared", "-ffp-contract=off",
           "-o", LIB + ".tmp"] + srcs
    subprocess.run(cmd, check=True)
    os.replace(LIB + ".tmp", LIB)
    return LIB


if __name__ == "__main__":
    print(build(force=True))

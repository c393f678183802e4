"""Build the FP64 CPU oracle (oracle/liboracle.so) with the host C++ compiler.

Test infrastructure: the oracle is what the CUDA path is checked against and
is never part of the product path.
"""
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
SOURCES = ["philox.cpp", "vegas.cpp", "phasespace.cpp", "pdf.cpp", "pdfset.cpp", "unweight.cpp", "channels.cpp", "matrix_elements.cpp",
           "integrand.cpp", "opcount.cpp"]
LIB = os.path.join(HERE, "liboracle.so")


def _stale():
    if not os.path.exists(LIB):
        return True
    t = os.path.getmtime(LIB)
    src = os.path.join(HERE, "src")
    return any(os.path.getmtime(os.path.join(src, f)) > t for f in os.listdir(src))


def build(force=False):
    if not force and not _stale():
        return LIB
    srcs = [os.path.join(HERE, "src", s) for s in SOURCES]
    cmd = ["g++", "-std=c++17", "-O2", "-fPIC", "-shared", "-fcx-fortran-rules", "-pthread",
           "-o", LIB] + srcs
    subprocess.run(cmd, check=True)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv))

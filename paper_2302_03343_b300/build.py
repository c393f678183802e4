"""Build libmcint.so (the CUDA library behind include/mcint.h) for sm_103a.

The library is built in-tree with nvcc: one shared object holding the fused
integrand kernel, the reduction and refinement kernels, the PDF kernel and the
C ABI.  The CUDA runtime is linked statically so the library needs only the
driver at run time.
"""
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
LIB = os.path.join(HERE, "libmcint.so")
SOURCES = ["kernels.cu", "api.cu", "noalloc.cu", "batch.cu", "tc_gemm.cu", "flow.cu", "pdfset.cu", "unweight.cu",
           "lhe.cu", "peak.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def nvcc():
    cand = os.path.join(os.environ.get("CUDA_HOME", "/usr/local/cuda"), "bin", "nvcc")
    return cand if os.path.exists(cand) else "nvcc"


def _stale(target, deps):
    if not os.path.exists(target):
        return True
    t = os.path.getmtime(target)
    return any(os.path.getmtime(d) > t for d in deps)


def build(force=False, verbose=False, extra=()):
    headers = [os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith((".cuh", ".h"))]
    headers.append(os.path.join(ROOT, "include", "mcint.h"))
    srcs = [os.path.join(CSRC, f) for f in SOURCES]
    if not force and not _stale(LIB, headers + srcs):
        return LIB
    objs = []
    for src in srcs:
        obj = os.path.splitext(src)[0] + ".o"
        # an object is rebuilt when its source or any header changed
        if force or extra or verbose or _stale(obj, headers + [src]):
            cmd = [nvcc(), *ARCH, "-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-I",
                   os.path.join(ROOT, "include"), "-c", src, "-o", obj, *extra]
            if verbose:
                cmd.insert(1, "-Xptxas=-v")
            subprocess.run(cmd, check=True)
        objs.append(obj)
    subprocess.run([nvcc(), *ARCH, "-shared", "-cudart", "static", "-o", LIB, *objs], check=True)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))

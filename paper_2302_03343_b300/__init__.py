"""B300-native per-event Monte Carlo evaluation of LO collider cross sections.

The compute path lives in the CUDA library libmcint.so (C ABI declared in
include/mcint.h); `paper_2302_03343_b300.mcint` is its thin ctypes binding.
"""

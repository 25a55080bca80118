"""GB300 (sm_103a) lattice Boltzmann-BGK library for high-frequency oscillating gas flows.

The compute path is liblbm.so (hand-written CUDA, include/lbm.h); ``lbm`` is its ctypes binding,
``build`` compiles it in-tree, and ``inputs`` holds the seeded workload generators.
"""
from .builder import build  # noqa: F401

"""GB300-native fluctuating D2Q9 lattice-Boltzmann hot path (Kaehler & Wagner,
arXiv:1204.6734): a CUDA library for sm_103a with a C ABI (include/flb.h) and a
thin ctypes binding (``flb``). Importing the package does not load the CUDA
library; ``flb.load()`` does, and raises if it is missing."""

__all__ = ["flb", "inputs", "build"]

"""B300-native nonbonded forces, MD and HMC (arXiv 2503.20541 hot path).

The compute path is the CUDA library ``libnbcore.so`` (sm_103a kernels behind a
C ABI, declared in include/nbcore.h); ``paper_2503_20541_b300.nbcore`` is its
thin ctypes binding.  Importing this package does not load the library; the
first call that needs it does, and raises if it is missing.
"""
__all__ = ["nbcore", "workloads"]

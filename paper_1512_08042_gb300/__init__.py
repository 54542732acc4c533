"""GB300-native hot path of the hybrid DSMC-LBM kinetic mapping method (arXiv 1512.08042).

The compute path is a CUDA library (`libdsmclbm.so`, C ABI declared in include/dsmclbm.h)
built for sm_103a; `binding` is a thin ctypes layer over it that only marshals arguments and
allocates device memory through PyTorch. Importing this package does not load the library;
the first use of `binding` does, and raises if it is missing.
"""
__all__ = ["binding", "workloads"]

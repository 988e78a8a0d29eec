"""fsmc: finite-state-machine multi-chain MCMC on one B300 GPU (arXiv 2503.17405).

The sampling path is CUDA (libfsmc.so, C ABI in include/fsmc.h); this package is its
thin Python binding (``fsmc``), the library build step (``build``) and the seeded
synthetic workload generators (``workloads``).
"""
from . import workloads  # noqa: F401

__all__ = ["workloads", "fsmc", "build"]

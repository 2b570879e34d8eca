"""GB300-native recursive-regularized BGK lattice Boltzmann (arXiv:1505.06900).

The compute path is the CUDA library ``liblbrr.so`` built from ``csrc/`` for
sm_103a; ``binding`` is a thin ctypes layer over its C ABI (``include/lbrr.h``).
Importing this package does not load the library; ``binding.load()`` does, and
raises if it is missing.
"""
__all__ = ["binding", "workloads"]

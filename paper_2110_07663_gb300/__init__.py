"""GB300-native spectral-element Poisson solver: matrix-free operator, p-multigrid with
Chebyshev-accelerated Schwarz/Jacobi smoothing, flexible Krylov solvers (libse.so, sm_103a).

The compute path is the CUDA library; ``se`` is its ctypes binding.  Importing the package
without a built library raises ImportError (there is no CPU fallback).
"""
from . import se  # noqa: F401

__all__ = ["se"]

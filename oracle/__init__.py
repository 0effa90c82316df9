"""FP64 CPU oracle of the spectral-element Poisson hot path.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s
cpu_baseline / reference arm may import or run anything in this package.  It shares no code with
the CUDA library (``paper_2110_07663_gb300``); the two meet only in the seeded inputs of
``workloads.py``.

Every function cites the passage of the paper (Phillips, Kerkemeier, Fischer, "Tuning Spectral
Element Preconditioners for Parallel Scalability on GPUs", arXiv 2110.07663) that it follows.
Pins (tests/test_oracle_*.py) tie each function to something other than itself: closed forms,
brute-force quadrature, dense inverses, dense eigenvalues, the Chebyshev closed form.
Parity unpinned against the paper's own printed numbers: the paper prints no iteration counts or
timings for these synthetic meshes (its Kershaw map and Navier-Stokes meshes are not available).
"""
from .se_oracle import *  # noqa: F401,F403

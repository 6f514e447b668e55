"""GB300-native (sm_103a) LOBPCG for the 7-point 3-D Dirichlet Laplacian.

The block LOBPCG iteration of Knyazev, Argentati, Lashuk and Ovtchinnikov (BLOPEX, Section 2.2,
with the soft locking of Section 2.3) preconditioned by a geometric-multigrid V-cycle, with every
step in hand-written CUDA kernels behind the C ABI of include/lobpcg_gb300.h.

  capi    -- ctypes binding with the C entry-point names (marshalling only)
  solver  -- ``Solver``: a handle with torch-provided device memory and stream
  build   -- compiles liblobpcg_gb300.so in-tree with nvcc for sm_103a
"""
from . import capi  # noqa: F401


def Solver(*args, **kwargs):
    from .solver import Solver as _S
    return _S(*args, **kwargs)

"""GB300-native p-multigrid-preconditioned Krylov pressure-Poisson solver for the
sigma-mapped nodal spectral element wave model of arXiv 2411.14977.

The compute path is the native library ``_lib/libpmg.so`` (hand-written sm_103a CUDA
kernels behind the C ABI of ``include/pmg.h``); ``pmg`` is a thin ctypes binding with the
same call names.  Importing this package does not load the library; ``pmg.load()`` does,
and raises if it is missing -- there is no CPU fallback.
"""
__all__ = ["pmg", "build"]

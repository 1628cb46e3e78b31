"""GB300 (sm_103a) implementation of the harmonic surface mapping algorithm (HSMA) for the
reaction potential of a spherical cavity in a linearized Poisson-Boltzmann continuum
(Fu & Gan, arXiv:1907.01724).

Layout:
  csrc/      CUDA kernels (sm_103a) and the C-ABI engine (libhsma.so)
  _native    in-tree nvcc build + ctypes loading (no CPU fallback)
  api        the Python binding of include/hsma.h (same names as the C entry points)
  inputs     seeded synthetic workloads (no arithmetic of the method)

Importing the package does not load CUDA; the library is built and loaded on first use.
"""
__all__ = ["api", "inputs"]


def __getattr__(name):
    if name in ("api", "_native", "inputs", "batch", "server", "autotune"):
        import importlib
        return importlib.import_module(f"{__name__}.{name}")
    raise AttributeError(name)

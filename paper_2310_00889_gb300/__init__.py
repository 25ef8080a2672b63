"""GB300 (sm_103a) implementation of the hot path of Malhotra & Barnett, "Efficient
Convergent Boundary Integral Methods for Slender Bodies" (arXiv 2310.00889): the
uncorrected Nystrom Stokes single-/double-layer pair sums, the combined-field operator
I/2 + D + eta S with a sparse correction, and its GMRES solve.

Submodules:
  inputs -- seeded synthetic geometries and densities (numpy only)
  sbq    -- ctypes binding of the CUDA C-ABI library libsbq.so (loaded on first access)
  build  -- nvcc build of libsbq.so
"""
import importlib

__all__ = ["inputs", "sbq", "build"]


def __getattr__(name):
    if name in __all__:
        return importlib.import_module("." + name, __name__)
    raise AttributeError(name)

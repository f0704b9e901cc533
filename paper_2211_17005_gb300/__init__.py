"""GB300-native (sm_103a) hierarchical pathwise-CVA hot path (arXiv 2211.17005).

Submodules:
  workload  seeded synthetic inputs (model parameters, swap portfolios)
  build     nvcc build of the CUDA library _build/libcva.so
  _native   ctypes binding of include/cva.h
  api       torch-facing wrappers (Simulation, regress, cva0)
"""
from . import workload  # noqa: F401

__all__ = ["workload", "build", "api"]

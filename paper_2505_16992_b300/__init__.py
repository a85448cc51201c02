"""B300-native (sm_103a) per-time-step PISO update of arXiv:2505.16992 (PICT).

Submodules:
  workloads  seeded synthetic inputs (no solver arithmetic)
  capi       ctypes binding of include/piso.h (needs the built libpiso.so)
  solver     torch-facing Domain / Batch / autograd wrappers
  losses     user-side loss code on the library's differentiable statistics
  _build     nvcc build of libpiso.so for sm_103a
"""
__all__ = ["workloads", "capi", "solver"]

// Adjoint step kernels, double storage: every instantiation of adj_kernel
// (2D/3D, 512/768 threads, plain / ILU(0); the non-orthogonal ones are in
// piso_kernels_adjno_f64.cu) in a translation unit of its own
// (built in parallel with the others); piso_capi.cu launches them through the
// addresses returned here.
#include "piso_adjoint.cuh"

namespace piso {

const void* adjno_kernel_addr_f64(int nd, bool wide);   // MODE 2, piso_kernels_adjno_f64.cu

template <int MODE>
static const void* adj_addr_f64(int nd, bool wide) {
  if (wide) return nd == 2 ? (const void*)adj_kernel<double, 2, 768, MODE> : (const void*)adj_kernel<double, 3, 768, MODE>;
  return nd == 2 ? (const void*)adj_kernel<double, 2, 512, MODE> : (const void*)adj_kernel<double, 3, 512, MODE>;
}

const void* adj_kernel_addr_f64(int nd, bool wide, int mode) {
  if (mode == 2) return adjno_kernel_addr_f64(nd, wide);
  return mode == 1 ? adj_addr_f64<1>(nd, wide) : adj_addr_f64<0>(nd, wide);
}

}  // namespace piso

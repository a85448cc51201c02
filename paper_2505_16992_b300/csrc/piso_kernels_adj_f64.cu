// Adjoint step kernels, double storage: every instantiation of adj_kernel
// (2D/3D, 512/768 threads, plain / ILU(0)) in a translation unit of its own
// (built in parallel with the others); piso_capi.cu launches them through the
// addresses returned here.
#include "piso_adjoint.cuh"

namespace piso {

template <bool ILU>
static const void* adj_addr_f64(int nd, bool wide) {
  if (wide) return nd == 2 ? (const void*)adj_kernel<double, 2, 768, ILU> : (const void*)adj_kernel<double, 3, 768, ILU>;
  return nd == 2 ? (const void*)adj_kernel<double, 2, 512, ILU> : (const void*)adj_kernel<double, 3, 512, ILU>;
}

const void* adj_kernel_addr_f64(int nd, bool wide, bool ilu) {
  return ilu ? adj_addr_f64<true>(nd, wide) : adj_addr_f64<false>(nd, wide);
}

}  // namespace piso

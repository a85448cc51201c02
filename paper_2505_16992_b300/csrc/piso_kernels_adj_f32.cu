// Adjoint step kernels, float storage: every instantiation of adj_kernel
// (2D/3D, 512/768 threads, plain / ILU(0)) in a translation unit of its own
// (built in parallel with the others); piso_capi.cu launches them through the
// addresses returned here.
#include "piso_adjoint.cuh"

namespace piso {

template <bool ILU>
static const void* adj_addr_f32(int nd, bool wide) {
  if (wide) return nd == 2 ? (const void*)adj_kernel<float, 2, 768, ILU> : (const void*)adj_kernel<float, 3, 768, ILU>;
  return nd == 2 ? (const void*)adj_kernel<float, 2, 512, ILU> : (const void*)adj_kernel<float, 3, 512, ILU>;
}

const void* adj_kernel_addr_f32(int nd, bool wide, bool ilu) {
  return ilu ? adj_addr_f32<true>(nd, wide) : adj_addr_f32<false>(nd, wide);
}

}  // namespace piso

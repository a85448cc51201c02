// Forward step kernels, double storage: every instantiation of fwd_kernel
// (2D/3D, 512/768 threads, modes plain / ILU(0); the non-orthogonal ones are
// in piso_kernels_fwdno_f64.cu) compiled in a translation unit of its own, so the library's units build in parallel;
// piso_capi.cu launches them through the addresses returned here.
#include "piso_forward.cuh"

namespace piso {

const void* fwdno_kernel_addr_f64(int nd, bool wide);   // MODE 2, piso_kernels_fwdno_f64.cu

template <int MODE>
static const void* fwd_addr_f64(int nd, bool wide) {
  if (wide) return nd == 2 ? (const void*)fwd_kernel<double, 2, 768, MODE> : (const void*)fwd_kernel<double, 3, 768, MODE>;
  return nd == 2 ? (const void*)fwd_kernel<double, 2, 512, MODE> : (const void*)fwd_kernel<double, 3, 512, MODE>;
}

const void* fwd_kernel_addr_f64(int nd, bool wide, int mode) {
  if (mode == 2) return fwdno_kernel_addr_f64(nd, wide);
  return mode == 1 ? fwd_addr_f64<1>(nd, wide) : fwd_addr_f64<0>(nd, wide);
}

}  // namespace piso

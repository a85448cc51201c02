// Forward step kernels of non-orthogonal meshes (MODE 2), double storage, in a
// translation unit of their own so they build in parallel with the others.
#include "piso_forward.cuh"

namespace piso {

const void* fwdno_kernel_addr_f64(int nd, bool wide) {
  if (wide) return nd == 2 ? (const void*)fwd_kernel<double, 2, 768, 2> : (const void*)fwd_kernel<double, 3, 768, 2>;
  return nd == 2 ? (const void*)fwd_kernel<double, 2, 512, 2> : (const void*)fwd_kernel<double, 3, 512, 2>;
}

}  // namespace piso

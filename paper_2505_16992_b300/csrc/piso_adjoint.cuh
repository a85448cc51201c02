#pragma once
#include "piso_forward.cuh"
namespace piso {
template <typename real, int ND>
__global__ void __launch_bounds__(512, 1) adj_kernel(int dummy) {}
}

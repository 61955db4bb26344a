// Device helpers shared by the learned-potential kernels (inference and
// training on the tcgen05 tensor cores): BF16 packing.
#pragma once
#include <cuda_bf16.h>

#include "kernels.cuh"

namespace espp {

__device__ __forceinline__ unsigned int pack_bf16x2(float lo, float hi) {
    const __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
    return *reinterpret_cast<const unsigned int*>(&v);
}

}  // namespace espp

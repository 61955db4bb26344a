// Device helpers shared by the learned-potential kernels (inference and
// training on the tcgen05 tensor cores): BF16 packing and the SiLU tangent
// in packed FP32x2 arithmetic.
#pragma once
#include <cuda_bf16.h>

#include "kernels.cuh"
#include "packed.cuh"

namespace espp {

__device__ __forceinline__ unsigned int pack_bf16x2(float lo, float hi) {
    const __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
    return *reinterpret_cast<const unsigned int*>(&v);
}

// For two units at once, with t = tanh(y):
//   silu'(z) dz = (1 + t)(1 + y (1 - t)) dy, written c dy with
//   c = a + t a, a = 1 + y (1 - t), 1 - t = t (-1) + 1
__device__ __forceinline__ f32x2 silu_tangent_factor(f32x2 y, f32x2 t) {
    const f32x2 one = f2(1.f, 1.f), mone = f2(-1.f, -1.f);
    const f32x2 omt = f2fma(t, mone, one);
    const f32x2 a = f2fma(y, omt, one);
    return f2fma(t, a, a);
}

}  // namespace espp

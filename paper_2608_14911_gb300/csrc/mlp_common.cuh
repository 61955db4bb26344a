// Device helpers shared by the learned-potential kernels (inference and
// training on the tcgen05 tensor cores): BF16 packing and packed FP32x2
// arithmetic.
#pragma once
#include <cuda_bf16.h>

#include "kernels.cuh"

namespace espp {

__device__ __forceinline__ unsigned int pack_bf16x2(float lo, float hi) {
    const __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
    return *reinterpret_cast<const unsigned int*>(&v);
}

// Pairs of FP32 values in one 64-bit register and the packed FP32x2
// arithmetic of the sm_100 family (two lanes per instruction, the same
// round-to-nearest results as the scalar operations).
typedef unsigned long long f32x2;
__device__ __forceinline__ f32x2 f2(float a, float b) {
    f32x2 r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(a), "f"(b));
    return r;
}
__device__ __forceinline__ void f2split(f32x2 v, float& a, float& b) {
    asm("mov.b64 {%0, %1}, %2;" : "=f"(a), "=f"(b) : "l"(v));
}
__device__ __forceinline__ f32x2 f2fma(f32x2 a, f32x2 b, f32x2 c) {
    f32x2 d;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
    return d;
}
__device__ __forceinline__ f32x2 f2mul(f32x2 a, f32x2 b) {
    f32x2 d;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ f32x2 f2add(f32x2 a, f32x2 b) {
    f32x2 d;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
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

// Device helpers shared by the learned-potential kernels (inference and
// training): BF16 packing, the m16n8k16 BF16 tensor-core MMA with FP32
// accumulation, SiLU and its derivatives, and the per-tile radial features.
//
// Fragment layouts of mma.m16n8k16 (row.col), lane = 4 g + t:
//   A (16x16): a0 = (g, 2t..2t+1), a1 = (g+8, 2t..), a2 = (g, 2t+8..), a3 = (g+8, 2t+8..)
//   B (16x8):  b0 = (k 2t..2t+1, n g), b1 = (k 2t+8.., n g)
//   C (16x8):  c0,c1 = (g, 2t..2t+1), c2,c3 = (g+8, 2t..2t+1)
// Two adjacent n-tiles of C therefore hold exactly one k-tile of A.
#pragma once
#include <cuda_bf16.h>

#include "kernels.cuh"

namespace espp {

constexpr int W1_LD = MLP_NB + 8;  // padded smem row strides (conflict-free B loads)
constexpr int W2_LD = MLP_H + 8;

__device__ __forceinline__ unsigned int pack_bf16x2(float lo, float hi) {
    const __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
    return *reinterpret_cast<const unsigned int*>(&v);
}

__device__ __forceinline__ void mma_bf16_16816(float c[4], const unsigned int a[4], unsigned int b0,
                                               unsigned int b1) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 "
        "{%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, {%0,%1,%2,%3};\n"
        : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

// logistic sigmoid from the hardware tanh: s(z) = (1 + tanh(z / 2)) / 2
__device__ __forceinline__ float sigm(float z) {
    float t;
    asm("tanh.approx.f32 %0, %1;" : "=f"(t) : "f"(0.5f * z));
    return fmaf(0.5f, t, 0.5f);
}

// B fragment (two 32-bit registers) of a [n][k] row-major BF16 matrix in
// shared memory with row stride ld: element (k, n) = M[n][k].
__device__ __forceinline__ void b_frag(const __nv_bfloat16* M, int ld, int n0, int k0, int g, int t,
                                       unsigned int& b0, unsigned int& b1) {
    const __nv_bfloat16* row = M + (n0 + g) * ld + k0 + 2 * t;
    b0 = *reinterpret_cast<const unsigned int*>(row);
    b1 = *reinterpret_cast<const unsigned int*>(row + 8);
}

// Radial features of tile rows a = g and b = g + 8 (distances ra, rb) as the
// A operands of the first layer: phi (aph) and dphi/dr (adp), two k-tiles.
__device__ __forceinline__ void rbf_fragments(float ra, float rb, float rc, int t, unsigned int aph[2][4],
                                              unsigned int adp[2][4]) {
    const float wid = rc / (MLP_NB - 1);
    const float inv2w2 = 0.5f / (wid * wid), invw2 = 1.0f / (wid * wid);
    const float pirc = 3.14159265358979f / rc;
    const float fca = 0.5f * (__cosf(pirc * ra) + 1.f), fcb = 0.5f * (__cosf(pirc * rb) + 1.f);
    const float dfca = -0.5f * pirc * __sinf(pirc * ra), dfcb = -0.5f * pirc * __sinf(pirc * rb);
#pragma unroll
    for (int kt = 0; kt < 2; ++kt) {
#pragma unroll
        for (int half = 0; half < 2; ++half) {
            const int col = kt * 16 + half * 8 + t * 2;
            float ph[2][2], dp[2][2];
#pragma unroll
            for (int q = 0; q < 2; ++q) {
                const float mu = wid * (float)(col + q);
                const float da = ra - mu, db = rb - mu;
                const float ga = __expf(-da * da * inv2w2), gb = __expf(-db * db * inv2w2);
                ph[0][q] = ga * fca;
                ph[1][q] = gb * fcb;
                dp[0][q] = ga * (dfca - da * invw2 * fca);
                dp[1][q] = gb * (dfcb - db * invw2 * fcb);
            }
            aph[kt][2 * half + 0] = pack_bf16x2(ph[0][0], ph[0][1]);
            aph[kt][2 * half + 1] = pack_bf16x2(ph[1][0], ph[1][1]);
            adp[kt][2 * half + 0] = pack_bf16x2(dp[0][0], dp[0][1]);
            adp[kt][2 * half + 1] = pack_bf16x2(dp[1][0], dp[1][1]);
        }
    }
}

// Weights into shared memory (padded rows); W2t is the transpose of W2, used
// by the training kernel's backward GEMM.
__device__ __forceinline__ void load_mlp_weights(const MlpWeights* __restrict__ W, __nv_bfloat16* w1s,
                                                 __nv_bfloat16* w2s, __nv_bfloat16* w2t, float* b1s,
                                                 float* b2s, float* w3s) {
    for (int e = threadIdx.x; e < MLP_H * MLP_NB; e += blockDim.x)
        w1s[(e / MLP_NB) * W1_LD + e % MLP_NB] = W->W1[e];
    for (int e = threadIdx.x; e < MLP_H * MLP_H; e += blockDim.x) {
        w2s[(e / MLP_H) * W2_LD + e % MLP_H] = W->W2[e];
        if (w2t) w2t[(e % MLP_H) * W2_LD + e / MLP_H] = W->W2[e];
    }
    for (int e = threadIdx.x; e < MLP_H; e += blockDim.x) {
        b1s[e] = W->b1[e];
        b2s[e] = W->b2[e];
        w3s[e] = W->w3[e];
    }
}

}  // namespace espp

// Learned coarse-grained pair potential on the tensor cores: a radial-basis
// MLP u(r) (32 Gaussian bases with a cosine cutoff envelope -> 64 SiLU -> 64
// SiLU -> 1), BF16 weights and activations, FP32 accumulation.  The force
// needs du/dr; it is carried forward through the same two GEMMs as a second
// set of 16 rows (the tangent d/dr of every activation), so one pass gives u
// and du/dr for 16 pairs:
//   [z1; dz1] = [phi; dphi/dr] W1^T            (2 x 16 x 32 . 32 x 64)
//   h1 = silu(z1 + b1),  dh1 = silu'(z1 + b1) dz1
//   [z2; dz2] = [h1; dh1] W2^T                 (2 x 16 x 64 . 64 x 64)
//   u = w3 . silu(z2 + b2) + b3,  du/dr = w3 . (silu'(z2 + b2) dz2)
// The accumulator fragments of the first GEMM are re-packed in registers as
// the A operand of the second (the m16n8 accumulator layout of two adjacent
// n-tiles equals the m16k16 A layout), so activations never touch memory.
//
// One warp per particle: its Verlet-list entries inside the MLP cutoff are
// compacted 32 at a time with a ballot and evaluated 16 per tile; the warp
// sums -du/dr r_hat over them (full list, so no atomics) and writes the
// particle's pair force, its pair-energy sum and its virial sum (each pair
// counted from both ends, as the step kernel's own pair loop does).
#include "mlp_common.cuh"

namespace espp {

constexpr int MLP_WARPS = 4;

template <class T>
__global__ void __launch_bounds__(32 * MLP_WARPS) k_mlp(DevSys<T> s, int cur) {
    __shared__ __align__(16) __nv_bfloat16 w1s[MLP_H * W1_LD];
    __shared__ __align__(16) __nv_bfloat16 w2s[MLP_H * W2_LD];
    __shared__ float b1s[MLP_H], b2s[MLP_H], w3s[MLP_H];
    __shared__ float4 pairs[MLP_WARPS][32];  // compacted (r, dx, dy, dz) per warp
    const MlpWeights* __restrict__ W = s.mlp;
    load_mlp_weights(W, w1s, w2s, nullptr, b1s, b2s, w3s);
    __syncthreads();
    if (s.ctrl->abort) return;
    const float b3 = W->b3;
    const float rc = W->rc, rc2 = rc * rc;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int g = lane >> 2, tig = lane & 3;
    const V4<T>* __restrict__ P = s.pos[cur];
    const size_t stride = (size_t)s.stride;

    for (int t = blockIdx.x; t < s.ntiles; t += gridDim.x) {
        const Tile tl = s.tiles[t];
        const RepGeom<T>& geo = s.reps[tl.rep];
        const T L0 = geo.L[0], L1 = geo.L[1], L2 = geo.L[2];
        for (int pi = warp; pi < tl.count; pi += MLP_WARPS) {
            const int i = tl.start + pi;
            const V4<T> xi = ld4<T>(P + i);
            const int n = s.nbr_cnt[i];
            float fx = 0.f, fy = 0.f, fz = 0.f, eu = 0.f, ew = 0.f;  // lane partials
            for (int c0 = 0; c0 < n; c0 += 32) {
                // ---- this lane's list entry, inside the cutoff or not --------
                const int c = c0 + lane;
                float r = rc, dx = 0.f, dy = 0.f, dz = 0.f;
                bool valid = false;
                if (c < n) {
                    const int e = s.nbr[4 * ((size_t)(c >> 2) * stride + i) + (c & 3)];
                    const V4<T> xj = ld4<T>(P + nbr_slot(e));
                    const int code = nbr_code(e);
                    const T ddx = shifted_diff(xi.x, (T)(xi.x - L0), xj.x, L0, code & 3);
                    const T ddy = shifted_diff(xi.y, (T)(xi.y - L1), xj.y, L1, (code >> 2) & 3);
                    const T ddz = shifted_diff(xi.z, (T)(xi.z - L2), xj.z, L2, code >> 4);
                    const float r2 = (float)(ddx * ddx + ddy * ddy + ddz * ddz);
                    if (r2 < rc2) {
                        valid = true;
                        r = sqrtf(r2);
                        dx = (float)ddx;
                        dy = (float)ddy;
                        dz = (float)ddz;
                    }
                }
                const unsigned int vm = __ballot_sync(0xffffffffu, valid);
                const int nv = __popc(vm);
                if (valid) pairs[warp][__popc(vm & ((1u << lane) - 1u))] = make_float4(r, dx, dy, dz);
                __syncwarp();
                for (int k0 = 0; k0 < nv; k0 += 16) {
                    // ---- the tile's 16 pairs: row p is the (k0+p)-th valid entry
                    const int p = lane & 15;
                    const bool pvalid = k0 + p < nv;
                    const float4 q4 = pvalid ? pairs[warp][k0 + p] : make_float4(rc, 0.f, 0.f, 0.f);
                    const float pr = q4.x, pdx = q4.y, pdy = q4.z, pdz = q4.w;
                    const float rr = pvalid ? pr : rc;  // invalid rows sit at the cutoff
                    // rows g and g + 8 of the tile
                    const float ra = __shfl_sync(0xffffffffu, rr, g);
                    const float rb = __shfl_sync(0xffffffffu, rr, g + 8);
                    unsigned int aph[2][4], adp[2][4];
                    rbf_fragments(ra, rb, rc, tig, aph, adp);
                    // ---- layer 1 GEMM, SiLU, re-packed as layer 2 A operands ----
                    unsigned int ah[4][4], adh[4][4];
#pragma unroll
                    for (int nt = 0; nt < 8; ++nt) {
                        float z[4] = {0.f, 0.f, 0.f, 0.f}, dzv[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
                        for (int kt = 0; kt < 2; ++kt) {
                            unsigned int b0, b1;
                            b_frag(w1s, W1_LD, nt * 8, kt * 16, g, tig, b0, b1);
                            mma_bf16_16816(z, aph[kt], b0, b1);
                            mma_bf16_16816(dzv, adp[kt], b0, b1);
                        }
                        const int ncol = nt * 8 + tig * 2;
                        float hv[4], dhv[4];
#pragma unroll
                        for (int e = 0; e < 4; ++e) {
                            const float zz = z[e] + b1s[ncol + (e & 1)];
                            const float sg = sigm(zz);
                            hv[e] = zz * sg;
                            dhv[e] = sg * (1.f + zz * (1.f - sg)) * dzv[e];
                        }
                        const int kt2 = nt >> 1, off = (nt & 1) * 2;
                        ah[kt2][off + 0] = pack_bf16x2(hv[0], hv[1]);
                        ah[kt2][off + 1] = pack_bf16x2(hv[2], hv[3]);
                        adh[kt2][off + 0] = pack_bf16x2(dhv[0], dhv[1]);
                        adh[kt2][off + 1] = pack_bf16x2(dhv[2], dhv[3]);
                    }
                    // ---- layer 2 GEMM and the output layer, one n-tile at a time -
                    float ua = 0.f, ub = 0.f, dua = 0.f, dub = 0.f;
#pragma unroll
                    for (int nt = 0; nt < 8; ++nt) {
                        float z[4] = {0.f, 0.f, 0.f, 0.f}, dzv[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
                        for (int kt = 0; kt < 4; ++kt) {
                            unsigned int b0, b1;
                            b_frag(w2s, W2_LD, nt * 8, kt * 16, g, tig, b0, b1);
                            mma_bf16_16816(z, ah[kt], b0, b1);
                            mma_bf16_16816(dzv, adh[kt], b0, b1);
                        }
                        const int ncol = nt * 8 + tig * 2;
#pragma unroll
                        for (int e = 0; e < 4; ++e) {
                            const float zz = z[e] + b2s[ncol + (e & 1)];
                            const float sg = sigm(zz);
                            const float w3v = w3s[ncol + (e & 1)];
                            const float uu = w3v * zz * sg;
                            const float dd = w3v * sg * (1.f + zz * (1.f - sg)) * dzv[e];
                            if (e < 2) {
                                ua += uu;
                                dua += dd;
                            } else {
                                ub += uu;
                                dub += dd;
                            }
                        }
                    }
                    // sum over the four lanes of a row group
#pragma unroll
                    for (int o = 1; o < 4; o <<= 1) {
                        ua += __shfl_xor_sync(0xffffffffu, ua, o);
                        ub += __shfl_xor_sync(0xffffffffu, ub, o);
                        dua += __shfl_xor_sync(0xffffffffu, dua, o);
                        dub += __shfl_xor_sync(0xffffffffu, dub, o);
                    }
                    // row p lives in lane 4 (p mod 8), first (p < 8) or second half
                    const int rs = 4 * (p & 7);
                    const float ufa = __shfl_sync(0xffffffffu, ua, rs), ufb = __shfl_sync(0xffffffffu, ub, rs);
                    const float dfa = __shfl_sync(0xffffffffu, dua, rs), dfb = __shfl_sync(0xffffffffu, dub, rs);
                    if (lane < 16 && pvalid) {
                        const float u = (p < 8 ? ufa : ufb) + b3;
                        const float du = p < 8 ? dfa : dfb;
                        const float fr = -du / pr;
                        fx += fr * pdx;
                        fy += fr * pdy;
                        fz += fr * pdz;
                        eu += u;
                        ew += fr * pr * pr;
                    }
                }
                __syncwarp();
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                fx += __shfl_xor_sync(0xffffffffu, fx, o);
                fy += __shfl_xor_sync(0xffffffffu, fy, o);
                fz += __shfl_xor_sync(0xffffffffu, fz, o);
                eu += __shfl_xor_sync(0xffffffffu, eu, o);
                ew += __shfl_xor_sync(0xffffffffu, ew, o);
            }
            if (lane == 0) {
                s.mlp_f[i] = make_float4(fx, fy, fz, eu);
                s.mlp_w[i] = ew;
            }
        }
    }
}

template <class T>
void Launch<T>::mlp(const DevSys<T>& s, int cur, cudaStream_t st) {
    k_mlp<T><<<s.ntiles, 32 * MLP_WARPS, 0, st>>>(s, cur);
}

template void Launch<float>::mlp(const DevSys<float>&, int, cudaStream_t);
template void Launch<double>::mlp(const DevSys<double>&, int, cudaStream_t);

}  // namespace espp

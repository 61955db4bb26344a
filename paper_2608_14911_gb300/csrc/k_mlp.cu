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
// Each unordered pair is evaluated once.  Three kernels:
//   k_mlp_rev     (list builds) for every list entry (i, j) with j > i, the
//                 index of the mirrored entry (j, i) in j's list
//   k_mlp_pairs   warp per 32 particles: their entries with j > i inside the
//                 MLP cutoff are compacted through a shared staging buffer
//                 into dense 16-pair tiles; -du/dr / r (and u) of each pair
//                 go to both entries of the pair (zero beyond the cutoff)
//   k_mlp_gather  thread per particle: force, energy and virial sums over
//                 its full list from the per-entry values, in list order
// Every entry is written once per evaluation and summed in a fixed order, so
// the forces do not depend on the order in which warps run.
#include "mlp_common.cuh"

namespace espp {

constexpr int MLP_WARPS = 4;
constexpr int MLP_STAGE = 48;  // < 16 pending + 32 new
#ifndef ESPP_MLP_MINB
#define ESPP_MLP_MINB 4  // resident blocks of k_mlp_pairs per SM the registers must allow
#endif

// The tile works with y = z / 2: the weights and biases are halved when they
// are staged (exact in BF16 and FP32), so that with t = tanh(y) (one hardware
// instruction)
//   silu(z)  = z (1 + tanh(z/2)) / 2      = y (1 + t)
//   silu'(z) dz = (1 + t)(1 + y (1 - t)) dy     (dz = 2 dy)
// and the biases start the accumulators instead of being added afterwards.
__device__ __forceinline__ float tanh_hw(float y) {
    float t;
    asm("tanh.approx.f32 %0, %1;" : "=f"(t) : "f"(y));
    return t;
}

// four 8x8 BF16 matrices from shared memory (rows given by lanes 8m..8m+7)
__device__ __forceinline__ void ldsm_x4(const __nv_bfloat16* p, unsigned int& r0, unsigned int& r1,
                                        unsigned int& r2, unsigned int& r3) {
    const unsigned int a = (unsigned int)__cvta_generic_to_shared(p);
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];\n"
                 : "=r"(r0), "=r"(r1), "=r"(r2), "=r"(r3)
                 : "r"(a));
}

__device__ __forceinline__ size_t entry_index(int i, int k, size_t stride) {
    return 4 * ((size_t)(k >> 2) * stride + i) + (k & 3);
}

// ---- mirrored entries (list builds) -----------------------------------------
template <class T>
__global__ void __launch_bounds__(TILE) k_mlp_rev(DevSys<T> s) {
    if (s.ctrl->abort) return;
    const size_t stride = (size_t)s.stride;
    const int4* __restrict__ nbr4 = reinterpret_cast<const int4*>(s.nbr);
    for (int t = blockIdx.x; t < s.ntiles; t += gridDim.x) {
        const Tile tl = s.tiles[t];
        if (!s.now[tl.rep] || (int)threadIdx.x >= tl.count) continue;
        const int i = tl.start + threadIdx.x;
        const int n = s.nbr_cnt[i];
        for (int k = 0; k < n; ++k) {
            const size_t e = entry_index(i, k, stride);
            const int j = nbr_slot(s.nbr[e]);
            if (j <= i) continue;
            // the list is symmetric: i is in j's list
            const int nj = s.nbr_cnt[j];
            size_t found = e;
            for (int g = 0; 4 * g < nj; ++g) {
                const int4 q = nbr4[(size_t)g * stride + j];
                const int hit = nbr_slot(q.x) == i ? 0 : nbr_slot(q.y) == i ? 1 : nbr_slot(q.z) == i ? 2
                                                                           : nbr_slot(q.w) == i ? 3 : -1;
                if (hit >= 0 && 4 * g + hit < nj) {
                    found = entry_index(j, 4 * g + hit, stride);
                    break;
                }
            }
            if (found == e) atomicOr(&s.ctrl->err, ERRBIT_ASYM);  // cannot happen for a symmetric list
            s.mlp_rev[e] = (int)found;
        }
    }
}

// ---- one 16-pair tile ----------------------------------------------------------
// stage[p] = (r bits, entry, mirrored entry, -) for rows p < cnt.  w1s, w2s,
// b1s, b2s hold the halved first- and second-layer weights and biases.
template <bool ENERGY>
__device__ __forceinline__ void mlp_tile(const int4* stage, int cnt, float rc, float b3, const __nv_bfloat16* w1s,
                                         const __nv_bfloat16* w2s, const float* b1s, const float* b2s,
                                         const float* w3s, float* __restrict__ pf, float* __restrict__ pu) {
    const int lane = threadIdx.x & 31;
    const int g = lane >> 2, tig = lane & 3;
    const int p = lane & 15;
    const bool pvalid = p < cnt;
    const int4 st = pvalid ? stage[p] : make_int4(__float_as_int(rc), 0, 0, 0);
    const float pr = __int_as_float(st.x);
    // rows g and g + 8 of the tile
    const float ra = __shfl_sync(0xffffffffu, pr, g);
    const float rb = __shfl_sync(0xffffffffu, pr, g + 8);
    unsigned int aph[2][4], adp[2][4];
    rbf_fragments(ra, rb, rc, tig, aph, adp);
    // ldmatrix row address of this lane: matrix lane / 8 covers k + 8 (lane / 8)
    const int lr = lane & 7, lm = lane >> 3;
    // ---- layer 1 GEMM, SiLU, re-packed as layer 2 A operands ----
    unsigned int ah[4][4], adh[4][4];
#pragma unroll
    for (int nt = 0; nt < 8; ++nt) {
        const int ncol = nt * 8 + tig * 2;
        const float2 bb = *reinterpret_cast<const float2*>(b1s + ncol);
        float y[4] = {bb.x, bb.y, bb.x, bb.y}, dy[4] = {0.f, 0.f, 0.f, 0.f};
        unsigned int b[4];
        ldsm_x4(w1s + (nt * 8 + lr) * W1_LD + 8 * lm, b[0], b[1], b[2], b[3]);
#pragma unroll
        for (int kt = 0; kt < 2; ++kt) {
            mma_bf16_16816(y, aph[kt], b[2 * kt], b[2 * kt + 1]);
            mma_bf16_16816(dy, adp[kt], b[2 * kt], b[2 * kt + 1]);
        }
        float hv[4], dhv[4];
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            const float t = tanh_hw(y[e]);
            hv[e] = fmaf(y[e], t, y[e]);
            const float a = fmaf(-y[e], t, y[e] + 1.f);
            dhv[e] = fmaf(t, a, a) * dy[e];
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
        const int ncol = nt * 8 + tig * 2;
        const float2 bb = *reinterpret_cast<const float2*>(b2s + ncol);
        const float2 ww = *reinterpret_cast<const float2*>(w3s + ncol);
        float y[4] = {bb.x, bb.y, bb.x, bb.y}, dy[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
        for (int kh = 0; kh < 2; ++kh) {
            unsigned int b[4];
            ldsm_x4(w2s + (nt * 8 + lr) * W2_LD + 32 * kh + 8 * lm, b[0], b[1], b[2], b[3]);
#pragma unroll
            for (int q = 0; q < 2; ++q) {
                mma_bf16_16816(y, ah[2 * kh + q], b[2 * q], b[2 * q + 1]);
                mma_bf16_16816(dy, adh[2 * kh + q], b[2 * q], b[2 * q + 1]);
            }
        }
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            const float t = tanh_hw(y[e]);
            const float w3v = (e & 1) ? ww.y : ww.x;
            const float a = fmaf(-y[e], t, y[e] + 1.f);
            const float dd = fmaf(t, a, a) * dy[e];
            if (e < 2) {
                if (ENERGY) ua = fmaf(w3v, fmaf(y[e], t, y[e]), ua);
                dua = fmaf(w3v, dd, dua);
            } else {
                if (ENERGY) ub = fmaf(w3v, fmaf(y[e], t, y[e]), ub);
                dub = fmaf(w3v, dd, dub);
            }
        }
    }
    // sum over the four lanes of a row group
#pragma unroll
    for (int o = 1; o < 4; o <<= 1) {
        if (ENERGY) {
            ua += __shfl_xor_sync(0xffffffffu, ua, o);
            ub += __shfl_xor_sync(0xffffffffu, ub, o);
        }
        dua += __shfl_xor_sync(0xffffffffu, dua, o);
        dub += __shfl_xor_sync(0xffffffffu, dub, o);
    }
    // row p lives in lane 4 (p mod 8), first (p < 8) or second half
    const int rs = 4 * (p & 7);
    const float dfa = __shfl_sync(0xffffffffu, dua, rs), dfb = __shfl_sync(0xffffffffu, dub, rs);
    float ufa = 0.f, ufb = 0.f;
    if (ENERGY) {
        ufa = __shfl_sync(0xffffffffu, ua, rs);
        ufb = __shfl_sync(0xffffffffu, ub, rs);
    }
    if (lane < 16 && pvalid) {
        // dd is silu'(z2) dz2 already (the halving cancels): du/dr = w3 . dd;
        // the force factor is -du/dr / r
        const float sv = -(p < 8 ? dfa : dfb) / pr;
        pf[st.y] = sv;
        pf[st.z] = sv;
        if (ENERGY) {
            const float u = (p < 8 ? ufa : ufb) + b3;
            pu[st.y] = u;
            pu[st.z] = u;
        }
    }
}

// ---- unique pairs -> per-entry values -------------------------------------------
template <class T, bool ENERGY>
__global__ void __launch_bounds__(32 * MLP_WARPS, ESPP_MLP_MINB) k_mlp_pairs(DevSys<T> s, int cur) {
    __shared__ __align__(16) __nv_bfloat16 w1s[MLP_H * W1_LD];
    __shared__ __align__(16) __nv_bfloat16 w2s[MLP_H * W2_LD];
    __shared__ __align__(16) float b1s[MLP_H];
    __shared__ __align__(16) float b2s[MLP_H];
    __shared__ __align__(16) float w3s[MLP_H];
    __shared__ int4 stage[MLP_WARPS][MLP_STAGE];
    const MlpWeights* __restrict__ W = s.mlp;
    // halved first- and second-layer weights and biases (exact)
    for (int e = threadIdx.x; e < MLP_H * MLP_NB; e += blockDim.x)
        w1s[(e / MLP_NB) * W1_LD + e % MLP_NB] = __float2bfloat16(0.5f * __bfloat162float(W->W1[e]));
    for (int e = threadIdx.x; e < MLP_H * MLP_H; e += blockDim.x)
        w2s[(e / MLP_H) * W2_LD + e % MLP_H] = __float2bfloat16(0.5f * __bfloat162float(W->W2[e]));
    for (int e = threadIdx.x; e < MLP_H; e += blockDim.x) {
        b1s[e] = 0.5f * W->b1[e];
        b2s[e] = 0.5f * W->b2[e];
        w3s[e] = W->w3[e];
    }
    __syncthreads();
    if (s.ctrl->abort) return;
    const float b3 = W->b3;
    const float rc = W->rc, rc2 = rc * rc;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const unsigned int lt_mask = (1u << lane) - 1u;
    const V4<T>* __restrict__ P = s.pos[cur];
    const size_t stride = (size_t)s.stride;
    float* __restrict__ pf = s.mlp_pf;
    float* __restrict__ pu = s.mlp_pu;
    int4* st = stage[warp];
    const int ntasks = s.ntiles * (TILE / 32);
    for (int task = blockIdx.x * MLP_WARPS + warp; task < ntasks; task += gridDim.x * MLP_WARPS) {
        const Tile tl = s.tiles[task / (TILE / 32)];
        const int p0 = (task % (TILE / 32)) * 32;
        if (p0 >= tl.count) continue;
        const int p1 = min(tl.count, p0 + 32);
        const RepGeom<T>& geo = s.reps[tl.rep];
        const T L0 = geo.L[0], L1 = geo.L[1], L2 = geo.L[2];
        int nst = 0;  // staged pairs, uniform over the warp
        for (int pi = p0; pi < p1; ++pi) {
            const int i = tl.start + pi;
            const V4<T> xi = ld4<T>(P + i);
            const int n = s.nbr_cnt[i];
            for (int c0 = 0; c0 < n; c0 += 32) {
                const int c = c0 + lane;
                bool valid = false, zero = false;
                float r = 0.f;
                size_t e = 0;
                if (c < n) {
                    e = entry_index(i, c, stride);
                    const int en = s.nbr[e];
                    const int j = nbr_slot(en);
                    if (j > i) {
                        const V4<T> xj = ld4<T>(P + j);
                        const int code = nbr_code(en);
                        const T ddx = shifted_diff(xi.x, (T)(xi.x - L0), xj.x, L0, code & 3);
                        const T ddy = shifted_diff(xi.y, (T)(xi.y - L1), xj.y, L1, (code >> 2) & 3);
                        const T ddz = shifted_diff(xi.z, (T)(xi.z - L2), xj.z, L2, code >> 4);
                        const float r2 = (float)(ddx * ddx + ddy * ddy + ddz * ddz);
                        if (r2 < rc2) {
                            valid = true;
                            r = sqrtf(r2);
                        } else {
                            zero = true;
                        }
                    }
                }
                const int erev = (valid || zero) ? s.mlp_rev[e] : 0;
                if (zero) {
                    pf[e] = 0.f;
                    pf[erev] = 0.f;
                    if (ENERGY) {
                        pu[e] = 0.f;
                        pu[erev] = 0.f;
                    }
                }
                const unsigned int vm = __ballot_sync(0xffffffffu, valid);
                if (valid) st[nst + __popc(vm & lt_mask)] = make_int4(__float_as_int(r), (int)e, erev, 0);
                nst += __popc(vm);
                __syncwarp();
                while (nst >= 16) {
                    mlp_tile<ENERGY>(st, 16, rc, b3, w1s, w2s, b1s, b2s, w3s, pf, pu);
                    const int rem = nst - 16;
                    int4 keep = make_int4(0, 0, 0, 0);
                    if (lane < rem) keep = st[16 + lane];
                    __syncwarp();
                    if (lane < rem) st[lane] = keep;
                    __syncwarp();
                    nst = rem;
                }
            }
        }
        if (nst > 0) mlp_tile<ENERGY>(st, nst, rc, b3, w1s, w2s, b1s, b2s, w3s, pf, pu);
        __syncwarp();
    }
}

// ---- per-particle sums over the full list -------------------------------------
template <class T, bool ENERGY>
__global__ void __launch_bounds__(TILE) k_mlp_gather(DevSys<T> s, int cur) {
    if (s.ctrl->abort) return;
    const V4<T>* __restrict__ P = s.pos[cur];
    const size_t stride = (size_t)s.stride;
    const int4* __restrict__ nbr4 = reinterpret_cast<const int4*>(s.nbr);
    const float4* __restrict__ pf4 = reinterpret_cast<const float4*>(s.mlp_pf);
    const float4* __restrict__ pu4 = reinterpret_cast<const float4*>(s.mlp_pu);
    for (int t = blockIdx.x; t < s.ntiles; t += gridDim.x) {
        const Tile tl = s.tiles[t];
        if ((int)threadIdx.x >= tl.count) continue;
        const RepGeom<T>& geo = s.reps[tl.rep];
        const T L0 = geo.L[0], L1 = geo.L[1], L2 = geo.L[2];
        const int i = tl.start + threadIdx.x;
        const V4<T> xi = ld4<T>(P + i);
        const T xim = xi.x - L0, yim = xi.y - L1, zim = xi.z - L2;
        const int n = s.nbr_cnt[i];
        float fx = 0.f, fy = 0.f, fz = 0.f, eu = 0.f, ew = 0.f;
        for (int g = 0; 4 * g < n; ++g) {
            const int4 q = nbr4[(size_t)g * stride + i];
            const float4 f4 = pf4[(size_t)g * stride + i];
            float4 u4 = make_float4(0.f, 0.f, 0.f, 0.f);
            if (ENERGY) u4 = pu4[(size_t)g * stride + i];
            const int en[4] = {q.x, q.y, q.z, q.w};
            const float sv[4] = {f4.x, f4.y, f4.z, f4.w};
            const float uv[4] = {u4.x, u4.y, u4.z, u4.w};
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                if (4 * g + k >= n) continue;
                if (ENERGY) eu += uv[k];
                if (sv[k] == 0.f) continue;  // beyond the cutoff (or a flat pair)
                const int code = nbr_code(en[k]);
                const V4<T> xj = ld4<T>(P + nbr_slot(en[k]));
                const float dx = (float)shifted_diff(xi.x, xim, xj.x, L0, code & 3);
                const float dy = (float)shifted_diff(xi.y, yim, xj.y, L1, (code >> 2) & 3);
                const float dz = (float)shifted_diff(xi.z, zim, xj.z, L2, code >> 4);
                fx = fmaf(sv[k], dx, fx);
                fy = fmaf(sv[k], dy, fy);
                fz = fmaf(sv[k], dz, fz);
                if (ENERGY) ew = fmaf(sv[k], dx * dx + dy * dy + dz * dz, ew);
            }
        }
        s.mlp_f[i] = make_float4(fx, fy, fz, eu);
        if (ENERGY) s.mlp_w[i] = ew;
    }
}

template <class T>
int Launch<T>::mlp(const DevSys<T>& s, int cur, bool energy, cudaStream_t st) {
    const int tasks = s.ntiles * (TILE / 32);
    const int blocks = std::max(1, std::min((tasks + MLP_WARPS - 1) / MLP_WARPS, 152 * 16));
    if (energy) {
        k_mlp_pairs<T, true><<<blocks, 32 * MLP_WARPS, 0, st>>>(s, cur);
        k_mlp_gather<T, true><<<s.ntiles, TILE, 0, st>>>(s, cur);
    } else {
        k_mlp_pairs<T, false><<<blocks, 32 * MLP_WARPS, 0, st>>>(s, cur);
        k_mlp_gather<T, false><<<s.ntiles, TILE, 0, st>>>(s, cur);
    }
    return 2;
}

template <class T>
int Launch<T>::mlp_rev(const DevSys<T>& s, cudaStream_t st) {
    k_mlp_rev<T><<<s.ntiles, TILE, 0, st>>>(s);
    return 1;
}

template int Launch<float>::mlp(const DevSys<float>&, int, bool, cudaStream_t);
template int Launch<double>::mlp(const DevSys<double>&, int, bool, cudaStream_t);
template int Launch<float>::mlp_rev(const DevSys<float>&, cudaStream_t);
template int Launch<double>::mlp_rev(const DevSys<double>&, cudaStream_t);

}  // namespace espp

// Learned coarse-grained pair potential on the tensor cores: a radial-basis
// MLP u(r) (32 Gaussian bases with a cosine cutoff envelope -> 64 SiLU -> 64
// SiLU -> 1), BF16 weights and activations, FP32 accumulation.  The force
// needs du/dr; it is carried forward through the same two GEMMs as the
// tangent d/dr of every activation, in the rows below the values, so one
// pass gives u and du/dr for 8 pairs (rows 0-7 values, rows 8-15 tangents):
//   [z1; dz1] = [phi; dphi/dr] W1^T            (16 x 32 . 32 x 64)
//   h1 = silu(z1 + b1),  dh1 = silu'(z1 + b1) dz1
//   [z2; dz2] = [h1; dh1] W2^T                 (16 x 64 . 64 x 64)
//   u = w3 . silu(z2 + b2) + b3,  du/dr = w3 . (silu'(z2 + b2) dz2)
// The accumulator fragments of the first GEMM are re-packed in registers as
// the A operand of the second (the m16n8 accumulator layout of two adjacent
// n-tiles equals the m16k16 A layout), so activations never touch memory.
//
// Each unordered pair is evaluated once.  Kernels:
//   k_mlp_rev     (list builds) for every list entry (i, j) with j > i, the
//                 index of the mirrored entry (j, i) in j's list, and the
//                 array of all unordered pairs of the list
//   k_mlp_stage   thread per unordered pair: the pairs inside the MLP cutoff
//                 go to a dense pair array (r, entry, mirrored entry)
//   k_mlp_tiles   warps stream the dense array in 8-pair tensor-core tiles;
//                 -du/dr / r (and u) of each pair go to both of its entries
//   k_mlp_gather  thread per particle: force, energy and virial sums over
//                 its full list from the per-entry values, in list order,
//                 over the entries inside the cutoff
// Every entry inside the cutoff is written once per evaluation and summed in
// a fixed order, so the forces do not depend on the order in which warps run.
#include "mlp_common.cuh"

namespace espp {

constexpr int MLP_WARPS = 4;
#ifndef ESPP_MLP_MINB
#define ESPP_MLP_MINB 4  // resident blocks of k_mlp_tiles per SM the registers must allow
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

// Squared distance of a list pair as both kernels that decide "inside the
// cutoff" compute it: the same operations with explicit rounding, so the
// decision taken from the pair's two entries agrees (the two displacements are
// exact negatives of each other).
template <class T>
__device__ __forceinline__ float mlp_r2(const V4<T>& xi, T xim, T yim, T zim, const V4<T>& xj, T L0, T L1, T L2,
                                        int code, float& dx, float& dy, float& dz) {
    dx = (float)shifted_diff(xi.x, xim, xj.x, L0, code & 3);
    dy = (float)shifted_diff(xi.y, yim, xj.y, L1, (code >> 2) & 3);
    dz = (float)shifted_diff(xi.z, zim, xj.z, L2, code >> 4);
    return __fadd_rn(__fadd_rn(__fmul_rn(dx, dx), __fmul_rn(dy, dy)), __fmul_rn(dz, dz));
}

// Per-warp shared buffer of int4 records, flushed to a global array at a
// warp-aggregated atomic offset (one atomic per ~500 records).
constexpr int STAGE_BUF = 512;

struct WarpAppender {
    int4* buf;
    int4* out;
    int* count;
    int cap;
    unsigned int* err;
    int fill;
    __device__ __forceinline__ void push(bool valid, int4 rec) {
        const int lane = threadIdx.x & 31;
        const unsigned int m = __ballot_sync(0xffffffffu, valid);
        if (valid) buf[fill + __popc(m & ((1u << lane) - 1u))] = rec;
        fill += __popc(m);
        __syncwarp();
        if (fill > STAGE_BUF - 32) flush();
    }
    __device__ __forceinline__ void flush() {
        const int lane = threadIdx.x & 31;
        int base = 0;
        if (lane == 0 && fill > 0) base = atomicAdd(count, fill);
        base = __shfl_sync(0xffffffffu, base, 0);
        const int room = cap - base;
        if (lane == 0 && fill > room) atomicOr(err, ERRBIT_OVERFLOW);  // cannot happen: sized for every pair
        for (int k = lane; k < fill && k < room; k += 32) out[base + k] = buf[k];
        __syncwarp();
        fill = 0;
    }
};

// ---- mirrored entries and the upper-pair array (list builds) -------------------
// Thread per particle.  For every entry (i, j) with j > i: the index of the
// mirrored entry (j, i), searched in j's list for the replicas just rebuilt
// and kept for the others, and the record (entry, mirrored entry, list entry,
// replica) in the array of all unordered pairs of the list.  A warp scan of
// the per-thread counts gives each thread a contiguous run of records at one
// atomic offset per warp.
template <class T>
__global__ void __launch_bounds__(TILE) k_mlp_rev(DevSys<T> s) {
    if (s.ctrl->abort) return;
    const int lane = threadIdx.x & 31;
    const size_t stride = (size_t)s.stride;
    const int4* __restrict__ nbr4 = reinterpret_cast<const int4*>(s.nbr);
    for (int t = blockIdx.x; t < s.ntiles; t += gridDim.x) {
        const Tile tl = s.tiles[t];
        const bool active = (int)threadIdx.x < tl.count;
        const bool fresh = s.now[tl.rep] != 0;
        const int i = tl.start + threadIdx.x;
        const int n = active ? s.nbr_cnt[i] : 0;
        int cnt = 0;
        for (int k = 0; k < n; ++k) cnt += nbr_slot(s.nbr[entry_index(i, k, stride)]) > i ? 1 : 0;
        int incl = cnt;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int u = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += u;
        }
        int base = 0;
        if (lane == 31 && incl > 0) base = atomicAdd(s.mlp_nupper, incl);
        base = __shfl_sync(0xffffffffu, base, 31) + incl - cnt;
        if (base + cnt > s.mlp_upper_cap) {
            atomicOr(&s.ctrl->err, ERRBIT_OVERFLOW);  // cannot happen: sized for every pair
            continue;
        }
        for (int k = 0; k < n; ++k) {
            const size_t e = entry_index(i, k, stride);
            const int en = s.nbr[e];
            const int j = nbr_slot(en);
            if (j <= i) continue;
            size_t found = e;
            if (fresh) {
                // the list is symmetric: i is in j's list
                const int nj = s.nbr_cnt[j];
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
            } else {
                found = (size_t)s.mlp_rev[e];
            }
            s.mlp_upper[base++] = make_int4((int)e, (int)found, en, tl.rep);
        }
    }
}

// ---- one 8-pair tile ------------------------------------------------------------
// Rows g and g + 8 of every m16n8k16 operand belong to the same pair g: row g
// carries the values (features, activations), row g + 8 their derivatives
// with respect to r.  A lane then holds, for its columns, both z and dz/dr of
// one pair, so the SiLU and its derivative stay inside the lane, and a tile
// needs half the registers of two separate 16-row streams.
//
// Features of pair g (distance r) for the first layer: phi in row g, dphi/dr
// in row g + 8, columns 2t, 2t+1 (+8) of both k-tiles.
__device__ __forceinline__ void rbf_rows(float r, float rc, int t, unsigned int a[2][4]) {
    const float wid = rc / (MLP_NB - 1);
    const float inv2w2 = 0.5f / (wid * wid), invw2 = 1.0f / (wid * wid);
    const float pirc = 3.14159265358979f / rc;
    const float fc = 0.5f * (__cosf(pirc * r) + 1.f);
    const float dfc = -0.5f * pirc * __sinf(pirc * r);
#pragma unroll
    for (int kt = 0; kt < 2; ++kt) {
#pragma unroll
        for (int half = 0; half < 2; ++half) {
            const int col = kt * 16 + half * 8 + t * 2;
            float ph[2], dp[2];
#pragma unroll
            for (int q = 0; q < 2; ++q) {
                const float d = r - wid * (float)(col + q);
                const float gq = __expf(-d * d * inv2w2);
                ph[q] = gq * fc;
                dp[q] = gq * (dfc - d * invw2 * fc);
            }
            a[kt][2 * half + 0] = pack_bf16x2(ph[0], ph[1]);
            a[kt][2 * half + 1] = pack_bf16x2(dp[0], dp[1]);
        }
    }
}

// stage[p] = (r bits, entry, mirrored entry, -) for pairs p < cnt (global
// memory).  w1s, w2s, b1s, b2s hold the halved first- and second-layer
// weights and biases.
template <bool ENERGY>
__device__ __forceinline__ void mlp_tile8(const int4* stage, int cnt, float rc, float b3, const __nv_bfloat16* w1s,
                                          const __nv_bfloat16* w2s, const float* b1s, const float* b2s,
                                          const float* w3s, float* __restrict__ pf, float* __restrict__ pu) {
    const int lane = threadIdx.x & 31;
    const int g = lane >> 2, tig = lane & 3;
    const bool gvalid = g < cnt;
    const int4 st = gvalid ? stage[g] : make_int4(__float_as_int(rc), 0, 0, 0);
    const float r = __int_as_float(st.x);
    unsigned int af[2][4];
    rbf_rows(r, rc, tig, af);
    const int lr = lane & 7, lm = lane >> 3;
    // ---- layer 1: [y; dy] = [phi; dphi] W1^T / 2 + [b1 / 2; 0] ----
    unsigned int ah[4][4];
#pragma unroll
    for (int nt = 0; nt < 8; ++nt) {
        const int ncol = nt * 8 + tig * 2;
        const float2 bb = *reinterpret_cast<const float2*>(b1s + ncol);
        float c[4] = {bb.x, bb.y, 0.f, 0.f};
        unsigned int b[4];
        ldsm_x4(w1s + (nt * 8 + lr) * W1_LD + 8 * lm, b[0], b[1], b[2], b[3]);
        mma_bf16_16816(c, af[0], b[0], b[1]);
        mma_bf16_16816(c, af[1], b[2], b[3]);
        float h[2], dh[2];
#pragma unroll
        for (int e = 0; e < 2; ++e) {
            const float y = c[e], t = tanh_hw(y);
            h[e] = fmaf(y, t, y);
            const float a = fmaf(-y, t, y + 1.f);
            dh[e] = fmaf(t, a, a) * c[2 + e];
        }
        const int kt2 = nt >> 1, off = (nt & 1) * 2;
        ah[kt2][off + 0] = pack_bf16x2(h[0], h[1]);
        ah[kt2][off + 1] = pack_bf16x2(dh[0], dh[1]);
    }
    // ---- layer 2 and the output layer -------------------------------
    float u = 0.f, du = 0.f;
#pragma unroll
    for (int nt = 0; nt < 8; ++nt) {
        const int ncol = nt * 8 + tig * 2;
        const float2 bb = *reinterpret_cast<const float2*>(b2s + ncol);
        const float2 ww = *reinterpret_cast<const float2*>(w3s + ncol);
        float c[4] = {bb.x, bb.y, 0.f, 0.f};
#pragma unroll
        for (int kh = 0; kh < 2; ++kh) {
            unsigned int b[4];
            ldsm_x4(w2s + (nt * 8 + lr) * W2_LD + 32 * kh + 8 * lm, b[0], b[1], b[2], b[3]);
            mma_bf16_16816(c, ah[2 * kh], b[0], b[1]);
            mma_bf16_16816(c, ah[2 * kh + 1], b[2], b[3]);
        }
#pragma unroll
        for (int e = 0; e < 2; ++e) {
            const float y = c[e], t = tanh_hw(y), w3v = e ? ww.y : ww.x;
            const float a = fmaf(-y, t, y + 1.f);
            du = fmaf(w3v, fmaf(t, a, a) * c[2 + e], du);
            if (ENERGY) u = fmaf(w3v, fmaf(y, t, y), u);
        }
    }
    // sum over the four lanes of pair g
#pragma unroll
    for (int o = 1; o < 4; o <<= 1) {
        du += __shfl_xor_sync(0xffffffffu, du, o);
        if (ENERGY) u += __shfl_xor_sync(0xffffffffu, u, o);
    }
    if (tig == 0 && gvalid) {
        // the halving cancels in the tangent: du/dr = w3 . (silu'(z2) dz2);
        // the force factor is -du/dr / r
        const float sv = -du / r;
        pf[st.y] = sv;
        pf[st.z] = sv;
        if (ENERGY) {
            pu[st.y] = u + b3;
            pu[st.z] = u + b3;
        }
    }
}

// ---- pairs inside the cutoff -> a dense pair array -------------------------------
// Thread per unordered pair of the list; the pairs inside the cutoff go to the
// dense array through per-warp shared buffers.  Their order there does not
// matter: every pair's result depends only on its own distance.
template <class T>
__global__ void __launch_bounds__(TILE) k_mlp_stage(DevSys<T> s, int cur) {
    __shared__ int4 buf[TILE / 32][STAGE_BUF];
    if (s.ctrl->abort) return;
    const float rc = s.mlp->rc, rc2 = rc * rc;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const V4<T>* __restrict__ P = s.pos[cur];
    const int stride = s.stride;
    const int nu = min(*s.mlp_nupper, s.mlp_upper_cap);
    WarpAppender ap{buf[warp], s.mlp_pairs, s.mlp_npairs, s.mlp_pairs_cap, &s.ctrl->err, 0};
    const int nthreads = gridDim.x * blockDim.x;
    for (int base = (blockIdx.x * blockDim.x + warp * 32); base < nu; base += nthreads) {
        const int k = base + lane;
        bool valid = false;
        int4 rec = make_int4(0, 0, 0, 0);
        if (k < nu) {
            const int4 up = s.mlp_upper[k];
            const int en = up.z;
            const int i = (up.x >> 2) % stride;
            const RepGeom<T>& geo = s.reps[up.w];
            const T L0 = geo.L[0], L1 = geo.L[1], L2 = geo.L[2];
            const V4<T> xi = ld4<T>(P + i);
            const V4<T> xj = ld4<T>(P + nbr_slot(en));
            float dx, dy, dz;
            const float r2 = mlp_r2(xi, (T)(xi.x - L0), (T)(xi.y - L1), (T)(xi.z - L2), xj, L0, L1, L2,
                                    nbr_code(en), dx, dy, dz);
            valid = r2 < rc2;
            rec = make_int4(__float_as_int(sqrtf(r2)), up.x, up.y, 0);
        }
        ap.push(valid, rec);
    }
    ap.flush();
}

// ---- dense pair tiles on the tensor cores -------------------------------------
template <class T, bool ENERGY>
__global__ void __launch_bounds__(32 * MLP_WARPS, ESPP_MLP_MINB) k_mlp_tiles(DevSys<T> s) {
    __shared__ __align__(16) __nv_bfloat16 w1s[MLP_H * W1_LD];
    __shared__ __align__(16) __nv_bfloat16 w2s[MLP_H * W2_LD];
    __shared__ __align__(16) float b1s[MLP_H];
    __shared__ __align__(16) float b2s[MLP_H];
    __shared__ __align__(16) float w3s[MLP_H];
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
    const float rc = W->rc;
    const int np = min(*s.mlp_npairs, s.mlp_pairs_cap);
    const int ntl = (np + 7) >> 3;
    const int warp = threadIdx.x >> 5;
    for (int t = blockIdx.x * MLP_WARPS + warp; t < ntl; t += gridDim.x * MLP_WARPS)
        mlp_tile8<ENERGY>(s.mlp_pairs + 8 * (size_t)t, min(8, np - 8 * t), rc, b3, w1s, w2s, b1s, b2s, w3s,
                          s.mlp_pf, s.mlp_pu);
}

// ---- per-particle sums over the full list -------------------------------------
template <class T, bool ENERGY>
__global__ void __launch_bounds__(TILE) k_mlp_gather(DevSys<T> s, int cur) {
    if (s.ctrl->abort) return;
    const float rc = s.mlp->rc, rc2 = rc * rc;
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
                const V4<T> xj = ld4<T>(P + nbr_slot(en[k]));
                float dx, dy, dz;
                const float r2 = mlp_r2(xi, xim, yim, zim, xj, L0, L1, L2, nbr_code(en[k]), dx, dy, dz);
                if (!(r2 < rc2)) continue;  // beyond the cutoff: the entry holds no value this step
                fx = fmaf(sv[k], dx, fx);
                fy = fmaf(sv[k], dy, fy);
                fz = fmaf(sv[k], dz, fz);
                if (ENERGY) {
                    eu += uv[k];
                    ew = fmaf(sv[k], r2, ew);
                }
            }
        }
        s.mlp_f[i] = make_float4(fx, fy, fz, eu);
        if (ENERGY) s.mlp_w[i] = ew;
    }
}

template <class T>
int Launch<T>::mlp(const DevSys<T>& s, int cur, bool energy, cudaStream_t st) {
    cudaMemsetAsync(s.mlp_npairs, 0, sizeof(int), st);
    const int tblocks = 152 * ESPP_MLP_MINB;
    k_mlp_stage<T><<<152 * 8, TILE, 0, st>>>(s, cur);
    if (energy) {
        k_mlp_tiles<T, true><<<tblocks, 32 * MLP_WARPS, 0, st>>>(s);
        k_mlp_gather<T, true><<<s.ntiles, TILE, 0, st>>>(s, cur);
    } else {
        k_mlp_tiles<T, false><<<tblocks, 32 * MLP_WARPS, 0, st>>>(s);
        k_mlp_gather<T, false><<<s.ntiles, TILE, 0, st>>>(s, cur);
    }
    return 3;
}

template <class T>
int Launch<T>::mlp_rev(const DevSys<T>& s, cudaStream_t st) {
    cudaMemsetAsync(s.mlp_nupper, 0, sizeof(int), st);
    k_mlp_rev<T><<<s.ntiles, TILE, 0, st>>>(s);
    return 1;
}

template int Launch<float>::mlp(const DevSys<float>&, int, bool, cudaStream_t);
template int Launch<double>::mlp(const DevSys<double>&, int, bool, cudaStream_t);
template int Launch<float>::mlp_rev(const DevSys<float>&, cudaStream_t);
template int Launch<double>::mlp_rev(const DevSys<double>&, cudaStream_t);

}  // namespace espp

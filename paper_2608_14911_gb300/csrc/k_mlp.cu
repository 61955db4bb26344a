// Learned coarse-grained pair potential on the tensor cores: a radial-basis
// MLP u(r) (32 Gaussian bases with a cosine cutoff envelope -> 64 SiLU -> 64
// SiLU -> 1), BF16 weights and activations, FP32 accumulation.  The force
// needs du/dr; it is carried forward through the same two GEMMs as the
// tangent d/dr of every activation, so one pass gives u and du/dr:
//   [z1; dz1] = [phi; dphi/dr] W1^T + [b1; 0]          (128 pairs x 32 . 32 x 64)
//   h1 = silu(z1),  dh1 = silu'(z1) dz1
//   [z2; dz2] = [h1; dh1] W2^T + [b2; 0]               (128 pairs x 64 . 64 x 64)
//   u = w3 . silu(z2) + b3,  du/dr = w3 . (silu'(z2) dz2)
// on the tcgen05 tensor cores with the accumulators in tensor memory.
//
// Each unordered pair is evaluated once.  Kernels:
//   k_mlp_rev     (list builds, after a count and a scan) for every list
//                 entry (i, j) with j > i, the index of the mirrored entry
//                 (j, i) in j's list, and the array of all unordered pairs of
//                 the list in an order that depends only on the list
//   k_mlp_stage   thread per unordered pair: the pairs inside the MLP cutoff
//                 go to a dense pair array (r, entry, mirrored entry)
//   k_mlp_tc      CTAs stream the dense array in 128-pair tiles on the
//                 tcgen05 tensor cores (accumulators in tensor memory);
//                 -du/dr / r (and u) of each pair go to both of its entries
//   k_mlp_gather  thread per particle: force, energy and virial sums over
//                 its full list from the per-entry values, in list order,
//                 over the entries inside the cutoff
// Every entry inside the cutoff is written once per evaluation and summed in
// a fixed order, so the forces do not depend on the order in which warps run.
#include <cstring>

#include <math_constants.h>

#include "mlp_common.cuh"
#include "scan.cuh"
#include "tc_ptx.cuh"

namespace espp {


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
// staging kernel: records buffered per warp, and blocks per SM (more
// resident warps hide the gathers; 4M CG sites: 6.21 ms per step at 256 / 24,
// 6.52 at 512 / 8)
#ifndef ESPP_STAGE_BUF
#define ESPP_STAGE_BUF 256
#endif
#ifndef ESPP_STAGE_GRID
#define ESPP_STAGE_GRID 24
#endif
constexpr int STAGE_BUF = ESPP_STAGE_BUF;

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
// Every unordered pair of the list gets one record (entry (i, j) with j > i,
// mirrored entry (j, i), the list entry, replica), at an offset from a scan of
// the per-particle counts, so the array's order depends only on the list.
template <class T>
__global__ void __launch_bounds__(TILE) k_mlp_count(DevSys<T> s) {
    if (s.ctrl->abort) return;
    const size_t stride = (size_t)s.stride;
    for (int t = blockIdx.x; t < s.ntiles; t += gridDim.x) {
        const Tile tl = s.tiles[t];
        if ((int)threadIdx.x >= tl.count) continue;
        const int i = tl.start + threadIdx.x;
        const int n = s.nbr_cnt[i];
        int cnt = 0;
        for (int k = 0; k < n; ++k) cnt += nbr_slot(s.nbr[entry_index(i, k, stride)]) > i ? 1 : 0;
        s.mlp_ucount[i] = cnt;
    }
}

__global__ void __launch_bounds__(SCAN_THREADS) k_uscan_reduce(const int* __restrict__ in, int n,
                                                             int* __restrict__ part) {
    const int base = blockIdx.x * SCAN_TILE + threadIdx.x * SCAN_ITEMS;
    int sum = 0;
#pragma unroll
    for (int k = 0; k < SCAN_ITEMS; ++k) sum += base + k < n ? in[base + k] : 0;
    int excl;
    const int total = block_excl_scan(sum, &excl);
    if (threadIdx.x == 0) part[blockIdx.x] = total;
}

__global__ void __launch_bounds__(SCAN_THREADS) k_uscan_top(int* __restrict__ part, int nb, int* __restrict__ total) {
    int carry = 0;
    for (int b0 = 0; b0 < nb; b0 += SCAN_THREADS) {
        const int b = b0 + threadIdx.x;
        const int v = b < nb ? part[b] : 0;
        int excl;
        const int t = block_excl_scan(v, &excl);
        if (b < nb) part[b] = carry + excl;
        carry += t;
    }
    if (threadIdx.x == 0) *total = carry;
}

__global__ void __launch_bounds__(SCAN_THREADS) k_uscan_down(const int* __restrict__ in, int n,
                                                           const int* __restrict__ part, int* __restrict__ out) {
    const int base = blockIdx.x * SCAN_TILE + threadIdx.x * SCAN_ITEMS;
    int v[SCAN_ITEMS];
    int sum = 0;
#pragma unroll
    for (int k = 0; k < SCAN_ITEMS; ++k) {
        v[k] = base + k < n ? in[base + k] : 0;
        sum += v[k];
    }
    int excl;
    block_excl_scan(sum, &excl);
    int run = part[blockIdx.x] + excl;
#pragma unroll
    for (int k = 0; k < SCAN_ITEMS; ++k) {
        if (base + k < n) out[base + k] = run;
        run += v[k];
    }
}

// Thread per particle: mirrored entries, searched in j's list for the
// replicas just rebuilt and kept for the others, and the particle's records.
template <class T>
__global__ void __launch_bounds__(TILE) k_mlp_rev(DevSys<T> s) {
    if (s.ctrl->abort) return;
    const size_t stride = (size_t)s.stride;
    const int4* __restrict__ nbr4 = reinterpret_cast<const int4*>(s.nbr);
    for (int t = blockIdx.x; t < s.ntiles; t += gridDim.x) {
        const Tile tl = s.tiles[t];
        if ((int)threadIdx.x >= tl.count) continue;
        const bool fresh = s.now[tl.rep] != 0;
        const int i = tl.start + threadIdx.x;
        const int n = s.nbr_cnt[i];
        int base = s.mlp_uoff[i];
        if (base + s.mlp_ucount[i] > s.mlp_upper_cap) {
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
                // the list is symmetric: i is in j's list; four groups per
                // probe keep four loads in flight
                const int nj = s.nbr_cnt[j];
                const int ngj = (nj + 3) >> 2;
                for (int g0 = 0; g0 < ngj && found == e; g0 += 4) {
                    int4 q[4];
#pragma unroll
                    for (int u = 0; u < 4; ++u)
                        q[u] = g0 + u < ngj ? nbr4[(size_t)(g0 + u) * stride + j] : make_int4(-1, -1, -1, -1);
#pragma unroll
                    for (int u = 0; u < 4; ++u) {
                        const int hit = nbr_slot(q[u].x) == i ? 0 : nbr_slot(q[u].y) == i ? 1
                                      : nbr_slot(q[u].z) == i ? 2 : nbr_slot(q[u].w) == i ? 3 : -1;
                        const int kk = 4 * (g0 + u) + hit;
                        if (hit >= 0 && kk < nj && found == e) found = entry_index(j, kk, stride);
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
    // four records per thread and pass: four independent gather chains in flight
    constexpr int U = 4;
    const int nthreads = gridDim.x * blockDim.x;
    for (int base = (blockIdx.x * blockDim.x + warp * 32) * U; base < nu; base += nthreads * U) {
        int4 up[U];
#pragma unroll
        for (int q = 0; q < U; ++q) {
            const int k = base + 32 * q + lane;
            up[q] = k < nu ? s.mlp_upper[k] : make_int4(-1, 0, 0, 0);
        }
        V4<T> xi[U], xj[U];
#pragma unroll
        for (int q = 0; q < U; ++q) {
            if (up[q].x >= 0) {
                xi[q] = ld4<T>(P + (up[q].x >> 2) % stride);
                xj[q] = ld4<T>(P + nbr_slot(up[q].z));
            }
        }
#pragma unroll
        for (int q = 0; q < U; ++q) {
            bool valid = false;
            int4 rec = make_int4(0, 0, 0, 0);
            if (up[q].x >= 0) {
                const RepGeom<T>& geo = s.reps[up[q].w];
                const T L0 = geo.L[0], L1 = geo.L[1], L2 = geo.L[2];
                float dx, dy, dz;
                const float r2 = mlp_r2(xi[q], (T)(xi[q].x - L0), (T)(xi[q].y - L1), (T)(xi[q].z - L2), xj[q],
                                        L0, L1, L2, nbr_code(up[q].z), dx, dy, dz);
                valid = r2 < rc2;
                rec = make_int4(__float_as_int(sqrtf(r2)), up[q].x, up[q].y, 0);
            }
            ap.push(valid, rec);
        }
    }
    ap.flush();
}

// ---- dense pair tiles on the 5th-generation tensor cores -------------------------
// CTA of 256 threads, two per pair: pair (row) p of a 128-pair tile belongs to
// tensor-memory lane p, read by warps p / 32 and 4 + p / 32; the first half
// of the CTA takes columns 0..31 of every 64-column block, the second half
// columns 32..63 (tensor memory caps the tiles in flight at four per SM, so
// the second thread per pair is what fills the SM with warps).  Per tile:
//   features   each half writes 16 of its pair's 32 phi (row of A0) and
//              dphi/dr (row of A1) as BF16; the first half adds a constant-1
//              column that carries the (halved) first-layer bias through the MMA
//   layer 1    one thread issues tcgen05.mma: D[0:64) = A0 W1^T / 2 and
//              D[64:128) = A1 W1^T / 2 (M 128, N 64, K 48), commit to an mbarrier
//   epilogue   each thread reads its 32 columns of its lane of D (y, dy), writes
//              h = y(1+t) and dh = (1+t)(1+y(1-t)) dy (t = tanh y) as BF16 into
//              the rows of A0/A1 (K 64)
//   layer 2    D[0:64) = A0 W2^T / 2, D[64:128) = A1 W2^T / 2
//   output     y += b2 / 2; du/dr = w3 . ((1+t)(1+y(1-t)) dy), u = w3 . y(1+t) + b3,
//              each half over its 32 units, summed through shared memory; the
//              force factor -du/dr / r goes to both entries of the pair
// The weights are staged once per CTA; the CTA walks tiles with a grid stride.
constexpr int TC_M = 128;
constexpr int TC_THREADS = 2 * TC_M;  // two threads per pair
constexpr int TC_N = MLP_H;           // 64 hidden units
constexpr int TC_K1 = 48;             // 32 features, bias column, zero padding
constexpr int TC_K2 = MLP_H;          // 64 units (the second-layer bias is added after the MMA)
constexpr uint32_t TC_COLS = 128;     // tensor-memory columns: values 0..63, tangents 64..127
constexpr int TC_WAIT = 1 << 22;      // polls of an mbarrier before giving up
constexpr int TC_CTAS_PER_SM = 4;     // tensor memory (4 x 128 columns) and shared memory allow four

struct __align__(128) TcShared {
    __nv_bfloat16 a[2 * TC_M * TC_K2];   // A0 | A1, layer 1 (K1) overlaid by layer 2 (K2)
    __nv_bfloat16 w1[TC_N * TC_K1];      // B operand of layer 1
    __nv_bfloat16 w2[TC_N * TC_K2];      // B operand of layer 2
    __align__(16) float w3[TC_N];
    __align__(16) float b2h[TC_N];        // halved second-layer bias
    __align__(8) float2 part[TC_M];       // second half's (u, du/dr) partial sums
    uint64_t mbar;
    uint32_t tmem;
    int stop;
};

__device__ __forceinline__ void st_row16(__nv_bfloat16* base, int row, int k, int K, uint4 v) {
    *reinterpret_cast<uint4*>(reinterpret_cast<char*>(base) + tc::core_offset(row, k, K)) = v;
}

template <bool ENERGY>
__global__ void __launch_bounds__(TC_THREADS, TC_CTAS_PER_SM) k_mlp_tc(DevSys<float> s) {
    extern __shared__ __align__(1024) unsigned char tc_smem[];
    TcShared& sh = *reinterpret_cast<TcShared*>(tc_smem);
    const int tid = threadIdx.x, warp = tid >> 5;
    const int row = tid & (TC_M - 1), half = tid >> 7;
    const MlpWeights* __restrict__ W = s.mlp;
    // B operands: halved weights, halved bias in the constant column
    for (int e = tid; e < TC_N * TC_K1; e += TC_THREADS) {
        const int n = e / TC_K1, k = e % TC_K1;
        const float v = k < MLP_NB ? __bfloat162float(W->W1[n * MLP_NB + k]) : (k == MLP_NB ? W->b1[n] : 0.f);
        *reinterpret_cast<__nv_bfloat16*>(reinterpret_cast<char*>(sh.w1) + tc::core_offset(n, k, TC_K1)) =
            __float2bfloat16(0.5f * v);
    }
    for (int e = tid; e < TC_N * TC_K2; e += TC_THREADS) {
        const int n = e / TC_K2, k = e % TC_K2;
        *reinterpret_cast<__nv_bfloat16*>(reinterpret_cast<char*>(sh.w2) + tc::core_offset(n, k, TC_K2)) =
            __float2bfloat16(0.5f * __bfloat162float(W->W2[n * MLP_H + k]));
    }
    for (int e = tid; e < TC_N; e += TC_THREADS) {
        sh.w3[e] = W->w3[e];
        sh.b2h[e] = 0.5f * W->b2[e];
    }
    if (tid == 0) {
        tc::mbar_init(&sh.mbar, 1);
        sh.stop = s.ctrl->abort;
    }
    if (warp == 0) tc::tmem_alloc(&sh.tmem, TC_COLS);
    tc::fence_async_smem();
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tmem = sh.tmem;
    const uint32_t lanes = tmem + ((uint32_t)((warp & 3) * 32) << 16);  // this warp's 32 lanes
    const int c0 = 32 * half;                                           // this half's columns
    const float rc = W->rc, b3 = W->b3;
    const float wid = rc / (MLP_NB - 1);
    const float invw2 = 1.0f / (wid * wid), inv_w = 1.0f / wid;
    const float pirc = 3.14159265358979f / rc;
    const int np = min(*s.mlp_npairs, s.mlp_pairs_cap);
    const int ntl = (np + TC_M - 1) / TC_M;
    const uint32_t idesc = tc::idesc_bf16(TC_M, TC_N);
    const uint32_t a_base = tc::smem_addr(sh.a), w1_base = tc::smem_addr(sh.w1), w2_base = tc::smem_addr(sh.w2);
    __nv_bfloat16* A0 = sh.a;
    float* __restrict__ pf = s.mlp_pf;
    float* __restrict__ pu = s.mlp_pu;
    uint32_t parity = 0;
    bool ok = sh.stop == 0;
    // fault injection: no MMA is issued and a short wait limit runs out
    const bool fault = s.tc_fault != 0;
    const int wait_limit = fault ? (1 << 12) : TC_WAIT;
    for (int tile = blockIdx.x; ok && tile < ntl; tile += gridDim.x) {
        const int p = tile * TC_M + row;
        const bool valid = p < np;
        const int4 rec = valid ? s.mlp_pairs[p] : make_int4(__float_as_int(rc), 0, 0, 0);
        const float r = __int_as_float(rec.x);
        // ---- features ----------------------------------------------------------
        {
            __nv_bfloat16* A1 = A0 + TC_M * TC_K1;
            const float fc = 0.5f * (__cosf(pirc * r) + 1.f);
            const float dfc = -0.5f * pirc * __sinf(pirc * r);
            // g_k = exp(-(t - k)^2 / 2), t = r / w, by the product recurrence
            // g_{k+2} = g_k exp(2 (t - k) - 2) (two exponentials per block of
            // eight bases instead of eight); dphi_k/dr = g_k (A + k B) with
            // A = dfc - r fc / w^2, B = fc / w.  Pairs of bases in packed FP32x2.
            const float t = r * inv_w;
            const float B = fc * inv_w;
            const f32x2 fc2 = f2(fc, fc);
            const f32x2 twoB = f2(2.f * B, 2.f * B);
            const float A = dfc - r * invw2 * fc;
            const f32x2 em4 = f2(0.018315638888734179f, 0.018315638888734179f);  // e^-4
#pragma unroll
            for (int gg = 0; gg < 2; ++gg) {
                const int g = 2 * half + gg;  // block of eight bases
                unsigned int ph[4], dp[4];
                const float u = t - (float)(8 * g);
                const float g0 = __expf(-0.5f * u * u);
                const float e1 = __expf(u - 0.5f);                  // g_{k+1} / g_k at k = 8g
                const float R0 = e1 * e1 * 0.36787944117144233f;    // g_{k+2} / g_k
                f32x2 gv = f2(g0, g0 * e1);
                f32x2 rv = f2(R0, R0 * 0.1353352832366127f);        // (g_{k+2}/g_k, g_{k+3}/g_{k+1})
                f32x2 cv = f2(A + (float)(8 * g) * B, A + (float)(8 * g + 1) * B);
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    float v0, v1, d0, d1;
                    f2split(f2mul(gv, fc2), v0, v1);
                    f2split(f2mul(gv, cv), d0, d1);
                    ph[q] = pack_bf16x2(v0, v1);
                    dp[q] = pack_bf16x2(d0, d1);
                    gv = f2mul(gv, rv);
                    rv = f2mul(rv, em4);
                    cv = f2add(cv, twoB);
                }
                st_row16(A0, row, 8 * g, TC_K1, make_uint4(ph[0], ph[1], ph[2], ph[3]));
                st_row16(A1, row, 8 * g, TC_K1, make_uint4(dp[0], dp[1], dp[2], dp[3]));
            }
            if (half == 0) {
                st_row16(A0, row, 32, TC_K1, make_uint4(pack_bf16x2(1.f, 0.f), 0u, 0u, 0u));
                st_row16(A0, row, 40, TC_K1, make_uint4(0u, 0u, 0u, 0u));
                st_row16(A1, row, 32, TC_K1, make_uint4(0u, 0u, 0u, 0u));
                st_row16(A1, row, 40, TC_K1, make_uint4(0u, 0u, 0u, 0u));
            }
        }
        tc::fence_async_smem();
        tc::fence_before_sync();
        __syncthreads();
        tc::fence_after_sync();
        if (tid == 0 && !fault) {
            constexpr uint32_t sbo = (TC_K1 / 8) * 128;
#pragma unroll
            for (int ks = 0; ks < TC_K1 / 16; ++ks) {
                const uint64_t db = tc::smem_desc(w1_base + ks * 256, 128, sbo);
                tc::mma(tmem, tc::smem_desc(a_base + ks * 256, 128, sbo), db, idesc, ks > 0);
                tc::mma(tmem + 64, tc::smem_desc(a_base + TC_M * TC_K1 * 2 + ks * 256, 128, sbo), db, idesc,
                        ks > 0);
            }
            tc::commit(&sh.mbar);
        }
        if (!__syncthreads_and(tc::mbar_wait(&sh.mbar, parity, wait_limit))) {
            ok = false;
            break;
        }
        parity ^= 1u;
        tc::fence_after_sync();
        // ---- layer-1 epilogue: h and dh rows of the layer-2 A operands -------------
        {
            __nv_bfloat16* A1 = A0 + TC_M * TC_K2;
#pragma unroll
            for (int c = c0; c < c0 + 32; c += 8) {
                float y[8], dy[8];
                tc::tmem_ld8x2(lanes + c, lanes + 64 + c, y, dy);
                unsigned int hw[4], dw[4];
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    const f32x2 yv = f2(y[2 * j], y[2 * j + 1]);
                    const f32x2 tv = f2(tanh_hw(y[2 * j]), tanh_hw(y[2 * j + 1]));
                    const f32x2 hv = f2fma(yv, tv, yv);  // y (1 + t)
                    const f32x2 dv = f2mul(silu_tangent_factor(yv, tv), f2(dy[2 * j], dy[2 * j + 1]));
                    float h0, h1, d0, d1;
                    f2split(hv, h0, h1);
                    f2split(dv, d0, d1);
                    hw[j] = pack_bf16x2(h0, h1);
                    dw[j] = pack_bf16x2(d0, d1);
                }
                st_row16(A0, row, c, TC_K2, make_uint4(hw[0], hw[1], hw[2], hw[3]));
                st_row16(A1, row, c, TC_K2, make_uint4(dw[0], dw[1], dw[2], dw[3]));
            }
        }
        tc::fence_async_smem();
        tc::fence_before_sync();
        __syncthreads();
        tc::fence_after_sync();
        if (tid == 0 && !fault) {
            constexpr uint32_t sbo = (TC_K2 / 8) * 128;
#pragma unroll
            for (int ks = 0; ks < TC_K2 / 16; ++ks) {
                const uint64_t db = tc::smem_desc(w2_base + ks * 256, 128, sbo);
                tc::mma(tmem, tc::smem_desc(a_base + ks * 256, 128, sbo), db, idesc, ks > 0);
                tc::mma(tmem + 64, tc::smem_desc(a_base + TC_M * TC_K2 * 2 + ks * 256, 128, sbo), db, idesc,
                        ks > 0);
            }
            tc::commit(&sh.mbar);
        }
        if (!__syncthreads_and(tc::mbar_wait(&sh.mbar, parity, wait_limit))) {
            ok = false;
            break;
        }
        parity ^= 1u;
        tc::fence_after_sync();
        // ---- output layer: this half's 32 units --------------------------------------
        f32x2 u2 = f2(0.f, 0.f), du2 = f2(0.f, 0.f);
#pragma unroll
        for (int c = c0; c < c0 + 32; c += 8) {
            float y[8], dy[8];
            tc::tmem_ld8x2(lanes + c, lanes + 64 + c, y, dy);
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const float2 bb = *reinterpret_cast<const float2*>(sh.b2h + c + 2 * j);
                const float2 ww = *reinterpret_cast<const float2*>(sh.w3 + c + 2 * j);
                const f32x2 yv = f2add(f2(y[2 * j], y[2 * j + 1]), f2(bb.x, bb.y));
                float y0, y1;
                f2split(yv, y0, y1);
                const f32x2 tv = f2(tanh_hw(y0), tanh_hw(y1));
                const f32x2 wv = f2(ww.x, ww.y);
                du2 = f2fma(wv, f2mul(silu_tangent_factor(yv, tv), f2(dy[2 * j], dy[2 * j + 1])), du2);
                if (ENERGY) u2 = f2fma(wv, f2fma(yv, tv, yv), u2);
            }
        }
        float u, du;
        {
            float a, b;
            f2split(du2, a, b);
            du = a + b;
            f2split(u2, a, b);
            u = a + b;
        }
        if (half == 1) sh.part[row] = make_float2(u, du);
        // tensor-memory reads and shared-memory operands of this tile are done
        tc::fence_before_sync();
        __syncthreads();
        tc::fence_after_sync();
        if (half == 0 && valid) {
            const float2 o = sh.part[row];
            const float sv = -(du + o.y) / r;
            pf[rec.y] = sv;
            pf[rec.z] = sv;
            if (ENERGY) {
                pu[rec.y] = u + o.x + b3;
                pu[rec.z] = u + o.x + b3;
            }
        }
    }
    if (!ok && sh.stop == 0) {
        // a commit never arrived: record it, give the MMAs in flight one more
        // bounded wait, then release the tensor memory
        if (tid == 0) {
            atomicOr(&s.ctrl->err, ERRBIT_TIMEOUT);
            s.ctrl->abort = 1;
        }
        tc::mbar_wait(&sh.mbar, parity, wait_limit);
    }
    tc::fence_before_sync();
    __syncthreads();
    if (warp == 0) tc::tmem_free(tmem, TC_COLS);
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

// ---- FP64 handles: the learned potential in double on the CUDA cores --------
// u(r) and du/dr of one pair in double from the BF16 weights (exact upcast):
// the same network as the tensor-core tile, without any rounding to BF16 of
// the features or activations, so an FP64 handle gets the network's exact
// value (to double rounding), as the reference path for the BF16 one.
__device__ __forceinline__ double silu_d(double z, double& dsilu) {
    const double sg = 1.0 / (1.0 + exp(-z));
    dsilu = sg * (1.0 + z * (1.0 - sg));
    return z * sg;
}

__device__ void mlp_pair_f64(const MlpWeights* __restrict__ W, double r, double& u, double& du) {
    const double rc = (double)W->rc;
    const double w = rc / (MLP_NB - 1);
    const double inv_2w2 = 1.0 / (2.0 * w * w);
    double sn, cs;
    sincospi(r / rc, &sn, &cs);
    const double fc = 0.5 * (cs + 1.0);
    const double dfc = -0.5 * (CUDART_PI / rc) * sn;
    double phi[MLP_NB], dphi[MLP_NB];
#pragma unroll 4
    for (int k = 0; k < MLP_NB; ++k) {
        const double d = r - rc * k / (MLP_NB - 1);
        const double g = exp(-d * d * inv_2w2);
        phi[k] = g * fc;
        dphi[k] = g * (dfc - 2.0 * d * inv_2w2 * fc);
    }
    double h1[MLP_H], dh1[MLP_H];
    for (int a = 0; a < MLP_H; ++a) {
        double z = (double)W->b1[a], dz = 0.0;
        const __nv_bfloat16* row = W->W1 + a * MLP_NB;
#pragma unroll 8
        for (int k = 0; k < MLP_NB; ++k) {
            const double wk = (double)__bfloat162float(row[k]);
            z = fma(wk, phi[k], z);
            dz = fma(wk, dphi[k], dz);
        }
        double s1;
        h1[a] = silu_d(z, s1);
        dh1[a] = s1 * dz;
    }
    u = (double)W->b3;
    du = 0.0;
    for (int a = 0; a < MLP_H; ++a) {
        double z = (double)W->b2[a], dz = 0.0;
        const __nv_bfloat16* row = W->W2 + a * MLP_H;
#pragma unroll 8
        for (int k = 0; k < MLP_H; ++k) {
            const double wk = (double)__bfloat162float(row[k]);
            z = fma(wk, h1[k], z);
            dz = fma(wk, dh1[k], dz);
        }
        double s1;
        const double h2 = silu_d(z, s1);
        u = fma((double)W->w3[a], h2, u);
        du = fma((double)W->w3[a], s1 * dz, du);
    }
}

// Thread per particle over its full list (each pair from both ends with the
// same arithmetic, so F_ij = -F_ji exactly): force, energy (u per pair, half
// of it to each end by the energy pass) and virial sums in list order.
template <bool ENERGY>
__global__ void __launch_bounds__(TILE) k_mlp_f64(DevSys<double> s, int cur) {
    if (s.ctrl->abort) return;
    const MlpWeights* __restrict__ W = s.mlp;
    const double rc = (double)W->rc, rc2 = rc * rc;
    const V4<double>* __restrict__ P = s.pos[cur];
    const int4* __restrict__ nbr4 = reinterpret_cast<const int4*>(s.nbr);
    const size_t stride = (size_t)s.stride;
    for (int t = blockIdx.x; t < s.ntiles; t += gridDim.x) {
        const Tile tl = s.tiles[t];
        if ((int)threadIdx.x >= tl.count) continue;
        const RepGeom<double>& g = s.reps[tl.rep];
        const double L0 = g.L[0], L1 = g.L[1], L2 = g.L[2];
        const int i = tl.start + threadIdx.x;
        const V4<double> xi = ld4<double>(P + i);
        const double xim = xi.x - L0, yim = xi.y - L1, zim = xi.z - L2;
        const int n = s.nbr_cnt[i];
        double fx = 0.0, fy = 0.0, fz = 0.0, eu = 0.0, ew = 0.0;
        for (int k = 0; k < n; ++k) {
            const int4 q = nbr4[(size_t)(k >> 2) * stride + i];
            const int e = (k & 3) == 0 ? q.x : (k & 3) == 1 ? q.y : (k & 3) == 2 ? q.z : q.w;
            const V4<double> xj = ld4<double>(P + nbr_slot(e));
            const int code = nbr_code(e);
            const double dx = shifted_diff(xi.x, xim, xj.x, L0, code & 3);
            const double dy = shifted_diff(xi.y, yim, xj.y, L1, (code >> 2) & 3);
            const double dz = shifted_diff(xi.z, zim, xj.z, L2, code >> 4);
            const double r2 = dx * dx + dy * dy + dz * dz;
            if (!(r2 < rc2)) continue;
            const double r = sqrt(r2);
            double u, du;
            mlp_pair_f64(W, r, u, du);
            const double fr = -du / r;  // F_i = -du/dr r_ij / r
            fx = fma(fr, dx, fx);
            fy = fma(fr, dy, fy);
            fz = fma(fr, dz, fz);
            if (ENERGY) {
                eu += u;
                ew = fma(fr, r2, ew);
            }
        }
        s.mlp_fT[i] = mk4<double>(fx, fy, fz, eu);
        if (ENERGY) s.mlp_wT[i] = ew;
    }
}

static_assert(sizeof(TcShared) <= 227 * 1024 / TC_CTAS_PER_SM, "tcgen05 tile CTA too large");

// The learned potential's force pass runs in FP32/BF16 for both precisions of
// the handle: the tensor-core kernel reads only the pair records and writes
// the per-entry values, so one FP32 instantiation serves both.
template <class T>
static DevSys<float> as_float(const DevSys<T>& s) {
    DevSys<float> f;
    memset(&f, 0, sizeof(f));
    f.ctrl = s.ctrl;
    f.mlp = s.mlp;
    f.mlp_pf = s.mlp_pf;
    f.mlp_pu = s.mlp_pu;
    f.mlp_pairs = s.mlp_pairs;
    f.mlp_pairs_cap = s.mlp_pairs_cap;
    f.mlp_npairs = s.mlp_npairs;
    f.tc_fault = s.tc_fault;
    return f;
}

cudaError_t prepare_mlp_tc() {
    cudaError_t e = cudaFuncSetAttribute(k_mlp_tc<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)sizeof(TcShared));
    if (e != cudaSuccess) return e;
    return cudaFuncSetAttribute(k_mlp_tc<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(TcShared));
}

template <class T>
int Launch<T>::mlp(const DevSys<T>& s, int cur, bool energy, cudaStream_t st) {
    if constexpr (sizeof(T) == 8) {
        // FP64 handle: the network in double on the CUDA cores
        if (energy) k_mlp_f64<true><<<s.ntiles, TILE, 0, st>>>(s, cur);
        else k_mlp_f64<false><<<s.ntiles, TILE, 0, st>>>(s, cur);
        return 1;
    }
    return mlp_tc(s, cur, energy, st);
}

template <class T>
int Launch<T>::mlp_tc(const DevSys<T>& s, int cur, bool energy, cudaStream_t st) {
    cudaMemsetAsync(s.mlp_npairs, 0, sizeof(int), st);
    const int tblocks = sm_count() * TC_CTAS_PER_SM;
    k_mlp_stage<T><<<sm_count() * ESPP_STAGE_GRID, TILE, 0, st>>>(s, cur);
    if (energy) {
        k_mlp_tc<true><<<tblocks, TC_THREADS, sizeof(TcShared), st>>>(as_float(s));
        k_mlp_gather<T, true><<<s.ntiles, TILE, 0, st>>>(s, cur);
    } else {
        k_mlp_tc<false><<<tblocks, TC_THREADS, sizeof(TcShared), st>>>(as_float(s));
        k_mlp_gather<T, false><<<s.ntiles, TILE, 0, st>>>(s, cur);
    }
    return 3;
}

template <class T>
int Launch<T>::mlp_rev(const DevSys<T>& s, cudaStream_t st) {
    const int nb = s.mlp_nuscan;
    k_mlp_count<T><<<s.ntiles, TILE, 0, st>>>(s);
    k_uscan_reduce<<<nb, SCAN_THREADS, 0, st>>>(s.mlp_ucount, s.N, s.mlp_uscan_part);
    k_uscan_top<<<1, SCAN_THREADS, 0, st>>>(s.mlp_uscan_part, nb, s.mlp_nupper);
    k_uscan_down<<<nb, SCAN_THREADS, 0, st>>>(s.mlp_ucount, s.N, s.mlp_uscan_part, s.mlp_uoff);
    k_mlp_rev<T><<<s.ntiles, TILE, 0, st>>>(s);
    return 5;
}

template int Launch<float>::mlp(const DevSys<float>&, int, bool, cudaStream_t);
template int Launch<double>::mlp(const DevSys<double>&, int, bool, cudaStream_t);
template int Launch<float>::mlp_tc(const DevSys<float>&, int, bool, cudaStream_t);
template int Launch<double>::mlp_tc(const DevSys<double>&, int, bool, cudaStream_t);
template int Launch<float>::mlp_rev(const DevSys<float>&, cudaStream_t);
template int Launch<double>::mlp_rev(const DevSys<double>&, cudaStream_t);

}  // namespace espp

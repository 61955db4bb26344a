// Force-matching training of the learned pair potential on the tensor cores.
//
// Loss over a batch of F frames of n sites: L = sum |e_i|^2 / (F n) with
// e_i = F_pair,i + F_bond,i - Y_i (Y: mapped forces).  Since
// F_pair,i = sum_j -u'(r_ij) r_ij_hat, the gradient is a sum over unordered
// pairs of w_ij d u'(r_ij) / d theta with
//   w_ij = -2 ((e_i - e_j) . r_ij_hat) / (F n)
// (the two ordered terms of a pair share u').  The pairs are the records of
// the list (each unordered pair once, in an order fixed by the list); those
// beyond the cutoff get w = 0 and contribute exact zeros.
//
// The gradient runs on the tcgen05 tensor cores (k_mlp_grad below: tiles of
// 128 pairs, accumulators in tensor memory).  Each CTA writes one partial in
// a fixed order and two small kernels add the partials in a fixed order: the
// gradient is deterministic.  Adam then updates FP32 master weights and
// refreshes the BF16 copy the kernels read.
#include "mlp_common.cuh"
#include "tc_ptx.cuh"

namespace espp {

constexpr int G_W1 = 0;
constexpr int G_B1 = MLP_H * MLP_NB;
constexpr int G_W2 = G_B1 + MLP_H;
constexpr int G_B2 = G_W2 + MLP_H * MLP_H;
constexpr int G_W3 = G_B2 + MLP_H;
constexpr int NGRAD = G_W3 + MLP_H;  // every parameter but b3 (whose gradient is 0)

// ---- the gradient tile on the tcgen05 tensor cores -------------------------------
// A CTA walks tiles of 128 pair records, one pair per tensor-memory lane.
// Per tile, with y = z / 2 and t = tanh(y) as in the inference tile (halved
// weights, the first-layer bias carried by a constant feature):
//   L1    [y1 | dy1] = [phi | dphi] W1^T / 2                  D1, tensor memory
//   epi1  h1 = y1 (1 + t1), dh1 = (1 + t1)(1 + y1 (1 - t1)) dy1   (BF16 rows)
//   L2    [y2 | dy2] = [h1 | dh1] W2^T / 2                      D2
//   epi2  with y2 += b2 / 2, dz2 = 2 dy2, s1 = silu'(z2), s2 = silu''(z2):
//         az2 = w w3 s2 dz2, adz2 = w w3 s1, w dh2 = w s1 dz2  (w: the row weight)
//   BW    [ah1 | adh1] = [az2 | adz2] W2                        D2 again
//   G2    dW2 += az2^T h1 + adz2^T dh1, db2 += az2^T 1, dw3 += (w dh2)^T 1
//   epi3  az1 = ah1 silu'(z1) + adh1 silu''(z1) dz1, adz1 = adh1 silu'(z1)
//   G1    dW1 += az1^T phi + adz1^T dphi, db1 += az1^T 1
// Each pair's quantities are written once, as 16-byte pieces of its row, into
// row buffers that serve twice: as K-major operands of the forward and
// backward products (rows = pairs) and, read through MN-major descriptors, as
// the operands of the G products, which contract over the tile's 128 pairs
// (K = pairs) and accumulate in tensor memory over all of the CTA's tiles.
// Bias and output-weight sums ride as a constant-1 column of the rows.  M is
// 128 throughout: dW2 is the top half of one product (rows az2, w dh2
// against [h1 | 1]) plus the bottom half of another (rows w dh2, adz2
// against dh1), dW1 likewise.  The CTA's 16 warps split the 64 units of
// every row four ways (warps w, w + 4, w + 8, w + 12 share the tensor-memory
// lanes of pairs 32 (w % 4) ..).  Each CTA writes one partial in a fixed
// order: the gradient is deterministic.
constexpr int GT_M = 128;                 // pairs per tile
constexpr int GT_NG = 4;                  // warps per tensor-memory lane quadrant (column groups)
constexpr int GT_THREADS = GT_M * GT_NG;
constexpr int GT_CW = MLP_H / GT_NG;      // units per thread in the epilogues (16)
constexpr int GT_K1 = 48;
constexpr int GT_H = MLP_H;
constexpr uint32_t GT_COLS = 512;
constexpr uint32_t GT_D1 = 0, GT_D2 = 128, GT_G2A = 256, GT_G2B = 336, GT_G1A = 400, GT_G1B = 448;
// row buffers, one row per pair (bf16 columns):
//   F  phi (0..31), 1 (32), 0 (33..47), dphi (48..79), 0 (80..95)
//   H  h1 (0..63), 1 (64), 0 (65..79), dh1 (80..143)
//   Z  az2 (0..63), w dh2 (64..127), adz2 (128..191)
//   A1 az1 (0..63), adz1 (64..127)
constexpr int F_COLS = 96, H_COLS = 144, Z_COLS = 192, A1_COLS = 128;
__host__ __device__ constexpr uint32_t rsbo(int cols) { return (uint32_t)(cols / 8) * 128; }  // stride of 8-pair groups
constexpr int GT_WAIT = 1 << 22;

struct __align__(1024) GradShared {
    unsigned char f[GT_M * F_COLS * 2];
    unsigned char h[GT_M * H_COLS * 2];
    unsigned char z[GT_M * Z_COLS * 2];
    unsigned char a1[GT_M * A1_COLS * 2];
    unsigned char w1h[GT_H * GT_K1 * 2];  // W1 / 2 with the bias column
    unsigned char w2h[GT_H * GT_H * 2];   // W2 / 2
    unsigned char w2t[GT_H * GT_H * 2];   // W2^T
    float b2h[GT_H];
    float w3[GT_H];
    float pr[2][GT_M];  // distance and row weight of each pair slot, this tile and the next
    float pw[2][GT_M];
    uint64_t mbar;
    uint32_t tmem;
    int stop;
};

__device__ __forceinline__ void st_bf(unsigned char* base, uint32_t off, float v) {
    *reinterpret_cast<__nv_bfloat16*>(base + off) = __float2bfloat16(v);
}
__device__ __forceinline__ float gt_tanh(float y) {
    float t;
    asm("tanh.approx.f32 %0, %1;" : "=f"(t) : "f"(y));
    return t;
}
// eight consecutive columns c.. of pair p's row in a buffer of `cols` columns
__device__ __forceinline__ void st_row8(unsigned char* base, int p, int c, int cols, uint4 v) {
    *reinterpret_cast<uint4*>(base + tc::core_offset(p, c, cols)) = v;
}
// a K-major descriptor (rows = pairs, K = columns) at column c0
__device__ __forceinline__ uint64_t row_desc(uint32_t base, int c0, int cols) {
    return tc::smem_desc(base + (c0 / 8) * 128, 128, rsbo(cols));
}
// an MN-major descriptor (M or N = columns from c0, K = the pairs of K-step ks)
__device__ __forceinline__ uint64_t col_desc(uint32_t base, int c0, int cols, int ks) {
    return tc::smem_desc(base + (c0 / 8) * 128 + ks * 2 * rsbo(cols), rsbo(cols), 128);
}

// Distance and row weight of pair record k (r = rc and w = 0 past the end or
// beyond the cutoff): w = scale ((e_i - e_j) . r_ij) / r.
template <class T>
__device__ __forceinline__ void pair_weight(const DevSys<T>& s, const V4<T>* __restrict__ P,
                                            const float4* __restrict__ err, int4 up, bool valid, float rc2,
                                            float scale, float& r, float& w) {
    if (!valid) return;
    const int stride = s.stride;
    const int i = (up.x >> 2) % stride, j = nbr_slot(up.z);
    const RepGeom<T>& geo = s.reps[up.w];
    const T L0 = geo.L[0], L1 = geo.L[1], L2 = geo.L[2];
    const V4<T> xi = ld4<T>(P + i), xj = ld4<T>(P + j);
    const float4 ei = err[i], ej = err[j];
    const int code = nbr_code(up.z);
    const float dx = (float)shifted_diff(xi.x, (T)(xi.x - L0), xj.x, L0, code & 3);
    const float dy = (float)shifted_diff(xi.y, (T)(xi.y - L1), xj.y, L1, (code >> 2) & 3);
    const float dz = (float)shifted_diff(xi.z, (T)(xi.z - L2), xj.z, L2, code >> 4);
    const float r2 = __fadd_rn(__fadd_rn(__fmul_rn(dx, dx), __fmul_rn(dy, dy)), __fmul_rn(dz, dz));
    if (r2 < rc2) {
        r = sqrtf(r2);
        w = scale * ((ei.x - ej.x) * dx + (ei.y - ej.y) * dy + (ei.z - ej.z) * dz) / r;
    }
}

template <class T>
__global__ void __launch_bounds__(GT_THREADS, 1) k_mlp_grad(DevSys<T> s, int cur, const float4* __restrict__ err,
                                                          float scale, float* __restrict__ partials) {
    extern __shared__ __align__(1024) unsigned char gsm_raw[];
    GradShared& sh = *reinterpret_cast<GradShared*>(gsm_raw);
    const int tid = threadIdx.x, warp = tid >> 5;
    const int p = 32 * (warp & 3) + (tid & 31);  // this thread's pair slot (tensor-memory lane)
    const int grp = warp >> 2;                   // its column group
    const MlpWeights* __restrict__ W = s.mlp;
    for (int e = tid; e < GT_H * GT_K1; e += GT_THREADS) {
        const int n = e / GT_K1, k = e % GT_K1;
        const float v = k < MLP_NB ? __bfloat162float(W->W1[n * MLP_NB + k]) : (k == MLP_NB ? W->b1[n] : 0.f);
        st_bf(sh.w1h, tc::core_offset(n, k, GT_K1), 0.5f * v);
    }
    for (int e = tid; e < GT_H * GT_H; e += GT_THREADS) {
        const int n = e / GT_H, k = e % GT_H;
        st_bf(sh.w2h, tc::core_offset(n, k, GT_H), 0.5f * __bfloat162float(W->W2[n * GT_H + k]));
        st_bf(sh.w2t, tc::core_offset(n, k, GT_H), __bfloat162float(W->W2[k * GT_H + n]));  // (i, o) = W2[o][i]
    }
    for (int e = tid; e < GT_H; e += GT_THREADS) {
        sh.w3[e] = W->w3[e];
        sh.b2h[e] = 0.5f * W->b2[e];
    }
    // the constant columns of this pair's rows
    if (grp == 0) {
        st_row8(sh.f, p, 32, F_COLS, make_uint4(pack_bf16x2(1.f, 0.f), 0u, 0u, 0u));
        st_row8(sh.f, p, 40, F_COLS, make_uint4(0u, 0u, 0u, 0u));
        st_row8(sh.f, p, 80, F_COLS, make_uint4(0u, 0u, 0u, 0u));
        st_row8(sh.f, p, 88, F_COLS, make_uint4(0u, 0u, 0u, 0u));
    } else if (grp == 1) {
        st_row8(sh.h, p, 64, H_COLS, make_uint4(pack_bf16x2(1.f, 0.f), 0u, 0u, 0u));
        st_row8(sh.h, p, 72, H_COLS, make_uint4(0u, 0u, 0u, 0u));
    }
    if (tid == 0) {
        tc::mbar_init(&sh.mbar, 1);
        sh.stop = s.ctrl->abort;
    }
    if (warp == 0) tc::tmem_alloc(&sh.tmem, GT_COLS);
    tc::fence_async_smem();
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tmem = sh.tmem;
    const uint32_t lanes = tmem + ((uint32_t)(32 * (warp & 3)) << 16);
    const float rc = W->rc, rc2 = rc * rc;
    const float wid = rc / (MLP_NB - 1);
    const float inv2w2 = 0.5f / (wid * wid), invw2 = 1.0f / (wid * wid);
    const float pirc = 3.14159265358979f / rc;
    const V4<T>* __restrict__ P = s.pos[cur];
    const int nu = min(*s.mlp_nupper, s.mlp_upper_cap);
    const int ntl = (nu + GT_M - 1) / GT_M;
    const uint32_t fb = tc::smem_addr(sh.f), hb = tc::smem_addr(sh.h), zb = tc::smem_addr(sh.z),
                   ab = tc::smem_addr(sh.a1), w1 = tc::smem_addr(sh.w1h), w2 = tc::smem_addr(sh.w2h),
                   w2t = tc::smem_addr(sh.w2t);
    const uint32_t id64 = tc::idesc_bf16(GT_M, 64);
    // G products: both operands MN-major (transpose bits 15 and 16)
    const uint32_t gt = (1u << 15) | (1u << 16);
    const uint32_t id80t = tc::idesc_bf16(GT_M, 80) | gt, id64t = id64 | gt, id48t = tc::idesc_bf16(GT_M, 48) | gt,
                   id32t = tc::idesc_bf16(GT_M, 32) | gt;
    const bool fault = s.tc_fault != 0;
    const int wait_limit = fault ? (1 << 12) : GT_WAIT;
    uint32_t parity = 0;
    bool ok = sh.stop == 0, acc = false;
    // one commit of the MMAs issued by thread 0, waited for by the whole CTA
    auto sync_mma = [&]() -> bool {
        if (tid == 0) tc::commit(&sh.mbar);
        const bool done = __syncthreads_and(tc::mbar_wait(&sh.mbar, parity, wait_limit));
        parity ^= 1u;
        tc::fence_after_sync();
        return done;
    };
    auto sync_smem = [&]() {
        tc::fence_async_smem();
        tc::fence_before_sync();
        __syncthreads();
        tc::fence_after_sync();
    };
    const int c0 = grp * GT_CW;  // this thread's 16 units of each layer
    // the pair data of the first tile (column group 0 loads and shares it)
    if (grp == 0) {
        const int k = blockIdx.x * GT_M + p;
        float r = rc, w = 0.f;
        pair_weight<T>(s, P, err, k < nu ? s.mlp_upper[k] : make_int4(0, 0, 0, 0), k < nu, rc2, scale, r, w);
        sh.pr[0][p] = r;
        sh.pw[0][p] = w;
    }
    __syncthreads();
    int buf = 0;
    for (int tile = blockIdx.x; ok && tile < ntl; tile += gridDim.x) {
        // ---- the pair: distance and row weight (shared by its four threads) ------
        const float r = sh.pr[buf][p], wrow = sh.pw[buf][p];
        // the next tile's record, requested now and used after epilogue 2
        const int kn = (tile + gridDim.x) * GT_M + p;
        const bool next_valid = grp == 0 && kn < nu;
        const int4 up_next = next_valid ? s.mlp_upper[kn] : make_int4(0, 0, 0, 0);
        // ---- features 8 grp .. 8 grp + 7 of phi and dphi ---------------------------
        {
            const float fc = 0.5f * (__cosf(pirc * r) + 1.f);
            const float dfc = -0.5f * pirc * __sinf(pirc * r);
            unsigned int ph[4], dp[4];
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                float v[2], dv[2];
#pragma unroll
                for (int hh = 0; hh < 2; ++hh) {
                    const float d = r - wid * (float)(8 * grp + 2 * q + hh);
                    const float gk = __expf(-d * d * inv2w2);
                    v[hh] = gk * fc;
                    dv[hh] = gk * (dfc - d * invw2 * fc);
                }
                ph[q] = pack_bf16x2(v[0], v[1]);
                dp[q] = pack_bf16x2(dv[0], dv[1]);
            }
            st_row8(sh.f, p, 8 * grp, F_COLS, make_uint4(ph[0], ph[1], ph[2], ph[3]));
            st_row8(sh.f, p, 48 + 8 * grp, F_COLS, make_uint4(dp[0], dp[1], dp[2], dp[3]));
        }
        sync_smem();
        if (tid == 0 && !fault) {
#pragma unroll
            for (int ks = 0; ks < GT_K1 / 16; ++ks) {
                const uint64_t db = tc::smem_desc(w1 + ks * 256, 128, (GT_K1 / 8) * 128);
                tc::mma(tmem + GT_D1, row_desc(fb, 16 * ks, F_COLS), db, id64, ks > 0);
                tc::mma(tmem + GT_D1 + 64, row_desc(fb, 48 + 16 * ks, F_COLS), db, id64, ks > 0);
            }
        }
        if (!sync_mma()) {
            ok = false;
            break;
        }
        // ---- epilogue 1: h1, dh1 (two units per packed instruction) -----------------
        {
            float y[16], dy[16];
            tc::tmem_ld16x2(lanes + GT_D1 + c0, lanes + GT_D1 + 64 + c0, y, dy);
            unsigned int hw[8], dw[8];
#pragma unroll
            for (int j = 0; j < 8; ++j) {
                const f32x2 yv = f2(y[2 * j], y[2 * j + 1]);
                const f32x2 tv = f2(gt_tanh(y[2 * j]), gt_tanh(y[2 * j + 1]));
                float h0, h1, d0, d1;
                f2split(f2fma(yv, tv, yv), h0, h1);  // y (1 + t)
                f2split(f2mul(silu_tangent_factor(yv, tv), f2(dy[2 * j], dy[2 * j + 1])), d0, d1);
                hw[j] = pack_bf16x2(h0, h1);
                dw[j] = pack_bf16x2(d0, d1);
            }
            st_row8(sh.h, p, c0, H_COLS, make_uint4(hw[0], hw[1], hw[2], hw[3]));
            st_row8(sh.h, p, c0 + 8, H_COLS, make_uint4(hw[4], hw[5], hw[6], hw[7]));
            st_row8(sh.h, p, 80 + c0, H_COLS, make_uint4(dw[0], dw[1], dw[2], dw[3]));
            st_row8(sh.h, p, 88 + c0, H_COLS, make_uint4(dw[4], dw[5], dw[6], dw[7]));
        }
        sync_smem();
        if (tid == 0 && !fault) {
#pragma unroll
            for (int ks = 0; ks < GT_H / 16; ++ks) {
                const uint64_t db = tc::smem_desc(w2 + ks * 256, 128, (GT_H / 8) * 128);
                tc::mma(tmem + GT_D2, row_desc(hb, 16 * ks, H_COLS), db, id64, ks > 0);
                tc::mma(tmem + GT_D2 + 64, row_desc(hb, 80 + 16 * ks, H_COLS), db, id64, ks > 0);
            }
        }
        if (!sync_mma()) {
            ok = false;
            break;
        }
        // ---- epilogue 2: the reverse seeds (two units per packed instruction) ---------
        // with z = 2 y, t = tanh(y): silu'(z) = (1 + t)(1 + y (1 - t)) / 2,
        // silu''(z) = (1 + t)(1 - t)(1 - y t) / 2
        {
            float y[16], dy[16];
            tc::tmem_ld16x2(lanes + GT_D2 + c0, lanes + GT_D2 + 64 + c0, y, dy);
            unsigned int aw[8], ww[8], dw[8];
            const f32x2 one = f2(1.f, 1.f), mone = f2(-1.f, -1.f), half = f2(0.5f, 0.5f);
            const f32x2 wv2 = f2(wrow, wrow);
#pragma unroll
            for (int j = 0; j < 8; ++j) {
                const int o = c0 + 2 * j;
                const float2 bb = *reinterpret_cast<const float2*>(sh.b2h + o);
                const float2 w3v = *reinterpret_cast<const float2*>(sh.w3 + o);
                const f32x2 yv = f2add(f2(y[2 * j], y[2 * j + 1]), f2(bb.x, bb.y));
                float ya, yb;
                f2split(yv, ya, yb);
                const f32x2 tv = f2(gt_tanh(ya), gt_tanh(yb));
                const f32x2 opt = f2add(tv, one), omt = f2fma(tv, mone, one);
                const f32x2 hopt = f2mul(half, opt);
                const f32x2 s1 = f2mul(hopt, f2fma(yv, omt, one));
                const f32x2 s2 = f2mul(f2mul(hopt, omt), f2fma(f2mul(yv, tv), mone, one));
                const f32x2 dz = f2(2.f * dy[2 * j], 2.f * dy[2 * j + 1]);
                const f32x2 wo = f2mul(wv2, f2(w3v.x, w3v.y));
                float a0, a1, w0, w1, d0, d1;
                f2split(f2mul(f2mul(wo, s2), dz), a0, a1);   // az2
                f2split(f2mul(f2mul(wv2, s1), dz), w0, w1);  // w dh2
                f2split(f2mul(wo, s1), d0, d1);              // adz2
                aw[j] = pack_bf16x2(a0, a1);
                ww[j] = pack_bf16x2(w0, w1);
                dw[j] = pack_bf16x2(d0, d1);
            }
            st_row8(sh.z, p, c0, Z_COLS, make_uint4(aw[0], aw[1], aw[2], aw[3]));
            st_row8(sh.z, p, c0 + 8, Z_COLS, make_uint4(aw[4], aw[5], aw[6], aw[7]));
            st_row8(sh.z, p, 64 + c0, Z_COLS, make_uint4(ww[0], ww[1], ww[2], ww[3]));
            st_row8(sh.z, p, 72 + c0, Z_COLS, make_uint4(ww[4], ww[5], ww[6], ww[7]));
            st_row8(sh.z, p, 128 + c0, Z_COLS, make_uint4(dw[0], dw[1], dw[2], dw[3]));
            st_row8(sh.z, p, 136 + c0, Z_COLS, make_uint4(dw[4], dw[5], dw[6], dw[7]));
        }
        if (grp == 0) {
            // the next tile's pair data, into the other buffer
            float rn = rc, wn = 0.f;
            pair_weight<T>(s, P, err, up_next, next_valid, rc2, scale, rn, wn);
            sh.pr[buf ^ 1][p] = rn;
            sh.pw[buf ^ 1][p] = wn;
        }
        sync_smem();
        if (tid == 0 && !fault) {
#pragma unroll
            for (int ks = 0; ks < GT_H / 16; ++ks) {
                const uint64_t db = tc::smem_desc(w2t + ks * 256, 128, (GT_H / 8) * 128);
                tc::mma(tmem + GT_D2, row_desc(zb, 16 * ks, Z_COLS), db, id64, ks > 0);
                tc::mma(tmem + GT_D2 + 64, row_desc(zb, 128 + 16 * ks, Z_COLS), db, id64, ks > 0);
            }
#pragma unroll
            for (int ks = 0; ks < GT_M / 16; ++ks) {
                tc::mma(tmem + GT_G2A, col_desc(zb, 0, Z_COLS, ks), col_desc(hb, 0, H_COLS, ks), id80t,
                        acc || ks > 0);
                tc::mma(tmem + GT_G2B, col_desc(zb, 64, Z_COLS, ks), col_desc(hb, 80, H_COLS, ks), id64t,
                        acc || ks > 0);
            }
        }
        if (!sync_mma()) {
            ok = false;
            break;
        }
        // ---- epilogue 3: layer-1 adjoints ---------------------------------------------
        {
            float ah[16], adh[16], y[16], dy[16];
            tc::tmem_ld16x2(lanes + GT_D2 + c0, lanes + GT_D2 + 64 + c0, ah, adh);
            tc::tmem_ld16x2(lanes + GT_D1 + c0, lanes + GT_D1 + 64 + c0, y, dy);
            unsigned int aw[8], dw[8];
            const f32x2 one = f2(1.f, 1.f), mone = f2(-1.f, -1.f), half = f2(0.5f, 0.5f);
#pragma unroll
            for (int j = 0; j < 8; ++j) {
                const f32x2 yv = f2(y[2 * j], y[2 * j + 1]);
                const f32x2 tv = f2(gt_tanh(y[2 * j]), gt_tanh(y[2 * j + 1]));
                const f32x2 opt = f2add(tv, one), omt = f2fma(tv, mone, one);
                const f32x2 hopt = f2mul(half, opt);
                const f32x2 s1 = f2mul(hopt, f2fma(yv, omt, one));
                const f32x2 s2 = f2mul(f2mul(hopt, omt), f2fma(f2mul(yv, tv), mone, one));
                const f32x2 adh2 = f2(adh[2 * j], adh[2 * j + 1]);
                const f32x2 dz = f2(2.f * dy[2 * j], 2.f * dy[2 * j + 1]);
                float a0, a1, d0, d1;
                f2split(f2fma(f2(ah[2 * j], ah[2 * j + 1]), s1, f2mul(f2mul(adh2, s2), dz)), a0, a1);  // az1
                f2split(f2mul(adh2, s1), d0, d1);                                                      // adz1
                aw[j] = pack_bf16x2(a0, a1);
                dw[j] = pack_bf16x2(d0, d1);
            }
            st_row8(sh.a1, p, c0, A1_COLS, make_uint4(aw[0], aw[1], aw[2], aw[3]));
            st_row8(sh.a1, p, c0 + 8, A1_COLS, make_uint4(aw[4], aw[5], aw[6], aw[7]));
            st_row8(sh.a1, p, 64 + c0, A1_COLS, make_uint4(dw[0], dw[1], dw[2], dw[3]));
            st_row8(sh.a1, p, 72 + c0, A1_COLS, make_uint4(dw[4], dw[5], dw[6], dw[7]));
        }
        sync_smem();
        if (tid == 0 && !fault) {
#pragma unroll
            for (int ks = 0; ks < GT_M / 16; ++ks) {
                const uint64_t da = col_desc(ab, 0, A1_COLS, ks);
                tc::mma(tmem + GT_G1A, da, col_desc(fb, 0, F_COLS, ks), id48t, acc || ks > 0);
                tc::mma(tmem + GT_G1B, da, col_desc(fb, 48, F_COLS, ks), id32t, acc || ks > 0);
            }
        }
        // the next tile rewrites the operands of these products
        if (!sync_mma()) {
            ok = false;
            break;
        }
        acc = true;
        buf ^= 1;
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
    // ---- this CTA's partial: rows 64..127 of the products hold the second
    //      halves (through shared memory), rows 0..63 the first ---------------
    float* out = partials + (size_t)blockIdx.x * NGRAD;
    float* part2 = reinterpret_cast<float*>(sh.z);  // dW2 part 2 [64][64], dW1 part 2 [64][32], dw3 [64]
    const bool lower = p >= 64;                      // uniform per warp
    if (ok && acc && lower) {
        const int o = p - 64;
        float a[16], b[16];
        tc::tmem_ld16x2(lanes + GT_G2B + c0, lanes + GT_G1B + (c0 & 16), a, b);
#pragma unroll
        for (int j = 0; j < 16; ++j) part2[o * 64 + c0 + j] = a[j];
        if (grp < 2)
#pragma unroll
            for (int j = 0; j < 16; ++j) part2[4096 + o * 32 + c0 + j] = b[j];
        if (grp == 0) {
            tc::tmem_ld16x2(lanes + GT_G2A + 64, lanes + GT_G2A + 64, a, b);
            part2[6144 + o] = a[0];
        } else {
            tc::tmem_ld16x2(lanes + GT_G2A + 64, lanes + GT_G2A + 64, a, b);  // the warp's collective read
        }
    }
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    if (!lower) {
        const int o = p;
        if (ok && acc) {
            float a[16], b[16];
            tc::tmem_ld16x2(lanes + GT_G2A + c0, lanes + GT_G1A + (c0 & 16), a, b);
#pragma unroll
            for (int j = 0; j < 16; ++j) out[G_W2 + o * 64 + c0 + j] = a[j] + part2[o * 64 + c0 + j];
            if (grp < 2)
#pragma unroll
                for (int j = 0; j < 16; ++j) out[G_W1 + o * 32 + c0 + j] = b[j] + part2[4096 + o * 32 + c0 + j];
            tc::tmem_ld16x2(lanes + GT_G2A + 64, lanes + GT_G1A + 32, a, b);
            if (grp == 0) {
                out[G_B2 + o] = a[0];
                out[G_B1 + o] = b[0];
                out[G_W3 + o] = part2[6144 + o];
            }
        } else {
            // no tile (or a failed wait): a zero partial
            for (int c = 0; c < GT_CW; ++c) out[G_W2 + o * 64 + c0 + c] = 0.f;
            if (grp < 2)
                for (int c = 0; c < GT_CW; ++c) out[G_W1 + o * 32 + c0 + c] = 0.f;
            if (grp == 0) {
                out[G_B2 + o] = 0.f;
                out[G_B1 + o] = 0.f;
                out[G_W3 + o] = 0.f;
            }
        }
    }
    tc::fence_before_sync();
    __syncthreads();
    if (warp == 0) tc::tmem_free(tmem, GT_COLS);
}

// e_i = F_pair,i + F_bond,i - Y_id(i); per-block sums of |e|^2 in double.
template <class T>
__global__ void __launch_bounds__(TILE) k_train_err(DevSys<T> s, int cur, const double* __restrict__ Y,
                                                    float4* __restrict__ err, double* __restrict__ loss_part) {
    __shared__ double red[TILE / 32];
    const V4<T>* __restrict__ P = s.pos[cur];
    double acc = 0.0;
    for (int t = blockIdx.x; t < s.ntiles; t += gridDim.x) {
        const Tile tl = s.tiles[t];
        if ((int)threadIdx.x >= tl.count) continue;
        const RepGeom<T>& geo = s.reps[tl.rep];
        const int i = tl.start + threadIdx.x;
        const V4<T> xi = P[i];
        const float4 fm = s.mlp_f[i];
        double fx = fm.x, fy = fm.y, fz = fm.z;
        if (s.bond.kind != 0) {
            const int2 b = s.bond_slot[i];
            for (int q = 0; q < 2; ++q) {
                const int pj = q == 0 ? b.x : b.y;
                if (pj < 0) continue;
                const V4<T> xp = P[pj];
                const T dx = min_image(xi.x, xp.x, geo.L[0], geo.halfL[0]);
                const T dy = min_image(xi.y, xp.y, geo.L[1], geo.halfL[1]);
                const T dz = min_image(xi.z, xp.z, geo.L[2], geo.halfL[2]);
                const T r2 = dx * dx + dy * dy + dz * dz;
                T fr = T(0);
                if (s.bond.kind == ESPP_FENE) {
                    const T one_m = T(1) - r2 * s.bond.inv_R02;
                    fr = one_m > T(0) ? -s.bond.K / one_m : T(0);
                } else {
                    const T r = sqrt(r2);
                    if (r < s.bond.rmax && r > T(0)) {
                        T u, F;
                        table_lookup(s.tab + s.bond.tab_off, s.bond.tab_n, s.bond.inv_dr, r, u, F);
                        fr = F / r;
                    }
                }
                fx += (double)(fr * dx);
                fy += (double)(fr * dy);
                fz += (double)(fr * dz);
            }
        }
        const size_t gid = (size_t)geo.p_off + bits_as_int(s.vel[i].w);
        const double ex = fx - Y[3 * gid], ey = fy - Y[3 * gid + 1], ez = fz - Y[3 * gid + 2];
        err[i] = make_float4((float)ex, (float)ey, (float)ez, 0.f);
        acc += ex * ex + ey * ey + ez * ez;
    }
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double a = 0.0;
        for (int w = 0; w < TILE / 32; ++w) a += red[w];
        loss_part[blockIdx.x] = a;
    }
}

// grad[k] += sum over blocks of partials in a fixed order, in two passes: 16
// chunks of consecutive blocks (each chunk summed in order) into chunk sums,
// then the chunk sums in order; loss += sum of parts.
constexpr int GRED_CHUNKS = 16;

__global__ void k_grad_chunks(const float* __restrict__ partials, int nblocks, float* __restrict__ chunk) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    const int c = blockIdx.y;
    const int per = (nblocks + GRED_CHUNKS - 1) / GRED_CHUNKS;
    if (k >= NGRAD) return;
    float a = 0.f;
    for (int b = c * per; b < min(nblocks, (c + 1) * per); ++b) a += partials[(size_t)b * NGRAD + k];
    chunk[(size_t)c * NGRAD + k] = a;
}

__global__ void k_grad_reduce(const float* __restrict__ chunk, float* __restrict__ grad,
                              const double* __restrict__ loss_part, int nloss, double* __restrict__ loss) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k < NGRAD) {
        float a = 0.f;
#pragma unroll
        for (int c = 0; c < GRED_CHUNKS; ++c) a += chunk[(size_t)c * NGRAD + k];
        grad[k] += a;
    }
    if (blockIdx.x == 0 && threadIdx.x < 32) {
        // lane q sums parts q, q + 32, ...; the lanes then add in a fixed tree
        double l = 0.0;
        for (int b = threadIdx.x; b < nloss; b += 32) l += loss_part[b];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) l += __shfl_down_sync(0xffffffffu, l, o);
        if (threadIdx.x == 0) *loss += l;
    }
}

// Adam on the FP32 master weights (b3 has no gradient), then the BF16 copy.
__global__ void k_adam(float* __restrict__ theta, float* __restrict__ m, float* __restrict__ v,
                       float* __restrict__ grad, float lr, float b1, float b2, float eps, int step,
                       MlpWeights* __restrict__ W) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= NGRAD) return;
    const float gk = grad[k];
    const float mk = b1 * m[k] + (1.f - b1) * gk;
    const float vk = b2 * v[k] + (1.f - b2) * gk * gk;
    m[k] = mk;
    v[k] = vk;
    const float mh = mk / (1.f - powf(b1, (float)step));
    const float vh = vk / (1.f - powf(b2, (float)step));
    const float th = theta[k] - lr * mh / (sqrtf(vh) + eps);
    theta[k] = th;
    grad[k] = 0.f;
    const __nv_bfloat16 hb = __float2bfloat16_rn(th);
    const float hf = __bfloat162float(hb);
    if (k < G_B1) W->W1[k] = hb;
    else if (k < G_W2) W->b1[k - G_B1] = hf;
    else if (k < G_B2) W->W2[k - G_W2] = hb;
    else if (k < G_W3) W->b2[k - G_B2] = hf;
    else W->w3[k - G_W3] = hf;
}

template <class T>
int Launch<T>::train_grad(const DevSys<T>& s, int cur, const double* Y, float4* err, double* loss_part,
                          float scale, float* partials, int grad_blocks, float* grad, double* loss,
                          cudaStream_t st) {
    k_train_err<T><<<s.ntiles, TILE, 0, st>>>(s, cur, Y, err, loss_part);
    k_mlp_grad<T><<<grad_blocks, GT_THREADS, sizeof(GradShared), st>>>(s, cur, err, scale, partials);
    // the chunk sums sit after the blocks' partials
    float* chunk = partials + (size_t)grad_blocks * NGRAD;
    k_grad_chunks<<<dim3((NGRAD + 255) / 256, GRED_CHUNKS), 256, 0, st>>>(partials, grad_blocks, chunk);
    k_grad_reduce<<<(NGRAD + 255) / 256, 256, 0, st>>>(chunk, grad, loss_part, s.ntiles, loss);
    return 4;
}

template <class T>
cudaError_t Launch<T>::prepare_train() {
    return cudaFuncSetAttribute(k_mlp_grad<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)sizeof(GradShared));
}

void launch_adam(float* theta, float* m, float* v, float* grad, float lr, float b1, float b2, float eps,
                 int step, MlpWeights* W, cudaStream_t st) {
    k_adam<<<(NGRAD + 255) / 256, 256, 0, st>>>(theta, m, v, grad, lr, b1, b2, eps, step, W);
}

int mlp_ngrad() { return NGRAD; }

template int Launch<float>::train_grad(const DevSys<float>&, int, const double*, float4*, double*, float, float*,
                                       int, float*, double*, cudaStream_t);
template int Launch<double>::train_grad(const DevSys<double>&, int, const double*, float4*, double*, float,
                                        float*, int, float*, double*, cudaStream_t);
template cudaError_t Launch<float>::prepare_train();
template cudaError_t Launch<double>::prepare_train();

}  // namespace espp

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
// A block of 4 warps works in rounds of 4 tiles of 16 pairs.  Each warp runs,
// for its tile, the forward pass of the inference kernel (activations and
// their r-tangents) and the reverse pass of the tangent output u' (rows
// scaled by w):
//   az2 = w w3 silu''(z2) dz2,  adz2 = w w3 silu'(z2)      (16 x 64)
//   [ah1; adh1] = [az2; adz2] W2                           (tensor cores)
//   az1 = ah1 silu'(z1) + adh1 silu''(z1) dz1,  adz1 = adh1 silu'(z1)
// and stages phi, dphi, h1, dh1 and the reverse rows in shared memory.  Then
// warp q accumulates rows 16q..16q+15 of
//   dW2 += az2^T h1 + adz2^T dh1,  dW1 += az1^T phi + adz1^T dphi
// over the round's 4 tiles in registers (tensor cores, K = 64 pairs), so the
// weight gradients never go through shared memory until the end.  The bias
// and output-weight sums collect per warp.  Each block writes one partial in
// a fixed order and a separate kernel adds the partials in a fixed order:
// the gradient is deterministic.  Adam then updates FP32 master weights and
// refreshes the BF16 copy the kernels read.
#include "mlp_common.cuh"

namespace espp {

constexpr int TR_WARPS = 4;
constexpr int PHI_LD = MLP_NB + 8;  // bf16 staging row strides
constexpr int H_LD = MLP_H + 8;
constexpr int G_W1 = 0;
constexpr int G_B1 = MLP_H * MLP_NB;
constexpr int G_W2 = G_B1 + MLP_H;
constexpr int G_B2 = G_W2 + MLP_H * MLP_H;
constexpr int G_W3 = G_B2 + MLP_H;
constexpr int NGRAD = G_W3 + MLP_H;  // every parameter but b3 (whose gradient is 0)

struct __align__(16) TrainWarp {
    __nv_bfloat16 phi[16 * PHI_LD], dphi[16 * PHI_LD];
    __nv_bfloat16 h1[16 * H_LD], dh1[16 * H_LD];
    __nv_bfloat16 az2[16 * H_LD], adz2[16 * H_LD];
    __nv_bfloat16 az1[16 * H_LD], adz1[16 * H_LD];
    float sums[3 * MLP_H];               // db1, db2, dw3 of this warp's tiles
};

struct __align__(16) TrainShared {
    __nv_bfloat16 w1s[MLP_H * W1_LD];
    __nv_bfloat16 w2s[MLP_H * W2_LD];
    __nv_bfloat16 w2t[MLP_H * W2_LD];
    float b1s[MLP_H], b2s[MLP_H], w3s[MLP_H];
    TrainWarp warp[TR_WARPS];
};

size_t train_smem_bytes() { return sizeof(TrainShared); }

// four 8x8 BF16 matrices from shared memory, transposed (rows of each source
// matrix given by lanes 8m..8m+7)
__device__ __forceinline__ void ldsm_x4_t(const __nv_bfloat16* p, unsigned int r[4]) {
    const unsigned int a = (unsigned int)__cvta_generic_to_shared(p);
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.trans.shared.b16 {%0,%1,%2,%3}, [%4];\n"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
                 : "r"(a));
}

// A fragment of M^T for a [16 rows = pairs][ld] staging matrix M: rows of the
// fragment are columns u0.. of M, columns are the 16 pairs.  Source matrix m
// of the load covers pairs 8 (m >> 1).. and columns u0 + 8 (m & 1)..
__device__ __forceinline__ void at_frag(const __nv_bfloat16* M, int ld, int u0, int lane, unsigned int a[4]) {
    const int m = lane >> 3, r = lane & 7;
    ldsm_x4_t(M + ((m >> 1) * 8 + r) * ld + u0 + (m & 1) * 8, a);
}

// B fragments of a [16 pairs (k)][ld] staging matrix M for columns n0..n0+7
// (b[0], b[1]) and n0+8..n0+15 (b[2], b[3]).  Source matrix m covers pairs
// 8 (m & 1).. and columns n0 + 8 (m >> 1)..
__device__ __forceinline__ void bk_frag2(const __nv_bfloat16* M, int ld, int n0, int lane, unsigned int b[4]) {
    const int m = lane >> 3, r = lane & 7;
    ldsm_x4_t(M + ((m & 1) * 8 + r) * ld + n0 + (m >> 1) * 8, b);
}

__device__ __forceinline__ void stage2(__nv_bfloat16* M, int ld, int row, int col, float lo, float hi) {
    *reinterpret_cast<unsigned int*>(M + row * ld + col) = pack_bf16x2(lo, hi);
}

// sum over the 8 lanes of equal t (rows of a C fragment), result in lanes 0..3
__device__ __forceinline__ float col_sum(float v) {
    v += __shfl_xor_sync(0xffffffffu, v, 4);
    v += __shfl_xor_sync(0xffffffffu, v, 8);
    v += __shfl_xor_sync(0xffffffffu, v, 16);
    return v;
}

template <class T>
__global__ void __launch_bounds__(32 * TR_WARPS, 2) k_mlp_grad(DevSys<T> s, int cur, const float4* __restrict__ err,
                                                             float scale, float* __restrict__ partials) {
    extern __shared__ __align__(16) unsigned char tsm_raw[];
    TrainShared& sh = *reinterpret_cast<TrainShared*>(tsm_raw);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int g = lane >> 2, tig = lane & 3;
    TrainWarp& ws = sh.warp[warp];
    load_mlp_weights(s.mlp, sh.w1s, sh.w2s, sh.w2t, sh.b1s, sh.b2s, sh.w3s);
    for (int k = lane; k < 3 * MLP_H; k += 32) ws.sums[k] = 0.f;
    __syncthreads();
    const float rc = s.mlp->rc, rc2 = rc * rc;
    const V4<T>* __restrict__ P = s.pos[cur];
    const int stride = s.stride;
    const int nu = min(*s.mlp_nupper, s.mlp_upper_cap);
    const int nrounds = (nu + 16 * TR_WARPS - 1) / (16 * TR_WARPS);
    // this warp's rows of dW2 (16 x 64) and dW1 (16 x 32), as MMA accumulators
    float acc2[8][4], acc1[4][4];
#pragma unroll
    for (int a = 0; a < 8; ++a)
#pragma unroll
        for (int e = 0; e < 4; ++e) acc2[a][e] = 0.f;
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int e = 0; e < 4; ++e) acc1[a][e] = 0.f;

    for (int round = blockIdx.x; round < nrounds; round += gridDim.x) {
        // ---- the pairs of this warp's tile: distance and row weight --------------
        const int p = lane & 15;
        const int k = (round * TR_WARPS + warp) * 16 + p;
        float rr = rc, wrow = 0.f;
        if (k < nu) {
            const int4 up = s.mlp_upper[k];
            const int i = (up.x >> 2) % stride, j = nbr_slot(up.z);
            const RepGeom<T>& geo = s.reps[up.w];
            const T L0 = geo.L[0], L1 = geo.L[1], L2 = geo.L[2];
            const V4<T> xi = ld4<T>(P + i), xj = ld4<T>(P + j);
            const int code = nbr_code(up.z);
            const float dx = (float)shifted_diff(xi.x, (T)(xi.x - L0), xj.x, L0, code & 3);
            const float dy = (float)shifted_diff(xi.y, (T)(xi.y - L1), xj.y, L1, (code >> 2) & 3);
            const float dz = (float)shifted_diff(xi.z, (T)(xi.z - L2), xj.z, L2, code >> 4);
            const float r2 = __fadd_rn(__fadd_rn(__fmul_rn(dx, dx), __fmul_rn(dy, dy)), __fmul_rn(dz, dz));
            if (r2 < rc2) {
                rr = sqrtf(r2);
                const float4 ei = err[i], ej = err[j];
                wrow = scale * ((ei.x - ej.x) * dx + (ei.y - ej.y) * dy + (ei.z - ej.z) * dz) / rr;
            }
        }
        const float ra = __shfl_sync(0xffffffffu, rr, g), rb = __shfl_sync(0xffffffffu, rr, g + 8);
        const float wa = __shfl_sync(0xffffffffu, wrow, g), wb = __shfl_sync(0xffffffffu, wrow, g + 8);
        // ---- features, staged for dW1 ---------------------------------
        unsigned int aph[2][4], adp[2][4];
        rbf_fragments(ra, rb, rc, tig, aph, adp);
#pragma unroll
        for (int kt = 0; kt < 2; ++kt) {
            const int col = kt * 16 + 2 * tig;
            *reinterpret_cast<unsigned int*>(ws.phi + g * PHI_LD + col) = aph[kt][0];
            *reinterpret_cast<unsigned int*>(ws.phi + (g + 8) * PHI_LD + col) = aph[kt][1];
            *reinterpret_cast<unsigned int*>(ws.phi + g * PHI_LD + col + 8) = aph[kt][2];
            *reinterpret_cast<unsigned int*>(ws.phi + (g + 8) * PHI_LD + col + 8) = aph[kt][3];
            *reinterpret_cast<unsigned int*>(ws.dphi + g * PHI_LD + col) = adp[kt][0];
            *reinterpret_cast<unsigned int*>(ws.dphi + (g + 8) * PHI_LD + col) = adp[kt][1];
            *reinterpret_cast<unsigned int*>(ws.dphi + g * PHI_LD + col + 8) = adp[kt][2];
            *reinterpret_cast<unsigned int*>(ws.dphi + (g + 8) * PHI_LD + col + 8) = adp[kt][3];
        }
        // ---- layer 1 forward: h1, dh1 as layer-2 operands, staged ---
        unsigned int ah[4][4], adh[4][4];
#pragma unroll
        for (int nt = 0; nt < 8; ++nt) {
            float z[4] = {0.f, 0.f, 0.f, 0.f}, dzv[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
            for (int kt = 0; kt < 2; ++kt) {
                unsigned int b0, b1;
                b_frag(sh.w1s, W1_LD, nt * 8, kt * 16, g, tig, b0, b1);
                mma_bf16_16816(z, aph[kt], b0, b1);
                mma_bf16_16816(dzv, adp[kt], b0, b1);
            }
            const int col = nt * 8 + 2 * tig;
            float hv[4], dhv[4];
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                const float zz = z[e] + sh.b1s[col + (e & 1)];
                const float sg = sigm(zz);
                hv[e] = zz * sg;
                dhv[e] = sg * (1.f + zz * (1.f - sg)) * dzv[e];
            }
            const int kt2 = nt >> 1, off = (nt & 1) * 2;
            ah[kt2][off + 0] = pack_bf16x2(hv[0], hv[1]);
            ah[kt2][off + 1] = pack_bf16x2(hv[2], hv[3]);
            adh[kt2][off + 0] = pack_bf16x2(dhv[0], dhv[1]);
            adh[kt2][off + 1] = pack_bf16x2(dhv[2], dhv[3]);
            *reinterpret_cast<unsigned int*>(ws.h1 + g * H_LD + col) = ah[kt2][off + 0];
            *reinterpret_cast<unsigned int*>(ws.h1 + (g + 8) * H_LD + col) = ah[kt2][off + 1];
            *reinterpret_cast<unsigned int*>(ws.dh1 + g * H_LD + col) = adh[kt2][off + 0];
            *reinterpret_cast<unsigned int*>(ws.dh1 + (g + 8) * H_LD + col) = adh[kt2][off + 1];
        }
        // ---- layer 2 forward and the reverse seeds az2, adz2 ---------
        unsigned int aaz[4][4], aadz[4][4];
#pragma unroll
        for (int nt = 0; nt < 8; ++nt) {
            float z[4] = {0.f, 0.f, 0.f, 0.f}, dzv[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
            for (int kt = 0; kt < 4; ++kt) {
                unsigned int b0, b1;
                b_frag(sh.w2s, W2_LD, nt * 8, kt * 16, g, tig, b0, b1);
                mma_bf16_16816(z, ah[kt], b0, b1);
                mma_bf16_16816(dzv, adh[kt], b0, b1);
            }
            const int col = nt * 8 + 2 * tig;
            float az[4], adz[4], gw3[2] = {0.f, 0.f}, gb2[2] = {0.f, 0.f};
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                const float zz = z[e] + sh.b2s[col + (e & 1)];
                const float sg = sigm(zz);
                const float s1 = sg * (1.f + zz * (1.f - sg));
                const float s2 = sg * (1.f - sg) * (2.f + zz * (1.f - 2.f * sg));
                const float w = e < 2 ? wa : wb;
                const float w3v = sh.w3s[col + (e & 1)];
                az[e] = w * w3v * s2 * dzv[e];
                adz[e] = w * w3v * s1;
                gw3[e & 1] += w * s1 * dzv[e];
                gb2[e & 1] += az[e];
            }
            const int kt2 = nt >> 1, off = (nt & 1) * 2;
            aaz[kt2][off + 0] = pack_bf16x2(az[0], az[1]);
            aaz[kt2][off + 1] = pack_bf16x2(az[2], az[3]);
            aadz[kt2][off + 0] = pack_bf16x2(adz[0], adz[1]);
            aadz[kt2][off + 1] = pack_bf16x2(adz[2], adz[3]);
            *reinterpret_cast<unsigned int*>(ws.az2 + g * H_LD + col) = aaz[kt2][off + 0];
            *reinterpret_cast<unsigned int*>(ws.az2 + (g + 8) * H_LD + col) = aaz[kt2][off + 1];
            *reinterpret_cast<unsigned int*>(ws.adz2 + g * H_LD + col) = aadz[kt2][off + 0];
            *reinterpret_cast<unsigned int*>(ws.adz2 + (g + 8) * H_LD + col) = aadz[kt2][off + 1];
#pragma unroll
            for (int q = 0; q < 2; ++q) {
                const float a3 = col_sum(gw3[q]), a2 = col_sum(gb2[q]);
                if (g == 0) {
                    ws.sums[2 * MLP_H + col + q] += a3;
                    ws.sums[MLP_H + col + q] += a2;
                }
            }
        }
        // ---- back through W2 and layer 1: az1, adz1, staged ----------
#pragma unroll
        for (int nt = 0; nt < 8; ++nt) {
            float a1[4] = {0.f, 0.f, 0.f, 0.f}, ad1[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
            for (int kt = 0; kt < 4; ++kt) {
                unsigned int b0, b1;
                b_frag(sh.w2t, W2_LD, nt * 8, kt * 16, g, tig, b0, b1);
                mma_bf16_16816(a1, aaz[kt], b0, b1);
                mma_bf16_16816(ad1, aadz[kt], b0, b1);
            }
            float z[4] = {0.f, 0.f, 0.f, 0.f}, dzv[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
            for (int kt = 0; kt < 2; ++kt) {
                unsigned int b0, b1;
                b_frag(sh.w1s, W1_LD, nt * 8, kt * 16, g, tig, b0, b1);
                mma_bf16_16816(z, aph[kt], b0, b1);
                mma_bf16_16816(dzv, adp[kt], b0, b1);
            }
            const int col = nt * 8 + 2 * tig;
            float az[4], adz[4], gb1[2] = {0.f, 0.f};
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                const float zz = z[e] + sh.b1s[col + (e & 1)];
                const float sg = sigm(zz);
                const float s1 = sg * (1.f + zz * (1.f - sg));
                const float s2 = sg * (1.f - sg) * (2.f + zz * (1.f - 2.f * sg));
                az[e] = a1[e] * s1 + ad1[e] * s2 * dzv[e];
                adz[e] = ad1[e] * s1;
                gb1[e & 1] += az[e];
            }
            stage2(ws.az1, H_LD, g, col, az[0], az[1]);
            stage2(ws.az1, H_LD, g + 8, col, az[2], az[3]);
            stage2(ws.adz1, H_LD, g, col, adz[0], adz[1]);
            stage2(ws.adz1, H_LD, g + 8, col, adz[2], adz[3]);
#pragma unroll
            for (int q = 0; q < 2; ++q) {
                const float a = col_sum(gb1[q]);
                if (g == 0) ws.sums[col + q] += a;
            }
        }
        __syncthreads();
        // ---- weight gradients: this warp's rows, K = the round's 4 x 16 pairs ----
        for (int src = 0; src < TR_WARPS; ++src) {
            const TrainWarp& ts = sh.warp[src];
            unsigned int A[4], AD[4];
            at_frag(ts.az2, H_LD, warp * 16, lane, A);
            at_frag(ts.adz2, H_LD, warp * 16, lane, AD);
#pragma unroll
            for (int nt = 0; nt < 8; nt += 2) {
                unsigned int b[4], d[4];
                bk_frag2(ts.h1, H_LD, nt * 8, lane, b);
                bk_frag2(ts.dh1, H_LD, nt * 8, lane, d);
                mma_bf16_16816(acc2[nt], A, b[0], b[1]);
                mma_bf16_16816(acc2[nt], AD, d[0], d[1]);
                mma_bf16_16816(acc2[nt + 1], A, b[2], b[3]);
                mma_bf16_16816(acc2[nt + 1], AD, d[2], d[3]);
            }
            at_frag(ts.az1, H_LD, warp * 16, lane, A);
            at_frag(ts.adz1, H_LD, warp * 16, lane, AD);
#pragma unroll
            for (int nt = 0; nt < 4; nt += 2) {
                unsigned int b[4], d[4];
                bk_frag2(ts.phi, PHI_LD, nt * 8, lane, b);
                bk_frag2(ts.dphi, PHI_LD, nt * 8, lane, d);
                mma_bf16_16816(acc1[nt], A, b[0], b[1]);
                mma_bf16_16816(acc1[nt], AD, d[0], d[1]);
                mma_bf16_16816(acc1[nt + 1], A, b[2], b[3]);
                mma_bf16_16816(acc1[nt + 1], AD, d[2], d[3]);
            }
        }
        __syncthreads();
    }
    // ---- this block's partial: register rows, then the warps' sums in order -----
    float* out = partials + (size_t)blockIdx.x * NGRAD;
    const int row = warp * 16 + g;
#pragma unroll
    for (int nt = 0; nt < 8; ++nt) {
        float* dst = out + G_W2 + row * MLP_H + nt * 8 + 2 * tig;
        dst[0] = acc2[nt][0];
        dst[1] = acc2[nt][1];
        dst[8 * MLP_H] = acc2[nt][2];
        dst[8 * MLP_H + 1] = acc2[nt][3];
    }
#pragma unroll
    for (int nt = 0; nt < 4; ++nt) {
        float* dst = out + G_W1 + row * MLP_NB + nt * 8 + 2 * tig;
        dst[0] = acc1[nt][0];
        dst[1] = acc1[nt][1];
        dst[8 * MLP_NB] = acc1[nt][2];
        dst[8 * MLP_NB + 1] = acc1[nt][3];
    }
    __syncthreads();
    for (int k = threadIdx.x; k < MLP_H; k += blockDim.x) {
        float b1v = 0.f, b2v = 0.f, w3v = 0.f;
#pragma unroll
        for (int w = 0; w < TR_WARPS; ++w) {
            b1v += sh.warp[w].sums[k];
            b2v += sh.warp[w].sums[MLP_H + k];
            w3v += sh.warp[w].sums[2 * MLP_H + k];
        }
        out[G_B1 + k] = b1v;
        out[G_B2 + k] = b2v;
        out[G_W3 + k] = w3v;
    }
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
    k_mlp_grad<T><<<grad_blocks, 32 * TR_WARPS, sizeof(TrainShared), st>>>(s, cur, err, scale, partials);
    // the chunk sums sit after the blocks' partials
    float* chunk = partials + (size_t)grad_blocks * NGRAD;
    k_grad_chunks<<<dim3((NGRAD + 255) / 256, GRED_CHUNKS), 256, 0, st>>>(partials, grad_blocks, chunk);
    k_grad_reduce<<<(NGRAD + 255) / 256, 256, 0, st>>>(chunk, grad, loss_part, s.ntiles, loss);
    return 4;
}

template <class T>
cudaError_t Launch<T>::prepare_train() {
    return cudaFuncSetAttribute(k_mlp_grad<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)sizeof(TrainShared));
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

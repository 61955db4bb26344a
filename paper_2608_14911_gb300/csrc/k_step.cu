// The per-step kernel: pair forces over the Verlet list (Lennard-Jones / WCA /
// capped LJ, paper "Software design": VerletListInteractionTemplate<Potential>
// with computeForce/computeEnergy; "Example usage": LennardJones(..., shift=
// 'auto'), LennardJonesCapped), FENE bonds, the Langevin thermostat
// ("Example usage": LangevinThermostat(gamma, temperature) attached through
// addExtension) and velocity Verlet ("Example usage": VelocityVerlet), fused
// into one pass per particle.
//
// One thread per particle, particles in cell (Hilbert) order, 128 per block.
// Each thread sums the forces on its own particle from both directions of the
// full list, so no force atomics are needed.  In MODE_STEP the thread then
// completes the step and starts the next one:
//   F_s  = F_pair + F_bond - gamma m v_{s-1/2} + sqrt(24 gamma m kT/dt) r_s
//   v_s  = v_{s-1/2} + dt/2 F_s/m           (the full-step velocity)
//   v_{s+1/2} = v_s + dt/2 F_s/m
//   x_{s+1}   = x_s + dt v_{s+1/2}           (wrapped; written to the other buffer)
// and checks the displacement since the last list build against skin/2.
#include "kernels.cuh"
#include "packed.cuh"
#include "pair_terms.cuh"
#include "philox.cuh"

// Launch shapes of the FP32 step kernel on the plain list path, chosen at run
// time by the autotuner (espp_tune_step_shape): int4 neighbour groups read per
// batch, the minimum resident blocks per SM the register budget is fitted to,
// and the tiles one block takes.  A block of several consecutive tiles holds
// a larger compact piece of the Hilbert order, so more of its neighbours'
// positions are shared in the SM's L1 (the halo of a piece shrinks relative
// to its volume).  Shape 0 is the default.
struct StepShape {
    int groups;  // list groups per batch
    int minb;    // minimum resident blocks per SM
    int tpb;     // tiles (of TILE particles) per block
};
constexpr StepShape STEP_SHAPES[ESPP_STEP_SHAPES] = {{1, 8, 1}, {2, 8, 1}, {1, 12, 1}, {1, 10, 1},
                                                     {1, 5, 2}, {1, 3, 3}, {1, 2, 4},  {1, 2, 5}};
#ifndef ESPP_STEP_MINB32
#define ESPP_STEP_MINB32 8  // KG 1M FP32: 0.1027 ms per step (8), 0.1123 (10)
#endif
#ifndef ESPP_STEP_MINB32_DPD  // the same for the DPD variants
#define ESPP_STEP_MINB32_DPD 10
#endif
#ifndef ESPP_STEP_LATE  // loads issued after the pair loop: 1 bond partners, 2 velocity and build position
#define ESPP_STEP_LATE 3  // KG 1M FP32 at 8 blocks per SM: 58.7 us (3), 61.5 (1); fewer values live across the loop
#endif
#ifndef ESPP_STEP_PREFETCH
#define ESPP_STEP_PREFETCH 2  // request the next batch's list groups early (see pair_loop)
#endif

namespace espp {

// Sum of the pair forces on particle i over its Verlet list.  The list is
// read in batches of int4 groups: all indices of a batch first, then all
// neighbour positions, then the arithmetic, so that each thread keeps several
// independent loads in flight; the next batch's indices are prefetched.
// With DPD the thermostat's pair term is added in the same pass, for pairs
// inside the DPD cutoff, from the neighbours' velocity snapshot.
// Entries with x code 3 cross a sheared face (Lees-Edwards): their x
// difference is taken from the current offset in *le.
template <class T, bool ENERGY, bool MULTI, bool FAST, bool DPD, bool LE, int GB32 = 1>
__device__ __forceinline__ void pair_loop(const DevSys<T>& s, const V4<T>* __restrict__ P, int i, int n,
                                          const V4<T>& xi, int ti, const PairRec<T>* pr1,
                                          T L0, T L1, T L2, T& fx, T& fy, T& fz, T& pe, T& vir, T& vxz,
                                          const LeCtx<T>* le, const DpdCtx<T>* dc = nullptr) {
    const T xim = xi.x - L0, yim = xi.y - L1, zim = xi.z - L2;
    constexpr int GB = sizeof(T) == 4 ? GB32 : 1;  // int4 groups per batch
    const int ng = (n + 3) >> 2;
    const int4* __restrict__ nb = reinterpret_cast<const int4*>(s.nbr) + i;
    const size_t stride = (size_t)s.stride;
    const int gcap = s.cap >> 2;  // groups allocated per particle (>= 2)
    // the groups of the next batch are requested before the positions of the
    // current one, so their latency overlaps the current batch; the first
    // batch is read without waiting for the count (groups past the count are
    // allocated, and dropped whole; the last group is padded with -1)
    // padding entries (the rest of the last group, and whole groups past the
    // count) name the padding slot, whose position is far outside the box:
    // every entry is loaded and evaluated without a test of its own
    const int pad = s.nbr_pad;
    const int4 pad4 = make_int4(pad, pad, pad, pad);
    // FP32 single-type Lennard-Jones without energies (the step's hot path):
    // two entries per packed FP32x2 instruction, forces summed in two lanes
    constexpr bool PACK = sizeof(T) == 4 && FAST && !ENERGY && !DPD;
    f32x2 px = 0ull, py = 0ull, pz = 0ull;
    f32x2 xi2 = 0ull, yi2 = 0ull, zi2 = 0ull, sg2 = 0ull, e24 = 0ull;
    if constexpr (PACK) {
        xi2 = f2(xi.x, xi.x);
        yi2 = f2(xi.y, xi.y);
        zi2 = f2(xi.z, xi.z);
        sg2 = f2(pr1->sig2, pr1->sig2);
        e24 = f2(pr1->eps24, pr1->eps24);
    }
    int4 nxt[GB];
#pragma unroll
    for (int q = 0; q < GB; ++q) nxt[q] = q < gcap ? __ldg(nb + q * stride) : pad4;
    for (int g0 = 0; g0 < ng || g0 == 0; g0 += GB) {
        int jj[4 * GB];
#pragma unroll
        for (int q = 0; q < GB; ++q) {
            if (!ESPP_STEP_PREFETCH && g0 > 0) nxt[q] = __ldg(nb + (g0 + q) * stride);
            int4 a = nxt[q];
            if (g0 + q >= ng) a = pad4;
            jj[4 * q + 0] = a.x;
            jj[4 * q + 1] = a.y;
            jj[4 * q + 2] = a.z;
            jj[4 * q + 3] = a.w;
        }
#pragma unroll
        for (int q = 0; q < GB; ++q) {
            const int gn = g0 + GB + q;
            // ESPP_STEP_PREFETCH 1: request while the count may be in flight
            // (reads one group past the list); 2: only groups inside the list
            if ((ESPP_STEP_PREFETCH == 1 && gn < gcap) || (ESPP_STEP_PREFETCH == 2 && gn < ng))
                nxt[q] = __ldg(nb + gn * stride);
        }
        int codes = 0;
#pragma unroll
        for (int q = 0; q < 4 * GB; ++q) codes |= jj[q];
        V4<T> xj[4 * GB];
#pragma unroll
        for (int q = 0; q < 4 * GB; ++q) xj[q] = ld4<T>(P + nbr_slot(jj[q]));
        if constexpr (PACK) {
            // entries two at a time; every entry goes through the same
            // arithmetic whichever batch it falls in, so the sums do not
            // depend on the batch shape
            const T rc2 = pr1->rc2;
            const f32x2 two = f2(2.f, 2.f), mone = f2(-1.f, -1.f);
            const bool plain = (codes & ~NBR_INDEX_MASK) == 0;  // no pair of the batch crosses a face
#pragma unroll
            for (int q = 0; q < 4 * GB; q += 2) {
                f32x2 dx, dy, dz;
                if (plain) {
                    dx = f2sub(xi2, f2(xj[q].x, xj[q + 1].x));
                    dy = f2sub(yi2, f2(xj[q].y, xj[q + 1].y));
                    dz = f2sub(zi2, f2(xj[q].z, xj[q + 1].z));
                } else {
                    T d[2][3];
#pragma unroll
                    for (int h = 0; h < 2; ++h) {
                        const int code = nbr_code(jj[q + h]);
                        if (LE && (code & 3) == 3)
                            d[h][0] = le_dx(xi.x, xj[q + h].x, (code >> 4) == 1 ? 1 : -1, le->d, L0, le->inv_Lx);
                        else
                            d[h][0] = shifted_diff(xi.x, xim, xj[q + h].x, L0, code & 3);
                        d[h][1] = shifted_diff(xi.y, yim, xj[q + h].y, L1, (code >> 2) & 3);
                        d[h][2] = shifted_diff(xi.z, zim, xj[q + h].z, L2, code >> 4);
                    }
                    dx = f2(d[0][0], d[1][0]);
                    dy = f2(d[0][1], d[1][1]);
                    dz = f2(d[0][2], d[1][2]);
                }
                float ra, rb;
                f2split(f2fma(dz, dz, f2fma(dy, dy, f2mul(dx, dx))), ra, rb);
                const f32x2 inv = f2(recip(ra), recip(rb));
                const f32x2 s2 = f2mul(sg2, inv);
                const f32x2 s6 = f2mul(f2mul(s2, s2), s2);
                float fa, fb;
                f2split(f2mul(f2mul(f2mul(e24, s6), f2fma(s6, two, mone)), inv), fa, fb);
                const f32x2 fr = f2(ra < rc2 ? fa : 0.f, rb < rc2 ? fb : 0.f);
                px = f2fma(fr, dx, px);
                py = f2fma(fr, dy, py);
                pz = f2fma(fr, dz, pz);
            }
        } else if ((codes & ~NBR_INDEX_MASK) == 0) {
            // no pair of this batch crosses a face (the common case)
#pragma unroll
            for (int q = 0; q < 4 * GB; ++q) {
                const T dx = xi.x - xj[q].x, dy = xi.y - xj[q].y, dz = xi.z - xj[q].z;
                pair_term<T, ENERGY, MULTI, FAST>(s, ti, pr1, dx, dy, dz, bits_as_int(xj[q].w), fx, fy, fz, pe,
                                                  vir, vxz);
                if (DPD) {
                    const T r2 = dx * dx + dy * dy + dz * dz;
                    if (r2 < s.ip->dpd_rc2)
                        dpd_term<T>(s.ip, *dc, dx, dy, dz, r2, ld4<T>(s.vsnap + nbr_slot(jj[q])), fx, fy, fz);
                }
            }
        } else {
#pragma unroll
            for (int q = 0; q < 4 * GB; ++q) {
                const int code = nbr_code(jj[q]);
                int nz = 0;
                T dx;
                if (LE && (code & 3) == 3) {
                    nz = (code >> 4) == 1 ? 1 : -1;
                    dx = le_dx(xi.x, xj[q].x, nz, le->d, L0, le->inv_Lx);
                } else {
                    dx = shifted_diff(xi.x, xim, xj[q].x, L0, code & 3);
                }
                const T dy = shifted_diff(xi.y, yim, xj[q].y, L1, (code >> 2) & 3);
                const T dz = shifted_diff(xi.z, zim, xj[q].z, L2, code >> 4);
                pair_term<T, ENERGY, MULTI, FAST>(s, ti, pr1, dx, dy, dz, bits_as_int(xj[q].w), fx, fy, fz,
                                                  pe, vir, vxz);
                if (DPD) {
                    const T r2 = dx * dx + dy * dy + dz * dz;
                    if (r2 < s.ip->dpd_rc2)
                        dpd_term<T>(s.ip, *dc, dx, dy, dz, r2, ld4<T>(s.vsnap + nbr_slot(jj[q])), fx, fy, fz,
                                    nz);
                }
            }
        }
    }
    if constexpr (PACK) {
        float a, b;
        f2split(px, a, b);
        fx += a + b;
        f2split(py, a, b);
        fy += a + b;
        f2split(pz, a, b);
        fz += a + b;
    }
}

// DPD thermostat forces on particle i as a pass of their own over the list,
// for the learned potential, whose pair forces come from k_mlp.
template <class T, bool LE>
__device__ __forceinline__ void dpd_loop(const DevSys<T>& s, const V4<T>* __restrict__ P, int i, int n,
                                         const V4<T>& xi, const DpdCtx<T>& c, const LeCtx<T>& le, T L0, T L1,
                                         T L2, T& fx, T& fy, T& fz) {
    const IntParams<T>* __restrict__ ip = s.ip;
    const T rc2 = ip->dpd_rc2;
    const T xim = xi.x - L0, yim = xi.y - L1, zim = xi.z - L2;
    const int4* __restrict__ nb = reinterpret_cast<const int4*>(s.nbr) + i;
    const V4<T>* __restrict__ VS = s.vsnap;
    const size_t stride = (size_t)s.stride;
    for (int g = 0; 4 * g < n; ++g) {
        const int4 a = __ldg(nb + g * stride);
        const int jj[4] = {a.x, a.y, a.z, a.w};
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            if (4 * g + q >= n) continue;
            const int j = nbr_slot(jj[q]), code = nbr_code(jj[q]);
            const V4<T> xj = ld4<T>(P + j);
            int nz = 0;
            T dx;
            if (LE && (code & 3) == 3) {
                nz = (code >> 4) == 1 ? 1 : -1;
                dx = le_dx(xi.x, xj.x, nz, le.d, L0, le.inv_Lx);
            } else {
                dx = shifted_diff(xi.x, xim, xj.x, L0, code & 3);
            }
            const T dy = shifted_diff(xi.y, yim, xj.y, L1, (code >> 2) & 3);
            const T dz = shifted_diff(xi.z, zim, xj.z, L2, code >> 4);
            const T r2 = dx * dx + dy * dy + dz * dz;
            if (!(r2 < rc2)) continue;
            dpd_term<T>(ip, c, dx, dy, dz, r2, ld4<T>(VS + j), fx, fy, fz, nz);
        }
    }
}

// velocities at the force evaluation, read by the DPD pass for the neighbours
template <class T>
__global__ void __launch_bounds__(TILE) k_vsnap(DevSys<T> s) {
    if (s.ctrl->abort) return;
    for (int t = blockIdx.x; t < s.ntiles; t += gridDim.x) {
        const Tile tl = s.tiles[t];
        if ((int)threadIdx.x < tl.count) s.vsnap[tl.start + threadIdx.x] = s.vel[tl.start + threadIdx.x];
    }
}

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    return v;
}

// SH: launch shape (STEP_SHAPES) of the plain FP32 list path.
template <class T, int MODE, bool ENERGY, bool FAST, bool DPD, bool LE, int SH = 0>
__global__ void __launch_bounds__(TILE * STEP_SHAPES[SH].tpb,
                                  sizeof(T) == 4 ? (DPD ? ESPP_STEP_MINB32_DPD
                                                        : (SH == 0 ? ESPP_STEP_MINB32 : STEP_SHAPES[SH].minb))
                                                 : 4)
    k_step(DevSys<T> s, int cur, double* __restrict__ f_out, unsigned long long next_cond) {
    // TPB consecutive tiles per block; the block-wide energy reduction below
    // is written for one
    constexpr int TPB = STEP_SHAPES[SH].tpb;
    static_assert(TPB == 1 || !ENERGY, "energy reductions take one tile per block");
    const int lt = TPB > 1 ? (int)threadIdx.x % TILE : (int)threadIdx.x;  // index inside the tile
    Ctrl* c = s.ctrl;
    const int t0 = blockIdx.x * TPB + (TPB > 1 ? (int)threadIdx.x / TILE : 0);
    // the first tile's record is requested together with the abort flag
    Tile tl0 = {0, 0, 0, 0};
    if (t0 < s.ntiles) tl0 = ld_tile_early(s.tiles + t0);
    if (MODE != MODE_FORCES && c->abort) return;
    const long long step = c->step + (MODE >= MODE_STEP ? 1 : 0);
    const V4<T>* __restrict__ P = s.pos[cur];
    V4<T>* __restrict__ Pn = s.pos[cur ^ 1];
    const IntParams<T>* __restrict__ ip = s.ip;
    __shared__ double red[NPART][TILE / 32];

    for (int t = t0; t < s.ntiles; t += gridDim.x * TPB) {
        const Tile tl = t == t0 ? tl0 : s.tiles[t];
        const bool active = lt < tl.count;
        const RepGeom<T>& g = s.reps[tl.rep];
        double acc[NPART];
        if (ENERGY) {
#pragma unroll
            for (int k = 0; k < NPART; ++k) acc[k] = 0.0;
        }
        // Lees-Edwards: the tile's offset now and, after the drift, the
        // displacement bound that keeps the list valid: pairs across a sheared
        // face also move apart by the change of delta since the build
        LeCtx<T> le;
        T skin_thr2 = s.half_skin2;
        if (LE) {
            double q[2] = {0.0, 0.0};
            if ((threadIdx.x & 31) == 0) {
                const double dnow = le_offset(s, g, step);
                q[0] = le_reduce(dnow, (double)g.L[0]);
                if (MODE == MODE_STEP) {
                    const double h = 0.5 * ((double)s.skin - fabs(le_offset(s, g, step + 1) - s.le_db[tl.rep]));
                    q[1] = h > 0.0 ? h * h : 0.0;
                }
            }
            q[0] = __shfl_sync(0xffffffffu, q[0], 0);
            q[1] = __shfl_sync(0xffffffffu, q[1], 0);
            le.d = (T)q[0];
            le.inv_Lx = T(1) / g.L[0];
            le.shear = (T)s.le_shear;
            le.vs = (T)(s.le_shear * (double)g.L[2]);
            if (MODE == MODE_STEP) skin_thr2 = (T)q[1];
        } else {
            le.d = le.inv_Lx = le.vs = le.shear = T(0);
        }
        if (active) {
            const int i = tl.start + lt;
            const T L0 = g.L[0], L1 = g.L[1], L2 = g.L[2];
            const T H0 = g.halfL[0], H1 = g.halfL[1], H2 = g.halfL[2];
            // independent loads first: own position, list count, bond slots,
            // velocity and build position, then the bond partners' positions
            const V4<T> xi = ld4<T>(P + i);
            const int ti = bits_as_int(xi.w);
            T fx = 0, fy = 0, fz = 0, pe = 0, pb = 0, vir = 0, vxz = 0;
            const int n = s.nbr_cnt[i];
            const bool bonded = s.bond.kind != 0;
            const int2 b = bonded ? s.bond_slot[i] : make_int2(-1, -1);
            // loads the pair loop does not need, issued before it (latency
            // hidden behind the loop) or after it (fewer registers held)
            constexpr bool LATE_BOND = (ESPP_STEP_LATE & 1) != 0;
            constexpr bool LATE_VEL = (ESPP_STEP_LATE & 2) != 0 && !DPD;
            V4<T> v, xbi, xp0, xp1;
            if (!LATE_VEL) {
                v = s.vel[i];
                if (MODE == MODE_STEP && (FAST || !s.cells_mode)) xbi = s.xb[i];
            }
            if (!LATE_BOND) {
                xp0 = b.x >= 0 ? ld4<T>(P + b.x) : xi;
                xp1 = b.y >= 0 ? ld4<T>(P + b.y) : xi;
            }
            DpdCtx<T> dc;
            if (DPD) {
                dc.vi = v;
                dc.seed = g.seed;
                dc.step = step;
                dc.le_vs = le.vs;
            }
            if (s.mlp_on) {
                // pair forces of the learned potential, computed by k_mlp
                if constexpr (sizeof(T) == 8) {
                    // FP64 handle: the network evaluated in double (k_mlp_f64)
                    const V4<T> fm = s.mlp_fT[i];
                    fx = fm.x;
                    fy = fm.y;
                    fz = fm.z;
                    if (ENERGY) {
                        pe = fm.w;
                        vir = s.mlp_wT[i];
                    }
                } else {
                    const float4 fm = s.mlp_f[i];
                    fx = (T)fm.x;
                    fy = (T)fm.y;
                    fz = (T)fm.z;
                    if (ENERGY) {
                        pe = (T)fm.w;
                        vir = (T)s.mlp_w[i];
                    }
                }
                if (DPD) dpd_loop<T, LE>(s, P, i, n, xi, dc, le, L0, L1, L2, fx, fy, fz);
            } else if (!FAST && s.cells_mode) {
                // list-free mode: pair forces (with the DPD pair term) from
                // the cell-stencil kernel
                const V4<T> f = s.cpf[i];
                fx = f.x;
                fy = f.y;
                fz = f.z;
                if (ENERGY) {
                    pe = f.w;
                    const V4<T> w = s.cpv[i];
                    vir = w.x;
                    vxz = w.y;
                }
            } else if (FAST) {
                PairRec<T> pr;
                pr.rc2 = s.pair[0].rc2;
                pr.sig2 = s.pair[0].sig2;
                pr.eps24 = s.pair[0].eps24;
                if (ENERGY) {
                    pr.eps4 = s.pair[0].eps4;
                    pr.shift = s.pair[0].shift;
                }
                pair_loop<T, ENERGY, false, true, DPD, LE, STEP_SHAPES[SH].groups>(s, P, i, n, xi, ti, &pr, L0, L1, L2,
                                                                                   fx, fy, fz, pe, vir, vxz, &le, &dc);
            } else if (s.ntypes == 1) {
                const PairRec<T> pr = s.pair[0];
                if (pr.kind != 0 || DPD)
                    pair_loop<T, ENERGY, false, false, DPD, LE>(s, P, i, n, xi, ti, &pr, L0, L1, L2, fx, fy, fz, pe,
                                                            vir, vxz, &le, &dc);
            } else {
                pair_loop<T, ENERGY, true, false, DPD, LE>(s, P, i, n, xi, ti, nullptr, L0, L1, L2, fx, fy, fz, pe,
                                                       vir, vxz, &le, &dc);
            }
            if (LATE_VEL) {
                v = s.vel[i];
                if (MODE == MODE_STEP && (FAST || !s.cells_mode)) xbi = s.xb[i];
            }
            if (LATE_BOND) {
                xp0 = b.x >= 0 ? ld4<T>(P + b.x) : xi;
                xp1 = b.y >= 0 ? ld4<T>(P + b.y) : xi;
            }
            // bonds (paper "Functionality": bonded interactions; FENE or tabulated)
            double blen = 0.0, bcnt = 0.0;
            if (bonded) {
#pragma unroll
                for (int q = 0; q < 2; ++q) {
                    const int p = q == 0 ? b.x : b.y;
                    if (p < 0) continue;
                    const V4<T> xp = q == 0 ? xp0 : xp1;
                    const T dz = min_image(xi.z, xp.z, L2, H2);
                    const T dy = min_image(xi.y, xp.y, L1, H1);
                    T dx;
                    if (LE && (xi.z - xp.z > H2 || xi.z - xp.z < -H2)) {
                        // bond across a sheared face
                        dx = le_dx(xi.x, xp.x, xi.z - xp.z > H2 ? 1 : -1, le.d, L0, le.inv_Lx);
                    } else {
                        dx = min_image(xi.x, xp.x, L0, H0);
                    }
                    const T r2 = dx * dx + dy * dy + dz * dz;
                    T fr, ub = T(0);
                    if (s.bond.kind == ESPP_FENE) {
                        T one_m = T(1) - r2 * s.bond.inv_R02;
                        if (!(one_m > T(0))) {
                            atomicOr(&c->err, ERRBIT_BOND);
                            c->abort = 1;
                            __threadfence();
                            one_m = T(1e-6);
                        }
                        fr = -s.bond.K * recip(one_m);
                        if (ENERGY) ub = -s.bond.halfKR02 * log(one_m);
                    } else {
                        T r = sqrt(r2), F;
                        if (!(r < s.bond.rmax)) {
                            atomicOr(&c->err, ERRBIT_BOND);
                            c->abort = 1;
                            __threadfence();
                            r = T(0);
                        }
                        table_lookup(s.tab + s.bond.tab_off, s.bond.tab_n, s.bond.inv_dr, r, ub, F);
                        fr = r > T(0) ? F / r : T(0);
                    }
                    fx += fr * dx;
                    fy += fr * dy;
                    fz += fr * dz;
                    if (ENERGY) {
                        pb += ub;
                        vir += fr * r2;
                        vxz += fr * dx * dz;
                        blen += sqrt((double)r2);
                        bcnt += 1.0;
                    }
                }
            }
            if (ENERGY) {
                acc[P_PE_PAIR] = 0.5 * (double)pe;
                acc[P_PE_BOND] = 0.5 * (double)pb;
                acc[P_VIRIAL] = 0.5 * (double)vir;
                acc[P_BOND_LEN] = 0.5 * blen;
                acc[P_BOND_CNT] = 0.5 * bcnt;
                acc[P_VIR_XZ] = 0.5 * (double)vxz;
            }
            if (MODE == MODE_FORCES) {
                if (f_out) {
                    const size_t gid = (size_t)g.p_off + bits_as_int(v.w);
                    f_out[3 * gid + 0] = (double)fx;
                    f_out[3 * gid + 1] = (double)fy;
                    f_out[3 * gid + 2] = (double)fz;
                }
                if (ENERGY) {
                    const double m = (double)ip->mass[ti];
                    // kinetic terms relative to the shear profile (Lees-Edwards)
                    const double vxp = LE ? (double)v.x - (double)le.shear * ((double)xi.z - (double)H2) : (double)v.x;
                    acc[P_KE] = 0.5 * m * (vxp * vxp + (double)v.y * v.y + (double)v.z * v.z);
                    acc[P_KIN_XZ] = m * vxp * (double)v.z;
                    acc[P_PX] = m * v.x;
                    acc[P_PY] = m * v.y;
                    acc[P_PZ] = m * v.z;
                }
            } else {
                const T m = ip->mass[ti], inv_m = ip->inv_mass[ti];
                if (!DPD && ip->gamma != T(0)) {
                    T rx, ry, rz;
                    langevin_noise<T>(g.seed, bits_as_int(v.w), step, rx, ry, rz);
                    const T amp = ip->noise_amp[ti];
                    const T gm = ip->gamma * m;
                    // friction relative to the shear profile (Lees-Edwards)
                    const T vxp = LE ? v.x - le.shear * (xi.z - H2) : v.x;
                    fx += -gm * vxp + amp * rx;
                    fy += -gm * v.y + amp * ry;
                    fz += -gm * v.z + amp * rz;
                }
                if (MODE == MODE_INIT) {
                    s.frc[i] = mk4<T>(fx, fy, fz, T(0));
                } else {
                    const T hdt = ip->half_dt;
                    v.x = half_kick(v.x, fx, hdt, inv_m);
                    v.y = half_kick(v.y, fy, hdt, inv_m);
                    v.z = half_kick(v.z, fz, hdt, inv_m);
                    if (MODE == MODE_FINAL) {
                        s.vel[i] = v;
                        s.frc[i] = mk4<T>(fx, fy, fz, T(0));
                    } else {
                        v.x = half_kick(v.x, fx, hdt, inv_m);
                        v.y = half_kick(v.y, fy, hdt, inv_m);
                        v.z = half_kick(v.z, fz, hdt, inv_m);
                        const T dt = ip->dt;
                        T x = drift(xi.x, v.x, dt), y = drift(xi.y, v.y, dt), z = drift(xi.z, v.z, dt);
                        // no wrap here: positions stay in the image frame of the
                        // last list build until the next build wraps them
                        if (!(fabs(x) < T(1e30) && fabs(y) < T(1e30) && fabs(z) < T(1e30))) {
                            atomicOr(&c->err, ERRBIT_NONFINITE);
                            c->abort = 1;
                            __threadfence();
                            x = xi.x; y = xi.y; z = xi.z;
                        }
                        if (!FAST && s.cells_mode) {
                            // list-free mode: every step is binned again
                            if (lt == 0) {
                                s.req[tl.rep] = 1;
                                c->any_req = 1;
                                __threadfence();
                            }
                        } else {
                            const T ex = x - xbi.x, ey = y - xbi.y, ez = z - xbi.z;
                            if (ex * ex + ey * ey + ez * ez > skin_thr2) {
                                s.req[tl.rep] = 1;
                                c->any_req = 1;
                                __threadfence();
                            }
                        }
                        Pn[i] = mk4<T>(x, y, z, xi.w);
                        s.vel[i] = v;
                    }
                }
            }
        }
        if (ENERGY) {
            const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
            for (int k = 0; k < NPART; ++k) {
                const double r = warp_sum(acc[k]);
                if (lane == 0) red[k][w] = r;
            }
            __syncthreads();
            if (threadIdx.x < NPART) {
                double sum = 0.0;
#pragma unroll
                for (int q = 0; q < TILE / 32; ++q) sum += red[threadIdx.x][q];
                s.partials[(size_t)t * NPART + threadIdx.x] = sum;
            }
            __syncthreads();
        }
    }

    if (MODE == MODE_STEP || MODE == MODE_FINAL) {
        // the last block to finish advances the step counter and arms the
        // conditional rebuild node of the next step
        __syncthreads();
        if (threadIdx.x == 0) {
            __threadfence();
            const unsigned int done = atomicAdd(&c->blocks_done, 1u);
            if (done == gridDim.x - 1) {
                __threadfence();
                c->step = step;
                if (MODE == MODE_FINAL) c->pos_ahead = 0;
                c->blocks_done = 0;
                if (next_cond) {
                    const unsigned int want = *(volatile unsigned int*)&c->any_req;
                    const unsigned int ab = *(volatile unsigned int*)&c->abort;
                    cudaGraphSetConditional(next_cond, (want && !ab) ? 1u : 0u);
                }
            }
        }
    }
}

// First half-kick and drift of an integrate call: v_{n+1/2}, x_{n+1}.
template <class T>
__global__ void __launch_bounds__(TILE) k_prologue(DevSys<T> s, int cur) {
    Ctrl* c = s.ctrl;
    if (c->abort) return;
    const V4<T>* __restrict__ P = s.pos[cur];
    V4<T>* __restrict__ Pn = s.pos[cur ^ 1];
    const IntParams<T>* __restrict__ ip = s.ip;
    // the stored positions become those of step + 1 (read by the rebuilds)
    if (blockIdx.x == 0 && threadIdx.x == 0) c->pos_ahead = 1;
    const long long step = c->step;
    for (int t = blockIdx.x; t < s.ntiles; t += gridDim.x) {
        const Tile tl = s.tiles[t];
        if ((int)threadIdx.x >= tl.count) continue;
        const int i = tl.start + threadIdx.x;
        T skin_thr2 = s.half_skin2;
        if (s.le_on) {
            // Lees-Edwards: the change of delta since the build uses up skin
            const double h = 0.5 * ((double)s.skin - fabs(le_offset(s, s.reps[tl.rep], step + 1) - s.le_db[tl.rep]));
            skin_thr2 = h > 0.0 ? (T)(h * h) : T(0);
        }
        const V4<T> xi = P[i];
        const int ti = bits_as_int(xi.w);
        const V4<T> f = s.frc[i];
        V4<T> v = s.vel[i];
        const T hdt = ip->half_dt, inv_m = ip->inv_mass[ti];
        v.x = half_kick(v.x, f.x, hdt, inv_m);
        v.y = half_kick(v.y, f.y, hdt, inv_m);
        v.z = half_kick(v.z, f.z, hdt, inv_m);
        const T dt = ip->dt;
        T x = drift(xi.x, v.x, dt), y = drift(xi.y, v.y, dt), z = drift(xi.z, v.z, dt);
        if (!(fabs(x) < T(1e30) && fabs(y) < T(1e30) && fabs(z) < T(1e30))) {
            atomicOr(&c->err, ERRBIT_NONFINITE);
            c->abort = 1;
            x = xi.x; y = xi.y; z = xi.z;
        }
        if (s.cells_mode) {
            // list-free mode: every step is binned again
            s.req[tl.rep] = 1;
            c->any_req = 1;
        } else {
            const V4<T> b = s.xb[i];
            const T ex = x - b.x, ey = y - b.y, ez = z - b.z;
            if (ex * ex + ey * ey + ez * ez > skin_thr2) {
                s.req[tl.rep] = 1;
                c->any_req = 1;
            }
        }
        Pn[i] = mk4<T>(x, y, z, xi.w);
        s.vel[i] = v;
    }
}

template <class T>
__global__ void k_set_cond(DevSys<T> s, unsigned long long h) {
    const unsigned int want = *(volatile unsigned int*)&s.ctrl->any_req;
    const unsigned int ab = *(volatile unsigned int*)&s.ctrl->abort;
    cudaGraphSetConditional(h, (want && !ab) ? 1u : 0u);
}

template <class T>
int Launch<T>::step(const DevSys<T>& s, int mode, bool energy, int cur, double* f_out,
                    unsigned long long next_cond, int grid, cudaStream_t st) {
    const int gr = grid > 0 ? grid : s.ntiles;
    int extra = s.mlp_on ? Launch<T>::mlp(s, cur, energy, st) : 0;
    const bool dpd = s.dpd && mode != MODE_FORCES;
    if (s.cells_mode) {
        // list-free: pair forces (and the DPD pair term) from the cell stencil
        extra += Launch<T>::cellforce(s, cur, energy, dpd, st);
    } else if (dpd) {
        k_vsnap<T><<<s.ntiles, TILE, 0, st>>>(s);
        extra += 1;
    }
    // the plain FP32 list path of a step takes the tuned launch shape
    const int sh = (sizeof(T) == 4 && s.lj_fast && !s.le_on && !s.cells_mode && !s.mlp_on &&
                    (mode == MODE_STEP || mode == MODE_FINAL) && !dpd) ? s.step_shape : 0;
#define ESPP_STEP_SHAPED(M, E, D, LE, K)                                                                   \
    k_step<T, M, E, true, D, LE, K>                                                                        \
        <<<(gr + STEP_SHAPES[K].tpb - 1) / STEP_SHAPES[K].tpb, TILE * STEP_SHAPES[K].tpb, 0, st>>>(s, cur, f_out, next_cond)
#define ESPP_STEP_SH(M, E, D, LE)                                                                          \
    do {                                                                                                   \
        if constexpr (sizeof(T) == 4 && !(D) && !(LE) && ((M) == MODE_STEP || (M) == MODE_FINAL)) {        \
            switch (sh) {                                                                                  \
                case 1: ESPP_STEP_SHAPED(M, E, D, LE, 1); break;                                           \
                case 2: ESPP_STEP_SHAPED(M, E, D, LE, 2); break;                                           \
                case 3: ESPP_STEP_SHAPED(M, E, D, LE, 3); break;                                           \
                case 4: ESPP_STEP_SHAPED(M, E, D, LE, 4); break;                                           \
                case 5: ESPP_STEP_SHAPED(M, E, D, LE, 5); break;                                           \
                case 6: ESPP_STEP_SHAPED(M, E, D, LE, 6); break;                                           \
                case 7: ESPP_STEP_SHAPED(M, E, D, LE, 7); break;                                           \
                default: break;                                                                            \
            }                                                                                              \
            if (sh != 0) break;                                                                            \
        }                                                                                                  \
        k_step<T, M, E, true, D, LE><<<gr, TILE, 0, st>>>(s, cur, f_out, next_cond);                       \
    } while (0)
#define ESPP_STEP_LE(M, E, D, LE)                                                                \
    do {                                                                                         \
        if (s.lj_fast) ESPP_STEP_SH(M, E, D, LE);                                                \
        else k_step<T, M, E, false, D, LE><<<gr, TILE, 0, st>>>(s, cur, f_out, next_cond);         \
    } while (0)
#define ESPP_STEP(M, E, D)                            \
    do {                                              \
        if (s.le_on) ESPP_STEP_LE(M, E, D, true);     \
        else ESPP_STEP_LE(M, E, D, false);            \
    } while (0)
    switch (mode) {
        case MODE_FORCES:
            if (energy) ESPP_STEP(MODE_FORCES, true, false); else ESPP_STEP(MODE_FORCES, false, false);
            break;
        case MODE_INIT:
            if (dpd) ESPP_STEP(MODE_INIT, false, true); else ESPP_STEP(MODE_INIT, false, false);
            break;
        case MODE_STEP:
            if (dpd) ESPP_STEP(MODE_STEP, false, true); else ESPP_STEP(MODE_STEP, false, false);
            break;
        default:
            if (dpd) ESPP_STEP(MODE_FINAL, false, true); else ESPP_STEP(MODE_FINAL, false, false);
            break;
    }
#undef ESPP_STEP
#undef ESPP_STEP_LE
#undef ESPP_STEP_SH
#undef ESPP_STEP_SHAPED
    return 1 + extra;
}

template <class T>
void Launch<T>::prologue(const DevSys<T>& s, int cur, int grid, cudaStream_t st) {
    k_prologue<T><<<grid > 0 ? grid : s.ntiles, TILE, 0, st>>>(s, cur);
}

template <class T>
void Launch<T>::set_cond(const DevSys<T>& s, unsigned long long cond, cudaStream_t st) {
    k_set_cond<T><<<1, 1, 0, st>>>(s, cond);
}

// The two precisions compile as separate units (k_step_f32.cu, k_step_f64.cu)
// that include this file with ESPP_STEP_PRECISION set, so they build in
// parallel; compiled alone, this file instantiates both.
#if !defined(ESPP_STEP_PRECISION) || ESPP_STEP_PRECISION == 32
template int Launch<float>::step(const DevSys<float>&, int, bool, int, double*, unsigned long long, int, cudaStream_t);
template void Launch<float>::prologue(const DevSys<float>&, int, int, cudaStream_t);
template void Launch<float>::set_cond(const DevSys<float>&, unsigned long long, cudaStream_t);
#endif
#if !defined(ESPP_STEP_PRECISION) || ESPP_STEP_PRECISION == 64
template int Launch<double>::step(const DevSys<double>&, int, bool, int, double*, unsigned long long, int, cudaStream_t);
template void Launch<double>::prologue(const DevSys<double>&, int, int, cudaStream_t);
template void Launch<double>::set_cond(const DevSys<double>&, unsigned long long, cudaStream_t);
#endif

}  // namespace espp

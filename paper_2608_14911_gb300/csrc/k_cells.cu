// List-free pair forces from the cell stencil (paper "Performance
// optimizations": linked cells and the sub-cell decomposition of Yao et al.,
// cells of edge rc / W).  In this mode the particles are binned every step
// (the rebuild pipeline without the Verlet search) and one thread per cell
// entry streams the (2W+1)^3 neighbouring cells' entries, which the binning
// left contiguous by rows, testing each against the cutoff.  No list is built
// or read, so nothing depends on a skin: the mode pays for the binning and a
// wider candidate set every step, and wins where a Verlet list would be
// rebuilt every step or two anyway (fast particles, large time steps).
//
// The kernel writes per storage slot the pair force and pair energy (and, in
// the energy pass, the virial and its xz part), which the step kernel adds
// in place of its list loop; the DPD thermostat's pair term (velocities from
// the cell-ordered copy written at binning) and the Lees-Edwards planes are
// evaluated here too.
#include "kernels.cuh"
#include "pair_terms.cuh"

// minimum resident blocks per SM the FP32 register budget is fitted to
#ifndef ESPP_CF_MINB32
#define ESPP_CF_MINB32 8
#endif

namespace espp {

template <class T>
__device__ __forceinline__ int cf_cell_coord(T x, T cpl, int nc) {
    int c = (int)(x * cpl);
    c = c < 0 ? 0 : c;
    return c >= nc ? nc - 1 : c;
}

// Pair and DPD terms of the candidates [p, e) of one contiguous range.
// SHIFT: shifted differences by the image codes xL/yL/zL and the shifted
// particle coordinates xo/yo/zo; LEX: the x difference is the nearest image
// of x_i - nz delta - x_j (a plane across a sheared face).
template <class T, bool ENERGY, bool MULTI, bool DPD, bool SHIFT, bool LEX>
__device__ __forceinline__ void cf_range(const DevSys<T>& s, const V4<T>* __restrict__ E,
                                         const V4<T>* __restrict__ VE, int p, int e, int i, int ti, int2 ex,
                                         const PairRec<T>* pr1, const V4<T>* __restrict__ P, T xo, T yo, T zo,
                                         T xL, T yL, T zL, T Lx,
                                         T inv_Lx, int nz, const DpdCtx<T>* dc, T& fx, T& fy, T& fz, T& pe,
                                         T& vir, T& vxz) {
    for (; p < e; ++p) {
        const V4<T> xj = ld4<T>(E + p);
        const int j = bits_as_int(xj.w);
        if (j == i) continue;
        if (s.excl_bonded && (j == ex.x || j == ex.y)) continue;
        T dx;
        if (LEX) {
            dx = (xo - xj.x) - xL;
            dx -= Lx * rint(dx * inv_Lx);
        } else {
            dx = SHIFT ? xo - (xj.x - xL) : xo - xj.x;
        }
        const T dy = SHIFT ? yo - (xj.y - yL) : yo - xj.y;
        const T dz = SHIFT ? zo - (xj.z - zL) : zo - xj.z;
        const int tj = MULTI ? bits_as_int(P[j].w) : 0;
        pair_term<T, ENERGY, MULTI, false>(s, ti, pr1, dx, dy, dz, tj, fx, fy, fz, pe, vir, vxz);
        if (DPD) {
            const T r2 = dx * dx + dy * dy + dz * dz;
            if (r2 < s.ip->dpd_rc2) dpd_term<T>(s.ip, *dc, dx, dy, dz, r2, ld4<T>(VE + p), fx, fy, fz, nz);
        }
    }
}

template <class T, int W, bool ENERGY, bool MULTI, bool DPD, bool LE>
__global__ void __launch_bounds__(TILE, sizeof(T) == 4 ? ESPP_CF_MINB32 : 2) k_cellforce(DevSys<T> s, int cur) {
    if (s.ctrl->abort) return;
    const V4<T>* __restrict__ P = s.pos[cur];  // type bits of the partners (several types)
    const V4<T>* __restrict__ E = s.cell_ent;
    const V4<T>* __restrict__ VE = s.cell_vel;
    const int* __restrict__ B = s.cell_beg;
    const long long step = s.ctrl->step + (long long)s.ctrl->pos_ahead;
    for (int t = blockIdx.x; t < s.ntiles; t += gridDim.x) {
        const Tile tl = s.tiles[t];
        if ((int)threadIdx.x >= tl.count) continue;
        const RepGeom<T>& g = s.reps[tl.rep];
        // threads follow the entry array (cell order); a replica's entries
        // fill the same index range as its slots
        const int idx = tl.start + threadIdx.x;
        const V4<T> xi = ld4<T>(E + idx);
        const int i = bits_as_int(xi.w);
        const int ti = MULTI ? bits_as_int(P[i].w) : 0;
        PairRec<T> prl;
        if (!MULTI) prl = s.pair[0];
        const PairRec<T>* pr1 = MULTI ? nullptr : &prl;
        const int2 ex = s.excl_bonded ? s.bond_slot[i] : make_int2(-1, -1);
        DpdCtx<T> dc;
        if (DPD) {
            dc.vi = ld4<T>(VE + idx);
            dc.seed = g.seed;
            dc.step = step;
            dc.le_vs = LE ? (T)(s.le_shear * (double)g.L[2]) : T(0);
        }
        const int nc0 = g.nc[0], nc1 = g.nc[1], nc2 = g.nc[2];
        const int cx = cf_cell_coord(xi.x, g.cells_per_len[0], nc0);
        const int cy = cf_cell_coord(xi.y, g.cells_per_len[1], nc1);
        const int cz = cf_cell_coord(xi.z, g.cells_per_len[2], nc2);
        const T L0 = g.L[0], L1 = g.L[1], L2 = g.L[2];
        const T inv_L0 = LE ? T(1) / L0 : T(0);
        // Lees-Edwards: delta of this step (binned with it) reduced into [0, Lx)
        const T le_d = LE ? (T)le_reduce(s.le_db[tl.rep], (double)L0) : T(0);
        T fx = 0, fy = 0, fz = 0, pe_ = 0, vir = 0, vxz = 0;
        constexpr int NR = 2 * W + 1;
#pragma unroll 1
        for (int dz = -W; dz <= W; ++dz) {
            int az = cz + dz, czc = 0;
            if (az < 0) { az += nc2; czc = 2; }
            else if (az >= nc2) { az -= nc2; czc = 1; }
            const T zo = (czc & 1) ? xi.z - L2 : xi.z, zL = (czc & 2) ? L2 : T(0);
            const bool sheared = LE && czc != 0;
            const int nz = czc == 1 ? 1 : czc == 2 ? -1 : 0;
            const T nd = sheared ? (T)nz * le_d : T(0);
            int cxr = cx;
            if (sheared) {
                // the partners' image is displaced by nz delta along x: its
                // cells are found around x_i - nz delta
                T xs = xi.x - nd;
                if (xs < T(0)) xs += L0;
                if (xs >= L0) xs -= L0;
                cxr = cf_cell_coord(xs, g.cells_per_len[0], nc0);
            }
            // the plane's rows share one cyclic x range: up to two pieces
            // [x0a, x0b] and [x1a, x1b] with their x image codes
            int x0a = cxr - W, x0b = cxr + W, x1a = 0, x1b = -1, c0 = 0, c1 = 0;
            if (x0a < 0) {
                x1a = 0;
                x1b = x0b;
                x0a += nc0;
                x0b = nc0 - 1;
                c0 = 2;
            } else if (x0b >= nc0) {
                x1a = 0;
                x1b = x0b - nc0;
                x0b = nc0 - 1;
                c1 = 1;
            }
            // all row ranges of the plane first, so their loads overlap
            int pb[NR][2], pe[NR][2], cyc[NR];
#pragma unroll
            for (int r = 0; r < NR; ++r) {
                int ay = cy + r - W, c = 0;
                if (ay < 0) { ay += nc1; c = 2; }
                else if (ay >= nc1) { ay -= nc1; c = 1; }
                cyc[r] = c;
                const int base = g.cell_off + (az * nc1 + ay) * nc0;
                pb[r][0] = __ldg(B + base + x0a);
                pe[r][0] = __ldg(B + base + x0b + 1);
                pb[r][1] = x1b >= 0 ? __ldg(B + base + x1a) : 0;
                pe[r][1] = x1b >= 0 ? __ldg(B + base + x1b + 1) : 0;
            }
#pragma unroll
            for (int r = 0; r < NR; ++r) {
                const T yo = (cyc[r] & 1) ? xi.y - L1 : xi.y, yL = (cyc[r] & 2) ? L1 : T(0);
#pragma unroll
                for (int part = 0; part < 2; ++part) {
                    if (sheared) {
                        cf_range<T, ENERGY, MULTI, DPD, true, true>(s, E, VE, pb[r][part], pe[r][part], i, ti, ex, pr1,
                                                                     P, xi.x, yo, zo, nd, yL, zL, L0, inv_L0, nz,
                                                                     &dc, fx, fy, fz, pe_, vir, vxz);
                        continue;
                    }
                    const int cxc = part ? c1 : c0;
                    const T xo = (cxc & 1) ? xi.x - L0 : xi.x, xL = (cxc & 2) ? L0 : T(0);
                    if ((cxc | cyc[r] | czc) == 0)
                        cf_range<T, ENERGY, MULTI, DPD, false, false>(s, E, VE, pb[r][part], pe[r][part], i, ti, ex,
                                                                       pr1, P, xo, yo, zo, xL, yL, zL, L0, inv_L0, 0,
                                                                       &dc, fx, fy, fz, pe_, vir, vxz);
                    else
                        cf_range<T, ENERGY, MULTI, DPD, true, false>(s, E, VE, pb[r][part], pe[r][part], i, ti, ex,
                                                                      pr1, P, xo, yo, zo, xL, yL, zL, L0, inv_L0, 0,
                                                                      &dc, fx, fy, fz, pe_, vir, vxz);
                }
            }
        }
        s.cpf[i] = mk4<T>(fx, fy, fz, pe_);
        if (ENERGY) s.cpv[i] = mk4<T>(vir, vxz, T(0), T(0));
    }
}

template <class T>
int Launch<T>::cellforce(const DevSys<T>& s, int cur, bool energy, bool dpd, cudaStream_t st) {
    const int gt = s.ntiles;
    const bool multi = s.ntypes > 1;
#define ESPP_CF(W, E, M, D, L) k_cellforce<T, W, E, M, D, L><<<gt, TILE, 0, st>>>(s, cur)
#define ESPP_CF_L(W, E, M, D)                    \
    do {                                         \
        if (s.le_on) ESPP_CF(W, E, M, D, true);  \
        else ESPP_CF(W, E, M, D, false);         \
    } while (0)
#define ESPP_CF_D(W, E, M)                       \
    do {                                         \
        if (dpd) ESPP_CF_L(W, E, M, true);       \
        else ESPP_CF_L(W, E, M, false);          \
    } while (0)
#define ESPP_CF_M(W, E)                          \
    do {                                         \
        if (multi) ESPP_CF_D(W, E, true);        \
        else ESPP_CF_D(W, E, false);             \
    } while (0)
    if (s.cell_w == 1) {
        if (energy) ESPP_CF_M(1, true);
        else ESPP_CF_M(1, false);
    } else {
        if (energy) ESPP_CF_M(2, true);
        else ESPP_CF_M(2, false);
    }
#undef ESPP_CF_M
#undef ESPP_CF_D
#undef ESPP_CF_L
#undef ESPP_CF
    return 1;
}

template int Launch<float>::cellforce(const DevSys<float>&, int, bool, bool, cudaStream_t);
template int Launch<double>::cellforce(const DevSys<double>&, int, bool, bool, cudaStream_t);

}  // namespace espp

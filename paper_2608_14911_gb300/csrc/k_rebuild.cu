// Rebuild pipeline: linked-cell binning, the periodic Hilbert resort of every
// particle array into cell order, and the full Verlet list with skin.  Paper
// "Software design" ("Parallelization": CellGrid linked cells;
// "Performance optimizations": cell decomposition and data sorting) and
// "Example usage" (VerletList(system, cutoff) with system.skin).
//
// Every rebuild (inside the step graphs, when a replica asked for it):
//   prep      latch the per-replica requests, clear those replicas' cell counts
//   bin       cell of every particle and its arrival index (atomic histogram)
//   scan x3   exclusive scan of the counts in cell-index order: first entry of
//             every cell in one compact entry array (no per-cell capacity)
//   place     every particle's entry (position, storage slot) into its cell
//   cellsort  entries of each cell in ascending storage slot, so the list does
//             not depend on the order of the atomics
//   verlet    stencil search from the cell entries, streamed as contiguous
//             row ranges; full list (both directions) as groups of four
//             indices, nbr4[g * stride + i]; records the build positions
// A resort (launched between step graphs every `resort_every` steps, and on
// every explicit build) additionally runs, between cellsort and verlet:
//   scan x3   exclusive scan of the cell counts in Hilbert-rank order
//   scatter   new slot of every entry (its cell's first slot + its rank in the
//             cell); the entries switch to the new slots
//   gather    permuted copies of positions, velocities, forces, images
//   copyback  copies back and maps bond partners to their new slots
// Replicas whose request flag is clear skip every per-particle and per-cell
// step after `prep`; their counts and entries stay those of their last build,
// so the global scan keeps every replica's entries in its own slot range.
#include "kernels.cuh"
#include "scan.cuh"

namespace espp {


template <class T>
__device__ __forceinline__ int cell_coord(T x, T cpl, int nc) {
    int c = (int)(x * cpl);
    c = c < 0 ? 0 : c;
    return c >= nc ? nc - 1 : c;
}

template <class T>
__device__ __forceinline__ int cell_of(const RepGeom<T>& g, const V4<T>& p) {
    const int cx = cell_coord(p.x, g.cells_per_len[0], g.nc[0]);
    const int cy = cell_coord(p.y, g.cells_per_len[1], g.nc[1]);
    const int cz = cell_coord(p.z, g.cells_per_len[2], g.nc[2]);
    return g.cell_off + (cz * g.nc[1] + cy) * g.nc[0] + cx;
}

template <class T>
__global__ void __launch_bounds__(256) k_prep(DevSys<T> s) {
    if (s.ctrl->abort) return;
    for (int h = blockIdx.x * blockDim.x + threadIdx.x; h < s.ncells; h += gridDim.x * blockDim.x)
        if (s.req[s.cell_rep[h]]) s.cell_cnt[h] = 0;
    if (blockIdx.x == 0) {
        // Lees-Edwards: the offset at this build, for the rebuild criterion
        // and the sheared rows of the search (kept as stored after a
        // checkpoint load)
        const long long pstep = s.ctrl->step + (long long)s.ctrl->pos_ahead;
        const bool keep = s.ctrl->le_keep != 0;
        for (int r = threadIdx.x; r < s.R; r += blockDim.x) {
            s.now[r] = s.req[r];
            if (s.le_on && s.req[r] && !keep) s.le_db[r] = le_offset(s, s.reps[r], pstep);
        }
        __syncthreads();
        if (threadIdx.x == 0) s.ctrl->le_keep = 0;
        if (threadIdx.x == 0 && s.ctrl->any_req) {
            s.ctrl->n_rebuilds += 1;
            s.ctrl->max_count = 0;
        }
    }
}

// Cell of every particle of a flagged replica and its arrival index in that
// cell (counting-sort histogram); positions are wrapped into the box here,
// at list builds only.
template <class T>
__global__ void __launch_bounds__(TILE) k_bin(DevSys<T> s, int cur) {
    // the first tile's record is requested together with the abort flag
    Tile tl0 = {0, 0, 0, 0};
    if ((int)blockIdx.x < s.ntiles) tl0 = ld_tile_early(s.tiles + blockIdx.x);
    if (s.ctrl->abort) return;
    if (blockIdx.x == 0) {
        for (int r = threadIdx.x; r < s.R; r += blockDim.x) s.req[r] = 0;
        if (threadIdx.x == 0) s.ctrl->any_req = 0;
    }
    V4<T>* __restrict__ P = s.pos[cur];
    for (int t = blockIdx.x; t < s.ntiles; t += gridDim.x) {
        const Tile tl = t == (int)blockIdx.x ? tl0 : s.tiles[t];
        if (!s.now[tl.rep] || (int)threadIdx.x >= tl.count) continue;
        const int i = tl.start + threadIdx.x;
        V4<T> p = P[i];
        const RepGeom<T>& g = s.reps[tl.rep];
        int wx, wy, wz;
        if (s.le_on && !(p.z >= T(0) && p.z < g.L[2])) {
            // across a sheared face: the image entered is displaced and moving
            const double L[3] = {(double)g.L[0], (double)g.L[1], (double)g.L[2]};
            double q[3] = {(double)p.x, (double)p.y, (double)p.z};
            V4<T> v = s.vel[i];
            double vx = (double)v.x;
            int k[3];
            le_wrap(q, vx, k, L, s.le_db[tl.rep], s.le_shear);
            p.x = (T)q[0];
            p.y = (T)q[1];
            p.z = (T)q[2];
            // a coordinate rounded up to L in the conversion stays in its
            // image, just below L
            if (!(p.x < g.L[0])) p.x = below(g.L[0]);
            if (!(p.y < g.L[1])) p.y = below(g.L[1]);
            if (!(p.z < g.L[2])) p.z = below(g.L[2]);
            v.x = (T)vx;
            s.vel[i] = v;
            wx = k[0];
            wy = k[1];
            wz = k[2];
        } else {
            wx = wrap_coord(p.x, g.L[0]);
            wy = wrap_coord(p.y, g.L[1]);
            wz = wrap_coord(p.z, g.L[2]);
        }
        if (wx | wy | wz) {
            P[i] = p;
            int4 im = s.img[i];
            im.x += wx;
            im.y += wy;
            im.z += wz;
            s.img[i] = im;
        }
        const int h = cell_of(g, p);
        s.cellh[i] = h;
        s.in_cell[i] = atomicAdd(&s.cell_cnt[h], 1);
    }
}

// Entry (wrapped position, storage slot in the w lane) of every particle of a
// flagged replica at its cell's first entry + its arrival index.
template <class T>
__global__ void __launch_bounds__(TILE) k_place(DevSys<T> s, int cur) {
    // the first tile's record is requested together with the abort flag
    Tile tl0 = {0, 0, 0, 0};
    if ((int)blockIdx.x < s.ntiles) tl0 = ld_tile_early(s.tiles + blockIdx.x);
    if (s.ctrl->abort) return;
    const V4<T>* __restrict__ P = s.pos[cur];
    for (int t = blockIdx.x; t < s.ntiles; t += gridDim.x) {
        const Tile tl = t == (int)blockIdx.x ? tl0 : s.tiles[t];
        if (!s.now[tl.rep] || (int)threadIdx.x >= tl.count) continue;
        const int i = tl.start + threadIdx.x;
        V4<T> p = ld4<T>(P + i);
        p.w = int_bits_as(T(0), i);
        s.cell_ent[s.cell_beg[s.cellh[i]] + s.in_cell[i]] = p;
    }
}

// Entries of each cell in ascending storage slot (a handful per cell), so the
// list does not depend on the order of the atomics.
template <class T>
__global__ void __launch_bounds__(256) k_cellsort(DevSys<T> s) {
    if (s.ctrl->abort) return;
    for (int h = blockIdx.x * blockDim.x + threadIdx.x; h < s.ncells; h += gridDim.x * blockDim.x) {
        if (!s.now[s.cell_rep[h]]) continue;
        V4<T>* p = s.cell_ent + s.cell_beg[h];
        const int e = s.cell_beg[h + 1] - s.cell_beg[h];
        for (int k = 1; k < e; ++k) {
            const V4<T> key = p[k];
            const int kk = bits_as_int(key.w);
            int q = k - 1;
            while (q >= 0 && bits_as_int(p[q].w) > kk) {
                p[q + 1] = p[q];
                --q;
            }
            p[q + 1] = key;
        }
        // list-free mode with DPD: the velocities in entry order as well
        if (s.cells_mode && s.dpd)
            for (int k = 0; k < e; ++k) s.cell_vel[s.cell_beg[h] + k] = s.vel[bits_as_int(p[k].w)];
    }
}

// ---- exclusive scan of the cell counts (three phases, no inter-block waits) --
// RANK = false: cells in index order -> cell_beg (every rebuild);
// RANK = true: cells in Hilbert-rank order -> rank_start (resort only).
template <class T, bool RANK>
__device__ __forceinline__ int scan_count(const DevSys<T>& s, int k) {
    return k < s.ncells ? s.cell_cnt[RANK ? s.cell_by_rank[k] : k] : 0;
}

template <class T, bool RANK>
__global__ void __launch_bounds__(SCAN_THREADS) k_scan_reduce(DevSys<T> s) {
    if (s.ctrl->abort) return;
    const int base = blockIdx.x * SCAN_TILE + threadIdx.x * SCAN_ITEMS;
    int sum = 0;
#pragma unroll
    for (int k = 0; k < SCAN_ITEMS; ++k) sum += scan_count<T, RANK>(s, base + k);
    int excl;
    const int total = block_excl_scan(sum, &excl);
    if (threadIdx.x == 0) s.scan_part[blockIdx.x] = total;
}

template <class T>
__global__ void __launch_bounds__(SCAN_THREADS) k_scan_top(DevSys<T> s) {
    if (s.ctrl->abort) return;
    int carry = 0;
    for (int b0 = 0; b0 < s.nscan_blocks; b0 += SCAN_THREADS) {
        const int b = b0 + threadIdx.x;
        const int v = b < s.nscan_blocks ? s.scan_part[b] : 0;
        int excl;
        const int total = block_excl_scan(v, &excl);
        if (b < s.nscan_blocks) s.scan_part[b] = carry + excl;
        carry += total;
    }
}

template <class T, bool RANK>
__global__ void __launch_bounds__(SCAN_THREADS) k_scan_down(DevSys<T> s) {
    if (s.ctrl->abort) return;
    const int base = blockIdx.x * SCAN_TILE + threadIdx.x * SCAN_ITEMS;
    int v[SCAN_ITEMS];
    int sum = 0;
#pragma unroll
    for (int k = 0; k < SCAN_ITEMS; ++k) {
        v[k] = scan_count<T, RANK>(s, base + k);
        sum += v[k];
    }
    int excl;
    block_excl_scan(sum, &excl);
    int run = s.scan_part[blockIdx.x] + excl;
    int* out = RANK ? s.rank_start : s.cell_beg;
#pragma unroll
    for (int k = 0; k < SCAN_ITEMS; ++k) {
        if (base + k < s.ncells) out[base + k] = run;
        run += v[k];
    }
}

// ---- resort ------------------------------------------------------------------
// Entry k of the cell of rank h moves to slot rank_start[h] + k; the entry
// follows.
template <class T>
__global__ void __launch_bounds__(256) k_resort_scatter(DevSys<T> s) {
    if (s.ctrl->abort) return;
    for (int h = blockIdx.x * blockDim.x + threadIdx.x; h < s.ncells; h += gridDim.x * blockDim.x) {
        const int c = s.cell_by_rank[h];
        if (!s.now[s.cell_rep[c]]) continue;
        V4<T>* p = s.cell_ent + s.cell_beg[c];
        const int b = s.rank_start[h], e = s.cell_beg[c + 1] - s.cell_beg[c];
        for (int k = 0; k < e; ++k) {
            s.perm[b + k] = bits_as_int(p[k].w);
            p[k].w = int_bits_as(T(0), b + k);
        }
    }
}

template <class T>
__global__ void __launch_bounds__(TILE) k_gather(DevSys<T> s, int cur, int permute_force) {
    if (s.ctrl->abort) return;
    const V4<T>* __restrict__ P = s.pos[cur];
    V4<T>* __restrict__ Q = s.pos[cur ^ 1];
    for (int t = blockIdx.x; t < s.ntiles; t += gridDim.x) {
        const Tile tl = s.tiles[t];
        if (!s.now[tl.rep] || (int)threadIdx.x >= tl.count) continue;
        const int n = tl.start + threadIdx.x;
        const int o = s.perm[n];
        Q[n] = ld4<T>(P + o);
        const V4<T> v = s.vel[o];
        s.vel_alt[n] = v;
        s.img_alt[n] = s.img[o];
        if (permute_force) s.frc_alt[n] = s.frc[o];
        s.slot_of_id[s.reps[tl.rep].p_off + bits_as_int(v.w)] = n;
    }
}

template <class T>
__global__ void __launch_bounds__(TILE) k_copyback(DevSys<T> s, int cur, int permute_force) {
    if (s.ctrl->abort) return;
    V4<T>* __restrict__ P = s.pos[cur];
    const V4<T>* __restrict__ Q = s.pos[cur ^ 1];
    for (int t = blockIdx.x; t < s.ntiles; t += gridDim.x) {
        const Tile tl = s.tiles[t];
        if (!s.now[tl.rep] || (int)threadIdx.x >= tl.count) continue;
        const int n = tl.start + threadIdx.x;
        P[n] = Q[n];
        const V4<T> v = s.vel_alt[n];
        s.vel[n] = v;
        s.img[n] = s.img_alt[n];
        if (permute_force) s.frc[n] = s.frc_alt[n];
        const int2 pg = s.bond_gid[s.reps[tl.rep].p_off + bits_as_int(v.w)];
        s.bond_slot[n] = make_int2(pg.x >= 0 ? s.slot_of_id[pg.x] : -1,
                                   pg.y >= 0 ? s.slot_of_id[pg.y] : -1);
    }
}

// ---- Verlet list ----------------------------------------------------------------
// One thread per particle, in cell order.  With cells of edge >= (rc + skin) / W
// (W = 1, or the sub-cells of W = 2) the stencil is (2W+1)^2 rows of 2W+1 cells.  The
// cells of a row are consecutive in index order, so a row is one contiguous
// range of the entry array (two where it wraps around the box in x).  The
// ranges of one plane of rows are loaded together, then each range is
// streamed with no further indirection.  Hits are packed into int4 groups in
// registers and stored as whole 16-byte groups, so the stores of a warp are
// contiguous.
// Candidates [p, e) of one contiguous range: distance test, hits packed into
// int4 groups.  SHIFT: the range lies across a face (the entries' and the
// particle's coordinates are shifted as the image codes say); without it the
// difference is the plain one, which equals the shifted form with zero shifts.
// LE: a row across a sheared face (Lees-Edwards): x is the nearest image of
// x_i - nz delta - x_j (xL holds nz delta, yL/zL the usual shifts).
// PUSH: how a hit enters the int4 group in registers.  false: at its place
// (cnt % 4), the group reset to padding once stored; true: pushed in at w,
// the others moving down one place, so a full group holds its four in order
// with no per-place select (the last, partial group is moved into place by
// verlet_last_group).  The lists are the same; which is faster depends on the
// hits per candidate and the registers left (the force-path tuner times both).
template <class T, bool EXCL, bool SHIFT, bool LE = false, bool PUSH = false>
__device__ __forceinline__ void verlet_range(const V4<T>* __restrict__ E, int p, int e, int i, int2 ex, T xo, T yo,
                                             T zo, T xL, T yL, T zL, T rl2, int tag, int cap, size_t stride,
                                             int pad, int& cnt, int4& grp, int4* __restrict__ out4, T Lx = T(0),
                                             T inv_Lx = T(0)) {
    for (; p < e; ++p) {
        const V4<T> xj = ld4<T>(E + p);
        const int j = bits_as_int(xj.w);
        T dx;
        if (LE) {
            dx = (xo - xj.x) - xL;
            dx -= Lx * rint(dx * inv_Lx);
        } else {
            dx = SHIFT ? xo - (xj.x - xL) : xo - xj.x;
        }
        const T dy = SHIFT ? yo - (xj.y - yL) : yo - xj.y;
        const T dz = SHIFT ? zo - (xj.z - zL) : zo - xj.z;
        bool hit = dx * dx + dy * dy + dz * dz < rl2 && j != i;
        if (EXCL) hit = hit && j != ex.x && j != ex.y;
        if (hit) {
            if constexpr (PUSH) {
                grp = make_int4(grp.y, grp.z, grp.w, j | tag);
                ++cnt;
                if ((cnt & 3) == 0 && cnt <= cap) out4[(size_t)((cnt >> 2) - 1) * stride] = grp;
            } else {
                const int l = cnt & 3;
                const int en = j | tag;
                if (l == 0) grp.x = en;
                else if (l == 1) grp.y = en;
                else if (l == 2) grp.z = en;
                else grp.w = en;
                ++cnt;
                if ((cnt & 3) == 0) {
                    if (cnt <= cap) out4[(size_t)((cnt >> 2) - 1) * stride] = grp;
                    grp = make_int4(pad, pad, pad, pad);
                }
            }
        }
    }
}

// The last, partial group of a list of cnt entries (cnt % 4 != 0) as stored:
// its entries first, in order, then the padding slot.
template <bool PUSH>
__device__ __forceinline__ int4 verlet_last_group(int4 grp, int cnt, int pad) {
    if constexpr (PUSH) {
        // the group's cnt % 4 entries sit at its top (w last)
        switch (cnt & 3) {
            case 1: return make_int4(grp.w, pad, pad, pad);
            case 2: return make_int4(grp.z, grp.w, pad, pad);
            default: return make_int4(grp.y, grp.z, grp.w, pad);
        }
    } else {
        (void)cnt;
        (void)pad;
        return grp;
    }
}

// replica index of a geometry record
template <class T>
__device__ __forceinline__ int g_rep(const DevSys<T>& s, const RepGeom<T>& g) {
    return (int)(&g - s.reps);
}

// One plane of rows across a sheared face (Lees-Edwards): x cells
// cxs - W .. cxs + W (cyclic) of rows cy - W .. cy + W, entries tagged with x
// code 3 (the x image is taken at evaluation time from the current delta).
template <class T, int W, bool EXCL, bool PUSH>
__device__ __forceinline__ void verlet_le_plane(const DevSys<T>& s, const RepGeom<T>& g, int i, const V4<T>& xi,
                                             int2 ex, int cxs, int az, int cy, T nd, T zo, T zL, T L0, T inv_L0,
                                             int czc, int& cnt, int4& grp, int4* __restrict__ out4) {
    const V4<T>* __restrict__ E = s.cell_ent;
    const int* __restrict__ B = s.cell_beg;
    const int nc0 = g.nc[0], nc1 = g.nc[1];
    const T L1 = g.L[1];
    for (int r = -W; r <= W; ++r) {
        int ay = cy + r, c = 0;
        if (ay < 0) { ay += nc1; c = 2; }
        else if (ay >= nc1) { ay -= nc1; c = 1; }
        const T yo = (c & 1) ? xi.y - L1 : xi.y, yL = (c & 2) ? L1 : T(0);
        const int tag = (3 | (c << 2) | (czc << 4)) << NBR_INDEX_BITS;
        const int base = g.cell_off + (az * nc1 + ay) * nc0;
        int lo = cxs - W, hi = cxs + W;
        // the cyclic x range as up to two contiguous pieces
        int p0b, p0e, p1b = 0, p1e = 0;
        if (lo < 0) {
            p0b = __ldg(B + base + lo + nc0);
            p0e = __ldg(B + base + nc0);
            p1b = __ldg(B + base);
            p1e = __ldg(B + base + hi + 1);
        } else if (hi >= nc0) {
            p0b = __ldg(B + base + lo);
            p0e = __ldg(B + base + nc0);
            p1b = __ldg(B + base);
            p1e = __ldg(B + base + hi - nc0 + 1);
        } else {
            p0b = __ldg(B + base + lo);
            p0e = __ldg(B + base + hi + 1);
        }
        verlet_range<T, EXCL, true, true, PUSH>(E, p0b, p0e, i, ex, xi.x, yo, zo, nd, yL, zL, s.rlist2, tag, s.cap,
                                          (size_t)s.stride, s.nbr_pad, cnt, grp, out4, L0, inv_L0);
        verlet_range<T, EXCL, true, true, PUSH>(E, p1b, p1e, i, ex, xi.x, yo, zo, nd, yL, zL, s.rlist2, tag, s.cap,
                                          (size_t)s.stride, s.nbr_pad, cnt, grp, out4, L0, inv_L0);
    }
}

// The full stencil of particle i: every row over the same x cells cx - W ..
// cx + W (whole cells: the trimmed form below costs more in registers and
// per-row work than the quarter of the candidates it saves).
template <class T, int W, bool EXCL, bool LE, bool PUSH>
__device__ __forceinline__ void verlet_stencil_full(const DevSys<T>& s, const RepGeom<T>& g, int i,
                                               const V4<T>& xi, int2 ex, int& cnt, int4& grp,
                                               int4* __restrict__ out4) {
    constexpr int NR = 2 * W + 1;
    const V4<T>* __restrict__ E = s.cell_ent;
    const int* __restrict__ B = s.cell_beg;
    const int nc0 = g.nc[0], nc1 = g.nc[1], nc2 = g.nc[2];
    const int cx = cell_coord(xi.x, g.cells_per_len[0], nc0);
    const int cy = cell_coord(xi.y, g.cells_per_len[1], nc1);
    const int cz = cell_coord(xi.z, g.cells_per_len[2], nc2);
    const T L0 = g.L[0], L1 = g.L[1], L2 = g.L[2];
    const T rl2 = s.rlist2;
    const int cap = s.cap;
    const size_t stride = (size_t)s.stride;
    // the x ranges are the same for every row: [sl0, sh0] and, where the row
    // wraps, [sl1, sh1] (image codes cxc0, cxc1)
    int sl0 = cx - W, sh0 = cx + W, cxc0 = 0, sl1 = 0, sh1 = -1, cxc1 = 0;
    if (sl0 < 0) {
        sl1 = 0;
        sh1 = sh0;
        sl0 += nc0;
        sh0 = nc0 - 1;
        cxc0 = 2;
    } else if (sh0 >= nc0) {
        sl1 = 0;
        sh1 = sh0 - nc0;
        cxc1 = 1;
        sh0 = nc0 - 1;
    }
    const T xo0 = (cxc0 & 1) ? xi.x - L0 : xi.x, xL0 = (cxc0 & 2) ? L0 : T(0);
    const T xo1 = (cxc1 & 1) ? xi.x - L0 : xi.x, xL1 = (cxc1 & 2) ? L0 : T(0);
    // Lees-Edwards: delta of this build reduced into [0, Lx)
    const T le_d = LE ? (T)le_reduce(s.le_db[g_rep(s, g)], (double)L0) : T(0);
    const T inv_L0 = LE ? T(1) / L0 : T(0);
#pragma unroll 1
    for (int dz = -W; dz <= W; ++dz) {
        int az = cz + dz, czc = 0;
        if (az < 0) { az += nc2; czc = 2; }
        else if (az >= nc2) { az -= nc2; czc = 1; }
        const T zo = (czc & 1) ? xi.z - L2 : xi.z, zL = (czc & 2) ? L2 : T(0);
        if (LE && czc != 0) {
            // a plane across a sheared face: the partners' image is displaced
            // by nz delta along x; its x cells are found around x_i - nz delta
            const int nz = czc == 1 ? 1 : -1;
            const T nd = (T)nz * le_d;
            T xs = xi.x - nd;
            if (xs < T(0)) xs += L0;
            if (xs >= L0) xs -= L0;
            const int cxs = cell_coord(xs, g.cells_per_len[0], nc0);
            verlet_le_plane<T, W, EXCL, PUSH>(s, g, i, xi, ex, cxs, az, cy, nd, zo, zL, L0, inv_L0, czc, cnt, grp, out4);
            continue;
        }
        int pb[NR][2], pe[NR][2], cyc[NR];
#pragma unroll
        for (int r = 0; r < NR; ++r) {
            int ay = cy + r - W, c = 0;
            if (ay < 0) { ay += nc1; c = 2; }
            else if (ay >= nc1) { ay -= nc1; c = 1; }
            cyc[r] = c;
            const int base = g.cell_off + (az * nc1 + ay) * nc0;
            pb[r][0] = __ldg(B + base + sl0);
            pe[r][0] = __ldg(B + base + sh0 + 1);
            pb[r][1] = sh1 >= 0 ? __ldg(B + base + sl1) : 0;
            pe[r][1] = sh1 >= 0 ? __ldg(B + base + sh1 + 1) : 0;
        }
#pragma unroll
        for (int r = 0; r < NR; ++r) {
            const T yo = (cyc[r] & 1) ? xi.y - L1 : xi.y, yL = (cyc[r] & 2) ? L1 : T(0);
#pragma unroll
            for (int part = 0; part < 2; ++part) {
                const T xo = part ? xo1 : xo0, xL = part ? xL1 : xL0;
                const int tag = ((part ? cxc1 : cxc0) | (cyc[r] << 2) | (czc << 4)) << NBR_INDEX_BITS;
                // a range that crosses no face (the common case) needs no shift
                if (tag == 0)
                    verlet_range<T, EXCL, false, false, PUSH>(E, pb[r][part], pe[r][part], i, ex, xo, yo, zo, xL, yL, zL, rl2,
                                                 tag, cap, stride, s.nbr_pad, cnt, grp, out4);
                else
                    verlet_range<T, EXCL, true, false, PUSH>(E, pb[r][part], pe[r][part], i, ex, xo, yo, zo, xL, yL, zL, rl2,
                                                tag, cap, stride, s.nbr_pad, cnt, grp, out4);
            }
        }
    }
}

// The stencil of particle i, trimmed to the list sphere: a row of cells (one
// y, one z) is searched only over the x cells that the sphere's chord at the
// row's nearest point reaches, and rows the sphere misses are skipped.  The
// nearest point of a row lies dmin_y, dmin_z away (cell units: the particle's
// offset inside its own cell to the row's slab), the chord's half-width is
// sqrt(rl^2 - dmin_y^2 - dmin_z^2).  Margins of 1e-4 cell widened every range
// against rounding, so no pair inside rl is missed (the distance test itself
// is unchanged); about a quarter (whole cells) to a third (half cells) of the
// candidates of the full stencil go.  Used with sub-cells (W >= 2), where
// rows are many and short; with whole cells the full stencil is faster.
template <class T, int W, bool EXCL, bool LE, bool PUSH>
__device__ __forceinline__ void verlet_stencil_trim(const DevSys<T>& s, const RepGeom<T>& g, int i,
                                               const V4<T>& xi, int2 ex, int& cnt, int4& grp,
                                               int4* __restrict__ out4) {
    constexpr int NR = 2 * W + 1;
    const V4<T>* __restrict__ E = s.cell_ent;
    const int* __restrict__ B = s.cell_beg;
    const int nc0 = g.nc[0], nc1 = g.nc[1], nc2 = g.nc[2];
    const int cx = cell_coord(xi.x, g.cells_per_len[0], nc0);
    const int cy = cell_coord(xi.y, g.cells_per_len[1], nc1);
    const int cz = cell_coord(xi.z, g.cells_per_len[2], nc2);
    const T L0 = g.L[0], L1 = g.L[1], L2 = g.L[2];
    const T rl2 = s.rlist2;
    const int cap = s.cap;
    const size_t stride = (size_t)s.stride;
    // position in cell units, offsets inside the own cell, cell edges
    const T ux = xi.x * g.cells_per_len[0];
    const T fy = xi.y * g.cells_per_len[1] - (T)cy, fz = xi.z * g.cells_per_len[2] - (T)cz;
    const T ey = L1 / (T)nc1, ez = L2 / (T)nc2;
    const T margin = T(1e-4);
    // Lees-Edwards: delta of this build reduced into [0, Lx)
    const T le_d = LE ? (T)le_reduce(s.le_db[g_rep(s, g)], (double)L0) : T(0);
    const T inv_L0 = LE ? T(1) / L0 : T(0);
#pragma unroll 1
    for (int dz = -W; dz <= W; ++dz) {
        int az = cz + dz, czc = 0;
        if (az < 0) { az += nc2; czc = 2; }
        else if (az >= nc2) { az -= nc2; czc = 1; }
        const T zo = (czc & 1) ? xi.z - L2 : xi.z, zL = (czc & 2) ? L2 : T(0);
        if (LE && czc != 0) {
            // a plane across a sheared face: the partners' image is displaced
            // by nz delta along x; its x cells are found around x_i - nz delta
            const int nz = czc == 1 ? 1 : -1;
            const T nd = (T)nz * le_d;
            T xs = xi.x - nd;
            if (xs < T(0)) xs += L0;
            if (xs >= L0) xs -= L0;
            const int cxs = cell_coord(xs, g.cells_per_len[0], nc0);
            verlet_le_plane<T, W, EXCL, PUSH>(s, g, i, xi, ex, cxs, az, cy, nd, zo, zL, L0, inv_L0, czc, cnt, grp, out4);
            continue;
        }
        T dmz = dz > 0 ? (T)dz - fz : (dz < 0 ? fz + (T)(-dz - 1) : T(0));
        dmz = dmz > margin ? (dmz - margin) * ez : T(0);
        const T dz2 = dmz * dmz;
        // rows whose ranges are loaded together (all of a plane for W <= 2;
        // one at a time for W = 3, whose seven rows would not fit the
        // registers)
        constexpr int RG = W <= 2 ? NR : 1;
#pragma unroll 1
        for (int r0 = 0; r0 < NR; r0 += RG) {
        int pb[RG][2], pe[RG][2], cyc[RG];
#pragma unroll
        for (int r = 0; r < RG; ++r) {
            const int dy = r0 + r - W;
            int ay = cy + dy, c = 0;
            if (ay < 0) { ay += nc1; c = 2; }
            else if (ay >= nc1) { ay -= nc1; c = 1; }
            T dmy = dy > 0 ? (T)dy - fy : (dy < 0 ? fy + (T)(-dy - 1) : T(0));
            dmy = dmy > margin ? (dmy - margin) * ey : T(0);
            const T d2 = dmy * dmy + dz2;
            // x cells of the chord, unwrapped, inside cx - W .. cx + W
            int lo = cx + 1, hi = cx;  // empty when the sphere misses the row
            if (d2 < rl2) {
                const T wc = sqrt(rl2 - d2) * g.cells_per_len[0] + margin;
                lo = max(cx - W, (int)floor(ux - wc));
                hi = min(cx + W, (int)floor(ux + wc));
            }
            // the chord as up to two contiguous ranges of the row
            int s0 = lo, h0 = hi, c0 = 0, s1 = 0, h1 = -1, c1 = 0;
            if (lo < 0) {
                if (hi < 0) {
                    s0 = lo + nc0;
                    h0 = hi + nc0;
                } else {
                    s0 = lo + nc0;
                    h0 = nc0 - 1;
                    s1 = 0;
                    h1 = hi;
                }
                c0 = 2;
            } else if (hi >= nc0) {
                if (lo >= nc0) {
                    s0 = lo - nc0;
                    h0 = hi - nc0;
                    c0 = 1;
                } else {
                    h0 = nc0 - 1;
                    s1 = 0;
                    h1 = hi - nc0;
                    c1 = 1;
                }
            }
            cyc[r] = c | (c0 << 2) | (c1 << 4);  // y code, then the x codes of both ranges
            const int base = g.cell_off + (az * nc1 + ay) * nc0;
            pb[r][0] = h0 >= s0 ? __ldg(B + base + s0) : 0;
            pe[r][0] = h0 >= s0 ? __ldg(B + base + h0 + 1) : 0;
            pb[r][1] = h1 >= s1 ? __ldg(B + base + s1) : 0;
            pe[r][1] = h1 >= s1 ? __ldg(B + base + h1 + 1) : 0;
        }
#pragma unroll
        for (int r = 0; r < RG; ++r) {
            const int cyr = cyc[r] & 3;
            const T yo = (cyr & 1) ? xi.y - L1 : xi.y, yL = (cyr & 2) ? L1 : T(0);
#pragma unroll
            for (int part = 0; part < 2; ++part) {
                const int cxc = (cyc[r] >> (2 + 2 * part)) & 3;
                const T xo = (cxc & 1) ? xi.x - L0 : xi.x, xL = (cxc & 2) ? L0 : T(0);
                const int tag = (cxc | (cyr << 2) | (czc << 4)) << NBR_INDEX_BITS;
                // a range that crosses no face (the common case) needs no shift
                if (tag == 0)
                    verlet_range<T, EXCL, false, false, PUSH>(E, pb[r][part], pe[r][part], i, ex, xo, yo, zo, xL, yL, zL, rl2,
                                                 tag, cap, stride, s.nbr_pad, cnt, grp, out4);
                else
                    verlet_range<T, EXCL, true, false, PUSH>(E, pb[r][part], pe[r][part], i, ex, xo, yo, zo, xL, yL, zL, rl2,
                                                tag, cap, stride, s.nbr_pad, cnt, grp, out4);
            }
        }
        }
    }
}

template <class T, int W, bool EXCL, bool LE, bool PUSH>
__global__ void __launch_bounds__(TILE, sizeof(T) == 4 ? (W > 1 ? 8 : (EXCL || LE ? 7 : 9)) : 5) k_verlet(DevSys<T> s, int cur) {
    // the first tile's record is requested together with the abort flag
    Tile tl0 = {0, 0, 0, 0};
    if ((int)blockIdx.x < s.ntiles) tl0 = ld_tile_early(s.tiles + blockIdx.x);
    if (s.ctrl->abort) return;
    for (int t = blockIdx.x; t < s.ntiles; t += gridDim.x) {
        const Tile tl = t == (int)blockIdx.x ? tl0 : s.tiles[t];
        if (!s.now[tl.rep]) continue;  // uniform over the block
        int cnt = 0;
        if ((int)threadIdx.x < tl.count) {
            const RepGeom<T>& g = s.reps[tl.rep];
            // threads follow the entry array (cell order: a warp walks a run of
            // cells along x, whose stencils share their rows), not the storage
            // order; a replica's entries fill the same index range as its slots
            const V4<T> xi = ld4<T>(s.cell_ent + tl.start + threadIdx.x);
            const int i = bits_as_int(xi.w);
            s.xb[i] = xi;
            // bonded partners left out of the list when 1-2 exclusions are on
            const int2 ex = EXCL ? s.bond_slot[i] : make_int2(-1, -1);
            int4* __restrict__ out4 = reinterpret_cast<int4*>(s.nbr) + i;
            int4 grp = make_int4(s.nbr_pad, s.nbr_pad, s.nbr_pad, s.nbr_pad);
            if constexpr (W == 1) verlet_stencil_full<T, W, EXCL, LE, PUSH>(s, g, i, xi, ex, cnt, grp, out4);
            else verlet_stencil_trim<T, W, EXCL, LE, PUSH>(s, g, i, xi, ex, cnt, grp, out4);
            const int cap = s.cap;
            if ((cnt & 3) != 0 && cnt <= cap) out4[(size_t)(cnt >> 2) * s.stride] = verlet_last_group<PUSH>(grp, cnt, s.nbr_pad);
            s.nbr_cnt[i] = cnt < cap ? cnt : cap;
            if (cnt > cap) {
                atomicMax(&s.ctrl->need_cap, (unsigned int)cnt);
                atomicOr(&s.ctrl->err, ERRBIT_OVERFLOW);
                s.ctrl->abort = 1;
            }
        }
        // largest count: one atomic per warp, no block barrier
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) cnt = max(cnt, __shfl_xor_sync(0xffffffffu, cnt, o));
        if ((threadIdx.x & 31) == 0 && cnt > 0) atomicMax(&s.ctrl->max_count, (unsigned int)cnt);
    }
}

template <class T>
__global__ void k_request_all(DevSys<T> s) {
    for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < s.R; r += gridDim.x * blockDim.x)
        s.req[r] = 1;
    if (blockIdx.x == 0 && threadIdx.x == 0) s.ctrl->any_req = 1;
}

// ---- launchers -------------------------------------------------------------------
static inline int grid_for(int n, int block) { return (n + block - 1) / block; }

template <class T>
int Launch<T>::rebuild(const DevSys<T>& s, int cur, bool resort, bool permute_force, cudaStream_t st) {
    const int gt = s.ntiles;
    const int gc = grid_for(s.ncells, 256);
    k_prep<T><<<gc, 256, 0, st>>>(s);
    k_bin<T><<<gt, TILE, 0, st>>>(s, cur);
    k_scan_reduce<T, false><<<s.nscan_blocks, SCAN_THREADS, 0, st>>>(s);
    k_scan_top<T><<<1, SCAN_THREADS, 0, st>>>(s);
    k_scan_down<T, false><<<s.nscan_blocks, SCAN_THREADS, 0, st>>>(s);
    k_place<T><<<gt, TILE, 0, st>>>(s, cur);
    k_cellsort<T><<<gc, 256, 0, st>>>(s);
    int launched = 7;
    if (resort) {
        k_scan_reduce<T, true><<<s.nscan_blocks, SCAN_THREADS, 0, st>>>(s);
        k_scan_top<T><<<1, SCAN_THREADS, 0, st>>>(s);
        k_scan_down<T, true><<<s.nscan_blocks, SCAN_THREADS, 0, st>>>(s);
        k_resort_scatter<T><<<gc, 256, 0, st>>>(s);
        k_gather<T><<<gt, TILE, 0, st>>>(s, cur, permute_force ? 1 : 0);
        k_copyback<T><<<gt, TILE, 0, st>>>(s, cur, permute_force ? 1 : 0);
        launched += 6;
    }
    // list-free mode: the binning is all that is needed
    if (s.cells_mode) return launched;
#define ESPP_VERLET(W, E, P)                                                  \
    do {                                                                      \
        if (s.le_on) k_verlet<T, W, E, true, P><<<gt, TILE, 0, st>>>(s, cur);  \
        else k_verlet<T, W, E, false, P><<<gt, TILE, 0, st>>>(s, cur);        \
    } while (0)
#define ESPP_VERLET_P(W, P)                       \
    do {                                         \
        if (s.excl_bonded) ESPP_VERLET(W, true, P);  \
        else ESPP_VERLET(W, false, P);            \
    } while (0)
    // the pushed stores are built for whole and third cells (on half cells
    // they only cost registers)
    if (s.cell_w == 1) {
        if (s.list_push) ESPP_VERLET_P(1, true);
        else ESPP_VERLET_P(1, false);
    } else if (s.cell_w == 2) {
        ESPP_VERLET_P(2, false);
    } else {
        if (s.list_push) ESPP_VERLET_P(3, true);
        else ESPP_VERLET_P(3, false);
    }
#undef ESPP_VERLET_P
#undef ESPP_VERLET
    launched += 1;
    // mirrored entries for the learned potential's pair-once evaluation
    if (s.mlp_on && s.mlp_rev) launched += Launch<T>::mlp_rev(s, st);
    return launched;
}

template <class T>
void Launch<T>::request_all(const DevSys<T>& s, cudaStream_t st) {
    k_request_all<T><<<grid_for(s.R, 256), 256, 0, st>>>(s);
}

template int Launch<float>::rebuild(const DevSys<float>&, int, bool, bool, cudaStream_t);
template int Launch<double>::rebuild(const DevSys<double>&, int, bool, bool, cudaStream_t);
template void Launch<float>::request_all(const DevSys<float>&, cudaStream_t);
template void Launch<double>::request_all(const DevSys<double>&, cudaStream_t);

int scan_blocks_for(int ncells) { return (ncells + SCAN_TILE - 1) / SCAN_TILE; }

}  // namespace espp

// Rebuild pipeline: linked-cell binning, the periodic Hilbert resort of every
// particle array into cell order, and the full Verlet list with skin.  Paper
// "Software design" ("Parallelization": CellGrid linked cells;
// "Performance optimizations": cell decomposition and data sorting) and
// "Example usage" (VerletList(system, cutoff) with system.skin).
//
// Every rebuild (inside the step graphs, when a replica asked for it):
//   prep      latch the per-replica requests, clear those replicas' cell counts
//   bin       cell of every particle; the particle's position and storage slot
//             go to an atomic slot of its cell's fixed-capacity entry array
//   cellsort  entries of each cell in ascending storage slot, so the list does
//             not depend on the order of the atomics
//   verlet    27-cell search from the cell entries (contiguous, no further
//             indirection), full list (both directions) as groups of four
//             indices, nbr4[g * stride + i]; records the build positions
// A resort (launched between step graphs every `resort_every` steps, and on
// every explicit build) additionally runs, between cellsort and verlet:
//   scan x3   exclusive scan of the cell counts in Hilbert-rank order
//   scatter   new slot of every entry (its cell's first slot + its rank in the
//             cell); the entries switch to the new slots
//   gather    permuted copies of positions, velocities, forces, images
//   copyback  copies back and maps bond partners to their new slots
// Replicas whose request flag is clear skip every step after `prep`.
#include "kernels.cuh"

namespace espp {

constexpr int SCAN_THREADS = 256;
constexpr int SCAN_ITEMS = 8;
constexpr int SCAN_TILE = SCAN_THREADS * SCAN_ITEMS;

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
        for (int r = threadIdx.x; r < s.R; r += blockDim.x) s.now[r] = s.req[r];
        if (threadIdx.x == 0 && s.ctrl->any_req) {
            s.ctrl->n_rebuilds += 1;
            s.ctrl->max_count = 0;
        }
    }
}

template <class T>
__global__ void __launch_bounds__(TILE) k_bin(DevSys<T> s, int cur) {
    if (s.ctrl->abort) return;
    if (blockIdx.x == 0) {
        for (int r = threadIdx.x; r < s.R; r += blockDim.x) s.req[r] = 0;
        if (threadIdx.x == 0) s.ctrl->any_req = 0;
    }
    V4<T>* __restrict__ P = s.pos[cur];
    for (int t = blockIdx.x; t < s.ntiles; t += gridDim.x) {
        const Tile tl = s.tiles[t];
        if (!s.now[tl.rep] || (int)threadIdx.x >= tl.count) continue;
        const int i = tl.start + threadIdx.x;
        V4<T> p = P[i];
        // positions are wrapped into the box at list builds only
        const RepGeom<T>& g = s.reps[tl.rep];
        const int wx = wrap_coord(p.x, g.L[0]), wy = wrap_coord(p.y, g.L[1]), wz = wrap_coord(p.z, g.L[2]);
        if (wx | wy | wz) {
            P[i] = p;
            int4 im = s.img[i];
            im.x += wx;
            im.y += wy;
            im.z += wz;
            s.img[i] = im;
        }
        const int h = cell_of(g, p);
        const int slot = atomicAdd(&s.cell_cnt[h], 1);
        if (slot < s.capc) {
            p.w = int_bits_as(T(0), i);
            s.cell_xyz[(size_t)h * s.capc + slot] = p;
        } else {
            atomicMax(&s.ctrl->need_capc, (unsigned int)(slot + 1));
            atomicOr(&s.ctrl->err, ERRBIT_CELL);
            s.ctrl->abort = 1;
        }
    }
}

// Entries of each cell in ascending storage slot (a handful per cell).
template <class T>
__global__ void __launch_bounds__(256) k_cellsort(DevSys<T> s) {
    if (s.ctrl->abort) return;
    for (int h = blockIdx.x * blockDim.x + threadIdx.x; h < s.ncells; h += gridDim.x * blockDim.x) {
        if (!s.now[s.cell_rep[h]]) continue;
        V4<T>* p = s.cell_xyz + (size_t)h * s.capc;
        const int e = min(s.cell_cnt[h], s.capc);
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
    }
}

// ---- exclusive scan of the cell counts (three phases, no inter-block waits) --
__device__ __forceinline__ int warp_incl_scan(int v) {
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        int u = __shfl_up_sync(0xffffffffu, v, o);
        if (lane >= o) v += u;
    }
    return v;
}

// block-wide exclusive scan of one int per thread; returns the block total
__device__ __forceinline__ int block_excl_scan(int v, int* excl_out) {
    __shared__ int wsum[SCAN_THREADS / 32];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    int inc = warp_incl_scan(v);
    if (lane == 31) wsum[w] = inc;
    __syncthreads();
    if (w == 0) {
        int t = lane < SCAN_THREADS / 32 ? wsum[lane] : 0;
        t = warp_incl_scan(t);
        if (lane < SCAN_THREADS / 32) wsum[lane] = t;
    }
    __syncthreads();
    const int base = w > 0 ? wsum[w - 1] : 0;
    *excl_out = base + inc - v;
    const int total = wsum[SCAN_THREADS / 32 - 1];
    __syncthreads();
    return total;
}

template <class T>
__global__ void __launch_bounds__(SCAN_THREADS) k_scan_reduce(DevSys<T> s) {
    if (s.ctrl->abort) return;
    const int base = blockIdx.x * SCAN_TILE + threadIdx.x * SCAN_ITEMS;
    int sum = 0;
#pragma unroll
    for (int k = 0; k < SCAN_ITEMS; ++k)
        if (base + k < s.ncells) sum += s.cell_cnt[s.cell_by_rank[base + k]];
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

template <class T>
__global__ void __launch_bounds__(SCAN_THREADS) k_scan_down(DevSys<T> s) {
    if (s.ctrl->abort) return;
    const int base = blockIdx.x * SCAN_TILE + threadIdx.x * SCAN_ITEMS;
    int v[SCAN_ITEMS];
    int sum = 0;
#pragma unroll
    for (int k = 0; k < SCAN_ITEMS; ++k) {
        v[k] = base + k < s.ncells ? s.cell_cnt[s.cell_by_rank[base + k]] : 0;
        sum += v[k];
    }
    int excl;
    block_excl_scan(sum, &excl);
    int run = s.scan_part[blockIdx.x] + excl;
#pragma unroll
    for (int k = 0; k < SCAN_ITEMS; ++k) {
        if (base + k < s.ncells) s.cell_start[base + k] = run;
        run += v[k];
    }
}

// ---- resort ------------------------------------------------------------------
// Entry k of the cell of rank h moves to slot start[h] + k; the entry follows.
template <class T>
__global__ void __launch_bounds__(256) k_resort_scatter(DevSys<T> s) {
    if (s.ctrl->abort) return;
    for (int h = blockIdx.x * blockDim.x + threadIdx.x; h < s.ncells; h += gridDim.x * blockDim.x) {
        const int c = s.cell_by_rank[h];
        if (!s.now[s.cell_rep[c]]) continue;
        V4<T>* p = s.cell_xyz + (size_t)c * s.capc;
        const int b = s.cell_start[h], e = min(s.cell_cnt[c], s.capc);
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
// One thread per particle.  The 27 neighbour cells are visited as three planes
// of nine; the nine counts of a plane are loaded together, then each cell's
// entries (position and slot, contiguous) are streamed with no further
// indirection.  Hits are packed into int4 groups in registers and stored as
// whole 16-byte groups, so the stores of a warp are contiguous.
template <class T>
__global__ void __launch_bounds__(TILE) k_verlet(DevSys<T> s, int cur) {
    if (s.ctrl->abort) return;
    __shared__ int smax;
    const V4<T>* __restrict__ P = s.pos[cur];
    for (int t = blockIdx.x; t < s.ntiles; t += gridDim.x) {
        const Tile tl = s.tiles[t];
        if (!s.now[tl.rep]) continue;  // uniform over the block
        if (threadIdx.x == 0) smax = 0;
        __syncthreads();
        if ((int)threadIdx.x < tl.count) {
            const RepGeom<T>& g = s.reps[tl.rep];
            const int i = tl.start + threadIdx.x;
            const V4<T> xi = ld4<T>(P + i);
            s.xb[i] = xi;
            const int nc0 = g.nc[0], nc1 = g.nc[1], nc2 = g.nc[2];
            const int cx = cell_coord(xi.x, g.cells_per_len[0], nc0);
            const int cy = cell_coord(xi.y, g.cells_per_len[1], nc1);
            const int cz = cell_coord(xi.z, g.cells_per_len[2], nc2);
            const int xm = cx == 0 ? nc0 - 1 : cx - 1, xp = cx == nc0 - 1 ? 0 : cx + 1;
            const int ym = cy == 0 ? nc1 - 1 : cy - 1, yp = cy == nc1 - 1 ? 0 : cy + 1;
            const T L0 = g.L[0], L1 = g.L[1], L2 = g.L[2];
            const T xim = xi.x - L0, yim = xi.y - L1, zim = xi.z - L2;
            const T rl2 = s.rlist2;
            const int cap = s.cap, capc = s.capc;
            const size_t stride = (size_t)s.stride;
            int4* __restrict__ out4 = reinterpret_cast<int4*>(s.nbr) + i;
            // bonded partners left out of the list when 1-2 exclusions are on
            const int2 ex = s.excl_bonded ? s.bond_slot[i] : make_int2(-1, -1);
            // image codes of the stencil rows: 1 = across the upper face, 2 = lower
            const int cxm = cx == 0 ? 2 : 0, cxp = cx == nc0 - 1 ? 1 : 0;
            const int cym = cy == 0 ? 2 : 0, cyp = cy == nc1 - 1 ? 1 : 0;
            int cnt = 0;
            int4 grp = make_int4(-1, -1, -1, -1);
#pragma unroll 1
            for (int pz = 0; pz < 3; ++pz) {
                int az = cz + pz - 1;
                int czc = 0;
                if (az < 0) { az += nc2; czc = 2; }
                if (az >= nc2) { az -= nc2; czc = 1; }
                int hh[9], cn[9];
#pragma unroll
                for (int q = 0; q < 9; ++q) {
                    const int ay = q / 3 == 0 ? ym : (q / 3 == 1 ? cy : yp);
                    const int ax = q % 3 == 0 ? xm : (q % 3 == 1 ? cx : xp);
                    hh[q] = g.cell_off + (az * nc1 + ay) * nc0 + ax;
                }
#pragma unroll
                for (int q = 0; q < 9; ++q) cn[q] = min(__ldg(s.cell_cnt + hh[q]), capc);
#pragma unroll
                for (int q = 0; q < 9; ++q) {
                    const int ccx = q % 3 == 0 ? cxm : (q % 3 == 2 ? cxp : 0);
                    const int ccy = q / 3 == 0 ? cym : (q / 3 == 2 ? cyp : 0);
                    const int code = ccx | (ccy << 2) | (czc << 4);
                    const int tag = code << NBR_INDEX_BITS;
                    const V4<T>* __restrict__ ent = s.cell_xyz + (size_t)hh[q] * capc;
                    for (int k = 0; k < cn[q]; ++k) {
                        const V4<T> xj = ld4<T>(ent + k);
                        const int j = bits_as_int(xj.w);
                        if (j == i || j == ex.x || j == ex.y) continue;
                        const T ddx = shifted_diff(xi.x, xim, xj.x, L0, ccx);
                        const T ddy = shifted_diff(xi.y, yim, xj.y, L1, ccy);
                        const T ddz = shifted_diff(xi.z, zim, xj.z, L2, czc);
                        if (ddx * ddx + ddy * ddy + ddz * ddz < rl2) {
                            const int l = cnt & 3;
                            const int e = j | tag;
                            if (l == 0) grp.x = e;
                            else if (l == 1) grp.y = e;
                            else if (l == 2) grp.z = e;
                            else grp.w = e;
                            ++cnt;
                            if ((cnt & 3) == 0) {
                                if (cnt <= cap) out4[(size_t)((cnt >> 2) - 1) * stride] = grp;
                                grp = make_int4(-1, -1, -1, -1);
                            }
                        }
                    }
                }
            }
            if ((cnt & 3) != 0 && cnt <= cap) out4[(size_t)(cnt >> 2) * stride] = grp;
            s.nbr_cnt[i] = cnt < cap ? cnt : cap;
            atomicMax(&smax, cnt);
            if (cnt > cap) {
                atomicMax(&s.ctrl->need_cap, (unsigned int)cnt);
                atomicOr(&s.ctrl->err, ERRBIT_OVERFLOW);
                s.ctrl->abort = 1;
            }
        }
        __syncthreads();
        if (threadIdx.x == 0) atomicMax(&s.ctrl->max_count, (unsigned int)smax);
        __syncthreads();
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
    k_cellsort<T><<<gc, 256, 0, st>>>(s);
    int launched = 4;
    if (resort) {
        k_scan_reduce<T><<<s.nscan_blocks, SCAN_THREADS, 0, st>>>(s);
        k_scan_top<T><<<1, SCAN_THREADS, 0, st>>>(s);
        k_scan_down<T><<<s.nscan_blocks, SCAN_THREADS, 0, st>>>(s);
        k_resort_scatter<T><<<gc, 256, 0, st>>>(s);
        k_gather<T><<<gt, TILE, 0, st>>>(s, cur, permute_force ? 1 : 0);
        k_copyback<T><<<gt, TILE, 0, st>>>(s, cur, permute_force ? 1 : 0);
        launched += 6;
    }
    k_verlet<T><<<gt, TILE, 0, st>>>(s, cur);
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

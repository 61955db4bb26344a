// Rebuild pipeline: linked-cell binning, the periodic Hilbert resort of every
// particle array into cell order, and the full Verlet list with skin.  Paper
// "Software design" ("Parallelization": CellGrid linked cells;
// "Performance optimizations": cell decomposition and data sorting) and
// "Example usage" (VerletList(system, cutoff) with system.skin).
//
// Every rebuild (inside the step graphs, when a replica asked for it):
//   prep      latch the per-replica requests, clear those replicas' cell counts
//   bin       cell of every particle (Hilbert rank space); atomic slot in a
//             fixed-capacity member array per cell
//   cellsort  members of each cell in ascending storage slot, so the list
//             does not depend on the order of the atomics
//   verlet    27-cell search, full list (both directions) as groups of four
//             indices, nbr4[g * stride + i]; records the build positions
// A resort (launched between step graphs every `resort_every` steps, and on
// every explicit build) additionally runs, between cellsort and verlet:
//   scan x3   exclusive scan of the cell counts -> first slot of each cell
//   scatter   new slot of every member; the member lists switch to new slots
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
    const V4<T>* __restrict__ P = s.pos[cur];
    for (int t = blockIdx.x; t < s.ntiles; t += gridDim.x) {
        const Tile tl = s.tiles[t];
        if (!s.now[tl.rep] || (int)threadIdx.x >= tl.count) continue;
        const RepGeom<T>& g = s.reps[tl.rep];
        const int i = tl.start + threadIdx.x;
        const V4<T> p = ld4<T>(P + i);
        const int cx = cell_coord(p.x, g.cells_per_len[0], g.nc[0]);
        const int cy = cell_coord(p.y, g.cells_per_len[1], g.nc[1]);
        const int cz = cell_coord(p.z, g.cells_per_len[2], g.nc[2]);
        const int h = s.cell_rank[g.cell_off + (cz * g.nc[1] + cy) * g.nc[0] + cx];
        const int slot = atomicAdd(&s.cell_cnt[h], 1);
        if (slot < s.capc) {
            s.cell_list[(size_t)h * s.capc + slot] = i;
        } else {
            atomicMax(&s.ctrl->need_capc, (unsigned int)(slot + 1));
            atomicOr(&s.ctrl->err, ERRBIT_CELL);
            s.ctrl->abort = 1;
        }
    }
}

// Members of each cell in ascending storage slot (a handful per cell).
template <class T>
__global__ void __launch_bounds__(256) k_cellsort(DevSys<T> s) {
    if (s.ctrl->abort) return;
    for (int h = blockIdx.x * blockDim.x + threadIdx.x; h < s.ncells; h += gridDim.x * blockDim.x) {
        if (!s.now[s.cell_rep[h]]) continue;
        int* p = s.cell_list + (size_t)h * s.capc;
        const int e = min(s.cell_cnt[h], s.capc);
        for (int k = 1; k < e; ++k) {
            const int key = p[k];
            int q = k - 1;
            while (q >= 0 && p[q] > key) {
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
        if (base + k < s.ncells) sum += s.cell_cnt[base + k];
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
        v[k] = base + k < s.ncells ? s.cell_cnt[base + k] : 0;
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
// Member k of cell h moves to slot start[h] + k; the member list follows.
template <class T>
__global__ void __launch_bounds__(256) k_resort_scatter(DevSys<T> s) {
    if (s.ctrl->abort) return;
    for (int h = blockIdx.x * blockDim.x + threadIdx.x; h < s.ncells; h += gridDim.x * blockDim.x) {
        if (!s.now[s.cell_rep[h]]) continue;
        int* p = s.cell_list + (size_t)h * s.capc;
        const int b = s.cell_start[h], e = min(s.cell_cnt[h], s.capc);
        for (int k = 0; k < e; ++k) {
            s.perm[b + k] = p[k];
            p[k] = b + k;
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
// of nine: the nine cell ranks and counts of a plane are loaded together
// (independent loads in flight), then each cell's members are read four at a
// time (one int4 of the member array, then their positions).  Hits are packed
// into int4 groups in registers and written as whole 16-byte groups, which
// makes the stores of a warp contiguous.
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
            const T L0 = g.L[0], L1 = g.L[1], L2 = g.L[2];
            const T H0 = g.halfL[0], H1 = g.halfL[1], H2 = g.halfL[2];
            const T rl2 = s.rlist2;
            const int cap = s.cap, capc = s.capc;
            const size_t stride = (size_t)s.stride;
            int4* __restrict__ out4 = reinterpret_cast<int4*>(s.nbr) + i;
            const int* __restrict__ crank = s.cell_rank + g.cell_off;
            int xs[3] = {cx == 0 ? nc0 - 1 : cx - 1, cx, cx == nc0 - 1 ? 0 : cx + 1};
            int ys[3] = {cy == 0 ? nc1 - 1 : cy - 1, cy, cy == nc1 - 1 ? 0 : cy + 1};
            int zs[3] = {cz == 0 ? nc2 - 1 : cz - 1, cz, cz == nc2 - 1 ? 0 : cz + 1};
            int cnt = 0;
            int4 grp = make_int4(-1, -1, -1, -1);
#pragma unroll 1
            for (int pz = 0; pz < 3; ++pz) {
                int hh[9], cn[9];
#pragma unroll
                for (int q = 0; q < 9; ++q)
                    hh[q] = __ldg(crank + (zs[pz] * nc1 + ys[q / 3]) * nc0 + xs[q % 3]);
#pragma unroll
                for (int q = 0; q < 9; ++q) cn[q] = min(__ldg(s.cell_cnt + hh[q]), capc);
#pragma unroll
                for (int q = 0; q < 9; ++q) {
                    const int4* __restrict__ row = reinterpret_cast<const int4*>(s.cell_list + (size_t)hh[q] * capc);
                    for (int k4 = 0; k4 < cn[q]; k4 += 4) {
                        const int4 m = __ldg(row + (k4 >> 2));
                        const int mm[4] = {m.x, m.y, m.z, m.w};
                        V4<T> pj[4];
#pragma unroll
                        for (int u = 0; u < 4; ++u) pj[u] = (k4 + u < cn[q]) ? ld4<T>(P + mm[u]) : xi;
#pragma unroll
                        for (int u = 0; u < 4; ++u) {
                            if (k4 + u >= cn[q] || mm[u] == i) continue;
                            const T ddx = min_image(xi.x, pj[u].x, L0, H0);
                            const T ddy = min_image(xi.y, pj[u].y, L1, H1);
                            const T ddz = min_image(xi.z, pj[u].z, L2, H2);
                            const T r2 = ddx * ddx + ddy * ddy + ddz * ddz;
                            if (r2 < rl2) {
                                const int l = cnt & 3;
                                if (l == 0) grp.x = mm[u];
                                else if (l == 1) grp.y = mm[u];
                                else if (l == 2) grp.z = mm[u];
                                else grp.w = mm[u];
                                ++cnt;
                                if ((cnt & 3) == 0) {
                                    if (cnt <= cap) out4[(size_t)((cnt >> 2) - 1) * stride] = grp;
                                    grp = make_int4(-1, -1, -1, -1);
                                }
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

// Rebuild pipeline: linked-cell binning as a counting sort over Hilbert-ranked
// cells, the resort of every particle array into cell order, and the full
// Verlet list with skin.  Paper "Software design", "Parallelization" (CellGrid
// linked cells), "Performance optimizations" (cell decomposition, data
// sorting) and "Example usage" (VerletList(system, cutoff) with system.skin).
//
// Per rebuild, in one stream:
//   bin        cell rank of every particle, atomic arrival index in its cell,
//              and the latch of the per-replica rebuild requests
//   scan x3    exclusive scan of the cell counts -> first slot of each cell
//              (the last phase also clears the counts for the next rebuild)
//   scatter    new slot of every particle of a rebuilding replica
//   cellsort   order inside each cell by previous slot (makes the counting
//              sort stable and the result independent of atomic timing)
//   gather     permuted copies of positions, velocities, forces, images
//   copyback   copies back, records the build positions, maps bond partners
//   verlet     27-cell search, full list (both directions) in column-major
//              (ELL) layout nbr[k * stride + i]
// Replicas whose request flag is clear skip every step after `bin`.
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
__global__ void __launch_bounds__(TILE) k_bin(DevSys<T> s, int cur) {
    if (s.ctrl->abort) return;
    if (blockIdx.x == 0) {
        for (int r = threadIdx.x; r < s.R; r += blockDim.x) {
            s.now[r] = s.req[r];
            s.req[r] = 0;
        }
        if (threadIdx.x == 0) {
            s.ctrl->any_req = 0;
            s.ctrl->n_rebuilds += 1;
            s.ctrl->max_count = 0;
        }
    }
    const V4<T>* __restrict__ P = s.pos[cur];
    for (int t = blockIdx.x; t < s.ntiles; t += gridDim.x) {
        const Tile tl = s.tiles[t];
        if ((int)threadIdx.x >= tl.count) continue;
        const RepGeom<T>& g = s.reps[tl.rep];
        const int i = tl.start + threadIdx.x;
        const V4<T> p = ld4<T>(P + i);
        const int cx = cell_coord(p.x, g.cells_per_len[0], g.nc[0]);
        const int cy = cell_coord(p.y, g.cells_per_len[1], g.nc[1]);
        const int cz = cell_coord(p.z, g.cells_per_len[2], g.nc[2]);
        const int h = s.cell_rank[g.cell_off + (cz * g.nc[1] + cy) * g.nc[0] + cx];
        s.cellh[i] = h;
        s.in_cell[i] = atomicAdd(&s.cell_cnt[h], 1);
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
        if (base + k < s.ncells) {
            s.cell_start[base + k] = run;
            s.cell_cnt[base + k] = 0;
        }
        run += v[k];
    }
}

// ---- permutation -------------------------------------------------------------
template <class T>
__global__ void __launch_bounds__(TILE) k_scatter(DevSys<T> s) {
    if (s.ctrl->abort) return;
    for (int t = blockIdx.x; t < s.ntiles; t += gridDim.x) {
        const Tile tl = s.tiles[t];
        if (!s.now[tl.rep] || (int)threadIdx.x >= tl.count) continue;
        const int i = tl.start + threadIdx.x;
        s.perm[s.cell_start[s.cellh[i]] + s.in_cell[i]] = i;
    }
}

// Sort each cell's old slots ascending: a stable counting sort overall.
template <class T>
__global__ void __launch_bounds__(TILE) k_cellsort(DevSys<T> s) {
    if (s.ctrl->abort) return;
    for (int h = blockIdx.x * blockDim.x + threadIdx.x; h < s.ncells; h += gridDim.x * blockDim.x) {
        if (!s.now[s.cell_rep[h]]) continue;
        const int b = s.cell_start[h], e = s.cell_start[h + 1];
        int* p = s.perm;
        for (int k = b + 1; k < e; ++k) {
            const int key = p[k];
            int q = k - 1;
            while (q >= b && p[q] > key) {
                p[q + 1] = p[q];
                --q;
            }
            p[q + 1] = key;
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
        const V4<T> x = Q[n];
        P[n] = x;
        s.xb[n] = x;
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
            const int cx = cell_coord(xi.x, g.cells_per_len[0], g.nc[0]);
            const int cy = cell_coord(xi.y, g.cells_per_len[1], g.nc[1]);
            const int cz = cell_coord(xi.z, g.cells_per_len[2], g.nc[2]);
            const T L0 = g.L[0], L1 = g.L[1], L2 = g.L[2];
            const T H0 = g.halfL[0], H1 = g.halfL[1], H2 = g.halfL[2];
            const T rl2 = s.rlist2;
            int cnt = 0;
            int* __restrict__ out = s.nbr + i;
            const int stride = s.stride, cap = s.cap;
            for (int dz = -1; dz <= 1; ++dz) {
                int az = cz + dz;
                az += az < 0 ? g.nc[2] : 0;
                az -= az >= g.nc[2] ? g.nc[2] : 0;
                for (int dy = -1; dy <= 1; ++dy) {
                    int ay = cy + dy;
                    ay += ay < 0 ? g.nc[1] : 0;
                    ay -= ay >= g.nc[1] ? g.nc[1] : 0;
                    for (int dx = -1; dx <= 1; ++dx) {
                        int ax = cx + dx;
                        ax += ax < 0 ? g.nc[0] : 0;
                        ax -= ax >= g.nc[0] ? g.nc[0] : 0;
                        const int h = s.cell_rank[g.cell_off + (az * g.nc[1] + ay) * g.nc[0] + ax];
                        const int b = s.cell_start[h], e = s.cell_start[h + 1];
                        for (int j = b; j < e; ++j) {
                            if (j == i) continue;
                            const V4<T> xj = ld4<T>(P + j);
                            const T ddx = min_image(xi.x, xj.x, L0, H0);
                            const T ddy = min_image(xi.y, xj.y, L1, H1);
                            const T ddz = min_image(xi.z, xj.z, L2, H2);
                            const T r2 = ddx * ddx + ddy * ddy + ddz * ddz;
                            if (r2 < rl2) {
                                if (cnt < cap) out[(size_t)cnt * stride] = j;
                                ++cnt;
                            }
                        }
                    }
                }
            }
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
void Launch<T>::rebuild(const DevSys<T>& s, int cur, bool permute_force, cudaStream_t st) {
    const int gt = s.ntiles;
    k_bin<T><<<gt, TILE, 0, st>>>(s, cur);
    k_scan_reduce<T><<<s.nscan_blocks, SCAN_THREADS, 0, st>>>(s);
    k_scan_top<T><<<1, SCAN_THREADS, 0, st>>>(s);
    k_scan_down<T><<<s.nscan_blocks, SCAN_THREADS, 0, st>>>(s);
    k_scatter<T><<<gt, TILE, 0, st>>>(s);
    k_cellsort<T><<<grid_for(s.ncells, TILE), TILE, 0, st>>>(s);
    k_gather<T><<<gt, TILE, 0, st>>>(s, cur, permute_force ? 1 : 0);
    k_copyback<T><<<gt, TILE, 0, st>>>(s, cur, permute_force ? 1 : 0);
    k_verlet<T><<<gt, TILE, 0, st>>>(s, cur);
}

template <class T>
void Launch<T>::verlet_only(const DevSys<T>& s, int cur, cudaStream_t st) {
    k_verlet<T><<<s.ntiles, TILE, 0, st>>>(s, cur);
}

template <class T>
void Launch<T>::request_all(const DevSys<T>& s, cudaStream_t st) {
    k_request_all<T><<<grid_for(s.R, 256), 256, 0, st>>>(s);
}

template struct Launch<float>;
template struct Launch<double>;

int scan_blocks_for(int ncells) { return (ncells + SCAN_TILE - 1) / SCAN_TILE; }

}  // namespace espp

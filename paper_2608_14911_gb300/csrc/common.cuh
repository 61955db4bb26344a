// Shared device-side types of the CUDA library (not used by the oracle).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>

#include "../../include/espp.h"

namespace espp {

// ---------------------------------------------------------------------------
// Precision-generic 4-vectors: float4 (16 B) or a 32-byte aligned double quad.
// The w lane carries an integer (particle type in positions, local particle id
// in velocities) stored bit-for-bit.
// ---------------------------------------------------------------------------
struct __align__(32) dquad {
    double x, y, z, w;
};

template <class T> struct VecOf;
template <> struct VecOf<float> { using type = float4; };
template <> struct VecOf<double> { using type = dquad; };
template <class T> using V4 = typename VecOf<T>::type;

__device__ __host__ __forceinline__ float int_bits_as(float, int v) {
#ifdef __CUDA_ARCH__
    return __int_as_float(v);
#else
    float f; memcpy(&f, &v, 4); return f;
#endif
}
__device__ __host__ __forceinline__ double int_bits_as(double, int v) {
#ifdef __CUDA_ARCH__
    return __longlong_as_double((long long)v);
#else
    long long l = v; double d; memcpy(&d, &l, 8); return d;
#endif
}
__device__ __forceinline__ int bits_as_int(float f) { return __float_as_int(f); }
__device__ __forceinline__ int bits_as_int(double d) { return (int)__double_as_longlong(d); }

template <class T>
__device__ __forceinline__ V4<T> ld4(const V4<T>* p) { return *p; }
template <>
__device__ __forceinline__ float4 ld4<float>(const float4* p) { return __ldg(p); }
template <>
__device__ __forceinline__ dquad ld4<double>(const dquad* p) {
    const double2* q = reinterpret_cast<const double2*>(p);
    double2 a = __ldg(q), b = __ldg(q + 1);
    dquad r; r.x = a.x; r.y = a.y; r.z = b.x; r.w = b.y;
    return r;
}

// plain (coherent) load, for arrays written earlier in the same kernel chain
template <class T>
__device__ __forceinline__ V4<T> ldc(const V4<T>* p) { return *p; }

template <class T> __device__ __forceinline__ V4<T> mk4(T x, T y, T z, T w) {
    V4<T> r; r.x = x; r.y = y; r.z = z; r.w = w; return r;
}

// ---------------------------------------------------------------------------
// Half kick and drift with a fixed rounding sequence (explicit intrinsics, so
// the compiler cannot contract them differently in different kernels): the
// result of a run does not depend on how it is split into integrate calls.
// ---------------------------------------------------------------------------
__device__ __forceinline__ float fma_rn(float a, float b, float c) { return __fmaf_rn(a, b, c); }
__device__ __forceinline__ double fma_rn(double a, double b, double c) { return __fma_rn(a, b, c); }
__device__ __forceinline__ float mul_rn(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ double mul_rn(double a, double b) { return __dmul_rn(a, b); }

// v + (dt/2 * f) / m, with 1/m precomputed
template <class T>
__device__ __forceinline__ T half_kick(T v, T f, T half_dt, T inv_m) {
    return fma_rn(mul_rn(half_dt, f), inv_m, v);
}
// x + dt * v
template <class T>
__device__ __forceinline__ T drift(T x, T v, T dt) {
    return fma_rn(dt, v, x);
}

// ---------------------------------------------------------------------------
// Minimum image of xi - xj for coordinates stored in [0, L).  The periodic
// shift is applied to the larger coordinate first; that subtraction is exact
// (Sterbenz: the coordinate lies in [L/2, L)), so the result carries a single
// rounding, as the plain difference of two nearby coordinates does.
// ---------------------------------------------------------------------------
template <class T>
__device__ __forceinline__ T min_image(T xi, T xj, T L, T halfL) {
    T d = xi - xj;
    if (d > halfL) d = (xi - L) - xj;
    else if (d < -halfL) d = xi - (xj - L);
    return d;
}

// ---------------------------------------------------------------------------
// Verlet-list entries carry the periodic image of the pair.  Bits 0..24 hold
// the neighbour's storage slot, bits 25..30 two bits per dimension: 1 = the
// neighbour lies across the upper face (use x_i - L), 2 = across the lower
// face (use x_j - L), 0 = no shift.  Positions are wrapped into the box only
// when the list is rebuilt, so the image fixed at the build stays valid until
// the next build.  Both shifted subtractions are exact (Sterbenz: the shifted
// coordinate lies in [L/2, 2L]); the difference carries one rounding, like
// the minimum image above.
// ---------------------------------------------------------------------------
constexpr int NBR_INDEX_BITS = 25;
constexpr int NBR_INDEX_MASK = (1 << NBR_INDEX_BITS) - 1;
constexpr int MAX_PARTICLES = 1 << NBR_INDEX_BITS;

__device__ __forceinline__ int nbr_slot(int e) { return e & NBR_INDEX_MASK; }
__device__ __forceinline__ int nbr_code(int e) { return e >> NBR_INDEX_BITS; }

template <class T>
__device__ __forceinline__ T shifted_diff(T xi, T xi_minus_L, T xj, T L, int c) {
    const T a = (c & 1) ? xi_minus_L : xi;
    const T b = (c & 2) ? xj - L : xj;
    return a - b;
}

// Wrap one coordinate into [0, L); returns the image change (-1, 0, +1).  A
// coordinate that rounds to exactly L after adding L (it lay less than half
// an ulp of L below 0) becomes 0 in its own image, so that x + img L stays
// continuous.
template <class T>
__device__ __forceinline__ int wrap_coord(T& x, T L) {
    if (x >= L) {
        x -= L;
        return 1;
    }
    if (x < T(0)) {
        x += L;
        if (x >= L) {
            x = T(0);
            return 0;
        }
        return -1;
    }
    return 0;
}

// The largest value of the type below L: a coordinate wrapped in double that
// rounds up to L in the stored precision is kept in its image there.
__device__ __forceinline__ float below(float L) { return nextafterf(L, 0.0f); }
__device__ __forceinline__ double below(double L) { return nextafter(L, 0.0); }

// ---------------------------------------------------------------------------
// Per-replica geometry, resident in device memory.
// ---------------------------------------------------------------------------
template <class T> struct RepGeom {
    T L[3];
    T halfL[3];
    T cells_per_len[3];  // nc / L
    int nc[3];
    int cell_off;        // first cell (rank space) of this replica
    int p_off;           // first particle slot
    int n;               // particles
    int pad;
    unsigned long long seed;
};

// Tile table: blocks walk tiles; a tile never straddles two replicas.
struct Tile {
    int start;  // first particle slot
    int count;  // particles in the tile (<= TILE)
    int rep;
    int pad;
};

// A tile record read ahead of a test that may end the block (an abort flag,
// a replica flag): the load is issued in program order before that test (a
// volatile read is never moved under the branch), so its round trip overlaps
// the flag's instead of following it.
__device__ __forceinline__ Tile ld_tile_early(const Tile* p) {
    Tile t;
    asm volatile("ld.global.nc.v4.s32 {%0, %1, %2, %3}, [%4];"
                 : "=r"(t.start), "=r"(t.count), "=r"(t.rep), "=r"(t.pad)
                 : "l"(p));
    return t;
}

// Pair potential record for one (type_i, type_j), derived on the host.
template <class T> struct PairRec {
    int kind;   // 0 none, ESPP_LJ, ESPP_LJ_CAPPED (WCA is LJ)
    int pad;
    T rc2;
    T sig2;
    T eps24;    // 24 eps
    T eps4;     // 4 eps
    T shift;    // U(rc) subtracted when shifted, else 0
    T cap2;     // caprad^2 (capped kind)
    T cap;      // caprad
    T capF;     // |F(caprad)|
    T capU;     // U(caprad) - shift
    int tab_off;  // tabulated kind: u at tab[tab_off + k], F at tab[tab_off + tab_n + k]
    int tab_n;
    T inv_dr;     // (tab_n - 1) / rc
};

template <class T> struct BondRec {
    int kind;   // 0 none, ESPP_FENE, ESPP_TAB_BOND
    int pad;
    T K;
    T inv_R02;
    T halfKR02;  // K R0^2 / 2
    int tab_off;
    int tab_n;
    T inv_dr;    // tabulated: (tab_n - 1) / rmax
    T rmax;
};

// Linear interpolation in a table of u(r_k) and F(r_k) (k < n) at r = x / inv_dr.
template <class T>
__device__ __forceinline__ void table_lookup(const T* __restrict__ tb, int n, T inv_dr, T r, T& u, T& F) {
    const T x = r * inv_dr;
    int k = (int)x;
    k = k > n - 2 ? n - 2 : k;
    const T t = x - (T)k;
    const T u0 = tb[k], u1 = tb[k + 1], f0 = tb[n + k], f1 = tb[n + k + 1];
    u = u0 + t * (u1 - u0);
    F = f0 + t * (f1 - f0);
}

// Control block in device memory (one per handle).
struct Ctrl {
    long long step;            // step number of the stored state
    unsigned int err;          // ESPP error bits (see below)
    unsigned int abort;        // non-zero freezes every later step kernel
    unsigned int any_req;      // some replica requested a rebuild
    unsigned int blocks_done;  // last-block counter of the step kernel
    unsigned int need_cap;     // largest neighbour count seen by an overflowing build
    unsigned int n_rebuilds;   // rebuild passes executed (any replica)
    unsigned int max_count;    // largest neighbour count of the last build
    unsigned int pos_ahead;    // 1 while the stored positions are those of step + 1
                               // (inside an integrate call, after the first drift)
    unsigned int le_keep;      // the next rebuild keeps the stored Lees-Edwards build
                               // offsets (a checkpoint load), then clears this
    unsigned int pad;
};

enum : unsigned int {
    ERRBIT_OVERFLOW = 1u,
    ERRBIT_BOND = 2u,
    ERRBIT_NONFINITE = 4u,
    ERRBIT_TIMEOUT = 8u,
    ERRBIT_ASYM = 16u,  // a list entry without its mirrored entry
};

// Streaming multiprocessors of the current device, for grids sized in whole
// waves (cached per device; 1 if the query fails, which only shrinks grids
// that stride over their work).
inline int sm_count() {
    static int cache[64] = {0};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return 1;
    if (cache[dev] <= 0) {
        int n = 0;
        if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n <= 0) return 1;
        cache[dev] = n;
    }
    return cache[dev];
}

constexpr int TILE = 128;          // particles per tile (= threads per block)
constexpr int MAX_TYPES = ESPP_MAX_TYPES;

}  // namespace espp

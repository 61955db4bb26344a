// Pair terms shared by the step kernel (pairs from the Verlet list) and the
// cell-pair force kernel (pairs from the cell stencil): the conservative pair
// force of every potential kind, and the DPD thermostat's pair term.
#pragma once
#include "kernels.cuh"
#include "philox.cuh"

namespace espp {

// 1/x: the hardware approximation in FP32 (error of order one ulp, far inside
// the 1e-5 force tolerance), the correctly rounded division in FP64.
__device__ __forceinline__ float recip(float x) {
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}
__device__ __forceinline__ double recip(double x) { return 1.0 / x; }

template <class T>
__device__ __forceinline__ void pair_force(const PairRec<T>& pr, const T* __restrict__ tab, T r2, T& fr, T& u) {
    // caller guarantees r2 < pr.rc2 and kind != 0
    if (pr.kind == ESPP_TAB_PAIR) {
        const T r = sqrt(r2);
        T F;
        table_lookup(tab + pr.tab_off, pr.tab_n, pr.inv_dr, r, u, F);
        fr = F / r;
        return;
    }
    if (pr.kind == ESPP_LJ_CAPPED && r2 < pr.cap2) {
        const T r = sqrt(r2);
        fr = pr.capF / r;
        u = pr.capU + pr.capF * (pr.cap - r);
        return;
    }
    const T inv_r2 = recip(r2);
    const T s2 = pr.sig2 * inv_r2;
    const T s6 = s2 * s2 * s2;
    fr = pr.eps24 * s6 * (T(2) * s6 - T(1)) * inv_r2;
    u = pr.eps4 * s6 * (s6 - T(1)) - pr.shift;
}

// One pair term: force (and energy, virial) of neighbour j at displacement d.
template <class T, bool ENERGY, bool MULTI, bool FAST>
__device__ __forceinline__ void pair_term(const DevSys<T>& s, int ti, const PairRec<T>* pr1, T dx, T dy,
                                          T dz, int tj, T& fx, T& fy, T& fz, T& pe, T& vir, T& vxz) {
    const T r2 = dx * dx + dy * dy + dz * dz;
    if (FAST) {
        // one type, plain Lennard-Jones: only rc^2, sigma^2, 24 eps live
        if (r2 < pr1->rc2) {
            const T inv_r2 = recip(r2);
            const T s2 = pr1->sig2 * inv_r2;
            const T s6 = s2 * s2 * s2;
            const T fr = pr1->eps24 * s6 * (T(2) * s6 - T(1)) * inv_r2;
            fx += fr * dx;
            fy += fr * dy;
            fz += fr * dz;
            if (ENERGY) {
                pe += pr1->eps4 * s6 * (s6 - T(1)) - pr1->shift;
                vir += fr * r2;
                vxz += fr * dx * dz;
            }
        }
        return;
    }
    const PairRec<T>& pr = MULTI ? s.pair[ti * s.ntypes + tj] : *pr1;
    if ((!MULTI || pr.kind != 0) && r2 < pr.rc2) {
        T fr, u;
        pair_force(pr, s.tab, r2, fr, u);
        fx += fr * dx;
        fy += fr * dy;
        fz += fr * dz;
        if (ENERGY) {
            pe += u;
            vir += fr * r2;
            vxz += fr * dx * dz;
        }
    }
}

// Lees-Edwards quantities of the current step, uniform over a tile: delta
// reduced into [0, Lx), 1 / Lx, the x velocity le_shear Lz of the image
// above, and le_shear (streaming profile le_shear (z - Lz / 2)).
template <class T>
struct LeCtx {
    T d;
    T inv_Lx;
    T vs;
    T shear;
};

// What the DPD pair term of particle i needs besides the displacement: its
// half-step velocity and id, the replica's seed and the step.
template <class T>
struct DpdCtx {
    V4<T> vi;
    unsigned long long seed;
    long long step;
    T le_vs;  // Lees-Edwards: x velocity of the image above (0 without shear)
};

// DPD pair term (paper "Functionality": dissipative particle dynamics) of a
// neighbour at displacement d (r2 = |d|^2 inside the DPD cutoff) whose
// velocity snapshot is vj: dissipative -gamma w^2 (e . v_ij) and random
// amp w theta_ij along e, w = 1 - r / rc.  e . v_ij and theta_ij are symmetric
// in the pair, so both sides add exactly opposite forces.  nz: the partner is
// the image above (+1) or below (-1) a sheared face (Lees-Edwards), whose
// velocity is vj + nz le_shear Lz along x.  dpd_value is the magnitude
// divided by r (the force on i is dpd_value * d).
template <class T>
__device__ __forceinline__ T dpd_value(const IntParams<T>* __restrict__ ip, const DpdCtx<T>& c, T dx, T dy, T dz,
                                       T r2, const V4<T>& vj, int nz = 0) {
    const T r = sqrt(r2), inv_r = T(1) / r;
    const T w = T(1) - r * ip->dpd_inv_rc;
    const T vjx = nz == 0 ? vj.x : vj.x + (T)nz * c.le_vs;
    const T ev = (dx * (c.vi.x - vjx) + dy * (c.vi.y - vj.y) + dz * (c.vi.z - vj.z)) * inv_r;
    const T th = dpd_theta<T>(c.seed, bits_as_int(c.vi.w), bits_as_int(vj.w), c.step);
    return (-ip->gamma * w * w * ev + ip->dpd_amp * w * th) * inv_r;
}

template <class T>
__device__ __forceinline__ void dpd_term(const IntParams<T>* __restrict__ ip, const DpdCtx<T>& c, T dx, T dy,
                                         T dz, T r2, const V4<T>& vj, T& fx, T& fy, T& fz, int nz = 0) {
    const T val = dpd_value<T>(ip, c, dx, dy, dz, r2, vj, nz);
    fx += val * dx;
    fy += val * dy;
    fz += val * dz;
}

}  // namespace espp

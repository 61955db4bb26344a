// State input/output in particle-id order, deterministic FP64 reductions of the
// observables (paper "Example usage": computeEnergy()), radius of gyration and
// pair-distance histograms.
#include "kernels.cuh"
#include "philox.cuh"

namespace espp {

// Load id-ordered doubles into storage order = id order (the order is reset on
// every set_state; the next rebuild resorts).  Coordinates are wrapped into
// [0, L) in double before rounding to T; a value that rounds up to L becomes 0
// of the next image.
template <class T>
__global__ void __launch_bounds__(TILE) k_set_state(DevSys<T> s, const double* __restrict__ x,
                                                    const double* __restrict__ v,
                                                    const int* __restrict__ img,
                                                    const int* __restrict__ types, int cur) {
    for (int t = blockIdx.x; t < s.ntiles; t += gridDim.x) {
        const Tile tl = s.tiles[t];
        if ((int)threadIdx.x >= tl.count) continue;
        const RepGeom<T>& g = s.reps[tl.rep];
        const int i = tl.start + threadIdx.x;  // slot == global id
        T p[3];
        int im[3];
        bool bad = false;
        for (int d = 0; d < 3; ++d) {
            const double L = (double)g.L[d];
            double xd = x[3 * (size_t)i + d];
            // a non-finite coordinate is reported (the call fails) and kept out
            // of the arithmetic below
            if (!isfinite(xd)) {
                bad = true;
                xd = 0.0;
            }
            const double fl = floor(xd / L);
            double w = xd - fl * L;
            int k = (int)fl + (img ? img[3 * (size_t)i + d] : 0);
            if (w < 0.0) { w += L; k -= 1; }
            if (w >= L) { w -= L; k += 1; }
            T wt = (T)w;
            if (wt >= g.L[d]) { wt = T(0); k += 1; }
            p[d] = wt;
            im[d] = k;
        }
        const int local = i - g.p_off;
        s.pos[cur][i] = mk4<T>(p[0], p[1], p[2], int_bits_as(T(0), types ? types[i] : 0));
        s.xb[i] = s.pos[cur][i];
        T vx = v ? (T)v[3 * (size_t)i] : T(0);
        T vy = v ? (T)v[3 * (size_t)i + 1] : T(0);
        T vz = v ? (T)v[3 * (size_t)i + 2] : T(0);
        if (!(isfinite(vx) && isfinite(vy) && isfinite(vz))) {
            bad = true;
            vx = vy = vz = T(0);
        }
        if (bad) atomicOr(&s.ctrl->err, ERRBIT_NONFINITE);
        s.vel[i] = mk4<T>(vx, vy, vz, int_bits_as(T(0), local));
        s.frc[i] = mk4<T>(T(0), T(0), T(0), T(0));
        s.img[i] = make_int4(im[0], im[1], im[2], 0);
        s.slot_of_id[i] = i;
        s.bond_slot[i] = s.bond_gid[i];
    }
}

template <class T>
__global__ void __launch_bounds__(TILE) k_get_state(DevSys<T> s, double* __restrict__ x,
                                                    double* __restrict__ v, int* __restrict__ img,
                                                    double* __restrict__ f, int cur) {
    for (int t = blockIdx.x; t < s.ntiles; t += gridDim.x) {
        const Tile tl = s.tiles[t];
        if ((int)threadIdx.x >= tl.count) continue;
        const RepGeom<T>& g = s.reps[tl.rep];
        const int i = tl.start + threadIdx.x;
        const V4<T> vv = s.vel[i];
        const size_t gid = (size_t)g.p_off + bits_as_int(vv.w);
        // stored positions may lie just outside the box (they are wrapped at
        // list builds only): report them wrapped, with the image counters to match
        const V4<T> p = s.pos[cur][i];
        const double pc[3] = {(double)p.x, (double)p.y, (double)p.z};
        double wc[3];
        int sh[3];
        double vx = (double)vv.x;
        if (s.le_on) {
            // Lees-Edwards: a crossing of a sheared face also moves x and v_x
            const double L[3] = {(double)g.L[0], (double)g.L[1], (double)g.L[2]};
            wc[0] = pc[0];
            wc[1] = pc[1];
            wc[2] = pc[2];
            le_wrap(wc, vx, sh, L, le_offset(s, g, s.ctrl->step + (long long)s.ctrl->pos_ahead), s.le_shear);
        } else {
            for (int d = 0; d < 3; ++d) {
                const double L = (double)g.L[d];
                double w = pc[d];
                int k = 0;
                if (w >= L) { w -= L; k = 1; }
                else if (w < 0.0) {
                    w += L;
                    k = -1;
                    if (w >= L) { w = 0.0; k = 0; }  // less than half an ulp below 0: its own image
                }
                wc[d] = w;
                sh[d] = k;
            }
        }
        if (x) {
            x[3 * gid] = wc[0];
            x[3 * gid + 1] = wc[1];
            x[3 * gid + 2] = wc[2];
        }
        if (v) {
            v[3 * gid] = vx;
            v[3 * gid + 1] = vv.y;
            v[3 * gid + 2] = vv.z;
        }
        if (img) {
            const int4 im = s.img[i];
            img[3 * gid] = im.x + sh[0];
            img[3 * gid + 1] = im.y + sh[1];
            img[3 * gid + 2] = im.z + sh[2];
        }
        if (f) {
            const V4<T> fi = s.frc[i];
            f[3 * gid] = fi.x;
            f[3 * gid + 1] = fi.y;
            f[3 * gid + 2] = fi.z;
        }
    }
}

// The stored total force of the current step (id-ordered doubles) back into
// its slots.
template <class T>
__global__ void __launch_bounds__(TILE) k_set_force(DevSys<T> s, const double* __restrict__ f) {
    for (int t = blockIdx.x; t < s.ntiles; t += gridDim.x) {
        const Tile tl = s.tiles[t];
        if ((int)threadIdx.x >= tl.count) continue;
        const int gid = tl.start + threadIdx.x;
        const int i = s.slot_of_id[gid];
        s.frc[i] = mk4<T>((T)f[3 * (size_t)gid], (T)f[3 * (size_t)gid + 1], (T)f[3 * (size_t)gid + 2], T(0));
    }
}

// One block per replica sums its tiles' partials in a fixed order.
template <class T>
__global__ void __launch_bounds__(256) k_reduce_obs(DevSys<T> s, double* __restrict__ out) {
    const int r = blockIdx.x;
    const int t0 = s.rep_tile_off[r], t1 = s.rep_tile_off[r + 1];
    __shared__ double sh[256];
    for (int k = 0; k < NPART; ++k) {
        double a = 0.0;
        for (int t = t0 + threadIdx.x; t < t1; t += blockDim.x) a += s.partials[(size_t)t * NPART + k];
        sh[threadIdx.x] = a;
        __syncthreads();
        for (int w = blockDim.x / 2; w > 0; w >>= 1) {
            if ((int)threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
            __syncthreads();
        }
        if (threadIdx.x == 0) out[(size_t)r * NPART + k] = sh[0];
        __syncthreads();
    }
}

// One warp per molecule: centre of the unwrapped positions, then the mean
// squared distance from it, both summed in a fixed lane order.
template <class T>
__global__ void k_rg2(DevSys<T> s, int cur, const int* __restrict__ members,
                      const int* __restrict__ off, const int* __restrict__ mrep, int nmol,
                      double* __restrict__ rg2) {
    const int lane = threadIdx.x & 31;
    const int m = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (m >= nmol) return;
    const RepGeom<T>& g = s.reps[mrep[m]];
    const int b = off[m], e = off[m + 1];
    // Lees-Edwards: the unwrapped x adds img_z delta(t) (delta not reduced)
    const double dle = s.le_on ? le_offset(s, g, s.ctrl->step + (long long)s.ctrl->pos_ahead) : 0.0;
    double c[3] = {0.0, 0.0, 0.0};
    for (int k = b + lane; k < e; k += 32) {
        const int slot = s.slot_of_id[members[k]];
        const V4<T> p = s.pos[cur][slot];
        const int4 im = s.img[slot];
        c[0] += (double)p.x + (double)im.x * (double)g.L[0] + (double)im.z * dle;
        c[1] += (double)p.y + (double)im.y * (double)g.L[1];
        c[2] += (double)p.z + (double)im.z * (double)g.L[2];
    }
    for (int d = 0; d < 3; ++d) {
        for (int o = 16; o > 0; o >>= 1) c[d] += __shfl_xor_sync(0xffffffffu, c[d], o);
        c[d] /= (double)(e - b);
    }
    double a = 0.0;
    for (int k = b + lane; k < e; k += 32) {
        const int slot = s.slot_of_id[members[k]];
        const V4<T> p = s.pos[cur][slot];
        const int4 im = s.img[slot];
        const double ux = (double)p.x + (double)im.x * (double)g.L[0] + (double)im.z * dle - c[0];
        const double uy = (double)p.y + (double)im.y * (double)g.L[1] - c[1];
        const double uz = (double)p.z + (double)im.z * (double)g.L[2] - c[2];
        a += ux * ux + uy * uy + uz * uz;
    }
    for (int o = 16; o > 0; o >>= 1) a += __shfl_xor_sync(0xffffffffu, a, o);
    if (lane == 0) rg2[m] = a / (double)(e - b);
}

// Unique pairs (slot i < slot j) of one replica with r < rmax; integer bin
// counts (exact under atomics).
template <class T>
__global__ void __launch_bounds__(256) k_rdf(DevSys<T> s, int cur, int rep, T rmax2, double inv_dr,
                                             int nbins, unsigned long long* __restrict__ counts) {
    extern __shared__ unsigned int hist[];
    for (int b = threadIdx.x; b < nbins; b += blockDim.x) hist[b] = 0;
    __syncthreads();
    const RepGeom<T>& g = s.reps[rep];
    const V4<T>* __restrict__ P = s.pos[cur];
    const int n = g.n;
    const T dle = s.le_on ? (T)le_reduce(le_offset(s, g, s.ctrl->step + (long long)s.ctrl->pos_ahead),
                                         (double)g.L[0])
                          : T(0);
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
      for (int j = i + 1; j < n; ++j) {
        const V4<T> a = P[g.p_off + i], c = P[g.p_off + j];
        const T dz = min_image(a.z, c.z, g.L[2], g.halfL[2]);
        const T dy = min_image(a.y, c.y, g.L[1], g.halfL[1]);
        const T zr = a.z - c.z;
        const T dx = (s.le_on && (zr > g.halfL[2] || zr < -g.halfL[2]))
                         ? le_dx(a.x, c.x, zr > g.halfL[2] ? 1 : -1, dle, g.L[0], T(1) / g.L[0])
                         : min_image(a.x, c.x, g.L[0], g.halfL[0]);
        const T r2 = dx * dx + dy * dy + dz * dz;
        if (r2 < rmax2) {
            int b = (int)(sqrt((double)r2) * inv_dr);
            if (b >= nbins) b = nbins - 1;
            atomicAdd(&hist[b], 1u);
        }
      }
    __syncthreads();
    for (int b = threadIdx.x; b < nbins; b += blockDim.x)
        if (hist[b]) atomicAdd(&counts[b], (unsigned long long)hist[b]);
}

// Unique pairs within rmax from the Verlet list (rmax <= list cutoff): each
// pair appears in both lists, counted from the lower storage slot.
template <class T>
__global__ void __launch_bounds__(256) k_rdf_list(DevSys<T> s, int cur, int rep, T rmax2, double inv_dr, int nbins,
                                                  unsigned long long* __restrict__ counts) {
    extern __shared__ unsigned int hist[];
    for (int b = threadIdx.x; b < nbins; b += blockDim.x) hist[b] = 0;
    __syncthreads();
    const RepGeom<T>& g = s.reps[rep];
    const V4<T>* __restrict__ P = s.pos[cur];
    const size_t stride = (size_t)s.stride;
    const T dle = s.le_on ? (T)le_reduce(le_offset(s, g, s.ctrl->step + (long long)s.ctrl->pos_ahead),
                                         (double)g.L[0])
                          : T(0);
    for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < g.n; q += gridDim.x * blockDim.x) {
        const int i = g.p_off + q;
        const V4<T> xi = P[i];
        const int n = s.nbr_cnt[i];
        for (int k = 0; k < n; ++k) {
            const int e = s.nbr[4 * ((size_t)(k >> 2) * stride + i) + (k & 3)];
            const int j = nbr_slot(e);
            if (j < i) continue;
            const V4<T> xj = P[j];
            const int code = nbr_code(e);
            const T dx = (code & 3) == 3 ? le_dx(xi.x, xj.x, (code >> 4) == 1 ? 1 : -1, dle, g.L[0], T(1) / g.L[0])
                                         : shifted_diff(xi.x, xi.x - g.L[0], xj.x, g.L[0], code & 3);
            const T dy = shifted_diff(xi.y, xi.y - g.L[1], xj.y, g.L[1], (code >> 2) & 3);
            const T dz = shifted_diff(xi.z, xi.z - g.L[2], xj.z, g.L[2], code >> 4);
            const T r2 = dx * dx + dy * dy + dz * dz;
            if (r2 < rmax2) {
                int b = (int)(sqrt((double)r2) * inv_dr);
                if (b >= nbins) b = nbins - 1;
                atomicAdd(&hist[b], 1u);
            }
        }
    }
    __syncthreads();
    for (int b = threadIdx.x; b < nbins; b += blockDim.x)
        if (hist[b]) atomicAdd(&counts[b], (unsigned long long)hist[b]);
}

// Coarse-graining map (4:1 style): site k is the centre of mass of beads
// [bps k, bps k + bps) of the id-ordered unwrapped positions, wrapped into the
// box; its force is the sum of the beads' forces.
__global__ void k_cg_map(const double* __restrict__ x, const int* __restrict__ img, const double* __restrict__ f,
                         long long nsites, int bps, double L0, double L1, double L2, double* __restrict__ xs,
                         double* __restrict__ fs) {
    const long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= nsites) return;
    const double L[3] = {L0, L1, L2};
    for (int d = 0; d < 3; ++d) {
        double c = 0.0, fsum = 0.0;
        for (int b = 0; b < bps; ++b) {
            const long long i = k * bps + b;
            c += x[3 * i + d] + (double)img[3 * i + d] * L[d];
            fsum += f[3 * i + d];
        }
        c /= bps;
        c -= L[d] * floor(c / L[d]);
        if (c >= L[d]) c -= L[d];
        xs[3 * k + d] = c;
        fs[3 * k + d] = fsum;
    }
}

void launch_cg_map(const double* x, const int* img, const double* f, long long nsites, int bps, const double* L,
                   double* xs, double* fs, cudaStream_t st) {
    if (nsites <= 0) return;
    k_cg_map<<<(unsigned int)((nsites + 255) / 256), 256, 0, st>>>(x, img, f, nsites, bps, L[0], L[1], L[2], xs, fs);
}

__global__ void k_noise(unsigned long long seed, long long step, long long n, double* out) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    double rx, ry, rz;
    langevin_noise<double>(seed, (int)i, step, rx, ry, rz);
    out[3 * i] = rx;
    out[3 * i + 1] = ry;
    out[3 * i + 2] = rz;
}

template <class T>
void Launch<T>::set_state(const DevSys<T>& s, const double* x, const double* v, const int* img,
                          const int* types_by_gid, int cur, cudaStream_t st) {
    k_set_state<T><<<s.ntiles, TILE, 0, st>>>(s, x, v, img, types_by_gid, cur);
}

template <class T>
void Launch<T>::get_state(const DevSys<T>& s, double* x, double* v, int* img, double* f, int cur,
                          cudaStream_t st) {
    k_get_state<T><<<s.ntiles, TILE, 0, st>>>(s, x, v, img, f, cur);
}

template <class T>
void Launch<T>::set_force(const DevSys<T>& s, const double* f, cudaStream_t st) {
    k_set_force<T><<<s.ntiles, TILE, 0, st>>>(s, f);
}

template <class T>
void Launch<T>::reduce_obs(const DevSys<T>& s, double* out, cudaStream_t st) {
    k_reduce_obs<T><<<s.R, 256, 0, st>>>(s, out);
}

template <class T>
void Launch<T>::rg2(const DevSys<T>& s, int cur, const int* members, const int* off,
                    const int* mrep, int nmol, double* out, cudaStream_t st) {
    if (nmol <= 0) return;
    const int warps_per_block = 4;
    k_rg2<T><<<(nmol + warps_per_block - 1) / warps_per_block, 32 * warps_per_block, 0, st>>>(
        s, cur, members, off, mrep, nmol, out);
}

template <class T>
void Launch<T>::rdf(const DevSys<T>& s, int cur, int rep, double rmax, int nbins,
                    unsigned long long* counts, cudaStream_t st) {
    k_rdf<T><<<4 * sm_count(), 256, sizeof(unsigned int) * nbins, st>>>(s, cur, rep, (T)(rmax * rmax),
                                                                 nbins / rmax, nbins, counts);
}

template <class T>
void Launch<T>::rdf_list(const DevSys<T>& s, int cur, int rep, double rmax, int nbins,
                         unsigned long long* counts, cudaStream_t st) {
    k_rdf_list<T><<<8 * sm_count(), 256, sizeof(unsigned int) * nbins, st>>>(s, cur, rep, (T)(rmax * rmax),
                                                                      nbins / rmax, nbins, counts);
}
template void Launch<float>::rdf_list(const DevSys<float>&, int, int, double, int, unsigned long long*, cudaStream_t);
template void Launch<double>::rdf_list(const DevSys<double>&, int, int, double, int, unsigned long long*, cudaStream_t);

void launch_noise(unsigned long long seed, long long step, long long n, double* out,
                  cudaStream_t st) {
    if (n <= 0) return;
    k_noise<<<(unsigned int)((n + 255) / 256), 256, 0, st>>>(seed, step, n, out);
}

template void Launch<float>::set_state(const DevSys<float>&, const double*, const double*, const int*, const int*, int, cudaStream_t);
template void Launch<double>::set_state(const DevSys<double>&, const double*, const double*, const int*, const int*, int, cudaStream_t);
template void Launch<float>::get_state(const DevSys<float>&, double*, double*, int*, double*, int, cudaStream_t);
template void Launch<double>::get_state(const DevSys<double>&, double*, double*, int*, double*, int, cudaStream_t);
template void Launch<float>::set_force(const DevSys<float>&, const double*, cudaStream_t);
template void Launch<double>::set_force(const DevSys<double>&, const double*, cudaStream_t);
template void Launch<float>::reduce_obs(const DevSys<float>&, double*, cudaStream_t);
template void Launch<double>::reduce_obs(const DevSys<double>&, double*, cudaStream_t);
template void Launch<float>::rg2(const DevSys<float>&, int, const int*, const int*, const int*, int, double*, cudaStream_t);
template void Launch<double>::rg2(const DevSys<double>&, int, const int*, const int*, const int*, int, double*, cudaStream_t);
template void Launch<float>::rdf(const DevSys<float>&, int, int, double, int, unsigned long long*, cudaStream_t);
template void Launch<double>::rdf(const DevSys<double>&, int, int, double, int, unsigned long long*, cudaStream_t);

}  // namespace espp

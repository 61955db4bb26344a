/*
 * Oracle implementation: see orc.h.  TEST INFRASTRUCTURE ONLY -- the product
 * path never loads or calls this code.
 *
 * Every function states the definition it writes out.  The paper (ESPResSo++)
 * names the ingredients but prints no formulas; the formulas here are the
 * textbook ones for the Kremer-Grest model, and the readings chosen where the
 * paper is silent are marked "Reading".
 */
#include "orc.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

int orc_num_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* ------------------------------------------------------------------------ */
/* Philox4x32-10, as defined in Salmon, Moraes, Dror and Shaw, "Parallel     */
/* random numbers: as easy as 1, 2, 3", SC'11: ten rounds of two 32x32->64   */
/* multiplies (multipliers 0xD2511F53, 0xCD9E8D57) with the counter words    */
/* permuted and xor-ed with the key, the key bumped by the Weyl constants    */
/* 0x9E3779B9, 0xBB67AE85 between rounds.                                    */
/* ------------------------------------------------------------------------ */
void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]) {
    uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int round = 0; round < 10; ++round) {
        if (round > 0) {
            k0 += 0x9E3779B9u;
            k1 += 0xBB67AE85u;
        }
        uint64_t p0 = (uint64_t)0xD2511F53u * (uint64_t)c0;
        uint64_t p1 = (uint64_t)0xCD9E8D57u * (uint64_t)c2;
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        uint32_t n0 = hi1 ^ c1 ^ k0;
        uint32_t n1 = lo1;
        uint32_t n2 = hi0 ^ c3 ^ k1;
        uint32_t n3 = lo0;
        c0 = n0; c1 = n1; c2 = n2; c3 = n3;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* Reading (noise distribution; the paper names only gamma and T for the
 * Langevin thermostat): the top 24 bits k of a word give the odd integer
 * 2k+1-2^24, scaled by 2^-25.  The result lies in (-1/2, 1/2), has mean 0 and
 * variance (1-2^-48)/12, and is exact in binary32 and binary64. */
double orc_uniform_centered(uint32_t w) {
    int32_t k = (int32_t)(w >> 8);
    int32_t odd = 2 * k + 1 - 16777216;
    return ldexp((double)odd, -25);
}

void orc_uniform_fill(const uint32_t* w, int64_t n, double* out) {
    for (int64_t i = 0; i < n; ++i) out[i] = orc_uniform_centered(w[i]);
}

/* Reading: key = (seed low word, seed high word); counter = (particle id,
 * step low word, step high word, stream tag 0 = Langevin).  Words 0..2 give
 * the x, y, z noise of that particle at that step. */
static void langevin_r(uint64_t seed, int64_t id, int64_t step, double r[3]) {
    uint32_t key[2] = {(uint32_t)(seed & 0xffffffffu), (uint32_t)(seed >> 32)};
    uint64_t s = (uint64_t)step;
    uint32_t ctr[4] = {(uint32_t)id, (uint32_t)(s & 0xffffffffu), (uint32_t)(s >> 32), 0u};
    uint32_t out[4];
    orc_philox4x32_10(ctr, key, out);
    r[0] = orc_uniform_centered(out[0]);
    r[1] = orc_uniform_centered(out[1]);
    r[2] = orc_uniform_centered(out[2]);
}

void orc_langevin_noise(uint64_t seed, int64_t step, int64_t n, double* out) {
    for (int64_t i = 0; i < n; ++i) langevin_r(seed, i, step, out + 3 * i);
}

/* ------------------------------------------------------------------------ */
/* Periodic box                                                              */
/* ------------------------------------------------------------------------ */

/* Minimum-image convention: the periodic copy of d nearest to zero. */
static double min_image(double d, double L) { return d - L * nearbyint(d / L); }

/* Lees-Edwards boundary conditions (paper "State of the field" and "New
 * features": Lees-Edwards; Lees & Edwards 1972).  Reading: steady shear with
 * the flow along x and the gradient along z at shear rate gdot; the periodic
 * image of the box at z + k Lz is displaced by k delta along x and moves with
 * velocity k gdot Lz along x, delta(t) = gdot Lz t (t = simulated time).
 * The state below is set by the callers (orc_set_lees_edwards). */
static int orc_le_on = 0;
static double orc_le_shear = 0.0, orc_le_time = 0.0;

void orc_set_lees_edwards(int on, double shear, double time) {
    orc_le_on = on ? 1 : 0;
    orc_le_shear = shear;
    orc_le_time = time;
}
double orc_le_get_time(void) { return orc_le_time; }

static double le_delta(const double* L) { return orc_le_on ? orc_le_shear * L[2] * orc_le_time : 0.0; }

/* Minimum image of x_i - x_j; *nz receives the z image index k of the copy
 * of j used (x_j + k (delta, 0, Lz)).  Under Lees-Edwards the z image is
 * chosen first, then x and y as in a plain periodic box. */
static void min_image_le(const double* xi, const double* xj, const double* L, double d[3], int* nz) {
    const double dz = xi[2] - xj[2];
    const double k = nearbyint(dz / L[2]);
    d[2] = dz - L[2] * k;
    double dx = xi[0] - xj[0];
    if (orc_le_on) dx -= k * le_delta(L);
    d[0] = min_image(dx, L[0]);
    d[1] = min_image(xi[1] - xj[1], L[1]);
    if (nz) *nz = (int)k;
}

static void min_image_vec(const double* xi, const double* xj, const double* L, double d[3]) {
    min_image_le(xi, xj, L, d, NULL);
}

/* Streaming velocity of the imposed shear at height z (Lees-Edwards):
 * gdot (z - Lz/2) along x, so that the images at z +- Lz move at +- gdot Lz. */
static double le_stream(double z, const double* L) { return orc_le_on ? orc_le_shear * (z - 0.5 * L[2]) : 0.0; }

/* ------------------------------------------------------------------------ */
/* Potentials                                                                */
/* ------------------------------------------------------------------------ */

/* 12-6 Lennard-Jones energy and -dU/dr / r at distance r (r2 = r*r). */
static void lj_raw(double eps, double sig, double r2, double* u, double* fr) {
    double s2 = sig * sig / r2;
    double s6 = s2 * s2 * s2;
    *u = 4.0 * eps * (s6 * s6 - s6);
    *fr = 24.0 * eps * (2.0 * s6 * s6 - s6) / r2;
}

/* Tabulated potentials (paper "Functionality": tabulated potentials).  A
 * table holds u(r_k) and F(r_k) = -dU/dr at r_k = k * rmax / (n - 1),
 * k = 0..n-1.  Reading: both are interpolated linearly in r between nodes. */
#define ORC_MAX_TABLES 16
static struct {
    int n;
    double rmax;
    double* u;
    double* f;
} orc_tables[ORC_MAX_TABLES];

int orc_set_table(int slot, double rmax, int n, const double* u, const double* f) {
    if (slot < 0 || slot >= ORC_MAX_TABLES || n < 2 || !(rmax > 0)) return -1;
    free(orc_tables[slot].u);
    free(orc_tables[slot].f);
    orc_tables[slot].n = n;
    orc_tables[slot].rmax = rmax;
    orc_tables[slot].u = (double*)malloc(sizeof(double) * (size_t)n);
    orc_tables[slot].f = (double*)malloc(sizeof(double) * (size_t)n);
    memcpy(orc_tables[slot].u, u, sizeof(double) * (size_t)n);
    memcpy(orc_tables[slot].f, f, sizeof(double) * (size_t)n);
    return 0;
}

/* Table `slot` at distance r (0 <= r < rmax): energy u and force F along r. */
static void table_eval(int slot, double r, double* u, double* F) {
    int n = orc_tables[slot].n;
    double dr = orc_tables[slot].rmax / (n - 1);
    double x = r / dr;
    int k = (int)floor(x);
    if (k > n - 2) k = n - 2;
    if (k < 0) k = 0;
    double t = x - k;
    const double* uu = orc_tables[slot].u;
    const double* ff = orc_tables[slot].f;
    *u = uu[k] + t * (uu[k + 1] - uu[k]);
    *F = ff[k] + t * (ff[k + 1] - ff[k]);
}

/* ------------------------------------------------------------------------ */
/* Learned radial-basis MLP pair potential (the learned CG model).            */
/* Reading (the paper prints no model; the shape is 32 Gaussian bases on     */
/* [0, rc], two hidden layers of 64 SiLU units, one output):                 */
/*   phi_k(r) = exp(-(r - mu_k)^2 / (2 w^2)) * fc(r),  mu_k = rc k / 31,    */
/*   w = rc / 31,  fc(r) = (cos(pi r / rc) + 1) / 2 (smooth cutoff);        */
/*   h1 = silu(W1 phi + b1), h2 = silu(W2 h1 + b2), u = w3 . h2 + b3.        */
/* The weights are given in double (the BF16 values upcast).  du/dr is the   */
/* exact derivative, propagated forward through the same layers.             */
/* ------------------------------------------------------------------------ */
#define ORC_MLP_NB 32
#define ORC_MLP_H 64
#define ORC_MLP_NPAR (ORC_MLP_H * ORC_MLP_NB + ORC_MLP_H + ORC_MLP_H * ORC_MLP_H + ORC_MLP_H + ORC_MLP_H + 1)
static double orc_mlp_par[ORC_MLP_NPAR];
static double orc_mlp_rc = 0.0;

int orc_set_mlp(const double* par, int64_t npar, double rc) {
    if (npar != ORC_MLP_NPAR || !(rc > 0)) return -1;
    memcpy(orc_mlp_par, par, sizeof(double) * ORC_MLP_NPAR);
    orc_mlp_rc = rc;
    return 0;
}

static double sigmoid(double z) { return 1.0 / (1.0 + exp(-z)); }

/* Energy of one pair at distance r and its derivative du/dr (r < rc).  If
 * grad is not NULL it receives d(du/dr)/d(parameters) (ORC_MLP_NPAR values,
 * same layout as the parameters), and if ugrad is not NULL it receives
 * du/d(parameters). */
void orc_mlp_pair(double r, double* u_out, double* dudr_out, double* grad, double* ugrad) {
    const double rc = orc_mlp_rc;
    const double* W1 = orc_mlp_par;
    const double* b1 = W1 + ORC_MLP_H * ORC_MLP_NB;
    const double* W2 = b1 + ORC_MLP_H;
    const double* b2 = W2 + ORC_MLP_H * ORC_MLP_H;
    const double* w3 = b2 + ORC_MLP_H;
    const double b3 = w3[ORC_MLP_H];
    double phi[ORC_MLP_NB], dphi[ORC_MLP_NB];
    const double w = rc / (ORC_MLP_NB - 1);
    const double fc = 0.5 * (cos(M_PI * r / rc) + 1.0);
    const double dfc = -0.5 * (M_PI / rc) * sin(M_PI * r / rc);
    for (int k = 0; k < ORC_MLP_NB; ++k) {
        const double mu = rc * k / (ORC_MLP_NB - 1);
        const double g = exp(-(r - mu) * (r - mu) / (2.0 * w * w));
        phi[k] = g * fc;
        dphi[k] = g * (-(r - mu) / (w * w)) * fc + g * dfc;
    }
    double z1[ORC_MLP_H], dz1[ORC_MLP_H], h1[ORC_MLP_H], dh1[ORC_MLP_H];
    for (int a = 0; a < ORC_MLP_H; ++a) {
        double s = b1[a], ds = 0.0;
        for (int k = 0; k < ORC_MLP_NB; ++k) {
            s += W1[a * ORC_MLP_NB + k] * phi[k];
            ds += W1[a * ORC_MLP_NB + k] * dphi[k];
        }
        z1[a] = s;
        dz1[a] = ds;
        const double sg = sigmoid(s);
        h1[a] = s * sg;
        dh1[a] = sg * (1.0 + s * (1.0 - sg)) * ds;
    }
    double z2[ORC_MLP_H], dz2[ORC_MLP_H], h2[ORC_MLP_H], dh2[ORC_MLP_H];
    double u = b3, du = 0.0;
    for (int a = 0; a < ORC_MLP_H; ++a) {
        double s = b2[a], ds = 0.0;
        for (int k = 0; k < ORC_MLP_H; ++k) {
            s += W2[a * ORC_MLP_H + k] * h1[k];
            ds += W2[a * ORC_MLP_H + k] * dh1[k];
        }
        z2[a] = s;
        dz2[a] = ds;
        const double sg = sigmoid(s);
        h2[a] = s * sg;
        dh2[a] = sg * (1.0 + s * (1.0 - sg)) * ds;
        u += w3[a] * h2[a];
        du += w3[a] * dh2[a];
    }
    *u_out = u;
    *dudr_out = du;
    if (!grad && !ugrad) return;
    /* Reverse pass through the pair (primal, tangent).  With s = sigmoid:
     * silu'(z) = s (1 + z (1 - s)),  silu''(z) = s (1 - s) (2 + z (1 - 2 s)).
     * Adjoints: for the tangent output du = w3 . dh2 and the primal output
     * u = w3 . h2 + b3. */
    double* gW1 = grad;
    double* gb1 = grad ? grad + ORC_MLP_H * ORC_MLP_NB : NULL;
    double* gW2 = grad ? gb1 + ORC_MLP_H : NULL;
    double* gb2 = grad ? gW2 + ORC_MLP_H * ORC_MLP_H : NULL;
    double* gw3 = grad ? gb2 + ORC_MLP_H : NULL;
    if (grad) {
        /* d(du)/d(w3_a) = dh2_a; layer-2 adjoints of the tangent path */
        double az2[ORC_MLP_H], adz2[ORC_MLP_H];
        for (int a = 0; a < ORC_MLP_H; ++a) {
            const double sg = sigmoid(z2[a]);
            const double s1 = sg * (1.0 + z2[a] * (1.0 - sg));
            const double s2 = sg * (1.0 - sg) * (2.0 + z2[a] * (1.0 - 2.0 * sg));
            gw3[a] = dh2[a];
            adz2[a] = w3[a] * s1;             /* d du / d dz2 */
            az2[a] = w3[a] * s2 * dz2[a];     /* d du / d z2 */
        }
        gw3[ORC_MLP_H] = 0.0; /* b3 */
        double ah1[ORC_MLP_H], adh1[ORC_MLP_H];
        for (int k = 0; k < ORC_MLP_H; ++k) {
            ah1[k] = 0.0;
            adh1[k] = 0.0;
        }
        for (int a = 0; a < ORC_MLP_H; ++a) {
            gb2[a] = az2[a];
            for (int k = 0; k < ORC_MLP_H; ++k) {
                gW2[a * ORC_MLP_H + k] = az2[a] * h1[k] + adz2[a] * dh1[k];
                ah1[k] += W2[a * ORC_MLP_H + k] * az2[a];
                adh1[k] += W2[a * ORC_MLP_H + k] * adz2[a];
            }
        }
        for (int a = 0; a < ORC_MLP_H; ++a) {
            const double sg = sigmoid(z1[a]);
            const double s1 = sg * (1.0 + z1[a] * (1.0 - sg));
            const double s2 = sg * (1.0 - sg) * (2.0 + z1[a] * (1.0 - 2.0 * sg));
            const double adz1 = adh1[a] * s1;
            const double az1 = ah1[a] * s1 + adh1[a] * s2 * dz1[a];
            gb1[a] = az1;
            for (int k = 0; k < ORC_MLP_NB; ++k) gW1[a * ORC_MLP_NB + k] = az1 * phi[k] + adz1 * dphi[k];
        }
    }
    if (ugrad) {
        double* uW1 = ugrad;
        double* ub1 = ugrad + ORC_MLP_H * ORC_MLP_NB;
        double* uW2 = ub1 + ORC_MLP_H;
        double* ub2 = uW2 + ORC_MLP_H * ORC_MLP_H;
        double* uw3 = ub2 + ORC_MLP_H;
        double az2[ORC_MLP_H], ah1[ORC_MLP_H];
        for (int a = 0; a < ORC_MLP_H; ++a) {
            const double sg = sigmoid(z2[a]);
            uw3[a] = h2[a];
            az2[a] = w3[a] * sg * (1.0 + z2[a] * (1.0 - sg));
            ah1[a] = 0.0;
        }
        uw3[ORC_MLP_H] = 1.0;
        for (int a = 0; a < ORC_MLP_H; ++a) {
            ub2[a] = az2[a];
            for (int k = 0; k < ORC_MLP_H; ++k) {
                uW2[a * ORC_MLP_H + k] = az2[a] * h1[k];
                ah1[k] += W2[a * ORC_MLP_H + k] * az2[a];
            }
        }
        for (int a = 0; a < ORC_MLP_H; ++a) {
            const double sg = sigmoid(z1[a]);
            const double az1 = ah1[a] * sg * (1.0 + z1[a] * (1.0 - sg));
            ub1[a] = az1;
            for (int k = 0; k < ORC_MLP_NB; ++k) uW1[a * ORC_MLP_NB + k] = az1 * phi[k];
        }
    }
}

/* Pair record [kind, eps, sigma, rc, shift_flag, caprad].
 * kind 1: Lennard-Jones cut at rc (r < rc strictly).  With shift_flag the
 *   energy is lowered by U(rc) so that it is zero at the cutoff; the force is
 *   not changed (the example script's shift='auto').  WCA is this with
 *   rc = 2^(1/6) sigma.
 * kind 3: tabulated, record [3, table slot, 0, rc]: u and F from the table.
 * kind 4: the learned MLP pair potential (orc_set_mlp), record [4, 0, 0, rc].
 * kind 2: capped Lennard-Jones (the example's LennardJonesCapped).  Reading:
 *   for r < caprad the force keeps the direction of r_ij and the magnitude
 *   |F(caprad)| it has at caprad; the energy continues linearly,
 *   U(caprad) + |F(caprad)| (caprad - r), so that F = -dU/dr everywhere. */
void orc_pair_eval(const double* pp, double r2, double* u, double* fr) {
    *u = 0.0;
    *fr = 0.0;
    int kind = (int)pp[0];
    double eps = pp[1], sig = pp[2], rc = pp[3];
    if (kind == 0 || r2 >= rc * rc) return;
    double shift = 0.0;
    if (pp[4] != 0.0) {
        double us, fs;
        lj_raw(eps, sig, rc * rc, &us, &fs);
        shift = us;
    }
    if (kind == 3) {
        double r = sqrt(r2), F;
        table_eval((int)pp[1], r, u, &F);
        *fr = F / r;
        return;
    }
    if (kind == 4) {
        double r = sqrt(r2), du;
        orc_mlp_pair(r, u, &du, NULL, NULL);
        *fr = -du / r;
        return;
    }
    if (kind == 1) {
        lj_raw(eps, sig, r2, u, fr);
        *u -= shift;
    } else if (kind == 2) {
        double cap = pp[5];
        if (r2 < cap * cap) {
            double uc, frc;
            lj_raw(eps, sig, cap * cap, &uc, &frc);
            double fmag = frc * cap; /* |F| at the capping radius */
            double r = sqrt(r2);
            *u = uc - shift + fmag * (cap - r);
            *fr = fmag / r;
        } else {
            lj_raw(eps, sig, r2, u, fr);
            *u -= shift;
        }
    }
}

/* Bond record [kind, K, R0].  kind 1: FENE, U = -1/2 K R0^2 ln(1 - r^2/R0^2),
 * F_i = -K r_ij / (1 - r^2/R0^2).  Reading: r >= R0 is an error (no bond
 * breaking); returns 1 then.  kind 2: tabulated bond, record [2, table slot]:
 * u and F from the table; r >= the table's rmax is an error like r >= R0. */
int orc_bond_eval(const double* bp, double r2, double* u, double* fr) {
    *u = 0.0;
    *fr = 0.0;
    int kind = (int)bp[0];
    if (kind == 0) return 0;
    if (kind == 2) {
        int slot = (int)bp[1];
        double r = sqrt(r2), F;
        if (r >= orc_tables[slot].rmax) return 1;
        table_eval(slot, r, u, &F);
        *fr = r > 0.0 ? F / r : 0.0;
        return 0;
    }
    if (kind == 1) {
        double K = bp[1], R0 = bp[2];
        double q = r2 / (R0 * R0);
        if (q >= 1.0) return 1;
        *u = -0.5 * K * R0 * R0 * log(1.0 - q);
        *fr = -K / (1.0 - q);
    }
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Linked cells (textbook head/next lists), used to find all pairs within a  */
/* cutoff.  When a box edge holds fewer than 3 cells every particle is       */
/* compared with every other one instead.                                    */
/* ------------------------------------------------------------------------ */
typedef struct {
    int nc[3];
    int brute;
    int64_t* head; /* per cell: first particle, or -1 */
    int64_t* next; /* per particle: next particle in the same cell, or -1 */
    int64_t* cell_of;
} cells_t;

static int64_t cell_coord(double xc, double L, int nc) {
    double w = xc - L * floor(xc / L); /* into [0, L) */
    int64_t c = (int64_t)floor(w / (L / nc));
    if (c < 0) c = 0;
    if (c >= nc) c = nc - 1;
    return c;
}

static void cells_build(cells_t* cl, int64_t n, const double* L, const double* x, double rcut) {
    cl->brute = 0;
    for (int c = 0; c < 3; ++c) {
        cl->nc[c] = (rcut > 0.0) ? (int)floor(L[c] / rcut) : 1;
        if (cl->nc[c] < 3) cl->brute = 1;
    }
    cl->head = NULL;
    cl->next = NULL;
    cl->cell_of = NULL;
    if (cl->brute) return;
    int64_t ncell = (int64_t)cl->nc[0] * cl->nc[1] * cl->nc[2];
    cl->head = (int64_t*)malloc(sizeof(int64_t) * ncell);
    cl->next = (int64_t*)malloc(sizeof(int64_t) * (n > 0 ? n : 1));
    cl->cell_of = (int64_t*)malloc(sizeof(int64_t) * (n > 0 ? n : 1));
    for (int64_t c = 0; c < ncell; ++c) cl->head[c] = -1;
    /* insert in descending id order so each cell's list runs in ascending id */
    for (int64_t i = n - 1; i >= 0; --i) {
        int64_t cx = cell_coord(x[3 * i + 0], L[0], cl->nc[0]);
        int64_t cy = cell_coord(x[3 * i + 1], L[1], cl->nc[1]);
        int64_t cz = cell_coord(x[3 * i + 2], L[2], cl->nc[2]);
        int64_t c = (cz * cl->nc[1] + cy) * cl->nc[0] + cx;
        cl->cell_of[i] = c;
        cl->next[i] = cl->head[c];
        cl->head[c] = i;
    }
}

static void cells_free(cells_t* cl) {
    free(cl->head);
    free(cl->next);
    free(cl->cell_of);
}

/* Calls visit(j) for every j != i in the 27 cells around i's cell (or every
 * j != i when the box is too small for cells).  Expressed as an iterator that
 * fills a caller buffer to keep the C plain. */
static int64_t cells_candidates(const cells_t* cl, int64_t n, int64_t i, int64_t* buf) {
    int64_t m = 0;
    if (cl->brute) {
        for (int64_t j = 0; j < n; ++j)
            if (j != i) buf[m++] = j;
        return m;
    }
    int64_t c = cl->cell_of[i];
    int64_t cx = c % cl->nc[0];
    int64_t cy = (c / cl->nc[0]) % cl->nc[1];
    int64_t cz = c / ((int64_t)cl->nc[0] * cl->nc[1]);
    for (int dz = -1; dz <= 1; ++dz) {
        /* under Lees-Edwards the rows across the z faces are displaced along
         * x by the shear offset: take the whole x row there */
        const int across = orc_le_on && (cz + dz < 0 || cz + dz >= cl->nc[2]);
        for (int dy = -1; dy <= 1; ++dy) {
            const int x0 = across ? 0 : -1, x1 = across ? cl->nc[0] - 1 : 1;
            for (int dx = x0; dx <= x1; ++dx) {
                int64_t ax = across ? dx : (cx + dx + cl->nc[0]) % cl->nc[0];
                int64_t ay = (cy + dy + cl->nc[1]) % cl->nc[1];
                int64_t az = (cz + dz + cl->nc[2]) % cl->nc[2];
                int64_t a = (az * cl->nc[1] + ay) * cl->nc[0] + ax;
                for (int64_t j = cl->head[a]; j >= 0; j = cl->next[j])
                    if (j != i) buf[m++] = j;
            }
        }
    }
    return m;
}

static int64_t max_candidates(const cells_t* cl, int64_t n) {
    if (cl->brute || orc_le_on) return n;
    int64_t ncell = (int64_t)cl->nc[0] * cl->nc[1] * cl->nc[2];
    int64_t* cnt = (int64_t*)calloc((size_t)ncell, sizeof(int64_t));
    for (int64_t i = 0; i < n; ++i) cnt[cl->cell_of[i]]++;
    int64_t mx = 0;
    for (int64_t c = 0; c < ncell; ++c)
        if (cnt[c] > mx) mx = cnt[c];
    free(cnt);
    return 27 * mx + 1;
}

/* ------------------------------------------------------------------------ */
/* Neighbour sets                                                            */
/* ------------------------------------------------------------------------ */
static int cmp_i64(const void* a, const void* b) {
    int64_t x = *(const int64_t*)a, y = *(const int64_t*)b;
    return (x > y) - (x < y);
}

/* Definition: all ordered pairs (i, j), j != i, whose minimum-image distance
 * is below rcut (strict).  O(n^2). */
int64_t orc_neighbors_brute(int64_t n, const double* L, const double* x, double rcut,
                            int64_t* row_ptr, int64_t* cols, int64_t cap) {
    int64_t m = 0;
    row_ptr[0] = 0;
    for (int64_t i = 0; i < n; ++i) {
        for (int64_t j = 0; j < n; ++j) {
            if (j == i) continue;
            double d[3];
            min_image_vec(x + 3 * i, x + 3 * j, L, d);
            double r2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
            if (r2 < rcut * rcut) {
                if (m >= cap) return -1;
                cols[m++] = j;
            }
        }
        row_ptr[i + 1] = m;
    }
    return m;
}

/* The same set found through linked cells of edge >= rcut. */
int64_t orc_neighbors_cells(int64_t n, const double* L, const double* x, double rcut,
                            int64_t* row_ptr, int64_t* cols, int64_t cap) {
    cells_t cl;
    cells_build(&cl, n, L, x, rcut);
    int64_t* buf = (int64_t*)malloc(sizeof(int64_t) * (size_t)max_candidates(&cl, n));
    int64_t m = 0;
    row_ptr[0] = 0;
    for (int64_t i = 0; i < n; ++i) {
        int64_t nc = cells_candidates(&cl, n, i, buf);
        int64_t row0 = m;
        for (int64_t k = 0; k < nc; ++k) {
            int64_t j = buf[k];
            double d[3];
            min_image_vec(x + 3 * i, x + 3 * j, L, d);
            double r2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
            if (r2 < rcut * rcut) {
                if (m >= cap) {
                    free(buf);
                    cells_free(&cl);
                    return -1;
                }
                cols[m++] = j;
            }
        }
        qsort(cols + row0, (size_t)(m - row0), sizeof(int64_t), cmp_i64);
        row_ptr[i + 1] = m;
    }
    free(buf);
    cells_free(&cl);
    return m;
}

/* ------------------------------------------------------------------------ */
/* Forces                                                                    */
/* ------------------------------------------------------------------------ */
typedef struct {
    int64_t* off; /* n+1 */
    int64_t* nbr; /* partner ids */
} adj_t;

static void adj_build(adj_t* a, int64_t n, int64_t nbonds, const int64_t* bonds) {
    a->off = (int64_t*)calloc((size_t)n + 1, sizeof(int64_t));
    a->nbr = (int64_t*)malloc(sizeof(int64_t) * (size_t)(2 * nbonds + 1));
    for (int64_t b = 0; b < nbonds; ++b) {
        a->off[bonds[2 * b] + 1]++;
        a->off[bonds[2 * b + 1] + 1]++;
    }
    for (int64_t i = 0; i < n; ++i) a->off[i + 1] += a->off[i];
    int64_t* fill = (int64_t*)malloc(sizeof(int64_t) * (size_t)(n + 1));
    memcpy(fill, a->off, sizeof(int64_t) * (size_t)(n + 1));
    for (int64_t b = 0; b < nbonds; ++b) {
        int64_t p = bonds[2 * b], q = bonds[2 * b + 1];
        a->nbr[fill[p]++] = q;
        a->nbr[fill[q]++] = p;
    }
    free(fill);
}

static void adj_free(adj_t* a) {
    free(a->off);
    free(a->nbr);
}

/* Reading (learned CG model): 1-2 bonded pairs can be excluded from the pair
 * interactions, so that the bonded (tabulated) potential alone acts between
 * them.  Off by default (Kremer-Grest keeps WCA between bonded beads). */
static int orc_exclude_bonded = 0;
void orc_set_exclude_bonded(int on) { orc_exclude_bonded = on ? 1 : 0; }

static int bonded_to(const adj_t* a, int64_t i, int64_t j) {
    for (int64_t k = a->off[i]; k < a->off[i + 1]; ++k)
        if (a->nbr[k] == j) return 1;
    return 0;
}

/* Definition: F_i = sum over j != i with r_ij < rc(t_i, t_j) of the pair force
 * plus the sum over bonds (i, p) of the bond force.  There are no exclusions:
 * bonded beads also interact through the pair potential (Kremer-Grest).
 * PE_pair = sum over unordered pairs of u, PE_bond = sum over bonds of u,
 * virial = sum over unordered pairs and bonds of r_ij . F_ij, and its xz
 * component W_xz = sum of (r_ij)_x (F_ij)_z.  Each particle accumulates its
 * own sum (both orders of every pair are evaluated). */
int orc_forces(int64_t n, const double* L, const double* x, const int32_t* type,
               int ntypes, const double* pair_params, int64_t nbonds,
               const int64_t* bonds, const double* bond_params, double* f,
               double* energies) {
    double rmax = 0.0;
    for (int t = 0; t < ntypes * ntypes; ++t) {
        const double* pp = pair_params + ORC_PAIR_STRIDE * t;
        if ((int)pp[0] != 0 && pp[3] > rmax) rmax = pp[3];
    }
    cells_t cl;
    cells_build(&cl, n, L, x, rmax);
    adj_t adj;
    adj_build(&adj, n, nbonds, bonds);
    double* pe_p = (double*)calloc((size_t)n + 1, sizeof(double));
    double* pe_b = (double*)calloc((size_t)n + 1, sizeof(double));
    double* vir = (double*)calloc((size_t)n + 1, sizeof(double));
    double* vxz = (double*)calloc((size_t)n + 1, sizeof(double));
    int64_t mc = max_candidates(&cl, n);
    int broken = 0;

#pragma omp parallel reduction(| : broken)
    {
        int64_t* buf = (int64_t*)malloc(sizeof(int64_t) * (size_t)mc);
#pragma omp for schedule(static)
        for (int64_t i = 0; i < n; ++i) {
            double fi[3] = {0.0, 0.0, 0.0};
            double ui = 0.0, ub = 0.0, wi = 0.0, wxz = 0.0;
            if (rmax > 0.0) {
                int64_t nc = cells_candidates(&cl, n, i, buf);
                for (int64_t k = 0; k < nc; ++k) {
                    int64_t j = buf[k];
                    if (orc_exclude_bonded && bonded_to(&adj, i, j)) continue;
                    double d[3];
                    min_image_vec(x + 3 * i, x + 3 * j, L, d);
                    double r2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
                    const double* pp = pair_params + ORC_PAIR_STRIDE * (type[i] * ntypes + type[j]);
                    double u, fr;
                    orc_pair_eval(pp, r2, &u, &fr);
                    for (int c = 0; c < 3; ++c) fi[c] += fr * d[c];
                    ui += 0.5 * u;
                    wi += 0.5 * fr * r2;
                    wxz += 0.5 * fr * d[0] * d[2];
                }
            }
            for (int64_t k = adj.off[i]; k < adj.off[i + 1]; ++k) {
                int64_t p = adj.nbr[k];
                double d[3];
                min_image_vec(x + 3 * i, x + 3 * p, L, d);
                double r2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
                double u, fr;
                if (orc_bond_eval(bond_params, r2, &u, &fr)) broken = 1;
                for (int c = 0; c < 3; ++c) fi[c] += fr * d[c];
                ub += 0.5 * u;
                wi += 0.5 * fr * r2;
                wxz += 0.5 * fr * d[0] * d[2];
            }
            for (int c = 0; c < 3; ++c) f[3 * i + c] = fi[c];
            pe_p[i] = ui;
            pe_b[i] = ub;
            vir[i] = wi;
            vxz[i] = wxz;
        }
        free(buf);
    }
    double sp = 0.0, sb = 0.0, sw = 0.0, sxz = 0.0;
    for (int64_t i = 0; i < n; ++i) {
        sp += pe_p[i];
        sb += pe_b[i];
        sw += vir[i];
        sxz += vxz[i];
    }
    if (energies) {
        energies[0] = sp;
        energies[1] = sb;
        energies[2] = sw;
        energies[3] = sxz;
    }
    free(pe_p);
    free(pe_b);
    free(vir);
    free(vxz);
    adj_free(&adj);
    cells_free(&cl);
    return broken ? -4 : 0;
}

/* The same definition as orc_forces, evaluated only for the particles listed
 * in sel[nsel] (for sampled checks of large systems): f_out is nsel*3. */
int orc_forces_subset(int64_t n, const double* L, const double* x, const int32_t* type,
                      int ntypes, const double* pair_params, int64_t nbonds,
                      const int64_t* bonds, const double* bond_params, int64_t nsel,
                      const int64_t* sel, double* f_out) {
    double rmax = 0.0;
    for (int t = 0; t < ntypes * ntypes; ++t) {
        const double* pp = pair_params + ORC_PAIR_STRIDE * t;
        if ((int)pp[0] != 0 && pp[3] > rmax) rmax = pp[3];
    }
    cells_t cl;
    cells_build(&cl, n, L, x, rmax);
    adj_t adj;
    adj_build(&adj, n, nbonds, bonds);
    int64_t mc = max_candidates(&cl, n);
    int broken = 0;
#pragma omp parallel reduction(| : broken)
    {
        int64_t* buf = (int64_t*)malloc(sizeof(int64_t) * (size_t)mc);
#pragma omp for schedule(dynamic, 16)
        for (int64_t q = 0; q < nsel; ++q) {
            int64_t i = sel[q];
            double fi[3] = {0.0, 0.0, 0.0};
            if (rmax > 0.0) {
                int64_t nc = cells_candidates(&cl, n, i, buf);
                for (int64_t k = 0; k < nc; ++k) {
                    int64_t j = buf[k];
                    if (orc_exclude_bonded && bonded_to(&adj, i, j)) continue;
                    double d[3];
                    min_image_vec(x + 3 * i, x + 3 * j, L, d);
                    double r2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
                    double u, fr;
                    orc_pair_eval(pair_params + ORC_PAIR_STRIDE * (type[i] * ntypes + type[j]), r2, &u, &fr);
                    for (int c = 0; c < 3; ++c) fi[c] += fr * d[c];
                }
            }
            for (int64_t k = adj.off[i]; k < adj.off[i + 1]; ++k) {
                int64_t p = adj.nbr[k];
                double d[3];
                min_image_vec(x + 3 * i, x + 3 * p, L, d);
                double r2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
                double u, fr;
                if (orc_bond_eval(bond_params, r2, &u, &fr)) broken = 1;
                for (int c = 0; c < 3; ++c) fi[c] += fr * d[c];
            }
            for (int c = 0; c < 3; ++c) f_out[3 * q + c] = fi[c];
        }
        free(buf);
    }
    adj_free(&adj);
    cells_free(&cl);
    return broken ? -4 : 0;
}

/* Force-matching loss of the learned pair potential and its gradient
 * (the learned CG model; reading: mean squared force error over all
 * frames and sites, the target being the mapped force minus the bonded
 * force).  For frame f with positions X_f and targets Y_f:
 *   e_i = F_pair,i(X_f) + F_bond,i(X_f) - Y_f,i,   loss = sum |e_i|^2 / (F n).
 * F_pair,i = sum_j -u'(r_ij) r_ij_hat, so
 *   d loss / d theta = sum_f sum_i sum_j -(2 / (F n)) (e_i . r_ij_hat)
 *                      d u'(r_ij) / d theta,
 * summed over ordered pairs with the exact parameter gradient of u'.  The
 * pair interactions are those of orc_forces (with the current bonded
 * exclusion setting); grad receives ORC_MLP_NPARAMS values. */
int orc_mlp_loss_grad(int64_t n, const double* L, int64_t nframes, const double* X, const double* Y,
                      const int32_t* type, int64_t nbonds, const int64_t* bonds,
                      const double* bond_params, double* loss_out, double* grad) {
    double pp[ORC_PAIR_STRIDE] = {4, 0, 0, orc_mlp_rc, 0, 0, 0, 0};
    for (int k = 0; k < ORC_MLP_NPAR; ++k) grad[k] = 0.0;
    double loss = 0.0;
    double* f = (double*)malloc(sizeof(double) * (size_t)(3 * n + 3));
    double* gtmp = (double*)malloc(sizeof(double) * ORC_MLP_NPAR);
    adj_t adj;
    adj_build(&adj, n, nbonds, bonds);
    for (int64_t fr = 0; fr < nframes; ++fr) {
        const double* x = X + 3 * n * fr;
        const double* y = Y + 3 * n * fr;
        double en[4];
        int st = orc_forces(n, L, x, type, 1, pp, nbonds, bonds, bond_params, f, en);
        if (st) {
            free(f);
            free(gtmp);
            adj_free(&adj);
            return st;
        }
        for (int64_t i = 0; i < 3 * n; ++i) {
            f[i] -= y[i];
            loss += f[i] * f[i];
        }
        /* pairs within the MLP cutoff, both orders, by brute force */
        const double c = -2.0 / ((double)nframes * (double)n);
        for (int64_t i = 0; i < n; ++i)
            for (int64_t j = 0; j < n; ++j) {
                if (j == i) continue;
                if (orc_exclude_bonded && bonded_to(&adj, i, j)) continue;
                double d[3];
                min_image_vec(x + 3 * i, x + 3 * j, L, d);
                double r2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
                if (r2 >= orc_mlp_rc * orc_mlp_rc) continue;
                double r = sqrt(r2), u, du;
                double w = c * (f[3 * i] * d[0] + f[3 * i + 1] * d[1] + f[3 * i + 2] * d[2]) / r;
                orc_mlp_pair(r, &u, &du, gtmp, NULL);
                for (int k = 0; k < ORC_MLP_NPAR; ++k) grad[k] += w * gtmp[k];
            }
    }
    *loss_out = loss / ((double)nframes * (double)n);
    free(f);
    free(gtmp);
    adj_free(&adj);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Integrator                                                                */
/* ------------------------------------------------------------------------ */

/* Wrap one coordinate into [0, L), counting crossings in the image counter.
 * Reading: a coordinate that rounds to exactly L after adding L is set to 0. */
static void wrap_coord(double* xc, int32_t* im, double L) {
    if (*xc >= L) {
        *xc -= L;
        *im += 1;
    } else if (*xc < 0.0) {
        *xc += L;
        *im -= 1;
        if (*xc >= L) {
            /* x lay less than half an ulp of L below 0: it stays at 0 in its
             * own image, so x + img L is continuous */
            *xc = 0.0;
            *im += 1;
        }
    }
}

/* Wrap under Lees-Edwards: crossing a z face by k boxes moves the particle
 * to the image it entered, displaced by -k delta along x and slower by
 * k gdot Lz along x; x and y are then wrapped as usual (x may need several
 * boxes).  The unwrapped position x + img_x Lx + img_z delta(t) is continuous
 * in time (delta the offset without reduction). */
static void le_wrap(double* xi, double* vi, int32_t* im, const double* L, double delta) {
    const int32_t z0 = im[2];
    wrap_coord(&xi[2], &im[2], L[2]);
    const int kz = im[2] - z0;
    if (kz != 0) {
        xi[0] -= kz * delta;
        vi[0] -= kz * orc_le_shear * L[2];
        double k = floor(xi[0] / L[0]);
        xi[0] -= k * L[0];
        if (xi[0] >= L[0]) {
            xi[0] -= L[0];
            k += 1.0;
        }
        if (xi[0] < 0.0) xi[0] = 0.0;
        im[0] += (int32_t)k;
    } else {
        wrap_coord(&xi[0], &im[0], L[0]);
    }
    wrap_coord(&xi[1], &im[1], L[1]);
}

/* Langevin force (added to the conservative force in the force step):
 * -gamma m v + sqrt(24 gamma m kT / dt) r, r from the Philox stream.
 * Reading (discretisation; the paper names only gamma and T): the friction
 * uses the velocity present when the force is evaluated (the half-step
 * velocity inside a step) and the uniform noise has the variance
 * 2 gamma m kT / dt of the continuous white noise over one step. */
static void add_langevin(int64_t n, const double* L, const double* x, const double* v, const int32_t* type,
                         const double* mass_of_type, double* f, double dt, double gamma,
                         double kT, uint64_t seed, int64_t step) {
    if (gamma == 0.0) return;
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; ++i) {
        double m = mass_of_type[type[i]];
        double amp = sqrt(24.0 * gamma * m * kT / dt);
        double r[3];
        langevin_r(seed, i, step, r);
        /* under Lees-Edwards the friction acts on the velocity relative to
         * the imposed streaming profile (reading) */
        double vp[3] = {v[3 * i + 0] - le_stream(x[3 * i + 2], L), v[3 * i + 1], v[3 * i + 2]};
        for (int c = 0; c < 3; ++c) f[3 * i + c] += -gamma * m * vp[c] + amp * r[c];
    }
}

/* Dissipative particle dynamics thermostat (paper "Functionality": DPD), the
 * pairwise alternative to the Langevin extension.  For every pair at
 * distance r < rc (r_ij = x_i - x_j, e = r_ij / r, v_ij = v_i - v_j):
 *   F_i += [-gamma w(r)^2 (e . v_ij) + sigma w(r) theta_ij / sqrt(dt)] e,
 *   w(r) = 1 - r / rc, sigma^2 = 2 gamma kT  (Espanol-Warren fluctuation-
 *   dissipation relation; Groot-Warren weight functions).
 * Reading: theta_ij has zero mean and unit variance: sqrt(12) times the
 * centred uniform of word 0 of Philox4x32-10 with key (seed lo, seed hi) and
 * counter (min id, max id | 2^31, step lo, step hi), so theta_ij = theta_ji
 * and the pair forces cancel exactly; the velocity is the one present at the
 * force evaluation (as for the Langevin friction).  Under Lees-Edwards the
 * image of j across the z faces moves at k gdot Lz along x: v_ij is taken
 * against that image's velocity.  Reading: the thermostat acts on the pairs
 * of the pair interaction, so with 1-2 bonded exclusions on (the learned CG
 * model) bonded pairs get no DPD force either. */
static int orc_dpd_on = 0;
static double orc_dpd_rc = 0.0;
void orc_set_dpd(int on, double rc) {
    orc_dpd_on = on ? 1 : 0;
    orc_dpd_rc = rc;
}

double orc_dpd_theta(uint64_t seed, int64_t a, int64_t b, int64_t step) {
    const int64_t lo = a < b ? a : b, hi = a < b ? b : a;
    uint32_t key[2] = {(uint32_t)(seed & 0xffffffffu), (uint32_t)(seed >> 32)};
    uint64_t s = (uint64_t)step;
    uint32_t ctr[4] = {(uint32_t)lo, (uint32_t)hi | 0x80000000u, (uint32_t)(s & 0xffffffffu), (uint32_t)(s >> 32)};
    uint32_t out[4];
    orc_philox4x32_10(ctr, key, out);
    return sqrt(12.0) * orc_uniform_centered(out[0]);
}

static void add_dpd(int64_t n, const double* L, const double* x, const double* v, int64_t nbonds,
                    const int64_t* bonds, double* f, double dt, double gamma, double kT, uint64_t seed,
                    int64_t step) {
    if (gamma == 0.0 && kT == 0.0) return;
    const double rc = orc_dpd_rc, sigma = sqrt(2.0 * gamma * kT), inv_sqdt = 1.0 / sqrt(dt);
    adj_t adj;
    adj_build(&adj, n, nbonds, bonds);
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t i = 0; i < n; ++i) {
        double fi[3] = {0.0, 0.0, 0.0};
        for (int64_t j = 0; j < n; ++j) {
            if (j == i) continue;
            if (orc_exclude_bonded && bonded_to(&adj, i, j)) continue;
            double d[3];
            int nz;
            min_image_le(x + 3 * i, x + 3 * j, L, d, &nz);
            const double r2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
            if (!(r2 < rc * rc)) continue;
            const double r = sqrt(r2), w = 1.0 - r / rc;
            double vij[3];
            for (int c = 0; c < 3; ++c) vij[c] = v[3 * i + c] - v[3 * j + c];
            if (orc_le_on) vij[0] -= nz * orc_le_shear * L[2];
            double ev = 0.0;
            for (int c = 0; c < 3; ++c) ev += d[c] / r * vij[c];
            const double mag = -gamma * w * w * ev + sigma * w * orc_dpd_theta(seed, i, j, step) * inv_sqdt;
            for (int c = 0; c < 3; ++c) fi[c] += mag * d[c] / r;
        }
        for (int c = 0; c < 3; ++c) f[3 * i + c] += fi[c];
    }
    adj_free(&adj);
}

/* the thermostat of the force step: DPD when selected, else Langevin */
static void add_thermostat(int64_t n, const double* L, const double* x, const double* v, const int32_t* type,
                           const double* mass_of_type, int64_t nbonds, const int64_t* bonds, double* f,
                           double dt, double gamma, double kT, uint64_t seed, int64_t step) {
    if (orc_dpd_on) add_dpd(n, L, x, v, nbonds, bonds, f, dt, gamma, kT, seed, step);
    else add_langevin(n, L, x, v, type, mass_of_type, f, dt, gamma, kT, seed, step);
}

/* Velocity Verlet (the example's VelocityVerlet) with the Langevin extension.
 * One step from step s-1 to s:
 *   1. v += dt/2 F/m            (F of step s-1)
 *   2. x += dt v, wrap into the box, update image counters
 *   3. F = conservative forces at the new x
 *   4. F += -gamma m v + sqrt(24 gamma m kT/dt) r(s)   (or the DPD pair terms)
 *   5. v += dt/2 F/m
 * Reading: when f is not valid on entry, F of step step0 is first computed
 * from x, v with the noise of step step0. */
int orc_integrate(int64_t n, const double* L, double* x, double* v, int32_t* img,
                  const int32_t* type, const double* mass_of_type, int ntypes,
                  const double* pair_params, int64_t nbonds, const int64_t* bonds,
                  const double* bond_params, double* f, int f_valid, double dt,
                  double gamma, double kT, uint64_t seed, int64_t step0, int64_t nsteps) {
    double en[4];
    int st = 0;
    const double t0 = orc_le_time;  /* simulated time of step0 (Lees-Edwards offset) */
    if (!f_valid) {
        st = orc_forces(n, L, x, type, ntypes, pair_params, nbonds, bonds, bond_params, f, en);
        if (st) return st;
        add_thermostat(n, L, x, v, type, mass_of_type, nbonds, bonds, f, dt, gamma, kT, seed, step0);
    }
    for (int64_t s = step0 + 1; s <= step0 + nsteps; ++s) {
        orc_le_time = t0 + (double)(s - step0) * dt;
        const double delta = le_delta(L);
#pragma omp parallel for schedule(static)
        for (int64_t i = 0; i < n; ++i) {
            double m = mass_of_type[type[i]];
            for (int c = 0; c < 3; ++c) {
                v[3 * i + c] += 0.5 * dt * f[3 * i + c] / m;
                x[3 * i + c] += dt * v[3 * i + c];
            }
            if (orc_le_on) {
                le_wrap(x + 3 * i, v + 3 * i, img + 3 * i, L, delta);
            } else {
                for (int c = 0; c < 3; ++c) wrap_coord(&x[3 * i + c], &img[3 * i + c], L[c]);
            }
        }
        st = orc_forces(n, L, x, type, ntypes, pair_params, nbonds, bonds, bond_params, f, en);
        if (st) return st;
        add_thermostat(n, L, x, v, type, mass_of_type, nbonds, bonds, f, dt, gamma, kT, seed, s);
#pragma omp parallel for schedule(static)
        for (int64_t i = 0; i < n; ++i) {
            double m = mass_of_type[type[i]];
            for (int c = 0; c < 3; ++c) v[3 * i + c] += 0.5 * dt * f[3 * i + c] / m;
        }
        for (int64_t i = 0; i < 3 * n; ++i)
            if (!isfinite(x[i]) || !isfinite(v[i])) return -5;
    }
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Observables                                                               */
/* ------------------------------------------------------------------------ */
static int64_t uf_find(int64_t* parent, int64_t a) {
    while (parent[a] != a) {
        parent[a] = parent[parent[a]];
        a = parent[a];
    }
    return a;
}

/* out[0] KE = sum 1/2 m v^2; out[1] PE_pair; out[2] PE_bond; out[3] virial W;
 * out[4..6] total momentum; out[7] T = 2 KE / (3 n) (Langevin: no constraint
 * removes degrees of freedom); out[8] P = (2 KE + W) / (3 V);
 * out[9] mean bond length; out[10] mean squared radius of gyration over
 * molecules (connected components of the bond graph with >= 2 beads, from
 * unwrapped positions x + img L); out[11] number of such molecules;
 * out[12] the xz component of the pressure tensor,
 * P_xz = (sum m v_x v_z + W_xz) / V.  Under Lees-Edwards the kinetic terms
 * (KE, T, P, P_xz) use the velocity relative to the streaming profile and
 * the unwrapped x adds img_z delta(t). */
int orc_observables(int64_t n, const double* L, const double* x, const double* v,
                    const int32_t* img, const int32_t* type, const double* mass_of_type,
                    int ntypes, const double* pair_params, int64_t nbonds,
                    const int64_t* bonds, const double* bond_params, double* out) {
    for (int k = 0; k < ORC_NOBS; ++k) out[k] = 0.0;
    double* f = (double*)malloc(sizeof(double) * (size_t)(3 * n + 1));
    double en[4];
    int st = orc_forces(n, L, x, type, ntypes, pair_params, nbonds, bonds, bond_params, f, en);
    free(f);
    double ke = 0.0, p[3] = {0, 0, 0}, kxz = 0.0;
    for (int64_t i = 0; i < n; ++i) {
        double m = mass_of_type[type[i]];
        /* kinetic terms from the velocity relative to the Lees-Edwards
         * streaming profile (the velocity itself without shear) */
        const double vp[3] = {v[3 * i + 0] - le_stream(x[3 * i + 2], L), v[3 * i + 1], v[3 * i + 2]};
        for (int c = 0; c < 3; ++c) {
            ke += 0.5 * m * vp[c] * vp[c];
            p[c] += m * v[3 * i + c];
        }
        kxz += m * vp[0] * vp[2];
    }
    double V = L[0] * L[1] * L[2];
    out[0] = ke;
    out[1] = en[0];
    out[2] = en[1];
    out[3] = en[2];
    out[4] = p[0];
    out[5] = p[1];
    out[6] = p[2];
    out[7] = n > 0 ? 2.0 * ke / (3.0 * (double)n) : 0.0;
    out[8] = (2.0 * ke + en[2]) / (3.0 * V);
    out[12] = (kxz + en[3]) / V;
    double bl = 0.0;
    for (int64_t b = 0; b < nbonds; ++b) {
        double d[3];
        min_image_vec(x + 3 * bonds[2 * b], x + 3 * bonds[2 * b + 1], L, d);
        bl += sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
    }
    out[9] = nbonds > 0 ? bl / (double)nbonds : 0.0;

    int64_t* parent = (int64_t*)malloc(sizeof(int64_t) * (size_t)(n + 1));
    for (int64_t i = 0; i < n; ++i) parent[i] = i;
    for (int64_t b = 0; b < nbonds; ++b) {
        int64_t ra = uf_find(parent, bonds[2 * b]), rb = uf_find(parent, bonds[2 * b + 1]);
        if (ra != rb) parent[ra] = rb;
    }
    double* com = (double*)calloc((size_t)(3 * n + 3), sizeof(double));
    int64_t* cnt = (int64_t*)calloc((size_t)(n + 1), sizeof(int64_t));
    double* rg = (double*)calloc((size_t)(n + 1), sizeof(double));
    for (int64_t i = 0; i < n; ++i) {
        int64_t r = uf_find(parent, i);
        cnt[r]++;
        for (int c = 0; c < 3; ++c) com[3 * r + c] += x[3 * i + c] + img[3 * i + c] * L[c];
        com[3 * r + 0] += img[3 * i + 2] * le_delta(L);
    }
    for (int64_t r = 0; r < n; ++r)
        if (cnt[r] > 0)
            for (int c = 0; c < 3; ++c) com[3 * r + c] /= (double)cnt[r];
    for (int64_t i = 0; i < n; ++i) {
        int64_t r = uf_find(parent, i);
        for (int c = 0; c < 3; ++c) {
            double u = x[3 * i + c] + img[3 * i + c] * L[c] - com[3 * r + c];
            if (c == 0) u += img[3 * i + 2] * le_delta(L);
            rg[r] += u * u;
        }
    }
    double rgsum = 0.0;
    int64_t nmol = 0;
    for (int64_t r = 0; r < n; ++r)
        if (cnt[r] >= 2) {
            rgsum += rg[r] / (double)cnt[r];
            nmol++;
        }
    out[10] = nmol > 0 ? rgsum / (double)nmol : 0.0;
    out[11] = (double)nmol;
    free(parent);
    free(com);
    free(cnt);
    free(rg);
    return st;
}

/* Unordered pairs with minimum-image distance r < rmax, counted in bin
 * floor(r / (rmax / nbins)).  O(n^2). */
void orc_rdf_counts(int64_t n, const double* L, const double* x, double rmax,
                    int nbins, int64_t* counts) {
    for (int b = 0; b < nbins; ++b) counts[b] = 0;
    double dr = rmax / nbins;
    for (int64_t i = 0; i < n; ++i)
        for (int64_t j = i + 1; j < n; ++j) {
            double d[3];
            min_image_vec(x + 3 * i, x + 3 * j, L, d);
            double r = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
            if (r < rmax) {
                int b = (int)(r / dr);
                if (b >= nbins) b = nbins - 1;
                counts[b]++;
            }
        }
}

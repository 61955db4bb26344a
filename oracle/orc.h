/*
 * Oracle for the short-range coarse-grained MD step (ESPResSo++, "Software
 * design" and "Example usage" sections): plain, slow, double-precision CPU
 * code written from the definitions of the method.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the CPU
 * baseline leg of the benchmark may load this library.  It shares no code,
 * header, table or helper with the CUDA library, and neither includes the other.
 *
 * Conventions (all arrays in particle-id order; particle i has id i):
 *   x, v, f   : n*3 doubles, row-major (x0,y0,z0,x1,...)
 *   img       : n*3 int32 periodic image counters (unwrapped = x + img*L)
 *   L         : 3 box edges of the orthorhombic periodic box
 *   pair_params: ntypes*ntypes records of ORC_PAIR_STRIDE doubles,
 *                [kind, eps, sigma, rc, shift_flag, caprad, 0, 0]
 *                kind: 0 none, 1 Lennard-Jones, 2 capped Lennard-Jones,
 *                3 tabulated [3, slot, 0, rc], 4 learned MLP [4, 0, 0, rc]
 *   bond_params: ORC_BOND_STRIDE doubles [kind, K, R0, 0]; kind 0 none, 1 FENE,
 *                2 tabulated [2, slot]
 *   bonds     : nbonds*2 int64 particle ids
 *
 * Readings of points the paper leaves open are listed beside each function.
 */
#ifndef ORC_H
#define ORC_H
#include <stdint.h>

#define ORC_PAIR_STRIDE 8
#define ORC_BOND_STRIDE 4
#define ORC_NOBS 13

#ifdef __cplusplus
extern "C" {
#endif

int orc_num_threads(void);

/* Philox4x32-10 counter-based generator (Salmon et al., SC'11). */
void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]);
/* One 32-bit Philox word -> odd multiple of 2^-25 in (-1/2, 1/2). */
double orc_uniform_centered(uint32_t w);
void orc_uniform_fill(const uint32_t* w, int64_t n, double* out);
/* Langevin noise words for particle ids [0,n) at a given step: out n*3. */
void orc_langevin_noise(uint64_t seed, int64_t step, int64_t n, double* out);

/* DPD thermostat instead of Langevin in orc_integrate (pair cutoff rc), and
 * the pair noise theta_ij of a step (zero mean, unit variance). */
void orc_set_dpd(int on, double rc);
double orc_dpd_theta(uint64_t seed, int64_t a, int64_t b, int64_t step);

/* Register a table (u, F = -dU/dr at r_k = k rmax/(n-1)) in slot [0, 16). */
int orc_set_table(int slot, double rmax, int n, const double* u, const double* f);

/* Learned MLP pair potential: parameters in the order W1 (64x32, row = output
 * unit), b1 (64), W2 (64x64), b2 (64), w3 (64), b3 (1); cutoff rc. */
#define ORC_MLP_NPARAMS (64 * 32 + 64 + 64 * 64 + 64 + 64 + 1)
int orc_set_mlp(const double* par, int64_t npar, double rc);
/* u(r), du/dr, and optionally d(du/dr)/dparams and du/dparams (NPARAMS each). */
void orc_mlp_pair(double r, double* u, double* dudr, double* grad_dudr, double* grad_u);

/* Force-matching loss of the learned potential over nframes frames
 * (X, Y: nframes*n*3 positions and target forces) and its gradient. */
int orc_mlp_loss_grad(int64_t n, const double* L, int64_t nframes, const double* X, const double* Y,
                      const int32_t* type, int64_t nbonds, const int64_t* bonds,
                      const double* bond_params, double* loss_out, double* grad);

/* Lees-Edwards boundary conditions: shear rate along x with the gradient
 * along z, and the simulated time t of the state (offset gdot Lz t).  The
 * time advances with orc_integrate; orc_le_get_time reads it back. */
void orc_set_lees_edwards(int on, double shear, double time);
double orc_le_get_time(void);

/* Exclude 1-2 bonded pairs from the pair interactions (default off). */
void orc_set_exclude_bonded(int on);

/* Pair and bond potentials at squared distance r2: energy u and scalar fr
 * such that the force on i is fr * (x_i - x_j). */
void orc_pair_eval(const double* pp, double r2, double* u, double* fr);
int orc_bond_eval(const double* bp, double r2, double* u, double* fr);

/* Conservative forces.  energies[0]=PE_pair, [1]=PE_bond, [2]=virial
 * (sum over pairs and bonds of r_ij . F_ij), [3]=its xz component.  Returns 0, or -4 if a FENE
 * bond is stretched to r >= R0. */
int orc_forces(int64_t n, const double* L, const double* x, const int32_t* type,
               int ntypes, const double* pair_params, int64_t nbonds,
               const int64_t* bonds, const double* bond_params, double* f,
               double* energies);

/* orc_forces restricted to the particles sel[nsel]; f_out is nsel*3. */
int orc_forces_subset(int64_t n, const double* L, const double* x, const int32_t* type,
                      int ntypes, const double* pair_params, int64_t nbonds,
                      const int64_t* bonds, const double* bond_params, int64_t nsel,
                      const int64_t* sel, double* f_out);

/* Neighbour sets {j != i : |x_i - x_j|_min-image < rcut} in CSR, id order,
 * columns ascending.  Returns the number of entries (or -1 if cap is short). */
int64_t orc_neighbors_brute(int64_t n, const double* L, const double* x, double rcut,
                            int64_t* row_ptr, int64_t* cols, int64_t cap);
int64_t orc_neighbors_cells(int64_t n, const double* L, const double* x, double rcut,
                            int64_t* row_ptr, int64_t* cols, int64_t cap);

/* Velocity Verlet with the Langevin thermostat, nsteps steps starting from
 * step number step0.  f holds the total force of step step0 on entry when
 * f_valid != 0; otherwise it is computed first.  x, v, img, f are updated. */
int orc_integrate(int64_t n, const double* L, double* x, double* v, int32_t* img,
                  const int32_t* type, const double* mass_of_type, int ntypes,
                  const double* pair_params, int64_t nbonds, const int64_t* bonds,
                  const double* bond_params, double* f, int f_valid, double dt,
                  double gamma, double kT, uint64_t seed, int64_t step0, int64_t nsteps);

/* Observables (see orc.c for the definitions). */
int orc_observables(int64_t n, const double* L, const double* x, const double* v,
                    const int32_t* img, const int32_t* type, const double* mass_of_type,
                    int ntypes, const double* pair_params, int64_t nbonds,
                    const int64_t* bonds, const double* bond_params, double* out);

/* Unique-pair distance histogram for r < rmax in nbins equal bins. */
void orc_rdf_counts(int64_t n, const double* L, const double* x, double rmax,
                    int nbins, int64_t* counts);

#ifdef __cplusplus
}
#endif
#endif

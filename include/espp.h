/*
 * espp.h -- C ABI of the GB300 short-range coarse-grained MD library
 * (libespp_gb.so).
 *
 * The library implements the per-timestep short-range force loop of the
 * ESPResSo++ package (paper "ESPResSo++: A Fast and Extensible Molecular
 * Simulation Package for Coarse-Grained Models", sections "Software design"
 * and "Example usage"): linked-cell binning, a Verlet list with a skin,
 * Lennard-Jones / WCA pair forces plus FENE bonds, and velocity Verlet with a
 * Langevin thermostat, for bead-spring polymer melts and LJ fluids.  All of it
 * runs in CUDA kernels for sm_103a; nothing falls back to the CPU.
 *
 * General rules
 *  - Every call returns an int status: ESPP_OK (0) or a negative ESPP_ERR_*.
 *    espp_last_error() gives a message for the last failing call on a handle;
 *    espp_last_error(NULL), for the calling thread's last failing call made
 *    without one (creation, espp_h5md_inspect).
 *  - Inputs are copied; the caller keeps ownership of every buffer it passes.
 *    Outputs are written into caller-allocated buffers.
 *  - Buffers tagged "where" are host pointers when where == ESPP_HOST and
 *    device pointers (e.g. torch tensors' data_ptr()) when where == ESPP_DEVICE.
 *  - All particle I/O is in particle-id order (id = index in the arrays the
 *    caller passed at creation), whatever order the library keeps internally.
 *  - Coordinates are double, row-major n x 3.  The library stores them in the
 *    handle's precision (ESPP_FP32 or ESPP_FP64, fixed at creation).
 *  - All work is issued on the CUDA stream given at creation (NULL = the
 *    legacy default stream).  Calls that return data to the host synchronise
 *    that stream.  A handle is not thread-safe; separate handles are
 *    independent.
 *  - A handle may hold several independent systems ("replicas", paper section
 *    "Software design": the example's System object, one per replica).  They
 *    share the interaction set and are stepped together; all per-particle
 *    arrays are the replicas' arrays concatenated in replica order.
 */
#ifndef ESPP_H
#define ESPP_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ------------------------------------------------------ */
#define ESPP_OK 0
#define ESPP_ERR_ARG (-1)            /* invalid argument */
#define ESPP_ERR_CUDA (-2)           /* a CUDA call failed */
#define ESPP_ERR_LIST_OVERFLOW (-3)  /* Verlet list still too small after retries */
#define ESPP_ERR_BOND_BROKEN (-4)    /* a FENE bond reached r >= R0 */
#define ESPP_ERR_NONFINITE (-5)      /* a position became NaN or infinite */
#define ESPP_ERR_TIMEOUT (-6)        /* a bounded device wait gave up */
#define ESPP_ERR_BOX_TOO_SMALL (-7)  /* fewer than 3 cells of rc+skin along an edge */
#define ESPP_ERR_STATE (-8)          /* call out of order (e.g. no positions set) */
#define ESPP_ERR_IO (-9)             /* checkpoint file error */

/* ---- enumerations -------------------------------------------------------- */
#define ESPP_FP32 1
#define ESPP_FP64 2

#define ESPP_HOST 0
#define ESPP_DEVICE 1

/* interaction kinds for espp_set_interaction */
#define ESPP_NONE 0
#define ESPP_LJ 1         /* params: eps, sigma, rc, shift (0/1)                */
#define ESPP_WCA 2        /* params: eps, sigma  (rc = 2^(1/6) sigma, shifted)  */
#define ESPP_LJ_CAPPED 3  /* params: eps, sigma, rc, shift (0/1), caprad        */
#define ESPP_FENE 4       /* params: K, R0  (applies to every bond)             */
#define ESPP_TAB_PAIR 5   /* params: rc, n, u[n], F[n] on r_k = k rc / (n-1)    */
#define ESPP_TAB_BOND 6   /* params: rmax, n, u[n], F[n] on r_k = k rmax / (n-1); every bond */
#define ESPP_MLP 7        /* params: rc; learned pair potential, weights by espp_mlp_set_weights */

#define ESPP_MAX_TYPES 8
#define ESPP_MAX_BONDS_PER_PARTICLE 2

typedef struct espp_system* espp_h;

/* One replica of a batched handle. */
typedef struct {
    double box[3];          /* orthorhombic periodic box edges */
    int64_t n;              /* particles */
    const int32_t* types;   /* n particle types in [0, ESPP_MAX_TYPES), or NULL = all 0 */
    int64_t n_bonds;
    const int64_t* bonds;   /* n_bonds x 2 local particle ids, or NULL */
    uint64_t seed;          /* Philox key of this replica's thermostat noise */
} espp_replica_desc;

/* Observables of one replica (paper: computeEnergy() in "Example usage").
 * Energies are sums over the replica; temperature = 2 ke / (3 n);
 * pressure = (2 ke + virial) / (3 V); virial = sum over pairs and bonds of
 * r_ij . F_ij; mean_bond over bonds; rg2 = mean over molecules (connected
 * components of the bond graph with >= 2 beads) of the squared radius of
 * gyration of the unwrapped positions; pxz = (sum m v_x v_z + sum over pairs
 * and bonds of (r_ij)_x (F_ij)_z) / V, the xz component of the pressure
 * tensor.  Under Lees-Edwards (espp_set_lees_edwards) ke, temperature,
 * pressure and pxz use the velocity relative to the shear profile and the
 * unwrapped x adds img_z delta(t). */
typedef struct {
    int64_t step;
    int64_t n;
    double ke, pe_pair, pe_bond, virial;
    double px, py, pz;
    double temperature, pressure;
    double mean_bond, rg2;
    int64_t n_molecules;
    int64_t n_rebuilds;
    uint32_t error_word;
    uint32_t reserved;
    double pxz;
} espp_obs_t;

/* ---- creation ------------------------------------------------------------ */

/* Create a handle holding one system: paper "Example usage" (System,
 * OrthorhombicBC(box), addParticles with ids/types, bonded topology).
 * box: 3 edges; n particles with types[n] (NULL = all type 0); bonds: n_bonds
 * pairs of particle ids (NULL if none; at most 2 bonds per particle);
 * precision ESPP_FP32 or ESPP_FP64; seed keys the Philox noise; cuda_stream is
 * a cudaStream_t (NULL = default stream).  On success *out owns all device
 * memory of the system until espp_system_destroy.  Errors: ESPP_ERR_ARG. */
int espp_system_create(const double box[3], int64_t n, const int32_t* types,
                       int64_t n_bonds, const int64_t* bonds, int precision,
                       uint64_t seed, void* cuda_stream, espp_h* out);

/* Create a handle holding R independent replicas (descs[R]), stepped together
 * in one graph-captured launch per step.  Particle arrays of all other calls
 * are the replicas' arrays concatenated in replica order. */
int espp_batch_create(int32_t R, const espp_replica_desc* descs, int precision,
                      void* cuda_stream, espp_h* out);

int espp_system_destroy(espp_h h);

/* ---- state --------------------------------------------------------------- */

/* Set positions x (n*3; wrapped into the box, crossings added to the image
 * counters), velocities v (n*3 or NULL = zero) and image counters img (n*3 or
 * NULL = zero), in id order, from host or device memory (where).  Marks the
 * neighbour list and the stored force stale.  A non-finite position or
 * velocity fails the call with ESPP_ERR_ARG and leaves the handle without a
 * state.  Paper "Example usage": addParticles(pos, v). */
int espp_set_state(espp_h h, const double* x, const double* v, const int32_t* img, int where);

/* Read positions (wrapped into [0,L)), velocities and image counters in id
 * order into caller buffers (each may be NULL).  Synchronises the stream.
 * Errors: ESPP_ERR_STATE (no state set), ESPP_ERR_ARG (where is neither
 * ESPP_HOST nor ESPP_DEVICE). */
int espp_get_state(espp_h h, double* x, double* v, int32_t* img, int where);

/* Set the step number of the state (keys the Philox noise counter).  The
 * simulated time of the handle is kept: it now belongs to this step. */
int espp_set_step(espp_h h, int64_t step);

/* ---- interactions -------------------------------------------------------- */

/* Paper "Software design" (VerletListInteractionTemplate<Potential>,
 * setPotential(type1, type2, potential)) and "Example usage"
 * (LennardJones(eps, sigma, rc, shift='auto'), LennardJonesCapped(...,
 * caprad)).  kind = ESPP_LJ | ESPP_WCA | ESPP_LJ_CAPPED | ESPP_NONE sets the
 * pair potential of types (type_a, type_b) and (type_b, type_a); kind =
 * ESPP_FENE sets the bond potential of every bond (types ignored).  params as
 * listed beside the kinds; shift = 1 lowers the energy by U(rc).  The cutoff
 * of every pair must not exceed the list cutoff of espp_build_neighbors.
 * Tabulated kinds (paper "Functionality": tabulated potentials) take the
 * energy u and the force F = -dU/dr on a uniform grid from r = 0 and
 * interpolate both linearly in r; a tabulated bond longer than rmax is an
 * error like a stretched FENE bond.  Marks the stored force stale.
 * Errors (ESPP_ERR_ARG, the handle unchanged): an unknown kind, a type outside
 * [0, ESPP_MAX_TYPES), too few or non-finite parameters, sigma, rc, caprad,
 * K or R0 not positive, a malformed table. */
int espp_set_interaction(espp_h h, int kind, int type_a, int type_b, const double* params,
                         int64_t n_params);

/* Learned coarse-grained pair potential (a learned CG model; the paper's
 * "tabulated potentials" are its fallback).  u(r) = w3 . silu(W2
 * silu(W1 phi(r) + b1) + b2) + b3 with 32 Gaussian radial bases phi_k(r) =
 * exp(-(r - mu_k)^2 / (2 w^2)) (cos(pi r / rc) + 1) / 2, mu_k = rc k / 31,
 * w = rc / 31.  Weights: bf16[ESPP_MLP_NPARAMS] bit patterns in the order W1
 * (64x32, rows = output units), b1 (64), W2 (64x64), b2 (64), w3 (64), b3.
 * On an FP32 handle it is evaluated on the tensor cores (BF16 operands:
 * the radial features and first-layer activations are rounded to BF16; FP32
 * accumulation) with the force from the exact derivative carried through
 * both layers.  On an FP64 handle the same network (the same BF16 weights)
 * is evaluated in double on the CUDA cores, with no rounding to BF16, as the
 * reference for the tensor-core path; it is much slower.  Select it
 * with espp_set_interaction(h, ESPP_MLP, 0, 0, {rc}, 1) on a single-type
 * system.  ESPP_ERR_ARG for n != ESPP_MLP_NPARAMS or a NaN or infinity
 * pattern among the weights. */
#define ESPP_MLP_NPARAMS 6337
int espp_mlp_set_weights(espp_h h, const uint16_t* bf16, int64_t n);

/* Coarse-graining map for learned-CG training data: site k is the centre of
 * mass of beads [b k, b k + b) (b = beads_per_site, consecutive ids; equal
 * masses) of the unwrapped positions, wrapped into replica 0's box, and its
 * force is the sum of the beads' conservative forces.  x_sites, f_sites:
 * device arrays of (n / b) x 3 doubles.  Synchronises. */
int espp_cg_map(espp_h h, int32_t beads_per_site, double* x_sites, double* f_sites);

/* Current learned-potential weights (BF16 bit patterns, ESPP_MLP_NPARAMS). */
int espp_mlp_get_weights(espp_h h, uint16_t* bf16, int64_t n);

/* Force-matching training of the learned potential (the learned CG model):
 * frames_x and frames_f are device arrays of nframes x n x 3 doubles
 * in id order, the site positions and the target forces for the pair
 * potential (the mapped forces minus the bonded forces of this handle's bond
 * potential).  Loss = mean over frames and sites of |F_pair + F_bond -
 * F_target|^2.  Each epoch visits the frames in an order shuffled by
 * shuffle_seed (splitmix64 Fisher-Yates) in batches of batch_frames; per
 * batch the gradient is computed on the tensor cores (BF16 operands, FP32
 * accumulation, deterministic reduction) and Adam (beta 0.9, 0.999, eps 1e-8,
 * step lr) updates FP32 master weights whose BF16 rounding becomes the
 * handle's weights.  loss_history[epochs] (host) receives the mean loss of
 * each epoch (computed before each batch's update).  The handle's positions
 * are overwritten. */
int espp_mlp_train(espp_h h, const double* frames_x, const double* frames_f, int32_t nframes,
                   int32_t batch_frames, int32_t epochs, double lr, uint64_t shuffle_seed,
                   double* loss_history);

/* The loss and its gradient for the current weights over all frames, without
 * updating them: loss (host, 1 value) and grad (host, ESPP_MLP_NPARAMS - 1
 * floats, the parameter order of the weights without b3). */
int espp_mlp_loss_grad(espp_h h, const double* frames_x, const double* frames_f, int32_t nframes,
                       double* loss, float* grad);

/* Leave 1-2 bonded pairs out of the Verlet list (and so out of every pair
 * potential); default off, as Kremer-Grest keeps WCA between bonded beads. */
int espp_set_exclude_bonded(espp_h h, int on);

/* Per-type mass (default 1 for every type).  ESPP_ERR_ARG unless the type is
 * in range and the mass finite and positive. */
int espp_set_mass(espp_h h, int type, double mass);

/* ---- neighbour list ------------------------------------------------------ */

/* Paper "Example usage": VerletList(system, cutoff=rc) with system.skin.
 * Sets the list cutoff rc and skin and builds the cell grid (cells of edge
 * >= rc + skin, at least 3 per box edge, else ESPP_ERR_BOX_TOO_SMALL), then
 * bins, resorts and builds the Verlet list of every replica now.  Later
 * rebuilds happen automatically when a particle has moved more than skin/2
 * since the last build.  ESPP_ERR_ARG for rc <= 0, skin < 0, non-finite
 * values or a pair cutoff above rc; that refusal keeps the earlier cutoff,
 * skin, grid and list. */
int espp_build_neighbors(espp_h h, double rc, double skin);

/* Tests: the current Verlet list as CSR in id order (global ids).  row_ptr has
 * n+1 entries; cols has room for cap entries.  Returns ESPP_ERR_ARG if cap is
 * too small (row_ptr[n] then holds the size needed). */
int espp_get_neighbors(espp_h h, int64_t* row_ptr, int64_t* cols, int64_t cap);

/* ---- forces and dynamics -------------------------------------------------- */

/* Conservative forces (pairs + bonds, no thermostat) at the current
 * positions, rebuilding the list first when it is stale.  f_out: n*3 doubles
 * in id order (host or device, where), or NULL.  The integrator's stored
 * force is not changed.  Errors: ESPP_ERR_STATE (no state, no list cutoff,
 * the learned potential without weights), ESPP_ERR_ARG (a pair cutoff above
 * the list cutoff, a bad where), ESPP_ERR_LIST_OVERFLOW, ESPP_ERR_BOND_BROKEN. */
int espp_compute_forces(espp_h h, double* f_out, int where);

/* Thermostat of espp_integrate (paper "Functionality": Langevin dynamics and
 * dissipative particle dynamics).  ESPP_THERMO_LANGEVIN (default; rc
 * ignored): per particle, as described at espp_integrate.  ESPP_THERMO_DPD:
 * per pair at distance r < rc (r_ij = x_i - x_j, e = r_ij / r,
 * v_ij = v_i - v_j, w = 1 - r / rc):
 *   F_i += [-gamma w^2 (e . v_ij) + sqrt(2 gamma kT) w theta_ij / sqrt(dt)] e,
 * theta_ij = sqrt(12) u, u uniform in (-1/2, 1/2) from Philox4x32-10 with key
 * (seed lo, seed hi) and counter (min id, max id | 2^31, step lo, step hi), so
 * theta_ij = theta_ji and total momentum is conserved.  The velocities are
 * those present at the force evaluation; ids are the particle ids within the
 * replica and seed the replica's seed.  The pairs are those of the Verlet
 * list: bonded pairs removed by espp_set_exclude_bonded get no DPD force.
 * rc must not exceed the list cutoff
 * of espp_build_neighbors (checked by espp_integrate: ESPP_ERR_ARG).  The
 * stored force becomes stale.  ESPP_ERR_ARG for an unknown kind or rc <= 0. */
#define ESPP_THERMO_LANGEVIN 0
#define ESPP_THERMO_DPD 1
int espp_set_thermostat(espp_h h, int32_t kind, double rc);

/* Pair-force method (paper "Performance optimizations": Verlet lists with a
 * skin, and linked cells with the sub-cell decomposition of Yao et al.).
 * ESPP_FORCES_VERLET (default): the Verlet list of espp_build_neighbors,
 * rebuilt when a particle moved more than skin/2.  ESPP_FORCES_CELLS: no
 * list; every step bins the particles into cells of edge rc / w (rc of
 * espp_build_neighbors; the skin is not used) and sums the pair forces (and
 * the DPD pair term) over the cell stencil; pays off where a list would be
 * rebuilt every step or two.  Both give the same forces up to rounding order.
 * espp_get_neighbors is unavailable, and espp_rdf_counts uses all pairs, in
 * the cell mode.  The cells are rebuilt for the new method.  Errors:
 * ESPP_ERR_ARG (unknown method), ESPP_ERR_STATE (the cell mode with the
 * learned potential). */
#define ESPP_FORCES_VERLET 0
#define ESPP_FORCES_CELLS 1
int espp_set_force_method(espp_h h, int32_t method);
/* How the Verlet build stores a particle's hits (a tuning knob; the list, its
 * order included, is the same either way): ESPP_LIST_STORE_PLACE (default)
 * writes each hit at its place in a 4-entry group held in registers,
 * ESPP_LIST_STORE_PUSH pushes it in at the group's end (the others move down
 * one place), which saves the per-place select on builds with many hits per
 * candidate.  Taken by builds over whole and third cells; half cells always
 * place.  Takes effect at the next list build.  ESPP_ERR_ARG for another
 * value. */
#define ESPP_LIST_STORE_PLACE 0
#define ESPP_LIST_STORE_PUSH 1
int espp_set_list_store(espp_h h, int32_t push);
/* Autotuner of the force path's shape: times nsteps integrate steps (dt,
 * gamma, kT) from the current state with each of ESPP_FORCE_SHAPES shapes,
 * 0 = the Verlet list over whole cells, 1 = the Verlet list over half cells
 * (subdivision 2), 2 = the Verlet list over third cells (subdivision 3), 3 =
 * the list-free cell forces over whole cells, 4 and 5 = shapes 0 and 2 with
 * ESPP_LIST_STORE_PUSH (the others place); restores the state (as
 * espp_set_state would, plus the step and simulated time) and keeps the
 * fastest shape (method, subdivision and list store).
 * ms_per_step[ESPP_FORCE_SHAPES] (may be NULL) receives the times (INFINITY
 * for a shape whose cells do not fit the box), *chosen (may be NULL) the
 * shape kept.  Synchronises. */
#define ESPP_FORCE_SHAPES 6
int espp_tune_force_method(espp_h h, int32_t nsteps, double dt, double gamma, double kT, double* ms_per_step,
                           int32_t* chosen);

/* Autotuner of the step kernel's launch shape and of the storage resort
 * (the batching pattern's "tile and list shapes picked by an autotuner"; the
 * paper's "Performance optimizations" name data sorting).  Shapes of the
 * FP32 step kernel on the plain list path (one particle type, Lennard-Jones,
 * no Lees-Edwards or DPD), as (int4 list groups per batch, resident blocks per
 * SM the registers are fitted to, 128-particle tiles per block): 0 = (1, 8,
 * 1) (the default), 1 = (2, 8, 1), 2 = (1, 12, 1), 3 = (1, 10, 1), 4 = (1, 5,
 * 2), 5 = (1, 3, 3), 6 = (1, 2, 4), 7 = (1, 2, 5).  Every shape computes the
 * same forces bit for bit; they differ in speed only.  espp_set_step_shape selects one (ESPP_ERR_ARG outside
 * [0, ESPP_STEP_SHAPES)).  espp_tune_step_shape times nsteps integrate steps
 * (dt, gamma, kT) from the current state with each shape, keeps the fastest,
 * then times max(nsteps, 1000) steps with each resort interval of 250, 500
 * and 1000 steps and keeps the fastest; it restores the state (as
 * espp_tune_force_method does).  ms_per_step[ESPP_STEP_SHAPES + 3] (may be
 * NULL) receives the times (shapes, then intervals), chosen[2] (may be NULL)
 * the shape and the interval kept.  Synchronises. */
#define ESPP_STEP_SHAPES 8
int espp_set_step_shape(espp_h h, int32_t shape);
int espp_tune_step_shape(espp_h h, int32_t nsteps, double dt, double gamma, double kT, double* ms_per_step,
                         int32_t* chosen);

/* Lees-Edwards boundary conditions (paper "State of the field" and "New
 * features": Lees-Edwards): steady shear with the flow along x and the
 * gradient along z at shear rate gdot (shear_rate).  The periodic image of a
 * replica's box at z + k Lz is displaced by k delta(t) along x and moves at
 * k gdot Lz along x, delta(t) = gdot Lz t, where t is the simulated time of
 * the handle (`time` sets t at the current step; every integrate step adds
 * its dt).  A particle crossing a z face by k boxes is moved by -k delta
 * along x and its v_x by -k gdot Lz; image counters count the wraps, so
 * x + img_x Lx + img_z delta(t) is the continuous unwrapped x.  Pair and bond
 * vectors take the sheared minimum image; the Langevin friction acts on
 * v - gdot (z - Lz/2) x; DPD relative velocities include the image velocity.
 * on = 0 restores the plain periodic box (time is kept).  Positions given to
 * espp_set_state must lie inside the box along z.  The list is rebuilt on
 * the next call; the change of delta since a build counts against the skin.
 * Errors: ESPP_ERR_ARG (non-finite values), ESPP_ERR_STATE (with the learned
 * potential or the CG mapping, which are not available under shear). */
int espp_set_lees_edwards(espp_h h, int32_t on, double shear_rate, double time);
/* Current setting and simulated time t of the handle (any pointer may be
 * NULL). */
int espp_get_lees_edwards(espp_h h, int32_t* on, double* shear_rate, double* time);

/* Paper "Example usage": VelocityVerlet + LangevinThermostat(gamma,
 * temperature) and integrator.run(nsteps).  Each step: v += dt/2 F/m;
 * x += dt v (wrap); rebuild the list if needed; F = conservative forces
 * - gamma m v + sqrt(24 gamma m kT / dt) r with r uniform in (-1/2, 1/2) from
 * Philox(seed; id, step); v += dt/2 F/m.  gamma = 0 gives plain velocity
 * Verlet.  Steps run as CUDA graphs on the handle's stream; the call returns
 * after the work is issued and checked (it synchronises once at the end).
 * Errors: ESPP_ERR_ARG (nsteps < 0, dt not finite and positive, gamma or kT
 * negative or not finite), ESPP_ERR_STATE (no state or list),
 * ESPP_ERR_BOND_BROKEN, ESPP_ERR_NONFINITE, ESPP_ERR_LIST_OVERFLOW. */
int espp_integrate(espp_h h, int64_t nsteps, double dt, double gamma, double kT);

/* Paper "Example usage": computeEnergy().  Observables of replica 0 (or of
 * the first R replicas into out[R] with espp_observables_batch; out is host
 * memory owned by the caller).  Synchronises.  Errors: ESPP_ERR_ARG (null out,
 * R outside [1, replica count]), ESPP_ERR_STATE (no state set), the errors of
 * a list rebuild the call may need (ESPP_ERR_LIST_OVERFLOW, ESPP_ERR_NONFINITE). */
int espp_observables(espp_h h, espp_obs_t* out);
int espp_observables_batch(espp_h h, espp_obs_t* out, int32_t R);

/* Unique-pair distance histogram of replica `replica` for r < rmax in nbins
 * equal bins (counts[nbins], host).  rmax must be below half the smallest
 * box edge.  Pairs come from the Verlet list when rmax <= rc + skin (with 1-2
 * exclusions on, bonded pairs are then not counted), else from all pairs of
 * the replica (limited to 200000 particles).  Errors: ESPP_ERR_ARG (replica
 * out of range, nbins outside [1, 12288], rmax not in (0, half the smallest
 * edge), null counts, an all-pairs histogram above the particle limit),
 * ESPP_ERR_STATE
 * (no state set). */
int espp_rdf_counts(espp_h h, int32_t replica, double rmax, int32_t nbins, int64_t* counts);

/* ---- checkpoint ------------------------------------------------------------ */

/* Paper "New features": checkpoint of the state and of the random number
 * generator.  The Philox noise is a pure function of (seed, id, step), so the
 * file holds the full internal state (storage order, positions at the last
 * list build, velocities, force, image counters, step, per-replica seeds and
 * pending rebuild requests, the Lees-Edwards setting, clock and build
 * offsets) and a resumed run is bit-identical to an uninterrupted one.  The
 * configuration is not in the file: interactions, masses, thermostat, force
 * method and list cutoff are set on the loading handle as on the saving one.
 * path: a NUL-terminated file name, written or read with stdio.
 * Save errors: ESPP_ERR_ARG (null path), ESPP_ERR_STATE (no state set),
 * ESPP_ERR_IO (open or write failed), the run's own error if the last step
 * failed.  Load needs espp_build_neighbors first (ESPP_ERR_STATE) and a handle
 * of the same precision, replica count, sizes and boxes (ESPP_ERR_ARG);
 * ESPP_ERR_IO for a file that cannot be opened, is not a checkpoint or is
 * truncated; ESPP_ERR_LIST_OVERFLOW if the saved list does not fit.  A load
 * that fails before the upload leaves the handle unchanged. */
int espp_checkpoint_save(espp_h h, const char* path);
int espp_checkpoint_load(espp_h h, const char* path);

/* Paper "New features": H5MD output and the checkpoint of the random number
 * generator.  espp_h5md_write writes the handle's state as an H5MD 1.1 file
 * (HDF5 format; no HDF5 library is used): /h5md (version 1.1, author,
 * creator), per replica /particles/<g>/{box (dimension 3, periodic
 * boundary, edges), position, velocity, image, force (one frame each: step,
 * time, value [1][n][3]), species [n]}, /connectivity/<g>/bonds [n_bonds][2] and
 * /parameters/espp (step, simulated time, precision, Lees-Edwards setting,
 * the replicas' Philox seeds [R]); <g> = "all" for a single system,
 * "replica_<r>" for a batch.  Particle data are in id order, positions
 * wrapped into the box with their image counters; force is the total force
 * the next velocity-Verlet step starts from (thermostat terms included),
 * written once the handle has one (after an integrate call).  Because the Philox noise
 * is a function of (seed, id, step), the seeds and the step restore the
 * random stream.  espp_h5md_read loads such a file into a handle of the same
 * replicas, sizes, boxes, types and Lees-Edwards setting (ESPP_ERR_ARG
 * otherwise, the handle unchanged): it takes the file's Philox seeds, step
 * and simulated time, then the positions, velocities and images as
 * espp_set_state does, and the force where the file holds one; the
 * interactions, thermostat and list are those of the loading handle.  A run resumed from it continues the same trajectory up to
 * rounding (the binary espp_checkpoint_* files resume bit for bit).  It reads
 * the HDF5 subset the writer produces (version-2 superblock and object
 * headers, compact groups, contiguous datasets) and refuses other files with
 * ESPP_ERR_IO, as it does a file that cannot be opened or fails a checksum.
 * Errors: ESPP_ERR_ARG (null path, a mismatched handle), ESPP_ERR_STATE
 * (write without a state), ESPP_ERR_IO. */
int espp_h5md_write(espp_h h, const char* path);
int espp_h5md_read(espp_h h, const char* path);
/* What an H5MD file written by espp_h5md_write holds, without a handle (host
 * code only; no GPU is touched): the number of replicas, their particles in
 * total, the step and the precision of the handle that wrote it.  The file is
 * parsed and checked as espp_h5md_read does (every checksum, every address
 * and length against the file's size, each object reached once, every
 * particle array of the size its shape says).  Any output pointer may be NULL.
 * Errors: ESPP_ERR_ARG (null path), ESPP_ERR_IO (a file that cannot be opened
 * or is refused); the message is espp_last_error(NULL). */
int espp_h5md_inspect(const char* path, int32_t* n_replicas, int64_t* n_particles, int64_t* step,
                      int32_t* precision);

/* ---- diagnostics ----------------------------------------------------------- */
const char* espp_last_error(espp_h h);
uint32_t espp_error_word(espp_h h);
int64_t espp_num_particles(espp_h h);
int32_t espp_num_replicas(espp_h h);
int64_t espp_num_rebuilds(espp_h h);
int64_t espp_step(espp_h h);
int32_t espp_list_capacity(espp_h h);
/* Number of kernel launches issued through this handle (graph replays count
 * every kernel node they hold once per replay; conditional bodies as run). */
int64_t espp_kernel_launches(espp_h h);

/* Kernel timing.  With timing enabled (espp_set_kernel_timing(h, 1)), the
 * CUDA graphs of espp_integrate record CUDA events around the conditional
 * rebuild node and the step kernel of every step; after each espp_integrate
 * call the durations of the last graph replay are added up.  out[4] receives
 * (sum of step-kernel ms, number of step-kernel launches timed, sum of
 * rebuild-node ms, number of steps timed); reset = 1 clears the sums.
 * Graphs with and without the timing events are cached side by side, so
 * switching does not rebuild them after the first use of each. */
int espp_set_kernel_timing(espp_h h, int enable);
int espp_kernel_timing(espp_h h, double* out, int reset);

/* Size of the current Verlet list: total entries over all particles and the
 * largest per-particle count (rebuilds first if the list is stale). */
int espp_list_stats(espp_h h, int64_t* total_entries, int32_t* max_count);

/* Steps between Hilbert resorts of the particle storage inside
 * espp_integrate (default 500; 0 = only on explicit builds).  A resort happens
 * before every step whose number is a multiple of the interval, so results do
 * not depend on how a run is split into calls. */
int espp_set_resort_interval(espp_h h, int64_t steps);

/* Cell sub-decomposition for the Verlet build (paper "Performance
 * optimizations": cells of rc/2 or rc/3 cut the volume searched per
 * particle).  w = 1: cells of edge >= rc + skin and a 3x3x3 stencil; w = 2
 * or 3: cells of edge >= (rc + skin) / w and a (2w+1)^3 stencil, each row of
 * it searched only over the cells the list sphere reaches; w = 0 (default):
 * chosen at each espp_build_neighbors, 2 when a full cell holds ten or more
 * particles on average (and every edge holds 5 half cells), else 1.  w needs
 * 2w + 1 cells along every edge of every replica (ESPP_ERR_BOX_TOO_SMALL
 * otherwise).  The list itself (its set of pairs) does not depend on w.  The
 * list-free mode (ESPP_FORCES_CELLS) takes w <= 2.  Takes effect at once when
 * a grid exists (the list is rebuilt), else at the next espp_build_neighbors.
 * ESPP_ERR_ARG unless 0 <= w <= 3, or for w = 3 in the list-free mode. */
int espp_set_cell_subdivision(espp_h h, int32_t w);

/* Steps captured per CUDA graph replay in espp_integrate (default 64).  0
 * launches every kernel directly instead (no graphs; for profilers, which do
 * not see kernels inside conditional graphs). */
int espp_set_graph_chunk(espp_h h, int32_t steps);

/* Tests: fill out[n*3] (device) with the Langevin noise of local ids [0,n) at
 * `step` under `seed`, as the force kernel draws it. */
int espp_langevin_noise(uint64_t seed, int64_t step, int64_t n, double* out_device,
                        void* cuda_stream);

/* Pair-distance histogram that allocates nothing.  The paper has no
 * counterpart: this entry point exists for callers that cannot call
 * cudaMalloc -- code inside a framework that reserved the device memory up
 * front and hands out only its own pool, or latency-critical loops that cannot
 * take the implicit synchronisation of cudaMalloc/cudaFree.
 *
 * Counts every unique pair i < j of the n positions whose plain periodic
 * minimum-image distance is r < rmax, in bin floor(r nbins / rmax): all
 * pairs, bonded ones included, with no Lees-Edwards offset.  That equals
 * espp_rdf_counts only where the handle path also counts all pairs of a
 * plain periodic box (rmax above the list radius, no shear); below the list
 * radius the handle path counts from the Verlet list, which leaves out
 * excluded bonded pairs.  Positions: caller-owned device memory x_device
 * (n*3 doubles, id order, each coordinate in [0, box) as espp_get_state
 * returns them); counts: caller-owned device memory counts_device[nbins]
 * (int64).  Work is queued on cuda_stream; the call does not wait for it.
 *
 * Working memory is a fixed file-scope device array of ESPP_NOALLOC_MAX_BINS
 * counters (32 KiB) inside the library; every GPU that loads the library holds
 * it until the process exits.  The first call on a device looks up the array's
 * device address (cudaGetSymbolAddress) with that device current; make that
 * first call before any stream capture, and do not reset the device
 * (cudaDeviceReset) while the library stays loaded, since the looked-up
 * address is kept.  All calls share the one array: each call clears the part
 * it uses, and calls whose work overlaps on the GPU (for instance on two
 * streams) race on it.  Errors (all checked on the host before any GPU work,
 * counts_device then untouched): ESPP_ERR_ARG for nbins outside
 * [1, ESPP_NOALLOC_MAX_BINS], n outside [0, ESPP_NOALLOC_MAX_N] (the kernel is
 * O(n^2)), rmax not in (0, half of every box edge), a box edge not positive,
 * or a null pointer; ESPP_ERR_CUDA if a launch fails.  Never calls
 * cudaMalloc, cudaFree or any allocating routine. */
#define ESPP_NOALLOC_MAX_BINS 4096
#define ESPP_NOALLOC_MAX_N 200000
int espp_rdf_counts_noalloc(const double* x_device, int64_t n, const double box[3], double rmax,
                            int32_t nbins, int64_t* counts_device, void* cuda_stream);

/* Host-side helper (no GPU work): the 3-D Hilbert-curve rank of each cell of an
 * nx x ny x nz grid (rank[cz*ny*nx + cy*nx + cx]), as used for the storage
 * order.  Returns ESPP_OK. */
int espp_hilbert_ranks(int32_t nx, int32_t ny, int32_t nz, int32_t* rank);

#ifdef __cplusplus
}
#endif
#endif /* ESPP_H */

// Device view of one handle and the host-side launchers of every kernel.
#pragma once
#include <cuda_bf16.h>

#include "common.cuh"

namespace espp {

// Integrator parameters, resident in device memory so captured graphs stay
// valid when they change.
template <class T> struct IntParams {
    T dt;
    T half_dt;
    T gamma;
    T kT;
    T mass[MAX_TYPES];
    T inv_mass[MAX_TYPES];
    T noise_amp[MAX_TYPES];  // sqrt(24 gamma m kT / dt)
    T dpd_rc2;               // DPD thermostat: cutoff^2, 1 / cutoff,
    T dpd_inv_rc;
    T dpd_amp;               // sqrt(2 gamma kT) sqrt(12) / sqrt(dt) (times w u gives the random force)
};

// Learned pair potential: 32 radial bases -> 64 -> 64 -> 1 (SiLU), weights
// in BF16 (W1 row-major 64x32, W2 64x64, rows = output units), biases and the
// output layer as the BF16 values in float.
constexpr int MLP_NB = 32;
constexpr int MLP_H = 64;
constexpr int MLP_NPARAMS = MLP_H * MLP_NB + MLP_H + MLP_H * MLP_H + MLP_H + MLP_H + 1;
struct MlpWeights {
    __nv_bfloat16 W1[MLP_H * MLP_NB];
    __nv_bfloat16 W2[MLP_H * MLP_H];
    float b1[MLP_H];
    float b2[MLP_H];
    float w3[MLP_H];
    float b3;
    float rc;
};

constexpr int NPART = 12;  // per-tile observable partials (doubles)
enum : int {
    P_PE_PAIR = 0, P_PE_BOND, P_VIRIAL, P_KE, P_BOND_LEN, P_BOND_CNT, P_PX, P_PY, P_PZ,
    P_VIR_XZ,  // sum over pairs and bonds of (r_ij)_x (F_ij)_z
    P_KIN_XZ,  // sum of m v_x v_z (velocities relative to the shear profile)
};

// Lees-Edwards clock in device memory: the simulated time of step s is
// t0 + (s - s0) dt (rewritten by the host before each integrate call, so
// captured graphs need no update).
struct LeClock {
    double t0;
    double dt;
    long long s0;
    long long pad;
};

template <class T> struct DevSys {
    // particle arrays in storage (cell-sorted) order, all replicas concatenated
    V4<T>* pos[2];      // double-buffered positions; w = type bits
    V4<T>* vel;         // w = local particle id bits
    V4<T>* vel_alt;
    V4<T>* frc;         // total force of the stored step
    V4<T>* frc_alt;
    V4<T>* xb;          // positions at the last list build
    int4* img;          // periodic image counters
    int4* img_alt;
    int2* bond_slot;    // storage slots of the (<= 2) bond partners, -1 = none
    const int2* bond_gid;  // by global id: global ids of bond partners, -1 = none
    int* slot_of_id;    // global id -> storage slot
    int* perm;          // new slot -> old slot (rebuild)
    int* cellh;         // per old slot: global cell rank
    int* in_cell;       // per old slot: arrival index in its cell
    // Verlet list in groups of four: entry k of particle i sits at
    // nbr[4 * ((k / 4) * stride + i) + k % 4]; k < nbr_cnt[i] <= cap; the last
    // group is padded with nbr_pad, the slot after the last particle, whose
    // position (in both position buffers) lies far outside every box, so a
    // padding entry is a pair beyond every cutoff
    int* nbr;
    int* nbr_cnt;
    int cap;
    int stride;
    int nbr_pad;
    // cells, all replicas concatenated; cell index cell_off + (cz * ny + cy) * nx + cx
    int* cell_cnt;
    // compact entries (position, storage slot in the w lane): those of cell h
    // are cell_ent[cell_beg[h] .. cell_beg[h + 1]), ascending slot
    V4<T>* cell_ent;
    int* cell_beg;          // ncells + 1; cell_beg[ncells] = N
    int* rank_start;        // first new slot of each cell in Hilbert-rank order (resort only)
    int cell_w;             // cell subdivision: cells of edge >= (rc + skin) / cell_w (1, 2 or 3)
    int list_push;          // Verlet build: hits pushed into the list group (1) or placed (0)
    const int* cell_by_rank;  // global Hilbert rank -> cell index
    const int* cell_rep;
    int ncells;
    int* scan_part;
    int nscan_blocks;
    // replicas and tiles
    const RepGeom<T>* reps;
    int R;
    const Tile* tiles;
    int ntiles;
    const int* rep_tile_off;  // R + 1: first tile of each replica
    int* req;           // rebuild requested (per replica), set by the step kernel
    int* now;           // rebuild running (per replica), latched at the rebuild start
    Ctrl* ctrl;
    const IntParams<T>* ip;
    const PairRec<T>* pair;
    const T* tab;       // concatenated tables (tabulated pair and bond kinds)
    int ntypes;
    int lj_fast;        // one particle type with a plain Lennard-Jones pair potential
    int step_shape;     // launch shape of the FP32 step kernel on the plain list path (autotuned)
    int mlp_on;         // pair forces come from the learned MLP (k_mlp) instead
    int excl_bonded;    // 1-2 bonded pairs are left out of the Verlet list
    const MlpWeights* mlp;
    float4* mlp_f;      // per particle: MLP pair force and sum of pair energies
    float* mlp_w;       // per particle: sum of r_ij . F_ij over its MLP pairs
    V4<T>* mlp_fT;      // FP64 handles: the same two sums in double (k_mlp_f64)
    T* mlp_wT;
    // per list entry (layout of nbr): -du/dr / r, u, and for entries (i, j)
    // with j > i the index of the mirrored entry (j, i)
    float* mlp_pf;
    float* mlp_pu;
    int* mlp_rev;
    int4* mlp_pairs;    // dense pairs inside the cutoff: (r bits, entry, mirrored entry, -)
    int mlp_pairs_cap;
    int* mlp_npairs;    // device counter of mlp_pairs
    int4* mlp_upper;    // every unordered list pair: (entry, mirrored entry, list entry, replica)
    int mlp_upper_cap;
    int* mlp_nupper;    // number of records in mlp_upper
    int* mlp_ucount;    // per particle: its list entries (i, j) with j > i
    int* mlp_uoff;      // per particle: first record in mlp_upper (scan of mlp_ucount)
    int* mlp_uscan_part;
    int mlp_nuscan;     // scan blocks over the particles
    int dpd;            // DPD thermostat instead of Langevin (integration modes)
    // list-free mode: particles binned every step, pair forces (with the DPD
    // pair term) from the cell stencil into cpf / cpv, read by the step kernel
    int cells_mode;
    V4<T>* cpf;         // per slot: pair force and pair energy
    V4<T>* cpv;         // per slot: pair virial and its xz part (energy pass)
    V4<T>* cell_vel;    // velocities in cell-entry order (with DPD), written at binning
    V4<T>* vsnap;       // DPD: velocities at the force evaluation, read for the neighbours
    int tc_fault;       // host fault injection: the tensor-core kernel issues no MMA and
                        // its bounded mbarrier wait runs out (tests of the timeout path)
    // Lees-Edwards boundary conditions: flow along x, gradient along z; the
    // image at z + k Lz is displaced by k delta(t) along x and moves at
    // k le_shear Lz, delta(t) = le_shear Lz t.  List entries of pairs across
    // the sheared faces carry x code 3 (x image taken at evaluation time).
    int le_on;
    double le_shear;
    const LeClock* le_clk;
    double* le_db;      // per replica: delta at the last list build (not reduced)
    int N;
    BondRec<T> bond;
    T rlist2;           // (rc + skin)^2
    T half_skin2;       // (skin / 2)^2
    T skin;
    double* partials;   // ntiles * NPART
};

// ---- Lees-Edwards helpers ----------------------------------------------------
// offset delta of replica g at step `step`, not reduced
template <class T>
__device__ __forceinline__ double le_offset(const DevSys<T>& s, const RepGeom<T>& g, long long step) {
    const LeClock* c = s.le_clk;
    return s.le_shear * (double)g.L[2] * (c->t0 + (double)(step - c->s0) * c->dt);
}

// d reduced into [0, L)
__device__ __forceinline__ double le_reduce(double d, double L) { return d - L * floor(d / L); }

// x displacement of a pair across the sheared faces: nz = +1 when the partner
// is the image above (z code 1), -1 below (z code 2); delta reduced into
// [0, Lx); the x image is the nearest one.
template <class T>
__device__ __forceinline__ T le_dx(T xi, T xj, int nz, T delta, T Lx, T inv_Lx) {
    T dx = (xi - xj) - (T)nz * delta;
    return dx - Lx * rint(dx * inv_Lx);
}

// Wrap of one position under Lees-Edwards, in double: a crossing of the z
// faces by k boxes moves x by -k delta and v_x by -k le_shear Lz (the image
// the particle entered), then x (possibly several boxes) and y are wrapped.
// k[] receives the image changes.
__device__ __forceinline__ void le_wrap(double p[3], double& vx, int k[3], const double L[3], double delta,
                                        double shear) {
    k[0] = k[1] = k[2] = 0;
    if (p[2] >= L[2]) {
        p[2] -= L[2];
        k[2] = 1;
    } else if (p[2] < 0.0) {
        p[2] += L[2];
        k[2] = -1;
        if (p[2] >= L[2]) {  // less than half an ulp below 0: its own image
            p[2] = 0.0;
            k[2] = 0;
        }
    }
    if (k[2] != 0) {
        p[0] -= k[2] * delta;
        vx -= k[2] * shear * L[2];
        double q = floor(p[0] / L[0]);
        p[0] -= q * L[0];
        if (p[0] >= L[0]) {
            p[0] -= L[0];
            q += 1.0;
        }
        if (p[0] < 0.0) p[0] = 0.0;
        k[0] = (int)q;
    } else if (p[0] >= L[0]) {
        p[0] -= L[0];
        k[0] = 1;
    } else if (p[0] < 0.0) {
        p[0] += L[0];
        k[0] = -1;
        if (p[0] >= L[0]) {
            p[0] = 0.0;
            k[0] = 0;
        }
    }
    if (p[1] >= L[1]) {
        p[1] -= L[1];
        k[1] = 1;
    } else if (p[1] < 0.0) {
        p[1] += L[1];
        k[1] = -1;
        if (p[1] >= L[1]) {
            p[1] = 0.0;
            k[1] = 0;
        }
    }
}

// kernels launched by one rebuild without a resort (Launch::rebuild)
constexpr int REBUILD_LAUNCHES = 8;

// step-kernel modes
enum : int {
    MODE_FORCES = 0,  // conservative forces only, written to an id-ordered double buffer
    MODE_INIT = 1,    // total force of the current step (with thermostat), stored; no kick
    MODE_STEP = 2,    // F_s, v_s, v_{s+1/2}, x_{s+1}
    MODE_FINAL = 3,   // F_s, v_s stored (end of an integrate call)
};

// ---- launchers (defined in the .cu files) ----------------------------------
template <class T> struct Launch {
    // rebuild pipeline on the positions in buffer `cur` (other buffer is
    // scratch); returns the number of kernels launched
    static int rebuild(const DevSys<T>& s, int cur, bool resort, bool permute_force, cudaStream_t st);
    static void request_all(const DevSys<T>& s, cudaStream_t st);
    // step kernels
    // one force evaluation (+ the learned potential's kernels); returns the
    // number of kernels launched
    static int step(const DevSys<T>& s, int mode, bool energy, int cur, double* f_out,
                    unsigned long long next_cond, int grid, cudaStream_t st);
    static void prologue(const DevSys<T>& s, int cur, int grid, cudaStream_t st);
    static void set_cond(const DevSys<T>& s, unsigned long long cond, cudaStream_t st);
    // the learned potential's pair forces: the tensor-core path (FP32 handles)
    // or the network in double (FP64 handles); mlp_tc: the tensor-core path
    // for either precision (per-entry values, as training reads them)
    static int mlp(const DevSys<T>& s, int cur, bool energy, cudaStream_t st);
    static int mlp_tc(const DevSys<T>& s, int cur, bool energy, cudaStream_t st);
    // list-free pair forces from the cell stencil (k_cells.cu)
    static int cellforce(const DevSys<T>& s, int cur, bool energy, bool dpd, cudaStream_t st);
    static int mlp_rev(const DevSys<T>& s, cudaStream_t st);
    // force-matching gradient of one frame (errors, tensor-core gradient,
    // deterministic reduction into grad and the loss)
    static int train_grad(const DevSys<T>& s, int cur, const double* Y, float4* err, double* loss_part,
                          float scale, float* partials, int grad_blocks, float* grad, double* loss,
                          cudaStream_t st);
    static cudaError_t prepare_train();
    // state I/O (id-ordered double buffers on the device)
    static void set_state(const DevSys<T>& s, const double* x, const double* v, const int* img,
                          const int* types_by_gid, int cur, cudaStream_t st);
    // f: the stored total force of the current step (thermostat terms included)
    static void get_state(const DevSys<T>& s, double* x, double* v, int* img, double* f, int cur,
                          cudaStream_t st);
    static void set_force(const DevSys<T>& s, const double* f, cudaStream_t st);
    static void reduce_obs(const DevSys<T>& s, double* out_R_NPART, cudaStream_t st);
    static void rg2(const DevSys<T>& s, int cur, const int* mol_members, const int* mol_off,
                    const int* mol_rep, int nmol, double* mol_rg2, cudaStream_t st);
    static void rdf(const DevSys<T>& s, int cur, int rep, double rmax, int nbins,
                    unsigned long long* counts, cudaStream_t st);
    static void rdf_list(const DevSys<T>& s, int cur, int rep, double rmax, int nbins,
                         unsigned long long* counts, cudaStream_t st);
};

void launch_adam(float* theta, float* m, float* v, float* grad, float lr, float b1, float b2, float eps,
                 int step, MlpWeights* W, cudaStream_t st);
int mlp_ngrad();
// once per process, before the learned potential's first launch
cudaError_t prepare_mlp_tc();

void launch_cg_map(const double* x, const int* img, const double* f, long long nsites, int bps, const double* L,
                   double* xs, double* fs, cudaStream_t st);

void launch_noise(unsigned long long seed, long long step, long long n, double* out,
                  cudaStream_t st);

}  // namespace espp

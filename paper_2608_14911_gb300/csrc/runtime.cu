// Host runtime behind the C ABI (include/espp.h): owns the device buffers of a
// handle, prepares geometry, cell grids, tiles and interaction tables, builds
// and caches the CUDA graphs that step the system, and turns the device error
// word into status codes.  Everything computed per particle runs in the
// kernels of k_rebuild.cu, k_step.cu and k_io.cu.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <memory>
#include <numeric>
#include <string>
#include <tuple>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "h5md.h"
#include "kernels.cuh"

namespace espp {

// NVTX range over a host call (shown by ncu's --nvtx filters and by
// timeline profilers; a no-op unless a tool is attached)
struct NvtxRange {
    explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange&) = delete;
    NvtxRange& operator=(const NvtxRange&) = delete;
};

void hilbert_ranks(int nx, int ny, int nz, int* rank);
int scan_blocks_for(int ncells);

#define CK(call)                                                                       \
    do {                                                                               \
        cudaError_t e_ = (call);                                                       \
        if (e_ != cudaSuccess) {                                                       \
            return fail(ESPP_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
        }                                                                              \
    } while (0)

struct SystemBase {
    std::string msg;
    virtual ~SystemBase() {}
    int fail(int code, const std::string& m) {
        msg = m;
        return code;
    }
    virtual int set_state(const double* x, const double* v, const int32_t* img, int where) = 0;
    virtual int get_state(double* x, double* v, int32_t* img, int where) = 0;
    virtual int set_step(int64_t step) = 0;
    virtual int set_interaction(int kind, int ta, int tb, const double* p, int64_t np) = 0;
    virtual int set_mass(int type, double m) = 0;
    virtual int mlp_set_weights(const uint16_t* bits, int64_t n) = 0;
    virtual int set_exclude_bonded(int on) = 0;
    virtual int mlp_get_weights(uint16_t* out, int64_t n) = 0;
    virtual int cg_map(int bps, double* xs, double* fs) = 0;
    virtual int mlp_train(const double* X, const double* Y, int nframes, int batch, int epochs, double lr,
                          uint64_t seed, double* loss_hist, float* grad_out) = 0;
    virtual int build_neighbors(double rc, double skin) = 0;
    virtual int get_neighbors(int64_t* row_ptr, int64_t* cols, int64_t cap) = 0;
    virtual int compute_forces(double* f, int where) = 0;
    virtual int integrate(int64_t nsteps, double dt, double gamma, double kT) = 0;
    virtual int observables(espp_obs_t* out, int R) = 0;
    virtual int rdf_counts(int rep, double rmax, int nbins, int64_t* counts) = 0;
    virtual int checkpoint_save(const char* path) = 0;
    virtual int checkpoint_load(const char* path) = 0;
    virtual uint32_t error_word() = 0;
    virtual int64_t num_particles() = 0;
    virtual int32_t num_replicas() = 0;
    virtual int64_t num_rebuilds() = 0;
    virtual int64_t step() = 0;
    virtual int32_t list_capacity() = 0;
    virtual int64_t kernel_launches() = 0;
    virtual int set_kernel_timing(int enable) = 0;
    virtual int kernel_timing(double* out, int reset) = 0;
    virtual int set_chunk(int steps) = 0;
    virtual int list_stats(int64_t* total, int32_t* maxc) = 0;
    virtual int set_resort_interval(int64_t steps) = 0;
    virtual int set_cell_subdivision(int w) = 0;
    virtual int set_thermostat(int kind, double rc) = 0;
    virtual int set_lees_edwards(int on, double shear, double time) = 0;
    virtual int get_lees_edwards(int* on, double* shear, double* time) = 0;
    virtual int set_force_method(int method) = 0;
    virtual int tune_force_method(int nsteps, double dt, double gamma, double kT, double* ms, int* chosen) = 0;
    virtual int set_step_shape(int shape) = 0;
    virtual int set_list_store(int push) = 0;
    virtual int h5md_write(const char* path) = 0;
    virtual int h5md_read(const char* path) = 0;
    virtual int tune_step_shape(int nsteps, double dt, double gamma, double kT, double* ms, int* chosen) = 0;
};

struct PairHost {
    int kind = ESPP_NONE;
    double eps = 0, sig = 0, rc = 0, cap = 0;
    bool shift = false;
    std::vector<double> tab;  // tabulated: u[n] then F[n]
};

template <class T>
class System : public SystemBase {
   public:
    cudaStream_t st = nullptr;
    int R = 0;
    int64_t N = 0;
    std::vector<double> box;  // R*3
    std::vector<int> rep_n, rep_poff;
    std::vector<unsigned long long> seeds;
    std::vector<Tile> tiles_h;
    std::vector<int> rep_tile_off_h;
    std::vector<int> types_gid;
    std::vector<int2> bond_gid_h;
    std::vector<int> mol_members_h, mol_off_h, mol_rep_h;
    int ntypes = 1;
    PairHost pair_h[MAX_TYPES][MAX_TYPES];
    int bond_kind = ESPP_NONE;
    double bond_K = 0, bond_R0 = 0;
    std::vector<double> bond_tab;  // tabulated bond: u[n] then F[n] over [0, bond_R0]
    std::vector<uint16_t> mlp_bits;  // learned potential, BF16 bit patterns
    MlpWeights* d_mlp = nullptr;
    void* tab_alloc = nullptr;
    size_t tab_elems = 0;
    double mass_h[MAX_TYPES];
    double rc_list = -1, skin = 0;
    bool cells_ready = false, state_set = false, f_valid = false, rebuild_pending = false;
    int cur = 0;
    std::vector<void*> allocs;
    std::vector<void*> cell_allocs;
    void* nbr_alloc = nullptr;
    void* mlp_buf = nullptr;  // per-entry buffers of the learned potential
    int mlp_buf_cap = 0;
    DevSys<T> d{};
    RepGeom<T>* d_geom = nullptr;
    IntParams<T>* d_ip = nullptr;
    PairRec<T>* d_pair = nullptr;
    Ctrl* d_ctrl = nullptr;
    int* d_types = nullptr;
    double* d_io_x = nullptr;
    double* d_io_v = nullptr;
    int* d_io_img = nullptr;
    double* d_obs = nullptr;
    int *d_mol_members = nullptr, *d_mol_off = nullptr, *d_mol_rep = nullptr;
    double* d_mol_rg2 = nullptr;
    unsigned long long* d_hist = nullptr;
    int hist_cap = 0;
    double ip_key[3] = {-1, -1, -1};
    struct ChunkGraph {
        cudaGraph_t graph = nullptr;
        cudaGraphExec_t exec = nullptr;
        std::vector<cudaEvent_t> ev;  // timing mode: 3 per step (before rebuild, before step, after step)
    };
    // key (steps, first position buffer, final step, timing events)
    std::map<std::tuple<int, int, int, int>, ChunkGraph> graphs;
    bool timing = false;
    double t_step_ms = 0, t_rebuild_ms = 0;
    int64_t t_step_n = 0;
    int64_t launches = 0;
    int chunk = 64;
    int64_t resort_every = 500;  // steps between Hilbert resorts inside integrate (0 = never)
    int cell_sub_req = 0;  // requested cell subdivision (0 = chosen per system)
    double dpd_rc = 0;     // DPD thermostat cutoff (d.dpd set)
    // simulated time t(step) = le_clk_h.t0 + (step - s0) dt, mirrored on the
    // device for the Lees-Edwards offset
    LeClock le_clk_h{0.0, 0.0, 0, 0};
    LeClock* d_le_clk = nullptr;
    int cell_sub = 1;      // subdivision in use (stencil half width)

    ~System() override {
        clear_graphs();
        for (void* p : cell_allocs) cudaFree(p);
        if (nbr_alloc) cudaFree(nbr_alloc);
        if (mlp_buf) cudaFree(mlp_buf);
        if (tab_alloc) cudaFree(tab_alloc);
        if (d_hist) cudaFree(d_hist);
        for (void* p : allocs) cudaFree(p);
    }

    template <class P>
    int alloc(P** out, size_t count, std::vector<void*>& pool) {
        void* p = nullptr;
        if (count == 0) count = 1;
        cudaError_t e = cudaMalloc(&p, count * sizeof(P));
        if (e != cudaSuccess) return fail(ESPP_ERR_CUDA, std::string("cudaMalloc: ") + cudaGetErrorString(e));
        cudaMemset(p, 0, count * sizeof(P));
        pool.push_back(p);
        *out = reinterpret_cast<P*>(p);
        return ESPP_OK;
    }

    void clear_graphs() {
        for (auto& kv : graphs) {
            cudaGraphExecDestroy(kv.second.exec);
            cudaGraphDestroy(kv.second.graph);
            for (cudaEvent_t e : kv.second.ev) cudaEventDestroy(e);
        }
        graphs.clear();
    }

    // ---------------------------------------------------------------- create
    int create(int Rr, const espp_replica_desc* descs, cudaStream_t stream) {
        st = stream;
        R = Rr;
        for (int a = 0; a < MAX_TYPES; ++a) mass_h[a] = 1.0;
        int64_t total = 0;
        for (int r = 0; r < R; ++r) {
            const espp_replica_desc& dsc = descs[r];
            if (dsc.n < 1) return fail(ESPP_ERR_ARG, "every replica needs at least one particle");
            for (int c = 0; c < 3; ++c)
                if (!(dsc.box[c] > 0) || !std::isfinite(dsc.box[c]))
                    return fail(ESPP_ERR_ARG, "box edges must be positive and finite");
            rep_poff.push_back((int)total);
            rep_n.push_back((int)dsc.n);
            total += dsc.n;
            if (total >= MAX_PARTICLES) return fail(ESPP_ERR_ARG, "too many particles (at most 2^25 per handle)");
            for (int c = 0; c < 3; ++c) box.push_back(dsc.box[c]);
            seeds.push_back(dsc.seed);
        }
        N = total;
        types_gid.assign(N, 0);
        bond_gid_h.assign(N, make_int2(-1, -1));
        int maxtype = 0;
        for (int r = 0; r < R; ++r) {
            const espp_replica_desc& dsc = descs[r];
            const int off = rep_poff[r];
            for (int64_t i = 0; i < dsc.n; ++i) {
                const int t = dsc.types ? dsc.types[i] : 0;
                if (t < 0 || t >= MAX_TYPES) return fail(ESPP_ERR_ARG, "particle type out of range");
                types_gid[off + i] = t;
                maxtype = std::max(maxtype, t);
            }
            if (dsc.n_bonds < 0 || (dsc.n_bonds > 0 && !dsc.bonds))
                return fail(ESPP_ERR_ARG, "bad bond list");
            for (int64_t b = 0; b < dsc.n_bonds; ++b) {
                const int64_t p = dsc.bonds[2 * b], q = dsc.bonds[2 * b + 1];
                if (p < 0 || q < 0 || p >= dsc.n || q >= dsc.n || p == q)
                    return fail(ESPP_ERR_ARG, "bond references an invalid particle id");
                for (int side = 0; side < 2; ++side) {
                    const int a = (int)(side == 0 ? p : q) + off, o = (int)(side == 0 ? q : p) + off;
                    int2& s = bond_gid_h[a];
                    if (s.x == o || s.y == o) return fail(ESPP_ERR_ARG, "duplicate bond");
                    if (s.x < 0) s.x = o;
                    else if (s.y < 0) s.y = o;
                    else return fail(ESPP_ERR_ARG, "more than 2 bonds on one particle");
                }
            }
        }
        ntypes = maxtype + 1;
        // molecules: connected components of the bond graph with >= 2 beads
        {
            std::vector<int> parent(N);
            std::iota(parent.begin(), parent.end(), 0);
            auto find = [&](int a) {
                while (parent[a] != a) {
                    parent[a] = parent[parent[a]];
                    a = parent[a];
                }
                return a;
            };
            for (int64_t i = 0; i < N; ++i) {
                const int2 b = bond_gid_h[i];
                for (int o : {b.x, b.y})
                    if (o >= 0) {
                        int ra = find((int)i), rb = find(o);
                        if (ra != rb) parent[std::max(ra, rb)] = std::min(ra, rb);
                    }
            }
            std::vector<int> cnt(N, 0);
            for (int64_t i = 0; i < N; ++i) cnt[find((int)i)]++;
            std::vector<int> mol_of_root(N, -1);
            int nm = 0;
            for (int64_t i = 0; i < N; ++i)
                if (find((int)i) == i && cnt[i] >= 2) mol_of_root[i] = nm++;
            mol_off_h.assign(nm + 1, 0);
            for (int64_t i = 0; i < N; ++i) {
                const int m = mol_of_root[find((int)i)];
                if (m >= 0) mol_off_h[m + 1]++;
            }
            for (int m = 0; m < nm; ++m) mol_off_h[m + 1] += mol_off_h[m];
            mol_members_h.assign(mol_off_h[nm], 0);
            mol_rep_h.assign(nm, 0);
            std::vector<int> fill(mol_off_h.begin(), mol_off_h.end() - 1);
            int r = 0;
            for (int64_t i = 0; i < N; ++i) {
                while (r + 1 < R && i >= rep_poff[r + 1]) ++r;
                const int m = mol_of_root[find((int)i)];
                if (m >= 0) {
                    mol_members_h[fill[m]++] = (int)i;
                    mol_rep_h[m] = r;
                }
            }
        }
        // tiles
        rep_tile_off_h.push_back(0);
        for (int r = 0; r < R; ++r) {
            for (int s0 = 0; s0 < rep_n[r]; s0 += TILE) {
                Tile t;
                t.start = rep_poff[r] + s0;
                t.count = std::min(TILE, rep_n[r] - s0);
                t.rep = r;
                t.pad = 0;
                tiles_h.push_back(t);
            }
            rep_tile_off_h.push_back((int)tiles_h.size());
        }
        // device buffers
        int rc = ESPP_OK;
        const size_t n = (size_t)N;
        if ((rc = alloc(&d.pos[0], n + 1, allocs)) || (rc = alloc(&d.pos[1], n + 1, allocs)) ||
            (rc = alloc(&d.vel, n, allocs)) || (rc = alloc(&d.vel_alt, n, allocs)) ||
            (rc = alloc(&d.frc, n, allocs)) || (rc = alloc(&d.frc_alt, n, allocs)) ||
            (rc = alloc(&d.xb, n, allocs)) || (rc = alloc(&d.img, n, allocs)) ||
            (rc = alloc(&d.img_alt, n, allocs)) || (rc = alloc(&d.bond_slot, n, allocs)) ||
            (rc = alloc(&d.cell_ent, n, allocs)))
            return rc;
        int2* bg = nullptr;
        int *sid, *perm, *cellh, *inc, *ncnt, *req, *now, *rto;
        Tile* tl;
        double* part;
        if ((rc = alloc(&bg, n, allocs)) || (rc = alloc(&sid, n, allocs)) ||
            (rc = alloc(&perm, n, allocs)) || (rc = alloc(&cellh, n, allocs)) ||
            (rc = alloc(&inc, n, allocs)) || (rc = alloc(&ncnt, n, allocs)) ||
            (rc = alloc(&req, R, allocs)) || (rc = alloc(&now, R, allocs)) ||
            (rc = alloc(&tl, tiles_h.size(), allocs)) || (rc = alloc(&rto, R + 1, allocs)) ||
            (rc = alloc(&part, tiles_h.size() * NPART, allocs)) ||
            (rc = alloc(&d_geom, R, allocs)) || (rc = alloc(&d_ip, 1, allocs)) ||
            (rc = alloc(&d_pair, MAX_TYPES * MAX_TYPES, allocs)) || (rc = alloc(&d_ctrl, 1, allocs)) ||
            (rc = alloc(&d_types, n, allocs)) || (rc = alloc(&d_io_x, 3 * n, allocs)) ||
            (rc = alloc(&d_io_v, 3 * n, allocs)) || (rc = alloc(&d_io_img, 3 * n, allocs)) ||
            (rc = alloc(&d_obs, (size_t)R * NPART, allocs)) ||
            (rc = alloc(&d_mol_members, mol_members_h.size(), allocs)) ||
            (rc = alloc(&d_mol_off, mol_off_h.size(), allocs)) ||
            (rc = alloc(&d_mol_rep, mol_rep_h.size(), allocs)) ||
            (rc = alloc(&d_mol_rg2, mol_rep_h.size(), allocs)) ||
            (rc = alloc(&d.mlp_f, n, allocs)) || (rc = alloc(&d.mlp_w, n, allocs)) ||
            (sizeof(T) == 8 && ((rc = alloc(&d.mlp_fT, n, allocs)) || (rc = alloc(&d.mlp_wT, n, allocs)))) ||
            (rc = alloc(&d_mlp, 1, allocs)) || (rc = alloc(&d_le_clk, 1, allocs)) ||
            (rc = alloc(&d.le_db, (size_t)R, allocs)))
            return rc;
        d.le_clk = d_le_clk;
        d.mlp = d_mlp;
        // the list's padding slot: one position past the particles, far
        // outside every box (type 0), in both position buffers
        {
            V4<T> far;
            far.x = far.y = far.z = (T)1e15;
            far.w = (T)0;
            CK(cudaMemcpy(d.pos[0] + n, &far, sizeof(far), cudaMemcpyHostToDevice));
            CK(cudaMemcpy(d.pos[1] + n, &far, sizeof(far), cudaMemcpyHostToDevice));
            d.nbr_pad = N;
        }
        // host-side fault injection for tests: the tensor-core kernel's wait runs out
        if (const char* f = getenv("ESPP_FAULT_TC_TIMEOUT")) d.tc_fault = atoi(f) > 0 ? 1 : 0;
        d.bond_gid = bg;
        d.slot_of_id = sid;
        d.perm = perm;
        d.cellh = cellh;
        d.in_cell = inc;
        d.nbr_cnt = ncnt;
        d.req = req;
        d.now = now;
        d.tiles = tl;
        d.ntiles = (int)tiles_h.size();
        d.rep_tile_off = rto;
        d.partials = part;
        d.reps = d_geom;
        d.R = R;
        d.ctrl = d_ctrl;
        d.ip = d_ip;
        d.pair = d_pair;
        d.ntypes = ntypes;
        d.N = (int)N;
        CK(cudaMemcpy(bg, bond_gid_h.data(), n * sizeof(int2), cudaMemcpyHostToDevice));
        CK(cudaMemcpy(tl, tiles_h.data(), tiles_h.size() * sizeof(Tile), cudaMemcpyHostToDevice));
        CK(cudaMemcpy(rto, rep_tile_off_h.data(), (R + 1) * sizeof(int), cudaMemcpyHostToDevice));
        CK(cudaMemcpy(d_types, types_gid.data(), n * sizeof(int), cudaMemcpyHostToDevice));
        if (!mol_members_h.empty()) {
            CK(cudaMemcpy(d_mol_members, mol_members_h.data(), mol_members_h.size() * sizeof(int), cudaMemcpyHostToDevice));
            CK(cudaMemcpy(d_mol_rep, mol_rep_h.data(), mol_rep_h.size() * sizeof(int), cudaMemcpyHostToDevice));
        }
        CK(cudaMemcpy(d_mol_off, mol_off_h.data(), mol_off_h.size() * sizeof(int), cudaMemcpyHostToDevice));
        upload_geometry();
        CK(upload_params());
        return ESPP_OK;
    }

    // reach of the cell stencil: the list radius rc + skin, or rc alone in
    // the list-free mode (no skin: every step is binned)
    double cell_reach() const { return rc_list + (d.cells_mode ? 0.0 : skin); }

    // cells per edge for stencil half width w: edge >= reach / w
    int cell_count(int r, int c, int w) const {
        return (int)std::floor(w * box[3 * r + c] / (cell_reach() * (1.0 + 1e-6)));
    }

    // Automatic choice: half cells (w = 2) pay off once a full cell holds about
    // ten particles (dense LJ: 19), where the 5x5x5 stencil of half cells
    // searches 42% less volume; for sparse cells (KG melt: 3) the longer
    // stencil loop costs more than it saves.  w = 2 also needs 5 cells per edge.
    int choose_subdivision() {
        if (cell_sub_req > 0) return cell_sub_req;
        // the list-free force kernel streams shorter ranges from half cells
        // and measured slower with them on every workload tried
        if (d.cells_mode) return 1;
        double n = 0, cells = 0;
        bool fits2 = true;
        for (int r = 0; r < R; ++r) {
            double c1 = 1;
            for (int c = 0; c < 3; ++c) {
                c1 *= std::max(1, cell_count(r, c, 1));
                fits2 = fits2 && cell_count(r, c, 2) >= 5;
            }
            n += rep_n[r];
            cells += c1;
        }
        return fits2 && n / cells >= 10.0 ? 2 : 1;
    }

    // every edge of replica r holds 2w + 1 distinct cells of the subdivision
    bool cells_fit(int r) const {
        bool ok = true;
        for (int c = 0; c < 3; ++c) ok = ok && cell_count(r, c, cell_sub) >= 2 * cell_sub + 1;
        return ok;
    }

    int upload_geometry() {
        std::vector<RepGeom<T>> g(R);
        int coff = 0;
        for (int r = 0; r < R; ++r) {
            const int w = cell_sub;
            for (int c = 0; c < 3; ++c) {
                g[r].L[c] = (T)box[3 * r + c];
                g[r].halfL[c] = g[r].L[c] * T(0.5);
                const int nc = cells_ready ? cell_count(r, c, w) : 1;
                g[r].nc[c] = nc;
                g[r].cells_per_len[c] = (T)((double)nc / (double)g[r].L[c]);
            }
            g[r].cell_off = coff;
            coff += g[r].nc[0] * g[r].nc[1] * g[r].nc[2];
            g[r].p_off = rep_poff[r];
            g[r].n = rep_n[r];
            g[r].pad = 0;
            g[r].seed = seeds[r];
        }
        cudaError_t e = cudaMemcpy(d_geom, g.data(), R * sizeof(RepGeom<T>), cudaMemcpyHostToDevice);
        return e == cudaSuccess ? ESPP_OK : fail(ESPP_ERR_CUDA, cudaGetErrorString(e));
    }

    cudaError_t upload_params() {
        // concatenated tables in the handle's precision
        std::vector<T> tab;
        std::vector<PairRec<T>> pr(MAX_TYPES * MAX_TYPES);
        for (int a = 0; a < ntypes; ++a)
            for (int b = 0; b < ntypes; ++b) {
                const PairHost& p = pair_h[a][b];
                PairRec<T>& q = pr[a * ntypes + b];
                memset(&q, 0, sizeof(q));
                q.kind = p.kind;
                if (p.kind == ESPP_NONE) continue;
                if (p.kind == ESPP_MLP) {
                    q.rc2 = (T)(p.rc * p.rc);
                    continue;
                }
                if (p.kind == ESPP_TAB_PAIR) {
                    const int nt = (int)(p.tab.size() / 2);
                    q.rc2 = (T)(p.rc * p.rc);
                    q.tab_off = (int)tab.size();
                    q.tab_n = nt;
                    q.inv_dr = (T)((nt - 1) / p.rc);
                    for (double v : p.tab) tab.push_back((T)v);
                    continue;
                }
                const double s2 = p.sig * p.sig;
                auto lj = [&](double r2, double& u, double& fr) {
                    const double x = s2 / r2, x6 = x * x * x;
                    u = 4 * p.eps * (x6 * x6 - x6);
                    fr = 24 * p.eps * (2 * x6 * x6 - x6) / r2;
                };
                double us = 0, fs = 0;
                if (p.shift) lj(p.rc * p.rc, us, fs);
                q.rc2 = (T)(p.rc * p.rc);
                q.sig2 = (T)s2;
                q.eps24 = (T)(24 * p.eps);
                q.eps4 = (T)(4 * p.eps);
                q.shift = (T)us;
                if (p.kind == ESPP_LJ_CAPPED) {
                    double uc, frc;
                    lj(p.cap * p.cap, uc, frc);
                    q.cap2 = (T)(p.cap * p.cap);
                    q.cap = (T)p.cap;
                    q.capF = (T)(frc * p.cap);
                    q.capU = (T)(uc - us);
                }
            }
        // the list-free mode reads its pair forces from the cell kernel, which
        // the general step-kernel variants take
        d.lj_fast = (!d.cells_mode && ntypes == 1 && pair_h[0][0].kind == ESPP_LJ) ? 1 : 0;
        d.mlp_on = (pair_h[0][0].kind == ESPP_MLP) ? 1 : 0;
        if (d.mlp_on && !mlp_bits.empty()) {
            MlpWeights w;
            memset(&w, 0, sizeof(w));
            auto f = [&](int k) {
                const uint32_t b = (uint32_t)mlp_bits[k] << 16;
                float v;
                memcpy(&v, &b, 4);
                return v;
            };
            memcpy(static_cast<void*>(w.W1), mlp_bits.data(), sizeof(w.W1));  // BF16 bit patterns
            const int o_b1 = MLP_H * MLP_NB, o_W2 = o_b1 + MLP_H, o_b2 = o_W2 + MLP_H * MLP_H;
            const int o_w3 = o_b2 + MLP_H, o_b3 = o_w3 + MLP_H;
            memcpy(static_cast<void*>(w.W2), mlp_bits.data() + o_W2, sizeof(w.W2));
            for (int a = 0; a < MLP_H; ++a) {
                w.b1[a] = f(o_b1 + a);
                w.b2[a] = f(o_b2 + a);
                w.w3[a] = f(o_w3 + a);
            }
            w.b3 = f(o_b3);
            w.rc = (float)pair_h[0][0].rc;
            cudaError_t e = cudaMemcpy(d_mlp, &w, sizeof(w), cudaMemcpyHostToDevice);
            if (e != cudaSuccess) return e;
        }
        d.bond.kind = bond_kind;
        d.bond.K = (T)bond_K;
        d.bond.inv_R02 = bond_kind ? (T)(1.0 / (bond_R0 * bond_R0)) : T(0);
        d.bond.halfKR02 = (T)(0.5 * bond_K * bond_R0 * bond_R0);
        d.bond.rmax = (T)bond_R0;
        if (bond_kind == ESPP_TAB_BOND) {
            const int nt = (int)(bond_tab.size() / 2);
            d.bond.tab_off = (int)tab.size();
            d.bond.tab_n = nt;
            d.bond.inv_dr = (T)((nt - 1) / bond_R0);
            for (double v : bond_tab) tab.push_back((T)v);
        }
        if (tab.size() > tab_elems || !tab_alloc) {
            if (tab_alloc) cudaFree(tab_alloc);
            tab_alloc = nullptr;
            tab_elems = std::max<size_t>(tab.size(), 1);
            cudaError_t e = cudaMalloc(&tab_alloc, tab_elems * sizeof(T));
            if (e != cudaSuccess) return e;
        }
        d.tab = reinterpret_cast<const T*>(tab_alloc);
        if (!tab.empty()) {
            cudaError_t e = cudaMemcpy(tab_alloc, tab.data(), tab.size() * sizeof(T), cudaMemcpyHostToDevice);
            if (e != cudaSuccess) return e;
        }
        return cudaMemcpy(d_pair, pr.data(), pr.size() * sizeof(PairRec<T>), cudaMemcpyHostToDevice);
    }

    int upload_int_params(double dt, double gamma, double kT) {
        if (ip_key[0] == dt && ip_key[1] == gamma && ip_key[2] == kT && !mass_dirty) return ESPP_OK;
        IntParams<T> ip;
        memset(&ip, 0, sizeof(ip));
        ip.dt = (T)dt;
        ip.half_dt = (T)(0.5 * dt);
        ip.gamma = (T)gamma;
        ip.kT = (T)kT;
        if (d.dpd) {
            ip.dpd_rc2 = (T)(dpd_rc * dpd_rc);
            ip.dpd_inv_rc = (T)(1.0 / dpd_rc);
            ip.dpd_amp = (T)(std::sqrt(2.0 * gamma * kT) * std::sqrt(12.0) / std::sqrt(dt));
        }
        for (int a = 0; a < MAX_TYPES; ++a) {
            ip.mass[a] = (T)mass_h[a];
            ip.inv_mass[a] = (T)(1.0 / mass_h[a]);
            ip.noise_amp[a] = dt > 0 ? (T)std::sqrt(24.0 * gamma * mass_h[a] * kT / dt) : T(0);
        }
        CK(cudaMemcpyAsync(d_ip, &ip, sizeof(ip), cudaMemcpyHostToDevice, st));
        CK(cudaStreamSynchronize(st));
        ip_key[0] = dt;
        ip_key[1] = gamma;
        ip_key[2] = kT;
        mass_dirty = false;
        return ESPP_OK;
    }
    bool mass_dirty = true;

    // ------------------------------------------------------------------ state
    int set_state(const double* x, const double* v, const int32_t* img, int where) override {
        if (!x) return fail(ESPP_ERR_ARG, "positions are required");
        const size_t n3 = 3 * (size_t)N;
        const double *dx = x, *dv = v;
        const int* di = img;
        if (where == ESPP_HOST) {
            CK(cudaMemcpyAsync(d_io_x, x, n3 * sizeof(double), cudaMemcpyHostToDevice, st));
            dx = d_io_x;
            if (v) {
                CK(cudaMemcpyAsync(d_io_v, v, n3 * sizeof(double), cudaMemcpyHostToDevice, st));
                dv = d_io_v;
            }
            if (img) {
                CK(cudaMemcpyAsync(d_io_img, img, n3 * sizeof(int), cudaMemcpyHostToDevice, st));
                di = d_io_img;
            }
        } else if (where != ESPP_DEVICE) {
            return fail(ESPP_ERR_ARG, "where must be ESPP_HOST or ESPP_DEVICE");
        }
        cur = 0;
        {
            // a new state clears any earlier error or freeze (the step number is kept)
            Ctrl c = read_ctrl();
            c.err = 0;
            c.abort = 0;
            c.any_req = 0;
            c.blocks_done = 0;
            c.need_cap = 0;
            CK(cudaMemcpyAsync(d_ctrl, &c, sizeof(Ctrl), cudaMemcpyHostToDevice, st));
        }
        Launch<T>::set_state(d, dx, dv, di, d_types, cur, st);
        Launch<T>::request_all(d, st);
        launches += 2;
        CK(cudaGetLastError());
        CK(cudaStreamSynchronize(st));
        {
            Ctrl c = read_ctrl();
            if (c.err & ERRBIT_NONFINITE) {
                // refuse the state: clear the flag, keep no half-set state
                c.err = 0;
                CK(cudaMemcpy(d_ctrl, &c, sizeof(Ctrl), cudaMemcpyHostToDevice));
                state_set = false;
                return fail(ESPP_ERR_ARG, "non-finite position or velocity");
            }
        }
        state_set = true;
        f_valid = false;
        rebuild_pending = true;
        return ESPP_OK;
    }

    int get_state(double* x, double* v, int32_t* img, int where) override {
        if (!state_set) return fail(ESPP_ERR_STATE, "no state set");
        const size_t n3 = 3 * (size_t)N;
        if (where == ESPP_DEVICE) {
            Launch<T>::get_state(d, x, v, img, nullptr, cur, st);
            launches++;
            CK(cudaGetLastError());
            CK(cudaStreamSynchronize(st));
            return ESPP_OK;
        }
        if (where != ESPP_HOST) return fail(ESPP_ERR_ARG, "where must be ESPP_HOST or ESPP_DEVICE");
        Launch<T>::get_state(d, x ? d_io_x : nullptr, v ? d_io_v : nullptr, img ? d_io_img : nullptr, nullptr, cur,
                             st);
        launches++;
        CK(cudaGetLastError());
        if (x) CK(cudaMemcpyAsync(x, d_io_x, n3 * sizeof(double), cudaMemcpyDeviceToHost, st));
        if (v) CK(cudaMemcpyAsync(v, d_io_v, n3 * sizeof(double), cudaMemcpyDeviceToHost, st));
        if (img) CK(cudaMemcpyAsync(img, d_io_img, n3 * sizeof(int), cudaMemcpyDeviceToHost, st));
        CK(cudaStreamSynchronize(st));
        return ESPP_OK;
    }

    Ctrl read_ctrl() {
        Ctrl c;
        memset(&c, 0, sizeof(c));
        cudaMemcpyAsync(&c, d_ctrl, sizeof(Ctrl), cudaMemcpyDeviceToHost, st);
        cudaStreamSynchronize(st);
        return c;
    }

    int set_step(int64_t s) override {
        // the simulated time stays; the step number it belongs to changes
        Ctrl c = read_ctrl();
        const double t = time_at(c.step);
        CK(cudaMemcpyAsync(&d_ctrl->step, &s, sizeof(long long), cudaMemcpyHostToDevice, st));
        CK(cudaStreamSynchronize(st));
        return set_clock(t, le_clk_h.dt, s);
    }

    // ---------------------------------------------------- Lees-Edwards clock
    double time_at(int64_t step) const { return le_clk_h.t0 + (double)(step - le_clk_h.s0) * le_clk_h.dt; }
    int set_clock(double t0, double dt, int64_t s0) {
        le_clk_h.t0 = t0;
        le_clk_h.dt = dt;
        le_clk_h.s0 = s0;
        // the kernels read the clock under Lees-Edwards only; switching it on
        // (or loading a sheared checkpoint) passes through here again
        if (!d.le_on) return ESPP_OK;
        CK(cudaMemcpyAsync(d_le_clk, &le_clk_h, sizeof(LeClock), cudaMemcpyHostToDevice, st));
        CK(cudaStreamSynchronize(st));
        return ESPP_OK;
    }

    int set_lees_edwards(int on, double shear, double time) override {
        if (!std::isfinite(shear) || !std::isfinite(time)) return fail(ESPP_ERR_ARG, "shear rate and time must be finite");
        if (on && d.mlp_on) return fail(ESPP_ERR_STATE, "Lees-Edwards is not available with the learned potential");
        Ctrl c = read_ctrl();
        d.le_on = on ? 1 : 0;
        d.le_shear = on ? shear : 0.0;
        int rcode = set_clock(time, le_clk_h.dt, c.step);
        if (rcode) return rcode;
        clear_graphs();          // the setting is a kernel argument of captured graphs
        rebuild_pending = true;  // the search across the sheared faces changes
        f_valid = false;
        return ESPP_OK;
    }

    int get_lees_edwards(int* on, double* shear, double* time) override {
        Ctrl c = read_ctrl();
        if (on) *on = d.le_on;
        if (shear) *shear = d.le_shear;
        if (time) *time = time_at(c.step);
        return ESPP_OK;
    }

    // ----------------------------------------------------------- interactions
    int set_interaction(int kind, int ta, int tb, const double* p, int64_t np) override {
        auto read_table = [&](double& rmax, std::vector<double>& out) -> int {
            if (!p || np < 2) return fail(ESPP_ERR_ARG, "a table needs rmax, n, u[n], F[n]");
            const double nd = p[1];
            if (!(p[0] > 0) || !(nd >= 2) || nd != std::floor(nd) || np != 2 + 2 * (int64_t)nd)
                return fail(ESPP_ERR_ARG, "a table needs rmax > 0, n >= 2 and exactly 2n values");
            rmax = p[0];
            out.assign(p + 2, p + 2 + 2 * (int64_t)nd);
            for (double v : out)
                if (!std::isfinite(v)) return fail(ESPP_ERR_ARG, "non-finite table entry");
            return ESPP_OK;
        };
        auto finite = [&](int count) {
            for (int k = 0; k < count; ++k)
                if (!std::isfinite(p[k])) return false;
            return true;
        };
        if (kind == ESPP_FENE) {
            if (!p || np < 2 || !(p[0] > 0) || !(p[1] > 0) || !finite(2))
                return fail(ESPP_ERR_ARG, "FENE needs finite K > 0, R0 > 0");
            bond_kind = ESPP_FENE;
            bond_K = p[0];
            bond_R0 = p[1];
        } else if (kind == ESPP_TAB_BOND) {
            double rmax;
            std::vector<double> t;
            int rc = read_table(rmax, t);
            if (rc) return rc;
            bond_kind = ESPP_TAB_BOND;
            bond_K = 0;
            bond_R0 = rmax;
            bond_tab = t;
        } else {
            if (ta < 0 || tb < 0 || ta >= MAX_TYPES || tb >= MAX_TYPES)
                return fail(ESPP_ERR_ARG, "type out of range");
            PairHost h;
            if (kind == ESPP_NONE) {
            } else if (kind == ESPP_LJ || kind == ESPP_LJ_CAPPED) {
                const int need = kind == ESPP_LJ ? 4 : 5;
                if (!p || np < need) return fail(ESPP_ERR_ARG, "too few parameters");
                if (!finite(need)) return fail(ESPP_ERR_ARG, "non-finite parameter");
                h.kind = kind;
                h.eps = p[0];
                h.sig = p[1];
                h.rc = p[2];
                h.shift = p[3] != 0.0;
                if (kind == ESPP_LJ_CAPPED) h.cap = p[4];
                if (!(h.sig > 0) || !(h.rc > 0) || (kind == ESPP_LJ_CAPPED && !(h.cap > 0)))
                    return fail(ESPP_ERR_ARG, "sigma, rc and caprad must be positive");
            } else if (kind == ESPP_TAB_PAIR) {
                int rc = read_table(h.rc, h.tab);
                if (rc) return rc;
                h.kind = ESPP_TAB_PAIR;
            } else if (kind == ESPP_MLP) {
                if (!p || np < 1 || !(p[0] > 0) || !finite(1))
                    return fail(ESPP_ERR_ARG, "the learned potential needs a finite rc > 0");
                if (ta != 0 || tb != 0 || ntypes != 1)
                    return fail(ESPP_ERR_ARG, "the learned potential applies to single-type systems (types 0, 0)");
                h.kind = ESPP_MLP;
                h.rc = p[0];
            } else if (kind == ESPP_WCA) {
                if (!p || np < 2 || !finite(2)) return fail(ESPP_ERR_ARG, "WCA needs finite eps, sigma");
                h.kind = ESPP_LJ;
                h.eps = p[0];
                h.sig = p[1];
                h.rc = std::pow(2.0, 1.0 / 6.0) * p[1];
                h.shift = true;
                if (!(h.sig > 0)) return fail(ESPP_ERR_ARG, "sigma must be positive");
            } else {
                return fail(ESPP_ERR_ARG, "unknown interaction kind");
            }
            pair_h[ta][tb] = h;
            pair_h[tb][ta] = h;
        }
        CK(upload_params());
        clear_graphs();  // the bond record is a kernel argument of captured graphs
        f_valid = false;
        return ESPP_OK;
    }

    int mlp_set_weights(const uint16_t* bits, int64_t n) override {
        if (!bits || n != MLP_NPARAMS) return fail(ESPP_ERR_ARG, "expected ESPP_MLP_NPARAMS BF16 weights");
        for (int64_t k = 0; k < n; ++k)
            if ((bits[k] & 0x7F80u) == 0x7F80u) return fail(ESPP_ERR_ARG, "non-finite BF16 weight");
        mlp_bits.assign(bits, bits + n);
        CK(upload_params());
        f_valid = false;
        return ESPP_OK;
    }

    // positions and conservative forces mapped onto sites of bps consecutive
    // beads (device outputs; replica 0's box)
    int cg_map(int bps, double* xs, double* fs) override {
        if (bps < 1 || N % bps != 0 || !xs || !fs) return fail(ESPP_ERR_ARG, "bad mapping arguments");
        if (d.le_on) return fail(ESPP_ERR_STATE, "the CG mapping is not available under Lees-Edwards");
        double* fdev = nullptr;
        CK(cudaMalloc(&fdev, 3 * (size_t)N * sizeof(double)));
        int rcode = compute_forces(fdev, ESPP_DEVICE);
        if (!rcode) {
            Launch<T>::get_state(d, d_io_x, nullptr, d_io_img, nullptr, cur, st);
            launch_cg_map(d_io_x, d_io_img, fdev, N / bps, bps, box.data(), xs, fs, st);
            launches += 2;
            cudaError_t e = cudaStreamSynchronize(st);
            if (e != cudaSuccess) rcode = fail(ESPP_ERR_CUDA, cudaGetErrorString(e));
        }
        cudaFree(fdev);
        return rcode;
    }

    int mlp_get_weights(uint16_t* out, int64_t n) override {
        if (!out || n != MLP_NPARAMS) return fail(ESPP_ERR_ARG, "expected room for ESPP_MLP_NPARAMS weights");
        if (mlp_bits.empty()) return fail(ESPP_ERR_STATE, "no weights set");
        memcpy(out, mlp_bits.data(), sizeof(uint16_t) * MLP_NPARAMS);
        return ESPP_OK;
    }

    // training state (allocated on first use)
    float4* t_err = nullptr;
    double* t_loss_part = nullptr;
    float* t_partials = nullptr;
    float *t_grad = nullptr, *t_theta = nullptr, *t_m = nullptr, *t_v = nullptr;
    double* t_loss = nullptr;
    int t_blocks = 0, t_epochs_alloc = 0, adam_step = 0;

    static uint64_t splitmix64(uint64_t& x) {
        uint64_t z = (x += 0x9E3779B97F4A7C15ull);
        z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
        z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
        return z ^ (z >> 31);
    }

    // Force-matching training (epochs >= 1), or one loss and gradient
    // evaluation of the current weights over all frames (epochs == 0).
    int mlp_train(const double* X, const double* Y, int nframes, int batch, int epochs, double lr, uint64_t seed,
                  double* loss_hist, float* grad_out) override {
        NvtxRange nvtx_range("espp_mlp_train");
        if (!X || !Y || nframes < 1 || epochs < 0 || (epochs > 0 && (batch < 1 || !(lr > 0))))
            return fail(ESPP_ERR_ARG, "bad training arguments");
        if (!d.mlp_on || mlp_bits.empty()) return fail(ESPP_ERR_STATE, "select the learned potential and set weights first");
        if (!cells_ready) return fail(ESPP_ERR_STATE, "call espp_build_neighbors first");
        {
            const int rb = ensure_mlp_buffers();
            if (rb) return rb;
        }
        const int ngrad = mlp_ngrad();
        const int nep = std::max(epochs, 1);
        if (!t_err) {
            t_blocks = sm_count();  // one gradient CTA per SM (tensor memory: 480 of 512 columns)
            int rc0;
            if ((rc0 = alloc(&t_err, (size_t)N, allocs)) || (rc0 = alloc(&t_loss_part, (size_t)d.ntiles, allocs)) ||
                (rc0 = alloc(&t_partials, (size_t)(t_blocks + 16) * ngrad, allocs)) || (rc0 = alloc(&t_grad, ngrad, allocs)) ||
                (rc0 = alloc(&t_theta, ngrad, allocs)) || (rc0 = alloc(&t_m, ngrad, allocs)) ||
                (rc0 = alloc(&t_v, ngrad, allocs)))
                return rc0;
            CK(Launch<T>::prepare_train());
        }
        if (t_epochs_alloc < nep) {
            int rc0 = alloc(&t_loss, (size_t)nep, allocs);
            if (rc0) return rc0;
            t_epochs_alloc = nep;
        }
        // FP32 master weights from the current BF16 weights (all but b3)
        {
            std::vector<float> th(ngrad);
            for (int k = 0; k < ngrad; ++k) {
                const uint32_t b = (uint32_t)mlp_bits[k] << 16;
                memcpy(&th[k], &b, 4);
            }
            CK(cudaMemcpy(t_theta, th.data(), ngrad * sizeof(float), cudaMemcpyHostToDevice));
            CK(cudaMemset(t_m, 0, ngrad * sizeof(float)));
            CK(cudaMemset(t_v, 0, ngrad * sizeof(float)));
            CK(cudaMemset(t_grad, 0, ngrad * sizeof(float)));
            CK(cudaMemset(t_loss, 0, nep * sizeof(double)));
        }
        adam_step = 0;
        const size_t n3 = 3 * (size_t)N;
        std::vector<int> order(nframes);
        std::iota(order.begin(), order.end(), 0);
        uint64_t rs = seed;
        for (int ep = 0; ep < nep; ++ep) {
            if (epochs > 0)
                for (int k = nframes - 1; k > 0; --k) std::swap(order[k], order[splitmix64(rs) % (uint64_t)(k + 1)]);
            const int bsz = epochs > 0 ? batch : nframes;
            for (int b0 = 0; b0 < nframes; b0 += bsz) {
                const int nb = std::min(bsz, nframes - b0);
                const float scale = (float)(-2.0 / ((double)nb * (double)N));
                for (int q = 0; q < nb; ++q) {
                    const int f = order[b0 + q];
                    int rcode = set_state(X + f * n3, nullptr, nullptr, ESPP_DEVICE);
                    if (rcode) return rcode;
                    // a training frame needs its list, not a new storage order
                    rcode = rebuild_now(false, false);
                    if (rcode) return rcode;
                    launches += Launch<T>::mlp_tc(d, cur, false, st);
                    launches += Launch<T>::train_grad(d, cur, Y + f * n3, t_err, t_loss_part, scale, t_partials,
                                                          t_blocks, t_grad, t_loss + ep, st);
                    CK(cudaGetLastError());
                }
                if (epochs > 0) {
                    ++adam_step;
                    launch_adam(t_theta, t_m, t_v, t_grad, (float)lr, 0.9f, 0.999f, 1e-8f, adam_step, d_mlp, st);
                    launches++;
                    CK(cudaGetLastError());
                }
            }
        }
        std::vector<double> lh(nep);
        CK(cudaMemcpyAsync(lh.data(), t_loss, nep * sizeof(double), cudaMemcpyDeviceToHost, st));
        if (grad_out && epochs == 0) CK(cudaMemcpyAsync(grad_out, t_grad, ngrad * sizeof(float), cudaMemcpyDeviceToHost, st));
        CK(cudaStreamSynchronize(st));
        if (loss_hist)
            for (int ep = 0; ep < nep; ++ep) loss_hist[ep] = lh[ep] / ((double)nframes * (double)N);
        if (epochs > 0) {
            // the trained BF16 weights become the handle's weights
            MlpWeights w;
            CK(cudaMemcpy(&w, d_mlp, sizeof(w), cudaMemcpyDeviceToHost));
            auto bits = [](float v) {
                uint32_t b;
                memcpy(&b, &v, 4);
                return (uint16_t)(b >> 16);  // these floats are BF16 values
            };
            const int o_b1 = MLP_H * MLP_NB, o_W2 = o_b1 + MLP_H, o_b2 = o_W2 + MLP_H * MLP_H, o_w3 = o_b2 + MLP_H;
            memcpy(mlp_bits.data(), w.W1, sizeof(w.W1));
            memcpy(mlp_bits.data() + o_W2, w.W2, sizeof(w.W2));
            for (int a = 0; a < MLP_H; ++a) {
                mlp_bits[o_b1 + a] = bits(w.b1[a]);
                mlp_bits[o_b2 + a] = bits(w.b2[a]);
                mlp_bits[o_w3 + a] = bits(w.w3[a]);
            }
        }
        f_valid = false;
        return ESPP_OK;
    }

    int set_exclude_bonded(int on) override {
        d.excl_bonded = on ? 1 : 0;
        clear_graphs();  // a kernel argument of the captured graphs
        rebuild_pending = true;
        if (state_set) {
            Launch<T>::request_all(d, st);
            launches++;
        }
        f_valid = false;
        return ESPP_OK;
    }

    int set_mass(int type, double m) override {
        if (type < 0 || type >= MAX_TYPES || !(m > 0) || !std::isfinite(m)) return fail(ESPP_ERR_ARG, "bad mass");
        mass_h[type] = m;
        mass_dirty = true;
        f_valid = false;
        return ESPP_OK;
    }

    int check_cutoffs() {
        for (int a = 0; a < ntypes; ++a)
            for (int b = 0; b < ntypes; ++b)
                if (pair_h[a][b].kind != ESPP_NONE && pair_h[a][b].rc > rc_list * (1 + 1e-12))
                    return fail(ESPP_ERR_ARG, "a pair cutoff exceeds the Verlet-list cutoff");
        return ESPP_OK;
    }

    // ---------------------------------------------------------- neighbour list
    int estimate_cap() const {
        double best = 0;
        const double rl = rc_list + skin;
        for (int r = 0; r < R; ++r) {
            const double V = box[3 * r] * box[3 * r + 1] * box[3 * r + 2];
            const double rho = rep_n[r] / V;
            best = std::max(best, rho * 4.0 / 3.0 * M_PI * rl * rl * rl);
        }
        int cap = (int)std::ceil(best * 1.4 + 8);
        // host-side fault injection for tests: start from a deliberately short list
        if (const char* f = getenv("ESPP_FAULT_LIST_CAP")) {
            const int forced = atoi(f);
            if (forced > 0) cap = forced;
        }
        return std::max(8, (cap + 3) & ~3);  // the step kernel reads two groups ahead
    }

    int alloc_list(int cap) {
        if (nbr_alloc) cudaFree(nbr_alloc);
        nbr_alloc = nullptr;
        d.stride = (int)((N + 31) / 32 * 32);
        void* p = nullptr;
        cudaError_t e = cudaMalloc(&p, (size_t)cap * d.stride * sizeof(int));
        if (e != cudaSuccess) return fail(ESPP_ERR_CUDA, std::string("list allocation: ") + cudaGetErrorString(e));
        nbr_alloc = p;
        e = cudaMemset(p, 0, (size_t)cap * d.stride * sizeof(int));
        if (e != cudaSuccess) return fail(ESPP_ERR_CUDA, std::string("list memset: ") + cudaGetErrorString(e));
        d.nbr = reinterpret_cast<int*>(p);
        d.cap = cap;
        clear_graphs();
        return d.mlp_on ? alloc_mlp_buffers() : ESPP_OK;
    }

    // per-entry values and mirrored-entry indices of the learned potential,
    // sized like the list (3 x 4 bytes per list slot), and the dense pair
    // array (16 bytes per unordered pair)
    int alloc_mlp_buffers() {
        {
            static cudaError_t prep = prepare_mlp_tc();  // kernel attributes, once per process
            if (prep != cudaSuccess) return fail(ESPP_ERR_CUDA, std::string("MLP kernel setup: ") + cudaGetErrorString(prep));
        }
        if (mlp_buf) cudaFree(mlp_buf);
        mlp_buf = nullptr;
        mlp_buf_cap = 0;
        d.mlp_pf = d.mlp_pu = nullptr;
        d.mlp_rev = nullptr;
        d.mlp_pairs = nullptr;
        d.mlp_npairs = nullptr;
        d.mlp_pairs_cap = 0;
        d.mlp_upper = nullptr;
        d.mlp_nupper = nullptr;
        d.mlp_upper_cap = 0;
        d.mlp_ucount = d.mlp_uoff = d.mlp_uscan_part = nullptr;
        const size_t slots = (size_t)d.cap * d.stride;
        // the pair arrays hold every unordered pair of the list; entry
        // indices are 32-bit
        const size_t npairs = slots / 2 + 64;
        if (4 * slots > (size_t)INT32_MAX) return fail(ESPP_ERR_ARG, "list too large for the learned potential");
        const int nus = scan_blocks_for((int)N);
        const size_t bytes = 3 * slots * sizeof(float) + 2 * npairs * sizeof(int4) + 64 +
                             (2 * (size_t)N + nus + 16) * sizeof(int);
        void* p = nullptr;
        cudaError_t e = cudaMalloc(&p, bytes);
        if (e != cudaSuccess) return fail(ESPP_ERR_CUDA, std::string("MLP buffers: ") + cudaGetErrorString(e));
        e = cudaMemset(p, 0, bytes);
        if (e != cudaSuccess) return fail(ESPP_ERR_CUDA, std::string("MLP buffers: ") + cudaGetErrorString(e));
        mlp_buf = p;
        mlp_buf_cap = d.cap;
        d.mlp_pairs = reinterpret_cast<int4*>(p);  // 256-byte aligned (cudaMalloc)
        d.mlp_pairs_cap = (int)npairs;
        d.mlp_upper = d.mlp_pairs + npairs;
        d.mlp_upper_cap = (int)npairs;
        d.mlp_pf = reinterpret_cast<float*>(d.mlp_upper + npairs);
        d.mlp_pu = d.mlp_pf + slots;
        d.mlp_rev = reinterpret_cast<int*>(d.mlp_pu + slots);
        d.mlp_npairs = d.mlp_rev + slots;
        d.mlp_nupper = d.mlp_npairs + 1;
        d.mlp_ucount = d.mlp_npairs + 16;
        d.mlp_uoff = d.mlp_ucount + N;
        d.mlp_uscan_part = d.mlp_uoff + N;
        d.mlp_nuscan = nus;
        clear_graphs();
        return ESPP_OK;
    }

    // the learned potential was selected after the list was sized: allocate its
    // buffers and rebuild every replica so the mirrored entries exist
    int ensure_mlp_buffers() {
        if (!d.mlp_on || !d.nbr || (mlp_buf && mlp_buf_cap == d.cap)) return ESPP_OK;
        int rcode = alloc_mlp_buffers();
        if (rcode) return rcode;
        Launch<T>::request_all(d, st);
        launches++;
        rebuild_pending = true;
        return ESPP_OK;
    }

    int build_neighbors(double rc, double sk) override {
        NvtxRange nvtx_range("espp_build_neighbors");
        if (!(rc > 0) || !(sk >= 0) || !std::isfinite(rc) || !std::isfinite(sk))
            return fail(ESPP_ERR_ARG, "rc must be positive and skin non-negative");
        const double rc_old = rc_list, sk_old = skin;
        rc_list = rc;
        skin = sk;
        int rcode = check_cutoffs();
        if (rcode) {
            rc_list = rc_old;  // refused: the grid and list of the old cutoff stay valid
            skin = sk_old;
            return rcode;
        }
        cell_sub = choose_subdivision();
        for (int r = 0; r < R; ++r)
            if (!cells_fit(r)) {
                cells_ready = false;
                return fail(ESPP_ERR_BOX_TOO_SMALL,
                            "box edge holds fewer than 2w + 1 cells of (rc + skin) / w (w: cell subdivision)");
            }
        cells_ready = true;
        // cell grids; Hilbert ranks for the resort order
        for (void* p : cell_allocs) cudaFree(p);
        cell_allocs.clear();
        clear_graphs();
        std::vector<int> rep_of, by_rank;
        int coff = 0;
        for (int r = 0; r < R; ++r) {
            const int w = cell_sub;
            const int nx = cell_count(r, 0, w), ny = cell_count(r, 1, w), nz = cell_count(r, 2, w);
            const int nc = nx * ny * nz;
            std::vector<int> rk(nc);
            hilbert_ranks(nx, ny, nz, rk.data());
            by_rank.resize(coff + nc);
            for (int k = 0; k < nc; ++k) {
                rep_of.push_back(r);
                by_rank[coff + rk[k]] = coff + k;
            }
            coff += nc;
        }
        const int C = coff;
        int *cnt, *beg, *rstart, *crep, *cbr, *part;
        int rc2 = ESPP_OK;
        d.nscan_blocks = scan_blocks_for(C);
        if ((rc2 = alloc(&cnt, C, cell_allocs)) || (rc2 = alloc(&beg, C + 1, cell_allocs)) ||
            (rc2 = alloc(&rstart, C, cell_allocs)) || (rc2 = alloc(&crep, C, cell_allocs)) ||
            (rc2 = alloc(&cbr, C, cell_allocs)) || (rc2 = alloc(&part, d.nscan_blocks, cell_allocs)))
            return rc2;
        CK(cudaMemcpy(crep, rep_of.data(), C * sizeof(int), cudaMemcpyHostToDevice));
        CK(cudaMemcpy(cbr, by_rank.data(), C * sizeof(int), cudaMemcpyHostToDevice));
        // every count starts at zero (a replica's counts sum to its particle
        // count after its first build); the entry array ends at N
        CK(cudaMemset(cnt, 0, C * sizeof(int)));
        const int nn = (int)N;
        CK(cudaMemcpy(beg + C, &nn, sizeof(int), cudaMemcpyHostToDevice));
        d.cell_w = cell_sub;
        d.cell_cnt = cnt;
        d.cell_beg = beg;
        d.rank_start = rstart;
        d.cell_rep = crep;
        d.cell_by_rank = cbr;
        d.ncells = C;
        d.scan_part = part;
        const double rl = rc + sk;
        d.rlist2 = (T)(rl * rl);
        d.half_skin2 = (T)(0.25 * sk * sk);
        d.skin = (T)sk;
        rcode = upload_geometry();
        if (rcode) return rcode;
        rcode = alloc_list(estimate_cap());
        if (rcode) return rcode;
        if (!state_set) return ESPP_OK;
        Launch<T>::request_all(d, st);
        launches++;
        return rebuild_now(f_valid);
    }

    // Direct (non-graph) rebuild, with a resort unless asked not to, with
    // capacity retries.  After
    // an overflow the list or the cell array is reallocated and every replica
    // is rebuilt (the old buffers of the other replicas are gone).
    int rebuild_now(bool permute_force, bool resort = true) {
        NvtxRange nvtx_range("espp_rebuild");
        if (!cells_ready) return fail(ESPP_ERR_STATE, "call espp_build_neighbors first");
        for (int attempt = 0; attempt < 6; ++attempt) {
            launches += Launch<T>::rebuild(d, cur, resort, permute_force, st);
            CK(cudaGetLastError());
            Ctrl c = read_ctrl();
            CK(cudaGetLastError());
            if (!(c.err & ERRBIT_OVERFLOW)) {
                rebuild_pending = false;
                return ESPP_OK;
            }
            int rcode = grow_capacity(c);
            if (rcode) return rcode;
        }
        return fail(ESPP_ERR_LIST_OVERFLOW, "Verlet list overflow persists after retries");
    }

    // grow the list after an overflow, clear the overflow state and request a
    // rebuild of every replica
    int grow_capacity(const Ctrl& c) {
        int rcode = ESPP_OK;
        if (c.err & ERRBIT_OVERFLOW) {
            int cap = (int)std::ceil(c.need_cap * 1.2 + 8);
            cap = (cap + 3) & ~3;
            rcode = alloc_list(std::max(cap, d.cap + 4));
            if (rcode) return rcode;
        }
        Ctrl w = read_ctrl();
        w.err &= ~ERRBIT_OVERFLOW;
        w.abort = 0;
        w.need_cap = 0;
        w.blocks_done = 0;
        CK(cudaMemcpyAsync(d_ctrl, &w, sizeof(Ctrl), cudaMemcpyHostToDevice, st));
        Launch<T>::request_all(d, st);
        launches++;
        CK(cudaStreamSynchronize(st));
        return ESPP_OK;
    }

    // Rebuilds the list when it is stale; *out (if given) receives the
    // control block as it stands afterwards.
    int ensure_list(Ctrl* out = nullptr) {
        if (!state_set) return fail(ESPP_ERR_STATE, "no state set");
        if (d.mlp_on && mlp_bits.empty()) return fail(ESPP_ERR_STATE, "learned potential selected but no weights set");
        if (d.mlp_on && d.le_on) return fail(ESPP_ERR_STATE, "Lees-Edwards is not available with the learned potential");
        if (d.mlp_on && d.cells_mode) return fail(ESPP_ERR_STATE, "the learned potential needs the Verlet list");
        if (!cells_ready) return fail(ESPP_ERR_STATE, "call espp_build_neighbors first");
        int rcode = check_cutoffs();
        if (rcode) return rcode;
        rcode = ensure_mlp_buffers();
        if (rcode) return rcode;
        Ctrl c = read_ctrl();
        if (c.abort) return status_from(c);
        if (rebuild_pending || c.any_req) {
            rcode = rebuild_now(f_valid);
            if (rcode) return rcode;
            if (out) c = read_ctrl();
        }
        if (out) *out = c;
        return ESPP_OK;
    }

    int status_from(const Ctrl& c) {
        if (c.err & ERRBIT_BOND) return fail(ESPP_ERR_BOND_BROKEN, "a bond reached r >= R0 (FENE) or the end of its table (tabulated)");
        if (c.err & ERRBIT_NONFINITE) return fail(ESPP_ERR_NONFINITE, "a position became non-finite or left the box");
        if (c.err & ERRBIT_TIMEOUT) return fail(ESPP_ERR_TIMEOUT, "a device wait timed out");
        if (c.err & ERRBIT_ASYM) return fail(ESPP_ERR_STATE, "Verlet list is not symmetric");
        if (c.err & ERRBIT_OVERFLOW) return fail(ESPP_ERR_LIST_OVERFLOW, "Verlet list overflow");
        if (c.abort) return fail(ESPP_ERR_STATE, "aborted");
        return ESPP_OK;
    }

    int get_neighbors(int64_t* row_ptr, int64_t* cols, int64_t cap) override {
        if (!row_ptr) return fail(ESPP_ERR_ARG, "row_ptr is required");
        if (d.cells_mode) return fail(ESPP_ERR_STATE, "no Verlet list in the list-free force mode");
        int rcode = ensure_list();
        if (rcode) return rcode;
        const size_t n = (size_t)N;
        std::vector<int> cnt(n), nb((size_t)d.cap * d.stride);
        std::vector<V4<T>> vel(n);
        CK(cudaMemcpy(cnt.data(), d.nbr_cnt, n * sizeof(int), cudaMemcpyDeviceToHost));
        CK(cudaMemcpy(nb.data(), d.nbr, nb.size() * sizeof(int), cudaMemcpyDeviceToHost));
        CK(cudaMemcpy(vel.data(), d.vel, n * sizeof(V4<T>), cudaMemcpyDeviceToHost));
        std::vector<int> gid_of_slot(n);
        for (int r = 0; r < R; ++r)
            for (int s0 = rep_poff[r]; s0 < rep_poff[r] + rep_n[r]; ++s0) {
                int id;
                if (sizeof(T) == 4) memcpy(&id, &vel[s0].w, 4);
                else { long long l; memcpy(&l, &vel[s0].w, 8); id = (int)l; }
                gid_of_slot[s0] = rep_poff[r] + id;
            }
        std::vector<int> slot_of_gid(n);
        for (size_t s0 = 0; s0 < n; ++s0) slot_of_gid[gid_of_slot[s0]] = (int)s0;
        row_ptr[0] = 0;
        for (size_t g = 0; g < n; ++g) row_ptr[g + 1] = row_ptr[g] + cnt[slot_of_gid[g]];
        if (row_ptr[n] > cap || !cols) return fail(ESPP_ERR_ARG, "cols capacity too small");
        for (size_t g = 0; g < n; ++g) {
            const int s0 = slot_of_gid[g];
            int64_t* out = cols + row_ptr[g];
            for (int k = 0; k < cnt[s0]; ++k)
                out[k] = gid_of_slot[nb[4 * ((size_t)(k >> 2) * d.stride + s0) + (k & 3)] & NBR_INDEX_MASK];
            std::sort(out, out + cnt[s0]);
        }
        return ESPP_OK;
    }

    // ------------------------------------------------------------------ forces
    int compute_forces(double* f, int where) override {
        NvtxRange nvtx_range("espp_compute_forces");
        int rcode = ensure_list();
        if (rcode) return rcode;
        double* target = f;
        if (f && where == ESPP_HOST) target = d_io_x;
        else if (f && where != ESPP_DEVICE) return fail(ESPP_ERR_ARG, "bad where");
        launches += Launch<T>::step(d, MODE_FORCES, false, cur, target, 0, 0, st);
        CK(cudaGetLastError());
        if (f && where == ESPP_HOST)
            CK(cudaMemcpyAsync(f, d_io_x, 3 * (size_t)N * sizeof(double), cudaMemcpyDeviceToHost, st));
        CK(cudaStreamSynchronize(st));
        return status_from(read_ctrl());
    }

    // -------------------------------------------------------------- integrate
    int make_chunk(int S, int p0, bool final_chunk, ChunkGraph** out) {
        auto key = std::make_tuple(S, p0, final_chunk ? 1 : 0, timing ? 1 : 0);
        auto it = graphs.find(key);
        if (it != graphs.end()) {
            *out = &it->second;
            return ESPP_OK;
        }
        ChunkGraph cg;
        if (timing) {
            cg.ev.resize(3 * (size_t)S);
            for (auto& e : cg.ev) CK(cudaEventCreate(&e));
        }
        cudaStream_t cs = nullptr, bs = nullptr;
        CK(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
        CK(cudaStreamCreateWithFlags(&bs, cudaStreamNonBlocking));
        cudaGraph_t g;
        CK(cudaGraphCreate(&g, 0));
        std::vector<cudaGraphConditionalHandle> h(S);
        for (int r = 0; r < S; ++r) CK(cudaGraphConditionalHandleCreate(&h[r], g, 0, cudaGraphCondAssignDefault));
        CK(cudaStreamBeginCaptureToGraph(cs, g, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed));
        Launch<T>::set_cond(d, h[0], cs);
        int p = p0;
        for (int r = 0; r < S; ++r) {
            if (timing) CK(cudaEventRecordWithFlags(cg.ev[3 * r], cs, cudaEventRecordExternal));
            cudaStreamCaptureStatus status;
            cudaGraph_t capg;
            const cudaGraphNode_t* deps = nullptr;
            size_t nd = 0;
            CK(cudaStreamGetCaptureInfo(cs, &status, nullptr, &capg, &deps, nullptr, &nd));
            // the parameter struct holds a union without a default constructor
            alignas(cudaGraphNodeParams) unsigned char raw[sizeof(cudaGraphNodeParams)];
            memset(raw, 0, sizeof(raw));
            cudaGraphNodeParams& np = *reinterpret_cast<cudaGraphNodeParams*>(raw);
            np.type = cudaGraphNodeTypeConditional;
            np.conditional.handle = h[r];
            np.conditional.type = cudaGraphCondTypeIf;
            np.conditional.size = 1;
            cudaGraphNode_t node;
            CK(cudaGraphAddNode(&node, capg, deps, nullptr, nd, &np));
            cudaGraph_t body = np.conditional.phGraph_out[0];
            CK(cudaStreamUpdateCaptureDependencies(cs, &node, nullptr, 1, cudaStreamSetCaptureDependencies));
            CK(cudaStreamBeginCaptureToGraph(bs, body, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed));
            Launch<T>::rebuild(d, p, false, false, bs);
            cudaGraph_t tmp;
            CK(cudaStreamEndCapture(bs, &tmp));
            const bool last = r == S - 1;
            const int mode = (final_chunk && last) ? MODE_FINAL : MODE_STEP;
            if (timing) CK(cudaEventRecordWithFlags(cg.ev[3 * r + 1], cs, cudaEventRecordExternal));
            Launch<T>::step(d, mode, false, p, nullptr, last ? 0ull : (unsigned long long)h[r + 1], 0, cs);
            if (timing) CK(cudaEventRecordWithFlags(cg.ev[3 * r + 2], cs, cudaEventRecordExternal));
            if (mode == MODE_STEP) p ^= 1;
        }
        cudaGraph_t done;
        CK(cudaStreamEndCapture(cs, &done));
        cudaGraphExec_t ex;
        CK(cudaGraphInstantiate(&ex, done, 0));
        cudaStreamDestroy(cs);
        cudaStreamDestroy(bs);
        cg.graph = done;
        cg.exec = ex;
        auto ins = graphs.emplace(key, std::move(cg));
        *out = &ins.first->second;
        return ESPP_OK;
    }

    // timing mode: add the event-measured durations of the last replay of a chunk
    int harvest_timing(ChunkGraph* cg) {
        const size_t S = cg->ev.size() / 3;
        for (size_t r = 0; r < S; ++r) {
            float a = 0, b = 0;
            CK(cudaEventElapsedTime(&a, cg->ev[3 * r], cg->ev[3 * r + 1]));
            CK(cudaEventElapsedTime(&b, cg->ev[3 * r + 1], cg->ev[3 * r + 2]));
            t_rebuild_ms += a;
            t_step_ms += b;
            t_step_n += 1;
        }
        return ESPP_OK;
    }

    int set_kernel_timing(int enable) override {
        // the graphs with timing events are cached beside the plain ones
        timing = enable != 0;
        t_step_ms = t_rebuild_ms = 0;
        t_step_n = 0;
        return ESPP_OK;
    }

    int kernel_timing(double* out, int reset) override {
        out[0] = t_step_ms;
        out[1] = (double)t_step_n;
        out[2] = t_rebuild_ms;
        out[3] = (double)t_step_n;
        if (reset) {
            t_step_ms = t_rebuild_ms = 0;
            t_step_n = 0;
        }
        return ESPP_OK;
    }

    // Step counts of the captured graphs: the chunk limit itself and every
    // power of two below it.  Any run splits into these (largest first, cut at
    // the next resort) plus the final step, so one set of graphs serves every
    // nsteps and no call captures a graph once prepare_graphs has run.
    std::vector<int> chunk_sizes() const {
        std::vector<int> out;
        if (chunk > 0) out.push_back(chunk);
        for (int k = 1 << 10; k >= 1; k >>= 1)
            if (k < chunk) out.push_back(k);
        return out;
    }
    int chunk_size_for(int64_t avail) const {
        if (avail >= chunk) return chunk;
        int k = 1;
        while (2 * (int64_t)k <= avail) k <<= 1;
        return k;
    }

    // Capture and instantiate every graph a run can use (both position
    // buffers, every chunk size, the final step), so that integrate calls
    // after the first one on a configuration launch cached graphs only.
    int prepare_graphs() {
        if (chunk <= 0) return ESPP_OK;
        for (int p = 0; p < 2; ++p) {
            ChunkGraph* cg = nullptr;
            for (int S : chunk_sizes()) {
                int rcode = make_chunk(S, p, false, &cg);
                if (rcode) return rcode;
            }
            int rcode = make_chunk(1, p, true, &cg);
            if (rcode) return rcode;
        }
        return ESPP_OK;
    }

    int integrate(int64_t nsteps, double dt, double gamma, double kT) override {
        NvtxRange nvtx_range("espp_integrate");
        if (nsteps < 0 || !(dt > 0) || !(gamma >= 0) || !(kT >= 0) || !std::isfinite(dt) || !std::isfinite(gamma) ||
            !std::isfinite(kT))
            return fail(ESPP_ERR_ARG, "need nsteps >= 0 and finite dt > 0, gamma >= 0, kT >= 0");
        if (nsteps == 0) return ESPP_OK;
        Ctrl c0;
        int rcode = ensure_list(&c0);
        if (rcode) return rcode;
        if (d.dpd && !(dpd_rc <= rc_list * (1 + 1e-12)))
            return fail(ESPP_ERR_ARG, "the DPD cutoff exceeds the list cutoff");
        rcode = upload_int_params(dt, gamma, kT);
        if (rcode) return rcode;
        rcode = prepare_graphs();
        if (rcode) return rcode;
        const int64_t step0 = c0.step;
        const int64_t target = step0 + nsteps;
        const int64_t rb0 = c0.n_rebuilds;
        // the clock of this call: t(step0) carried over, this call's dt
        rcode = set_clock(time_at(step0), dt, step0);
        if (rcode) return rcode;
        if (!f_valid) {
            if (d.cells_mode && d.dpd) {
                // the DPD pair term reads the cell-ordered velocities: bin again
                Launch<T>::request_all(d, st);
                launches += 1 + Launch<T>::rebuild(d, cur, false, false, st);
            }
            launches += Launch<T>::step(d, MODE_INIT, false, cur, nullptr, 0, 0, st);
            f_valid = true;
        }
        const int c_start = cur;
        Launch<T>::prologue(d, cur, 0, st);
        launches++;
        CK(cudaGetLastError());
        int64_t done = step0;  // last completed step
        for (int attempt = 0; attempt < 8; ++attempt) {
            // positions of step done+1 live in buffer (1 - c_start) ^ ((done - step0) & 1)
            int p = (1 - c_start) ^ (int)((done - step0) & 1);
            int64_t next = done + 1;  // step the next graph computes first
            int64_t host_rebuilds = 0;  // rebuilds launched here rather than by graph nodes
            while (next <= target) {
                // Hilbert resort (with a list rebuild) before every step that is
                // a multiple of resort_every: a function of the step number only
                if (resort_every > 0 && next % resort_every == 0) {
                    Launch<T>::request_all(d, st);
                    launches += 1 + Launch<T>::rebuild(d, p, true, false, st);
                    host_rebuilds++;
                }
                // steps before the final one, up to the next resort
                int64_t avail = target - next;
                if (resort_every > 0) avail = std::min<int64_t>(avail, resort_every - (next % resort_every));
                const bool fin = avail == 0;  // only the final step is left
                if (chunk == 0) {
                    // direct launches (profilers cannot see kernels inside
                    // conditional graphs): early-exit rebuild kernels + step
                    host_rebuilds = -1;  // every kernel is counted as launched
                    const int64_t S = fin ? 1 : avail;
                    for (int64_t r = 0; r < S; ++r) {
                        launches += Launch<T>::rebuild(d, p, false, false, st);
                        launches += Launch<T>::step(d, fin ? MODE_FINAL : MODE_STEP, false, p, nullptr, 0ull, 0, st);
                        if (!fin) p ^= 1;
                    }
                    CK(cudaGetLastError());
                    next += S;
                    continue;
                }
                const int S = fin ? 1 : chunk_size_for(avail);
                ChunkGraph* cg = nullptr;
                rcode = make_chunk(S, p, fin, &cg);
                if (rcode) return rcode;
                CK(cudaGraphLaunch(cg->exec, st));
                launches += 1 + (int64_t)S * step_kernels();
                if (timing) {
                    // every replay is read back (a graph's events hold its last replay only)
                    CK(cudaStreamSynchronize(st));
                    rcode = harvest_timing(cg);
                    if (rcode) return rcode;
                }
                if (!fin) p ^= S & 1;
                next += S;
            }
            Ctrl c = read_ctrl();
            CK(cudaGetLastError());
            if (host_rebuilds >= 0)
                launches += (REBUILD_LAUNCHES - (d.cells_mode ? 1 : 0) + (d.mlp_on ? 5 : 0)) *
                            ((int64_t)(c.n_rebuilds - (unsigned)rb0) - host_rebuilds);
            if (c.err & (ERRBIT_BOND | ERRBIT_NONFINITE | ERRBIT_TIMEOUT)) return status_from(c);
            if (c.err & ERRBIT_OVERFLOW) {
                // frozen after step c.step with the positions of the next step in
                // buffer pm: grow, rebuild every replica there, go on
                done = c.step;
                const int pm = (1 - c_start) ^ (int)((done - step0) & 1);
                rcode = grow_capacity(c);
                if (rcode) return rcode;
                launches += Launch<T>::rebuild(d, pm, true, false, st);
                CK(cudaGetLastError());
                rcode = prepare_graphs();  // the grown list is a new kernel argument
                if (rcode) return rcode;
                continue;
            }
            if (c.step != target) return fail(ESPP_ERR_STATE, "step counter mismatch after integrate");
            cur = (1 - c_start) ^ (int)((nsteps - 1) & 1);
            return ESPP_OK;
        }
        return fail(ESPP_ERR_LIST_OVERFLOW, "Verlet list overflow persists after retries");
    }

    // ------------------------------------------------------------ observables
    int observables(espp_obs_t* out, int Rq) override {
        NvtxRange nvtx_range("espp_observables");
        if (!out || Rq < 1 || Rq > R) return fail(ESPP_ERR_ARG, "bad output");
        int rcode = ensure_list();
        if (rcode) return rcode;
        rcode = upload_int_params(ip_key[0] > 0 ? ip_key[0] : 1.0, std::max(ip_key[1], 0.0), std::max(ip_key[2], 0.0));
        if (rcode) return rcode;
        launches += Launch<T>::step(d, MODE_FORCES, true, cur, nullptr, 0, 0, st);
        Launch<T>::reduce_obs(d, d_obs, st);
        Launch<T>::rg2(d, cur, d_mol_members, d_mol_off, d_mol_rep, (int)mol_rep_h.size(), d_mol_rg2, st);
        launches += 2;
        CK(cudaGetLastError());
        std::vector<double> part((size_t)R * NPART), rg(mol_rep_h.size());
        CK(cudaMemcpyAsync(part.data(), d_obs, part.size() * sizeof(double), cudaMemcpyDeviceToHost, st));
        if (!rg.empty()) CK(cudaMemcpyAsync(rg.data(), d_mol_rg2, rg.size() * sizeof(double), cudaMemcpyDeviceToHost, st));
        Ctrl c = read_ctrl();
        CK(cudaGetLastError());
        std::vector<double> rgsum(R, 0.0);
        std::vector<int64_t> nmol(R, 0);
        for (size_t m = 0; m < rg.size(); ++m) {
            rgsum[mol_rep_h[m]] += rg[m];
            nmol[mol_rep_h[m]]++;
        }
        for (int r = 0; r < Rq; ++r) {
            const double* q = &part[(size_t)r * NPART];
            espp_obs_t& o = out[r];
            memset(&o, 0, sizeof(o));
            o.step = c.step;
            o.n = rep_n[r];
            o.ke = q[P_KE];
            o.pe_pair = q[P_PE_PAIR];
            o.pe_bond = q[P_PE_BOND];
            o.virial = q[P_VIRIAL];
            o.px = q[P_PX];
            o.py = q[P_PY];
            o.pz = q[P_PZ];
            o.temperature = 2.0 * o.ke / (3.0 * rep_n[r]);
            const double V = box[3 * r] * box[3 * r + 1] * box[3 * r + 2];
            o.pressure = (2.0 * o.ke + o.virial) / (3.0 * V);
            o.pxz = (q[P_KIN_XZ] + q[P_VIR_XZ]) / V;
            o.mean_bond = q[P_BOND_CNT] > 0 ? q[P_BOND_LEN] / q[P_BOND_CNT] : 0.0;
            o.rg2 = nmol[r] > 0 ? rgsum[r] / nmol[r] : 0.0;
            o.n_molecules = nmol[r];
            o.n_rebuilds = c.n_rebuilds;
            o.error_word = c.err;
        }
        return ESPP_OK;
    }

    int rdf_counts(int rep, double rmax, int nbins, int64_t* counts) override {
        if (rep < 0 || rep >= R || nbins < 1 || !(rmax > 0) || !counts) return fail(ESPP_ERR_ARG, "bad rdf arguments");
        for (int c = 0; c < 3; ++c)
            if (rmax >= 0.5 * box[3 * rep + c]) return fail(ESPP_ERR_ARG, "rmax must be below half the box");
        if (!state_set) return fail(ESPP_ERR_STATE, "no state set");
        if (nbins > 12288) return fail(ESPP_ERR_ARG, "too many bins");
        if (hist_cap < nbins) {
            if (d_hist) cudaFree(d_hist);
            d_hist = nullptr;
            hist_cap = 0;
            CK(cudaMalloc(&d_hist, nbins * sizeof(unsigned long long)));
            hist_cap = nbins;
        }
        CK(cudaMemsetAsync(d_hist, 0, nbins * sizeof(unsigned long long), st));
        // from the Verlet list when it reaches far enough (with 1-2
        // exclusions on, bonded pairs are then not counted), else all pairs
        const double rl = rc_list + skin;
        bool use_list = false;
        if (cells_ready && rmax <= rl && !d.cells_mode) {
            int rcode = ensure_list();
            if (rcode) return rcode;
            use_list = true;
        }
        if (use_list) Launch<T>::rdf_list(d, cur, rep, rmax, nbins, d_hist, st);
        else if (rep_n[rep] > 200000) return fail(ESPP_ERR_ARG, "all-pairs histogram of a replica this large; use rmax <= rc + skin");
        else Launch<T>::rdf(d, cur, rep, rmax, nbins, d_hist, st);
        launches++;
        CK(cudaGetLastError());
        std::vector<unsigned long long> h(nbins);
        CK(cudaMemcpyAsync(h.data(), d_hist, nbins * sizeof(unsigned long long), cudaMemcpyDeviceToHost, st));
        CK(cudaStreamSynchronize(st));
        for (int b = 0; b < nbins; ++b) counts[b] = (int64_t)h[b];
        return ESPP_OK;
    }

    // ------------------------------------------------------------- checkpoint
    // File layout: header, per replica (box, n, seed), then the storage-order
    // arrays (positions, velocities, force, build positions, images, bond
    // slots, slot of every id), the pending rebuild requests and the
    // Lees-Edwards build offsets of every replica.  Loading puts
    // every array back in the same order and rebuilds the Verlet list from the
    // build positions, so the list equals the one of the saved run.
    struct CkptHeader {
        char magic[8];
        int32_t version, precision, R, f_valid;
        int64_t N, step, n_rebuilds;
        double rc_list, skin;
        int32_t le_on, pad;
        double le_shear, le_time, le_dt;  // Lees-Edwards setting and the simulated time
    };

    template <class P>
    int dl(std::vector<P>& h, const P* dptr, size_t n) {
        h.resize(n);
        CK(cudaMemcpy(h.data(), dptr, n * sizeof(P), cudaMemcpyDeviceToHost));
        return ESPP_OK;
    }
    template <class P>
    int ul(P* dptr, const std::vector<P>& h) {
        CK(cudaMemcpy(dptr, h.data(), h.size() * sizeof(P), cudaMemcpyHostToDevice));
        return ESPP_OK;
    }

    int checkpoint_save(const char* path) override {
        NvtxRange nvtx_range("espp_checkpoint_save");
        if (!path) return fail(ESPP_ERR_ARG, "path is required");
        if (!state_set) return fail(ESPP_ERR_STATE, "no state set");
        CK(cudaStreamSynchronize(st));
        Ctrl c = read_ctrl();
        if (c.abort) return status_from(c);
        CkptHeader hd;
        memset(&hd, 0, sizeof(hd));
        memcpy(hd.magic, "ESPPCKP2", 8);
        hd.version = 2;
        hd.precision = sizeof(T) == 4 ? ESPP_FP32 : ESPP_FP64;
        hd.R = R;
        hd.f_valid = f_valid ? 1 : 0;
        hd.N = N;
        hd.step = c.step;
        hd.n_rebuilds = c.n_rebuilds;
        hd.rc_list = rc_list;
        hd.skin = skin;
        hd.le_on = d.le_on;
        hd.le_shear = d.le_shear;
        hd.le_time = time_at(c.step);
        hd.le_dt = le_clk_h.dt;
        const size_t n = (size_t)N;
        std::vector<V4<T>> pos, vel, frc, xb;
        std::vector<int4> img;
        std::vector<int2> bs;
        std::vector<int> sid, req;
        std::vector<double> ledb;
        int rcode;
        // the list-free mode keeps no build positions: the positions, binned
        // at this step, serve (a handle with a list rebuilds from them)
        if ((rcode = dl(pos, d.pos[cur], n)) || (rcode = dl(vel, d.vel, n)) || (rcode = dl(frc, d.frc, n)) ||
            (rcode = dl(xb, d.cells_mode ? d.pos[cur] : d.xb, n)) || (rcode = dl(img, d.img, n)) ||
            (rcode = dl(bs, d.bond_slot, n)) ||
            (rcode = dl(sid, d.slot_of_id, n)) || (rcode = dl(req, d.req, (size_t)R)) ||
            (rcode = dl(ledb, d.le_db, (size_t)R)))
            return rcode;
        FILE* fh = fopen(path, "wb");
        if (!fh) return fail(ESPP_ERR_IO, std::string("cannot open ") + path);
        bool ok = fwrite(&hd, sizeof(hd), 1, fh) == 1;
        for (int r = 0; r < R && ok; ++r) {
            const int64_t nr = rep_n[r];
            ok = fwrite(&box[3 * r], sizeof(double), 3, fh) == 3 && fwrite(&nr, sizeof(nr), 1, fh) == 1 &&
                 fwrite(&seeds[r], sizeof(seeds[r]), 1, fh) == 1;
        }
        auto wr = [&](const void* p, size_t bytes) { ok = ok && fwrite(p, 1, bytes, fh) == bytes; };
        wr(pos.data(), n * sizeof(V4<T>));
        wr(vel.data(), n * sizeof(V4<T>));
        wr(frc.data(), n * sizeof(V4<T>));
        wr(xb.data(), n * sizeof(V4<T>));
        wr(img.data(), n * sizeof(int4));
        wr(bs.data(), n * sizeof(int2));
        wr(sid.data(), n * sizeof(int));
        wr(req.data(), (size_t)R * sizeof(int));
        wr(ledb.data(), (size_t)R * sizeof(double));
        ok = (fclose(fh) == 0) && ok;
        return ok ? ESPP_OK : fail(ESPP_ERR_IO, std::string("write failed: ") + path);
    }

    int checkpoint_load(const char* path) override {
        NvtxRange nvtx_range("espp_checkpoint_load");
        if (!path) return fail(ESPP_ERR_ARG, "path is required");
        if (!cells_ready) return fail(ESPP_ERR_STATE, "call espp_build_neighbors before loading");
        FILE* fh = fopen(path, "rb");
        if (!fh) return fail(ESPP_ERR_IO, std::string("cannot open ") + path);
        CkptHeader hd;
        bool ok = fread(&hd, sizeof(hd), 1, fh) == 1 && memcmp(hd.magic, "ESPPCKP2", 8) == 0;
        if (!ok) {
            fclose(fh);
            return fail(ESPP_ERR_IO, "not a checkpoint file");
        }
        if (hd.precision != (sizeof(T) == 4 ? ESPP_FP32 : ESPP_FP64) || hd.R != R || hd.N != N) {
            fclose(fh);
            return fail(ESPP_ERR_ARG, "checkpoint does not match this handle (precision, replicas, size)");
        }
        // the handle changes only once the whole file has been read and checked
        std::vector<unsigned long long> sds((size_t)R);
        for (int r = 0; r < R && ok; ++r) {
            double b[3];
            int64_t nr;
            ok = fread(b, sizeof(double), 3, fh) == 3 && fread(&nr, sizeof(nr), 1, fh) == 1 &&
                 fread(&sds[r], sizeof(sds[r]), 1, fh) == 1;
            if (ok && (nr != rep_n[r] || b[0] != box[3 * r] || b[1] != box[3 * r + 1] || b[2] != box[3 * r + 2])) {
                fclose(fh);
                return fail(ESPP_ERR_ARG, "checkpoint replica geometry differs from this handle");
            }
        }
        const size_t n = (size_t)N;
        std::vector<V4<T>> pos(n), vel(n), frc(n), xb(n);
        std::vector<int4> img(n);
        std::vector<int2> bs(n);
        std::vector<int> sid(n), req((size_t)R);
        std::vector<double> ledb((size_t)R);
        auto rd = [&](void* p, size_t bytes) { ok = ok && fread(p, 1, bytes, fh) == bytes; };
        rd(pos.data(), n * sizeof(V4<T>));
        rd(vel.data(), n * sizeof(V4<T>));
        rd(frc.data(), n * sizeof(V4<T>));
        rd(xb.data(), n * sizeof(V4<T>));
        rd(img.data(), n * sizeof(int4));
        rd(bs.data(), n * sizeof(int2));
        rd(sid.data(), n * sizeof(int));
        rd(req.data(), (size_t)R * sizeof(int));
        rd(ledb.data(), (size_t)R * sizeof(double));
        fclose(fh);
        if (!ok) return fail(ESPP_ERR_IO, "checkpoint file is truncated");
        if (hd.le_on && d.mlp_on) return fail(ESPP_ERR_STATE, "Lees-Edwards is not available with the learned potential");
        CK(cudaStreamSynchronize(st));
        for (int r = 0; r < R; ++r) seeds[r] = sds[r];
        int rcode = upload_geometry();  // seeds
        if (rcode) return rcode;
        cur = 0;
        if ((rcode = ul(d.pos[0], pos)) || (rcode = ul(d.pos[1], xb)) || (rcode = ul(d.vel, vel)) ||
            (rcode = ul(d.frc, frc)) || (rcode = ul(d.xb, xb)) || (rcode = ul(d.img, img)) ||
            (rcode = ul(d.bond_slot, bs)) || (rcode = ul(d.slot_of_id, sid)) || (rcode = ul(d.le_db, ledb)))
            return rcode;
        // Lees-Edwards setting and clock of the saved run
        d.le_on = hd.le_on;
        d.le_shear = hd.le_shear;
        clear_graphs();
        rcode = set_clock(hd.le_time, hd.le_dt, hd.step);
        if (rcode) return rcode;
        Ctrl c = read_ctrl();
        c.step = hd.step;
        c.pos_ahead = 0;
        c.le_keep = 1;  // the list below is rebuilt with the saved build offsets
        c.err = 0;
        c.abort = 0;
        c.any_req = 0;
        c.blocks_done = 0;
        c.need_cap = 0;
        CK(cudaMemcpy(d_ctrl, &c, sizeof(Ctrl), cudaMemcpyHostToDevice));
        // the list of the saved run was built from the build positions: rebuild
        // it from them (buffer 1 holds a copy), without a resort
        // (list-free mode: bin the saved positions, which the last step binned)
        Launch<T>::request_all(d, st);
        launches += 1 + Launch<T>::rebuild(d, d.cells_mode ? 0 : 1, false, false, st);
        CK(cudaGetLastError());
        rebuild_pending = false;  // the loaded state is complete
        c = read_ctrl();
        if (c.err & ERRBIT_OVERFLOW) return fail(ESPP_ERR_LIST_OVERFLOW, "list capacity too small for the checkpoint");
        // restore the pending requests and the rebuild counter of the saved run
        CK(cudaMemcpy(d.req, req.data(), (size_t)R * sizeof(int), cudaMemcpyHostToDevice));
        int any = 0;
        for (int v : req) any |= v != 0;
        c.any_req = any;
        c.n_rebuilds = (unsigned int)hd.n_rebuilds;
        CK(cudaMemcpy(d_ctrl, &c, sizeof(Ctrl), cudaMemcpyHostToDevice));
        state_set = true;
        f_valid = hd.f_valid != 0;
        rebuild_pending = false;
        return ESPP_OK;
    }

    // ------------------------------------------------------------ diagnostics
    uint32_t error_word() override { return read_ctrl().err; }
    int64_t num_particles() override { return N; }
    int32_t num_replicas() override { return R; }
    int64_t num_rebuilds() override { return read_ctrl().n_rebuilds; }
    int64_t step() override { return read_ctrl().step; }
    int32_t list_capacity() override { return d.cap; }
    int64_t kernel_launches() override { return launches; }
    int list_stats(int64_t* total, int32_t* maxc) override {
        if (d.cells_mode) {
            // no list is built in the list-free mode
            if (total) *total = 0;
            if (maxc) *maxc = 0;
            return ESPP_OK;
        }
        int rcode = ensure_list();
        if (rcode) return rcode;
        std::vector<int> cnt((size_t)N);
        CK(cudaMemcpy(cnt.data(), d.nbr_cnt, (size_t)N * sizeof(int), cudaMemcpyDeviceToHost));
        int64_t t = 0;
        int m = 0;
        for (int c : cnt) {
            t += c;
            m = std::max(m, c);
        }
        if (total) *total = t;
        if (maxc) *maxc = m;
        return ESPP_OK;
    }

    int set_resort_interval(int64_t steps) override {
        if (steps < 0) return fail(ESPP_ERR_ARG, "resort interval must be >= 0");
        resort_every = steps;
        return ESPP_OK;
    }

    int set_thermostat(int kind, double rc) override {
        if (kind == ESPP_THERMO_LANGEVIN) {
            d.dpd = 0;
        } else if (kind == ESPP_THERMO_DPD) {
            if (!(rc > 0) || !std::isfinite(rc)) return fail(ESPP_ERR_ARG, "the DPD cutoff must be > 0");
            if (!d.vsnap) {
                const int rb = alloc(&d.vsnap, (size_t)N, allocs);
                if (rb) return rb;
            }
            d.dpd = 1;
            dpd_rc = rc;
        } else {
            return fail(ESPP_ERR_ARG, "unknown thermostat kind");
        }
        clear_graphs();   // the thermostat is a template argument of captured kernels
        mass_dirty = true;  // the DPD constants live in the integrator parameters
        f_valid = false;
        return ESPP_OK;
    }

    // kernels of one step inside the step graphs (Launch::step)
    int step_kernels() const {
        // the learned potential: stage + tile + gather (FP32), one kernel (FP64)
        int k = 1 + (d.mlp_on ? (sizeof(T) == 8 ? 1 : 3) : 0);
        if (d.cells_mode) k += 1;  // cell-stencil forces
        else if (d.dpd) k += 1;    // velocity snapshot
        return k;
    }

    // ------------------------------------------------------- force method
    int set_force_method(int method) override {
        if (method != ESPP_FORCES_VERLET && method != ESPP_FORCES_CELLS)
            return fail(ESPP_ERR_ARG, "unknown force method");
        const int cells = method == ESPP_FORCES_CELLS ? 1 : 0;
        if (cells && d.mlp_on) return fail(ESPP_ERR_STATE, "the learned potential needs the Verlet list");
        if (cells && cell_sub_req == 3) return fail(ESPP_ERR_ARG, "the list-free mode takes whole or half cells");
        if (cells == d.cells_mode) return ESPP_OK;
        if (cells && !d.cpf) {
            int rc;
            if ((rc = alloc(&d.cpf, (size_t)N, allocs)) || (rc = alloc(&d.cpv, (size_t)N, allocs)) ||
                (rc = alloc(&d.cell_vel, (size_t)N, allocs)))
                return rc;
        }
        d.cells_mode = cells;
        CK(upload_params());  // the fast Lennard-Jones variant is for the list
        clear_graphs();
        f_valid = false;
        // the cells' edge depends on the method (the list's skin is no part of it)
        return cells_ready ? build_neighbors(rc_list, skin) : ESPP_OK;
    }

    // Times nsteps steps of each candidate shape from the current state and
    // keeps the fastest: the Verlet list over whole, half or third cells, the
    // list-free cell forces (whole cells).  The state is
    // then restored through set_state (so the next integrate recomputes the
    // force of the current step); a candidate whose cells do not fit the box
    // is skipped.  The subdivision request of the caller is replaced.
    int tune_force_method(int nsteps, double dt, double gamma, double kT, double* ms, int* chosen) override {
        NvtxRange nvtx_range("espp_tune_force_method");
        if (nsteps < 1) return fail(ESPP_ERR_ARG, "nsteps must be positive");
        if (!state_set || !cells_ready) return fail(ESPP_ERR_STATE, "set the state and build the cells first");
        const size_t n3 = 3 * (size_t)N;
        std::vector<double> x(n3), v(n3);
        std::vector<int32_t> img(n3);
        int rcode = get_state(x.data(), v.data(), img.data(), ESPP_HOST);
        if (rcode) return rcode;
        const int64_t step0 = read_ctrl().step;
        const double t0 = time_at(step0), dt0 = le_clk_h.dt;
        auto restore = [&]() -> int {
            int rc = set_state(x.data(), v.data(), img.data(), ESPP_HOST);
            if (rc) return rc;
            if ((rc = set_step(step0))) return rc;
            return set_clock(t0, dt0, step0);
        };
        constexpr int NSH = ESPP_FORCE_SHAPES;
        const int method_of[NSH] = {ESPP_FORCES_VERLET, ESPP_FORCES_VERLET, ESPP_FORCES_VERLET,
                                    ESPP_FORCES_CELLS,  ESPP_FORCES_VERLET, ESPP_FORCES_VERLET};
        const int w_of[NSH] = {1, 2, 3, 1, 1, 3};
        const int push_of[NSH] = {0, 0, 0, 0, 1, 1};
        auto apply = [&](int k) -> int {
            // the subdivision and the list store first (the list-free shape
            // takes whole cells), then the method (a change of method
            // rebuilds the grid)
            cell_sub_req = w_of[k];
            int rc = set_list_store(push_of[k]);
            if (rc) return rc;
            if ((rc = set_force_method(method_of[k]))) return rc;
            return build_neighbors(rc_list, skin);
        };
        double t[NSH];
        for (double& q : t) q = INFINITY;
        cudaEvent_t e0, e1;
        CK(cudaEventCreate(&e0));
        CK(cudaEventCreate(&e1));
        for (int k = 0; k < NSH && !rcode; ++k) {
            if (method_of[k] == ESPP_FORCES_CELLS && d.mlp_on) continue;
            const int rc = apply(k);
            if (rc == ESPP_ERR_BOX_TOO_SMALL) continue;  // this shape does not fit
            if ((rcode = rc) || (rcode = restore()) || (rcode = integrate(2, dt, gamma, kT))) break;
            CK(cudaEventRecord(e0, st));
            rcode = integrate(nsteps, dt, gamma, kT);
            if (rcode) break;
            CK(cudaEventRecord(e1, st));
            CK(cudaEventSynchronize(e1));
            float el = 0;
            CK(cudaEventElapsedTime(&el, e0, e1));
            t[k] = el / nsteps;
        }
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        if (rcode) return rcode;
        int best = 0;
        for (int k = 1; k < NSH; ++k)
            if (t[k] < t[best]) best = k;
        if (!std::isfinite(t[best])) return fail(ESPP_ERR_BOX_TOO_SMALL, "no cell shape fits the box");
        if ((rcode = apply(best)) || (rcode = restore())) return rcode;
        if (ms)
            for (int k = 0; k < NSH; ++k) ms[k] = t[k];
        if (chosen) *chosen = best;
        return ESPP_OK;
    }

    // ---- H5MD files ----------------------------------------------------------
    int h5md_write(const char* path) override {
        NvtxRange nvtx_range("espp_h5md_write");
        if (!path) return fail(ESPP_ERR_ARG, "path is required");
        if (!state_set) return fail(ESPP_ERR_STATE, "no state set");
        const size_t n3 = 3 * (size_t)N;
        std::vector<double> x(n3), v(n3);
        std::vector<int32_t> img(n3);
        int rcode = get_state(x.data(), v.data(), img.data(), ESPP_HOST);
        if (rcode) return rcode;
        // the stored total force of this step, when there is one: velocity
        // Verlet starts the next step from it (its Langevin friction was taken
        // at the half-step velocity, which the file does not hold otherwise)
        std::vector<double> f;
        if (f_valid) {
            f.resize(n3);
            Launch<T>::get_state(d, nullptr, nullptr, nullptr, d_io_x, cur, st);
            launches++;
            CK(cudaGetLastError());
            CK(cudaMemcpyAsync(f.data(), d_io_x, n3 * sizeof(double), cudaMemcpyDeviceToHost, st));
            CK(cudaStreamSynchronize(st));
        }
        const Ctrl c = read_ctrl();
        H5mdState hs;
        hs.step = c.step;
        hs.time = time_at(c.step);
        hs.precision = sizeof(T) == 4 ? ESPP_FP32 : ESPP_FP64;
        hs.lees_edwards = d.le_on;
        hs.shear_rate = d.le_shear;
        hs.reps.resize(R);
        for (int r = 0; r < R; ++r) {
            H5mdReplica& rp = hs.reps[r];
            const int off = rep_poff[r], n = rep_n[r];
            for (int k = 0; k < 3; ++k) rp.box[k] = box[3 * r + k];
            rp.n = n;
            rp.x.assign(x.begin() + 3 * (size_t)off, x.begin() + 3 * (size_t)(off + n));
            rp.v.assign(v.begin() + 3 * (size_t)off, v.begin() + 3 * (size_t)(off + n));
            rp.img.assign(img.begin() + 3 * (size_t)off, img.begin() + 3 * (size_t)(off + n));
            if (f_valid) rp.f.assign(f.begin() + 3 * (size_t)off, f.begin() + 3 * (size_t)(off + n));
            rp.species.assign(types_gid.begin() + off, types_gid.begin() + off + n);
            for (int a = 0; a < n; ++a) {
                const int2 b = bond_gid_h[off + a];
                for (int o : {b.x, b.y})
                    if (o > off + a) {
                        rp.bonds.push_back(a);
                        rp.bonds.push_back(o - off);
                    }
            }
            rp.seed = seeds[r];
        }
        std::string err;
        if (espp::h5md_write(path, hs, err)) return fail(ESPP_ERR_IO, "H5MD write: " + err);
        return ESPP_OK;
    }

    int h5md_read(const char* path) override {
        NvtxRange nvtx_range("espp_h5md_read");
        if (!path) return fail(ESPP_ERR_ARG, "path is required");
        H5mdState hs;
        std::string err;
        if (espp::h5md_read(path, hs, err)) return fail(ESPP_ERR_IO, "H5MD read: " + err);
        if ((int)hs.reps.size() != R) return fail(ESPP_ERR_ARG, "the file holds another number of replicas");
        const size_t n3 = 3 * (size_t)N;
        std::vector<double> x, v, f;
        std::vector<int32_t> img;
        x.reserve(n3);
        v.reserve(n3);
        img.reserve(n3);
        const bool with_f = !hs.reps.empty() && !hs.reps[0].f.empty();
        for (int r = 0; r < R; ++r) {
            const H5mdReplica& rp = hs.reps[r];
            if (rp.f.empty() == with_f) return fail(ESPP_ERR_IO, "H5MD read: a force element in some replicas only");
            f.insert(f.end(), rp.f.begin(), rp.f.end());
            if (rp.n != rep_n[r]) return fail(ESPP_ERR_ARG, "a replica of the file has another particle count");
            for (int k = 0; k < 3; ++k)
                if (rp.box[k] != box[3 * r + k]) return fail(ESPP_ERR_ARG, "a replica of the file has another box");
            for (int a = 0; a < rep_n[r]; ++a)
                if (rp.species[a] != types_gid[rep_poff[r] + a])
                    return fail(ESPP_ERR_ARG, "the file's particle types differ from the handle's");
            x.insert(x.end(), rp.x.begin(), rp.x.end());
            v.insert(v.end(), rp.v.begin(), rp.v.end());
            img.insert(img.end(), rp.img.begin(), rp.img.end());
        }
        if (hs.lees_edwards != d.le_on || (d.le_on && hs.shear_rate != d.le_shear))
            return fail(ESPP_ERR_ARG, "the file's Lees-Edwards setting differs from the handle's");
        // the Philox seeds, step and clock of the file, then the particles
        // (wrapped under the clock of the saved step)
        CK(cudaStreamSynchronize(st));
        for (int r = 0; r < R; ++r) seeds[r] = hs.reps[r].seed;
        int rcode = upload_geometry();
        if (rcode) return rcode;
        const long long step = hs.step;
        CK(cudaMemcpyAsync(&d_ctrl->step, &step, sizeof(long long), cudaMemcpyHostToDevice, st));
        CK(cudaStreamSynchronize(st));
        if ((rcode = set_clock(hs.time, le_clk_h.dt, hs.step))) return rcode;
        if ((rcode = set_state(x.data(), v.data(), img.data(), ESPP_HOST))) return rcode;
        if (with_f) {
            CK(cudaMemcpyAsync(d_io_x, f.data(), n3 * sizeof(double), cudaMemcpyHostToDevice, st));
            Launch<T>::set_force(d, d_io_x, st);
            launches++;
            CK(cudaGetLastError());
            CK(cudaStreamSynchronize(st));
            f_valid = true;
        }
        return ESPP_OK;
    }

    // ---- launch shape of the step kernel and the resort interval ----------
    int set_step_shape(int shape) override {
        if (shape < 0 || shape >= ESPP_STEP_SHAPES) return fail(ESPP_ERR_ARG, "unknown step shape");
        d.step_shape = shape;
        clear_graphs();  // a kernel argument of the captured graphs
        return ESPP_OK;
    }

    int set_list_store(int push) override {
        if (push != ESPP_LIST_STORE_PLACE && push != ESPP_LIST_STORE_PUSH)
            return fail(ESPP_ERR_ARG, "unknown list store");
        d.list_push = push;
        clear_graphs();  // a kernel argument of the captured graphs
        return ESPP_OK;
    }

    // Times the step-kernel shapes, then the resort intervals, from the
    // current state (restored after each trial and at the end), keeping the
    // fastest of each.
    int tune_step_shape(int nsteps, double dt, double gamma, double kT, double* ms, int* chosen) override {
        NvtxRange nvtx_range("espp_tune_step_shape");
        if (nsteps < 1) return fail(ESPP_ERR_ARG, "nsteps must be positive");
        if (!state_set || !cells_ready) return fail(ESPP_ERR_STATE, "set the state and build the cells first");
        const size_t n3 = 3 * (size_t)N;
        std::vector<double> x(n3), v(n3);
        std::vector<int32_t> img(n3);
        int rcode = get_state(x.data(), v.data(), img.data(), ESPP_HOST);
        if (rcode) return rcode;
        const int64_t step0 = read_ctrl().step;
        const double t0 = time_at(step0), dt0 = le_clk_h.dt;
        auto restore = [&]() -> int {
            int rc = set_state(x.data(), v.data(), img.data(), ESPP_HOST);
            if (rc) return rc;
            if ((rc = set_step(step0))) return rc;
            return set_clock(t0, dt0, step0);
        };
        cudaEvent_t e0, e1;
        CK(cudaEventCreate(&e0));
        CK(cudaEventCreate(&e1));
        auto timed = [&](int steps, double* out) -> int {
            int rc;
            if ((rc = restore()) || (rc = integrate(2, dt, gamma, kT))) return rc;
            CK(cudaEventRecord(e0, st));
            if ((rc = integrate(steps, dt, gamma, kT))) return rc;
            CK(cudaEventRecord(e1, st));
            CK(cudaEventSynchronize(e1));
            float el = 0;
            CK(cudaEventElapsedTime(&el, e0, e1));
            *out = el / steps;
            return ESPP_OK;
        };
        const int resort_of[3] = {250, 500, 1000};
        double t[ESPP_STEP_SHAPES + 3];
        for (double& q : t) q = INFINITY;
        int best = 0, best_r = 1;
        for (int k = 0; k < ESPP_STEP_SHAPES && !rcode; ++k)
            if (!(rcode = set_step_shape(k))) rcode = timed(nsteps, &t[k]);
        if (!rcode) {
            for (int k = 1; k < ESPP_STEP_SHAPES; ++k)
                if (t[k] < t[best]) best = k;
            rcode = set_step_shape(best);
        }
        const int64_t resort0 = resort_every;
        for (int k = 0; k < 3 && !rcode; ++k) {
            resort_every = resort_of[k];
            rcode = timed(std::max(nsteps, 1000), &t[ESPP_STEP_SHAPES + k]);
        }
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        if (rcode) {
            resort_every = resort0;
            return rcode;
        }
        for (int k = 1; k < 3; ++k)
            if (t[ESPP_STEP_SHAPES + k] < t[ESPP_STEP_SHAPES + best_r]) best_r = k;
        resort_every = resort_of[best_r];
        if ((rcode = restore())) return rcode;
        if (ms)
            for (int k = 0; k < ESPP_STEP_SHAPES + 3; ++k) ms[k] = t[k];
        if (chosen) {
            chosen[0] = best;
            chosen[1] = resort_of[best_r];
        }
        return ESPP_OK;
    }

    int set_cell_subdivision(int w) override {
        if (w < 0 || w > 3) return fail(ESPP_ERR_ARG, "cell subdivision must be 0, 1, 2 or 3");
        if (w == 3 && d.cells_mode) return fail(ESPP_ERR_ARG, "the list-free mode takes whole or half cells");
        cell_sub_req = w;
        // an existing grid is rebuilt with the new cells
        return cells_ready ? build_neighbors(rc_list, skin) : ESPP_OK;
    }

    int set_chunk(int steps) override {
        if (steps < 0 || steps > 1024) return fail(ESPP_ERR_ARG, "chunk must be in [0, 1024]");
        chunk = steps;
        clear_graphs();
        return ESPP_OK;
    }
};

}  // namespace espp

struct espp_system {
    std::unique_ptr<espp::SystemBase> impl;
    std::string create_msg;
};

static thread_local std::string g_create_error;

template <class F>
static int guarded(espp_h h, F&& f) {
    if (!h || !h->impl) return ESPP_ERR_ARG;
    // a failed runtime call elsewhere in this thread leaves a non-sticky
    // "last error" behind; drop it so launch checks see only our launches
    (void)cudaGetLastError();
    try {
        return f(*h->impl);
    } catch (const std::exception& e) {
        h->impl->msg = e.what();
        return ESPP_ERR_STATE;
    }
}

extern "C" {

int espp_batch_create(int32_t R, const espp_replica_desc* descs, int precision, void* stream, espp_h* out) {
    if (!out || R < 1 || !descs) {
        g_create_error = "invalid arguments";
        return ESPP_ERR_ARG;
    }
    *out = nullptr;
    std::unique_ptr<espp_system> h(new espp_system());
    int rc;
    if (precision == ESPP_FP32) {
        auto* s = new espp::System<float>();
        h->impl.reset(s);
        rc = s->create(R, descs, (cudaStream_t)stream);
    } else if (precision == ESPP_FP64) {
        auto* s = new espp::System<double>();
        h->impl.reset(s);
        rc = s->create(R, descs, (cudaStream_t)stream);
    } else {
        g_create_error = "precision must be ESPP_FP32 or ESPP_FP64";
        return ESPP_ERR_ARG;
    }
    if (rc != ESPP_OK) {
        g_create_error = h->impl->msg;
        return rc;
    }
    *out = h.release();
    return ESPP_OK;
}

int espp_system_create(const double box[3], int64_t n, const int32_t* types, int64_t n_bonds,
                       const int64_t* bonds, int precision, uint64_t seed, void* stream, espp_h* out) {
    if (!box) return ESPP_ERR_ARG;
    espp_replica_desc d;
    d.box[0] = box[0];
    d.box[1] = box[1];
    d.box[2] = box[2];
    d.n = n;
    d.types = types;
    d.n_bonds = n_bonds;
    d.bonds = bonds;
    d.seed = seed;
    return espp_batch_create(1, &d, precision, stream, out);
}

int espp_system_destroy(espp_h h) {
    if (!h) return ESPP_ERR_ARG;
    delete h;
    return ESPP_OK;
}

int espp_set_state(espp_h h, const double* x, const double* v, const int32_t* img, int where) {
    return guarded(h, [&](espp::SystemBase& s) { return s.set_state(x, v, img, where); });
}
int espp_get_state(espp_h h, double* x, double* v, int32_t* img, int where) {
    return guarded(h, [&](espp::SystemBase& s) { return s.get_state(x, v, img, where); });
}
int espp_set_step(espp_h h, int64_t step) {
    return guarded(h, [&](espp::SystemBase& s) { return s.set_step(step); });
}
int espp_set_interaction(espp_h h, int kind, int ta, int tb, const double* p, int64_t np) {
    return guarded(h, [&](espp::SystemBase& s) { return s.set_interaction(kind, ta, tb, p, np); });
}
int espp_mlp_set_weights(espp_h h, const uint16_t* bf16, int64_t n) {
    return guarded(h, [&](espp::SystemBase& s) { return s.mlp_set_weights(bf16, n); });
}
int espp_cg_map(espp_h h, int32_t beads_per_site, double* x_sites, double* f_sites) {
    return guarded(h, [&](espp::SystemBase& s) { return s.cg_map(beads_per_site, x_sites, f_sites); });
}
int espp_mlp_get_weights(espp_h h, uint16_t* bf16, int64_t n) {
    return guarded(h, [&](espp::SystemBase& s) { return s.mlp_get_weights(bf16, n); });
}
int espp_mlp_train(espp_h h, const double* frames_x, const double* frames_f, int32_t nframes,
                   int32_t batch_frames, int32_t epochs, double lr, uint64_t shuffle_seed, double* loss_history) {
    return guarded(h, [&](espp::SystemBase& s) {
        return s.mlp_train(frames_x, frames_f, nframes, batch_frames, epochs, lr, shuffle_seed, loss_history, nullptr);
    });
}
int espp_mlp_loss_grad(espp_h h, const double* frames_x, const double* frames_f, int32_t nframes, double* loss,
                       float* grad) {
    return guarded(h, [&](espp::SystemBase& s) {
        return s.mlp_train(frames_x, frames_f, nframes, 0, 0, 0.0, 0, loss, grad);
    });
}
int espp_set_exclude_bonded(espp_h h, int on) {
    return guarded(h, [&](espp::SystemBase& s) { return s.set_exclude_bonded(on); });
}
int espp_set_mass(espp_h h, int type, double m) {
    return guarded(h, [&](espp::SystemBase& s) { return s.set_mass(type, m); });
}
int espp_build_neighbors(espp_h h, double rc, double skin) {
    return guarded(h, [&](espp::SystemBase& s) { return s.build_neighbors(rc, skin); });
}
int espp_get_neighbors(espp_h h, int64_t* row_ptr, int64_t* cols, int64_t cap) {
    return guarded(h, [&](espp::SystemBase& s) { return s.get_neighbors(row_ptr, cols, cap); });
}
int espp_compute_forces(espp_h h, double* f, int where) {
    return guarded(h, [&](espp::SystemBase& s) { return s.compute_forces(f, where); });
}
int espp_integrate(espp_h h, int64_t nsteps, double dt, double gamma, double kT) {
    return guarded(h, [&](espp::SystemBase& s) { return s.integrate(nsteps, dt, gamma, kT); });
}
int espp_observables(espp_h h, espp_obs_t* out) {
    return guarded(h, [&](espp::SystemBase& s) { return s.observables(out, 1); });
}
int espp_observables_batch(espp_h h, espp_obs_t* out, int32_t R) {
    return guarded(h, [&](espp::SystemBase& s) { return s.observables(out, R); });
}
int espp_rdf_counts(espp_h h, int32_t rep, double rmax, int32_t nbins, int64_t* counts) {
    return guarded(h, [&](espp::SystemBase& s) { return s.rdf_counts(rep, rmax, nbins, counts); });
}
int espp_checkpoint_save(espp_h h, const char* path) {
    return guarded(h, [&](espp::SystemBase& s) { return s.checkpoint_save(path); });
}
int espp_checkpoint_load(espp_h h, const char* path) {
    return guarded(h, [&](espp::SystemBase& s) { return s.checkpoint_load(path); });
}
const char* espp_last_error(espp_h h) {
    if (!h || !h->impl) return g_create_error.c_str();
    return h->impl->msg.c_str();
}
uint32_t espp_error_word(espp_h h) { return (h && h->impl) ? h->impl->error_word() : 0u; }
int64_t espp_num_particles(espp_h h) { return (h && h->impl) ? h->impl->num_particles() : -1; }
int32_t espp_num_replicas(espp_h h) { return (h && h->impl) ? h->impl->num_replicas() : -1; }
int64_t espp_num_rebuilds(espp_h h) { return (h && h->impl) ? h->impl->num_rebuilds() : -1; }
int64_t espp_step(espp_h h) { return (h && h->impl) ? h->impl->step() : -1; }
int32_t espp_list_capacity(espp_h h) { return (h && h->impl) ? h->impl->list_capacity() : -1; }
int64_t espp_kernel_launches(espp_h h) { return (h && h->impl) ? h->impl->kernel_launches() : -1; }

int espp_set_kernel_timing(espp_h h, int enable) {
    return guarded(h, [&](espp::SystemBase& s) { return s.set_kernel_timing(enable); });
}
int espp_kernel_timing(espp_h h, double* out, int reset) {
    if (!out) return ESPP_ERR_ARG;
    return guarded(h, [&](espp::SystemBase& s) { return s.kernel_timing(out, reset); });
}
int espp_list_stats(espp_h h, int64_t* total_entries, int32_t* max_count) {
    return guarded(h, [&](espp::SystemBase& s) { return s.list_stats(total_entries, max_count); });
}
int espp_set_resort_interval(espp_h h, int64_t steps) {
    return guarded(h, [&](espp::SystemBase& s) { return s.set_resort_interval(steps); });
}

int espp_set_lees_edwards(espp_h h, int32_t on, double shear_rate, double time) {
    return guarded(h, [&](espp::SystemBase& s) { return s.set_lees_edwards(on, shear_rate, time); });
}
int espp_get_lees_edwards(espp_h h, int32_t* on, double* shear_rate, double* time) {
    return guarded(h, [&](espp::SystemBase& s) { return s.get_lees_edwards(on, shear_rate, time); });
}
int espp_set_force_method(espp_h h, int32_t method) {
    return guarded(h, [&](espp::SystemBase& s) { return s.set_force_method(method); });
}
int espp_tune_force_method(espp_h h, int32_t nsteps, double dt, double gamma, double kT, double* ms_per_step,
                           int32_t* chosen) {
    return guarded(h, [&](espp::SystemBase& s) {
        int c = 0;
        const int rc = s.tune_force_method(nsteps, dt, gamma, kT, ms_per_step, &c);
        if (chosen) *chosen = c;
        return rc;
    });
}
int espp_h5md_write(espp_h h, const char* path) {
    return guarded(h, [&](espp::SystemBase& s) { return s.h5md_write(path); });
}
int espp_h5md_read(espp_h h, const char* path) {
    return guarded(h, [&](espp::SystemBase& s) { return s.h5md_read(path); });
}
int espp_h5md_inspect(const char* path, int32_t* n_replicas, int64_t* n_particles, int64_t* step,
                      int32_t* precision) {
    espp::NvtxRange nvtx_range("espp_h5md_inspect");
    if (!path) {
        g_create_error = "path is required";
        return ESPP_ERR_ARG;
    }
    try {
        espp::H5mdState hs;
        std::string err;
        if (espp::h5md_read(path, hs, err)) {
            g_create_error = "H5MD read: " + err;
            return ESPP_ERR_IO;
        }
        int64_t n = 0;
        for (const espp::H5mdReplica& r : hs.reps) n += r.n;
        if (n_replicas) *n_replicas = (int32_t)hs.reps.size();
        if (n_particles) *n_particles = n;
        if (step) *step = hs.step;
        if (precision) *precision = hs.precision;
        return ESPP_OK;
    } catch (const std::exception& e) {
        g_create_error = std::string("H5MD read: ") + e.what();
        return ESPP_ERR_IO;
    }
}
int espp_set_list_store(espp_h h, int32_t push) {
    return guarded(h, [&](espp::SystemBase& s) { return s.set_list_store(push); });
}
int espp_set_step_shape(espp_h h, int32_t shape) {
    return guarded(h, [&](espp::SystemBase& s) { return s.set_step_shape(shape); });
}
int espp_tune_step_shape(espp_h h, int32_t nsteps, double dt, double gamma, double kT, double* ms,
                         int32_t* chosen) {
    return guarded(h, [&](espp::SystemBase& s) {
        int c[2] = {0, 0};
        const int rc = s.tune_step_shape(nsteps, dt, gamma, kT, ms, c);
        if (rc == ESPP_OK && chosen) {
            chosen[0] = c[0];
            chosen[1] = c[1];
        }
        return rc;
    });
}
int espp_set_thermostat(espp_h h, int32_t kind, double rc) {
    return guarded(h, [&](espp::SystemBase& s) { return s.set_thermostat(kind, rc); });
}
int espp_set_cell_subdivision(espp_h h, int32_t w) {
    return guarded(h, [&](espp::SystemBase& s) { return s.set_cell_subdivision(w); });
}
int espp_set_graph_chunk(espp_h h, int32_t steps) {
    return guarded(h, [&](espp::SystemBase& s) { return s.set_chunk(steps); });
}

int espp_langevin_noise(uint64_t seed, int64_t step, int64_t n, double* out, void* stream) {
    if (n < 0 || (n > 0 && !out)) return ESPP_ERR_ARG;
    espp::launch_noise(seed, step, n, out, (cudaStream_t)stream);
    if (cudaGetLastError() != cudaSuccess) return ESPP_ERR_CUDA;
    if (cudaStreamSynchronize((cudaStream_t)stream) != cudaSuccess) return ESPP_ERR_CUDA;
    return ESPP_OK;
}

}  // extern "C"

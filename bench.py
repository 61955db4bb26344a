"""Benchmark: particle-steps/s of the short-range MD step on a 1M-bead
Kremer-Grest melt (1000 chains x 1000 beads, density 0.85, WCA + FENE,
Langevin T=1, gamma=1, dt=0.005, skin 0.4) in FP32, with the plain FP64 path
timed beside it, an end-to-end figure through the C ABI with host buffers, the
roofline of the step kernel and the CPU oracle on the host cores.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

One rank per GPU (torchrun for N > 1).  Each rank steps its own independent
melt (seed 42 + rank): the ranks share no data, so the aggregate is weak
scaling and the only collectives are the barrier and the max of the timings.
Rank 0 prints one JSON line.
"""
import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "particle-steps/s @1M beads: FP32 & learned-CG vs FP64 plain, at stated force error"
WCA_RC = 2.0 ** (1.0 / 6.0)
L2_MB = 129.0


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10000)
    ap.add_argument("--warmup", type=int, default=500)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--nchains", type=int, default=1000)
    ap.add_argument("--nbeads", type=int, default=1000)
    ap.add_argument("--fp64-steps", type=int, default=2000)
    ap.add_argument("--no-fp64", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--profile-steps", type=int, default=1024)
    ap.add_argument("--direct", action="store_true",
                    help="launch every kernel directly instead of through CUDA graphs (for ncu)")
    ap.add_argument("--no-suite", action="store_true",
                    help="skip the secondary workloads (4M LJ, 512 replicas, learned CG)")
    ap.add_argument("--suite-steps", type=int, default=5000)
    ap.add_argument("--suite-only", default="",
                    help="comma-separated names of the suite entries to run (default: all)")
    ap.add_argument("--cg-frames", type=int, default=2000)
    ap.add_argument("--cg-epochs", type=int, default=10)
    ap.add_argument("--cg-batch", type=int, default=16)
    ap.add_argument("--ibi-iters", type=int, default=40)
    ap.add_argument("--ibi-damping", type=float, default=0.5)
    ap.add_argument("--refine-damping", type=float, default=0.5)
    ap.add_argument("--refine-iters", type=int, default=40,
                    help="structure refinement iterations of the learned potential (0: force matching alone)")
    ap.add_argument("--refine-frames", type=int, default=64)
    ap.add_argument("--refine-epochs", type=int, default=10)
    ap.add_argument("--cg-eq", type=int, default=2000)
    ap.add_argument("--cg-snap", type=int, default=20)
    ap.add_argument("--cg-warm", type=int, default=1000)
    ap.add_argument("--cg-steps", type=int, default=1000)
    ap.add_argument("--cg-probe", type=int, default=0,
                    help="only: N-site CG system with the learned potential, a few force evaluations (for ncu)")
    ap.add_argument("--train-probe", type=int, default=0,
                    help="time force-matching training on this many CG sites and exit (for ncu)")
    ap.add_argument("--step-shape", type=int, default=-1,
                    help="launch shape of the headline's step kernel after the tuner has run (for profiling; "
                         "default: the tuner's pick)")
    ap.add_argument("--quick-start", action="store_true",
                    help="lattice start with a short equilibration (for profiler runs)")
    return ap.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


# ---- the multi-GPU bookkeeping: one independent melt per rank (replicas only) ----
def rank_seed(rank):
    """Each rank steps its own melt, seeded by its rank."""
    return 42 + rank


def reduce_max(pg, x, device):
    """Largest value over the ranks of process group pg (None: one process)."""
    if pg is None:
        return x
    import torch
    t = torch.tensor([x], dtype=torch.float64, device=device)
    pg.all_reduce(t, op=pg.ReduceOp.MAX)
    return float(t.item())


def aggregate_rate(world, n, steps, ms_max):
    """Whole-job particle-steps/s: every rank's particles over the slowest rank's time."""
    return world * n * steps / (ms_max / 1e3)


def workload_name(a):
    return "kg_melt_%dx%d_rho0.85_wca_fene_langevin" % (a.nchains, a.nbeads)


def host_cores():
    try:
        return len(os.sched_getaffinity(0))
    except Exception:
        return os.cpu_count() or 1


def cpu_model():
    try:
        with open("/proc/cpuinfo") as fh:
            for line in fh:
                if line.lower().startswith(("model name", "cpu part", "hardware")):
                    return line.split(":", 1)[1].strip()
    except Exception:
        pass
    import platform
    return platform.machine()


# ---------------------------------------------------------------------------
# clocks during the timed region
# ---------------------------------------------------------------------------
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        # raw samples (the JSON line carries their summary); ESPP_CLOCK_DIR
        # keeps them somewhere else than the temporary directory
        out_dir = os.environ.get("ESPP_CLOCK_DIR") or tempfile.gettempdir()
        self.path = os.path.join(out_dir, "clocks_bench_%d.csv" % os.getpid())

    def __enter__(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.FIELDS,
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=self.fh, stderr=subprocess.DEVNULL)
            time.sleep(0.3)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
            self.fh.close()

    def summary(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        rows = []
        with open(self.path) as fh:
            for line in fh:
                p = [t.strip() for t in line.split(",")]
                if len(p) < 9:
                    continue
                try:
                    rows.append((float(p[1]), float(p[2]), float(p[3]), p[4], p[5], p[6], p[7], p[8]))
                except ValueError:
                    continue
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        busy = [r for r in rows if r[2] > 200.0] or rows
        reasons = set()
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        for r in rows:
            for nm, val in zip(names, r[4:]):
                if val.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(r[0] for r in busy), "sm_max_mhz": max(r[1] for r in rows),
                "samples": len(rows), "reasons": sorted(reasons)}


# ---------------------------------------------------------------------------
# the system
# ---------------------------------------------------------------------------
def make_melt(a, seed, precision, nchains=None, nbeads=None):
    """KG melt: random-walk chains, soft push-off with a growing force cap,
    then plain WCA; falls back to an overlap-free lattice start."""
    from paper_2608_14911_gb300 import espp, inputs
    nchains = a.nchains if nchains is None else nchains
    nbeads = a.nbeads if nbeads is None else nbeads
    cfg = inputs.kg_random_walk(nchains, nbeads, density=0.85, seed=seed, bond=0.97)
    v = inputs.maxwell_velocities(cfg.n, 1.0, seed=seed)
    s = espp.System(cfg.box, cfg.n, cfg.types, cfg.bonds, precision=precision, seed=seed)
    s.set_fene(30.0, 1.5)
    start = "random_walk+pushoff"
    try:
        if a.quick_start:
            raise espp.EsppError(0, "quick start requested")
        s.set_lj_capped(1.0, 1.0, WCA_RC, 1.05)
        s.set_state(cfg.x, v, cfg.img)
        s.build_neighbors(WCA_RC, 0.4)
        for cap in (1.05, 1.0, 0.95, 0.9, 0.85, 0.8):
            s.set_lj_capped(1.0, 1.0, WCA_RC, cap)
            s.integrate(400, 1e-3, 1.0, 1.0)
        s.set_wca(1.0, 1.0)
        s.integrate(1000, 0.002, 1.0, 1.0)
        s.integrate(1000, 0.005, 1.0, 1.0)
    except espp.EsppError:
        start = "lattice"
        s.close()
        cfg = inputs.kg_lattice(nchains, nbeads, density=0.85, seed=seed)
        s = espp.System(cfg.box, cfg.n, cfg.types, cfg.bonds, precision=precision, seed=seed)
        s.set_fene(30.0, 1.5)
        s.set_wca(1.0, 1.0)
        s.set_state(cfg.x, v, cfg.img)
        s.build_neighbors(WCA_RC, 0.4)
        s.integrate(200 if a.quick_start else 2000, 0.005, 1.0, 1.0)
    return s, cfg, start


def copy_system(src, cfg, precision, seed):
    from paper_2608_14911_gb300 import espp
    x, v, img = src.get_state()
    s = espp.System(cfg.box, cfg.n, cfg.types, cfg.bonds, precision=precision, seed=seed)
    s.set_fene(30.0, 1.5)
    s.set_wca(1.0, 1.0)
    s.set_state(x, v, img)
    s.build_neighbors(WCA_RC, 0.4)
    s.set_step(src.step)
    return s, (x, v, img)


def timed_integrate(s, steps, stream_sync):
    import torch
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    stream_sync()
    e0.record()
    # NVTX range: profilers can restrict a capture to the timed steps
    torch.cuda.nvtx.range_push("timed_region")
    s.integrate(steps, 0.005, 1.0, 1.0)
    torch.cuda.nvtx.range_pop()
    e1.record()
    stream_sync()
    return e0.elapsed_time(e1)


def step_kernel_bytes(n, list_entries, precision):
    """Algorithmic HBM bytes of one step-kernel launch (MODE_STEP).
    Per particle: position read + write, velocity read + write, build position
    read (4-vectors of 16 B in FP32, 32 B in FP64), bond slots (8 B), list
    count (4 B); plus 4 B per Verlet-list entry.  Neighbour positions are
    reads of the same position array and are not counted again."""
    v4 = 16 if precision == 1 else 32
    return n * (5 * v4 + 8 + 4) + 4 * list_entries


def step_kernel_digest():
    """Digest of the sources the step kernel is compiled from."""
    h = hashlib.sha256()
    for f in ("k_step.cu", "pair_terms.cuh", "kernels.cuh", "common.cuh", "philox.cuh", "packed.cuh"):
        h.update(open(os.path.join(ROOT, "paper_2608_14911_gb300", "csrc", f), "rb").read())
    return h.hexdigest()[:16]


def read_traffic_record():
    """DRAM bytes per step-kernel launch from the committed ncu summary, or
    None when the kernel source changed since the capture."""
    path = os.path.join(ROOT, "profiles", "step_kernel_traffic.txt")
    if not os.path.exists(path):
        return None
    rec = {}
    with open(path) as fh:
        for line in fh:
            if ":" in line and not line.startswith("#"):
                k, val = line.split(":", 1)
                rec[k.strip()] = val.strip()
    if rec.get("k_step_sha") != step_kernel_digest():
        return None
    try:
        return float(rec["dram_bytes_per_particle_step"])
    except (KeyError, ValueError):
        return None


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            return json.load(fh), "measured"
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}, "fallback"


# ---------------------------------------------------------------------------
# the CPU oracle (the reference arm and the cpu_baseline leg)
# ---------------------------------------------------------------------------
def oracle_rate(cfg, x, v, img, budget_s):
    """Time the oracle's own velocity-Verlet + Langevin steps on the full
    system for about budget_s seconds; returns (particle-steps/s, steps, s)."""
    import oracle as O
    model = O.Model(1, {(0, 0): ("wca", 1.0, 1.0)}, ("fene", 30.0, 1.5))
    st = O.State(cfg.box, x, v, img, cfg.types, cfg.bonds)
    O.integrate(model, st, 0, 0.005, 1.0, 1.0, seed=42)  # force of the start state
    t0 = time.perf_counter()
    O.integrate(model, st, 1, 0.005, 1.0, 1.0, seed=42)
    one = time.perf_counter() - t0
    k = max(1, min(200, int(budget_s / max(one, 1e-6)) - 1))
    t0 = time.perf_counter()
    O.integrate(model, st, k, 0.005, 1.0, 1.0, seed=42)
    dt_s = time.perf_counter() - t0
    steps = k + 1
    total = dt_s + one
    return cfg.n * steps / total, steps, total, O.num_threads()


def run_reference(a):
    rank, world, _ = dist_env()
    if rank != 0:
        return 0
    from paper_2608_14911_gb300 import inputs
    cfg = inputs.kg_lattice(a.nchains, a.nbeads, density=0.85, seed=42)
    v = inputs.maxwell_velocities(cfg.n, 1.0, seed=42)
    # the oracle as it stands, on a bounded sample of the same workload
    value, steps_per_run, secs, threads = oracle_rate(cfg, cfg.x, v, cfg.img, a.cpu_seconds)
    sample = "%d oracle steps of the full %d-bead melt (lattice start), %.1f s" % (steps_per_run, cfg.n, secs)
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "particle-steps/s",
        "n_gpus": world, "steps": a.steps, "warmup": a.warmup,
        "ms_per_step": 1e3 * cfg.n / value, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": workload_name(a), "n_particles": cfg.n},
        "cpu_baseline": {"value": value, "unit": "particle-steps/s", "cores": threads,
                         "kind": "oracle", "sample": sample, "cpu": cpu_model()},
        "e2e": {"value": value, "unit": "particle-steps/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


# ---------------------------------------------------------------------------
# our arm
# ---------------------------------------------------------------------------
def run_ours(a):
    import torch
    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    pg = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
        pg = dist
    import __graft_entry__ as g
    if rank == 0 or world == 1:
        g.build()
    if pg:
        pg.barrier()
        g.build()
    from paper_2608_14911_gb300 import espp

    def barrier():
        if pg:
            pg.barrier()
        torch.cuda.synchronize()

    def max_over_ranks(x):
        return reduce_max(pg, x, "cuda")

    seed = rank_seed(rank)
    s, cfg, start = make_melt(a, seed, espp.ESPP_FP32)
    # the autotuner picks the step kernel's launch shape and the resort
    # interval for this melt (untimed; the state is restored afterwards)
    shape_ms, resort_ms, (shape, resort) = s.tune_step_shape(200, 0.005, 1.0, 1.0)
    if a.step_shape >= 0:
        shape = a.step_shape
        s.set_step_shape(shape)
    if a.direct:
        s.set_graph_chunk(0)
    n = cfg.n
    assert a.warmup >= 3
    s.integrate(a.warmup, 0.005, 1.0, 1.0)
    total_entries, max_count = s.list_stats()
    launches0 = s.kernel_launches
    rb0 = s.n_rebuilds

    # ---- FP32 timed region -------------------------------------------------
    with ClockSampler(local) as clk:
        barrier()
        ms = timed_integrate(s, a.steps, barrier)
        barrier()
    ms = max_over_ranks(ms)
    clocks = clk.summary()
    gpu_launches = s.kernel_launches - launches0
    rebuilds = s.n_rebuilds - rb0
    value = aggregate_rate(world, n, a.steps, ms)
    obs = s.observables()

    # ---- step-kernel duration by CUDA events inside the graphs -------------
    if a.direct:
        s.set_graph_chunk(64)
    s.set_kernel_timing(True)
    prof_steps = max(64, a.profile_steps // 64 * 64)
    for _ in range(prof_steps // 64):
        s.integrate(64, 0.005, 1.0, 1.0)
    kt = s.kernel_timing(reset=True)
    s.set_kernel_timing(False)
    total_entries2, _ = s.list_stats()
    mean_entries = 0.5 * (total_entries + total_entries2)
    avg_step_ms = kt["step_ms"] / max(1, kt["step_launches"])
    peaks, peak_kind = measured_peaks()
    alg_bytes = step_kernel_bytes(n, mean_entries, 1)
    achieved = alg_bytes / (avg_step_ms * 1e-3) / 1e9
    dram_pp = read_traffic_record()
    roofline = {"bound": "hbm", "achieved": achieved, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                "frac": achieved / peaks["hbm_gbs"],
                "traffic": None if dram_pp is None else dram_pp * n,
                "kernel": "k_step<float, MODE_STEP>",
                "algorithmic_bytes_per_launch": alg_bytes,
                "avg_launch_ms": avg_step_ms, "launches_timed": kt["step_launches"],
                "peak_kind": peak_kind + " (hbm_gbs, STREAM-style copy)",
                "rebuild_node_ms_per_step": kt["rebuild_ms"] / max(1, kt["steps"])}

    # ---- FP64 plain path ------------------------------------------------------
    fp64 = None
    if not a.no_fp64:
        s64, _ = copy_system(s, cfg, espp.ESPP_FP64, seed)
        if a.direct:
            s64.set_graph_chunk(0)
        s64.integrate(max(3, a.warmup // 5), 0.005, 1.0, 1.0)
        barrier()
        ms64 = max_over_ranks(timed_integrate(s64, a.fp64_steps, barrier))
        v64 = world * n * a.fp64_steps / (ms64 / 1e3)
        fp64 = {"value": v64, "unit": "particle-steps/s", "steps": a.fp64_steps,
                "ms_per_step": ms64 / a.fp64_steps, "dtype": "f64",
                "fp32_speedup": value / v64}
        s64.close()

    # ---- end to end through the C ABI with pinned host buffers ---------------
    e2e = None
    if not a.no_e2e:
        x, v, img = s.get_state()
        hx = torch.from_numpy(x).pin_memory()
        hv = torch.from_numpy(v).pin_memory()
        hi = torch.from_numpy(img).pin_memory()
        barrier()
        t0 = time.perf_counter()
        s.set_state(hx, hv, hi)
        s.integrate(a.steps, 0.005, 1.0, 1.0)
        s.get_state((hx, hv, hi))
        torch.cuda.synchronize()
        t_e2e = max_over_ranks(time.perf_counter() - t0)
        bi = hx.numel() * 8 + hv.numel() * 8 + hi.numel() * 4
        e2e = {"value": world * n * a.steps / t_e2e, "unit": "particle-steps/s",
               "h2d_bytes_per_step": bi / a.steps, "d2h_bytes_per_step": bi / a.steps,
               "timed": "set_state(host) + integrate(%d) + get_state(host), wall clock" % a.steps}

    # ---- CPU oracle on the host cores (rank 0, N = 1 only) --------------------
    cpu = None
    if not a.no_cpu_baseline and world == 1:
        x, v, img = s.get_state()
        rate, k, secs, threads = oracle_rate(cfg, x, v, img, a.cpu_seconds)
        cpu = {"value": rate, "unit": "particle-steps/s", "cores": threads, "kind": "oracle",
               "sample": "%d oracle steps of the full %d-bead melt, %.1f s" % (k, n, secs),
               "cpu": cpu_model(), "host_cores": host_cores()}

    suite = None
    if not a.no_suite and world == 1:
        suite = {}
        for name, fn in (("cfg0_fp64", lambda o: o.update(suite_cfg0(a, barrier))),
                         ("kg1m_dpd", lambda o: o.update(suite_dpd(a, barrier, s, cfg, seed, ms / a.steps))),
                         ("dpd_fluid_786k", lambda o: o.update(suite_dpd_fluid(a, barrier))),
                         ("lj4m", lambda o: o.update(suite_lj4m(a, barrier, peaks))),
                         ("batched512", lambda o: o.update(suite_batched(a, barrier))),
                         ("learned_cg", lambda o: suite_learned_cg(a, barrier, o))):
            if a.suite_only and name not in a.suite_only.split(","):
                continue
            part = {}
            t0 = time.perf_counter()
            try:
                fn(part)
            except Exception as exc:  # reported, never hidden; partial results kept
                part["error"] = "%s: %s" % (type(exc).__name__, exc)
            part["wall_s"] = time.perf_counter() - t0
            suite[name] = part

    ws_mb = alg_bytes / 1e6
    line = {
        "metric": METRIC, "value": value, "unit": "particle-steps/s", "n_gpus": world,
        "steps": a.steps, "warmup": a.warmup, "ms_per_step": ms / a.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic",
        "config": {"workload": workload_name(a), "n_particles": n, "start": start,
                   "rc": WCA_RC, "skin": 0.4, "dt": 0.005, "gamma": 1.0, "kT": 1.0,
                   "parallelism": "replicas" if world > 1 else "single",
                   "l2": "inputs larger than L2: per-step working set %.0f MB > %.0f MB L2, no flush"
                         % (ws_mb, L2_MB),
                   "rebuilds_in_timed_region": rebuilds,
                   "step_shape": {"chosen": shape, "groups_per_batch": espp.STEP_SHAPE_TABLE[shape][0],
                                  "min_blocks_per_sm": espp.STEP_SHAPE_TABLE[shape][1],
                                  "tiles_per_block": espp.STEP_SHAPE_TABLE[shape][2], "resort_interval": resort,
                                  "tuner_ms_per_step": {"shapes": shape_ms, "resort_250_500_1000": resort_ms}},
                   "mean_list_entries_per_particle": mean_entries / n, "max_list_entries": max_count,
                   "observables_after_run": {k: obs[k] for k in ("temperature", "mean_bond", "rg2", "pe_pair")},
                   "force_error_gate": "FP32 <= 1e-5 relative RMS vs the FP64 oracle (tests/test_gpu_parity.py)"},
        "fp64": fp64,
        "roofline": roofline,
        "cpu_baseline": cpu,
        "e2e": e2e,
        "gpu_launches": gpu_launches,
        "clocks": clocks,
        "suite": suite,
    }
    if rank == 0:
        print(json.dumps(line), flush=True)
    s.close()
    if pg:
        pg.destroy_process_group()
    return 0


# ---------------------------------------------------------------------------
# secondary workloads (reported under "suite")
# ---------------------------------------------------------------------------
def _timed(s, steps, dt, gamma, kT, sync):
    import torch
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    sync()
    e0.record()
    s.integrate(steps, dt, gamma, kT)
    e1.record()
    sync()
    return e0.elapsed_time(e1)


def _step_kernel_ms(s, dt, gamma, kT, steps=256):
    s.set_kernel_timing(True)
    for _ in range(max(1, steps // 64)):
        s.integrate(64, dt, gamma, kT)
    kt = s.kernel_timing(reset=True)
    s.set_kernel_timing(False)
    return kt["step_ms"] / max(1, kt["step_launches"]), kt["rebuild_ms"] / max(1, kt["steps"])


def suite_cfg0(a, sync):
    """The FP64 sanity workload: a Kremer-Grest melt of 20 chains x 50 beads
    at density 0.85 (random walks, capped push-off, seed 42), 1000 timed
    Langevin steps in FP64 (its parity with the oracle is checked by the
    tests, not here)."""
    from paper_2608_14911_gb300 import espp
    s, cfg, start = make_melt(a, 42, espp.ESPP_FP64, nchains=20, nbeads=50)
    steps = 1000
    ms = _timed(s, steps, 0.005, 1.0, 1.0, sync)
    o = s.observables()
    s.close()
    return {"workload": "kg_melt_20x50_rho0.85_fp64", "n_particles": cfg.n, "start": start, "steps": steps,
            "value": cfg.n * steps / (ms / 1e3), "unit": "particle-steps/s", "ms_per_step": ms / steps,
            "dtype": "f64", "temperature": o["temperature"], "mean_bond": o["mean_bond"],
            "note": "launch-bound at 1000 beads; FP64 parity with the oracle: tests/test_gpu_parity.py"}


def suite_dpd(a, sync, src, cfg, seed, langevin_ms):
    """The KG melt of the headline line under the DPD thermostat (pair cutoff
    2^(1/6), gamma 1, kT 1) in place of Langevin: each step adds a velocity
    snapshot and a pass over the list for the pair friction and noise."""
    from paper_2608_14911_gb300 import espp
    s, _ = copy_system(src, cfg, espp.ESPP_FP32, seed)
    s.set_thermostat(espp.ESPP_THERMO_DPD, WCA_RC)
    s.integrate(200, 0.005, 1.0, 1.0)
    p0 = s.observables()
    steps = a.suite_steps
    ms = _timed(s, steps, 0.005, 1.0, 1.0, sync)
    k_ms, rb_ms = _step_kernel_ms(s, 0.005, 1.0, 1.0)
    o = s.observables()
    _, v, _ = s.get_state()
    out = {"workload": workload_name(a) + "_dpd_rc1.1225_gamma1", "n_particles": cfg.n,
           "value": cfg.n * steps / (ms / 1e3), "unit": "particle-steps/s", "steps": steps,
           "ms_per_step": ms / steps, "langevin_ms_per_step": langevin_ms,
           "step_kernel_avg_launch_ms": k_ms, "rebuild_node_ms_per_step": rb_ms,
           "temperature_after": o["temperature"], "temperature_before": p0["temperature"],
           "net_momentum_per_particle": float(abs(v.sum(axis=0)).max() / cfg.n)}
    s.close()
    return out


def suite_dpd_fluid(a, sync):
    """Groot-Warren DPD fluid: 786,432 particles at density 3 in a 64^3 box,
    soft repulsion F = 25 (1 - r) (tabulated) and the DPD thermostat (rc 1,
    gamma 4.5, kT 1, dt 0.04), at rest and under Lees-Edwards shear 0.01; the
    force method (Verlet list or list-free cells) is the tuner's choice."""
    from paper_2608_14911_gb300 import espp, inputs
    L, a_rep, n_tab = 64.0, 25.0, 1001
    box = np.array([L, L, L])
    n = int(3 * L ** 3)
    cfg = inputs.random_positions(n, box, seed=11)
    v = inputs.maxwell_velocities(n, 1.0, seed=11)
    r = np.linspace(0.0, 1.0, n_tab)
    u_tab, f_tab = 0.5 * a_rep * (1.0 - r) ** 2, a_rep * (1.0 - r)
    out = {"workload": "dpd_fluid_786432_rho3_a25_gamma4.5_dt0.04", "n_particles": n}
    for label, shear in (("rest", None), ("lees_edwards_0.01", 0.01)):
        s = espp.System(box, n, cfg.types, cfg.bonds, precision=espp.ESPP_FP32, seed=11)
        s.set_table_pair(1.0, u_tab, f_tab)
        s.set_state(cfg.x, v, cfg.img)
        if shear is not None:
            s.set_lees_edwards(True, shear, 0.0)
        s.build_neighbors(1.0, 0.6)
        s.set_thermostat(espp.ESPP_THERMO_DPD, 1.0)
        s.integrate(300, 0.04, 4.5, 1.0)
        # Verlet list (skin 0.6) or list-free cells, whichever the tuner times faster
        tuned_ms, method = s.tune_force_method(100, 0.04, 4.5, 1.0)
        s.integrate(50, 0.04, 4.5, 1.0)
        rb0 = s.n_rebuilds
        steps = a.suite_steps
        ms = _timed(s, steps, 0.04, 4.5, 1.0, sync)
        rb = s.n_rebuilds - rb0
        obs = []
        for _ in range(10):  # after the timed region: averages over 10 snapshots
            s.integrate(20, 0.04, 4.5, 1.0)
            obs.append(s.observables())
        mean = {k: float(np.mean([q[k] for q in obs])) for k in ("temperature", "pressure", "pxz")}
        part = {"value": n * steps / (ms / 1e3), "unit": "particle-steps/s", "steps": steps,
                "ms_per_step": ms / steps, "rebuilds": rb,
                "force_shape": espp.FORCE_SHAPE_NAMES[method],
                "tuner_ms_per_step": dict(zip(espp.FORCE_SHAPE_NAMES, tuned_ms)), **mean}
        if shear is not None:
            part["viscosity_estimate"] = -mean["pxz"] / shear
        out[label] = part
        s.close()
    return out


def suite_lj4m(a, sync, peaks):
    """4,194,304-particle LJ fluid: fcc 128x128x64 at density 0.8442, Maxwell
    T = 0.72, rc 2.5 (shifted), skin 0.3, Langevin gamma 1 at T = 0.72."""
    from paper_2608_14911_gb300 import espp, inputs
    cfg = inputs.lj_fcc(128, 128, 64, density=0.8442)
    v = inputs.maxwell_velocities(cfg.n, 0.72, seed=42)
    out = {"workload": "lj_fluid_4194304_fcc_rho0.8442_T0.72_rc2.5_skin0.3", "n_particles": cfg.n}
    for prec, steps in ((espp.ESPP_FP32, a.suite_steps), (espp.ESPP_FP64, max(50, a.suite_steps // 10))):
        s = espp.System(cfg.box, cfg.n, cfg.types, cfg.bonds, precision=prec, seed=42)
        s.set_lj(1.0, 1.0, 2.5, True)
        s.set_state(cfg.x, v, cfg.img)
        s.build_neighbors(2.5, 0.3)
        s.integrate(100, 0.005, 1.0, 0.72)
        tuned = None
        if prec == espp.ESPP_FP32:
            # the autotuners pick the force path (list over whole, half or
            # third cells, or list-free cells), then the step kernel's launch
            # shape and the resort interval
            force_ms, force_shape = s.tune_force_method(100, 0.005, 1.0, 0.72)
            shape_ms, resort_ms, (shape, resort) = s.tune_step_shape(200, 0.005, 1.0, 0.72)
            tuned = {"force_shape": espp.FORCE_SHAPE_NAMES[force_shape],
                     "force_tuner_ms_per_step": dict(zip(espp.FORCE_SHAPE_NAMES, force_ms)),
                     "chosen": shape, "shape": espp.STEP_SHAPE_TABLE[shape], "resort_interval": resort,
                     "tuner_ms_per_step": {"shapes": shape_ms, "resort_250_500_1000": resort_ms}}
            s.integrate(20, 0.005, 1.0, 0.72)
        rb0 = s.n_rebuilds
        ms = _timed(s, steps, 0.005, 1.0, 0.72, sync)
        key = "fp32" if prec == espp.ESPP_FP32 else "fp64"
        out[key] = {"value": cfg.n * steps / (ms / 1e3), "unit": "particle-steps/s", "steps": steps,
                    "steps_spec": 10000,
                    "ms_per_step": ms / steps, "rebuilds": s.n_rebuilds - rb0}
        if prec == espp.ESPP_FP32:
            total, _ = s.list_stats()
            k_ms, rb_ms = _step_kernel_ms(s, 0.005, 1.0, 0.72)
            byt = step_kernel_bytes(cfg.n, total, 1) - 8 * cfg.n  # no bonds
            out[key]["step_kernel"] = {"avg_launch_ms": k_ms, "algorithmic_bytes": byt,
                                       "achieved_gbs": byt / (k_ms * 1e-3) / 1e9,
                                       "frac_of_measured_hbm": byt / (k_ms * 1e-3) / 1e9 / peaks["hbm_gbs"],
                                       "mean_list_entries": total / cfg.n,
                                       "rebuild_node_ms_per_step": rb_ms}
            out[key]["step_shape"] = tuned
        s.close()
    out["fp32_speedup_vs_fp64"] = out["fp32"]["value"] / out["fp64"]["value"]
    return out


def suite_batched(a, sync):
    """512 independent KG melts of uneven size (chains uniform 10-400, length
    uniform 20-200, density 0.85), one seed each, stepped together."""
    from paper_2608_14911_gb300 import espp, inputs
    sizes = inputs.replica_sizes(512, seed=42)
    cfgs = [inputs.kg_random_walk(nc, nb, density=0.85, seed=42 + r) for r, (nc, nb) in enumerate(sizes)]
    reps = [dict(box=c.box, n=c.n, types=c.types, bonds=c.bonds, seed=42 + r) for r, c in enumerate(cfgs)]
    s = espp.System(replicas=reps, precision=espp.ESPP_FP32)
    n = s.n
    x = np.concatenate([c.x for c in cfgs])
    img = np.concatenate([c.img for c in cfgs])
    v = inputs.maxwell_velocities(n, 1.0, seed=7)
    s.set_fene(30.0, 1.5)
    s.set_lj_capped(1.0, 1.0, WCA_RC, 1.05)
    s.set_state(x, v, img)
    s.build_neighbors(WCA_RC, 0.4)
    for cap in (1.05, 1.0, 0.95, 0.9, 0.85, 0.8):
        s.set_lj_capped(1.0, 1.0, WCA_RC, cap)
        s.integrate(400, 1e-3, 1.0, 1.0)
    s.set_wca(1.0, 1.0)
    s.integrate(1000, 0.002, 1.0, 1.0)
    s.integrate(200, 0.005, 1.0, 1.0)
    # the autotuner picks the force path for this batch, then the step
    # kernel's launch shape and the resort interval
    tuned_ms, shape = s.tune_force_method(100, 0.005, 1.0, 1.0)
    shape_ms, resort_ms, (step_shape, resort) = s.tune_step_shape(200, 0.005, 1.0, 1.0)
    s.integrate(50, 0.005, 1.0, 1.0)
    rb0 = s.n_rebuilds
    l0 = s.kernel_launches
    steps = a.suite_steps
    ms = _timed(s, steps, 0.005, 1.0, 1.0, sync)
    obs = s.observables()
    temps = np.array([o["temperature"] for o in obs])
    out = {"workload": "kg_batched_512_replicas_chains10-400_len20-200_rho0.85", "replicas": 512,
           "n_particles": n, "min_replica": min(s.rep_n), "max_replica": max(s.rep_n),
           "value": n * steps / (ms / 1e3), "unit": "particle-steps/s", "steps": steps, "steps_spec": 5000,
           "ms_per_step": ms / steps, "rebuild_passes": s.n_rebuilds - rb0,
           "kernel_launches_per_step": (s.kernel_launches - l0) / steps,
           "force_shape": espp.FORCE_SHAPE_NAMES[shape],
           "tuner_ms_per_step": dict(zip(espp.FORCE_SHAPE_NAMES, tuned_ms)),
           "step_shape": {"chosen": step_shape, "shape": espp.STEP_SHAPE_TABLE[step_shape],
                          "resort_interval": resort,
                          "tuner_ms_per_step": {"shapes": shape_ms, "resort_250_500_1000": resort_ms}},
           "temperature_mean_over_replicas": float(temps.mean())}
    s.close()
    return out


def _bond_table_boltzmann(xs, nchains, sites_per_chain, box, kT=1.0, dr=0.02, rmax=6.0, min_count=100):
    """Boltzmann-inverted CG bond potential from mapped frames:
    U(b) = -kT ln(P(b) / b^2) on the bins holding at least min_count bonds,
    smoothed over five bins, continued linearly outside them with restoring
    slopes (at least kT / sigma); F = -dU/db on a grid from 0 to rmax."""
    b = []
    for x in xs:
        x = x.reshape(nchains, sites_per_chain, 3)
        d = x[:, 1:] - x[:, :-1]
        d -= box * np.round(d / box)
        b.append(np.linalg.norm(d, axis=2).ravel())
    b = np.concatenate(b)
    edges = np.arange(0.0, rmax + dr, dr)
    hist, _ = np.histogram(b, bins=edges)
    centres = 0.5 * (edges[1:] + edges[:-1])
    ok = np.nonzero(hist >= min_count)[0]
    lo, hi = ok[0], ok[-1]
    U = np.interp(centres, centres[ok], -kT * np.log(hist[ok] / centres[ok] ** 2))
    pad = 2
    U[lo:hi + 1] = np.convolve(np.pad(U[lo:hi + 1], pad, mode="edge"), np.ones(5) / 5.0, mode="valid")
    # linear continuation with the edge slopes (restoring at both ends)
    sl = min((U[lo + 3] - U[lo]) / (3 * dr), -1.0)
    sh = max((U[hi] - U[hi - 3]) / (3 * dr), 1.0)
    U[:lo] = U[lo] + sl * (centres[:lo] - centres[lo])
    U[hi + 1:] = U[hi] + sh * (centres[hi + 1:] - centres[hi])
    grid = np.linspace(0.0, rmax, 1201)
    Ug = np.interp(grid, centres, U, left=U[0] + sl * (0 - centres[0]))
    Fg = -np.gradient(Ug, grid)
    return rmax, Ug - Ug.min(), Fg, float(b.mean())


RCM, SKIN_CG, DR_G = 3.5, 0.5, 0.02
# handles that evaluate independent frames (training, held-out forces) build
# a fresh list for every frame, so a skin would only lengthen it
SKIN_FRAMES = 0.0


def _gofr(counts, n, box, dr=DR_G):
    """g(r) of unique-pair counts per bin (ideal-gas shell normalisation)."""
    r0 = np.arange(counts.size) * dr
    shell = 4.0 / 3.0 * np.pi * ((r0 + dr) ** 3 - r0 ** 3)
    rho = n / np.prod(box)
    return counts / (0.5 * n * rho * shell)


def _rdf_l2(ga, gb, dr=DR_G, rmax=RCM):
    """L2 distance of two g(r): sqrt(sum (ga - gb)^2 dr / rmax)."""
    return float(np.sqrt(((ga - gb) ** 2).sum() * dr / rmax))


def _cg_handle(box, n, bonds, bond_tab, pair, seed):
    """A CG handle: the Boltzmann-inverted bond table, 1-2 bonded pairs out of
    the pair potential, and pair = ("mlp", bits) | ("table", u, F) | None."""
    from paper_2608_14911_gb300 import espp
    h = espp.System(box, n, None, bonds, precision=espp.ESPP_FP32, seed=seed)
    if pair is not None and pair[0] == "mlp":
        h.set_mlp(RCM, pair[1])
    elif pair is not None:
        h.set_table_pair(RCM, pair[1], pair[2])
    h.set_table_bond(*bond_tab[:3])
    h.set_exclude_bonded(True)
    return h


def _sampled_rdf(h, x0, v0, eq, nsnap, every):
    """Mean unique non-bonded pair counts (bins of DR_G up to RCM) over nsnap
    snapshots every `every` steps after `eq` steps from (x0, v0)."""
    h.set_state(x0, v0)
    h.build_neighbors(RCM, SKIN_FRAMES)
    h.integrate(eq, 0.005, 1.0, 1.0)
    counts = np.zeros(int(round(RCM / DR_G)))
    for _ in range(nsnap):
        h.integrate(every, 0.005, 1.0, 1.0)
        counts += h.rdf_counts(RCM, counts.size)
    return counts / nsnap


def _table_from_potential(U_bins, rt):
    """Pair table (u, F = -du/dr) on the grid rt from a potential on the bin
    centres: linear interpolation, a cosine taper over the last 0.5 sigma so
    that u and F reach 0 at the cutoff, F by central differences."""
    rc_b = (np.arange(U_bins.size) + 0.5) * DR_G
    U = np.interp(rt, rc_b, U_bins)
    U = U - np.interp(RCM, rc_b, U_bins)
    taper = np.where(rt < RCM - 0.5, 1.0, 0.5 * (1.0 + np.cos(np.pi * (rt - (RCM - 0.5)) / 0.5)))
    U = U * taper
    F = -np.gradient(U, rt)
    return U, F


def _reliable_from(counts_total, min_count=100):
    """First bin from which every bin holds at least min_count pairs (summed
    over the sampled snapshots): below it the core is too sparsely sampled
    for a logarithm."""
    ok = counts_total >= min_count
    bad = np.nonzero(~ok)[0]
    return 0 if bad.size == 0 else int(bad[-1]) + 1


def _core_extrapolate(U, first, min_slope=-2.0):
    """U below bin `first` continued linearly, repulsive (U grows toward r = 0)
    with the slope of the first sampled bins, at least |min_slope|."""
    k = min(first + 5, U.size - 1)
    slope = min((U[k] - U[first]) / ((k - first) * DR_G), min_slope)
    idx = np.arange(first)
    U[:first] = U[first] + slope * (idx - first) * DR_G
    return U


def _smooth(v, width=3):
    pad = width // 2
    w = np.pad(v, pad, mode="edge")
    return np.convolve(w, np.ones(width) / width, mode="valid")


def _boltzmann_start(g_t, counts_total, kT=1.0):
    """U_0(r) = -kT ln g_target(r) where the target is well sampled, smoothed
    over three bins, continued linearly (repulsive) into the core."""
    first = _reliable_from(counts_total)
    U = np.zeros(g_t.size)
    U[first:] = -kT * np.log(g_t[first:])
    U[first:] = _smooth(U[first:])
    return _core_extrapolate(U, first), first


def _ibi_update(U, g, g_t, counts_g, first_t, damping=0.3):
    """One iterative Boltzmann inversion step, U += damping kT ln(g / g_t), on
    the bins both samples hold well (the correction smoothed over five
    bins), the core re-extrapolated from the first of them."""
    first = max(first_t, _reliable_from(counts_g))
    corr = np.zeros_like(U)
    corr[first:] = damping * np.log(g[first:] / g_t[first:])
    corr[first:] = _smooth(corr[first:], 5)
    U = U + corr
    return _core_extrapolate(U, first)


def _correction_update(C, g, g_t, counts_g, first_t, damping=0.3):
    """The structural correction of the learned potential, one iterative
    Boltzmann inversion step: C += damping kT ln(g / g_t) on the bins both
    samples hold well (smoothed over five bins); below them C is held at its
    first reliable value (no force: the core stays the learned one)."""
    first = max(first_t, _reliable_from(counts_g))
    corr = np.zeros_like(C)
    corr[first:] = damping * np.log(g[first:] / g_t[first:])
    corr[first:] = _smooth(corr[first:], 5)
    C = C + corr
    C[:first] = C[first]
    return C


def _pair_forces_of_table(box, n, bonds, ut, ft, frames):
    """Pair forces (1-2 bonded pairs excluded, no bond term) of a tabulated
    potential on each frame, through the library."""
    import torch
    from paper_2608_14911_gb300 import espp
    h = espp.System(box, n, None, bonds, precision=espp.ESPP_FP32, seed=5)
    h.set_table_pair(RCM, ut, ft)
    h.set_exclude_bonded(True)
    out = torch.zeros_like(frames)
    for k in range(frames.shape[0]):
        h.set_state(frames[k])
        if k == 0:
            h.build_neighbors(RCM, SKIN_CG)
        h.compute_forces(out[k])
    h.close()
    return out


def suite_learned_cg(a, sync, out):
    """Learned CG: a fine KG melt of 2000 chains x 200 beads is mapped 4:1 onto
    100k sites every 200 steps; the CG bond table comes from Boltzmann
    inversion; the MLP pair potential is force-matched on the frames; its
    yardstick is an independent tabulated pair potential made from the mapped
    g(r) alone (Boltzmann inversion refined by iterative Boltzmann
    inversion).  Both are compared with the mapped fine melt (g(r) and
    held-out forces); then a 4M-site CG melt runs with the MLP on the tensor
    cores and with the IBI table.  Results go into `out` as they are
    measured, and `out["stage"]` names the part that ran last."""
    import torch
    from paper_2608_14911_gb300 import espp, inputs
    # ---- fine run and frames --------------------------------------------------
    out["stage"] = "fine melt"
    nch, nb, bps = 2000, 200, 4
    f, cfg, start = make_melt(a, 42, espp.ESPP_FP32, nchains=nch, nbeads=nb)
    f.integrate(1000, 0.005, 1.0, 1.0)
    out["fine_start"] = start
    ns = cfg.n // bps
    F = a.cg_frames
    X = torch.zeros((F, ns, 3), dtype=torch.float64, device="cuda")
    Y = torch.zeros_like(X)
    t0 = time.perf_counter()
    for k in range(F):
        f.integrate(200, 0.005, 1.0, 1.0)
        f.cg_map(bps, X[k], Y[k])
    sync()
    frames_s = time.perf_counter() - t0
    f.close()
    sites_per_chain = nb // bps
    every = max(1, F // 200)
    bond_tab = _bond_table_boltzmann(X[::every].cpu().numpy(), nch, sites_per_chain, cfg.box)
    x_start = X[F - max(1, F // 10)].cpu().numpy()  # first held-out frame: the start of the CG runs
    cg_bonds = inputs.chain_bonds(nch, sites_per_chain)
    n_hold = max(1, F // 10)
    n_train = F - n_hold
    out["frames"] = {"frames": F, "frames_spec": 2000, "steps_between": 200, "sites": ns,
                     "train": n_train, "held_out": n_hold, "generation_s": frames_s}
    # ---- target: the mapped fine melt's non-bonded g(r) ----------------------
    out["stage"] = "mapped g(r)"
    probe = _cg_handle(cfg.box, ns, cg_bonds, bond_tab, None, 43)
    nbin = int(round(RCM / DR_G))
    tgt_total = np.zeros(nbin)
    tframes = list(range(0, F, every))
    for k in tframes:
        probe.set_state(X[k])
        if k == 0:
            probe.build_neighbors(RCM, SKIN_FRAMES)
        tgt_total += probe.rdf_counts(RCM, nbin)
    g_t = _gofr(tgt_total / len(tframes), ns, cfg.box)
    # ---- IBI table: Boltzmann inversion + iterative Boltzmann inversion -----
    out["stage"] = "IBI table (IBI)"
    rt = np.linspace(0.0, RCM, 4096)
    U, first_t = _boltzmann_start(g_t, tgt_total)
    vmax = inputs.maxwell_velocities(ns, 1.0, seed=47)
    ibi_l2, ibi_fmax, best = [], [], None
    for it in range(a.ibi_iters):
        ut, ft = _table_from_potential(U, rt)
        ibi_fmax.append(float(np.abs(ft).max()))
        h = _cg_handle(cfg.box, ns, cg_bonds, bond_tab, ("table", ut, ft), 100 + it)
        c = _sampled_rdf(h, x_start, vmax, a.cg_eq, a.cg_snap, 25)
        h.close()
        g = _gofr(c, ns, cfg.box)
        l2 = _rdf_l2(g, g_t)
        ibi_l2.append(l2)
        if best is None or l2 < best[0]:
            best = (l2, ut.copy(), ft.copy(), U.copy())
        U = _ibi_update(U, g, g_t, c * a.cg_snap, first_t, damping=a.ibi_damping)
    _, ut, ft, _ = best
    out["ibi_table"] = {"method": "Boltzmann inversion of the mapped non-bonded g(r) (bins with >= 100 sampled "
                                    "pairs; the core continued linearly), then %d iterations of iterative Boltzmann "
                                    "inversion (damping %.2f), the best kept" % (a.ibi_iters, a.ibi_damping),
                          "rdf_l2_per_iteration": ibi_l2, "max_abs_force_per_iteration": ibi_fmax,
                          "core_below_r": first_t * DR_G}
    probe.close()
    # ---- training -------------------------------------------------------------
    out["stage"] = "training"
    g = np.random.default_rng(4)
    lim1, lim2, lim3 = np.sqrt(6 / (32 + 64)), np.sqrt(6 / 128), np.sqrt(6 / 65)
    w0 = np.concatenate([g.uniform(-lim1, lim1, 64 * 32), np.zeros(64), g.uniform(-lim2, lim2, 64 * 64),
                         np.zeros(64), g.uniform(-lim3, lim3, 64), [0.0]])
    bits = espp.to_bf16_bits(w0)
    c = _cg_handle(cfg.box, ns, cg_bonds, bond_tab, ("mlp", bits), 43)
    c.set_state(X[0])
    c.build_neighbors(RCM, SKIN_FRAMES)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    sync()
    e0.record()
    loss = c.mlp_train(X[:n_train], Y[:n_train], batch_frames=a.cg_batch, epochs=a.cg_epochs, lr=1e-3, seed=4)
    e1.record()
    sync()
    train_ms = e0.elapsed_time(e1)
    trained = c.mlp_weights()
    # tensor work of one frame: unique pairs inside the cutoff x (24576 flop
    # forward, values and tangents, + 2 x 24576 backward to the weights)
    tr_pairs = float(c.rdf_counts(RCM, nbin).sum())
    tr_flop = 3 * 24576.0 * tr_pairs
    tr_s = train_ms / 1e3 / a.cg_epochs / n_train
    peaks_t, peak_kind_t = measured_peaks()
    tr_peak = peaks_t.get("bf16_tflops_sustained", peaks_t["bf16_tflops"])
    c.close()
    # ---- held-out forces and losses: zero pair force, IBI table, MLP ------
    out["stage"] = "held-out forces"
    models = {"zero_pair": None, "ibi_table": ("table", ut, ft), "mlp": ("mlp", trained)}
    held = {}
    for name, pair in models.items():
        h = _cg_handle(cfg.box, ns, cg_bonds, bond_tab, pair, 44)
        se = den = 0.0
        fq = torch.zeros((ns, 3), dtype=torch.float64, device="cuda")
        for q in range(n_hold):
            h.set_state(X[n_train + q])
            if q == 0:
                h.build_neighbors(RCM, SKIN_FRAMES)
            h.compute_forces(fq)
            yq = Y[n_train + q]
            se += float(((fq - yq) ** 2).sum())
            den += float((yq ** 2).sum())
        h.close()
        held[name] = {"loss": se / (n_hold * ns), "force_rel_rms": float(np.sqrt(se / den))}
    out["training"] = {"workload": "kg_2000x200_mapped_4to1_100000_sites", "frames_train": n_train,
                       "frames_spec": 2000, "epochs": a.cg_epochs, "epochs_spec": 50, "batch_frames": a.cg_batch,
                       "adam_steps": a.cg_epochs * (-(-n_train // a.cg_batch)),
                       "s_per_epoch": train_ms / 1e3 / a.cg_epochs,
                       "s_per_epoch_per_frame": tr_s,
                       "loss_per_epoch": [float(v) for v in loss],
                       "held_out": held,
                       "loss_note": "force-matching loss = mean over frames and sites of |F_pair + F_bond - F_mapped|^2; "
                                    "training loss per epoch on the training frames, held-out losses on the last "
                                    "%d frames; zero_pair = bonds only (the floor any pair model must beat)" % n_hold,
                       "cg_mean_bond": bond_tab[3],
                       "roofline": {"bound": "tensor", "unique_pairs_per_frame": tr_pairs,
                                    "flop_per_frame": tr_flop, "achieved": tr_flop / tr_s / 1e12,
                                    "unit": "TFLOP/s", "peak": tr_peak, "frac": tr_flop / tr_s / 1e12 / tr_peak,
                                    "peak_kind": peak_kind_t + " (bf16_tflops_sustained)",
                                    "timed": "whole epochs: state upload, list build, forces, gradient, Adam"}}
    # ---- structure: MLP and IBI table against the mapped g(r) ---------------
    out["stage"] = "structure at 100k sites"
    gs = {}
    for name in ("mlp", "ibi_table"):
        h = _cg_handle(cfg.box, ns, cg_bonds, bond_tab, models[name], 61)
        gs[name] = _gofr(_sampled_rdf(h, x_start, vmax, a.cg_eq, 2 * a.cg_snap, 25), ns, cfg.box)
        h.close()
    out["structure"] = {"rdf_l2_mlp_vs_mapped": _rdf_l2(gs["mlp"], g_t),
                        "rdf_l2_table_vs_mapped": _rdf_l2(gs["ibi_table"], g_t),
                        "rdf_l2_mlp_vs_table": _rdf_l2(gs["mlp"], gs["ibi_table"]),
                        "protocol": "100k CG sites from a held-out mapped frame, Langevin T 1, %d steps, then g(r) "
                                    "(non-bonded pairs, dr %.2f to %.1f) over %d snapshots 25 steps apart; target: "
                                    "the mapped g(r) of %d frames" % (a.cg_eq, DR_G, RCM, 2 * a.cg_snap, len(tframes))}
    # ---- structure refinement of the learned potential ------------------------
    # Force matching fixes the potential of mean force only as far as a pair
    # potential can project the mapped forces; the structure it gives is off
    # by the many-body part.  Each refinement iteration simulates the current
    # MLP, turns its g(r) error into a pair correction (one iterative
    # Boltzmann inversion step) and trains the MLP, from its current weights,
    # to the forces of the current MLP plus the correction's pair forces on
    # mapped training frames (targets free of the mapped forces' noise, so the
    # fit takes the correction up exactly).  The best iteration (g(r) against
    # the mapped one) is kept.
    refined = trained
    if a.refine_iters > 0:
        out["stage"] = "structure refinement"
        n_ref = min(n_train, a.refine_frames)
        idx = torch.linspace(0, n_train - 1, n_ref).round().long().to(X.device)
        Xr, Yr = X[idx].contiguous(), Y[idx].contiguous()
        C = np.zeros(nbin)
        w = trained
        ref_l2, ref_loss, best_r = [], [], None
        t0 = time.perf_counter()
        for it in range(a.refine_iters):
            h = _cg_handle(cfg.box, ns, cg_bonds, bond_tab, ("mlp", w), 300 + it)
            cnt = _sampled_rdf(h, x_start, vmax, a.cg_eq, a.cg_snap, 25)
            h.close()
            gk = _gofr(cnt, ns, cfg.box)
            l2 = _rdf_l2(gk, g_t)
            ref_l2.append(l2)
            if best_r is None or l2 < best_r[0]:
                best_r = (l2, w, it)
            if it == a.refine_iters - 1:
                break
            dC = _correction_update(np.zeros(nbin), gk, g_t, cnt * a.cg_snap, first_t, damping=a.refine_damping)
            C = C + dC
            uc, fc = _table_from_potential(dC, rt)
            h = _cg_handle(cfg.box, ns, cg_bonds, bond_tab, ("mlp", w), 43)
            Yc = _pair_forces_of_table(cfg.box, ns, cg_bonds, uc, fc, Xr)
            fk = torch.zeros((ns, 3), dtype=torch.float64, device="cuda")
            for k in range(n_ref):
                h.set_state(Xr[k])
                if k == 0:
                    h.build_neighbors(RCM, SKIN_FRAMES)
                h.compute_forces(fk)
                Yc[k] += fk
            lh = h.mlp_train(Xr, Yc, batch_frames=a.cg_batch, epochs=a.refine_epochs, lr=1e-3, seed=5 + it)
            ref_loss.append(float(lh[-1]))
            w = h.mlp_weights()
            h.close()
        refined = best_r[1]
        out["refinement"] = {"iterations": a.refine_iters, "frames": n_ref, "epochs_per_iteration": a.refine_epochs,
                             "rdf_l2_per_iteration": ref_l2, "fine_tune_loss_per_iteration": ref_loss,
                             "kept_iteration": best_r[2], "wall_s": time.perf_counter() - t0,
                             "correction_max_abs": float(np.abs(C).max()),
                             "method": "iteration k: g(r) of the current MLP (100k sites, %d steps, %d snapshots); "
                                       "correction dC = %.2f kT ln(g / g_mapped) (IBI step on the well-sampled "
                                       "bins); target forces on %d mapped training frames = the current MLP's "
                                       "forces + dC's pair forces; %d epochs of force matching on them from the "
                                       "current weights (Adam, lr 1e-3)" % (a.cg_eq, a.cg_snap, a.refine_damping,
                                                                          n_ref, a.refine_epochs)}
        # held-out forces and structure of the refined model
        h = _cg_handle(cfg.box, ns, cg_bonds, bond_tab, ("mlp", refined), 44)
        se = den = 0.0
        fq = torch.zeros((ns, 3), dtype=torch.float64, device="cuda")
        for q in range(n_hold):
            h.set_state(X[n_train + q])
            if q == 0:
                h.build_neighbors(RCM, SKIN_FRAMES)
            h.compute_forces(fq)
            yq = Y[n_train + q]
            se += float(((fq - yq) ** 2).sum())
            den += float((yq ** 2).sum())
        h.close()
        out["training"]["held_out"]["mlp_refined"] = {"loss": se / (n_hold * ns),
                                                      "force_rel_rms": float(np.sqrt(se / den))}
        h = _cg_handle(cfg.box, ns, cg_bonds, bond_tab, ("mlp", refined), 61)
        g_ref = _gofr(_sampled_rdf(h, x_start, vmax, a.cg_eq, 2 * a.cg_snap, 25), ns, cfg.box)
        h.close()
        out["structure"]["rdf_l2_mlp_refined_vs_mapped"] = _rdf_l2(g_ref, g_t)
        out["structure"]["rdf_l2_mlp_refined_vs_table"] = _rdf_l2(g_ref, gs["ibi_table"])
    # ---- 4M CG sites: MLP on tensor cores vs the IBI table -------------------
    out["stage"] = "4M CG melt"
    cg = inputs.kg_lattice(16000, 250, density=0.2125, seed=44, jitter=0.1)
    res = {}
    forces = {}
    n_snap, snap_every = 40, 20
    for mode in ("mlp", "table"):
        out["stage"] = "4M CG melt, " + mode
        s = espp.System(cg.box, cg.n, None, cg.bonds, precision=espp.ESPP_FP32, seed=45)
        if mode == "mlp":
            s.set_mlp(RCM, refined)
        else:
            s.set_table_pair(RCM, ut, ft)
        s.set_table_bond(*bond_tab[:3])
        s.set_exclude_bonded(True)
        s.set_state(cg.x, inputs.maxwell_velocities(cg.n, 1.0, seed=46), cg.img)
        s.build_neighbors(RCM, SKIN_CG)
        forces[mode] = s.compute_forces()
        s.integrate(a.cg_warm, 0.005, 1.0, 1.0)
        steps = a.cg_steps
        ms = _timed(s, steps, 0.005, 1.0, 1.0, sync)
        # force-evaluation time per step (the learned potential's kernels and
        # the step kernel), from events around the graph's step nodes
        s.set_kernel_timing(True)
        for _ in range(2):
            s.integrate(64, 0.005, 1.0, 1.0)
        kt = s.kernel_timing(reset=True)
        s.set_kernel_timing(False)
        counts = np.zeros(nbin)
        for _ in range(n_snap):
            s.integrate(snap_every, 0.005, 1.0, 1.0)
            counts += s.rdf_counts(RCM, nbin)
        counts /= n_snap
        res[mode] = {"value": cg.n * steps / (ms / 1e3), "unit": "site-steps/s", "steps": steps,
                     "steps_spec": 10000, "ms_per_step": ms / steps,
                     "fine_bead_equivalent": 4 * cg.n * steps / (ms / 1e3),
                     "force_eval_ms": kt["step_ms"] / max(1, kt["step_launches"])}
        res[mode]["_rdf"] = counts
        s.close()
    cm = res["mlp"].pop("_rdf")
    ct = res["table"].pop("_rdf")
    ga, gb = _gofr(cm, cg.n, cg.box), _gofr(ct, cg.n, cg.box)
    # tensor-core work of the learned potential: unique non-bonded pairs inside
    # the cutoff x 24576 flop (two 32x64 and two 64x64 multiply-adds per pair:
    # u and its r-derivative)
    pairs = float(cm.sum())
    flop = 24576.0 * pairs
    peaks, peak_kind = measured_peaks()
    fe = res["mlp"]["force_eval_ms"]
    res["mlp"]["roofline"] = {"bound": "tensor", "unique_pairs": pairs, "flop_per_step": flop,
                              "achieved": flop / (fe * 1e-3) / 1e12, "unit": "TFLOP/s",
                              "peak": peaks.get("bf16_tflops_sustained", peaks["bf16_tflops"]),
                              "frac": flop / (fe * 1e-3) / 1e12 / peaks.get("bf16_tflops_sustained",
                                                                            peaks["bf16_tflops"]),
                              "peak_kind": peak_kind + " (bf16_tflops_sustained: timed inside a long run)",
                              "timed": "all force kernels of a step (pairs, gather, step kernel)"}
    out["cg4m"] = {"workload": "cg_melt_16000x250_4000000_sites_rho0.2125", "n_sites": cg.n,
                   "mlp": res["mlp"], "table": res["table"],
                   "force_rel_rms_mlp_vs_table": float(np.sqrt(((forces["mlp"] - forces["table"]) ** 2).sum()
                                                               / (forces["table"] ** 2).sum())),
                   "rdf_l2_mlp_vs_table": _rdf_l2(ga, gb),
                   "rdf_note": "g(r), dr 0.02, averaged over %d snapshots %d steps apart after %d + %d + 128 steps "
                               "from the same lattice start, for both potentials" % (n_snap, snap_every, a.cg_warm,
                                                                                     a.cg_steps)}
    out["stage"] = "done"


def run_cg_probe(a):
    """A CG melt of a.cg_probe sites (density 0.2125, chains of 250) with a
    random learned potential and a tabulated bond: five force evaluations."""
    import torch
    import __graft_entry__ as g
    g.build()
    from paper_2608_14911_gb300 import espp, inputs
    nch = max(1, a.cg_probe // 250)
    cg = inputs.kg_lattice(nch, 250, density=0.2125, seed=44, jitter=0.1)
    rng = np.random.default_rng(4)
    w = np.concatenate([rng.normal(0, 0.18, 64 * 32), np.zeros(64), rng.normal(0, 0.125, 64 * 64), np.zeros(64),
                        rng.normal(0, 0.06, 64), [0.0]])
    s = espp.System(cg.box, cg.n, None, cg.bonds, precision=espp.ESPP_FP32, seed=1)
    s.set_mlp(3.5, espp.to_bf16_bits(w))
    rb = np.linspace(0.0, 4.0, 801)
    s.set_table_bond(4.0, 5.0 * (rb - 2.0) ** 2, -10.0 * (rb - 2.0))
    s.set_exclude_bonded(True)
    s.set_state(cg.x, None, cg.img)
    s.build_neighbors(3.5, 0.5)
    out = torch.zeros((cg.n, 3), dtype=torch.float64, device="cuda")
    for _ in range(5):
        s.compute_forces(out)
    torch.cuda.synchronize()
    print(json.dumps({"cg_probe_sites": cg.n}))
    return 0


def run_train_probe(a):
    """Force-matching training on a.train_probe CG sites (chains of 50 at
    density 0.2125, 8 jittered frames with random target forces, random
    BF16 weights): one warm-up epoch, then two timed epochs."""
    import torch
    import __graft_entry__ as g
    g.build()
    from paper_2608_14911_gb300 import espp, inputs
    c = inputs.kg_lattice(max(1, a.train_probe // 50), 50, density=0.2125, seed=44, jitter=0.3)
    rng = np.random.default_rng(4)
    w = np.concatenate([rng.normal(0, 0.18, 64 * 32), np.zeros(64), rng.normal(0, 0.125, 64 * 64), np.zeros(64),
                        rng.normal(0, 0.06, 64), [0.0]])
    nf = 8
    X = np.stack([inputs.f32(np.mod(c.x + rng.normal(0, 0.3, c.x.shape), c.box)) for _ in range(nf)])
    X[X >= c.box] = 0.0
    Xd = torch.tensor(X, device="cuda")
    Yd = torch.tensor(rng.normal(0, 1.0, X.shape), device="cuda")
    s = espp.System(c.box, c.n, None, c.bonds, precision=espp.ESPP_FP32, seed=1)
    s.set_mlp(RCM, espp.to_bf16_bits(w))
    rb = np.linspace(0.0, 6.0, 1201)
    s.set_table_bond(6.0, 2.0 * (rb - 2.0) ** 2, -4.0 * (rb - 2.0))
    s.set_exclude_bonded(True)
    s.set_state(X[0])
    s.build_neighbors(RCM, SKIN_CG)
    s.mlp_train(Xd, Yd, batch_frames=4, epochs=1, lr=1e-3, seed=1)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record()
    loss = s.mlp_train(Xd, Yd, batch_frames=4, epochs=2, lr=1e-3, seed=1)
    e1.record()
    torch.cuda.synchronize()
    print(json.dumps({"train_probe_sites": c.n, "ms_per_frame_epoch": e0.elapsed_time(e1) / (2 * nf),
                      "loss": [float(v) for v in loss]}))
    return 0


def main():
    a = parse()
    if a.cg_probe:
        return run_cg_probe(a)
    if a.train_probe:
        return run_train_probe(a)
    if a.impl == "reference":
        return run_reference(a)
    return run_ours(a)


if __name__ == "__main__":
    sys.exit(main())

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
    ap.add_argument("--quick-start", action="store_true",
                    help="lattice start with a short equilibration (for profiler runs)")
    return ap.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


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
        self.path = os.path.join(ROOT, "gpurun_out", "clocks_bench_%d.csv" % os.getpid())

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
def make_melt(a, seed, precision):
    """KG melt: random-walk chains, soft push-off with a growing force cap,
    then plain WCA; falls back to an overlap-free lattice start."""
    from paper_2608_14911_gb300 import espp, inputs
    cfg = inputs.kg_random_walk(a.nchains, a.nbeads, density=0.85, seed=seed, bond=0.97)
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
        cfg = inputs.kg_lattice(a.nchains, a.nbeads, density=0.85, seed=seed)
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
    s.integrate(steps, 0.005, 1.0, 1.0)
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


def read_traffic_record():
    """DRAM bytes per step-kernel launch from the committed ncu summary, or
    None when the kernel source changed since the capture."""
    path = os.path.join(ROOT, "profiles", "step_kernel_traffic.txt")
    src = os.path.join(ROOT, "paper_2608_14911_gb300", "csrc", "k_step.cu")
    if not os.path.exists(path):
        return None
    rec = {}
    with open(path) as fh:
        for line in fh:
            if ":" in line and not line.startswith("#"):
                k, val = line.split(":", 1)
                rec[k.strip()] = val.strip()
    digest = hashlib.sha256(open(src, "rb").read()).hexdigest()[:16]
    if rec.get("k_step_sha") != digest:
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
        if not pg:
            return x
        t = torch.tensor([x], dtype=torch.float64, device="cuda")
        pg.all_reduce(t, op=pg.ReduceOp.MAX)
        return float(t.item())

    seed = 42 + rank
    s, cfg, start = make_melt(a, seed, espp.ESPP_FP32)
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
    value = world * n * a.steps / (ms / 1e3)
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
                   "mean_list_entries_per_particle": mean_entries / n, "max_list_entries": max_count,
                   "observables_after_run": {k: obs[k] for k in ("temperature", "mean_bond", "rg2", "pe_pair")},
                   "force_error_gate": "FP32 <= 1e-5 relative RMS vs the FP64 oracle (tests/test_gpu_parity.py)"},
        "fp64": fp64,
        "roofline": roofline,
        "cpu_baseline": cpu,
        "e2e": e2e,
        "gpu_launches": gpu_launches,
        "clocks": clocks,
    }
    if rank == 0:
        print(json.dumps(line), flush=True)
    s.close()
    if pg:
        pg.destroy_process_group()
    return 0


def main():
    a = parse()
    if a.impl == "reference":
        return run_reference(a)
    return run_ours(a)


if __name__ == "__main__":
    sys.exit(main())

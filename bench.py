"""Benchmark of the SIDM scattering pass on GB300.

Workload (one "step" = one pass of the whole hot path over the halo):
  NFW halo, r_s = 1, truncated at 10 r_s, N = 1,048,576 equal-mass particles,
  isotropic Maxwellian velocities with the Jeans dispersion (seed 1),
  sigma(v)/m = 100 / (1 + (v/v_max)^2)^2 with v_max the halo's maximum circular
  velocity, N_ngb = 64, FP32 storage with exact/FP64 reductions (mixed form),
  fixed dt from the SIDM time-step proxy dt = 0.04 / q99.9(sum_j P_ij / dt)
  on the initial state.  Synthetic inputs (seeded), no datasets.
  A step = ballistic drift + cell build + kernel sizes + pair probabilities,
  draws and scatter + per-halo energy/momentum (exact integer sums of the
  FP32 velocities).  L2 is flushed (256 MiB write)
  before every timed step, outside the step's events.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
Under torchrun (N > 1) every rank runs an independent halo (seed + rank):
weak scaling, no data-path collective; rank 0 prints one JSON line.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

N_PART = 1 << 20
N_NGB = 64
S0 = 100.0
SEED_IC = 1
TAU = 0.04
DT_PROBE = 1e-6            # probe time step of the dt rule (sum_j P_ij / dt is dt-independent)
METRIC = "SIDM particle-steps/s"
UNIT = "particle-steps/s"
WORKLOAD = "nfw_rcut10_N1048576_ngb64_veldep_s0_100_w_vmax"
PEAKS = os.path.join(ROOT, "MEASURED_PEAKS.json")
# issue slots of the FP32/INT32 pipes: SMs x lanes per SM (GB300, 152 SMs x 128)
N_SM, LANES_PER_SM = 152, 128
# algorithmic lane operations per unit of the two ALU-bound kernels: the operation
# counts of the formulas as written, not counts of issued instructions
OPS_PER_TEST = 10          # canonical d^2 (3 sub, 1 mul, 2 fma), sum, square, compare, ballot
OPS_PER_PAIR = 121         # |v_ij| + sigma(v) + Philox4x32-10 + upper bound of P + draw decision + bookkeeping
OPS_PER_LAMBDA = 50        # sqrt(d^2) + Lambda table (bicubic, 16 loads) + P + exact decision, when looked up
OPS_PER_KNN_CAND = 8       # canonical d^2 (6) + key compare (2)
# the kernel-size search as the scope table counts it: about 6 N_ngb candidate
# distances of about 9 FP32 operations per particle
KNN_SCOPE_CANDS_PER_NGB, KNN_SCOPE_OPS_PER_CAND = 6, 9
PAIR_SCOPE_OPS = 130              # per in-range pair: ~60 FP32 with the Lambda table + ~70 INT32 of Philox
BUILD_BUDGET_BYTES = 184           # 12 + 12 + 4 sort passes x 24 + 32 + 32

# the paper's top resolution: cored-isothermal inner profile joined to NFW
CFG3_N, CFG3_SEED, CFG3_SWEEP = 50_000_000, 2, (16, 32, 64, 128)
CFG3_WORKLOAD = "cored_nfw_N50000000_core0.05rs_rho1e3rhos_ngb16-128_veldep_s0_100_w_vmax"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--n", type=int, default=N_PART)
    ap.add_argument("--fp64-steps", type=int, default=3)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--use-tma", type=int, default=0)
    ap.add_argument("--no-batched", action="store_true")
    ap.add_argument("--no-tune", action="store_true")
    ap.add_argument("--only", choices=["all", "streaming"], default="all",
                    help="streaming: time only the HBM-bound kernels (profiling runs; prints their block)")
    ap.add_argument("--stream-n", type=int, default=1 << 25)
    return ap.parse_args()


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def make_halo(n, seed):
    from paper_2506_06269_gb300 import ics
    h = ics.nfw(n, seed)
    return h, ics.nfw_vmax()


def load_peaks():
    try:
        with open(PEAKS) as f:
            return json.load(f), "measured"
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "sm_max_mhz": 2070.0}, "fallback"


class ClockSampler:
    """nvidia-smi clock / throttle sampling during the timed region."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0])); mx.append(float(parts[1]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[4:8]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def source_sha(path):
    import hashlib
    with open(path, "rb") as f:
        return hashlib.sha256(f.read()).hexdigest()[:16]


def load_traffic():
    """DRAM bytes per launch from the committed ncu summary, if still current.

    profiles/ncu_traffic.json maps kernel -> {"bytes_per_launch", "units_per_launch",
    "source_sha"}; an entry whose kernel source changed since the capture is ignored.
    """
    p = os.path.join(ROOT, "profiles", "ncu_traffic.json")
    src = {"pairs": "sidm_pairs.cu", "knn": "sidm_knn.cu"}
    out = {}
    try:
        with open(p) as f:
            d = json.load(f)
    except Exception:
        return out
    for k, v in d.items():
        f = os.path.join(ROOT, "paper_2506_06269_gb300", "csrc", src.get(k, ""))
        if os.path.isfile(f) and v.get("source_sha") == source_sha(f):
            out[k] = v
    return out


def dt_rule(ctx_cls, halo, vmax, device):
    """dt = 0.04 / q99.9(sum_j P_ij / dt) on the initial state (SIDM time-step proxy)."""
    import torch
    from paper_2506_06269_gb300 import sidm
    n = halo.n
    c = ctx_cls(n_max=n, halo_max=1, ngb_max=N_NGB, event_cap=16, precision="mixed", device=device,
                flags=sidm.SIDM_FLAG_SUM_P)
    dev = c.device
    pos = torch.tensor(halo.pos, device=dev)
    vel = torch.tensor(halo.vel.astype(np.float32), device=dev)
    ids = torch.tensor(halo.ids.astype(np.int64), device=dev).to(torch.int32)
    h = torch.zeros(n, dtype=torch.float32, device=dev)
    c.build_cells([0, n], pos, vel, ids)
    c.kernel_sizes([N_NGB], h)
    # sum_j P_ij / dt does not depend on dt: probe with a tiny dt so that
    # (almost) no event fires
    c.scatter_step(0, 0, c.xs_tensor([(1, S0, vmax)]), c.f64([DT_PROBE]), c.f64([halo.mass]), vel)
    c.status()
    sp = c.sum_p(n).cpu().numpy().astype(np.float64) / DT_PROBE
    c.close()
    q = float(np.quantile(sp, 0.999))
    return TAU / q, q


def max_over_ranks(value, device):
    """MAX of a per-rank scalar over the process group (timing only)."""
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(n_per_rank, world, steps, max_ms):
    """Whole-job particle-steps/s: every rank advances its own halo."""
    return world * n_per_rank * steps / (max_ms * 1e-3)


def time_steps(ctx, step_fn, k, flush, first_step):
    import torch
    s = torch.cuda.current_stream()
    e0 = [torch.cuda.Event(enable_timing=True) for _ in range(k)]
    e1 = [torch.cuda.Event(enable_timing=True) for _ in range(k)]
    for i in range(k):
        flush.zero_()
        e0[i].record(s)
        step_fn(first_step + i, i)
        e1[i].record(s)
    torch.cuda.synchronize()
    return [a.elapsed_time(b) for a, b in zip(e0, e1)]


def run_ours(args):
    import torch
    from paper_2506_06269_gb300 import build, sidm
    ws, rank, local = dist_env()
    if ws > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    build.build()
    torch.cuda.set_device(local)
    n = args.n
    halo, vmax = make_halo(n, SEED_IC + rank)
    dt, q999 = dt_rule(sidm.Context, halo, vmax, local)
    # launch knobs tuned on this workload before the timed region (none changes a result)
    knobs, tuning = {"use_tma": args.use_tma}, []
    if not args.no_tune:
        from paper_2506_06269_gb300 import tune

        def make_inputs(c):
            return (torch.tensor(halo.pos, device=c.device), torch.tensor(halo.vel.astype(np.float32), device=c.device),
                    torch.tensor(halo.ids.astype(np.int64), device=c.device).to(torch.int32))

        knobs, tuning = tune.autotune(make_inputs, [N_NGB], [(1, S0, vmax)], [dt], [halo.mass], [0, n],
                                      tma=(0, 1) if args.use_tma else (0,))
    ctx = sidm.Context(n_max=n, halo_max=1, ngb_max=N_NGB, event_cap=max(1 << 16, n // 8), precision="mixed",
                       device=local, flags=sidm.SIDM_FLAG_TIMING | sidm.SIDM_FLAG_LOCAL_DIAG, **knobs)
    dev = ctx.device
    off = [0, n]
    pos = torch.tensor(halo.pos, device=dev)
    vel = torch.tensor(halo.vel.astype(np.float32), device=dev)
    ids = torch.tensor(halo.ids.astype(np.int64), device=dev).to(torch.int32)
    h = torch.zeros(n, dtype=torch.float32, device=dev)
    xs = ctx.xs_tensor([(1, S0, vmax)])
    dt_t = ctx.f64([dt])
    mass_t = ctx.f64([halo.mass])
    K, W = args.steps, args.warmup
    stats = torch.zeros((max(K, W, 1), sidm.STATS_DTYPE.itemsize), dtype=torch.uint8, device=dev)
    energy = torch.zeros((max(K, W, 1) + 1, 4), dtype=torch.float64, device=dev)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    seed = 20250617 + rank

    def step(step_no, slot):
        ctx.drift(dt_t, pos, vel)
        ctx.build_cells(off, pos, vel, ids)
        ctx.kernel_sizes([N_NGB], h)
        ctx.scatter_step(seed, step_no, xs, dt_t, mass_t, vel, stats[slot])
        ctx.energy_momentum(mass_t, vel, energy[slot + 1])

    ctx.build_cells(off, pos, vel, ids)          # layout upload happens here, once
    for i in range(W):
        step(i, i)
    torch.cuda.synchronize()
    if ctx.status() != 0:
        raise RuntimeError(f"device status after warm-up: {ctx.status()}")
    ctx.energy_momentum(mass_t, vel, energy[0])
    ctx.kernel_times(reset=True)
    ctx.diagnostics(reset=True)
    l0 = ctx.launch_count()
    if ws > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    clk = ClockSampler(local)
    clk.start()
    times = time_steps(ctx, step, K, flush, W)
    clocks = clk.stop()
    gpu_launches = ctx.launch_count() - l0
    kms, kcnt = ctx.kernel_times(reset=True)
    diag = ctx.diagnostics(reset=True)
    status = ctx.status()
    # the kernel-size search from scratch (no previous h), same particles
    ctx.warm_start(False)
    ctx.build_cells(off, pos, vel, ids)
    for _ in range(3):
        ctx.kernel_sizes([N_NGB], h)
    torch.cuda.synchronize()
    kms_cold, kcnt_cold = ctx.kernel_times(reset=True)
    ctx.diagnostics(reset=True)
    ctx.warm_start(True)
    knn_cold_ms = float(kms_cold[1] / max(kcnt_cold[1], 1))
    # local diagnostics of the evolved halo (one fused pair traversal + finalize)
    ctx.local_diagnostics(xs, mass_t, vel, n)
    d0, d1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    d0.record()
    diag_out = ctx.local_diagnostics(xs, mass_t, vel, n)
    d1.record()
    torch.cuda.synchronize()
    hl = diag_out["h_over_l"].double(); kn = diag_out["kn"].double()
    local_diag = {"ms": d0.elapsed_time(d1), "h_over_l_median": float(hl.median()), "h_over_l_max": float(hl.max()),
                  "h_over_l_q99": float(torch.quantile(hl[::16], 0.99)), "kn_median": float(kn.median()),
                  "kn_min": float(kn.min()), "G": 1.0,
                  "note": "per particle: SPH density over its kernel, kernel-weighted dispersion, sigma_eff, "
                          "h/l (Eq. hDl), Knudsen number (Eq. knudsen_number)"}
    total_ms = max_over_ranks(float(sum(times)), dev) if ws > 1 else float(sum(times))
    st = [sidm.parse_stats(stats[i]) for i in range(K)]
    E = energy.cpu().numpy()
    e0 = E[0, 0]
    drift = float(np.max(np.abs(E[1:K + 1, 0] - e0)) / abs(e0)) if K else 0.0
    book = float(sum(s.d_energy for s in st))
    n_pairs = sum(s.n_pairs for s in st)
    n_tested = sum(s.n_tested for s in st)
    n_events = sum(s.n_events for s in st)

    res = {
        "ctx": ctx, "halo": halo, "vmax": vmax, "dt": dt, "q999": q999, "times": times, "total_ms": total_ms,
        "clocks": clocks, "gpu_launches": gpu_launches, "kms": kms, "kcnt": kcnt, "status": status,
        "drift": drift, "book": book, "n_pairs": n_pairs, "n_tested": n_tested, "n_events": n_events,
        "stats": st, "ws": ws, "rank": rank, "local": local, "tensors": (pos, vel, ids, h, xs, dt_t, mass_t),
        "step": step, "seed": seed, "diag": diag, "knn_cold_ms": knn_cold_ms, "local_diag": local_diag,
        "knn_candidates_per_step": float(diag[1]) / max(K, 1), "knobs": knobs, "tuning": tuning,
    }
    return res


def run_e2e(res, steps):
    """Same metric through the C ABI with host buffers: every step copies its
    inputs (positions, velocities, ids) from pinned host memory and reads the
    results (the reordered positions and ids, the velocities and the
    energy/momentum) back; the positions and ids are read back on a second
    stream while the kernel sizes and pairs run."""
    import torch
    ctx = res["ctx"]
    halo = res["halo"]
    n = halo.n
    pos, vel, ids, h, xs, dt_t, mass_t = res["tensors"]
    # the particle state lives on the host: every step uploads it, runs the
    # pass and downloads the evolved (reordered) state and the energy
    hp = torch.tensor(pos.cpu().numpy()).pin_memory()
    hv = torch.tensor(vel.cpu().numpy()).pin_memory()
    hi = torch.tensor(ids.cpu().numpy()).pin_memory()
    out_e = torch.empty((steps, 4), dtype=torch.float64).pin_memory()
    energy = torch.zeros(4, dtype=torch.float64, device=ctx.device)
    s = torch.cuda.current_stream()
    # positions and ids are final once the cells are built (the kernel sizes
    # and the scatter change only velocities), so their download runs on a
    # second stream beside the kernel-size and pair kernels; the next upload
    # waits for it
    side = torch.cuda.Stream(device=ctx.device)
    built, copied = torch.cuda.Event(), torch.cuda.Event()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(s)
    for i in range(steps):
        if i > 0:
            s.wait_event(copied)
        pos.copy_(hp, non_blocking=True)
        vel.copy_(hv, non_blocking=True)
        ids.copy_(hi, non_blocking=True)
        ctx.drift(dt_t, pos, vel)
        ctx.build_cells([0, n], pos, vel, ids)
        built.record(s)
        side.wait_event(built)
        with torch.cuda.stream(side):
            hp.copy_(pos, non_blocking=True)
            hi.copy_(ids, non_blocking=True)
            copied.record(side)
        ctx.kernel_sizes([N_NGB], h)
        ctx.scatter_step(res["seed"], 10_000 + i, xs, dt_t, mass_t, vel)
        ctx.energy_momentum(mass_t, vel, energy)
        hv.copy_(vel, non_blocking=True)
        out_e[i].copy_(energy, non_blocking=True)
    s.wait_event(copied)
    e1.record(s)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    h2d = hp.numel() * 8 + hv.numel() * 4 + hi.numel() * 4
    d2h = hp.numel() * 8 + hv.numel() * 4 + hi.numel() * 4 + 4 * 8
    return {"value": n * steps / (ms * 1e-3), "unit": UNIT, "h2d_bytes_per_step": int(h2d),
            "d2h_bytes_per_step": int(d2h), "steps": steps, "ms": ms}


def run_fp64(res, steps):
    """All-FP64 form of the same pass on identical inputs (FP64 positions,
    velocities, distances, kernel sizes, probabilities and updates)."""
    import torch
    from paper_2506_06269_gb300 import sidm
    halo, vmax, dt = res["halo"], res["vmax"], res["dt"]
    n = halo.n
    c = sidm.Context(n_max=n, halo_max=1, ngb_max=N_NGB, event_cap=max(1 << 16, n // 8), precision="fp64",
                     device=res["local"])
    dev = c.device
    pos = torch.tensor(halo.pos, device=dev)
    vel = torch.tensor(halo.vel.astype(np.float32).astype(np.float64), device=dev)
    ids = torch.tensor(halo.ids.astype(np.int64), device=dev).to(torch.int32)
    h = torch.zeros(n, dtype=torch.float64, device=dev)
    xs = c.xs_tensor([(1, S0, vmax)]); dt_t = c.f64([dt]); mass_t = c.f64([halo.mass])
    energy = torch.zeros((steps + 1, 4), dtype=torch.float64, device=dev)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)

    def step(step_no, slot):
        c.drift(dt_t, pos, vel)
        c.build_cells([0, n], pos, vel, ids)
        c.kernel_sizes([N_NGB], h)
        c.scatter_step(res["seed"], step_no, xs, dt_t, mass_t, vel)
        c.energy_momentum(mass_t, vel, energy[slot + 1])

    c.build_cells([0, n], pos, vel, ids)
    step(0, 0)
    torch.cuda.synchronize()
    c.energy_momentum(mass_t, vel, energy[0])
    times = time_steps(c, step, steps, flush, 1)
    E = energy.cpu().numpy()
    st = c.status()
    c.close()
    ms = float(sum(times))
    return {"value": n * steps / (ms * 1e-3), "unit": UNIT, "ms_per_step": ms / steps, "steps": steps,
            "energy_drift": float(np.max(np.abs(E[1:, 0] - E[0, 0])) / abs(E[0, 0])), "status": st}


def cpu_baseline(dt, vmax, threads=None, ns=N_PART // 2):
    """The oracle as it stands, on the host cores: one full oracle step of a
    2^19-particle realisation of the benchmark halo (same NFW profile, N_ngb,
    sigma(v), dt), about 10 s of CPU work on 16 cores; per-particle work
    depends on N_ngb, and on N only through the tree depth."""
    from oracle import oracle as O
    from paper_2506_06269_gb300 import ics
    th = threads or os.cpu_count() or 1
    O.set_num_threads(th)
    halo = ics.nfw(ns, SEED_IC)
    vel = halo.vel.astype(np.float32).astype(np.float64)
    t0 = time.perf_counter()
    r = O.step(halo.pos, vel, halo.ids, [0, ns], [N_NGB], [halo.mass], [(1, S0, vmax)], [dt], 1, 0, O.MODE_MIXED)
    sec = time.perf_counter() - t0
    cores = int(O.num_threads())
    # the same oracle on one core, on a 32,768-particle halo (about 8 s)
    n1 = 32768
    O.set_num_threads(1)
    h1 = ics.nfw(n1, SEED_IC)
    v1 = h1.vel.astype(np.float32).astype(np.float64)
    t1 = time.perf_counter()
    O.step(h1.pos, v1, h1.ids, [0, n1], [N_NGB], [h1.mass], [(1, S0, vmax)], [dt], 1, 0, O.MODE_MIXED)
    sec1 = time.perf_counter() - t1
    O.set_num_threads(th)
    return {"value": ns / sec, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"one full oracle step (kNN, pair probabilities with exact Lambda quadrature, draws, "
                      f"sequential scatter) of a {ns}-particle NFW halo drawn like the workload's, same N_ngb/sigma(v)/dt; "
                      f"{sec:.2f} s", "seconds": sec, "pairs": int(r["stats"][0]["n_pairs"]),
            "one_core": {"value": n1 / sec1, "unit": UNIT, "cores": 1,
                         "sample": f"one oracle step of a {n1}-particle halo drawn the same way; {sec1:.2f} s"}}


def run_config3(local, steps=3, n=CFG3_N, oracle_sample=True):
    """The paper's top resolution: N = 5e7 particles of a cored-isothermal halo
    (King-like core of 0.05 r_s at 1e3 rho_s joined to NFW, truncated at
    10 r_s; seed 2), sigma(v)/m of the main workload, dt by the same rule at
    N_ngb = 64.  For each N_ngb of {16, 32, 64, 128}: the initial state, one
    warm-up step (a new N_ngb starts the kernel-size search cold), then `steps`
    timed steps (drift + cell build + kernel sizes + scatter + exact E,p) with
    CUDA events and the per-kernel split.  The all-FP64 form runs the same
    steps at N_ngb = 64 on identical inputs.  The oracle baseline is one full
    oracle step of an N/64-particle realisation of the same profile."""
    import torch
    from paper_2506_06269_gb300 import ics, sidm
    halo = ics.cored_nfw(n, CFG3_SEED)
    vmax = ics.nfw_vmax()
    dt, q999 = dt_rule(sidm.Context, halo, vmax, local)
    torch.cuda.empty_cache()
    dev = torch.device("cuda", local)
    pos_h = torch.tensor(halo.pos).pin_memory()
    ids_h = torch.tensor(halo.ids.astype(np.int64)).to(torch.int32).pin_memory()
    out = {"workload": CFG3_WORKLOAD, "n_particles": n, "dt": dt,
           "dt_rule": "0.04 / q99.9(sum_j P_ij/dt) on the initial state at N_ngb = 64",
           "cross_section": f"sigma/m = {S0}/(1+(v/{vmax:.4f})^2)^2", "steps_timed": steps,
           "l2": "inputs far larger than L2 (2.4 GB of particle state)"}

    def run_form(precision, ks):
        vdt = torch.float32 if precision == "mixed" else torch.float64
        vel_h = torch.tensor(halo.vel.astype(np.float32).astype(np.float64 if precision == "fp64" else np.float32))
        vel_h = vel_h.pin_memory()
        ctx = sidm.Context(n_max=n, halo_max=1, ngb_max=max(ks), event_cap=1 << 22, precision=precision,
                           device=local, flags=sidm.SIDM_FLAG_TIMING)
        pos = torch.empty((3, n), dtype=torch.float64, device=dev)
        vel = torch.empty((3, n), dtype=vdt, device=dev)
        ids = torch.empty(n, dtype=torch.int32, device=dev)
        h = torch.zeros(n, dtype=vdt, device=dev)
        xs = ctx.xs_tensor([(1, S0, vmax)]); dt_t = ctx.f64([dt]); mass_t = ctx.f64([halo.mass])
        stats = torch.zeros((steps + 1, sidm.STATS_DTYPE.itemsize), dtype=torch.uint8, device=dev)
        energy = torch.zeros((steps + 2, 4), dtype=torch.float64, device=dev)
        rows = []
        for k in ks:
            pos.copy_(pos_h); vel.copy_(vel_h); ids.copy_(ids_h)

            def step(i, slot):
                ctx.drift(dt_t, pos, vel)
                ctx.build_cells([0, n], pos, vel, ids)
                ctx.kernel_sizes([k], h)
                ctx.scatter_step(20250617, i, xs, dt_t, mass_t, vel, stats[slot])
                ctx.energy_momentum(mass_t, vel, energy[slot + 1])

            ctx.build_cells([0, n], pos, vel, ids)
            step(0, 0)                                   # warm-up (cold kernel-size search)
            torch.cuda.synchronize()
            ctx.energy_momentum(mass_t, vel, energy[0])
            ctx.kernel_times(reset=True)
            s = torch.cuda.current_stream()
            ev = [torch.cuda.Event(enable_timing=True) for _ in range(2 * steps)]
            for i in range(steps):
                ev[2 * i].record(s)
                step(1 + i, i)
                ev[2 * i + 1].record(s)
            torch.cuda.synchronize()
            ms = [ev[2 * i].elapsed_time(ev[2 * i + 1]) for i in range(steps)]
            kms, _ = ctx.kernel_times(reset=True)
            st = [sidm.parse_stats(stats[i]) for i in range(steps)]
            E = energy.cpu().numpy()
            tot = float(sum(ms))
            rows.append({"n_ngb": k, "value": n * steps / (tot * 1e-3), "unit": UNIT, "ms_per_step": tot / steps,
                         "kernel_ms_per_step": {"build": kms[0] / steps, "knn": kms[1] / steps,
                                                "pairs": kms[2] / steps, "resolve": kms[3] / steps,
                                                "other": tot / steps - sum(kms) / steps},
                         "pair_evals_per_s": sum(x.n_pairs for x in st) / (tot * 1e-3),
                         "events_per_step": sum(x.n_events for x in st) / steps,
                         "energy_drift": float(np.max(np.abs(E[1:steps + 1, 0] - E[0, 0])) / abs(E[0, 0])),
                         "device_status": ctx.status()})
        ctx.close()
        del pos, vel, ids, h
        torch.cuda.empty_cache()
        return rows

    out["sweep"] = run_form("mixed", CFG3_SWEEP)
    out["fp64_form"] = run_form("fp64", (64,))[0]
    mixed64 = [r for r in out["sweep"] if r["n_ngb"] == 64][0]
    out["mixed_over_fp64_ngb64"] = mixed64["value"] / out["fp64_form"]["value"]
    if oracle_sample:
        from oracle import oracle as O
        ns = n // 64
        th = os.cpu_count() or 1
        O.set_num_threads(th)
        small = ics.cored_nfw(ns, CFG3_SEED)
        vel = small.vel.astype(np.float32).astype(np.float64)
        t0 = time.perf_counter()
        O.step(small.pos, vel, small.ids, [0, ns], [64], [small.mass], [(1, S0, vmax)], [dt], 1, 0, O.MODE_MIXED)
        sec = time.perf_counter() - t0
        out["cpu_baseline"] = {"value": ns / sec, "unit": UNIT, "cores": int(O.num_threads()), "kind": "oracle",
                               "sample": f"one full oracle step (kNN, pair probabilities with exact Lambda "
                                         f"quadrature, draws, sequential scatter) of an N/64 = {ns}-particle "
                                         f"realisation of the same cored profile, N_ngb = 64, same sigma(v) and dt; "
                                         f"{sec:.1f} s", "seconds": sec}
    return out


def run_resolve_dense(res, steps=3, dt_scale=40.0):
    """The resolve (a4) where events are dense: the benchmark halo with its
    dt times dt_scale, so particles scatter several times per step.  The
    claim-based resolve (one CTA) against the per-particle-list resolve
    (cooperative launch over all SMs, SIDM_FLAG_DRAG contexts) on the same
    events: rounds, events and CUDA-event time of each."""
    import torch
    from paper_2506_06269_gb300 import sidm
    halo, vmax = res["halo"], res["vmax"]
    n = halo.n
    out = {"workload": f"benchmark halo, dt x {dt_scale:g}", "dt": res["dt"] * dt_scale}
    for name, flags in (("claims_one_cta", 0), ("lists_all_sms", sidm.SIDM_FLAG_DRAG)):
        c = sidm.Context(n_max=n, halo_max=1, ngb_max=N_NGB, event_cap=1 << 22, device=res["local"],
                         flags=flags | sidm.SIDM_FLAG_TIMING)
        dev = c.device
        pos = torch.tensor(halo.pos, device=dev)
        vel = torch.tensor(halo.vel.astype(np.float32), device=dev)
        ids = torch.tensor(halo.ids.astype(np.int64), device=dev).to(torch.int32)
        h = torch.zeros(n, dtype=torch.float32, device=dev)
        xs, dt, mass = c.xs_tensor([(1, S0, vmax)]), c.f64([res["dt"] * dt_scale]), c.f64([halo.mass])
        c.build_cells([0, n], pos, vel, ids)
        c.kernel_sizes([N_NGB], h)
        c.scatter_step(5, 0, xs, dt, mass, vel)                # warm-up
        c.kernel_times(reset=True)
        st = []
        for i in range(steps):
            c.scatter_step(5, 1 + i, xs, dt, mass, vel)
            st.append(c.stats())
        ms, cnt = c.kernel_times(reset=True)
        out[name] = {"ms_per_step": ms[3] / steps, "events_per_step": float(np.mean([x.n_events for x in st])),
                     "rounds": int(max(x.rounds for x in st)), "multi_hit_particles": int(st[-1].n_multi),
                     "device_status": c.status()}
        c.close()
    return out


def run_satellite(local, big_steps=8, n=1 << 22, n_bins=4, dt_max=0.02):
    """NFW subhalo of 2^22 particles at the paper's initial position and velocity
    (123.6 kpc, 109 km/s) in its six-part Milky-Way-like host (NFW halo,
    Hernquist bulge, four Miyamoto-Nagai disks), in the code units of the
    subhalo: kick-drift-kick with the host's analytic force on 4 power-of-two
    individual steps, bins from the SIDM time-step criterion (tau = 0.04) of
    the previous big step, sigma(v) of the main workload; cells and kernel
    sizes every sub-step."""
    import torch
    from paper_2506_06269_gb300 import ics, sidm
    halo = ics.nfw(n, 4)
    vmax = ics.nfw_vmax()
    host = ics.milky_way_host()
    x0, v0 = ics.satellite_orbit()
    ctx = sidm.Context(n_max=n, halo_max=1, ngb_max=N_NGB, event_cap=max(1 << 16, n // 8), device=local,
                       flags=sidm.SIDM_FLAG_SUM_P)
    dev = ctx.device
    pos = torch.tensor(halo.pos + x0[:, None], device=dev)
    vel = torch.tensor((halo.vel + v0[:, None]).astype(np.float32), device=dev)
    ids = torch.tensor(halo.ids.astype(np.int64), device=dev).to(torch.int32)
    h = torch.zeros(n, dtype=torch.float32, device=dev)
    phi = torch.zeros(n, dtype=torch.float64, device=dev)
    xs = ctx.xs_tensor([(1, S0, vmax)])
    mass = ctx.f64([halo.mass])
    S = 1 << (n_bins - 1)
    dtt = ctx.f64([dt_max / S])
    dtm = ctx.f64([dt_max])
    bins = torch.zeros(n, dtype=torch.int32, device=dev)
    stats = torch.zeros((big_steps * S, sidm.STATS_DTYPE.itemsize), dtype=torch.uint8, device=dev)

    def energy():
        ctx.host_potential(host, pos, phi)
        return float((0.5 * (vel.double() ** 2).sum(0) + phi).sum().item()) * halo.mass

    def big_step(k, record):
        nonlocal bins
        nxt = bins
        for s in range(S):
            ctx.host_kick(host, dt_max, n_bins, s, 0, bins, pos, vel)
            ctx.build_cells([0, n], pos, vel, ids)
            pm = ctx.perm(n).to(torch.int64)
            bins, nxt = bins[pm], nxt[pm]                     # bins travel with their particles
            ctx.kernel_sizes([N_NGB], h)
            ctx.scatter_step_binned(SEED_IC, k * S + s, xs, dt_max, n_bins, s, bins, mass, vel,
                                    stats[k * S + s] if record else None)
            if s == 0:                                        # every step opens: rates of all pairs
                _, nxt, _ = ctx.timestep_criterion(0.04, 0.0, dt_max, n_bins, dtm, n, 1)
            ctx.drift(dtt, pos, vel)
            ctx.host_kick(host, dt_max, n_bins, s, 1, bins, pos, vel)
        bins = nxt                                            # the next big step's bins

    ctx.build_cells([0, n], pos, vel, ids)                   # layout for the first kicks
    big_step(0, False)
    torch.cuda.synchronize()
    e0 = energy()
    t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    t0.record()
    for k in range(big_steps):
        big_step(k, True)
    t1.record()
    torch.cuda.synchronize()
    ms = t0.elapsed_time(t1)
    e1 = energy()
    st = [sidm.parse_stats(stats[i]) for i in range(big_steps * S)]
    hist = torch.bincount(bins.long(), minlength=n_bins).cpu().tolist()
    status = ctx.status()
    ctx.close()
    return {"workload": "NFW subhalo N=2^22 from 123.6 kpc at 109 km/s in the six-part Milky-Way-like host "
                        "(NFW + Hernquist bulge + 4 Miyamoto-Nagai disks), "
                        "KDK with the host force, 4 power-of-two bins from the SIDM criterion (tau 0.04), "
                        f"sigma/m = {S0}/(1+(v/v_max)^2)^2, N_ngb = {N_NGB}",
            "n_particles": n, "big_steps": big_steps, "substeps_per_big_step": S, "dt_max": dt_max,
            "particle_substeps_per_s": n * big_steps * S / (ms * 1e-3),
            "particle_big_steps_per_s": n * big_steps / (ms * 1e-3), "ms_per_big_step": ms / big_steps,
            "energy_drift_rel": abs(e1 - e0) / abs(e0),
            "events_total": int(sum(x.n_events for x in st)),
            "events_by_substep_index": [float(np.mean([st[k * S + s].n_events for k in range(big_steps)]))
                                        for s in range(S)],
            "bins_last": hist, "device_status": status}


def run_streaming(local, n=1 << 25, reps=5):
    """The HBM-bound kernels of the step on a halo far larger than L2: 2^25
    particles uniform in a cube (seeded, generated on the device), FP32
    velocities.  Times the cell build (Morton keys, 7-pass radix sort, gather,
    leaf boxes, tree), the drift and the energy/momentum sums with CUDA
    events, and reports algorithmic bytes / time against the measured HBM
    peak.  Algorithmic bytes per particle: build 456 (bbox 24, keys 24 + 12,
    digit counts 8, 7 sort passes x 24, gather 52 + 64, copy-back 80, leaf
    boxes 24), drift 60 (pos 24 read + 24 write, vel 12), energy 12 (one read
    of the velocities).  The build is also given against the 184 B/particle
    budget of a build with 4 sort passes and 32-byte records (pos 12 read,
    key + index 12 written, 4 x 24, gather 32 + 32).  After the first build the
    particles arrive in the previous build's order, as they do in a step."""
    import torch
    from paper_2506_06269_gb300 import sidm
    peaks, src = load_peaks()
    g = torch.Generator(device=f"cuda:{local}")
    g.manual_seed(SEED_IC)
    ctx = sidm.Context(n_max=n, halo_max=1, ngb_max=N_NGB, event_cap=1 << 16, device=local)
    dev = ctx.device
    pos = torch.rand((3, n), generator=g, dtype=torch.float64, device=dev)
    vel = torch.randn((3, n), generator=g, dtype=torch.float32, device=dev)
    ids = torch.arange(n, dtype=torch.int32, device=dev)
    dt = ctx.f64([1e-6])
    mass = ctx.f64([1.0 / n])
    out = torch.zeros((1, 4), dtype=torch.float64, device=dev)
    ctx.build_cells([0, n], pos, vel, ids)

    def timed(fn):
        fn()
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        for _ in range(reps):
            fn()
        b.record()
        torch.cuda.synchronize()
        return a.elapsed_time(b) / reps

    legs = {"build": (lambda: ctx.build_cells([0, n], pos, vel, ids), 456),
            "drift": (lambda: ctx.drift(dt, pos, vel), 60),
            "energy_momentum": (lambda: ctx.energy_momentum(mass, vel, out), 12)}
    res = {"n_particles": n, "workload": f"uniform cube, {n} particles (seeded, on the device)",
           "peak_gbs": peaks["hbm_gbs"], "peak_source": src}
    for name, (fn, bpp) in legs.items():
        ms = timed(fn)
        gbs = bpp * n / (ms * 1e-3) / 1e9
        res[name] = {"ms": ms, "bytes_per_particle": bpp, "achieved_gbs": gbs, "frac": gbs / peaks["hbm_gbs"]}
    sg = BUILD_BUDGET_BYTES * n / (res["build"]["ms"] * 1e-3) / 1e9
    res["build"]["against_budget"] = {"bytes_per_particle": BUILD_BUDGET_BYTES, "achieved_gbs": sg,
                                      "frac": sg / peaks["hbm_gbs"]}
    res["device_status"] = ctx.status()
    ctx.close()
    return res


def run_batched(local, graph_steps=50, seq_steps=2):
    """64 independent NFW halos in one persistent launch per kernel, 50 steps
    captured in one CUDA graph, against 64 sequential single-halo contexts."""
    import torch
    from paper_2506_06269_gb300 import ics, sidm, tune
    rng = np.random.default_rng(3)
    H = 64
    sizes = np.round(10.0 ** rng.uniform(4.0, math.log10(2e6), H)).astype(np.int64)
    halos = [ics.nfw(int(sizes[h]), 3 * 1000 + h) for h in range(H)]
    b = ics.batch(halos)
    n = b.n
    ks = [[16, 32, 64, 128][h % 4] for h in range(H)]
    xs_list = [(0, 10.0, 1.0)] * H
    dev = torch.device("cuda", local)
    # Δt per halo by the same rule (q99.9 of sum_j P_ij/Δt on the initial state)
    c = sidm.Context(n_max=n, halo_max=H, ngb_max=128, event_cap=16, device=local, flags=sidm.SIDM_FLAG_SUM_P)
    pos = torch.tensor(b.pos, device=dev); vel = torch.tensor(b.vel.astype(np.float32), device=dev)
    ids = torch.tensor(b.ids.astype(np.int64), device=dev).to(torch.int32)
    hbuf = torch.zeros(n, dtype=torch.float32, device=dev)
    c.build_cells(b.offsets, pos, vel, ids); c.kernel_sizes(ks, hbuf)
    c.scatter_step(0, 0, c.xs_tensor(xs_list), c.f64([DT_PROBE] * H), c.f64(b.mass), vel)
    c.status()
    sp = c.sum_p(n).cpu().numpy().astype(np.float64) / DT_PROBE
    c.close()
    dts = [TAU / float(np.quantile(sp[b.offsets[h]:b.offsets[h + 1]], 0.999)) for h in range(H)]

    def make_inputs(ctx):
        return (torch.tensor(b.pos, device=dev), torch.tensor(b.vel.astype(np.float32), device=dev),
                torch.tensor(b.ids.astype(np.int64), device=dev).to(torch.int32))

    choice, table = tune.autotune(make_inputs, ks, xs_list, dts, b.mass, b.offsets, tma=(0, 1))
    ctx = sidm.Context(n_max=n, halo_max=H, ngb_max=128, event_cap=max(1 << 16, n // 8), device=local, **choice)
    pos, vel, ids = make_inputs(ctx)
    xs = ctx.xs_tensor(xs_list); dt_t = ctx.f64(dts); mass_t = ctx.f64(b.mass)
    E = torch.zeros((graph_steps + 1, H, 4), dtype=torch.float64, device=dev)

    def step(i, slot):
        ctx.drift(dt_t, pos, vel)
        ctx.build_cells(b.offsets, pos, vel, ids)
        ctx.kernel_sizes(ks, hbuf)
        ctx.scatter_step(777, i, xs, dt_t, mass_t, vel)
        ctx.energy_momentum(mass_t, vel, E[slot])

    ctx.build_cells(b.offsets, pos, vel, ids)
    s = torch.cuda.Stream(device=dev)
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        for i in range(2):                         # warm-up outside the graph
            step(i, 0)
        ctx.energy_momentum(mass_t, vel, E[0])
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    lc0 = ctx.launch_count()
    with torch.cuda.graph(g, stream=s):
        for i in range(graph_steps):
            step(2 + i, i + 1)
    per_step_launches = (ctx.launch_count() - lc0) / graph_steps   # kernels captured per step
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record()
    g.replay()
    e1.record()
    torch.cuda.synchronize()
    ms_graph = e0.elapsed_time(e1)
    status = ctx.status()
    Eh = E[:, :, 0].cpu().numpy()
    drift = float(np.max(np.abs(Eh[1:] - Eh[0]) / np.abs(Eh[0])))
    ctx.close()
    del g
    # 64 sequential single-halo contexts, eager launches
    ctxs = []
    for hh, halo in enumerate(halos):
        cc = sidm.Context(n_max=halo.n, halo_max=1, ngb_max=ks[hh], event_cap=max(4096, halo.n // 8), device=local,
                          **choice)
        t = (torch.tensor(halo.pos, device=dev), torch.tensor(halo.vel.astype(np.float32), device=dev),
             torch.tensor(halo.ids.astype(np.int64), device=dev).to(torch.int32),
             torch.zeros(halo.n, dtype=torch.float32, device=dev), cc.xs_tensor([xs_list[hh]]), cc.f64([dts[hh]]),
             cc.f64([halo.mass]), torch.zeros(4, dtype=torch.float64, device=dev))
        cc.build_cells([0, halo.n], t[0], t[1], t[2])
        ctxs.append((cc, t, halo.n, ks[hh]))

    def seq_step(i):
        for cc, t, nh, kh in ctxs:
            cc.drift(t[5], t[0], t[1])
            cc.build_cells([0, nh], t[0], t[1], t[2])
            cc.kernel_sizes([kh], t[3])
            cc.scatter_step(777, i, t[4], t[5], t[6], t[1])
            cc.energy_momentum(t[6], t[1], t[7])

    seq_step(0)
    torch.cuda.synchronize()
    e0.record()
    for i in range(seq_steps):
        seq_step(1 + i)
    e1.record()
    torch.cuda.synchronize()
    ms_seq = e0.elapsed_time(e1) / seq_steps
    for cc, *_ in ctxs:
        cc.close()
    return {"workload": "64 NFW halos, N log-uniform in [1e4, 2e6] (seed 3), N_ngb 16/32/64/128 round-robin, "
                        "sigma/m = 10, 50 steps in one CUDA graph",
            "n_particles": int(n), "halos": H, "graph_steps": graph_steps,
            "value": n * graph_steps / (ms_graph * 1e-3), "unit": UNIT, "ms_per_step": ms_graph / graph_steps,
            "sequential_single_halo": {"value": n / (ms_seq * 1e-3), "ms_per_step": ms_seq},
            "batched_over_sequential": (ms_seq) / (ms_graph / graph_steps),
            "energy_drift_max_halo": drift, "device_status": status, "tuned": choice, "tuning": table,
            "kernels_per_step_in_graph": per_step_launches,
            "gpu_launches": int(round(per_step_launches * graph_steps))}


def roofline(res, peaks, peak_src, name=None):
    """Roofline of one hot kernel, by default the dominant one (by measured
    event time)."""
    kms, kcnt = res["kms"], res["kcnt"]
    K = max(1, len(res["times"]))
    clock_mhz = float(peaks.get("sm_max_mhz", 2070.0))
    alu_peak = N_SM * LANES_PER_SM * clock_mhz * 1e6 / 1e12          # T lane-ops/s
    traffic = load_traffic()
    names = {0: "build", 1: "knn", 2: "pairs", 3: "resolve"}
    dom = max(range(4), key=lambda i: kms[i]) if name is None else [i for i in names if names[i] == name][0]
    name = names[dom]
    launches = max(1, int(kcnt[dom]))
    per_launch_ms = kms[dom] / launches
    n = res["halo"].n
    if name == "pairs":
        ops = (res["n_tested"] * OPS_PER_TEST + res["n_pairs"] * OPS_PER_PAIR + res["diag"][6] * OPS_PER_LAMBDA) / K
        achieved = ops / (per_launch_ms * 1e-3) / 1e12
        tr = traffic.get("pairs")
        return {"kernel": "k_pairs", "bound": "alu", "achieved": achieved, "peak": alu_peak, "unit": "Tops/s",
                "frac": achieved / alu_peak, "traffic": (tr["bytes_per_launch"] * n / tr["units_per_launch"]) if tr else None,
                "peak_source": f"derived: {N_SM} SMs x {LANES_PER_SM} FP32/INT32 lanes x {clock_mhz:.0f} MHz "
                               f"({peak_src} sm_max_mhz)",
                "ops_per_unit": {"candidate_test": OPS_PER_TEST, "pair_eval": OPS_PER_PAIR,
                                 "lambda_lookup": OPS_PER_LAMBDA},
                "scope_table_count": {"ops_per_pair": PAIR_SCOPE_OPS,
                                      "achieved": res["n_pairs"] / K * PAIR_SCOPE_OPS / (per_launch_ms * 1e-3) / 1e12,
                                      "frac": res["n_pairs"] / K * PAIR_SCOPE_OPS / (per_launch_ms * 1e-3) / 1e12
                                      / alu_peak},
                "ms_per_launch": per_launch_ms}
    if name == "knn":
        # algorithmic work = the scope table's per-particle figure (6 N_ngb
        # candidate distances of 9 operations) x the particles of one search;
        # the distances the kernels actually computed are given beside it.  A
        # warm-started search is two launches (k_knn_warm, then k_knn on the
        # leaves it hands on), so the time is per search call
        per_launch_ms = kms[dom] / K
        cand = res.get("knn_candidates_per_step")
        tr = traffic.get("knn")
        ops_pp = KNN_SCOPE_CANDS_PER_NGB * N_NGB * KNN_SCOPE_OPS_PER_CAND
        achieved = n * ops_pp / (per_launch_ms * 1e-3) / 1e12
        impl = (cand * OPS_PER_KNN_CAND) / (per_launch_ms * 1e-3) / 1e12 if cand else None
        return {"kernel": "k_knn", "bound": "alu", "achieved": achieved, "peak": alu_peak, "unit": "Tops/s",
                "frac": achieved / alu_peak,
                "traffic": (tr["bytes_per_launch"] * n / tr["units_per_launch"]) if tr else None,
                "peak_source": f"derived: {N_SM} SMs x {LANES_PER_SM} lanes x {clock_mhz:.0f} MHz ({peak_src})",
                "ops_per_unit": {"particle": ops_pp},
                "computed_distances": {"per_particle": (cand / n) if cand else None,
                                       "ops_per_distance": OPS_PER_KNN_CAND, "achieved": impl,
                                       "frac": (impl / alu_peak) if impl else None},
                "ms_per_call": per_launch_ms, "launches_per_call": launches / K}
    # the cell build is a streaming (HBM) sequence
    hbm = float(peaks.get("hbm_gbs", 6800.0))
    bytes_per_particle = 456.0
    achieved = bytes_per_particle * n / (per_launch_ms * 1e-3) / 1e9
    return {"kernel": name, "bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s",
            "frac": achieved / hbm, "traffic": None, "peak_source": f"{peak_src} hbm_gbs",
            "ms_per_launch": per_launch_ms}


def emit(line):
    print(json.dumps(line), flush=True)


def main_ours(args):
    import torch
    res = run_ours(args)
    ws, rank = res["ws"], res["rank"]
    K, W = args.steps, args.warmup
    n = res["halo"].n
    total_ms = res["total_ms"]
    value = job_throughput(n, ws, K, total_ms)
    peaks, peak_src = load_peaks()
    line = None
    # end to end on every rank at once (each its own halo): the whole-job rate
    # takes the slowest rank's time, like the device-timed value
    if ws > 1:
        torch.distributed.barrier()
    e2e = run_e2e(res, min(K, 10))
    e2e_ms = e2e.pop("ms")
    if ws > 1:
        e2e_ms = max_over_ranks(e2e_ms, torch.device("cuda", res["local"]))
    e2e["value"] = job_throughput(n, ws, e2e["steps"], e2e_ms)
    if rank == 0:
        # the legs below describe one GPU: they run at N = 1 only
        fp64 = run_fp64(res, args.fp64_steps) if args.fp64_steps > 0 and ws == 1 else None
        kms = res["kms"]
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": K, "warmup": W,
            "ms_per_step": total_ms / K, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32", "data": "synthetic",
            "config": {"workload": WORKLOAD, "n_particles": n, "n_ngb": N_NGB,
                       "cross_section": f"sigma/m = {S0}/(1+(v/{res['vmax']:.4f})^2)^2", "dt": res["dt"],
                       "dt_rule": "0.04 / q99.9(sum_j P_ij/dt) on the initial state", "precision": "mixed",
                       "step": "drift + cell build + kernel sizes + pairs/draws/scatter + exact E,p",
                       "l2": "flushed before every timed step (256 MiB write, outside the step events)",
                       "parallelism": f"replicas x{ws}" if ws > 1 else "1 GPU",
                       "launch_knobs": res["knobs"],
                       "autotuned": "coordinate descent over the launch knobs on this workload before the timed "
                                    "region (none changes a result)" if res["tuning"] else "defaults"},
            "pair_evals_per_s": ws * res["n_pairs"] / (total_ms * 1e-3),
            "events_per_step": res["n_events"] / K,
            "energy_drift": res["drift"],
            "energy_bookkeeping_dE": res["book"],
            "kernel_ms_per_step": {"build": kms[0] / K, "knn": kms[1] / K, "pairs": kms[2] / K, "resolve": kms[3] / K},
            "roofline": roofline(res, peaks, peak_src),
            "roofline_knn": roofline(res, peaks, peak_src, "knn"),
            "e2e": e2e,
            "clocks": res["clocks"],
            "gpu_launches": int(res["gpu_launches"]),
            "device_status": res["status"],
            "work_per_step": {"knn_tiles": float(res["diag"][0]) / K, "knn_candidates": float(res["diag"][1]) / K,
                              "knn_heap_inserts": float(res["diag"][2]) / K, "knn_max_tiles_one_leaf": int(res["diag"][3]),
                              "pair_tiles": float(res["diag"][4]) / K, "pair_max_tiles_one_leaf": int(res["diag"][5]),
                              "pair_tests": res["n_tested"] / K, "pair_evals": res["n_pairs"] / K,
                              "pair_lambda_lookups": float(res["diag"][6]) / K,
                              "knn_redone_cold": float(res["diag"][7]) / K},
            "local_diagnostics": res["local_diag"],
            "tuning_trials": len(res["tuning"]),
            "knn_warm_start": {"ms_per_call_warm": kms[1] / K, "ms_per_call_cold": res["knn_cold_ms"],
                               "note": "kernel sizes start from the previous step's h (bound knn_slack h_prev); "
                                       "particles with fewer than N_ngb candidates inside are redone cold; "
                                       "results bit-identical to the cold search"},
        }
        if fp64:
            line["fp64_form"] = fp64
            line["mixed_over_fp64"] = value / ws / fp64["value"]
        if not args.no_batched and ws == 1:
            line["batched"] = run_batched(res["local"])
            line["satellite"] = run_satellite(res["local"])
            line["streaming_kernels"] = run_streaming(res["local"], n=args.stream_n)
            line["config3"] = run_config3(res["local"], oracle_sample=not args.no_cpu_baseline)
            line["resolve_dense"] = run_resolve_dense(res)
            if fp64:
                line["batched_over_fp64_single_halo"] = line["batched"]["value"] / fp64["value"]
        if not args.no_cpu_baseline and ws == 1:
            line["cpu_baseline"] = cpu_baseline(res["dt"], res["vmax"], ns=max(1, res["halo"].n // 2))
        emit(line)
    res["ctx"].close()
    if ws > 1:
        torch.distributed.barrier()
        torch.distributed.destroy_process_group()


def main_reference(args):
    """The oracle (CPU, FP64, as it stands) timed on the host cores: each step
    is one full oracle step on a bounded sample of the workload."""
    ws, rank, _ = dist_env()
    if rank != 0:
        return
    from oracle import oracle as O
    from paper_2506_06269_gb300 import ics
    O.build()
    ns = 32768
    th = os.cpu_count() or 1
    O.set_num_threads(th)
    halo = ics.nfw(ns, SEED_IC)
    vmax = ics.nfw_vmax()
    # dt of the same rule, evaluated on the oracle's own sample
    h, _, _ = O.knn(halo.pos, halo.ids, N_NGB, O.MODE_MIXED)
    vel = halo.vel.astype(np.float32).astype(np.float64)
    _, _, sump = O.pairs(halo.pos, vel, halo.ids, h, O.MODE_MIXED, (1, S0, vmax), halo.mass, DT_PROBE, 0, 0, 0,
                         ev_cap=1 << 16)
    dt = TAU / float(np.quantile(sump / DT_PROBE, 0.999))
    pos = halo.pos.copy()

    def one(step_no):
        nonlocal pos, vel
        pos = pos + vel * dt
        r = O.step(pos, vel.astype(np.float32).astype(np.float64), halo.ids, [0, ns], [N_NGB], [halo.mass],
                   [(1, S0, vmax)], [dt], 7, step_no, O.MODE_MIXED)
        vel = r["vel_out"]
        O.energy_momentum(halo.mass, vel)

    for i in range(args.warmup):
        one(i)
    t0 = time.perf_counter()
    for i in range(args.steps):
        one(args.warmup + i)
    sec = time.perf_counter() - t0
    value = ns * args.steps / sec
    emit({"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws,
          "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * sec / max(args.steps, 1),
          "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
          "config": {"workload": WORKLOAD, "sample_particles": ns, "n_ngb": N_NGB, "dt": dt},
          "cpu_baseline": {"value": value, "unit": UNIT, "cores": int(O.num_threads()), "kind": "oracle",
                           "sample": f"each step: drift + full oracle step of a {ns}-particle NFW halo "
                                     f"(same profile, N_ngb, sigma(v), dt rule)"},
          "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}})


if __name__ == "__main__":
    a = parse()
    if a.impl == "reference":
        main_reference(a)
    elif a.only == "streaming":
        from paper_2506_06269_gb300 import build as _b
        _b.build()
        emit({"streaming_kernels": run_streaming(dist_env()[2], n=a.stream_n)})
    else:
        main_ours(a)

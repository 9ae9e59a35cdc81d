"""Autotuner of the launch knobs of the two hot kernels.

Every knob of sidm_config tuned here changes work, never a result (the tests
require identical kernel sizes, events and velocities for every setting; the
leaf size that defines the canonical FP32 distance is not a knob):

  kernel-size search (k_knn)     knn_warps (CTA size), knn_groups (lane groups of
                                 the candidate mask), knn_chains (independent
                                 distance chains), knn_batch (loop per staged leaf,
                                 over compacted batches, or those plus the
                                 fixed-bound warm-start kernel), knn_flush (merge
                                 threshold before node tests), knn_slack
                                 (warm-start bound)
  pair kernel (k_pairs)          pair_warps, pair_per_round (pairs a lane queues
                                 per round)
  candidate staging              use_tma (plain loads or bulk async copies)

The search is coordinate descent from the defaults: one knob at a time over
its values, keeping the fastest, two sweeps.  A trial builds a context with the
knobs (they are fixed at creation) on the caller's workload, runs a cell build,
a cold step and two warm-started steps (drift, build, kernel sizes, scatter),
then times `reps` more warm-started steps by the library's CUDA-event kernel
timers; the score of a knob is the time of the kernel it acts on.
"""
from __future__ import annotations

import numpy as np

KNN_KNOBS = {
    "knn_warps": (4, 8),
    "knn_batch": (1, 2, 3),
    "knn_groups": (2, 4, 8),
    "knn_chains": (4, 8),
    "knn_flush": (8, 16, 32),
    "knn_slack": (1.04, 1.05, 1.07, 1.08, 1.1),
}
PAIR_KNOBS = {
    "pair_warps": (4, 8),
    "pair_per_round": (3, 4),
}
DEFAULTS = {"knn_warps": 8, "knn_batch": 3, "knn_groups": 2, "knn_chains": 4, "knn_flush": 32, "knn_slack": 1.07,
            "pair_warps": 8, "pair_per_round": 4, "use_tma": 0}


def _trial(make_inputs, ks, xs_list, dts, masses, halo_off, precision, kw, reps, settle=2):
    import torch
    from paper_2506_06269_gb300 import sidm
    n = int(halo_off[-1])
    ctx = sidm.Context(n_max=n, halo_max=len(halo_off) - 1, ngb_max=int(max(ks)), precision=precision,
                       event_cap=max(1 << 16, n // 8), flags=sidm.SIDM_FLAG_TIMING, **kw)
    try:
        pos, vel, ids = make_inputs(ctx)
        h = torch.zeros(n, dtype=ctx.vdtype, device=ctx.device)
        xs, dt, mass = ctx.xs_tensor(xs_list), ctx.f64(dts), ctx.f64(masses)

        def step(i):
            ctx.drift(dt, pos, vel)
            ctx.build_cells(halo_off, pos, vel, ids)
            ctx.kernel_sizes(ks, h)
            ctx.scatter_step(12345, i, xs, dt, mass, vel)

        ctx.build_cells(halo_off, pos, vel, ids)
        for i in range(1 + settle):               # a cold search, then warm-started ones settle
            step(i)
        ctx.kernel_times(reset=True)
        for i in range(reps):
            step(1 + settle + i)
        ms, _ = ctx.kernel_times(reset=True)
        status = ctx.status()
    finally:
        ctx.close()
    if status:
        raise RuntimeError(f"device status {status} during tuning")
    return float(ms[1]) / reps, float(ms[2]) / reps


def autotune(make_inputs, ks, xs_list, dts, masses, halo_off, precision="mixed", reps=4, sweeps=2, tma=(0,)):
    """Return (knobs for sidm.Context, table of trials).

    make_inputs(ctx) -> (pos, vel, ids): fresh device copies of the workload.
    """
    best = dict(DEFAULTS)
    table = []
    cache = {}

    def score(kw):
        key = tuple(sorted(kw.items()))
        if key not in cache:
            try:
                cache[key] = _trial(make_inputs, ks, xs_list, dts, masses, halo_off, precision, kw, reps)
                table.append({**kw, "knn_ms": cache[key][0], "pairs_ms": cache[key][1]})
            except Exception as e:       # a shape that does not fit (shared memory, registers) is skipped
                cache[key] = None
                table.append({**kw, "error": str(e)})
        return cache[key]

    for _ in range(sweeps):
        for knobs, slot in ((KNN_KNOBS, 0), (PAIR_KNOBS, 1)):
            for name, values in knobs.items():
                timed = []
                for v in values:
                    kw = dict(best)
                    kw[name] = v
                    if kw["knn_chains"] == 8 and kw["knn_groups"] != 4:
                        continue                  # eight chains are built with four lane groups
                    r = score(kw)
                    if r is not None:
                        timed.append((r[slot], v))
                if timed:
                    best[name] = min(timed)[1]
    for t in tma:
        if t != best["use_tma"]:
            kw = dict(best)
            kw["use_tma"] = t
            kw["knn_batch"] = 1                   # bulk copies stage leaves for the per-leaf loop
            r, r0 = score(kw), score(best)
            if r is not None and r0 is not None and sum(r) < sum(r0):
                best = kw
    return best, table

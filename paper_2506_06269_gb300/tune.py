"""Autotuner for the launch shape of the two hot kernels.

Tunes, by measured CUDA-event kernel time on the caller's own workload:
  * warps per CTA of the kernel-size kernel (k_knn)   in {2, 4, 8}
  * warps per CTA of the pair kernel (k_pairs)        in {2, 4, 8}
  * candidate staging: plain 128-bit loads or bulk async copies (TMA)
Every choice gives bit-identical kernel sizes, events and velocities (the
leaf size that defines the canonical FP32 distance is not tuned), so tuning
never changes a result.  Each trial builds a fresh context (the launch shape
is fixed at creation), runs the cell build, kernel sizes and one scatter step
twice, and keeps the second timing.
"""
from __future__ import annotations

import itertools

import numpy as np


def _trial(make_inputs, ks, xs_list, dts, masses, halo_off, n, halo_max, ngb_max, precision, kw):
    import torch
    from paper_2506_06269_gb300 import sidm
    ctx = sidm.Context(n_max=n, halo_max=halo_max, ngb_max=ngb_max, precision=precision,
                       event_cap=max(1 << 16, n // 8), flags=sidm.SIDM_FLAG_TIMING, **kw)
    pos, vel, ids = make_inputs(ctx)
    h = torch.zeros(n, dtype=ctx.vdtype, device=ctx.device)
    xs = ctx.xs_tensor(xs_list)
    dt = ctx.f64(dts)
    mass = ctx.f64(masses)
    best = None
    for rep in range(2):
        ctx.build_cells(halo_off, pos, vel, ids)
        ctx.kernel_sizes(ks, h)
        ctx.scatter_step(12345, rep, xs, dt, mass, vel)
        ms, _ = ctx.kernel_times(reset=True)
        best = ms
    status = ctx.status()
    ctx.close()
    if status:
        raise RuntimeError(f"device status {status} during tuning")
    return best


def autotune(make_inputs, ks, xs_list, dts, masses, halo_off, precision="mixed",
             warps=(2, 4, 8), tma=(0, 1)):
    """Return ({knn_warps, pair_warps, use_tma}, table of trials).

    make_inputs(ctx) -> (pos, vel, ids) fresh device copies of the workload.
    """
    n = int(halo_off[-1])
    H = len(halo_off) - 1
    kmax = int(max(ks))
    table = []
    for w, t in itertools.product(warps, tma):
        try:
            ms = _trial(make_inputs, ks, xs_list, dts, masses, halo_off, n, H, kmax, precision,
                        dict(knn_warps=w, pair_warps=w, use_tma=t))
        except Exception as e:   # a shape that does not fit (shared memory, pair CTAs > 8 warps) is skipped
            table.append({"warps": w, "use_tma": t, "error": str(e)})
            continue
        table.append({"warps": w, "use_tma": t, "knn_ms": float(ms[1]), "pairs_ms": float(ms[2])})
    ok = [r for r in table if "error" not in r]
    if not ok:
        return {"knn_warps": 4, "pair_warps": 4, "use_tma": 0}, table
    best_t = min(tma, key=lambda t: min(r["knn_ms"] + r["pairs_ms"] for r in ok if r["use_tma"] == t)
                 if any(r["use_tma"] == t for r in ok) else np.inf)
    sub = [r for r in ok if r["use_tma"] == best_t]
    kw = min(sub, key=lambda r: r["knn_ms"])["warps"]
    pw = min(sub, key=lambda r: r["pairs_ms"])["warps"]
    return {"knn_warps": int(kw), "pair_warps": int(pw), "use_tma": int(best_t)}, table

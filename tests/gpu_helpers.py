"""Helpers for the GPU parity tests: run the CUDA pass through the C ABI and
compare with the oracle on the same seeded inputs.  Imports torch/CUDA lazily."""
from __future__ import annotations

import numpy as np

from oracle import oracle as O


def gpu_step(batch, ks, xs_list, dts, seed, step, precision="mixed", want_nbrs=False, ctx_kw=None,
             ctx=None, event_cap=None):
    """One build + kernel sizes + scatter step on cuda:0; results in input order."""
    import torch
    from paper_2506_06269_gb300 import sidm
    n, H = batch.n, batch.n_halos
    kw = dict(ctx_kw or {})
    own = ctx is None
    if own:
        ctx = sidm.Context(n_max=n, halo_max=H, ngb_max=max(ks), precision=precision,
                           event_cap=event_cap if event_cap is not None else max(4096, n), **kw)
    dev = ctx.device
    vdt = ctx.vdtype
    pos = torch.tensor(batch.pos, dtype=torch.float64, device=dev).contiguous()
    vel_in = batch.vel.astype(np.float32).astype(np.float64) if precision == "mixed" else batch.vel
    vel = torch.tensor(vel_in, dtype=vdt, device=dev).contiguous()
    ids = torch.tensor(batch.ids.astype(np.int64), dtype=torch.int64, device=dev).to(torch.int32).contiguous()
    h = torch.zeros(n, dtype=vdt, device=dev)
    ctx.build_cells(batch.offsets, pos, vel, ids)
    perm = ctx.perm(n).cpu().numpy().astype(np.int64)
    ctx.kernel_sizes(ks, h)
    nbr = ctx.neighbours(ks, n, max(ks)).cpu().numpy().view(np.uint32) if want_nbrs else None
    xs = ctx.xs_tensor(xs_list)
    dt = ctx.f64(dts)
    mass = ctx.f64(batch.mass)
    ctx.scatter_step(seed, step, xs, dt, mass, vel)
    status = ctx.status()
    stats = ctx.stats()
    n_ev, ev = ctx.events()
    out = {
        "perm": perm,
        "h": _unperm(h.cpu().numpy().astype(np.float64), perm),
        "vel": _unperm_v(vel.cpu().numpy().astype(np.float64), perm),
        "pos_sorted": pos.cpu().numpy(),
        "ids_sorted": ids.cpu().numpy().view(np.uint32),
        "events": ev.copy(),
        "n_events": n_ev,
        "stats": stats,
        "status": status,
        "nbr": None,
        "vel_in": vel_in,
    }
    if nbr is not None:
        nb = np.zeros_like(nbr)
        nb[perm] = nbr
        out["nbr"] = nb
    if len(ev):
        ev2 = ev.copy()
        ev2["i"] = perm[ev["i"]]
        ev2["j"] = perm[ev["j"]]
        out["events"] = np.sort(ev2, order="key")
    if own:
        ctx.close()
    return out


def _unperm(a_sorted, perm):
    out = np.empty_like(a_sorted)
    out[perm] = a_sorted
    return out


def _unperm_v(v_sorted, perm):
    out = np.empty_like(v_sorted)
    out[:, perm] = v_sorted
    return out


def oracle_step(batch, ks, xs_list, dts, seed, step, precision="mixed"):
    vel_in = batch.vel.astype(np.float32).astype(np.float64) if precision == "mixed" else batch.vel
    mode = O.MODE_MIXED if precision == "mixed" else O.MODE_FP64
    return O.step(batch.pos, vel_in, batch.ids, batch.offsets, ks, batch.mass, xs_list, dts, seed, step, mode)


def compare_events(g_ev, o_ev, tol=1e-6):
    """Event key sets must agree except for pairs with |P - u| < tol (oracle P)."""
    gk = set(int(k) for k in g_ev["key"])
    ok = {int(e["key"]): e for e in o_ev}
    only_o = [k for k in ok if k not in gk]
    only_g = [k for k in gk if k not in ok]
    for k in only_o:
        e = ok[k]
        assert abs(e["P"] - e["u"]) < tol, f"oracle-only event with |P-u|={abs(e['P'] - e['u'])}"
    gmap = {int(e["key"]): e for e in g_ev}
    for k in only_g:
        e = gmap[k]
        u = float(e["x0"]) * 2.0 ** -32
        assert abs(float(e["P"]) - u) < tol, f"GPU-only event with |P-u|={abs(float(e['P']) - u)}"
    return only_o, only_g


def tainted_particles(o_ev, g_ev, only_keys, n):
    """Particles event-connected to a differing event (union-find over all events)."""
    parent = np.arange(n)

    def find(x):
        while parent[x] != x:
            parent[x] = parent[parent[x]]
            x = parent[x]
        return x

    for ev in (o_ev, g_ev):
        for e in ev:
            a, b = find(int(e["i"])), find(int(e["j"]))
            if a != b:
                parent[a] = b
    bad_roots = set()
    allev = {int(e["key"]): e for e in list(o_ev) + list(g_ev)}
    for k in only_keys:
        e = allev[k]
        bad_roots.add(find(int(e["i"])))
    mask = np.zeros(n, bool)
    if bad_roots:
        roots = np.array([find(i) for i in range(n)])
        mask = np.isin(roots, list(bad_roots))
    return mask


def velocity_scale(o_ev, vel_in, masses):
    """Per-particle speed scale of the scatter arithmetic: for a particle in one
    event, its own speed plus its partner's at the step start; for a particle in
    several, the largest such pair speed, each taken from the velocities the
    oracle's sequential application (ascending key order) has just before that
    event.  A particle without events keeps its own speed.

    o_ev: the oracle's events (key order, global indices); vel_in [3, n] the
    step-start velocities; masses [n] per-particle masses."""
    cur = np.array(vel_in, dtype=np.float64, copy=True)
    scale = np.linalg.norm(cur, axis=0)
    for e in np.sort(np.asarray(o_ev), order="key") if len(o_ev) else []:
        i, j = int(e["i"]), int(e["j"])
        s = np.linalg.norm(cur[:, i]) + np.linalg.norm(cur[:, j])
        scale[i] = max(scale[i], s)
        scale[j] = max(scale[j], s)
        loc = np.array([e]).copy()
        loc["i"], loc["j"] = 0, 1
        v2, _ = O.apply_events(loc, np.array([masses[i], masses[j]]), cur[:, [i, j]])
        cur[:, [i, j]] = v2
    return scale

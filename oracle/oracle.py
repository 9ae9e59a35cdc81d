"""Python face of the FP64 CPU oracle (``sidm_oracle.c``).

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` are the only
callers.  It shares nothing with the CUDA path; its inputs come from the seeded
generators in ``paper_2506_06269_gb300.ics`` or from literal test values.

Functions follow the paper (Fischer, Yu & Dolag 2025): Sect. 2 (spline kernel,
N_ngb-adaptive size, energy/momentum conserving scatter), Sect. 3.5 (geometric
factor Lambda of the interaction probability, Eq. hDl), Sect. 3.8 (Eq. vel_dep),
Sect. 5 (conservation independent of the kernel); local diagnostics: Eq. hDl
(Sect. 3.5), Eq. knudsen_number (Sect. 3.6), Eq. effective_cross_section
(App. C).  The readings where the paper
is silent are documented in the C source header.

Parity status: every function here is pinned by a ``-m "not gpu"`` test
(``tests/test_oracle_*.py``) against something other than itself.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "sidm_oracle.c")
_LIB = os.path.join(_HERE, "_build", "liboracle.so")
_lock = threading.Lock()
_lib = None

MODE_MIXED = 0
MODE_FP64 = 1

EVENT_DTYPE = np.dtype([("key", "<u8"), ("i", "<u4"), ("j", "<u4"), ("x1", "<u4"),
                        ("x2", "<u4"), ("P", "<f8"), ("u", "<f8")])
assert EVENT_DTYPE.itemsize == 40


class _PairStats(C.Structure):
    _fields_ = [("n_pairs", C.c_int64), ("n_events", C.c_int64), ("n_p_gt1", C.c_int64),
                ("n_near", C.c_int64), ("max_sum_p", C.c_double)]


def build(force: bool = False) -> str:
    """Compile the oracle (gcc, -O2, no fast-math, no FP contraction, OpenMP)."""
    os.makedirs(os.path.dirname(_LIB), exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-fPIC", "-shared", "-ffp-contract=off", "-fno-fast-math",
               "-fopenmp", _SRC, "-o", tmp, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB)
    return _LIB


def lib():
    global _lib
    with _lock:
        if _lib is None:
            build()
            L = C.CDLL(_LIB)
            P = C.POINTER
            d, i32, i64, u32, u64 = C.c_double, C.c_int, C.c_int64, C.c_uint32, C.c_uint64
            vp = C.c_void_p
            L.orc_philox4x32_10.argtypes = [vp, vp, vp]
            L.orc_kernel_w.argtypes = [d, d]; L.orc_kernel_w.restype = d
            L.orc_lambda.argtypes = [d, d, d]; L.orc_lambda.restype = d
            L.orc_sigma.argtypes = [i32, d, d, d]; L.orc_sigma.restype = d
            L.orc_knn_halo.argtypes = [i32, vp, vp, vp, vp, i32, i32, i32, vp, vp, vp, vp]
            L.orc_knn_halo.restype = i32
            L.orc_knn_sample.argtypes = [i32, vp, vp, vp, vp, i32, i32, i64, vp, vp]
            L.orc_knn_sample.restype = i32
            L.orc_sigma_eff.argtypes = [i32, d, d, d]; L.orc_sigma_eff.restype = d
            L.orc_local_diag.argtypes = [i32, vp, vp, vp, vp, vp, vp, vp, d, i32, i32, d, d, d, vp]
            L.orc_local_diag.restype = i32
            L.orc_timestep.argtypes = [i32, vp, d, d, d, d, i32, vp, vp]
            L.orc_pairs_halo.argtypes = [i32, vp, vp, vp, vp, vp, vp, vp, vp, i32, i32, d, d, d, d,
                                         u64, u64, u32, vp, i64, P(_PairStats), vp, vp, vp, i32, i32, d, i32]
            L.orc_apply_drag.argtypes = [vp, i64, vp, i32, d, d, vp, vp, vp, vp, vp]
            L.orc_host_mass.argtypes = [d, d, d]; L.orc_host_mass.restype = d
            L.orc_host_phi.argtypes = [vp, d, d, d]; L.orc_host_phi.restype = d
            L.orc_host_accel.argtypes = [vp, d, d, d, vp]
            L.orc_host_kick.argtypes = [i32, vp, vp, vp, vp, vp, vp, vp, i32, i32, i32, d, vp]
            L.orc_reflect.argtypes = [i32, vp, vp, vp, vp, vp, vp, d, d, d, d]
            L.orc_pairs_halo.restype = i32
            L.orc_sort_events.argtypes = [vp, i64]
            L.orc_apply_events.argtypes = [vp, i64, vp, vp, vp, vp, vp]
            L.orc_energy_momentum.argtypes = [i32, d, vp, vp, vp, vp]
            L.orc_exact_sum.argtypes = [vp, i64]; L.orc_exact_sum.restype = d
            L.orc_geometry.argtypes = [i32, vp, vp, vp, vp, vp, vp, vp, vp]
            L.orc_d2_mixed_pairs.argtypes = [i32, vp, vp, vp, i64, vp, vp, vp]
            L.orc_num_threads.restype = i32
            L.orc_set_num_threads.argtypes = [i32]
            _lib = L
    return _lib


def _p(a: np.ndarray):
    return a.ctypes.data_as(C.c_void_p) if a is not None else None


def _c(a, dtype):
    return np.ascontiguousarray(a, dtype=dtype)


def num_threads() -> int:
    return int(lib().orc_num_threads())


def set_num_threads(t: int) -> None:
    lib().orc_set_num_threads(int(t))


# --------------------------------------------------------------------------
# elementary functions
# --------------------------------------------------------------------------
def philox4x32_10(ctr, key) -> np.ndarray:
    """Philox4x32-10 block (Salmon et al. 2011) of a 4-word counter, 2-word key."""
    c = _c(ctr, np.uint32); k = _c(key, np.uint32); o = np.zeros(4, np.uint32)
    lib().orc_philox4x32_10(_p(c), _p(k), _p(o))
    return o


def kernel_w(r: float, h: float) -> float:
    """Cubic spline kernel W(r, h), support h, unit integral (Sect. 2)."""
    return float(lib().orc_kernel_w(float(r), float(h)))


def lam(d: float, hi: float, hj: float) -> float:
    """Geometric factor Lambda(d; h_i, h_j): overlap integral of two kernels."""
    return float(lib().orc_lambda(float(d), float(hi), float(hj)))


def sigma(kind: int, s0: float, w: float, v: float) -> float:
    """sigma/m of Eq. vel_dep (kind 1) or a constant (kind 0)."""
    return float(lib().orc_sigma(int(kind), float(s0), float(w), float(v)))


def exact_sum(x) -> float:
    a = _c(x, np.float64)
    return float(lib().orc_exact_sum(_p(a), a.size))


def energy_momentum(m: float, vel: np.ndarray) -> np.ndarray:
    """Exact (expansion) sums of 1/2 m |v|^2 and m v; vel is [3, n]."""
    v = _c(vel, np.float64); out = np.zeros(4)
    n = v.shape[1]
    lib().orc_energy_momentum(n, float(m), _p(v[0]), _p(v[1]), _p(v[2]), _p(out))
    return out


# --------------------------------------------------------------------------
# canonical FP32 geometry (mixed form)
# --------------------------------------------------------------------------
def geometry(pos: np.ndarray):
    """Sorted order, FP32 offsets [3][n] (input order), leaf cells [nleaf][3], E, O."""
    p = _c(pos, np.float64); n = p.shape[1]
    order = np.zeros(n, np.uint32); off = np.zeros((n, 3), np.float32)
    nleaf = (n + 31) // 32
    cell = np.zeros((max(nleaf, 1), 3), np.float32)
    E = C.c_int(0); O = np.zeros(3)
    lib().orc_geometry(n, _p(p[0]), _p(p[1]), _p(p[2]), _p(order), _p(off), _p(cell), C.byref(E), _p(O))
    return order, off.T.copy(), cell[:nleaf], int(E.value), O


def d2_mixed(pos: np.ndarray, qi, qj) -> np.ndarray:
    """Canonical FP32 d^2 from i (its leaf frame) to j, for local index pairs."""
    p = _c(pos, np.float64); n = p.shape[1]
    a = _c(qi, np.uint32); b = _c(qj, np.uint32); out = np.zeros(a.size, np.float32)
    lib().orc_d2_mixed_pairs(n, _p(p[0]), _p(p[1]), _p(p[2]), a.size, _p(a), _p(b), _p(out))
    return out


# --------------------------------------------------------------------------
# the pass, halo by halo
# --------------------------------------------------------------------------
def knn(pos: np.ndarray, ids: np.ndarray, k: int, mode: int = MODE_MIXED, brute: bool = False,
        query_mask=None, want_nbrs: bool = False):
    """Kernel sizes h of one halo: distance to the k-th nearest other particle.

    Returns (h float64[n], d2k_bits uint64[n], nbr_ids uint32[n,k] or None).
    For the mixed form h holds FP32 values.
    """
    p = _c(pos, np.float64); n = p.shape[1]
    idv = _c(ids, np.uint32)
    h = np.full(n, np.nan); d2k = np.zeros(n, np.uint64)
    nb = np.zeros((n, k), np.uint32) if want_nbrs else None
    qm = _c(query_mask, np.uint8) if query_mask is not None else None
    rc = lib().orc_knn_halo(n, _p(p[0]), _p(p[1]), _p(p[2]), _p(idv), int(k), int(mode),
                            1 if brute else 0, _p(qm), _p(h), _p(d2k), _p(nb))
    if rc != 0:
        raise ValueError(f"oracle kNN failed ({rc}): need 1 <= k <= n-1 (k={k}, n={n})")
    return h, d2k, nb


def knn_sample(pos: np.ndarray, ids: np.ndarray, k: int, qidx, mode: int = MODE_MIXED):
    """Kernel sizes of the listed particles for every N_ngb = 1..k: returns
    h[len(qidx), k] with h[t, r] the distance to the (r+1)-th nearest other
    particle of particle qidx[t] (the same definition as knn)."""
    p = _c(pos, np.float64); n = p.shape[1]
    idv = _c(ids, np.uint32)
    q = _c(qidx, np.int64)
    h = np.full((q.size, k), np.nan)
    rc = lib().orc_knn_sample(n, _p(p[0]), _p(p[1]), _p(p[2]), _p(idv), int(k), int(mode), q.size, _p(q), _p(h))
    if rc != 0:
        raise ValueError(f"oracle kNN failed ({rc}): need 1 <= k <= n-1 (k={k}, n={n})")
    return h


def sigma_eff(kind: int, s0: float, w: float, nu: float) -> float:
    """Effective cross-section per mass at 1-D velocity dispersion nu."""
    return float(lib().orc_sigma_eff(int(kind), float(s0), float(w), float(nu)))


def local_diag(pos, vel, h, mass: float, nngb: int, xs, G: float = 1.0) -> dict:
    """Per-particle rho, nu, sigma_eff/m, h/l (Eq. hDl) and Kn of one halo (FP64)."""
    p = _c(pos, np.float64); v = _c(vel, np.float64); hh = _c(h, np.float64); n = p.shape[1]
    out = np.zeros((5, n))
    kind, s0, w = xs
    lib().orc_local_diag(n, _p(p[0]), _p(p[1]), _p(p[2]), _p(v[0]), _p(v[1]), _p(v[2]), _p(hh), float(mass),
                         int(nngb), int(kind), float(s0), float(w), float(G), _p(out))
    return {"rho": out[0], "nu": out[1], "sigma_eff": out[2], "h_over_l": out[3], "kn": out[4]}


def timestep(sum_p, tau: float, dt: float, dt_min: float, dt_max: float, n_bins: int):
    """SIDM time step per particle from its summed pair probabilities, and its
    power-of-two bin (see orc_timestep)."""
    sp = _c(sum_p, np.float64); n = sp.size
    dto = np.zeros(n); bo = np.zeros(n, np.int32)
    lib().orc_timestep(n, _p(sp), float(tau), float(dt), float(dt_min), float(dt_max), int(n_bins), _p(dto), _p(bo))
    return dto, bo


def host_params(host) -> np.ndarray:
    """Flat FP64 parameter array of an analytic host (the layout orc_host_phi reads).

    host: dict with G, center (3), and any of nfw = (rho_s, r_s),
    bulge = (M_H, a_H), disks = [(M_d, a_d, b_d), ...] (at most 4)."""
    disks = list(host.get("disks", ()))
    if len(disks) > 4:
        raise ValueError("at most 4 disks")
    rho_s, r_s = host.get("nfw") or (0.0, 1.0)
    m_h, a_h = host.get("bulge") or (0.0, 1.0)
    out = [float(host["G"]), *[float(c) for c in host.get("center", (0.0, 0.0, 0.0))],
           float(rho_s), float(r_s), float(m_h), float(a_h), float(len(disks))]
    for m, a, b in disks:
        out += [float(m), float(a), float(b)]
    return np.array(out, dtype=np.float64)


def host_mass(r, rho_s, r_s):
    """NFW mass inside r (see orc_host_mass)."""
    return float(lib().orc_host_mass(float(r), float(rho_s), float(r_s)))


def host_phi(host, x):
    """Host potential at the points x [3] or [3][n] (see orc_host_phi)."""
    hp = host_params(host)
    pts = np.asarray(x, dtype=np.float64).reshape(3, -1)
    out = np.array([lib().orc_host_phi(_p(hp), float(p[0]), float(p[1]), float(p[2])) for p in pts.T])
    return out if np.ndim(x) > 1 else float(out[0])


def host_accel(host, x):
    """Host acceleration at the points x [3] or [3][n] (see orc_host_accel)."""
    hp = host_params(host)
    pts = np.asarray(x, dtype=np.float64).reshape(3, -1)
    out = np.zeros((3, pts.shape[1]))
    a = np.zeros(3)
    for k in range(pts.shape[1]):
        lib().orc_host_accel(_p(hp), float(pts[0, k]), float(pts[1, k]), float(pts[2, k]), _p(a))
        out[:, k] = a
    return out if np.ndim(x) > 1 else out[:, 0]


def host_kick(pos, vel, host, dt_max, bins=None, n_bins=1, substep=0, phase=0):
    """Half kick of the particles due at this sub-step (see orc_host_kick); returns new vel."""
    p = _c(pos, np.float64); v = np.array(vel, dtype=np.float64, copy=True, order="C"); n = p.shape[1]
    bn = None if bins is None else _c(bins, np.int32)
    hp = host_params(host)
    lib().orc_host_kick(n, _p(p[0]), _p(p[1]), _p(p[2]), _p(v[0]), _p(v[1]), _p(v[2]), _p(bn), int(n_bins),
                        int(substep), int(phase), float(dt_max), _p(hp))
    return v


def reflect(pos, vel, center, r_b):
    """Reflecting sphere of radius r_b about center (see orc_reflect); returns new vel."""
    p = _c(pos, np.float64); v = np.array(vel, dtype=np.float64, copy=True, order="C"); n = p.shape[1]
    lib().orc_reflect(n, _p(p[0]), _p(p[1]), _p(p[2]), _p(v[0]), _p(v[1]), _p(v[2]),
                      float(center[0]), float(center[1]), float(center[2]), float(r_b))
    return v


def pairs(pos, vel, ids, h, mode, xs, mass, dt, seed, step, halo, ev_cap=None, mask=None, bins=None,
          n_bins=1, substep=0, dt_max=0.0):
    """Pair probabilities and draws of one halo.

    xs = (kind, s0, w) or (kind, s0, w, angular): angular 1 is the
    forward-dominated (frictional) limit (Sect. 3.8), where every in-range
    pair is returned as a record whose "P" field holds G = m_j Lambda_ij dt
    (u = -1, no draw), to be applied by apply_drag; n_p_gt1 then counts pairs
    whose step-start D = P/3 exceeds 1, and n_near is 0.

    bins (int [n], optional): individual power-of-two steps; only pairs whose
    particles both open a step at `substep` are evaluated, on the longer step
    dt_max / 2^min(b_i, b_j) (dt is then unused); sum_p then holds the sums of
    P scaled to dt_max.

    xs = (kind, s0, w).  Returns (events [EVENT_DTYPE], stats dict, sum_p[n]).
    Event indices are local (halo) input indices; i has the smaller id.
    mask (bool [n], optional): only pairs with a masked endpoint are evaluated
    (stats and sum_p then cover those pairs only).
    """
    p = _c(pos, np.float64); v = _c(vel, np.float64); n = p.shape[1]
    idv = _c(ids, np.uint32); hh = _c(h, np.float64)
    cap = int(ev_cap if ev_cap is not None else max(1024, n))
    ev = np.zeros(cap, EVENT_DTYPE)
    st = _PairStats(); sump = np.zeros(n)
    pm = None if mask is None else _c(mask, np.uint8)
    bn = None if bins is None else _c(bins, np.int32)
    kind, s0, w = xs[:3]
    angular = int(xs[3]) if len(xs) > 3 else 0
    rc = lib().orc_pairs_halo(n, _p(p[0]), _p(p[1]), _p(p[2]), _p(v[0]), _p(v[1]), _p(v[2]),
                              _p(idv), _p(hh), int(mode), int(kind), float(s0), float(w),
                              float(mass), float(dt), C.c_uint64(int(seed)), C.c_uint64(int(step)),
                              C.c_uint32(int(halo)), _p(ev), cap, C.byref(st), _p(sump),
                              _p(pm), _p(bn), int(n_bins), int(substep), float(dt_max), angular)
    if rc != 0:
        raise RuntimeError(f"oracle pair pass failed ({rc}): event buffer too small")
    ne = int(st.n_events)
    ev = ev[:ne].copy()
    lib().orc_sort_events(_p(ev), ne)
    stats = {"n_pairs": int(st.n_pairs), "n_events": ne, "n_p_gt1": int(st.n_p_gt1),
             "n_near": int(st.n_near), "max_sum_p": float(st.max_sum_p)}
    return ev, stats, sump


def apply_events(events: np.ndarray, masses: np.ndarray, vel: np.ndarray):
    """Apply key-sorted events one after another (current velocities), FP64.

    Returns (new vel [3,n] float64, per-event pair kinetic-energy change).
    """
    ev = np.ascontiguousarray(events, dtype=EVENT_DTYPE)
    v = np.array(vel, dtype=np.float64, copy=True, order="C")
    m = _c(masses, np.float64)
    dE = np.zeros(max(ev.size, 1))
    lib().orc_apply_events(_p(ev), ev.size, _p(m), _p(v[0]), _p(v[1]), _p(v[2]), _p(dE))
    return v, dE[:ev.size]


def apply_drag(records: np.ndarray, masses: np.ndarray, xs, vel: np.ndarray):
    """Forward-dominated (frictional) scattering of key-sorted pair records,
    one after another from the current FP64 velocities (Sect. 3.8, App. A).

    records: pairs(..., xs with angular 1) output ("P" = G = m_j Lambda dt);
    xs = (kind, s0, w[, angular]) gives sigma_V / m.  Returns (new vel [3,n],
    per-record pair kinetic-energy change, per-record D).
    """
    ev = np.ascontiguousarray(records, dtype=EVENT_DTYPE)
    v = np.array(vel, dtype=np.float64, copy=True, order="C")
    m = _c(masses, np.float64)
    dE = np.zeros(max(ev.size, 1)); D = np.zeros(max(ev.size, 1))
    lib().orc_apply_drag(_p(ev), ev.size, _p(m), int(xs[0]), float(xs[1]), float(xs[2]),
                         _p(v[0]), _p(v[1]), _p(v[2]), _p(dE), _p(D))
    return v, dE[:ev.size], D[:ev.size]


def step(pos, vel, ids, offsets, k_per_halo, masses, xs_per_halo, dt_per_halo, seed, step_no,
         mode: int = MODE_MIXED):
    """One full SIDM scattering pass of a batch of halos (oracle form).

    pos float64 [3,N]; vel [3,N] (FP32 values in the mixed form); ids uint32;
    offsets int64 [H+1].  Returns dict with h, events (global indices, key
    order), vel_out (FP64), per-halo stats.
    """
    offsets = np.asarray(offsets, np.int64)
    H = len(offsets) - 1
    N = int(offsets[-1])
    h_all = np.zeros(N)
    evs, stats = [], []
    for hidx in range(H):
        a, b = int(offsets[hidx]), int(offsets[hidx + 1])
        if b - a == 0:
            stats.append({"n_pairs": 0, "n_events": 0, "n_p_gt1": 0, "n_near": 0, "max_sum_p": 0.0})
            continue
        hh, _, _ = knn(pos[:, a:b], ids[a:b], int(k_per_halo[hidx]), mode)
        h_all[a:b] = hh
        xs = xs_per_halo[hidx]
        # forward-dominated halos return every in-range pair (about 2 N_ngb per particle)
        cap = (b - a) * 8 * int(k_per_halo[hidx]) if len(xs) > 3 and int(xs[3]) == 1 else None
        ev, st, _ = pairs(pos[:, a:b], vel[:, a:b], ids[a:b], hh, mode, xs,
                          float(masses[hidx]), float(dt_per_halo[hidx]), seed, step_no, hidx, ev_cap=cap)
        ev["i"] += a; ev["j"] += a
        evs.append(ev); stats.append(st)
    events = np.concatenate(evs) if evs else np.zeros(0, EVENT_DTYPE)
    events = np.sort(events, order="key")
    pm = np.repeat(np.asarray(masses, np.float64), np.diff(offsets))
    # halos hold disjoint particles: isotropic events and forward-dominated pair
    # records are applied halo by halo, each in key order
    vout = np.array(vel, dtype=np.float64, copy=True)
    dE = np.zeros(events.size)
    hof = (events["key"] >> np.uint64(54)).astype(np.int64)
    for hidx in range(H):
        sel = np.flatnonzero(hof == hidx)
        if sel.size == 0:
            continue
        xs = xs_per_halo[hidx]
        if len(xs) > 3 and int(xs[3]) == 1:
            vout, dE[sel], _ = apply_drag(events[sel], pm, xs, vout)
        else:
            vout, dE[sel] = apply_events(events[sel], pm, vout)
    return {"h": h_all, "events": events, "vel_out": vout, "dE": dE, "stats": stats}

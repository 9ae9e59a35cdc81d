"""Thin Python binding of libsidm (the C ABI declared in include/sidm.h).

Argument marshalling only: every step of the scattering pass runs in the CUDA
kernels of ``libsidm.so``.  PyTorch provides device memory and streams.  There
is no CPU fallback: if the library is missing, cannot be loaded, or no CUDA
device is present, these functions raise.

Functions carry the C names (``sidm_create``, ``sidm_build_cells``, ...);
``Context`` bundles them for convenience.
"""
from __future__ import annotations

import ctypes as C
import os
from dataclasses import dataclass

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_build", "libsidm.so")

SIDM_OK, SIDM_EINVAL, SIDM_ECAPACITY, SIDM_ECUDA, SIDM_EROUNDS, SIDM_EDEVICE = 0, -1, -2, -3, -4, -5
SIDM_DEV_EVENT_OVERFLOW, SIDM_DEV_ROUNDS, SIDM_DEV_STACK, SIDM_DEV_BAD_INPUT, SIDM_DEV_WAIT_TIMEOUT = 1, 2, 4, 8, 16
SIDM_MIXED, SIDM_FP64 = 0, 1
SIDM_FLAG_SUM_P = 1
SIDM_FLAG_LOCAL_DIAG = 4
SIDM_FLAG_DRAG = 8
SIDM_FLAG_TIMING = 2
SIDM_STATIC_MAX_HALOS, SIDM_STATIC_MAX_CHUNKS = 64, 4096

XS_DTYPE = np.dtype([("kind", "<i4"), ("angular", "<i4"), ("s0", "<f8"), ("w", "<f8")])
STATS_DTYPE = np.dtype([("n_pairs", "<u8"), ("n_events", "<u8"), ("n_p_gt1", "<u8"), ("n_near", "<u8"),
                        ("n_multi", "<u8"), ("rounds", "<u4"), ("status", "<u4"), ("d_energy", "<f8"),
                        ("max_sum_p", "<f4"), ("pad", "<f4"), ("n_tested", "<u8")])
EVENT_DTYPE = np.dtype([("key", "<u8"), ("i", "<u4"), ("j", "<u4"), ("x1", "<u4"), ("x2", "<u4"),
                        ("P", "<f4"), ("x0", "<u4")])
assert XS_DTYPE.itemsize == 24 and STATS_DTYPE.itemsize == 72 and EVENT_DTYPE.itemsize == 32


class SidmConfig(C.Structure):
    _fields_ = [("n_max", C.c_int64), ("halo_max", C.c_int32), ("ngb_max", C.c_int32),
                ("event_cap", C.c_int64), ("precision", C.c_int32), ("device", C.c_int32),
                ("knn_warps", C.c_int32), ("pair_warps", C.c_int32), ("max_rounds", C.c_int32),
                ("flags", C.c_int32), ("grid_ctas", C.c_int32), ("use_tma", C.c_int32),
                ("knn_groups", C.c_int32), ("knn_chains", C.c_int32), ("knn_flush", C.c_int32),
                ("knn_slack", C.c_float), ("pair_per_round", C.c_int32), ("knn_batch", C.c_int32)]


class SidmHost(C.Structure):
    _fields_ = [("G", C.c_double), ("center", C.c_double * 3), ("rho_s", C.c_double), ("r_s", C.c_double),
                ("M_H", C.c_double), ("a_H", C.c_double), ("n_disks", C.c_int32), ("pad_", C.c_int32),
                ("M_d", C.c_double * 4), ("a_d", C.c_double * 4), ("b_d", C.c_double * 4)]


def host_struct(host) -> SidmHost:
    """sidm_host from a dict: G, center, and any of nfw = (rho_s, r_s),
    bulge = (M_H, a_H), disks = [(M_d, a_d, b_d), ...] (at most 4)."""
    disks = list(host.get("disks", ()))
    if len(disks) > 4:
        raise ValueError("at most 4 disks")
    rho_s, r_s = host.get("nfw") or (0.0, 1.0)
    m_h, a_h = host.get("bulge") or (0.0, 1.0)
    pad = disks + [(0.0, 0.0, 1.0)] * (4 - len(disks))
    return SidmHost(float(host["G"]), (C.c_double * 3)(*[float(x) for x in host.get("center", (0.0, 0.0, 0.0))]),
                    float(rho_s), float(r_s), float(m_h), float(a_h), len(disks), 0,
                    (C.c_double * 4)(*[float(d[0]) for d in pad]), (C.c_double * 4)(*[float(d[1]) for d in pad]),
                    (C.c_double * 4)(*[float(d[2]) for d in pad]))


class SidmError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"libsidm error {code}: {msg}")
        self.code = code


_lib = None


def load_library():
    """Load libsidm.so (built by paper_2506_06269_gb300.build).  Raises if absent."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"libsidm.so not built ({LIB_PATH}); run __graft_entry__.build()")
    L = C.CDLL(LIB_PATH)
    vp, i32, i64, u64 = C.c_void_p, C.c_int32, C.c_int64, C.c_uint64
    L.sidm_create.argtypes = [C.POINTER(vp), C.POINTER(SidmConfig)]
    L.sidm_destroy.argtypes = [vp]
    L.sidm_last_error.argtypes = [vp]; L.sidm_last_error.restype = C.c_char_p
    L.sidm_create_error.restype = C.c_char_p
    L.sidm_build_cells.argtypes = [vp, i32, vp, vp, vp, vp, vp]
    L.sidm_kernel_sizes.argtypes = [vp, vp, vp, vp]
    L.sidm_scatter_step.argtypes = [vp, u64, u64, vp, vp, vp, vp, vp, vp]
    L.sidm_energy_momentum.argtypes = [vp, vp, vp, vp, vp, vp]
    L.sidm_status.argtypes = [vp, vp, C.POINTER(C.c_uint32)]
    L.sidm_get_perm.argtypes = [vp, vp, vp]
    L.sidm_neighbours.argtypes = [vp, vp, i32, vp, vp]
    L.sidm_get_events.argtypes = [vp, i64, vp, C.POINTER(C.c_int64), vp]
    L.sidm_lambda_eval.argtypes = [vp, i64, vp, vp, vp, vp, vp]
    L.sidm_drift.argtypes = [vp, vp, vp, vp, vp]
    L.sidm_get_sum_p.argtypes = [vp, vp, vp]
    L.sidm_launch_count.argtypes = [vp]; L.sidm_launch_count.restype = i64
    L.sidm_kernel_times.argtypes = [vp, vp, vp, i32]
    L.sidm_diagnostics.argtypes = [vp, vp, i32]
    L.sidm_warm_start.argtypes = [vp, i32]
    L.sidm_local_diagnostics.argtypes = [vp, vp, vp, vp, C.c_double, vp, vp]
    L.sidm_timestep_criterion.argtypes = [vp, C.c_double, C.c_double, C.c_double, i32, vp, vp, vp, vp, vp]
    L.sidm_scatter_step_binned.argtypes = [vp, u64, u64, vp, C.c_double, i32, i32, vp, vp, vp, vp, vp]
    L.sidm_host_kick.argtypes = [vp, C.POINTER(SidmHost), C.c_double, i32, i32, i32, vp, vp, vp, vp]
    L.sidm_host_potential.argtypes = [vp, C.POINTER(SidmHost), vp, vp, vp]
    L.sidm_reflect_boundary.argtypes = [vp, vp, vp, vp, vp]
    L.sidm_energy_momentum_static.argtypes = [i32, vp, i32, vp, vp, vp, vp, vp]
    L.sidm_static_last_error.restype = C.c_char_p
    for f in ("sidm_create", "sidm_destroy", "sidm_build_cells", "sidm_kernel_sizes", "sidm_scatter_step",
              "sidm_energy_momentum", "sidm_status", "sidm_get_perm", "sidm_neighbours", "sidm_get_events",
              "sidm_lambda_eval", "sidm_drift", "sidm_get_sum_p", "sidm_kernel_times", "sidm_diagnostics",
              "sidm_energy_momentum_static", "sidm_warm_start", "sidm_local_diagnostics", "sidm_timestep_criterion",
              "sidm_scatter_step_binned", "sidm_host_kick", "sidm_host_potential", "sidm_reflect_boundary"):
        getattr(L, f).restype = C.c_int
    _lib = L
    return L


EXPORTED = ["sidm_create", "sidm_destroy", "sidm_last_error", "sidm_create_error", "sidm_build_cells",
            "sidm_kernel_sizes", "sidm_scatter_step", "sidm_energy_momentum", "sidm_status", "sidm_get_perm",
            "sidm_neighbours", "sidm_get_events", "sidm_lambda_eval", "sidm_drift", "sidm_get_sum_p",
            "sidm_launch_count", "sidm_kernel_times", "sidm_diagnostics", "sidm_energy_momentum_static",
            "sidm_warm_start", "sidm_local_diagnostics", "sidm_timestep_criterion", "sidm_scatter_step_binned",
            "sidm_host_kick", "sidm_host_potential", "sidm_reflect_boundary", "sidm_static_last_error"]


def _torch():
    import torch
    if not torch.cuda.is_available():
        raise RuntimeError("libsidm needs a CUDA device; there is no CPU fallback")
    return torch


def _ptr(t):
    return None if t is None else C.c_void_p(t.data_ptr())


def _stream(stream):
    torch = _torch()
    s = stream if stream is not None else torch.cuda.current_stream()
    return C.c_void_p(s.cuda_stream)


def _check(ctx, rc):
    if rc != SIDM_OK:
        raise SidmError(rc, load_library().sidm_last_error(ctx).decode())


# ------------------------------------------------------------------ C names
def sidm_create(cfg: SidmConfig):
    L = load_library()
    h = C.c_void_p()
    rc = L.sidm_create(C.byref(h), C.byref(cfg))
    if rc != SIDM_OK:
        raise SidmError(rc, L.sidm_create_error().decode())
    return h


def sidm_destroy(ctx):
    load_library().sidm_destroy(ctx)


def sidm_build_cells(ctx, halo_off, pos, vel, ids, stream=None):
    off = np.ascontiguousarray(halo_off, dtype=np.int64)
    _check(ctx, load_library().sidm_build_cells(ctx, len(off) - 1, off.ctypes.data_as(C.c_void_p), _ptr(pos),
                                                _ptr(vel), _ptr(ids), _stream(stream)))


def sidm_kernel_sizes(ctx, n_ngb, h, stream=None):
    k = np.ascontiguousarray(n_ngb, dtype=np.int32)
    _check(ctx, load_library().sidm_kernel_sizes(ctx, k.ctypes.data_as(C.c_void_p), _ptr(h), _stream(stream)))


def sidm_scatter_step_binned(ctx, seed, step, xs, dt_max, n_bins, substep, bins, mass, vel, stats=None,
                             stream=None):
    _check(ctx, load_library().sidm_scatter_step_binned(ctx, C.c_uint64(int(seed)), C.c_uint64(int(step)), _ptr(xs),
                                                        float(dt_max), int(n_bins), int(substep), _ptr(bins),
                                                        _ptr(mass), _ptr(vel), _ptr(stats), _stream(stream)))


def sidm_host_kick(ctx, host, dt_max, n_bins, substep, phase, bins, pos, vel, stream=None):
    """host: a dict as host_struct takes; see include/sidm.h."""
    hs = host_struct(host)
    _check(ctx, load_library().sidm_host_kick(ctx, C.byref(hs), float(dt_max), int(n_bins), int(substep), int(phase),
                                              _ptr(bins), _ptr(pos), _ptr(vel), _stream(stream)))


def sidm_host_potential(ctx, host, pos, phi, stream=None):
    """Host potential at every particle into phi (f64 [N]); see include/sidm.h."""
    hs = host_struct(host)
    _check(ctx, load_library().sidm_host_potential(ctx, C.byref(hs), _ptr(pos), _ptr(phi), _stream(stream)))


def sidm_reflect_boundary(ctx, bound, pos, vel, stream=None):
    """bound: device f64 [H][4] = (cx, cy, cz, R) per halo; see include/sidm.h."""
    _check(ctx, load_library().sidm_reflect_boundary(ctx, _ptr(bound), _ptr(pos), _ptr(vel), _stream(stream)))


def sidm_scatter_step(ctx, seed, step, xs, dt, mass, vel, stats=None, stream=None):
    _check(ctx, load_library().sidm_scatter_step(ctx, C.c_uint64(int(seed)), C.c_uint64(int(step)), _ptr(xs),
                                                 _ptr(dt), _ptr(mass), _ptr(vel), _ptr(stats), _stream(stream)))


def sidm_energy_momentum(ctx, mass, vel, out, comp=None, stream=None):
    _check(ctx, load_library().sidm_energy_momentum(ctx, _ptr(mass), _ptr(vel), _ptr(out), _ptr(comp),
                                                    _stream(stream)))


def sidm_status(ctx, stream=None):
    """Synchronise; return the device status bits (raises on none of them)."""
    v = C.c_uint32(0)
    load_library().sidm_status(ctx, _stream(stream), C.byref(v))
    return int(v.value)


def sidm_get_perm(ctx, perm, stream=None):
    _check(ctx, load_library().sidm_get_perm(ctx, _ptr(perm), _stream(stream)))


def sidm_neighbours(ctx, n_ngb, k_stride, nbr, stream=None):
    k = np.ascontiguousarray(n_ngb, dtype=np.int32)
    _check(ctx, load_library().sidm_neighbours(ctx, k.ctypes.data_as(C.c_void_p), int(k_stride), _ptr(nbr),
                                               _stream(stream)))


def sidm_get_events(ctx, cap, ev, stream=None):
    n = C.c_int64(0)
    _check(ctx, load_library().sidm_get_events(ctx, int(cap), _ptr(ev), C.byref(n), _stream(stream)))
    return int(n.value)


def sidm_lambda_eval(ctx, d, hi, hj, out, stream=None):
    _check(ctx, load_library().sidm_lambda_eval(ctx, int(d.numel()), _ptr(d), _ptr(hi), _ptr(hj), _ptr(out),
                                                _stream(stream)))


def sidm_drift(ctx, dt, pos, vel, stream=None):
    _check(ctx, load_library().sidm_drift(ctx, _ptr(dt), _ptr(pos), _ptr(vel), _stream(stream)))


def sidm_get_sum_p(ctx, out, stream=None):
    _check(ctx, load_library().sidm_get_sum_p(ctx, _ptr(out), _stream(stream)))


def sidm_launch_count(ctx) -> int:
    return int(load_library().sidm_launch_count(ctx))


def sidm_energy_momentum_static(halo_off, precision, mass, vel, out, comp=None, stream=None):
    """Allocation-free per-halo energy and momentum (no context; see include/sidm.h)."""
    off = np.ascontiguousarray(halo_off, dtype=np.int64)
    prec = SIDM_FP64 if precision in ("fp64", SIDM_FP64) else SIDM_MIXED
    rc = load_library().sidm_energy_momentum_static(len(off) - 1, off.ctypes.data_as(C.c_void_p), prec, _ptr(mass),
                                                    _ptr(vel), _ptr(out), _ptr(comp), _stream(stream))
    if rc != SIDM_OK:
        raise SidmError(rc, load_library().sidm_static_last_error().decode())


def sidm_local_diagnostics(ctx, xs, mass, vel, G, out, stream=None):
    """Per-particle rho, nu, sigma_eff/m, h/l, Kn into out ([5][N], f32 or f64 by precision)."""
    _check(ctx, load_library().sidm_local_diagnostics(ctx, _ptr(xs), _ptr(mass), _ptr(vel), float(G), _ptr(out),
                                                      _stream(stream)))


def sidm_timestep_criterion(ctx, tau, dt_min, dt_max, n_bins, dt, dt_out=None, bin_out=None, dt_halo_min=None,
                            stream=None):
    """SIDM time step and power-of-two bin per particle, smallest step per halo."""
    _check(ctx, load_library().sidm_timestep_criterion(ctx, float(tau), float(dt_min), float(dt_max), int(n_bins),
                                                       _ptr(dt), _ptr(dt_out), _ptr(bin_out), _ptr(dt_halo_min),
                                                       _stream(stream)))


def sidm_warm_start(ctx, enable=True):
    """Enable/disable seeding the kernel-size search with the last kernel sizes."""
    _check(ctx, load_library().sidm_warm_start(ctx, 1 if enable else 0))


def sidm_diagnostics(ctx, reset=True):
    """Work counters of the kernel-size and pair kernels (see include/sidm.h)."""
    out = np.zeros(8, np.uint64)
    _check(ctx, load_library().sidm_diagnostics(ctx, out.ctypes.data_as(C.c_void_p), 1 if reset else 0))
    return out


def sidm_kernel_times(ctx, reset=True):
    """(ms[4], counts[4]) of {build, kernel sizes, pairs, resolve} since the last reset."""
    ms = np.zeros(4); cnt = np.zeros(4, np.int64)
    _check(ctx, load_library().sidm_kernel_times(ctx, ms.ctypes.data_as(C.c_void_p),
                                                 cnt.ctypes.data_as(C.c_void_p), 1 if reset else 0))
    return ms, cnt


# ------------------------------------------------------------------ convenience
@dataclass
class Stats:
    n_pairs: int
    n_events: int
    n_p_gt1: int
    n_near: int
    n_multi: int
    rounds: int
    status: int
    d_energy: float
    max_sum_p: float
    n_tested: int


def parse_stats(buf) -> Stats:
    a = np.frombuffer(buf.cpu().numpy().tobytes(), dtype=STATS_DTYPE)[0]
    return Stats(int(a["n_pairs"]), int(a["n_events"]), int(a["n_p_gt1"]), int(a["n_near"]), int(a["n_multi"]),
                 int(a["rounds"]), int(a["status"]), float(a["d_energy"]), float(a["max_sum_p"]),
                 int(a["n_tested"]))


class Context:
    """One libsidm context on one device, plus device copies of per-halo parameters."""

    def __init__(self, n_max, halo_max=1, ngb_max=64, event_cap=None, precision="mixed", device=0,
                 knn_warps=0, pair_warps=0, max_rounds=0, flags=0, grid_ctas=0, use_tma=0,
                 knn_groups=0, knn_chains=0, knn_flush=0, knn_slack=0.0, pair_per_round=0, knn_batch=0):
        torch = _torch()
        self.torch = torch
        self.precision = SIDM_FP64 if precision in ("fp64", SIDM_FP64) else SIDM_MIXED
        self.vdtype = torch.float64 if self.precision == SIDM_FP64 else torch.float32
        self.device = torch.device("cuda", device)
        cfg = SidmConfig(n_max=int(n_max), halo_max=int(halo_max), ngb_max=int(ngb_max),
                         event_cap=int(event_cap if event_cap is not None else max(4096, n_max // 4)),
                         precision=self.precision, device=int(device), knn_warps=int(knn_warps),
                         pair_warps=int(pair_warps), max_rounds=int(max_rounds), flags=int(flags),
                         grid_ctas=int(grid_ctas), use_tma=int(use_tma), knn_groups=int(knn_groups),
                         knn_chains=int(knn_chains), knn_flush=int(knn_flush), knn_slack=float(knn_slack),
                         pair_per_round=int(pair_per_round), knn_batch=int(knn_batch))
        self.cfg = cfg
        self.handle = sidm_create(cfg)
        self.stats_buf = torch.zeros(STATS_DTYPE.itemsize, dtype=torch.uint8, device=self.device)

    def close(self):
        if self.handle:
            sidm_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def xs_tensor(self, xs_list):
        """Device sidm_xs array from (kind, s0, w) or (kind, s0, w, angular) tuples."""
        a = np.zeros(len(xs_list), XS_DTYPE)
        for i, xs in enumerate(xs_list):
            kind, s0, w = xs[:3]
            a[i] = (int(kind), int(xs[3]) if len(xs) > 3 else 0, float(s0), float(w))
        return self.torch.from_numpy(np.frombuffer(a.tobytes(), np.uint8).copy()).to(self.device)

    def f64(self, values):
        return self.torch.as_tensor(np.asarray(values, np.float64), device=self.device)

    def build_cells(self, halo_off, pos, vel, ids, stream=None):
        sidm_build_cells(self.handle, halo_off, pos, vel, ids, stream)

    def kernel_sizes(self, n_ngb, h, stream=None):
        sidm_kernel_sizes(self.handle, n_ngb, h, stream)

    def scatter_step(self, seed, step, xs, dt, mass, vel, stats=None, stream=None):
        sidm_scatter_step(self.handle, seed, step, xs, dt, mass, vel,
                          self.stats_buf if stats is None else stats, stream)

    def scatter_step_binned(self, seed, step, xs, dt_max, n_bins, substep, bins, mass, vel, stats=None,
                            stream=None):
        sidm_scatter_step_binned(self.handle, seed, step, xs, dt_max, n_bins, substep, bins, mass, vel,
                                 self.stats_buf if stats is None else stats, stream)

    def host_kick(self, host, dt_max, n_bins, substep, phase, bins, pos, vel, stream=None):
        sidm_host_kick(self.handle, host, dt_max, n_bins, substep, phase, bins, pos, vel, stream)

    def host_potential(self, host, pos, phi, stream=None):
        sidm_host_potential(self.handle, host, pos, phi, stream)

    def reflect_boundary(self, bound, pos, vel, stream=None):
        sidm_reflect_boundary(self.handle, bound, pos, vel, stream)

    def energy_momentum(self, mass, vel, out, comp=None, stream=None):
        sidm_energy_momentum(self.handle, mass, vel, out, comp, stream)

    def status(self, stream=None):
        return sidm_status(self.handle, stream)

    def perm(self, n):
        t = self.torch.empty(n, dtype=self.torch.int32, device=self.device)
        sidm_get_perm(self.handle, t)
        return t

    def neighbours(self, n_ngb, n, k_stride):
        t = self.torch.zeros((n, k_stride), dtype=self.torch.int32, device=self.device)
        sidm_neighbours(self.handle, n_ngb, k_stride, t)
        return t

    def events(self, cap=None):
        cap = int(cap if cap is not None else self.cfg.event_cap)
        buf = self.torch.zeros(max(cap, 1) * EVENT_DTYPE.itemsize, dtype=self.torch.uint8, device=self.device)
        n = sidm_get_events(self.handle, cap, buf)
        m = min(n, cap)
        return n, np.frombuffer(buf[: m * EVENT_DTYPE.itemsize].cpu().numpy().tobytes(), EVENT_DTYPE)

    def stats(self):
        return parse_stats(self.stats_buf)

    def lambda_eval(self, d, hi, hj):
        out = self.torch.empty_like(d)
        sidm_lambda_eval(self.handle, d, hi, hj, out)
        return out

    def drift(self, dt, pos, vel, stream=None):
        sidm_drift(self.handle, dt, pos, vel, stream)

    def sum_p(self, n):
        t = self.torch.empty(n, dtype=self.torch.float32, device=self.device)
        sidm_get_sum_p(self.handle, t)
        return t

    def launch_count(self):
        return sidm_launch_count(self.handle)

    def kernel_times(self, reset=True):
        return sidm_kernel_times(self.handle, reset)

    def diagnostics(self, reset=True):
        return sidm_diagnostics(self.handle, reset)

    def warm_start(self, enable=True):
        sidm_warm_start(self.handle, enable)

    def timestep_criterion(self, tau, dt_min, dt_max, n_bins, dt, n, n_halos, stream=None):
        """(dt f64[n], bin int32[n], smallest dt per halo f64[n_halos]) in the current order."""
        torch = self.torch
        dto = torch.empty(n, dtype=torch.float64, device=self.device)
        bo = torch.empty(n, dtype=torch.int32, device=self.device)
        hm = torch.empty(n_halos, dtype=torch.float64, device=self.device)
        sidm_timestep_criterion(self.handle, tau, dt_min, dt_max, n_bins, dt, dto, bo, hm, stream)
        return dto, bo, hm

    def local_diagnostics(self, xs, mass, vel, n, G=1.0, stream=None):
        """dict of per-particle rho, nu, sigma_eff, h_over_l, kn (tensors of the form's precision, current order)."""
        out = self.torch.empty((5, n), dtype=self.vdtype, device=self.device)
        sidm_local_diagnostics(self.handle, xs, mass, vel, G, out, stream)
        return {"rho": out[0], "nu": out[1], "sigma_eff": out[2], "h_over_l": out[3], "kn": out[4]}

"""Satellite pieces on the GPU against the FP64 oracle: the analytic host's
kick on individual power-of-two steps and its potential, the scatter step on
individual steps, and a short kick-drift-kick run of a satellite in the host
(Sect. 4.1 evolves the satellite in an external potential of six parts --
NFW halo, Hernquist bulge, four Miyamoto-Nagai disks -- from a given position
and velocity; individual time steps).

Tolerances: the kick adds an FP64 acceleration to FP32 velocities, so one
kick agrees to 1e-6 of the speed; the potential is FP64 on both sides with
different library logarithms and square roots (1e-13); the binned scatter step
obeys the scatter tolerances (event sets equal except |P - u| < 1e-6,
velocities to 1e-5 of the pair speed scale, per-particle sums to 1e-5); the
run without scattering (neighbouring orbits in a smooth potential do not
diverge) keeps positions to 1e-6 and velocities to 1e-5 relative over three
big steps.
"""
import math

import numpy as np
import pytest

from oracle import oracle as O
from paper_2506_06269_gb300 import ics

from gpu_helpers import compare_events

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

HOST = ics.milky_way_host()
NB, DT_MAX = 4, 0.02


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2506_06269_gb300 import build
    build.build()


def _satellite(n, seed, where="orbit"):
    """An NFW subhalo at the paper's initial position and velocity in the host
    ("orbit"), or at rest at the host's centre, twice enlarged, so that its
    particles sample the bulge and the disks ("centre")."""
    halo = ics.nfw(n, seed)
    if where == "orbit":
        x0, v0 = ics.satellite_orbit()
        pos = halo.pos + x0[:, None]
        vel = (halo.vel + v0[:, None]).astype(np.float32).astype(np.float64)
    else:
        pos = 2.0 * halo.pos
        vel = halo.vel.astype(np.float32).astype(np.float64)
    return halo, pos, vel


def _context(pos, vel, ids, k=32, flags=0, n_halo=None):
    from paper_2506_06269_gb300 import sidm
    n = pos.shape[1]
    ctx = sidm.Context(n_max=n, halo_max=1, ngb_max=k, event_cap=1 << 16, flags=flags)
    dev = ctx.device
    t = (torch.tensor(pos, device=dev), torch.tensor(vel.astype(np.float32), device=dev),
         torch.tensor(ids.astype(np.int64), device=dev).to(torch.int32))
    ctx.build_cells([0, n], *t)
    perm = ctx.perm(n).cpu().numpy().astype(np.int64)
    return ctx, t, perm


@pytest.mark.parametrize("where", ["orbit", "centre"])
def test_host_kick_matches_oracle(where):
    halo, pos, vel = _satellite(20000, 51, where)
    n = halo.n
    bins = np.random.default_rng(2).integers(0, NB, n).astype(np.int32)
    ctx, (p, v, ids), perm = _context(pos, vel, halo.ids)
    bins_g = torch.tensor(bins[perm], device=ctx.device)
    vo = vel.copy()
    for substep, phase in ((0, 0), (1, 1), (3, 1), (4, 0), (6, 0), (7, 1)):
        ctx.host_kick(HOST, DT_MAX, NB, substep, phase, bins_g, p, v)
        vo = O.host_kick(pos, vo, HOST, DT_MAX, bins, NB, substep, phase)
    assert ctx.status() == 0
    got = np.empty((3, n)); got[:, perm] = v.cpu().numpy().astype(np.float64)
    speed = np.linalg.norm(vo, axis=0)
    assert np.all(np.abs(got - vo).max(axis=0) <= 1e-6 * speed)
    assert not np.allclose(vo, vel)
    ctx.close()


@pytest.mark.parametrize("where", ["orbit", "centre"])
def test_host_potential_matches_oracle(where):
    halo, pos, vel = _satellite(5000, 54, where)
    n = halo.n
    ctx, (p, v, ids), perm = _context(pos, vel, halo.ids)
    phi = torch.zeros(n, dtype=torch.float64, device=ctx.device)
    ctx.host_potential(HOST, p, phi)
    assert ctx.status() == 0
    got = np.empty(n); got[perm] = phi.cpu().numpy()
    ctx.close()
    want = O.host_phi(HOST, pos)
    np.testing.assert_allclose(got, want, rtol=1e-13, atol=0)


def test_host_arguments_are_checked():
    from paper_2506_06269_gb300 import sidm
    halo, pos, vel = _satellite(300, 55)
    ctx, (p, v, ids), perm = _context(pos, vel, halo.ids)
    phi = torch.zeros(halo.n, dtype=torch.float64, device=ctx.device)
    bad = [dict(HOST, disks=HOST["disks"] + [(1.0, 1.0, 1.0)]),      # five disks
           dict(HOST, disks=[(1.0, 1.0, 0.0)]),                     # b_d = 0
           dict(HOST, nfw=(1.0, 0.0)),                              # r_s = 0
           dict(HOST, bulge=(-1.0, 1.0))]                           # negative mass
    for host in bad:
        with pytest.raises((sidm.SidmError, ValueError)):
            ctx.host_potential(host, p, phi)
        with pytest.raises((sidm.SidmError, ValueError)):
            ctx.host_kick(host, DT_MAX, NB, 0, 0, None, p, v)
    ctx.close()


@pytest.mark.parametrize("substep", [0, 2, 5])
def test_binned_scatter_step_matches_oracle(substep):
    from paper_2506_06269_gb300 import sidm
    h = ics.hernquist(16384, 52)
    n = h.n
    vin = h.vel.astype(np.float32).astype(np.float64)
    # bins skewed towards short steps, so that every sub-step tests some pairs
    bins = np.random.default_rng(substep).choice(NB, n, p=[0.1, 0.15, 0.25, 0.5]).astype(np.int32)
    ctx, (p, v, ids), perm = _context(h.pos, vin, h.ids, k=32, flags=sidm.SIDM_FLAG_SUM_P)
    hg = torch.zeros(n, dtype=torch.float32, device=ctx.device)
    ctx.kernel_sizes([32], hg)
    xs = (0, 300.0, 1.0)
    dt_max = 0.4
    ctx.scatter_step_binned(3, 7, ctx.xs_tensor([xs]), dt_max, NB, substep, torch.tensor(bins[perm], device=ctx.device),
                            ctx.f64([h.mass]), v)
    assert ctx.status() == 0
    n_ev, ev = ctx.events()
    sump = np.empty(n); sump[perm] = ctx.sum_p(n).cpu().numpy().astype(np.float64)
    vg = np.empty((3, n)); vg[:, perm] = v.cpu().numpy().astype(np.float64)
    ctx.close()
    ev = ev.copy(); ev["i"] = perm[ev["i"]]; ev["j"] = perm[ev["j"]]
    oh, _, _ = O.knn(h.pos, h.ids, 32, O.MODE_MIXED)
    oev, _, osum = O.pairs(h.pos, vin, h.ids, oh, O.MODE_MIXED, xs, h.mass, 0.0, 3, 7, 0, ev_cap=1 << 20,
                           bins=bins, n_bins=NB, substep=substep, dt_max=dt_max)
    oev = np.sort(oev, order="key")
    assert len(oev) > (100 if substep == 0 else 5)
    only_o, only_g = compare_events(ev, oev)
    # in this deliberately dense case single pairs reach P ~ 1, and the FP32
    # table's absolute error of Lambda adds up over hundreds of partners
    np.testing.assert_allclose(sump, osum, rtol=5e-5, atol=1e-7 * osum.max())
    # velocities of particles in exactly one (oracle) event, others untouched
    vo, _ = O.apply_events(oev, np.full(n, h.mass), vin)
    cnt = np.bincount(np.concatenate([oev["i"], oev["j"]]).astype(np.int64), minlength=n)
    differ = set(only_o) | set(only_g)
    single = [e for e in oev if cnt[e["i"]] == 1 and cnt[e["j"]] == 1 and int(e["key"]) not in differ]
    for e in single:
        i, j = int(e["i"]), int(e["j"])
        scale = np.linalg.norm(vin[:, i]) + np.linalg.norm(vin[:, j])
        assert np.abs(vg[:, [i, j]] - vo[:, [i, j]]).max() <= 1e-5 * scale
    quiet = (cnt == 0)
    gcnt = np.bincount(np.concatenate([ev["i"], ev["j"]]).astype(np.int64), minlength=n)
    quiet &= gcnt == 0
    assert np.array_equal(vg[:, quiet], vin[:, quiet])


def test_satellite_run_without_scattering_matches_oracle():
    halo, pos, vel = _satellite(8192, 53)
    n = halo.n
    r = np.linalg.norm(halo.pos, axis=0)
    assert np.linalg.norm(pos.mean(axis=1)) > 90.0          # far out on the paper's orbit
    bins = np.clip((3 - np.log2(np.maximum(r, 1e-3) / 0.25)).astype(np.int32), 0, NB - 1).astype(np.int32)
    ctx, (p, v, ids), perm = _context(pos, vel, halo.ids)
    hg = torch.zeros(n, dtype=torch.float32, device=ctx.device)
    bins_g = torch.tensor(bins[perm], device=ctx.device)
    order = perm.copy()                                       # current position -> input index
    xs0 = ctx.xs_tensor([(0, 0.0, 1.0)])
    mass = ctx.f64([halo.mass])
    S = 1 << (NB - 1)
    delta = DT_MAX / S
    dtt = ctx.f64([delta])
    xo, vo = pos.copy(), vel.copy()
    for big in range(3):
        for s in range(S):
            ctx.host_kick(HOST, DT_MAX, NB, s, 0, bins_g, p, v)
            ctx.kernel_sizes([32], hg)
            ctx.scatter_step_binned(1, big * S + s, xs0, DT_MAX, NB, s, bins_g, mass, v)
            ctx.drift(dtt, p, v)
            ctx.host_kick(HOST, DT_MAX, NB, s, 1, bins_g, p, v)
            ctx.build_cells([0, n], p, v, ids)                # the positions moved: new order
            pm = ctx.perm(n).to(torch.int64)
            bins_g = bins_g[pm]
            order = order[pm.cpu().numpy()]
            vo = O.host_kick(xo, vo, HOST, DT_MAX, bins, NB, s, 0)
            xo = xo + vo * delta
            vo = O.host_kick(xo, vo, HOST, DT_MAX, bins, NB, s, 1)
    assert ctx.status() == 0
    xg = np.empty((3, n)); xg[:, order] = p.cpu().numpy()
    vg = np.empty((3, n)); vg[:, order] = v.cpu().numpy().astype(np.float64)
    ctx.close()
    assert np.abs(xg - xo).max() <= 1e-6 * np.abs(xo).max()
    assert np.all(np.abs(vg - vo).max(axis=0) <= 1e-5 * np.linalg.norm(vo, axis=0))
    assert np.abs(xo - pos).max() > 1e-3                      # it moved

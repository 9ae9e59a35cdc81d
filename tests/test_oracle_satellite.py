"""Pins of the oracle's satellite pieces (no GPU): the analytic NFW host, the
kick-drift-kick schedule with individual power-of-two steps, and the pair pass
on individual steps (Sect. 4.1 evolves the satellite in an external
potential; individual time steps, Sect. 3.1)."""
import math

import numpy as np
import pytest
from scipy import integrate

from oracle import oracle as O
from paper_2506_06269_gb300 import ics

G, MN, RS = 1.0, 1000.0 / (math.log(11.0) - 10.0 / 11.0), 15.3


def test_host_mass_and_potential():
    # M(<r) is the integral of the NFW density rho = M_n / (4 pi R^3 x (1+x)^2);
    # the acceleration is -dPhi/dr and Phi vanishes at infinity
    rho = lambda r: MN / (4 * math.pi * RS ** 3) / ((r / RS) * (1 + r / RS) ** 2)
    for r in (0.01, 1.0, 15.3, 30.0, 153.0):
        m = integrate.quad(lambda x: 4 * math.pi * x * x * rho(x), 0, r, epsrel=1e-12, limit=200)[0]
        assert O.host_mass(r, MN, RS) == pytest.approx(m, rel=1e-9)
        eps = 1e-5 * r
        dphi = (O.host_phi(r + eps, G, MN, RS) - O.host_phi(r - eps, G, MN, RS)) / (2 * eps)
        assert dphi == pytest.approx(G * O.host_mass(r, MN, RS) / r ** 2, rel=1e-7)
    assert O.host_mass(10 * RS, MN, RS) == pytest.approx(1000.0, rel=1e-14)
    assert abs(O.host_phi(1e16, G, MN, RS)) < 1e-11
    assert O.host_phi(1e-9, G, MN, RS) == pytest.approx(O.host_phi(0.0, G, MN, RS), rel=1e-9)


def _run_schedule(pos, vel, bins, n_bins, dt_max, big_steps):
    """Block-step KDK: per sub-step, opening kicks, drift by the smallest step, closing kicks."""
    host = (G, MN, RS, (0.0, 0.0, 0.0))
    S = 1 << (n_bins - 1)
    delta = dt_max / S
    x, v = pos.copy(), vel.copy()
    for _ in range(big_steps):
        for s in range(S):
            v = O.host_kick(x, v, host, dt_max, bins, n_bins, s, 0)
            x = x + v * delta
            v = O.host_kick(x, v, host, dt_max, bins, n_bins, s, 1)
    return x, v


def test_block_steps_reduce_to_kick_drift_kick_of_each_bin():
    # a particle of bin b moves exactly as a plain KDK with its own step dt_max / 2^b
    rng = np.random.default_rng(3)
    n, n_bins, dt_max = 8, 4, 0.5
    pos = rng.uniform(20, 40, (3, n)); vel = rng.normal(0, 3, (3, n))
    bins = np.arange(n) % n_bins
    x, v = _run_schedule(pos, vel, bins, n_bins, dt_max, 3)
    host = (G, MN, RS, (0.0, 0.0, 0.0))
    for i in range(n):
        dtb = dt_max / 2 ** bins[i]
        xi, vi = pos[:, [i]].copy(), vel[:, [i]].copy()
        for _ in range(3 * 2 ** bins[i]):
            vi = O.host_kick(xi, vi, host, dtb)                       # half kick dtb / 2
            xi = xi + vi * dtb
            vi = O.host_kick(xi, vi, host, dtb)
        assert np.allclose(x[:, [i]], xi, rtol=1e-12, atol=1e-12), i
        assert np.allclose(v[:, [i]], vi, rtol=1e-12, atol=1e-12), i


def test_circular_orbit_energy_bounded():
    # kick-drift-kick is symplectic: the energy error of a circular orbit at 30 stays
    # small and bounded over 20 orbits, and the radius stays put
    r0 = 30.0
    vc = math.sqrt(G * O.host_mass(r0, MN, RS) / r0)
    period = 2 * math.pi * r0 / vc
    pos = np.array([[r0], [0.0], [0.0]]); vel = np.array([[0.0], [vc], [0.0]])
    e0 = 0.5 * vc * vc + O.host_phi(r0, G, MN, RS)
    x, v = pos, vel
    steps_per_orbit = 200
    dt = period / steps_per_orbit
    worst = 0.0
    for k in range(20):
        x, v = _run_schedule(x, v, np.zeros(1, np.int32), 1, dt, steps_per_orbit)
        r = float(np.linalg.norm(x))
        e = 0.5 * float((v ** 2).sum()) + O.host_phi(r, G, MN, RS)
        worst = max(worst, abs(e / e0 - 1))
        assert abs(r / r0 - 1) < 1e-3
    assert worst < 1e-4


def test_binned_pairs_reduce_to_the_plain_pass():
    h = ics.hernquist(3000, 12)
    vel = h.vel.astype(np.float32).astype(np.float64)
    hh, _, _ = O.knn(h.pos, h.ids, 32, O.MODE_MIXED)
    xs = (0, 10.0, 1.0)
    dt_max = 0.2
    # every particle in bin 0: the plain pass with dt = dt_max
    ev0, _, sp0 = O.pairs(h.pos, vel, h.ids, hh, O.MODE_MIXED, xs, h.mass, dt_max, 1, 5, 0)
    evb, _, spb = O.pairs(h.pos, vel, h.ids, hh, O.MODE_MIXED, xs, h.mass, 0.0, 1, 5, 0,
                          bins=np.zeros(h.n, np.int32), n_bins=4, substep=0, dt_max=dt_max)
    # (per-particle sums are accumulated by parallel atomics: equal up to summation order)
    assert np.array_equal(ev0, evb) and np.allclose(sp0, spb, rtol=1e-12, atol=0)
    # mixed bins at sub-step 2 of 8: only pairs whose particles both open a step there
    # (bins 2 and 3, periods 2 and 1), each on the longer step; sums are rates
    # scaled to dt_max
    bins = np.random.default_rng(5).integers(0, 4, h.n).astype(np.int32)
    evs, _, sps = O.pairs(h.pos, vel, h.ids, hh, O.MODE_MIXED, xs, h.mass, 0.0, 1, 5, 0,
                          bins=bins, n_bins=4, substep=2, dt_max=dt_max)
    assert evs.size > 0
    assert np.all(bins[evs["i"]] >= 2) and np.all(bins[evs["j"]] >= 2)
    full = {int(e["key"]): e for e in ev0}
    for e in evs:
        dtp = dt_max / 2 ** min(bins[e["i"]], bins[e["j"]])
        if int(e["key"]) in full:
            assert e["P"] == pytest.approx(full[int(e["key"])]["P"] * dtp / dt_max, rel=1e-12)
    opened = bins >= 2
    assert np.all(sps[~opened] == 0.0)
    assert np.all(sps[opened] <= sp0[opened] * (1 + 1e-12))

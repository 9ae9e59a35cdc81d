"""Pins of the oracle's satellite pieces (no GPU): the analytic host, the
kick-drift-kick schedule with individual power-of-two steps, and the pair pass
on individual steps (Sect. 4.1 evolves the satellite in an external potential
of six parts -- an NFW halo, a Hernquist bulge and four Miyamoto-Nagai disks --
on individual time steps).

The host's potential and acceleration are pinned by what fixes them apart from
their own formulas: the enclosed mass of the NFW density, the acceleration as
minus the numerical gradient of the potential, Poisson's equation against the
textbook densities of each part, the Plummer special case of a disk, the point
mass far field, and the paper's numbers for the orbit and the Milky Way.
"""
import math

import numpy as np
import pytest
from scipy import integrate

from oracle import oracle as O
from paper_2506_06269_gb300 import ics

RHO_S, RS = 1000.0 / (4 * math.pi * (math.log(11.0) - 10.0 / 11.0) * 15.3 ** 3), 15.3
NFW_HOST = {"G": 1.0, "center": (0.0, 0.0, 0.0), "nfw": (RHO_S, RS)}
MW = ics.milky_way_host()
G = 1.0


def _parts(host):
    """The host split into one-part hosts."""
    out = []
    if host.get("nfw"):
        out.append({"G": host["G"], "center": host["center"], "nfw": host["nfw"]})
    if host.get("bulge"):
        out.append({"G": host["G"], "center": host["center"], "bulge": host["bulge"]})
    for d in host.get("disks", ()):
        out.append({"G": host["G"], "center": host["center"], "disks": [d]})
    return out


def _density(part, x):
    """Textbook density of a one-part host at x (Binney & Tremaine: NFW; Hernquist
    1990; Miyamoto & Nagai 1975), G = 1 units."""
    d = np.asarray(x, float) - np.asarray(part["center"], float)
    r = float(np.linalg.norm(d))
    if part.get("nfw"):
        rho_s, r_s = part["nfw"]
        u = r / r_s
        return rho_s / (u * (1 + u) ** 2)
    if part.get("bulge"):
        m, a = part["bulge"]
        return m * a / (2 * math.pi * r * (r + a) ** 3)
    (m, a, b), = part["disks"]
    R2, z = d[0] ** 2 + d[1] ** 2, d[2]
    zeta = math.sqrt(z * z + b * b)
    D = R2 + (a + zeta) ** 2
    return b * b * m / (4 * math.pi) * (a * R2 + (a + 3 * zeta) * (a + zeta) ** 2) / (D ** 2.5 * zeta ** 3)


_PTS = [np.array(p) for p in ([45.4, 31.3, 79.2], [3.0, -2.0, 0.01], [0.5, 0.2, -0.3], [6.0, 1.0, 0.05],
                               [-1.2, 0.4, 1.7], [20.0, -15.0, -4.0], [0.03, 0.02, 0.02])]


def test_nfw_mass_and_potential():
    # M(<r) is the integral of the NFW density; -dPhi/dr = G M(<r) / r^2; Phi -> 0 at infinity
    rho = lambda r: RHO_S / ((r / RS) * (1 + r / RS) ** 2)
    for r in (0.01, 1.0, 15.3, 30.0, 153.0):
        m = integrate.quad(lambda x: 4 * math.pi * x * x * rho(x), 0, r, epsrel=1e-12, limit=200)[0]
        assert O.host_mass(r, RHO_S, RS) == pytest.approx(m, rel=1e-9)
        eps = 1e-5 * r
        dphi = (O.host_phi(NFW_HOST, [r + eps, 0, 0]) - O.host_phi(NFW_HOST, [r - eps, 0, 0])) / (2 * eps)
        assert dphi == pytest.approx(G * O.host_mass(r, RHO_S, RS) / r ** 2, rel=1e-7)
    assert O.host_mass(10 * RS, RHO_S, RS) == pytest.approx(1000.0, rel=1e-14)
    assert abs(O.host_phi(NFW_HOST, [1e16, 0, 0])) < 1e-11
    assert O.host_phi(NFW_HOST, [1e-9, 0, 0]) == pytest.approx(O.host_phi(NFW_HOST, [0, 0, 0]), rel=1e-9)


@pytest.mark.parametrize("k", range(len(_PTS)))
def test_acceleration_is_minus_the_gradient_of_the_potential(k):
    x = _PTS[k]
    for host in [MW] + _parts(MW):
        a = O.host_accel(host, x)
        scale = max(1e-3, 1e-3 * float(np.linalg.norm(x)))
        g = np.zeros(3)
        for c in range(3):
            e = np.zeros(3); e[c] = 1e-3 * scale
            # fourth-order central difference
            g[c] = (-O.host_phi(host, x + 2 * e) + 8 * O.host_phi(host, x + e) - 8 * O.host_phi(host, x - e)
                    + O.host_phi(host, x - 2 * e)) / (12 * e[c])
        assert np.abs(a + g).max() <= 1e-7 * np.linalg.norm(a) + 1e-12, (k, host)


@pytest.mark.parametrize("k", range(len(_PTS)))
def test_poisson_equation_gives_the_textbook_densities(k):
    # -div a = 4 pi G rho for each part, and for the sum of the six
    x = _PTS[k]
    total = 0.0
    for part in _parts(MW):
        h = 1e-4 * max(0.02, min(1.0, float(np.linalg.norm(x))))
        div = 0.0
        for c in range(3):
            e = np.zeros(3); e[c] = h
            div += (-O.host_accel(part, x + 2 * e)[c] + 8 * O.host_accel(part, x + e)[c]
                    - 8 * O.host_accel(part, x - e)[c] + O.host_accel(part, x - 2 * e)[c]) / (12 * h)
        rho = _density(part, x)
        total += rho
        assert -div == pytest.approx(4 * math.pi * G * rho, rel=2e-6, abs=1e-9 * abs(div) + 1e-12), (k, part)
    h = 1e-4 * max(0.02, min(1.0, float(np.linalg.norm(x))))
    div = sum((O.host_accel(MW, x + h * np.eye(3)[c])[c] - O.host_accel(MW, x - h * np.eye(3)[c])[c]) / (2 * h)
              for c in range(3))
    assert -div == pytest.approx(4 * math.pi * G * total, rel=1e-4)


def test_disk_special_cases_and_far_field():
    # a = 0: the Miyamoto-Nagai disk is a Plummer sphere of scale b
    m, b = 2.5, 0.7
    pl = {"G": 1.0, "center": (1.0, -2.0, 0.5), "disks": [(m, 0.0, b)]}
    for x in _PTS:
        r = np.linalg.norm(x - np.array(pl["center"]))
        assert O.host_phi(pl, x) == pytest.approx(-m / math.sqrt(r * r + b * b), rel=1e-14)
        a = O.host_accel(pl, x)
        np.testing.assert_allclose(a, -m * (x - np.array(pl["center"])) / (r * r + b * b) ** 1.5, rtol=1e-13)
    # far away the bulge and the disks act as a point of their total mass
    nobulge = {k: v for k, v in MW.items() if k != "nfw"}
    mt = MW["bulge"][0] + sum(d[0] for d in MW["disks"])
    for u in ([1, 0, 0], [0, 0, 1], [0.6, 0.0, 0.8]):
        x = 1e7 * np.array(u, float)
        assert O.host_phi(nobulge, x) * 1e7 == pytest.approx(-mt, rel=1e-6)
        np.testing.assert_allclose(O.host_accel(nobulge, x), -mt * x / 1e21, rtol=1e-6)
    # axisymmetric about z and even in z
    x = np.array([3.0, 4.0, 0.2])
    for y in ([5.0, 0.0, 0.2], [0.0, -5.0, 0.2], [-3.0, -4.0, -0.2]):
        assert O.host_phi(MW, y) == pytest.approx(O.host_phi(MW, x), rel=1e-14)


def test_paper_orbit_and_milky_way_rotation():
    # Sect. 4.1: the satellite starts 123.6 kpc from the host's centre at 109 km/s
    L, M, V = ics.satellite_units()
    p, v = ics.satellite_orbit()
    assert np.linalg.norm(p) * L == pytest.approx(123.6, abs=0.05)
    assert np.linalg.norm(v) * V == pytest.approx(109.0, abs=0.1)
    # the halo of Sect. 2: about 2.8e9 M_sun in all (c ~ 22); inside 10 r_s somewhat less
    assert 1.0e9 < M < 2.8e9
    # the host mimics the Milky Way: a nearly flat rotation curve near 220 km/s
    vc = [math.sqrt(-O.host_accel(MW, [R / L, 0.0, 0.0])[0] * R / L) * V for R in (4.0, 8.0, 15.0, 30.0, 50.0)]
    assert 200.0 < vc[1] < 250.0
    assert max(vc) / min(vc) < 1.1


def _run_schedule(pos, vel, bins, n_bins, dt_max, big_steps):
    """Block-step KDK: per sub-step, opening kicks, drift by the smallest step, closing kicks."""
    host = MW
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
    host = MW
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
    # kick-drift-kick is symplectic: the energy error of a circular orbit in the
    # disk plane at R = 30 stays small and bounded over 20 orbits, the radius stays put
    r0 = 30.0
    vc = math.sqrt(-O.host_accel(MW, [r0, 0.0, 0.0])[0] * r0)
    period = 2 * math.pi * r0 / vc
    pos = np.array([[r0], [0.0], [0.0]]); vel = np.array([[0.0], [vc], [0.0]])
    e0 = 0.5 * vc * vc + O.host_phi(MW, pos[:, 0])
    x, v = pos, vel
    steps_per_orbit = 200
    dt = period / steps_per_orbit
    worst = 0.0
    for k in range(20):
        x, v = _run_schedule(x, v, np.zeros(1, np.int32), 1, dt, steps_per_orbit)
        r = float(np.linalg.norm(x))
        e = 0.5 * float((v ** 2).sum()) + O.host_phi(MW, x[:, 0])
        worst = max(worst, abs(e / e0 - 1))
        assert abs(r / r0 - 1) < 1e-3
        assert abs(x[2, 0]) < 1e-9
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


def test_host_edge_cases():
    # a host with no parts exerts nothing; moving the centre with the point
    # changes nothing; the spherical parts pull towards the centre
    empty = {"G": 1.0, "center": (1.0, 2.0, 3.0)}
    x = np.array([4.0, -1.0, 0.5])
    assert O.host_phi(empty, x) == 0.0
    assert np.all(O.host_accel(empty, x) == 0.0)
    shift = np.array([7.0, -3.0, 11.0])
    moved = dict(MW, center=tuple(shift))
    assert O.host_phi(moved, x + shift) == pytest.approx(O.host_phi(MW, x), rel=1e-13)
    np.testing.assert_allclose(O.host_accel(moved, x + shift), O.host_accel(MW, x), rtol=1e-12)
    for part in _parts(MW)[:2]:                      # the NFW halo and the bulge
        a = O.host_accel(part, x)
        assert np.dot(a, x) < 0 and np.linalg.norm(np.cross(a, x)) <= 1e-12 * np.linalg.norm(a) * np.linalg.norm(x)
    # at the centre itself the spherical parts add nothing (and stay finite)
    assert np.all(np.isfinite(O.host_accel(MW, [0.0, 0.0, 0.0])))
    np.testing.assert_allclose(O.host_accel({"G": 1.0, "center": (0, 0, 0), "nfw": MW["nfw"], "bulge": MW["bulge"]},
                                            [0.0, 0.0, 0.0]), 0.0, atol=0)

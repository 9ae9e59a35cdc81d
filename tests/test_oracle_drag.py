"""Pins of the oracle's forward-dominated (frictional) scattering (no GPU).

Paper: Sect. 3.8 (the forward-dominated cross-section is the limit of a
vanishing scattering angle at constant momentum transfer), App. A (strengths
are given as the viscosity cross-section sigma_V, normalised to the total
cross-section for isotropic scattering), Sect. 2 and Sect. 5 (every
interaction conserves pair energy and momentum).

What pins it, other than its own formulas:
  - conservation: every interaction keeps the pair's momentum and kinetic
    energy, so the totals of a dense multi-interaction step are unchanged;
  - the viscosity normalisation: sigma_V weights the scattering angle by
    (3/2) sin^2 theta = 1 - P_2(cos theta), the relaxation of the l = 2 moment
    of the relative-velocity direction.  An isotropic event relaxes it fully,
    so at equal sigma_V the turn alpha of each interaction, read off the
    output velocities, must give (3/2) sin^2 alpha = P (1 - P/6) with P the
    isotropic collision probability (sigma_V/m) m_j |u| Lambda dt -- equal to
    first order in P;
  - the drag: averaged over the random direction, u' = (1 - D) u, and the
    turn is isotropic about u in any orthonormal frame of the normal plane
    (the test builds its own frame);
  - the closed-form rate: in a uniform Maxwellian box the summed l = 2
    relaxation per particle and unit time equals the isotropic collision
    rate rho (sigma_V/m) 4 sigma_v / sqrt(pi);
  - a zero cross-section leaves every velocity bit-unchanged.
"""
import math

import numpy as np
import pytest

from oracle import oracle as O
from paper_2506_06269_gb300 import ics


def _box(n, seed, hval, sigma_v=(1.0, 1.0, 1.0)):
    rng = np.random.default_rng(seed)
    pos = rng.random((3, n))
    vel = (rng.standard_normal((3, n)) * np.asarray(sigma_v)[:, None]).astype(np.float32).astype(np.float64)
    ids = np.arange(n, dtype=np.uint32)
    return pos, vel, ids, np.full(n, np.float64(np.float32(hval)))


def test_drag_records_every_in_range_pair_with_its_geometric_factor():
    h = ics.hernquist(3000, 41)
    vel = h.vel.astype(np.float32).astype(np.float64)
    hh, _, _ = O.knn(h.pos, h.ids, 32, O.MODE_MIXED)
    rec, st, _ = O.pairs(h.pos, vel, h.ids, hh, O.MODE_MIXED, (0, 10.0, 1.0, 1), h.mass, 0.01, 3, 0, 0,
                         ev_cap=1 << 20)
    iso, st_iso, _ = O.pairs(h.pos, vel, h.ids, hh, O.MODE_MIXED, (0, 1e300, 1.0), h.mass, 0.01, 3, 0, 0,
                             ev_cap=1 << 20)
    assert st["n_pairs"] == st_iso["n_pairs"] == rec.size == st["n_events"] > 10000
    assert st["n_near"] == 0 and np.all(rec["u"] == -1.0)
    # every pair with a nonzero overlap fires in the huge-sigma isotropic pass
    assert set(iso["key"].tolist()) <= set(rec["key"].tolist())
    for e in rec[:: rec.size // 50]:
        i, j = int(e["i"]), int(e["j"])
        d = np.linalg.norm(h.pos[:, i] - h.pos[:, j])
        assert e["P"] == pytest.approx(h.mass * O.lam(d, hh[i], hh[j]) * 0.01, rel=1e-12, abs=0)


def test_drag_conserves_pair_energy_and_momentum_in_a_dense_step():
    n = 4000
    pos, vel, ids, h = _box(n, 42, 0.12)
    m = 1.0 / n
    rec, st, _ = O.pairs(pos, vel, ids, h, O.MODE_FP64, (1, 50.0, 0.7, 1), m, 0.05, 9, 2, 0, ev_cap=n * 600)
    assert rec.size > 40 * n                          # every particle takes part in about 90 interactions
    v1, dE, D = O.apply_drag(rec, np.full(n, m), (1, 50.0, 0.7), vel)
    e0, e1 = O.energy_momentum(m, vel), O.energy_momentum(m, v1)
    assert abs(e1[0] - e0[0]) <= 1e-13 * e0[0]
    assert np.all(np.abs(e1[1:] - e0[1:]) <= 1e-14 * m * np.abs(vel).sum())
    assert np.all(np.abs(dE) <= 1e-14 * e0[0])
    assert D.max() > 1e-3 and np.any(v1 != vel)


def test_drag_turn_angle_matches_the_viscosity_normalisation():
    # replay the records one by one and read the turn of u off the velocities
    n, s0 = 1500, 30.0
    pos, vel, ids, h = _box(n, 43, 0.1)
    m = np.full(n, 1.0 / n)
    rec, _, _ = O.pairs(pos, vel, ids, h, O.MODE_FP64, (0, s0, 1.0, 1), m[0], 0.02, 5, 1, 0, ev_cap=n * 200)
    assert rec.size > 5000
    cur = vel.copy()
    worst, checked = 0.0, 0
    for e in rec[: 6000]:
        i, j = int(e["i"]), int(e["j"])
        u = cur[:, i] - cur[:, j]
        un = np.linalg.norm(u)
        loc = np.array([e]).copy(); loc["i"], loc["j"] = 0, 1
        v2, _, _ = O.apply_drag(loc, m[[i, j]], (0, s0, 1.0), cur[:, [i, j]])
        u2 = v2[:, 0] - v2[:, 1]
        assert np.linalg.norm(u2) == pytest.approx(un, rel=1e-14)                      # energy
        scale = np.linalg.norm(cur[:, i]) + np.linalg.norm(cur[:, j])
        assert np.allclose(v2.sum(axis=1), cur[:, [i, j]].sum(axis=1), rtol=0, atol=4e-15 * scale)  # momentum
        sin2 = np.sum(np.cross(u, u2) ** 2) / un ** 4                                # sin^2(alpha)
        P = s0 * un * e["P"]                                                          # isotropic probability
        if P >= 1e-5:                     # smaller turns drown in the rounding of reading them back
            worst = max(worst, abs(1.5 * sin2 - P * (1.0 - P / 6.0)) / P)
            checked += 1
        cur[:, [i, j]] = v2
    assert checked > 1000 and worst < 1e-6


def test_drag_mean_change_and_azimuthal_isotropy():
    # many copies of one pair (same u and G, different azimuth words)
    copies, s0, G = 40000, 1.0, 0.09
    rng = np.random.default_rng(44)
    u = np.array([0.3, -1.1, 0.7]); un = np.linalg.norm(u)
    vel = np.zeros((3, 2 * copies)); vel[:, 0::2] = (0.5 * u)[:, None]; vel[:, 1::2] = (-0.5 * u)[:, None]
    rec = np.zeros(copies, O.EVENT_DTYPE)
    rec["i"] = np.arange(copies) * 2; rec["j"] = rec["i"] + 1
    rec["key"] = np.arange(copies); rec["P"] = G; rec["u"] = -1.0
    rec["x1"] = rng.integers(0, 2 ** 32, copies, dtype=np.uint64).astype(np.uint32)
    rec["x2"] = rng.integers(0, 2 ** 32, copies, dtype=np.uint64).astype(np.uint32)
    v1, _, D = O.apply_drag(rec, np.ones(2 * copies), (0, s0, 1.0), vel)
    up = v1[:, 0::2] - v1[:, 1::2]
    Dv = s0 * un * G / 3.0
    assert np.allclose(D, Dv)
    sa2 = Dv * (2.0 - Dv)
    noise = math.sqrt(sa2 / copies) * un
    assert np.all(np.abs(up.mean(axis=1) - (1.0 - Dv) * u) < 5 * noise)             # the drag
    # the test's own frame of the normal plane
    a = np.cross(u, [1.0, 0.0, 0.0]); a /= np.linalg.norm(a)
    b = np.cross(u / un, a)
    pa, pb = a @ up, b @ up
    want = un ** 2 * sa2 / 2.0
    assert abs(np.mean(pa ** 2) / want - 1) < 0.03 and abs(np.mean(pb ** 2) / want - 1) < 0.03
    assert abs(np.mean(pa * pb)) < 0.03 * want and abs(np.mean(pa)) < 5 * noise


def test_drag_rate_closed_form_uniform_maxwellian_box():
    # sum over partners of (3/2) sin^2(alpha) = 3D - 3D^2/2 per unit time against
    # rho (sigma_V/m) <|v_i - v_j|> (N-1)/N for interior particles (fixed h)
    n, hval, s0, dt = 30000, 0.06, 2.0, 1e-3
    pos, vel, ids, h = _box(n, 45, hval)
    rec, _, _ = O.pairs(pos, vel, ids, h, O.MODE_FP64, (0, s0, 1.0, 1), 1.0 / n, dt, 8, 0, 0, ev_cap=n * 200)
    _, _, D = O.apply_drag(rec, np.full(n, 1.0 / n), (0, s0, 1.0), vel)
    relax = 3.0 * D - 1.5 * D * D
    S = np.zeros(n)
    np.add.at(S, rec["i"], relax); np.add.at(S, rec["j"], relax)
    inner = np.all((pos > 2 * hval) & (pos < 1 - 2 * hval), axis=0)
    expect = s0 * 1.0 * 4.0 / math.sqrt(math.pi) * (n - 1) / n
    got = S[inner].mean() / dt
    sem = S[inner].std() / math.sqrt(inner.sum()) / dt
    assert abs(got / expect - 1) < 4e-3 and abs(got - expect) < 6 * sem * 3


def test_zero_cross_section_drag_is_identity():
    n = 2000
    pos, vel, ids, h = _box(n, 46, 0.1)
    rec, _, _ = O.pairs(pos, vel, ids, h, O.MODE_FP64, (0, 0.0, 1.0, 1), 1.0 / n, 0.01, 1, 0, 0, ev_cap=n * 200)
    assert rec.size > 1000
    v1, dE, D = O.apply_drag(rec, np.full(n, 1.0 / n), (0, 0.0, 1.0), vel)
    assert np.array_equal(v1, vel) and np.all(dE == 0.0) and np.all(D == 0.0)


def test_oracle_step_applies_drag_and_isotropic_halos_side_by_side():
    # a batch mixing the two angular dependences: each halo follows its own rule
    a, b = ics.hernquist(1200, 47), ics.hernquist(900, 48)
    bt = ics.batch([a, b])
    vel = bt.vel.astype(np.float32).astype(np.float64)
    xs = [(0, 10.0, 1.0, 1), (0, 10.0, 1.0)]
    r = O.step(bt.pos, vel, bt.ids, bt.offsets, [32, 32], bt.mass, xs, [0.05, 0.2], 6, 0, O.MODE_MIXED)
    n0 = int(bt.offsets[1])
    ev0 = r["events"][r["events"]["key"] >> np.uint64(54) == 0]
    v_drag, _, _ = O.apply_drag(ev0, np.repeat(bt.mass, np.diff(bt.offsets)), xs[0], vel)
    assert np.array_equal(r["vel_out"][:, :n0], v_drag[:, :n0])
    assert r["stats"][0]["n_events"] == r["stats"][0]["n_pairs"] > 1000
    assert 0 < r["stats"][1]["n_events"] < r["stats"][1]["n_pairs"]

"""Pins of the oracle's kNN, pair pass and scatter against brute force, a
library kNN, closed forms and invariants (no GPU).

Paper passages: Sect. 2 (kernel size set by the next N_ngb neighbours;
explicit energy and momentum conservation), Eq. hDl (h is the radius of the
sphere holding N_ngb particles), Sect. 3.5 (Lambda in the interaction
probability), Sect. 5 (conservation does not depend on the probability)."""
import math

import numpy as np
import pytest
from scipy import spatial, special, stats

from oracle import oracle as O
from paper_2506_06269_gb300 import ics


# ---------------------------------------------------------------- kNN
@pytest.mark.parametrize("k", [1, 16, 32, 64, 128])
def test_knn_tree_equals_brute_force(k):
    h = ics.hernquist(3000, 1)
    for mode in (O.MODE_MIXED, O.MODE_FP64):
        hb, db, nb = O.knn(h.pos, h.ids, k, mode, brute=True, want_nbrs=True)
        hg, dg, ng = O.knn(h.pos, h.ids, k, mode, brute=False, want_nbrs=True)
        assert np.array_equal(hb, hg) and np.array_equal(db, dg) and np.array_equal(nb, ng)


@pytest.mark.parametrize("k", [16, 64])
def test_knn_tree_equals_brute_force_on_a_cored_halo(k):
    # 10^3 rho_s core of radius 0.05 inside NFW: a density contrast of ~10^6
    # between the core and the truncation radius, where a wrong box skip shows
    h = ics.cored_nfw(4000, 12)
    for mode in (O.MODE_MIXED, O.MODE_FP64):
        hb, db, nb = O.knn(h.pos, h.ids, k, mode, brute=True, want_nbrs=True)
        ht, dt_, nt = O.knn(h.pos, h.ids, k, mode, brute=False, want_nbrs=True)
        assert np.array_equal(hb, ht) and np.array_equal(db, dt_) and np.array_equal(nb, nt)


def test_pair_pass_finds_every_in_range_pair_of_a_cored_halo():
    # The pair pass (k-d tree) against a brute-force list of the in-range pairs,
    # canonical d2 < RN32(RN32(h_i + h_j)^2) over all N(N-1)/2 pairs (mixed
    # form).  A huge cross-section makes P > 1 for every in-range pair with a
    # nonzero overlap, so the event set is that list (less pairs whose FP64
    # distance rounds onto the support edge, where Lambda is exactly zero).
    h = ics.cored_nfw(3000, 13)
    n = h.n
    vel = h.vel.astype(np.float32).astype(np.float64)
    hh, _, _ = O.knn(h.pos, h.ids, 32, O.MODE_MIXED)
    ev, st, _ = O.pairs(h.pos, vel, h.ids, hh, O.MODE_MIXED, (0, 1e300, 1.0), h.mass, 1.0, 1, 0, 0,
                        ev_cap=n * n // 2)
    got = {(int(e["key"]) >> 27 & ((1 << 27) - 1), int(e["key"]) & ((1 << 27) - 1)) for e in ev}
    order, _, _, _, _ = O.geometry(h.pos)
    rank = np.empty(n, np.int64); rank[order] = np.arange(n)
    ii, jj = np.triu_indices(n, 1)
    lower_first = rank[ii] // 32 <= rank[jj] // 32          # each pair in its lower leaf's frame
    qi, qj = np.where(lower_first, ii, jj), np.where(lower_first, jj, ii)
    d2 = O.d2_mixed(h.pos, qi, qj)
    hs = hh.astype(np.float32)[ii] + hh.astype(np.float32)[jj]
    inr = d2 < hs * hs
    ids = h.ids.astype(np.int64)
    want = {(min(a, b), max(a, b)): (a_, b_)
            for a, b, a_, b_ in zip(ids[ii[inr]], ids[jj[inr]], ii[inr], jj[inr])}
    assert st["n_pairs"] == len(want) > 30000
    assert got <= set(want)
    for key in set(want) - got:
        a_, b_ = want[key]
        d = np.linalg.norm(h.pos[:, a_] - h.pos[:, b_])
        assert d >= (hh[a_] + hh[b_]) * (1 - 1e-6), key


def test_knn_sample_equals_knn_for_every_k():
    # the sampled entry (all N_ngb up to k from one search) against separate calls
    h = ics.nfw(5000, 4)
    q = np.random.default_rng(3).choice(h.n, 200, replace=False)
    for mode in (O.MODE_MIXED, O.MODE_FP64):
        hs = O.knn_sample(h.pos, h.ids, 64, q, mode)
        for k in (1, 16, 33, 64):
            hk, _, _ = O.knn(h.pos, h.ids, k, mode)
            assert np.array_equal(hs[:, k - 1], hk[q]), (mode, k)


def test_knn_matches_library_kdtree():
    # exact FP64 kNN distances from scipy's kd-tree (its own arithmetic)
    h = ics.nfw(6000, 2)
    k = 32
    tree = spatial.cKDTree(h.pos.T)
    dist, idx = tree.query(h.pos.T, k=k + 1)
    h64, _, nb64 = O.knn(h.pos, h.ids, k, O.MODE_FP64, want_nbrs=True)
    assert np.allclose(h64, dist[:, k], rtol=1e-14, atol=0)
    # neighbour sets agree except where the k-th and (k+1)-th are a near tie
    clear = (dist[:, k + 0] < dist[:, k] * (1 + 1e-12)) & True
    gap = np.array([np.partition(np.linalg.norm(h.pos.T - h.pos.T[i], axis=1), k + 1)[k + 1]
                    for i in range(0, 6000, 97)])
    sel = np.arange(0, 6000, 97)
    for t, i in enumerate(sel):
        if gap[t] > dist[i, k] * (1 + 1e-12):
            assert set(nb64[i]) == set(h.ids[idx[i, 1:]])
    # mixed form: FP32 canonical distances, same h to FP32 rounding
    h32, _, _ = O.knn(h.pos, h.ids, k, O.MODE_MIXED)
    assert np.all(np.abs(h32 - h64) <= 4e-6 * h64)
    assert clear.any()


def test_knn_uniform_box_mean_h_matches_hdl_reading():
    # Eq. hDl reading: h is the radius of the sphere holding N_ngb particles.
    # For a Poisson field the k-th neighbour distance has
    # E[r_k] = (3/(4 pi n))^(1/3) Gamma(k+1/3)/Gamma(k).
    n, k = 40000, 32
    b = ics.uniform_box(n, 7)
    hh, _, _ = O.knn(b.pos, b.ids, k, O.MODE_MIXED)
    inner = np.all((b.pos > 0.15) & (b.pos < 0.85), axis=0)
    expect = (3.0 / (4 * math.pi * n)) ** (1 / 3) * math.exp(special.gammaln(k + 1 / 3) - special.gammaln(k))
    got = hh[inner].mean()
    sem = hh[inner].std() / math.sqrt(inner.sum())
    assert abs(got - expect) < 6 * sem


def test_knn_rejects_too_few_particles():
    b = ics.uniform_box(10, 1)
    with pytest.raises(ValueError):
        O.knn(b.pos, b.ids, 10, O.MODE_MIXED)
    hh, _, _ = O.knn(b.pos, b.ids, 9, O.MODE_MIXED)
    assert np.all(np.isfinite(hh))


def test_canonical_geometry_offsets():
    h = ics.nfw(5000, 4)
    order, off, cell, E, Og = O.geometry(h.pos)
    n = h.n
    assert sorted(order.tolist()) == list(range(n))
    ext = (h.pos.max(1) - h.pos.min(1)).max()
    assert 2.0 ** E > ext >= 2.0 ** (E - 1)
    # cube [O, O + 2^(E+1)) holds the halo, O a multiple of 2^E
    assert np.all(h.pos >= Og[:, None]) and np.all(h.pos < Og[:, None] + 2.0 ** (E + 1))
    assert np.all(np.mod(Og, 2.0 ** E) == 0)
    fine = 2.0 ** (E + 1 - 17)
    assert np.all(np.mod(cell.astype(np.float64), fine) == 0)
    leaf = np.empty(n, np.int64)
    leaf[order] = np.arange(n) // 32
    Cabs = Og[None, :] + cell[leaf].astype(np.float64)
    # offsets are the correctly rounded FP32 values of x - (O + c)
    assert np.array_equal(off, (h.pos - Cabs.T).astype(np.float32))
    # and stay within the leaf's extent (frame next to the leaf)
    for L in range(0, len(cell), 7):
        mem = order[L * 32:(L + 1) * 32]
        span = (h.pos[:, mem].max(1) - h.pos[:, mem].min(1)).max()
        assert np.abs(off[:, mem]).max() <= span * (1 + 1e-6) + fine


def test_canonical_distance_error_bound():
    h = ics.nfw(4000, 5)
    rng = np.random.default_rng(0)
    qi = rng.integers(0, h.n, 20000).astype(np.uint32)
    qj = rng.integers(0, h.n, 20000).astype(np.uint32)
    d2 = O.d2_mixed(h.pos, qi, qj).astype(np.float64)
    ex = ((h.pos[:, qj] - h.pos[:, qi]) ** 2).sum(0)
    _, _, _, E, _ = O.geometry(h.pos)
    tol = 2.0 ** (E + 1 - 22)
    assert np.all(np.abs(np.sqrt(d2) - np.sqrt(ex)) <= 1e-6 * np.sqrt(ex) + tol)
    # same leaf: exactly symmetric
    order, _, _, _, _ = O.geometry(h.pos)
    a, b = order[:32], order[:32][::-1]
    assert np.array_equal(O.d2_mixed(h.pos, a, b), O.d2_mixed(h.pos, b, a))


# ---------------------------------------------------------------- pair pass
def _box_fixed_h(n, seed, hval, sigma_v=1.0):
    b = ics.uniform_box(n, seed, sigma_v=sigma_v)
    vel32 = b.vel.astype(np.float32).astype(np.float64)
    return b, vel32, np.full(n, np.float64(np.float32(hval)))


def test_rate_closed_form_uniform_maxwellian_box():
    # Expected sum_j P_ij for an interior particle with a fixed kernel size:
    # (sigma/m) dt rho <|v_i - v_j|> (N-1)/N, since int Lambda d^3x = 1 and the
    # relative speed of two Maxwellian particles has mean 4 sigma_v / sqrt(pi).
    n, hval, s0, dt = 30000, 0.06, 2.0, 1e-3
    b, vel, hh = _box_fixed_h(n, 21, hval)
    ev, st, sump = O.pairs(b.pos, vel, b.ids, hh, O.MODE_FP64, (0, s0, 1.0), b.mass, dt, 99, 0, 0)
    inner = np.all((b.pos > 2 * hval) & (b.pos < 1 - 2 * hval), axis=0)
    rho = 1.0
    expect = s0 * dt * rho * 4.0 / math.sqrt(math.pi) * (n - 1) / n
    got = sump[inner].mean()
    sem = sump[inner].std() / math.sqrt(inner.sum())
    assert abs(got / expect - 1) < 4e-3 and abs(got - expect) < 6 * sem * 3
    # realised events: Poisson around the summed probabilities
    lam_tot = 0.5 * sump.sum()
    assert abs(st["n_events"] - lam_tot) < 5 * math.sqrt(lam_tot)
    # every unordered in-range pair once: compare with a kd-tree pair count
    tree = spatial.cKDTree(b.pos.T)
    npairs = len(tree.query_pairs(2 * hval * (1 - 1e-6)))
    assert abs(st["n_pairs"] - npairs) <= len(tree.query_pairs(2 * hval * (1 + 1e-6))) - npairs


def test_zero_cross_section_leaves_velocities_unchanged():
    h = ics.hernquist(2000, 3)
    vel = h.vel.astype(np.float32).astype(np.float64)
    offs = np.array([0, h.n])
    res = O.step(h.pos, vel, h.ids, offs, [32], [h.mass], [(0, 0.0, 1.0)], [1e-3], 5, 0)
    assert res["events"].size == 0
    assert np.array_equal(res["vel_out"], vel)


def test_event_keys_sorted_unique_and_draws_below_p():
    h = ics.hernquist(4000, 8)
    vel = h.vel.astype(np.float32).astype(np.float64)
    offs = np.array([0, h.n])
    res = O.step(h.pos, vel, h.ids, offs, [32], [h.mass], [(0, 10.0, 1.0)], [0.25], 1, 3)
    ev = res["events"]
    assert ev.size > 50
    assert np.all(np.diff(ev["key"].astype(np.int64)) > 0)
    assert np.all(ev["u"] < ev["P"])
    # u is word 0 of Philox at (step, min id, max id, halo), key = seed
    for e in ev[:20]:
        a, b = int(h.ids[e["i"]]), int(h.ids[e["j"]])
        assert a < b
        x = O.philox4x32_10([3, a, b, 0], [1, 0])
        assert e["u"] == x[0] * 2.0 ** -32 and e["x1"] == x[1] and e["x2"] == x[2]


def test_pair_mask_selects_exactly_the_masked_pairs():
    # the sampled pair pass used at full size evaluates the same pairs, with the
    # same draws and probabilities, as the full pass restricted to the sample
    h = ics.hernquist(4000, 9)
    vel = h.vel.astype(np.float32).astype(np.float64)
    hh, _, _ = O.knn(h.pos, h.ids, 32, O.MODE_MIXED)
    full, _, _ = O.pairs(h.pos, vel, h.ids, hh, O.MODE_MIXED, (0, 10.0, 1.0), h.mass, 0.25, 1, 3, 0)
    mask = np.zeros(h.n, bool)
    mask[np.random.default_rng(2).choice(h.n, 600, replace=False)] = True
    part, _, _ = O.pairs(h.pos, vel, h.ids, hh, O.MODE_MIXED, (0, 10.0, 1.0), h.mass, 0.25, 1, 3, 0, mask=mask)
    want = full[mask[full["i"]] | mask[full["j"]]]
    assert want.size > 10 and want.size < full.size
    assert np.array_equal(part, want)


# ---------------------------------------------------------------- scatter
def _random_events(n_part, n_ev, seed, chain=False):
    rng = np.random.default_rng(seed)
    ev = np.zeros(n_ev, O.EVENT_DTYPE)
    i = rng.integers(0, n_part, n_ev)
    j = (i + 1 + rng.integers(0, n_part - 1, n_ev)) % n_part
    ev["i"], ev["j"] = np.minimum(i, j), np.maximum(i, j)
    ev["key"] = (ev["i"].astype(np.uint64) << np.uint64(27)) | ev["j"].astype(np.uint64)
    w = np.array([O.philox4x32_10([s, 1, 2, 3], [seed, 9]) for s in range(n_ev)], dtype=np.uint32)
    ev["x1"], ev["x2"] = w[:, 1], w[:, 2]
    return np.sort(ev, order="key")


def test_per_event_conservation_and_multi_hit_chains():
    rng = np.random.default_rng(2)
    n = 50
    vel = rng.standard_normal((3, n))
    m = np.full(n, 0.02)
    ev = _random_events(n, 400, 4)          # dense: every particle hit many times
    vout, dE = O.apply_events(ev, m, vel)
    p0, p1 = (m * vel).sum(1), (m * vout).sum(1)
    e0, e1 = 0.5 * (m * vel ** 2).sum(), 0.5 * (m * vout ** 2).sum()
    scale = 0.5 * (m * vel ** 2).sum()
    # holds only if every event starts from the *current* velocities
    assert np.all(np.abs(p1 - p0) < 1e-13 * np.abs(m * vel).sum())
    assert abs(e1 - e0) < 1e-13 * scale
    assert np.all(np.abs(dE) < 1e-14 * scale * 10)


def test_unequal_masses_conserve_pair_energy_and_momentum():
    rng = np.random.default_rng(6)
    vel = rng.standard_normal((3, 2))
    m = np.array([0.3, 1.7])
    ev = _random_events(2, 1, 1)
    vout, _ = O.apply_events(ev, m, vel)
    assert np.allclose((m * vout).sum(1), (m * vel).sum(1), rtol=0, atol=1e-15)
    assert 0.5 * (m * vout ** 2).sum() == pytest.approx(0.5 * (m * vel ** 2).sum(), rel=1e-15)
    # relative speed is preserved (elastic), direction re-drawn
    assert np.linalg.norm(vout[:, 0] - vout[:, 1]) == pytest.approx(np.linalg.norm(vel[:, 0] - vel[:, 1]), rel=1e-14)


def test_isotropy_chi_square():
    # post-scatter CM-frame directions over many independent events
    n_ev = 60000
    rng = np.random.default_rng(12)
    vel = rng.standard_normal((3, 2 * n_ev))
    m = np.ones(2 * n_ev)
    ev = np.zeros(n_ev, O.EVENT_DTYPE)
    ev["i"] = np.arange(0, 2 * n_ev, 2); ev["j"] = ev["i"] + 1
    ev["key"] = np.arange(n_ev, dtype=np.uint64)
    w = rng.integers(0, 2 ** 32, (n_ev, 2), dtype=np.uint64).astype(np.uint32)
    ev["x1"], ev["x2"] = w[:, 0], w[:, 1]
    vout, _ = O.apply_events(ev, m, vel)
    rel = vout[:, ev["i"]] - vout[:, ev["j"]]
    nh = rel / np.linalg.norm(rel, axis=0)
    ct = nh[2]
    phi = np.mod(np.arctan2(nh[1], nh[0]), 2 * math.pi)
    for x, lo, hi in ((ct, -1, 1), (phi, 0, 2 * math.pi)):
        cnt, _ = np.histogram(x, bins=20, range=(lo, hi))
        p = stats.chisquare(cnt).pvalue
        assert p > 1e-3
    # and independent of the incoming direction
    inc = (vel[:, ev["i"]] - vel[:, ev["j"]])
    inc /= np.linalg.norm(inc, axis=0)
    assert abs(np.mean((inc * nh).sum(0))) < 5 / math.sqrt(n_ev)


# ---------------------------------------------------------------- local diagnostics
def test_local_density_dispersion_and_ratios_in_a_uniform_box():
    # Sums over each particle's own kernel (itself included), recomputed from a
    # library neighbour search (scipy kd-tree) and numpy; the kernel W itself is
    # pinned in test_oracle_math.
    n = 20000
    b = ics.uniform_box(n, 31)
    rng = np.random.default_rng(4)
    hh = rng.uniform(0.06, 0.12, n)
    d = O.local_diag(b.pos, b.vel, hh, b.mass, 64, (1, 100.0, 0.3811))
    tree = spatial.cKDTree(b.pos.T)
    for i in rng.choice(n, 200, replace=False):
        nb = np.array(tree.query_ball_point(b.pos[:, i], hh[i]))
        r = np.linalg.norm(b.pos[:, nb] - b.pos[:, [i]], axis=0)
        nb, r = nb[r < hh[i]], r[r < hh[i]]
        wt = b.mass * np.array([O.kernel_w(x, hh[i]) for x in r])
        rho = wt.sum()
        mean = (wt * b.vel[:, nb]).sum(1) / rho
        nu = math.sqrt(max(((wt * (b.vel[:, nb] ** 2).sum(0)).sum() / rho - (mean ** 2).sum()) / 3.0, 0.0))
        assert d["rho"][i] == pytest.approx(rho, rel=1e-12)
        assert d["nu"][i] == pytest.approx(nu, rel=1e-9)
        assert d["sigma_eff"][i] == pytest.approx(O.sigma_eff(1, 100.0, 0.3811, nu), rel=1e-12)
    # statistics of a unit-density Maxwellian box (1-D dispersion 1): the interior
    # density is ~ 1 + m W(0, h) up to the ~1 % count fluctuation of the region;
    # a weighted variance of independent velocities has expectation
    # 1 - sum w^2 / (sum w)^2 per component
    inner = np.all((b.pos > 0.12) & (b.pos < 0.88), axis=0)
    self_term = b.mass * 8.0 / (math.pi * hh ** 3)
    assert abs((d["rho"] - self_term)[inner].mean() - 1.0) < 0.03
    pick = rng.choice(np.where(inner)[0], 2000, replace=False)
    expect = []
    for i in pick:
        nb = np.array(tree.query_ball_point(b.pos[:, i], hh[i]))
        r = np.linalg.norm(b.pos[:, nb] - b.pos[:, [i]], axis=0)
        wt = np.array([O.kernel_w(x, hh[i]) for x in r[r < hh[i]]])
        expect.append(1.0 - (wt ** 2).sum() / wt.sum() ** 2)
    assert (d["nu"][pick] ** 2).mean() == pytest.approx(np.mean(expect), rel=0.03)
    # h/l (Eq. hDl) is sqrt(2) rho sigma_eff/m times the kernel size of a sphere
    # holding N_ngb particles at density rho; Kn (Eq. knudsen_number) is the mean
    # free path 1/(rho sigma_eff/m) over the Jeans length nu / sqrt(4 pi G rho)
    r = d["rho"]; se = d["sigma_eff"]
    h_est = (3.0 * b.mass * 64 / (4.0 * math.pi * r)) ** (1.0 / 3.0)
    assert np.allclose(d["h_over_l"], math.sqrt(2.0) * r * se * h_est, rtol=1e-12)
    lam = 1.0 / (r * se)
    jeans = d["nu"] / np.sqrt(4.0 * math.pi * r)
    assert np.allclose(d["kn"], lam / jeans, rtol=1e-12)


def test_local_dispersion_vanishes_for_equal_velocities():
    b = ics.uniform_box(3000, 32)
    vel = np.tile(np.array([[0.3], [-1.2], [2.0]]), (1, b.n))
    d = O.local_diag(b.pos, vel, np.full(b.n, 0.2), b.mass, 32, (1, 100.0, 0.38))
    assert np.all(d["nu"] < 1e-7)
    # a particle alone in its kernel has the self term only
    lone = O.local_diag(np.array([[0.0, 5.0], [0.0, 5.0], [0.0, 5.0]]), np.zeros((3, 2)), np.array([1.0, 1.0]),
                        0.5, 1, (0, 1.0, 1.0))
    assert lone["rho"][0] == 0.5 * O.kernel_w(0.0, 1.0)

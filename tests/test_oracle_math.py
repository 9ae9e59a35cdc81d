"""Pins of the oracle's elementary pieces against what the paper and the
mathematics fix (no GPU).  Kernel: Sect. 2 (Monaghan spline); Lambda:
Sect. 3.5 (kernel-overlap geometric factor); sigma(v): Eq. vel_dep (Sect. 3.8);
draws: Philox4x32-10 from its published known-answer vectors."""
import math
import os

import numpy as np
import pytest
from scipy import integrate, stats

from oracle import oracle as O

GOLD = os.path.join(os.path.dirname(__file__), "golden")


# ---------------------------------------------------------------- Philox
def test_philox_known_answer_vectors():
    rows = [l.split() for l in open(os.path.join(GOLD, "philox4x32_10_kat.txt"))
            if l.strip() and not l.startswith("#")]
    assert len(rows) == 3
    for r in rows:
        v = [int(x, 16) for x in r]
        out = O.philox4x32_10(v[0:4], v[4:6])
        assert [int(x) for x in out] == v[6:10]


def test_philox_words_uniform():
    # 4 words x 20000 counters: each word uniform on [0, 2^32) (KS test)
    w = np.array([O.philox4x32_10([c, 7, 11, 0], [123, 456]) for c in range(20000)], dtype=np.float64)
    for col in range(4):
        p = stats.kstest(w[:, col] / 2.0 ** 32, "uniform").pvalue
        assert p > 1e-4


# ---------------------------------------------------------------- kernel W
def test_kernel_normalised_and_shape():
    for h in (0.3, 1.0, 2.5):
        val = integrate.quad(lambda r: 4 * math.pi * r * r * O.kernel_w(r, h), 0, h,
                             points=[0.5 * h], epsabs=0, epsrel=1e-13)[0]
        assert abs(val - 1.0) < 1e-12
        assert O.kernel_w(0.0, h) == pytest.approx(8.0 / (math.pi * h ** 3), rel=1e-15)
        assert O.kernel_w(h, h) == 0.0 and O.kernel_w(1.5 * h, h) == 0.0
        # continuity (value and slope) at q = 1/2
        e = 1e-7 * h
        assert O.kernel_w(0.5 * h - e, h) == pytest.approx(O.kernel_w(0.5 * h + e, h), rel=1e-5)
        s1 = (O.kernel_w(0.5 * h - e, h) - O.kernel_w(0.5 * h - 2 * e, h)) / e
        s2 = (O.kernel_w(0.5 * h + 2 * e, h) - O.kernel_w(0.5 * h + e, h)) / e
        assert s1 == pytest.approx(s2, rel=1e-4)


# ---------------------------------------------------------------- Lambda
def _lambda_breaks(hi, hj):
    c = [abs(a * hi + b * hj) for a in (0.5, 1.0, -0.5, -1.0) for b in (0.5, 1.0, -0.5, -1.0)]
    return sorted({x for x in c if 0 < x < hi + hj})


@pytest.mark.parametrize("hi,hj", [(1.0, 1.0), (1.0, 0.5), (0.3, 1.0), (1.0, 0.07), (2.0, 1.7)])
def test_lambda_integrates_to_one(hi, hj):
    # convolution of two unit-normalised kernels is unit-normalised
    f = lambda d: 4 * math.pi * d * d * O.lam(d, hi, hj)
    brk = [0.0] + _lambda_breaks(hi, hj) + [hi + hj]
    tot = 0.0
    for a, b in zip(brk[:-1], brk[1:]):
        tot += integrate.quad(f, a, b, epsabs=0, epsrel=1e-13, limit=200)[0]
    assert abs(tot - 1.0) < 1e-12


def test_lambda_symmetry_support_and_limits():
    rng = np.random.default_rng(3)
    for _ in range(200):
        hi, hj = rng.uniform(0.05, 2.0, 2)
        d = rng.uniform(0, hi + hj)
        a, b = O.lam(d, hi, hj), O.lam(d, hj, hi)
        assert a == pytest.approx(b, rel=1e-12, abs=1e-300)
        assert a >= 0.0
    assert O.lam(2.0, 1.0, 1.0) == 0.0 and O.lam(2.5, 1.0, 1.0) == 0.0
    # small second kernel -> Lambda(d) tends to W(d, h_i)  (O(eps^2) error)
    for d in (0.0, 0.1, 0.3, 0.49, 0.6, 0.9):
        assert O.lam(d, 1.0, 1e-4) == pytest.approx(O.kernel_w(d, 1.0), rel=2e-6, abs=1e-9)
    # continuity at d -> 0 (switch to the analytic limit)
    assert O.lam(1e-7, 1.0, 0.6) == pytest.approx(O.lam(0.0, 1.0, 0.6), rel=1e-9)


def test_lambda_zero_separation_closed_form():
    # Lambda(0; h, h) = int W^2 d^3x, closed form by symbolic integration
    sp = pytest.importorskip("sympy")
    r = sp.symbols("r", positive=True)
    n = 8 / sp.pi
    w1 = n * (1 - 6 * r ** 2 + 6 * r ** 3)
    w2 = n * 2 * (1 - r) ** 3
    exact = 4 * sp.pi * (sp.integrate(r ** 2 * w1 ** 2, (r, 0, sp.Rational(1, 2)))
                         + sp.integrate(r ** 2 * w2 ** 2, (r, sp.Rational(1, 2), 1)))
    val = float(sp.N(exact, 30))
    for h in (1.0, 0.25):
        assert O.lam(0.0, h, h) == pytest.approx(val / h ** 3, rel=1e-13)


def test_lambda_monte_carlo():
    # brute-force 3-D Monte Carlo of int W(|x|,h) W(|x-d e_z|,h) d^3x
    rng = np.random.default_rng(11)
    h, d = 1.0, 0.7
    n = 400_000
    pts = rng.uniform(-h, h, (n, 3))
    vol = (2 * h) ** 3
    r1 = np.linalg.norm(pts, axis=1)
    r2 = np.linalg.norm(pts - np.array([0, 0, d]), axis=1)
    wv = np.vectorize(O.kernel_w)
    vals = wv(r1, h) * wv(r2, h) * vol
    est, err = vals.mean(), vals.std() / math.sqrt(n)
    assert abs(O.lam(d, h, h) - est) < 5 * err


# ---------------------------------------------------------------- sigma(v)
def test_cross_section_law():
    s0, w = 100.0, 0.3811
    assert O.sigma(1, s0, w, 0.0) == s0
    assert O.sigma(1, s0, w, w) == pytest.approx(s0 / 4, rel=1e-15)
    assert O.sigma(1, s0, w, 3 * w) == pytest.approx(s0 / 100, rel=1e-15)
    assert O.sigma(0, 10.0, w, 5.0) == 10.0


# ---------------------------------------------------------------- exact sums
def test_exact_sum_matches_fsum():
    rng = np.random.default_rng(5)
    x = rng.standard_normal(20000) * 10.0 ** rng.integers(-20, 20, 20000)
    x = np.concatenate([x, -x[:5000] * (1 + 1e-16)])
    assert O.exact_sum(x) == math.fsum(x)
    vel = rng.standard_normal((3, 5000)).astype(np.float32).astype(np.float64)
    m = 1.0 / 5000
    em = O.energy_momentum(m, vel)
    terms = [(0.5 * m) * ((vel[0, i] * vel[0, i] + vel[1, i] * vel[1, i]) + vel[2, i] * vel[2, i])
             for i in range(5000)]
    assert em[0] == math.fsum(terms)
    for a in range(3):
        assert em[1 + a] == math.fsum(m * vel[a])


def test_sigma_eff_matches_its_definition():
    # App. C: <v^5 sigma_V(v)> / <v^5> over the relative-speed Maxwellian of two
    # particles of 1-D dispersion nu; evaluated here by scipy's adaptive
    # quadrature in the substituted variable t = v^2 / (4 nu^2)
    from scipy import integrate
    s0, w = 100.0, 0.3811
    assert O.sigma_eff(0, 7.5, w, 0.2) == 7.5
    for nu in (0.01, 0.1, 0.3811, 1.0, 3.0):
        a = 4.0 * nu * nu
        num = integrate.quad(lambda t: t ** 3 * math.exp(-t) / (1.0 + a * t / w ** 2) ** 2, 0, math.inf,
                             epsabs=0, epsrel=1e-13, limit=400)[0]
        want = s0 * num / 6.0
        assert O.sigma_eff(1, s0, w, nu) == pytest.approx(want, rel=1e-10), nu
    # limits: nu -> 0 recovers sigma(0) = s0; large nu falls like (w / 2nu)^4 * 2 / 6
    assert O.sigma_eff(1, s0, w, 1e-4) == pytest.approx(s0, rel=1e-5)
    nu = 200.0
    assert O.sigma_eff(1, s0, w, nu) == pytest.approx(s0 * (w * w / (4 * nu * nu)) ** 2 * 1.0 / 6.0, rel=1e-3)


def test_timestep_criterion_and_bins():
    # dt_i = tau dt / sum_j P_ij (expected scatterings per step = tau), bounded by
    # [dt_min, dt_max]; bin b: the largest dt_max / 2^b not above dt_i
    rng = np.random.default_rng(8)
    sp = 10.0 ** rng.uniform(-6, 1, 5000)
    sp[:7] = 0.0
    tau, dt, dmin, dmax, nb = 0.04, 1e-3, 1e-6, 4e-3, 4
    dto, bo = O.timestep(sp, tau, dt, dmin, dmax, nb)
    safe = np.where(sp > 0, sp, 1.0)
    free = (sp > 0) & (tau * dt / safe > dmin) & (tau * dt / safe < dmax)
    assert np.all(dto[free] * sp[free] == pytest.approx(tau * dt, rel=1e-14))
    assert np.all(dto[:7] == dmax) and dto.min() >= dmin and dto.max() <= dmax
    step = dmax / 2.0 ** bo
    top = bo < nb - 1
    assert np.all(step[top] <= dto[top]) and np.all((bo == 0) | (2 * step > dto))
    # a step longer than the criterion only where no smaller bin exists
    assert np.all(bo[step > dto] == nb - 1) and np.any(step > dto)

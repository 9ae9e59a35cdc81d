"""The rounding argument behind the mixed form's exact candidate filter.

In a warm-started kernel-size search every candidate is shifted exactly into
the query leaf's frame, and a candidate c is dropped for a group of queries when
the squared gap between c and the group's box, formed with every operation
rounded down, exceeds the largest bound of the group.  That is exact only if the
rounded-down gap never exceeds the canonical FP32 distance of c from any query q
in the box, d2 = RN(dz dz + RN(dy dy + RN(dx dx))) with dx = RN(c_x - q_x)
(reading C2').  Here both sides are evaluated in exact rational arithmetic with
explicit FP32 rounding, for random and for adversarial points: on the box's
faces, inside it, at binade edges and at tiny and equal offsets.
"""
from fractions import Fraction

import numpy as np
import pytest

F32 = np.float32


def _round32(x: Fraction, mode: str) -> Fraction:
    """x rounded to FP32: 'rn' to nearest (ties to even) or 'rd' downwards."""
    f = F32(float(x))                      # within an ulp or two of x
    while Fraction(float(f)) > x:
        f = np.nextafter(f, F32(-np.inf))
    lo = f                                 # largest FP32 <= x
    if mode == "rd" or Fraction(float(lo)) == x:
        return Fraction(float(lo))
    hi = np.nextafter(lo, F32(np.inf))
    dl, dh = x - Fraction(float(lo)), Fraction(float(hi)) - x
    if dl < dh:
        return Fraction(float(lo))
    if dh < dl:
        return Fraction(float(hi))
    even = lo if (int(np.frombuffer(lo.tobytes(), np.uint32)[0]) & 1) == 0 else hi
    return Fraction(float(even))


def _canonical_d2(c, q) -> Fraction:
    d = [_round32(Fraction(float(c[a])) - Fraction(float(q[a])), "rn") for a in range(3)]
    t = _round32(d[0] * d[0], "rn")
    t = _round32(d[1] * d[1] + t, "rn")        # fma: one rounding of the exact sum
    return _round32(d[2] * d[2] + t, "rn")


def _gap2_rd(c, lo, hi) -> Fraction:
    g = []
    for a in range(3):
        ca, la, ha = Fraction(float(c[a])), Fraction(float(lo[a])), Fraction(float(hi[a]))
        g.append(max(Fraction(0), _round32(la - ca, "rd"), _round32(ca - ha, "rd")))
    s = _round32(_round32(g[0] * g[0], "rd") + _round32(g[1] * g[1], "rd"), "rd")
    return _round32(s + _round32(g[2] * g[2], "rd"), "rd")


def _check_group(queries, cands):
    lo = queries.min(axis=0)
    hi = queries.max(axis=0)
    for c in cands:
        g2 = _gap2_rd(c, lo, hi)
        for q in queries:
            assert g2 <= _canonical_d2(c, q), (c, q, lo, hi)


def test_round32_agrees_with_numpy_rounding():
    rng = np.random.default_rng(1)
    for x in rng.normal(size=200) * 10.0 ** rng.integers(-8, 8, size=200):
        assert _round32(Fraction(float(x)), "rn") == Fraction(float(F32(x)))
        assert _round32(Fraction(float(x)), "rd") <= Fraction(float(x))


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_box_gap_rounded_down_bounds_canonical_distance(seed):
    rng = np.random.default_rng(seed)
    for _ in range(12):
        scale = F32(2.0 ** rng.integers(-12, 3))
        queries = (rng.uniform(-1, 1, size=(8, 3)) * scale).astype(F32)
        spread = F32(rng.uniform(0.5, 4.0))
        cands = (rng.uniform(-spread, spread, size=(24, 3)) * scale).astype(F32)
        _check_group(queries, cands)


def test_box_gap_bound_on_faces_edges_and_binade_boundaries():
    q = np.array([[0.5, 0.25, 1.0], [0.75, 0.125, 1.5], [0.5, 0.375, 2.0]], F32)
    lo, hi = q.min(axis=0), q.max(axis=0)
    up = lambda v: np.nextafter(F32(v), F32(np.inf))
    dn = lambda v: np.nextafter(F32(v), F32(-np.inf))
    cands = np.array([
        lo, hi, (lo + hi) / 2,                                   # on a corner, the other, inside
        [dn(lo[0]), lo[1], lo[2]], [up(hi[0]), hi[1], hi[2]],    # one ulp outside a face
        [dn(dn(lo[0])), dn(lo[1]), up(hi[2])],                   # just outside an edge
        [1.0, 0.5, 2.0], [dn(1.0), dn(0.5), up(2.0)],            # binade boundaries
        [0.5, 0.25, 1.0 + 2.0 ** -20], [-0.5, -0.25, -1.0],      # tiny offset, far side
    ], F32)
    _check_group(q, cands)
    # a single query: the box is a point and the gap is the distance rounded down
    _check_group(q[:1], cands)

"""Pins of the oracle's reflecting boundary (no GPU).  Sect. 2 keeps the
isolated halos inside a sphere that turns outward-moving particles back
without changing the energy; the oracle mirrors the velocity in the sphere's
tangent plane.  Checked here with numpy geometry written apart from it: the
speed is kept, the radial component flips, the tangential part (the cross
product with the normal) is unchanged, everything inside or moving inwards is
untouched, and a second application changes nothing."""
import numpy as np

from oracle import oracle as O


def _state(n=4000, seed=5):
    rng = np.random.default_rng(seed)
    pos = rng.normal(0.0, 1.0, (3, n)) * rng.uniform(0.2, 3.0, n)
    vel = rng.normal(0.0, 1.0, (3, n))
    return pos, vel


def test_reflection_keeps_speed_and_flips_the_radial_part():
    c, rb = np.array([0.1, -0.2, 0.05]), 1.5
    pos, vel = _state()
    out = O.reflect(pos, vel, c, rb)
    d = pos - c[:, None]
    r = np.linalg.norm(d, axis=0)
    nrm = d / r
    vn = (vel * nrm).sum(0)
    hit = (r > rb) & (vn > 0)
    assert 200 < hit.sum() < len(r) - 200
    np.testing.assert_allclose(np.linalg.norm(out, axis=0), np.linalg.norm(vel, axis=0), rtol=1e-15)
    np.testing.assert_allclose((out * nrm).sum(0)[hit], -vn[hit], rtol=1e-13, atol=1e-15)
    np.testing.assert_allclose(np.cross(out.T, nrm.T)[hit], np.cross(vel.T, nrm.T)[hit], rtol=1e-13, atol=1e-15)
    assert np.array_equal(out[:, ~hit], vel[:, ~hit])
    assert np.all((out * nrm).sum(0)[r > rb] <= 0)
    assert np.array_equal(O.reflect(pos, out, c, rb), out)


def test_radial_motion_is_reversed_and_no_boundary_is_a_no_op():
    pos = np.array([[3.0, 0.0, -2.0], [0.0, 4.0, 2.0], [0.0, 0.0, 1.0]])
    vel = pos * np.array([0.5, 2.0, 1.0])                  # purely radial, outwards
    out = O.reflect(pos, vel, (0.0, 0.0, 0.0), 2.5)
    np.testing.assert_allclose(out, -vel, rtol=1e-15)
    assert np.array_equal(O.reflect(pos, vel, (0.0, 0.0, 0.0), 0.0), vel)
    assert np.array_equal(O.reflect(pos, -vel, (0.0, 0.0, 0.0), 2.5), -vel)

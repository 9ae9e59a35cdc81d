"""Seeded synthetic initial conditions (halos) for the SIDM scattering pass.

This module is shared by the tests, ``bench.py`` and ``smoke()``: it draws
particle positions, velocities and ids and holds none of the scattering
method's arithmetic (no kernel, no overlap factor, no probability, no draw).

Profiles (code units, G = 1, total mass inside the truncation radius = 1):

* Hernquist, scale radius a = 1, truncated at 20 a, radii by the inverse CDF
  ``r = a sqrt(u) / (1 - sqrt(u))`` with ``u`` in ``[0, (20/21)^2)``.
* NFW, scale radius r_s = 1, truncated at ``r_cut`` (10 r_s by default); the
  paper samples its NFW halo up to 10 or 15 r_s (Sect. 2) -- the radii come
  from a tabulated inverse of M(<r).
* Cored: a King-like core ``rho_c (1 + (r/r_c)^2)^(-3/2)`` with r_c = 0.05 r_s
  and rho_c = 1e3 rho_s, joined to the NFW profile where the two cross
  (continuous density), truncated at 10 r_s.
* Uniform box: positions uniform in ``[0, L)^3``, Maxwellian velocities with a
  fixed one-dimensional dispersion.

The satellite set-up of Sect. 4.1 (a Milky-Way-like host of six analytic parts
and the satellite's initial position and velocity) is given in the paper in
kpc, M_sun and km/s; ``milky_way_host`` and ``satellite_orbit`` convert it to
the code units of the NFW halo above, read as the paper's halo of Sect. 2
(rho_0 = 4.42e7 M_sun/kpc^3, r_s = 1.28 kpc): length unit r_s, mass unit the
mass inside ``r_cut``, G = 1.

Velocities of the halos are isotropic Maxwellian with the local Jeans
dispersion of the *untruncated* profile,
``sigma_r^2(r) = (1/rho) int_r^inf rho(r') M(r') / r'^2 dr'``, evaluated by
FP64 quadrature on a logarithmic grid.

Particles of one halo get ids ``0 .. N_h-1`` (unique within the halo) and the
input order is shuffled, so that nothing downstream can rely on ids matching
array positions.
"""
from __future__ import annotations

from dataclasses import dataclass, field
import functools
import math

import numpy as np
from scipy import integrate

__all__ = [
    "Halo", "Batch", "hernquist", "nfw", "cored_nfw", "uniform_box",
    "batch", "nfw_vmax", "NFW_RHO_S", "satellite_units", "milky_way_host", "satellite_orbit",
]

# NFW normalisation: mass inside 10 r_s equals 1.
NFW_RHO_S = 1.0 / (4.0 * math.pi * (math.log(11.0) - 10.0 / 11.0))


@dataclass
class Halo:
    """One halo: SoA FP64 positions/velocities [3][N], u32 ids, particle mass."""
    pos: np.ndarray          # float64 [3, N]
    vel: np.ndarray          # float64 [3, N]
    ids: np.ndarray          # uint32 [N]
    mass: float              # mass of one particle
    name: str = ""
    meta: dict = field(default_factory=dict)

    @property
    def n(self) -> int:
        return int(self.pos.shape[1])


@dataclass
class Batch:
    """Several halos concatenated: offsets[h] .. offsets[h+1] is halo h."""
    pos: np.ndarray          # float64 [3, N]
    vel: np.ndarray          # float64 [3, N]
    ids: np.ndarray          # uint32 [N]
    offsets: np.ndarray      # int64 [H+1]
    mass: np.ndarray         # float64 [H]
    halos: list

    @property
    def n(self) -> int:
        return int(self.pos.shape[1])

    @property
    def n_halos(self) -> int:
        return int(len(self.offsets) - 1)


def _isotropic(rng: np.random.Generator, r: np.ndarray) -> np.ndarray:
    """Points at radii r with uniformly distributed directions, [3, N]."""
    n = r.shape[0]
    mu = rng.uniform(-1.0, 1.0, n)
    phi = rng.uniform(0.0, 2.0 * math.pi, n)
    s = np.sqrt(np.maximum(0.0, 1.0 - mu * mu))
    return np.stack([r * s * np.cos(phi), r * s * np.sin(phi), r * mu])


def _jeans_sigma(rho, mass, r_eval: np.ndarray, r_max: float = 1e6) -> np.ndarray:
    """Isotropic Jeans dispersion sigma_r(r) of an untruncated profile (G=1).

    sigma_r^2(r) = (1/rho(r)) * int_r^inf rho(s) M(s)/s^2 ds, tabulated on a
    log grid with Gauss-Kronrod quadrature per interval and interpolated in
    log r.
    """
    lo = max(float(np.min(r_eval)) * 0.5, 1e-7)
    grid = np.geomspace(lo, r_max, 1200)
    f = lambda s: rho(s) * mass(s) / (s * s)
    seg = np.array([integrate.quad(f, a, b, limit=200, epsabs=0.0, epsrel=1e-11)[0]
                    for a, b in zip(grid[:-1], grid[1:])])
    tail = np.concatenate([np.cumsum(seg[::-1])[::-1], [0.0]])
    sig2 = tail / np.array([rho(s) for s in grid])
    out = np.exp(np.interp(np.log(r_eval), np.log(grid), np.log(np.maximum(sig2, 1e-300))))
    return np.sqrt(out)


def _finish(rng, r, sigma, name, meta) -> Halo:
    n = r.shape[0]
    pos = _isotropic(rng, r)
    vel = rng.standard_normal((3, n)) * sigma[None, :]
    perm = rng.permutation(n)
    ids = np.arange(n, dtype=np.uint32)
    return Halo(pos=np.ascontiguousarray(pos[:, perm]),
                vel=np.ascontiguousarray(vel[:, perm]),
                ids=np.ascontiguousarray(ids[perm]),
                mass=1.0 / n, name=name, meta=meta)


def hernquist(n: int, seed: int, r_trunc: float = 20.0) -> Halo:
    """Hernquist halo, a = M = G = 1, truncated at r_trunc, mass 1 inside."""
    rng = np.random.default_rng(seed)
    umax = (r_trunc / (r_trunc + 1.0)) ** 2
    u = rng.uniform(0.0, umax, n)
    su = np.sqrt(u)
    r = su / (1.0 - su)
    rho = lambda s: 1.0 / (2.0 * math.pi) / (s * (1.0 + s) ** 3)
    mass = lambda s: s * s / (1.0 + s) ** 2
    sigma = _jeans_sigma(rho, mass, np.maximum(r, 1e-6))
    return _finish(rng, r, sigma, "hernquist", {"r_trunc": r_trunc})


def _nfw_mass(r):
    return 4.0 * math.pi * NFW_RHO_S * (np.log1p(r) - r / (1.0 + r))


def nfw_vmax() -> float:
    """Maximum circular velocity of the normalised NFW halo (at r ~ 2.163 r_s)."""
    r = np.linspace(1.5, 3.0, 20001)
    return float(np.sqrt(np.max(_nfw_mass(r) / r)))


def _sample_table(rng, n, r_grid, m_grid):
    u = rng.uniform(m_grid[0], m_grid[-1], n)
    return np.interp(u, m_grid, r_grid)


@functools.lru_cache(maxsize=None)
def _nfw_tables(r_cut: float):
    """Inverse-CDF table and Jeans dispersion table of the NFW profile (cached)."""
    r_grid = np.concatenate([[0.0], np.geomspace(1e-7, r_cut, 200001)])
    m_grid = _nfw_mass(r_grid)
    rho = lambda s: NFW_RHO_S / (s * (1.0 + s) ** 2)
    mass = lambda s: float(_nfw_mass(np.array(s)))
    r_sig = np.geomspace(1e-7, r_cut, 4001)
    sig = _jeans_sigma(rho, mass, r_sig)
    return r_grid, m_grid, r_sig, sig


def nfw(n: int, seed: int, r_cut: float = 10.0) -> Halo:
    """NFW halo, r_s = 1, truncated at r_cut, total sampled mass rescaled to 1."""
    rng = np.random.default_rng(seed)
    r_grid, m_grid, r_sig, sig = _nfw_tables(float(r_cut))
    r = _sample_table(rng, n, r_grid, m_grid)
    r = np.maximum(r, 1e-7)
    sigma = np.exp(np.interp(np.log(r), np.log(r_sig), np.log(sig)))
    return _finish(rng, r, sigma, "nfw", {"r_cut": r_cut})


# The paper's halo (Sect. 2) and Milky-Way-like host (Sect. 4.1), physical units.
G_KPC_KMS2_PER_MSUN = 4.30091727e-6          # gravitational constant in kpc (km/s)^2 / M_sun
HALO_RHO0_MSUN_KPC3, HALO_RS_KPC = 4.42e7, 1.28
HOST_NFW = (8.54e6, 19.6)                     # rho_s [M_sun/kpc^3], r_s [kpc]
HOST_BULGE = (9.23e9, 1.3)                    # M_H [M_sun], a_H [kpc]
HOST_DISKS = ((3.52e10, 2.5, 0.3),            # thin stellar: M_d [M_sun], a_d, b_d [kpc]
              (1.05e10, 3.02, 0.9),           # thick stellar
              (1.2e9, 1.5, 0.045),            # thin gas
              (1.1e10, 7.0, 0.085))           # thick gas
SATELLITE_POS_KPC = (58.16, 40.12, 101.41)
SATELLITE_VEL_KMS = (45.94, 83.42, 53.12)


def satellite_units(r_cut: float = 10.0):
    """(length kpc, mass M_sun, velocity km/s) of the code units of ``nfw(r_cut=...)``
    read as the paper's halo: length r_s, mass inside r_cut, G = 1."""
    length = HALO_RS_KPC
    mass = 4.0 * math.pi * HALO_RHO0_MSUN_KPC3 * length ** 3 * (math.log1p(r_cut) - r_cut / (1.0 + r_cut))
    return length, mass, math.sqrt(G_KPC_KMS2_PER_MSUN * mass / length)


def milky_way_host(r_cut: float = 10.0) -> dict:
    """The six-part host of Sect. 4.1 in code units (G = 1, centre at the origin)."""
    L, M, _ = satellite_units(r_cut)
    return {"G": 1.0, "center": (0.0, 0.0, 0.0),
            "nfw": (HOST_NFW[0] * L ** 3 / M, HOST_NFW[1] / L),
            "bulge": (HOST_BULGE[0] / M, HOST_BULGE[1] / L),
            "disks": [(m / M, a / L, b / L) for m, a, b in HOST_DISKS]}


def satellite_orbit(r_cut: float = 10.0):
    """Initial position and velocity of the satellite's centre (Sect. 4.1), code units."""
    L, _, V = satellite_units(r_cut)
    return (np.array(SATELLITE_POS_KPC) / L, np.array(SATELLITE_VEL_KMS) / V)


def cored_nfw(n: int, seed: int, r_core: float = 0.05, contrast: float = 1e3,
              r_cut: float = 10.0) -> Halo:
    """King-like core matched to an NFW outer profile (continuous density)."""
    rng = np.random.default_rng(seed)
    rho_core = lambda s: contrast * NFW_RHO_S * (1.0 + (s / r_core) ** 2) ** -1.5
    rho_nfw = lambda s: NFW_RHO_S / (s * (1.0 + s) ** 2)
    # outermost crossing radius of the two profiles
    rs = np.geomspace(1e-4, r_cut, 200001)
    diff = rho_core(rs) - rho_nfw(rs)
    idx = np.nonzero(np.sign(diff[:-1]) != np.sign(diff[1:]))[0]
    r_x = float(rs[idx[-1]]) if idx.size else r_cut
    rho = lambda s: rho_core(s) if s < r_x else rho_nfw(s)
    r_grid = np.concatenate([[0.0], np.geomspace(1e-7, r_cut, 200001)])
    dens = np.where(r_grid < r_x, rho_core(r_grid),
                    NFW_RHO_S / (np.maximum(r_grid, 1e-300) * (1.0 + r_grid) ** 2))
    shell = 4.0 * math.pi * r_grid ** 2 * dens
    m_grid = np.concatenate([[0.0], np.cumsum(0.5 * (shell[1:] + shell[:-1]) * np.diff(r_grid))])
    r = np.maximum(_sample_table(rng, n, r_grid, m_grid), 1e-7)
    m_tab = lambda s: float(np.interp(s, r_grid, m_grid)) if s <= r_cut else \
        float(m_grid[-1] + _nfw_mass(np.array(s)) - _nfw_mass(np.array(r_cut)))
    sigma = _jeans_sigma(rho, m_tab, r)
    return _finish(rng, r, sigma, "cored_nfw", {"r_core": r_core, "contrast": contrast, "r_cross": r_x})


def uniform_box(n: int, seed: int, box: float = 1.0, sigma_v: float = 1.0) -> Halo:
    """Uniform-density box [0, box)^3 with Maxwellian velocities (1-D dispersion sigma_v).

    The particle mass is 1/n, so the mass density is 1/box^3.
    """
    rng = np.random.default_rng(seed)
    pos = rng.uniform(0.0, box, (3, n))
    vel = rng.standard_normal((3, n)) * sigma_v
    ids = rng.permutation(n).astype(np.uint32)
    return Halo(pos=pos, vel=vel, ids=ids, mass=1.0 / n, name="box",
                meta={"box": box, "sigma_v": sigma_v})


def batch(halos: list) -> Batch:
    """Concatenate halos into one batch (halo h occupies offsets[h]..offsets[h+1])."""
    offs = np.zeros(len(halos) + 1, dtype=np.int64)
    for i, h in enumerate(halos):
        offs[i + 1] = offs[i] + h.n
    pos = np.concatenate([h.pos for h in halos], axis=1) if halos else np.zeros((3, 0))
    vel = np.concatenate([h.vel for h in halos], axis=1) if halos else np.zeros((3, 0))
    ids = np.concatenate([h.ids for h in halos]) if halos else np.zeros(0, np.uint32)
    return Batch(pos=np.ascontiguousarray(pos), vel=np.ascontiguousarray(vel),
                 ids=np.ascontiguousarray(ids.astype(np.uint32)), offsets=offs,
                 mass=np.array([h.mass for h in halos], dtype=np.float64), halos=halos)

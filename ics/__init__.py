"""Seeded synthetic initial conditions shared by the tests, the oracle checks and the benchmark.

This module only draws bodies; it holds none of the Barnes-Hut arithmetic (no keys, no tree,
no forces, no integration).  Every generator returns float64 arrays in the structure-of-arrays
layout the library uses:

    pos  : (3, N)  rows x, y, z
    vel  : (3, N)
    mass : (N,)

Workloads follow the paper's test problem (§5: colliding Plummer clusters of equal-mass stars,
G = 1, total mass 1) scaled up, plus the forest and disk+bulge stress cases:

* ``plummer``      one Plummer sphere, radii by inverse CDF, speeds by von Neumann rejection
                   (Aarseth, Henon & Wielen 1974), centre-of-mass frame.
* ``two_plummer``  two equal clusters of N/2 bodies each, centres at -d and +d on x, closing
                   speed ``v_rel`` along x.
* ``forest``       S independent Plummer systems with N_s log-uniform in [n_min, n_max], packed
                   back to back with an offsets table.
* ``disk_bulge``   exponential disk (sech^2 vertical profile) + Hernquist bulge, cold circular
                   velocities from the enclosed mass.

Random numbers come from numpy's PCG64 seeded by the caller, so every input is reproducible.
"""
from __future__ import annotations

import numpy as np

# Radii are drawn from the Plummer mass fraction u in (0, U_MAX]; capping u keeps the rare
# far outliers (r -> infinity as u -> 1) out of the box, as is usual for Plummer generators.
U_MAX = 0.999


def _isotropic(rng: np.random.Generator, n: int) -> np.ndarray:
    """Unit vectors uniform on the sphere, shape (3, n)."""
    cos_t = rng.uniform(-1.0, 1.0, n)
    phi = rng.uniform(0.0, 2.0 * np.pi, n)
    sin_t = np.sqrt(np.maximum(0.0, 1.0 - cos_t * cos_t))
    return np.stack([sin_t * np.cos(phi), sin_t * np.sin(phi), cos_t])


def _plummer_speed_fraction(rng: np.random.Generator, n: int) -> np.ndarray:
    """q = v / v_escape with density g(q) ~ q^2 (1 - q^2)^(7/2), by rejection (max of g < 0.1)."""
    out = np.empty(n)
    filled = 0
    while filled < n:
        want = n - filled
        m = int(want * 1.25) + 64
        q = rng.uniform(0.0, 1.0, m)
        y = rng.uniform(0.0, 0.1, m)
        keep = q[y < q * q * (1.0 - q * q) ** 3.5]
        take = min(want, keep.size)
        out[filled:filled + take] = keep[:take]
        filled += take
    return out


def plummer(n: int, seed: int, a: float = 1.0, total_mass: float = 1.0, G: float = 1.0,
            com_frame: bool = True):
    """One Plummer sphere of ``n`` equal-mass bodies (scale radius ``a``), virialised velocities."""
    rng = np.random.Generator(np.random.PCG64(seed))
    n = int(n)
    if n == 0:
        return np.zeros((3, 0)), np.zeros((3, 0)), np.zeros(0)
    u = rng.uniform(0.0, U_MAX, n)
    u = np.maximum(u, 1e-300)
    r = a / np.sqrt(u ** (-2.0 / 3.0) - 1.0)
    pos = r * _isotropic(rng, n)
    v_esc = np.sqrt(2.0 * G * total_mass) * (r * r + a * a) ** (-0.25)
    vel = (_plummer_speed_fraction(rng, n) * v_esc) * _isotropic(rng, n)
    mass = np.full(n, total_mass / n)
    if com_frame:
        pos -= pos.mean(axis=1, keepdims=True)
        vel -= vel.mean(axis=1, keepdims=True)
    return np.ascontiguousarray(pos), np.ascontiguousarray(vel), mass


def two_plummer(n: int, seeds=(4, 5), separation: float = 5.0, v_rel: float = 0.5,
                a: float = 1.0, total_mass: float = 1.0):
    """Two equal Plummer clusters (n/2 bodies each, mass total/2 each) at x = -sep and x = +sep.

    The left cluster moves with +v_rel/2 along x and the right one with -v_rel/2, so the
    clusters close at ``v_rel``.  The first n//2 bodies belong to the left cluster.
    """
    n1 = n // 2
    n2 = n - n1
    p1, v1, m1 = plummer(n1, seeds[0], a=a, total_mass=total_mass * n1 / n)
    p2, v2, m2 = plummer(n2, seeds[1], a=a, total_mass=total_mass * n2 / n)
    p1[0] -= separation
    p2[0] += separation
    v1[0] += 0.5 * v_rel
    v2[0] -= 0.5 * v_rel
    pos = np.ascontiguousarray(np.concatenate([p1, p2], axis=1))
    vel = np.ascontiguousarray(np.concatenate([v1, v2], axis=1))
    mass = np.concatenate([m1, m2])
    return pos, vel, mass


def forest_sizes(n_systems: int, seed: int, n_min: int = 1024, n_max: int = 65536) -> np.ndarray:
    """System sizes log-uniform in [n_min, n_max] (rounded), int64."""
    rng = np.random.Generator(np.random.PCG64(seed))
    ln = rng.uniform(np.log(n_min), np.log(n_max), n_systems)
    return np.clip(np.rint(np.exp(ln)), n_min, n_max).astype(np.int64)


def forest(n_systems: int = 512, seed: int = 6, n_min: int = 1024, n_max: int = 65536):
    """Packed forest of independent Plummer systems.

    Returns pos (3, sum N), vel (3, sum N), mass (sum N), offsets (S+1,) int64.  System s owns
    the columns offsets[s]:offsets[s+1]; its bodies come from ``plummer(N_s, seed*100003 + s)``.
    """
    sizes = forest_sizes(n_systems, seed, n_min, n_max)
    offsets = np.zeros(n_systems + 1, dtype=np.int64)
    offsets[1:] = np.cumsum(sizes)
    total = int(offsets[-1])
    pos = np.empty((3, total))
    vel = np.empty((3, total))
    mass = np.empty(total)
    for s in range(n_systems):
        p, v, m = plummer(int(sizes[s]), seed * 100003 + s)
        lo, hi = offsets[s], offsets[s + 1]
        pos[:, lo:hi] = p
        vel[:, lo:hi] = v
        mass[lo:hi] = m
    return pos, vel, mass, offsets


def disk_bulge(n: int, seed: int = 7, r_d: float = 3.0, z0: float = 0.3, disk_frac: float = 0.8,
               a_bulge: float = 0.5, total_mass: float = 1.0, G: float = 1.0):
    """Exponential disk + Hernquist bulge, equal masses, cold circular velocities.

    Disk: surface density ~ exp(-R/r_d), so R ~ Gamma(2, r_d); vertical density ~ sech^2(z/z0),
    so z = z0 * atanh(2u - 1).  Bulge: Hernquist, r = a sqrt(w) / (1 - sqrt(w)) with the mass
    fraction w in (0, U_MAX].  Speeds: v_c^2 = G M(<r) / r with the enclosed mass of both
    components taken as spherical (a stated simplification); disk bodies move along phi-hat,
    bulge bodies along a random direction perpendicular to their radius vector.
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    n_disk = int(round(n * disk_frac))
    n_bulge = n - n_disk
    m_disk = total_mass * n_disk / n
    m_bulge = total_mass - m_disk

    R = rng.gamma(2.0, r_d, n_disk)
    phi = rng.uniform(0.0, 2.0 * np.pi, n_disk)
    uz = rng.uniform(1e-12, 1.0 - 1e-12, n_disk)
    z = z0 * np.arctanh(2.0 * uz - 1.0)
    pd = np.stack([R * np.cos(phi), R * np.sin(phi), z])

    w = rng.uniform(0.0, U_MAX, n_bulge)
    sw = np.sqrt(w)
    rb = a_bulge * sw / (1.0 - sw)
    pb = rb * _isotropic(rng, n_bulge)

    def m_enc(r):
        disk = m_disk * (1.0 - (1.0 + r / r_d) * np.exp(-r / r_d))
        bulge = m_bulge * r * r / (r + a_bulge) ** 2
        return disk + bulge

    rs_d = np.sqrt(R * R + z * z)
    vc_d = np.sqrt(G * m_enc(rs_d) / np.maximum(rs_d, 1e-12))
    vd = np.stack([-np.sin(phi) * vc_d, np.cos(phi) * vc_d, np.zeros(n_disk)])

    vc_b = np.sqrt(G * m_enc(rb) / np.maximum(rb, 1e-12))
    rnd = _isotropic(rng, n_bulge)
    rhat = pb / np.maximum(rb, 1e-12)
    perp = rnd - (rnd * rhat).sum(axis=0) * rhat
    perp /= np.maximum(np.linalg.norm(perp, axis=0), 1e-12)
    vb = perp * vc_b

    pos = np.ascontiguousarray(np.concatenate([pd, pb], axis=1))
    vel = np.ascontiguousarray(np.concatenate([vd, vb], axis=1))
    mass = np.full(n, total_mass / n)
    return pos, vel, mass


def uniform_cube(n: int, seed: int, side: float = 1.0):
    """Bodies uniform in [0, side)^3 with random masses in [0.5, 1.5) / n (edge-case tests)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    pos = np.ascontiguousarray(rng.uniform(0.0, side, (3, n)))
    vel = np.ascontiguousarray(rng.normal(0.0, 0.1, (3, n)))
    mass = rng.uniform(0.5, 1.5, n) / max(n, 1)
    return pos, vel, mass


# Named workloads: the five configurations the library is measured and tested on.
WORKLOADS = {
    "plummer_4k": dict(kind="plummer", n=4096, seed=1, eps=0.01, theta=0.5, dt=1e-3, steps=10),
    "plummer_1m": dict(kind="plummer", n=1048576, seed=2, eps=0.005, theta=0.5, dt=5e-4,
                       steps=20),
    "two_plummer_16m": dict(kind="two_plummer", n=16777216, seeds=(4, 5), eps=0.002, theta=0.5,
                            dt=5e-4, steps=10),
    "forest_512": dict(kind="forest", systems=512, seed=6, eps=0.01, theta=0.6, dt=1e-3,
                       steps=100),
    "disk_bulge_64m": dict(kind="disk_bulge", n=67108864, seed=7, eps=0.001, theta=0.5,
                           dt=2e-4, steps=5),
}

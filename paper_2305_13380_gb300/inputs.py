"""Seeded synthetic initial conditions for the SPH neighbour loops.

This module only draws particles: it holds none of the SPH arithmetic.  The
tests, the benchmark and the oracle checks all take their inputs from here.

Random numbers come from a counter-based generator: SplitMix64 (Steele, Lea &
Flood 2014, "Fast splittable pseudorandom number generators") evaluated at
position ``counter`` of the stream whose start is a hash of (workload, seed,
field).  Every value depends only on those keys and the particle index, so the
draw does not depend on generation order (the same property the paper asks of
its random numbers in Sec. 9.4).

Workloads (the paper's simulation inputs are not available; these stand in):
  * ``lattice``   -- n^3 jittered lattice in a periodic box (uniform gas);
  * ``clustered`` -- Plummer spheres plus a uniform background (clustered gas,
                     smoothing lengths spanning two orders of magnitude);
  * ``batch``     -- many independent small boxes of uneven size;
  * ``two_spheres`` -- two uniform-density spheres on a collision course.
"""
from __future__ import annotations

import math

import numpy as np

ETA = 1.2348

_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)

# field identifiers of the stream keys
_F = {name: k for k, name in enumerate(
    ["jx", "jy", "jz", "u", "vx1", "vx2", "vy1", "vy2", "vz1", "vz2", "sphere", "rad", "dir1",
     "dir2", "bgx", "bgy", "bgz", "scale", "cx", "cy", "cz", "lnu1", "lnu2", "nbox", "kind",
     "radius", "speed", "pos1", "pos2", "pos3", "perm"])}


def _mix(z: np.ndarray) -> np.ndarray:
    z = (z ^ (z >> np.uint64(30))) * _M1
    z = (z ^ (z >> np.uint64(27))) * _M2
    return z ^ (z >> np.uint64(31))


def _key(workload: int, seed: int, field: str) -> np.uint64:
    mask = (1 << 64) - 1
    k = ((workload * 0x100000001B3) ^ (seed * 0xC2B2AE3D27D4EB4F) ^
         (_F[field] * 0x165667B19E3779F9)) & mask
    with np.errstate(over="ignore"):
        s = _mix(np.array([k], dtype=np.uint64) + _GOLDEN)
    return s[0]


def bits(workload: int, seed: int, field: str, counter: np.ndarray) -> np.ndarray:
    """64 random bits per counter (SplitMix64 output at that stream position)."""
    c = np.asarray(counter, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = _key(workload, seed, field) + (c + np.uint64(1)) * _GOLDEN
        return _mix(z)


def uniform(workload: int, seed: int, field: str, counter: np.ndarray) -> np.ndarray:
    """Uniform doubles in [0, 1) from the top 53 bits."""
    return (bits(workload, seed, field, counter) >> np.uint64(11)).astype(np.float64) * 2.0 ** -53


def normal(workload: int, seed: int, f1: str, f2: str, counter: np.ndarray) -> np.ndarray:
    """Standard normal deviates by the Box-Muller transform."""
    u1 = uniform(workload, seed, f1, counter)
    u2 = uniform(workload, seed, f2, counter)
    return np.sqrt(-2.0 * np.log1p(-u1)) * np.cos(2.0 * math.pi * u2)


def _wrap(x: np.ndarray, L: float) -> np.ndarray:
    x = np.mod(x, L)
    x[x >= L] -= L  # np.mod may return L for tiny negative inputs
    return x


def lattice(n_side: int, seed: int = 0, L: float = 1.0, jitter: float = 0.1,
            sigma_v: float = 0.01, u0: float = 1.0, u_noise: float = 0.01,
            workload: int = 1) -> dict:
    """Jittered n_side^3 lattice: x = (i + 1/2 + U(-jitter, jitter)) d, equal
    masses summing to 1, u = u0 (1 + u_noise U(-1, 1)), Gaussian velocities.
    Particle index i = ix + n (iy + n iz).  h0 = eta d is the starting guess."""
    n = n_side ** 3
    d = L / n_side
    i = np.arange(n, dtype=np.int64)
    ix, iy, iz = i % n_side, (i // n_side) % n_side, i // (n_side * n_side)
    c = i.astype(np.uint64)
    jx = uniform(workload, seed, "jx", c) * 2.0 - 1.0
    jy = uniform(workload, seed, "jy", c) * 2.0 - 1.0
    jz = uniform(workload, seed, "jz", c) * 2.0 - 1.0
    x = _wrap((ix + 0.5 + jitter * jx) * d, L)
    y = _wrap((iy + 0.5 + jitter * jy) * d, L)
    z = _wrap((iz + 0.5 + jitter * jz) * d, L)
    u = u0 * (1.0 + u_noise * (uniform(workload, seed, "u", c) * 2.0 - 1.0))
    vx = sigma_v * normal(workload, seed, "vx1", "vx2", c)
    vy = sigma_v * normal(workload, seed, "vy1", "vy2", c)
    vz = sigma_v * normal(workload, seed, "vz1", "vz2", c)
    m = np.full(n, 1.0 / n)
    h0 = np.full(n, ETA * d)
    return dict(L=L, x=x, y=y, z=z, vx=vx, vy=vy, vz=vz, m=m, u=u, h0=h0)


def clustered(n: int, n_spheres: int = 64, seed: int = 0, L: float = 1.0,
              frac_clustered: float = 0.7, a_min: float = 0.002, a_max: float = 0.02,
              sigma_v: float = 0.05, workload: int = 3) -> dict:
    """Plummer spheres plus a uniform background in a periodic box.

    frac_clustered of the particles are split evenly over n_spheres spheres
    (remainder to the first ones); sphere s has scale radius a_s log-uniform in
    [a_min, a_max] and a uniform centre.  Radii follow the Plummer cumulative
    mass profile r = a / sqrt(X^(-2/3) - 1) with isotropic directions, and
    positions are wrapped into the box (no truncation).  u is log-normal with
    sigma 1, velocities Gaussian with sigma_v, equal masses summing to 1.
    The starting guess h0 is eta times the local mean spacing estimated from
    each particle's own sphere (or the background)."""
    n_cl = int(round(frac_clustered * n))
    n_bg = n - n_cl
    per = np.full(n_spheres, n_cl // n_spheres, dtype=np.int64)
    per[: n_cl - per.sum()] += 1
    sph = np.arange(n_spheres, dtype=np.uint64)
    a = a_min * (a_max / a_min) ** uniform(workload, seed, "scale", sph)
    cen = np.stack([uniform(workload, seed, f, sph) * L for f in ("cx", "cy", "cz")], axis=1)
    owner = np.repeat(np.arange(n_spheres), per)
    c = np.arange(n_cl, dtype=np.uint64)
    X = uniform(workload, seed, "rad", c)
    X = np.clip(X, 1e-300, 1.0 - 2.0 ** -53)
    r = a[owner] / np.sqrt(X ** (-2.0 / 3.0) - 1.0)
    cth = uniform(workload, seed, "dir1", c) * 2.0 - 1.0
    phi = uniform(workload, seed, "dir2", c) * 2.0 * math.pi
    sth = np.sqrt(np.maximum(0.0, 1.0 - cth * cth))
    px = cen[owner, 0] + r * sth * np.cos(phi)
    py = cen[owner, 1] + r * sth * np.sin(phi)
    pz = cen[owner, 2] + r * cth
    cb = np.arange(n_cl, n, dtype=np.uint64)
    bx = uniform(workload, seed, "bgx", cb) * L
    by = uniform(workload, seed, "bgy", cb) * L
    bz = uniform(workload, seed, "bgz", cb) * L
    x = _wrap(np.concatenate([px, bx]), L)
    y = _wrap(np.concatenate([py, by]), L)
    z = _wrap(np.concatenate([pz, bz]), L)
    ci = np.arange(n, dtype=np.uint64)
    u = np.exp(normal(workload, seed, "lnu1", "lnu2", ci))
    vx = sigma_v * normal(workload, seed, "vx1", "vx2", ci)
    vy = sigma_v * normal(workload, seed, "vy1", "vy2", ci)
    vz = sigma_v * normal(workload, seed, "vz1", "vz2", ci)
    m = np.full(n, 1.0 / n)
    # starting guess: Plummer density rho(r) = 3M/(4 pi a^3) (1 + r^2/a^2)^(-5/2)
    # expressed as a number density of the sphere's particles, plus the background
    n_bg_dens = n_bg / L ** 3
    nd = np.full(n, n_bg_dens)
    if n_cl:
        nd_sph = 3.0 * per[owner] / (4.0 * math.pi * a[owner] ** 3) * \
            (1.0 + (r / a[owner]) ** 2) ** -2.5
        nd[:n_cl] += nd_sph
    h0 = ETA * nd ** (-1.0 / 3.0)
    h0 = np.minimum(h0, 0.1 * L)
    return dict(L=L, x=x, y=y, z=z, vx=vx, vy=vy, vz=vz, m=m, u=u, h0=h0)


def batch_sizes(n_boxes: int, seed0: int = 0, n_min: float = 1e3, n_max: float = 1e5,
                workload: int = 4):
    """Particle counts log-uniform in [n_min, n_max] and the kind of each box
    (even box index: lattice, odd: clustered); lattice counts are rounded to
    a cube."""
    out = []
    for b in range(n_boxes):
        uu = uniform(workload, seed0 + b, "nbox", np.zeros(1, dtype=np.uint64))[0]
        nb = int(math.floor(n_min * (n_max / n_min) ** uu))
        if b % 2 == 0:
            side = max(4, int(round(nb ** (1.0 / 3.0))))
            out.append(("lattice", side ** 3, side))
        else:
            out.append(("clustered", nb, None))
    return out


# A periodic box needs at least 3 cells of the largest support per side; a
# uniform background of at least this many particles keeps the background
# support below a third of the unit box.
MIN_BACKGROUND = 800


def batch(n_boxes: int, seed0: int = 0, **kw) -> list:
    """Independent periodic unit boxes: box b uses seed seed0 + b; even b is a
    jittered lattice, odd b a clustered box with 4 Plummer spheres whose
    background holds 30 % of the particles but at least MIN_BACKGROUND."""
    boxes = []
    for b, (kind, nb, side) in enumerate(batch_sizes(n_boxes, seed0, **kw)):
        if kind == "lattice":
            boxes.append(lattice(side, seed=seed0 + b, workload=41))
        else:
            frac = min(0.7, 1.0 - MIN_BACKGROUND / nb)
            boxes.append(clustered(nb, n_spheres=4, seed=seed0 + b, frac_clustered=frac,
                                   workload=43))
    return boxes


def two_spheres(seed: int, L: float = 2.0, n_min: float = 1e3, n_max: float = 5e5,
                u0: float = 0.05, workload: int = 5) -> dict:
    """Two uniform-density spheres on a collision course along x.

    Radii U(0.1, 0.3); total count log-uniform in [n_min, n_max] split in
    proportion to r^3 (equal particle mass and density); centres separated by
    r1 + r2 + 0.05 around the box centre; relative speed U(0.5, 2) split
    symmetrically; u = u0; equal masses summing to 1."""
    k = np.arange(4, dtype=np.uint64)
    rr = uniform(workload, seed, "radius", k)
    r1, r2 = 0.1 + 0.2 * rr[0], 0.1 + 0.2 * rr[1]
    ntot = int(math.floor(n_min * (n_max / n_min) ** rr[2]))
    vrel = 0.5 + 1.5 * uniform(workload, seed, "speed", k)[0]
    n1 = max(1, int(round(ntot * r1 ** 3 / (r1 ** 3 + r2 ** 3))))
    n2 = max(1, ntot - n1)
    pts = []
    off = 0
    for s, (ns, rs) in enumerate(((n1, r1), (n2, r2))):
        c = np.arange(off, off + ns, dtype=np.uint64)
        rad = rs * uniform(workload, seed, "pos1", c) ** (1.0 / 3.0)
        cth = uniform(workload, seed, "pos2", c) * 2.0 - 1.0
        phi = uniform(workload, seed, "pos3", c) * 2.0 * math.pi
        sth = np.sqrt(np.maximum(0.0, 1.0 - cth * cth))
        pts.append(np.stack([rad * sth * np.cos(phi), rad * sth * np.sin(phi), rad * cth], 1))
        off += ns
    sep = r1 + r2 + 0.05
    c1 = np.array([0.5 * L - 0.5 * sep, 0.5 * L, 0.5 * L])
    c2 = np.array([0.5 * L + 0.5 * sep, 0.5 * L, 0.5 * L])
    p = np.concatenate([pts[0] + c1, pts[1] + c2])
    n = p.shape[0]
    v = np.zeros((n, 3))
    v[:n1, 0] = 0.5 * vrel
    v[n1:, 0] = -0.5 * vrel
    dens = n / (4.0 / 3.0 * math.pi * (r1 ** 3 + r2 ** 3))
    h0 = np.full(n, ETA * dens ** (-1.0 / 3.0))
    return dict(L=L, x=_wrap(p[:, 0].copy(), L), y=_wrap(p[:, 1].copy(), L),
                z=_wrap(p[:, 2].copy(), L), vx=v[:, 0].copy(), vy=v[:, 1].copy(),
                vz=v[:, 2].copy(), m=np.full(n, 1.0 / n), u=np.full(n, u0), h0=h0)

"""Seeded synthetic inputs for the short-range MD hot path.

This module only *makes inputs*: lattices, thermal velocities, jitter,
slab/nanoparticle geometries and species labels.  It holds none of the
method's arithmetic (no cell lists, no neighbour tests, no forces, no
integration), so both the CUDA path and the independent CPU oracle can be
fed from it without sharing any of the computation they are compared on.

Every random number comes from one counter-based generator, SplitMix64
(Steele, Lea and Flood, "Fast splittable pseudorandom number generators",
OOPSLA 2014), evaluated at (seed, stream, counter), so the same seed gives the
same bits on every machine and numpy version.

The workloads mirror the paper's benchmark shapes (Sec. III: a homogeneous
fcc bulk crystal of about 1e6 atoms, and strongly inhomogeneous systems - a
nanoparticle in vacuum, porous sintered particles), with a Lennard-Jones
fluid, and the paper's copper crystal with Cleri and Rosato's published
parameters of its many-body potential.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def splitmix64(seed: int, stream: int, n: int, offset: int = 0) -> np.ndarray:
    """Return n uint64 words: SplitMix64 output for counters offset..offset+n-1.

    The state for counter k of (seed, stream) is seed' + (k+1)*golden, where
    seed' mixes the stream id into the seed; the output is the published
    SplitMix64 finaliser applied to that state.
    """
    with np.errstate(over="ignore"):
        base = np.uint64((seed * 0x100000001B3 + stream * 0x2545F4914F6CDD1D) & 0xFFFFFFFFFFFFFFFF)
        k = np.arange(offset + 1, offset + n + 1, dtype=np.uint64)
        z = base + k * _GOLDEN
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        z = z ^ (z >> np.uint64(31))
    return z


def uniform01(seed: int, stream: int, n: int, offset: int = 0) -> np.ndarray:
    """n doubles uniform in the open interval (0, 1): top 53 bits + half an ulp."""
    w = splitmix64(seed, stream, n, offset) >> np.uint64(11)
    return (w.astype(np.float64) + 0.5) * (1.0 / 9007199254740992.0)


def normal(seed: int, stream: int, n: int) -> np.ndarray:
    """n standard normal doubles by the Box-Muller transform of paired uniforms."""
    m = (n + 1) // 2
    u1 = uniform01(seed, stream, m, 0)
    u2 = uniform01(seed, stream, m, m)
    r = np.sqrt(-2.0 * np.log(u1))
    t = 2.0 * np.pi * u2
    z = np.empty(2 * m)
    z[0::2] = r * np.cos(t)
    z[1::2] = r * np.sin(t)
    return z[:n]


def lattice_constant(rho: float) -> float:
    """Cubic fcc lattice constant for number density rho (4 atoms per unit cell)."""
    return (4.0 / rho) ** (1.0 / 3.0)


_FCC_BASIS = np.array([[0.0, 0.0, 0.0], [0.5, 0.5, 0.0], [0.5, 0.0, 0.5], [0.0, 0.5, 0.5]])


def fcc_lattice(nx: int, ny: int, nz: int, a: float):
    """fcc sites of nx*ny*nz cubic unit cells, unit cells x fastest, 4 basis atoms each.

    Returns (pos (N,3) float64 in [0, L), box (3,) float64).
    """
    iz, iy, ix = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    cells = np.stack([ix.ravel(), iy.ravel(), iz.ravel()], axis=1).astype(np.float64)
    pos = (cells[:, None, :] + _FCC_BASIS[None, :, :]).reshape(-1, 3) * a
    box = np.array([nx * a, ny * a, nz * a])
    return pos, box


def wrap(pos: np.ndarray, box: np.ndarray) -> np.ndarray:
    """Map positions into [0, L) per dimension."""
    out = pos - box * np.floor(pos / box)
    out = np.where(out >= box, out - box, out)
    return np.where(out < 0.0, 0.0, out)


def thermal_velocities(masses: np.ndarray, T: float, seed: int, stream: int = 1) -> np.ndarray:
    """Gaussian velocities with zero total momentum, rescaled to temperature T exactly.

    T is defined with 3N-3 degrees of freedom (momentum removed), k_B = 1.
    """
    n = masses.shape[0]
    v = normal(seed, stream, 3 * n).reshape(n, 3) / np.sqrt(masses)[:, None]
    p = (masses[:, None] * v).sum(axis=0)
    v -= p / masses.sum()
    twice_ke = float((masses[:, None] * v * v).sum())
    dof = max(3 * n - 3, 1)
    v *= math.sqrt(T * dof / twice_ke)
    return v


def gaussian_jitter(pos: np.ndarray, box: np.ndarray, amp: float, seed: int, stream: int = 2):
    """Displace every coordinate by amp * N(0,1) and wrap back into the box."""
    d = normal(seed, stream, pos.size).reshape(pos.shape) * amp
    return wrap(pos + d, box)


@dataclass
class System:
    """One synthetic workload: positions, velocities, species and the box."""
    pos: np.ndarray       # (N,3) float64, in [0, L)
    vel: np.ndarray       # (N,3) float64
    species: np.ndarray   # (N,) int32
    box: np.ndarray       # (3,) float64
    name: str = ""

    @property
    def n(self) -> int:
        return int(self.pos.shape[0])


def lj_fcc(n_cells: int, rho: float = 0.8442, T: float = 0.72, seed: int = 1,
           jitter: float = 0.0, name: str = "") -> System:
    """Single-species LJ system started from an fcc lattice of n_cells^3 unit cells.

    With jitter > 0 every coordinate is displaced by a Gaussian of that width,
    which gives liquid-like disorder (non-zero forces) without overlaps.
    """
    a = lattice_constant(rho)
    pos, box = fcc_lattice(n_cells, n_cells, n_cells, a)
    if jitter > 0.0:
        pos = gaussian_jitter(pos, box, jitter, seed, stream=2)
    masses = np.ones(pos.shape[0])
    vel = thermal_velocities(masses, T, seed, stream=1)
    species = np.zeros(pos.shape[0], dtype=np.int32)
    return System(pos, vel, species, box, name or f"lj_fcc_{n_cells}")


def random_gas(n: int, box, seed: int, stream: int = 3) -> np.ndarray:
    """n positions uniform in the box (overlaps allowed: for neighbour-set tests only)."""
    box = np.asarray(box, dtype=np.float64)
    u = uniform01(seed, stream, 3 * n).reshape(n, 3)
    return wrap(u * box, box)


def threshold_pairs(n_pairs: int, box, r: float, rel: float, seed: int, stream: int = 4):
    """Atom pairs placed at separations r*(1-rel) and r*(1+rel), alternately.

    Pairs are put far apart from each other on a coarse grid so that each
    pair probes one neighbour-list comparison right at its threshold.
    Returns positions (2*n_pairs, 3).
    """
    box = np.asarray(box, dtype=np.float64)
    u = uniform01(seed, stream, 3 * n_pairs).reshape(n_pairs, 3)
    g = int(math.ceil(n_pairs ** (1.0 / 3.0)))
    idx = np.arange(n_pairs)
    centers = np.stack([idx % g, (idx // g) % g, idx // (g * g)], axis=1) + 0.5
    centers = centers * (box / g)
    theta = np.arccos(2.0 * u[:, 0] - 1.0)
    phi = 2.0 * np.pi * u[:, 1]
    dirs = np.stack([np.sin(theta) * np.cos(phi), np.sin(theta) * np.sin(phi), np.cos(theta)], axis=1)
    sep = np.where(idx % 2 == 0, r * (1.0 - rel), r * (1.0 + rel))
    a = centers - 0.5 * sep[:, None] * dirs
    b = centers + 0.5 * sep[:, None] * dirs
    return wrap(np.concatenate([a, b], axis=0), box)


def _fcc_ball(center: np.ndarray, radius: float, a: float) -> np.ndarray:
    """fcc sites (axis-aligned lattice, origin at center) within radius of center."""
    m = int(math.ceil(radius / a)) + 1
    r = np.arange(-m, m + 1)
    iz, iy, ix = np.meshgrid(r, r, r, indexing="ij")
    cells = np.stack([ix.ravel(), iy.ravel(), iz.ravel()], axis=1).astype(np.float64)
    pts = (cells[:, None, :] + _FCC_BASIS[None, :, :]).reshape(-1, 3) * a
    keep = (pts * pts).sum(axis=1) <= radius * radius
    return pts[keep] + center


def slab_nanoparticles(L: float, rho: float = 0.8442, T: float = 0.3, slab_frac: float = 0.3,
                       n_particles: int = 40, r_min: float = 8.0, r_max: float = 20.0,
                       gap: float = 2.8, seed: int = 3, max_tries: int = 200000) -> System:
    """Strongly inhomogeneous workload: an fcc slab plus fcc nanoparticles in vacuum.

    The slab fills z in [0, slab_frac*L) of a periodic cube of side L.  Particle
    radii are uniform in [r_min, r_max]; centres are drawn uniformly in the
    vacuum region and accepted only if the particle keeps a surface gap of at
    least `gap` to the slab (through the periodic z boundary too) and to every
    particle already placed.
    """
    a = lattice_constant(rho)
    nxy = max(int(math.floor(L / a)), 1)
    nz = max(int(math.floor(slab_frac * L / a)), 1)
    # the slab is commensurate with the box in x and y; its thickness is nz cells
    box = np.array([nxy * a, nxy * a, nxy * a])
    slab, _ = fcc_lattice(nxy, nxy, nz, a)
    z_top = nz * a
    Lz = box[2]
    u = uniform01(seed, 5, 4 * max_tries).reshape(max_tries, 4)
    centers, radii = [], []
    k = 0
    while len(centers) < n_particles and k < max_tries:
        rad = r_min + (r_max - r_min) * u[k, 0]
        c = np.array([u[k, 1] * box[0], u[k, 2] * box[1], u[k, 3] * Lz])
        k += 1
        # vacuum region is z in [z_top, Lz): keep the surface gap to the slab on both sides
        if c[2] - rad < z_top + gap or c[2] + rad > Lz - gap:
            continue
        ok = True
        for c2, r2 in zip(centers, radii):
            d = c - c2
            d -= box * np.rint(d / box)
            if np.sqrt((d * d).sum()) < rad + r2 + gap:
                ok = False
                break
        if ok:
            centers.append(c)
            radii.append(rad)
    parts = [slab] + [_fcc_ball(c, r, a) for c, r in zip(centers, radii)]
    pos = wrap(np.concatenate(parts, axis=0), box)
    masses = np.ones(pos.shape[0])
    vel = thermal_velocities(masses, T, seed, stream=1)
    species = np.zeros(pos.shape[0], dtype=np.int32)
    sysm = System(pos, vel, species, box, "slab_nanoparticles")
    sysm.n_particles_placed = len(centers)  # type: ignore[attr-defined]
    return sysm


def species_shuffle(n: int, frac_b: float, seed: int, stream: int = 6) -> np.ndarray:
    """Species labels 0/1 with round(frac_b*n) of species 1, in a seeded random order."""
    nb = int(round(frac_b * n))
    keys = splitmix64(seed, stream, n)
    order = np.argsort(keys, kind="stable")
    sp = np.zeros(n, dtype=np.int32)
    sp[order[:nb]] = 1
    return sp


def fcc_vacancies(n: int, rho: float, T: float, seed: int, jitter: float = 0.05, name: str = "") -> System:
    """n atoms at exactly density rho: the fcc lattice of the smallest n_c^3 cells holding n
    sites, scaled into the cube of side (n/rho)^(1/3), with a seeded random set of sites
    left empty; Gaussian jitter and velocities at temperature T."""
    nc = 1
    while 4 * nc ** 3 < n:
        nc += 1
    L = (n / rho) ** (1.0 / 3.0)
    sites, _ = fcc_lattice(nc, nc, nc, L / nc)
    keys = splitmix64(seed, 7, sites.shape[0])
    keep = np.sort(np.argsort(keys, kind="stable")[:n])
    box = np.array([L, L, L])
    pos = sites[keep]
    if jitter > 0.0:
        pos = gaussian_jitter(pos, box, jitter, seed, stream=2)
    masses = np.ones(n)
    vel = thermal_velocities(masses, T, seed, stream=1)
    return System(pos, vel, np.zeros(n, dtype=np.int32), box, name or f"fcc_vacancies_{n}")


def copper_tbsma() -> dict:
    """Cleri and Rosato's published tight-binding second-moment parameters for copper
    (A, xi in eV; p, q; r0 the fcc nearest-neighbour distance at a = 3.615 A), the cutoff
    halfway between the fifth and sixth fcc shells (A), and the mass (amu)."""
    r0 = 3.615 / math.sqrt(2.0)
    return dict(A=0.0855, xi=1.224, p=10.960, q=2.278, r0=r0, rc=0.5 * (math.sqrt(5.0) + math.sqrt(6.0)) * r0,
                mass=63.546)


def batch_ensemble(n_systems: int = 512, seed: int = 4, n_min: int = 256, n_max: int = 32768,
                   rho_range=(0.7, 0.95), T_range=(0.5, 1.5)) -> list:
    """Independent periodic LJ systems of uneven size: atom counts log-uniform in
    [n_min, n_max], densities and temperatures uniform in the given ranges, all seeded."""
    u = uniform01(seed, 11, 3 * n_systems).reshape(n_systems, 3)
    out = []
    for k in range(n_systems):
        n = int(round(math.exp(math.log(n_min) + u[k, 0] * (math.log(n_max) - math.log(n_min)))))
        rho = rho_range[0] + u[k, 1] * (rho_range[1] - rho_range[0])
        T = T_range[0] + u[k, 2] * (T_range[1] - T_range[0])
        out.append(fcc_vacancies(n, rho, T, seed * 100003 + k, name=f"batch_{k}"))
    return out

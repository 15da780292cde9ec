"""Seeded synthetic inputs shaped like the paper's workloads.

This module draws geometry and per-atom free-atom parameters only; it holds none of
the MBD arithmetic, so both the CUDA path and the CPU oracle can take their inputs
from it.  The paper's own systems (urethane supercells, Sec. 3.2; L7 complexes,
Sec. 4.1) are not available, so clusters and cells with the same atom counts,
densities and parameter ranges stand in for them.

Parameter recipe (per atom, drawn in this order, independent uniforms):
  alpha0_ref ~ U[4, 12] bohr^3, c6_ref ~ U[5, 50] Ha bohr^6,
  rvdw_ref ~ U[3, 4] bohr, volume ratio ~ U[0.7, 1.0].
Seeds: workload k, instance i -> seed = 1000 k + i.

All lengths are in bohr (Hartree atomic units).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

BOHR_PER_ANGSTROM = 1.0 / 0.529177210903
# Cluster density: 0.08 atoms per cubic angstrom expressed in atoms per cubic bohr.
DENSITY_CLUSTER = 0.08 / BOHR_PER_ANGSTROM**3


@dataclass
class System:
    """One input system: coordinates [N,3], four per-atom parameter arrays [N],
    optional lattice [3,3] (rows are lattice vectors) and k-grid (3 ints)."""
    coords: np.ndarray
    alpha0_ref: np.ndarray
    c6_ref: np.ndarray
    rvdw_ref: np.ndarray
    ratio: np.ndarray
    lattice: np.ndarray | None = None
    k_grid: tuple | None = None
    name: str = ""
    meta: dict = field(default_factory=dict)

    @property
    def n_atoms(self) -> int:
        return int(self.coords.shape[0])


def draw_params(rng: np.random.Generator, n: int):
    """Free-atom parameters in the fixed draw order alpha0, C6, R_vdW, ratio."""
    a0 = rng.uniform(4.0, 12.0, n)
    c6 = rng.uniform(5.0, 50.0, n)
    rv = rng.uniform(3.0, 4.0, n)
    vr = rng.uniform(0.7, 1.0, n)
    return a0, c6, rv, vr


def nl_ratios(n: int, seed: int):
    """Density-functional ratios for MBD-NL inputs, drawn from their own stream (seed):
    ra = alpha0_df/alpha0_df,ref ~ U[0.7, 1.0] (like the volume ratio: compression in the
    system), then rw = omega_df/omega_df,ref ~ U[0.85, 1.2]."""
    rng = np.random.default_rng(seed)
    ra = rng.uniform(0.7, 1.0, n)
    rw = rng.uniform(0.85, 1.2, n)
    return ra, rw


class _Grid:
    """Bucket grid for minimum-separation rejection sampling (open boundaries)."""

    def __init__(self, lo: np.ndarray, hi: np.ndarray, h: float):
        self.lo, self.h = lo, h
        self.dims = np.maximum(1, np.ceil((hi - lo) / h).astype(int))
        self.cells: dict = {}

    def key(self, p):
        return tuple(np.clip(((p - self.lo) / self.h).astype(int), 0, self.dims - 1))

    def near(self, p, pts, dmin):
        k = self.key(p)
        for dx in (-1, 0, 1):
            for dy in (-1, 0, 1):
                for dz in (-1, 0, 1):
                    for idx in self.cells.get((k[0] + dx, k[1] + dy, k[2] + dz), ()):
                        d = p - pts[idx]
                        if d @ d < dmin * dmin:
                            return True
        return False

    def add(self, p, idx):
        self.cells.setdefault(self.key(p), []).append(idx)


def _rsa(rng, n, sample, lo, hi, dmin, max_tries=2_000_000):
    """Random sequential addition: draw candidates from `sample`, keep those at least
    dmin from every kept point."""
    grid = _Grid(lo, hi, dmin)
    pts = np.zeros((n, 3))
    k = tries = 0
    while k < n:
        tries += 1
        if tries > max_tries:
            raise RuntimeError("random sequential addition jammed")
        p = sample()
        if grid.near(p, pts[:k], dmin):
            continue
        pts[k] = p
        grid.add(p, k)
        k += 1
    return pts


def cube_cluster(n_atoms=32, edge=14.0, dmin=2.5, seed=0, name="cube") -> System:
    """Atoms uniform in [0, edge]^3 with minimum separation dmin (rejection sampling)."""
    rng = np.random.default_rng(seed)
    lo, hi = np.zeros(3), np.full(3, edge)
    pts = _rsa(rng, n_atoms, lambda: rng.uniform(0.0, edge, 3), lo, hi, dmin)
    a0, c6, rv, vr = draw_params(rng, n_atoms)
    return System(pts, a0, c6, rv, vr, name=name,
                  meta=dict(edge=edge, dmin=dmin, seed=seed))


def sphere_cluster(n_atoms=2000, density=DENSITY_CLUSTER, dmin=2.2, seed=1000,
                   name="sphere") -> System:
    """Random sequential addition in a sphere of radius (3N/(4 pi rho))^(1/3)."""
    rng = np.random.default_rng(seed)
    radius = (3.0 * n_atoms / (4.0 * math.pi * density)) ** (1.0 / 3.0)

    def sample():
        while True:
            p = rng.uniform(-radius, radius, 3)
            if p @ p <= radius * radius:
                return p

    pts = _rsa(rng, n_atoms, sample, np.full(3, -radius), np.full(3, radius), dmin)
    a0, c6, rv, vr = draw_params(rng, n_atoms)
    return System(pts, a0, c6, rv, vr, name=name,
                  meta=dict(radius=radius, density=density, dmin=dmin, seed=seed))


def fcc_jitter_cluster(n_atoms=400, density=0.08, jitter=0.2, seed=1099,
                       name="fcc-dense") -> System:
    """Jittered FCC ball at `density` atoms/bohr^3 (the literal high-density reading
    of the N=2000 cluster, kept as a negative case)."""
    rng = np.random.default_rng(seed)
    a = (4.0 / density) ** (1.0 / 3.0)
    m = int(math.ceil((n_atoms / 4.0) ** (1.0 / 3.0))) + 3
    basis = np.array([[0, 0, 0], [0.5, 0.5, 0], [0.5, 0, 0.5], [0, 0.5, 0.5]])
    g = np.arange(-m, m + 1)
    cells = np.array(np.meshgrid(g, g, g, indexing="ij")).reshape(3, -1).T
    lat = (cells[:, None, :] + basis[None, :, :]).reshape(-1, 3) * a
    order = np.argsort(np.einsum("ij,ij->i", lat, lat), kind="stable")
    pts = lat[order[:n_atoms]] + rng.uniform(-jitter, jitter, (n_atoms, 3))
    a0, c6, rv, vr = draw_params(rng, n_atoms)
    return System(pts, a0, c6, rv, vr, name=name,
                  meta=dict(density=density, jitter=jitter, seed=seed))


def triclinic_cell(n_atoms=256, edge=(20.0, 26.0), angle=(80.0, 100.0), dmin=2.5,
                   k_grid=(4, 4, 4), seed=2000, name="cell") -> System:
    """Triclinic cell: edges U[edge], angles U[angle] degrees, a along x, b in the
    xy plane; atoms uniform in fractional coordinates with minimum-image separation
    at least dmin."""
    rng = np.random.default_rng(seed)
    la, lb, lc = rng.uniform(*edge, 3)
    al, be, ga = np.radians(rng.uniform(*angle, 3))
    ax = np.array([la, 0.0, 0.0])
    bx = np.array([lb * math.cos(ga), lb * math.sin(ga), 0.0])
    cx_ = lc * math.cos(be)
    cy_ = lc * (math.cos(al) - math.cos(be) * math.cos(ga)) / math.sin(ga)
    cz_ = math.sqrt(max(lc * lc - cx_ * cx_ - cy_ * cy_, 1e-12))
    A = np.array([ax, bx, [cx_, cy_, cz_]])
    frac = np.zeros((n_atoms, 3))
    shifts = np.array(np.meshgrid([-1, 0, 1], [-1, 0, 1], [-1, 0, 1],
                                  indexing="ij")).reshape(3, -1).T @ A
    k = tries = 0
    while k < n_atoms:
        tries += 1
        if tries > 2_000_000:
            raise RuntimeError("cell packing jammed")
        f = rng.uniform(0.0, 1.0, 3)
        if k:
            d = (frac[:k] - f)
            d -= np.round(d)
            cart = d @ A
            dd = cart[:, None, :] + shifts[None, :, :]
            if np.min(np.einsum("ijk,ijk->ij", dd, dd)) < dmin * dmin:
                continue
        frac[k] = f
        k += 1
    a0, c6, rv, vr = draw_params(rng, n_atoms)
    return System(frac @ A, a0, c6, rv, vr, lattice=A, k_grid=tuple(k_grid), name=name,
                  meta=dict(seed=seed, dmin=dmin))


def cluster_batch(n_clusters=4096, n_range=(50, 500), density=DENSITY_CLUSTER, dmin=2.2,
                  seed0=4000):
    """Varlen batch of sphere clusters, cluster i seeded 4000 + i, size U{lo..hi}."""
    sizes = np.random.default_rng(seed0 - 1).integers(n_range[0], n_range[1] + 1, n_clusters)
    return [sphere_cluster(int(s), density, dmin, seed0 + i, name=f"cl{i}")
            for i, s in enumerate(sizes)]


# The named workloads (sizes as the paper-shaped benchmark configurations).
def workload(name: str, instance: int = 0) -> System:
    if name == "finite32":      # N=32 in a 14 bohr cube, min separation 2.5
        return cube_cluster(32, 14.0, 2.5, seed=0 * 1000 + instance, name=name)
    if name == "finite2000":    # N=2000 sphere, 0.08 atoms/A^3, min separation 2.2
        return sphere_cluster(2000, DENSITY_CLUSTER, 2.2, seed=1000 + instance, name=name)
    if name == "cell256":       # 256-atom triclinic cell, 4x4x4 k-grid
        return triclinic_cell(256, seed=2000 + instance, name=name)
    if name == "finite8000":    # N=8000 sphere at the cluster density
        return sphere_cluster(8000, DENSITY_CLUSTER, 2.2, seed=3000 + instance, name=name)
    raise KeyError(name)

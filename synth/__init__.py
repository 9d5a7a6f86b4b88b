"""Seeded synthetic inputs for the Moment Tensor Potential workloads.

This module only draws numbers and builds geometry (lattices, displacements,
species labels, periodic cells, raw random coefficients).  It holds none of
the potential's arithmetic: no radial basis, no moments, no contractions.
Both the CUDA path and the oracle are fed from here.

Cell convention: ``cell`` is a 3x3 float64 array whose ROWS are the lattice
vectors a, b, c (LAMMPS lower-triangular form for generated triclinic cells).
Positions are Cartesian, in Angstrom, wrapped into the cell.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

BASE_SEED = 20251000


def rng(stream: int, sub: int = 0) -> np.random.Generator:
    """PCG64 generator for workload ``stream`` and sub-stream ``sub``."""
    return np.random.Generator(np.random.PCG64(np.random.SeedSequence([BASE_SEED + stream, sub])))


@dataclasses.dataclass
class Structure:
    x: np.ndarray          # [N, 3] float64, Cartesian, wrapped into the cell
    z: np.ndarray          # [N] int32 species index (0-based)
    cell: np.ndarray       # [3, 3] float64, rows = lattice vectors
    pbc: tuple = (1, 1, 1)

    @property
    def n(self) -> int:
        return int(self.x.shape[0])


_BASIS = {
    "bcc": np.array([[0.0, 0.0, 0.0], [0.5, 0.5, 0.5]]),
    "fcc": np.array([[0.0, 0.0, 0.0], [0.0, 0.5, 0.5], [0.5, 0.0, 0.5], [0.5, 0.5, 0.0]]),
}


def lattice(kind: str, cells: tuple, a: float) -> tuple[np.ndarray, np.ndarray]:
    """Undisplaced cubic lattice of ``cells`` = (n1, n2, n3) unit cells; atom
    order is cell-major (i1 slowest), basis atom fastest."""
    n1, n2, n3 = cells
    b = _BASIS[kind]
    g = np.stack(np.meshgrid(np.arange(n1), np.arange(n2), np.arange(n3), indexing="ij"), -1).reshape(-1, 3)
    frac = (g[:, None, :] + b[None, :, :]).reshape(-1, 3)
    cell = np.diag([n1 * a, n2 * a, n3 * a]).astype(np.float64)
    return frac * a, cell


def wrap(x: np.ndarray, cell: np.ndarray) -> np.ndarray:
    """Wrap Cartesian positions into the parallelepiped spanned by the cell rows."""
    s = x @ np.linalg.inv(cell)
    s = s - np.floor(s)
    s[s >= 1.0] = 0.0
    return s @ cell


def balanced_species(n: int, n_species: int, g: np.random.Generator) -> np.ndarray:
    """Random permutation of balanced labels (counts differ by at most one)."""
    lab = np.arange(n) % n_species
    return g.permutation(lab).astype(np.int32)


def crystal(kind: str, cells: tuple, a: float, sigma: float, n_species: int, stream: int,
            sub: int = 0) -> Structure:
    """Lattice with i.i.d. Gaussian displacements (std ``sigma`` per Cartesian
    component), wrapped into the cell, with balanced random species."""
    x0, cell = lattice(kind, cells, a)
    g = rng(stream, 10 + sub)
    x = x0 + g.normal(0.0, sigma, size=x0.shape)
    z = balanced_species(x.shape[0], n_species, rng(stream, 20 + sub))
    return Structure(wrap(x, cell), z, cell)


def random_triclinic_cell(n_atoms: int, density: float, g: np.random.Generator) -> np.ndarray:
    """Lower-triangular cell: diagonal aspect ratios U[0.8, 1.25], tilts
    U[-0.3, 0.3] times the matching diagonal, scaled to volume n/density."""
    d = g.uniform(0.8, 1.25, size=3)
    xy = g.uniform(-0.3, 0.3) * d[0]
    xz = g.uniform(-0.3, 0.3) * d[0]
    yz = g.uniform(-0.3, 0.3) * d[1]
    h = np.array([[d[0], 0.0, 0.0], [xy, d[1], 0.0], [xz, yz, d[2]]])
    vol = n_atoms / density
    h *= (vol / abs(np.linalg.det(h))) ** (1.0 / 3.0)
    return h


def _image_shifts(cell: np.ndarray, reach: int) -> np.ndarray:
    r = np.arange(-reach, reach + 1)
    n = np.stack(np.meshgrid(r, r, r, indexing="ij"), -1).reshape(-1, 3).astype(np.float64)
    return n @ cell


def random_gas(n_atoms: int, density: float, min_sep: float, n_species: int, g: np.random.Generator,
               max_attempts: int = 400000, chunk: int = 256) -> Structure | None:
    """Random sequential insertion in a random triclinic cell, rejecting any
    trial point closer than ``min_sep`` to an accepted one under every
    periodic image.  Trial points are drawn ``chunk`` at a time (the same
    sequence as one at a time).  Distances use the fractional difference
    wrapped to [-0.5, 0.5] plus the images n in [-R, R]^3 with
    R = floor(0.5 + min_sep / h_min), h_min the smallest plane spacing: every
    image closer than min_sep lies in that set.  Returns None if the attempt
    budget runs out."""
    cell = random_triclinic_cell(n_atoms, density, g)
    inv = np.linalg.inv(cell)
    heights = 1.0 / np.linalg.norm(inv, axis=0)
    reach = int(math.floor(0.5 + min_sep / heights.min()))
    r = np.arange(-reach, reach + 1)
    imgs = np.stack(np.meshgrid(r, r, r, indexing="ij"), -1).reshape(-1, 3).astype(np.float64)
    lim = min_sep * min_sep
    acc = np.zeros((n_atoms, 3))        # fractional coordinates of accepted points
    count = 0
    attempts = 0

    def dist2(tr, pts):
        d = tr[:, None, :] - pts[None, :, :]
        d -= np.round(d)
        v = (d[:, :, None, :] + imgs[None, None, :, :]) @ cell
        return np.einsum("tpsk,tpsk->tps", v, v).min(axis=(1, 2))

    while count < n_atoms:
        if attempts >= max_attempts:
            return None
        trials = g.uniform(0.0, 1.0, size=(chunk, 3))
        best = dist2(trials, acc[:count]) if count else np.full(chunk, np.inf)
        for t in range(chunk):
            attempts += 1
            if best[t] < lim:
                continue
            acc[count] = trials[t]
            count += 1
            if count == n_atoms or attempts >= max_attempts:
                break
            if t + 1 < chunk:
                best[t + 1:] = np.minimum(best[t + 1:], dist2(trials[t + 1:], trials[t:t + 1]))
    z = balanced_species(n_atoms, n_species, g)
    return Structure(wrap(acc @ cell, cell), z, cell)


def _gas_job(args):
    stream, k, n, density, min_sep, n_species = args
    gk = rng(stream, 1000 + k)
    s = None
    while s is None:
        s = random_gas(int(n), density, min_sep, n_species, gk)
    return s


def batch_sizes(n_cfg: int, lo: int, hi: int, g: np.random.Generator) -> np.ndarray:
    """Configuration sizes floor(exp(U[ln lo, ln (hi+1))))."""
    return np.floor(np.exp(g.uniform(math.log(lo), math.log(hi + 1), size=n_cfg))).astype(np.int64)


def random_gas_batch(n_cfg: int, lo: int, hi: int, density: float, min_sep: float, n_species: int,
                     stream: int, workers: int = 0) -> list[Structure]:
    """Batch of random periodic gases with log-uniform sizes; each
    configuration has its own sub-stream, and a failed insertion is redrawn
    from it.  ``workers`` > 1 generates in that many spawned processes (the
    result does not depend on it); 0 = one per CPU core for large batches."""
    g = rng(stream, 30)
    sizes = batch_sizes(n_cfg, lo, hi, g)
    jobs = [(stream, k, int(n), density, min_sep, n_species) for k, n in enumerate(sizes)]
    if workers == 0:
        import os
        workers = (os.cpu_count() or 1) if n_cfg >= 64 else 1
    if workers <= 1:
        return [_gas_job(j) for j in jobs]
    import multiprocessing as mp
    with mp.get_context("spawn").Pool(workers) as pool:
        return pool.map(_gas_job, jobs, chunksize=max(1, n_cfg // (8 * workers)))


@dataclasses.dataclass
class RawPotential:
    """Random coefficients before any normalisation.

    radial[mu, k, zi, zj]: Chebyshev coefficients of radial function mu for an
    ordered species pair; species_energy[z]; xi_raw[alpha] linear coefficients.
    """
    level: int
    n_species: int
    n_q: int
    r_min: float
    r_cut: float
    n_mu: int
    species_energy: np.ndarray
    radial: np.ndarray
    xi_raw: np.ndarray


def raw_potential(level: int, n_species: int, n_q: int, r_min: float, r_cut: float, n_mu: int,
                  m: int, stream: int) -> RawPotential:
    """c ~ N(0, 0.1^2), species energies ~ N(0, 1), xi ~ N(0, 0.1^2)."""
    g = rng(stream, 40)
    radial = g.normal(0.0, 0.1, size=(n_mu, n_q, n_species, n_species))
    s = rng(stream, 41).normal(0.0, 1.0, size=n_species)
    xi = rng(stream, 42).normal(0.0, 0.1, size=m)
    return RawPotential(level, n_species, n_q, r_min, r_cut, n_mu, s, radial, xi)


def random_neighbourhoods(n_hoods: int, n_nb: int, n_mu: int, g: np.random.Generator):
    """Random unit vectors (uniform on the sphere) and free radial values per
    neighbour, used to probe linear dependence among basis functions."""
    v = g.normal(size=(n_hoods, n_nb, 3))
    v /= np.linalg.norm(v, axis=-1, keepdims=True)
    f = g.normal(size=(n_hoods, n_nb, n_mu))
    return v, f


def target_forces(n: int, stream: int) -> np.ndarray:
    """Seeded target forces ~ N(0, 0.5^2) eV/A per component."""
    return rng(stream, 50).normal(0.0, 0.5, size=(n, 3))

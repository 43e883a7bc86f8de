"""Seeded synthetic crystal-structure batches.

This module draws inputs only: lattices, atom lists, scattering-coefficient
tables and option sets. It holds none of the diffraction arithmetic, so both
the CUDA path and the FP64 oracle can be fed the same bytes from it.

The five workloads stand in for the paper's MC3D and COD benchmark sets
(Sec. 4), which are not available here:

* ``nacl``     -- rock-salt NaCl, a = 5.64 A, conventional cell of 8 atoms.
* ``small``    -- 1024 P1 cells, edges 3-15 A, 1-64 atoms (MC3D-like sizes,
                  the paper's MC3D set holds 1-80 atoms, Sec. 4.1).
* ``large``    -- 256 P1 cells, edges 15-40 A, 200-2000 atoms, 20 % partially
                  occupied sites (COD-like large cells, Sec. 3 and 4.2).
* ``mixed``    -- 100 000 cells, lognormal atom counts (median 20) and edges
                  (median 7 A): spans all reflection-count bins of Sec. 4.2.
* ``stress``   -- one 50 A cell of 940 atoms at Mo K-alpha, 2-theta 2-60 deg
                  (about 600 000 Friedel-unique reflections): the shape of the
                  largest single structure of Sec. 4.2.
* ``grad``     -- 512 cells of 8-128 atoms for the broadened-pattern gradient.
* ``hexdis``   -- 256 cells, half hexagonal (a = b U[2.5, 6] A, c U[3, 12] A,
                  gamma 120 deg) and half P1, 2-24 sites each, a third of the
                  sites shared by 2-3 species with occupancies summing to 1
                  (real COD/MC3D entries carry both: Sec. 1 inputs).
* ``augment``  -- per-structure experimental effects of ML training patterns
                  (Sec. 1): pseudo-Voigt FWHM 0.05-0.3 deg and mixing 0-1,
                  March-Dollase r 0.6-1.4 about a low-index direction, noise
                  scale 0-1 with standard normal draws.

All arrays follow the C ABI layout: ``lattice`` float64 [n, 6] (a, b, c in
angstrom; alpha, beta, gamma in degrees), ``atom_off`` int64 [n + 1],
``frac`` float64 [N, 3], ``Z`` int16 [N], ``occ`` float64 [N], ``B`` float64
[N] (angstrom^2), ``coef`` float64 [zmax + 1, 4, 2] holding (a_i, b_i).
"""
from __future__ import annotations

import dataclasses
import numpy as np

ZMAX = 83
CU_KA = 1.54184
MO_KA = 0.71073


@dataclasses.dataclass
class Batch:
    lattice: np.ndarray
    atom_off: np.ndarray
    frac: np.ndarray
    Z: np.ndarray
    occ: np.ndarray
    B: np.ndarray
    coef: np.ndarray
    zmax: int = ZMAX

    @property
    def n_struct(self) -> int:
        return int(self.lattice.shape[0])

    @property
    def n_atoms(self) -> int:
        return int(self.frac.shape[0])

    def atoms_of(self, s: int) -> slice:
        return slice(int(self.atom_off[s]), int(self.atom_off[s + 1]))

    def subset(self, idx) -> "Batch":
        """Batch made of the structures ``idx`` (in that order)."""
        idx = np.asarray(idx, dtype=np.int64)
        parts = [np.arange(self.atom_off[s], self.atom_off[s + 1]) for s in idx]
        sel = np.concatenate(parts) if parts else np.zeros(0, np.int64)
        counts = np.array([len(p) for p in parts], dtype=np.int64)
        off = np.zeros(len(idx) + 1, dtype=np.int64)
        off[1:] = np.cumsum(counts)
        return Batch(self.lattice[idx].copy(), off, self.frac[sel].copy(), self.Z[sel].copy(),
                     self.occ[sel].copy(), self.B[sel].copy(), self.coef, self.zmax)


@dataclasses.dataclass
class Opts:
    wavelength: float = CU_KA
    tt_min: float = 0.0
    tt_max: float = 90.0
    tt_tol: float = 1e-5
    rel_cutoff: float = 1e-3
    scaled: int = 1
    point_group: object = None  # operations [n][3][3] on (h, k, l): families by its orbits (None: default)


def coef_table(rng: np.random.Generator, zmax: int = ZMAX) -> np.ndarray:
    """One (a_i, b_i) set per element, a_i ~ U[0.5, 4], b_i ~ U[0.5, 50]."""
    t = np.zeros((zmax + 1, 4, 2), dtype=np.float64)
    t[1:, :, 0] = rng.uniform(0.5, 4.0, size=(zmax, 4))
    t[1:, :, 1] = rng.uniform(0.5, 50.0, size=(zmax, 4))
    return t


def _volume_factor(ang_deg: np.ndarray) -> np.ndarray:
    c = np.cos(np.radians(ang_deg))
    return 1.0 - (c ** 2).sum(axis=1) + 2.0 * c.prod(axis=1)


def _angles(rng: np.random.Generator, n: int, lo=60.0, hi=120.0, min_factor=0.1) -> np.ndarray:
    """Uniform cell angles, redrawing cells whose volume factor is below ``min_factor``."""
    ang = rng.uniform(lo, hi, size=(n, 3))
    bad = _volume_factor(ang) < min_factor
    while bad.any():
        ang[bad] = rng.uniform(lo, hi, size=(int(bad.sum()), 3))
        bad = _volume_factor(ang) < min_factor
    return ang


def _atoms(rng, counts, bmax, partial=False):
    n = int(counts.sum())
    off = np.zeros(len(counts) + 1, dtype=np.int64)
    off[1:] = np.cumsum(counts)
    frac = rng.random(size=(n, 3))
    Z = rng.integers(1, ZMAX + 1, size=n).astype(np.int16)
    B = rng.uniform(0.0, bmax, size=n)
    occ = np.ones(n)
    if partial:
        part = rng.random(n) < 0.2
        occ[part] = rng.uniform(0.5, 1.0, size=int(part.sum()))
    return off, frac, Z, occ, B


def hexdis(seed: int = 8, n: int = 256) -> tuple[Batch, Opts]:
    """Hexagonal and P1 cells whose sites may be shared by several species.

    A shared site is one atom record per species at the same coordinates, with
    the species' occupancies (Dirichlet(1, ..)) summing to 1 and one B per record.
    """
    rng = np.random.default_rng(seed)
    coef = coef_table(rng)
    lat = np.zeros((n, 6))
    for s in range(n):
        if s % 2 == 0:
            a = rng.uniform(2.5, 6.0)
            lat[s] = [a, a, rng.uniform(3.0, 12.0), 90.0, 90.0, 120.0]
        else:
            lat[s, :3] = rng.uniform(3.0, 10.0, 3)
            lat[s, 3:] = _angles(rng, 1)[0]
    frac, Z, occ, B, counts = [], [], [], [], []
    for s in range(n):
        n_sites = int(rng.integers(2, 25))
        c = 0
        for _ in range(n_sites):
            x = rng.random(3)
            k = int(rng.integers(2, 4)) if rng.random() < 1.0 / 3.0 else 1
            w = rng.dirichlet(np.ones(k)) if k > 1 else np.ones(1)
            for j in range(k):
                frac.append(x)
                Z.append(rng.integers(1, ZMAX + 1))
                occ.append(w[j])
                B.append(rng.uniform(0.0, 1.5))
            c += k
        counts.append(c)
    off = np.zeros(n + 1, dtype=np.int64)
    off[1:] = np.cumsum(counts)
    return (Batch(lat, off, np.array(frac), np.array(Z, dtype=np.int16), np.array(occ), np.array(B), coef),
            Opts(CU_KA, 5.0, 110.0, 1e-5, 1e-3, 1))


def nacl(seed: int = 1) -> tuple[Batch, Opts]:
    """Rock salt: Na on the fcc sites, Cl shifted by (1/2, 0, 0); occ 1, B = 0.5."""
    rng = np.random.default_rng(seed)
    coef = coef_table(rng)
    fcc = np.array([[0, 0, 0], [0, .5, .5], [.5, 0, .5], [.5, .5, 0]], dtype=np.float64)
    cl = (fcc + np.array([.5, 0, 0])) % 1.0
    frac = np.vstack([fcc, cl])
    Z = np.array([11] * 4 + [17] * 4, dtype=np.int16)
    b = Batch(np.array([[5.64, 5.64, 5.64, 90.0, 90.0, 90.0]]), np.array([0, 8], dtype=np.int64),
              frac, Z, np.ones(8), np.full(8, 0.5), coef)
    return b, Opts(CU_KA, 0.0, 90.0, 1e-5, 1e-3, 1)


def small(seed: int = 2, n: int = 1024) -> tuple[Batch, Opts]:
    rng = np.random.default_rng(seed)
    coef = coef_table(rng)
    edges = rng.uniform(3.0, 15.0, size=(n, 3))
    ang = _angles(rng, n)
    counts = rng.integers(1, 65, size=n)
    off, frac, Z, occ, B = _atoms(rng, counts, 2.0)
    return Batch(np.hstack([edges, ang]), off, frac, Z, occ, B, coef), Opts(CU_KA, 0.0, 90.0)


def large(seed: int = 3, n: int = 256) -> tuple[Batch, Opts]:
    rng = np.random.default_rng(seed)
    coef = coef_table(rng)
    edges = rng.uniform(15.0, 40.0, size=(n, 3))
    ang = _angles(rng, n)
    counts = rng.integers(200, 2001, size=n)
    off, frac, Z, occ, B = _atoms(rng, counts, 3.0, partial=True)
    return Batch(np.hstack([edges, ang]), off, frac, Z, occ, B, coef), Opts(CU_KA, 5.0, 120.0)


def stress(seed: int = 9, n: int = 1) -> tuple[Batch, Opts]:
    """The shape of the largest single-structure case of Sec. 4.2 (a COD entry with a ~50 A cell,
    940 atoms and more than 600 000 reflections at Mo K-alpha, 2-theta 2-60 deg): edges 50 A,
    angles U[60, 120] deg (volume-factor rejection), 940 atoms, Z U{1..83}, B U[0, 3] A^2, 20 %
    of sites with occ U[0.5, 1]; lambda 0.71073 A, 2-theta 2-60 deg."""
    rng = np.random.default_rng(seed)
    coef = coef_table(rng)
    edges = np.full((n, 3), 50.0)
    ang = _angles(rng, n)
    off, frac, Z, occ, B = _atoms(rng, np.full(n, 940), 3.0, partial=True)
    return Batch(np.hstack([edges, ang]), off, frac, Z, occ, B, coef), Opts(MO_KA, 2.0, 60.0)


def mixed(seed: int = 4, n: int = 100_000) -> tuple[Batch, Opts]:
    rng = np.random.default_rng(seed)
    coef = coef_table(rng)
    counts = np.clip(np.rint(np.exp(np.log(20.0) + 1.0 * rng.standard_normal(n))), 1, 500).astype(np.int64)
    edges = np.clip(np.exp(np.log(7.0) + 0.5 * rng.standard_normal((n, 3))), 3.0, 30.0)
    ang = _angles(rng, n)
    off, frac, Z, occ, B = _atoms(rng, counts, 2.0)
    return Batch(np.hstack([edges, ang]), off, frac, Z, occ, B, coef), Opts(CU_KA, 0.0, 90.0)


@dataclasses.dataclass
class Grid:
    """Uniform 2-theta grid t_k = t0 + k * dt, k = 0 .. n_pts - 1, Gaussian FWHM in degrees."""
    t0: float = 5.0
    dt: float = 85.0 / 4095.0
    n_pts: int = 4096
    fwhm: float = 0.1


def grad(seed: int = 5, n: int = 512) -> tuple[Batch, Batch, Opts, Grid]:
    """Structures plus a perturbed copy used as the fitting target.

    Target: coordinates + N(0, 0.01) wrapped into [0, 1), B + U(-0.1, 0.1)
    clipped at 0, edges x (1 + U(-0.005, 0.005)), angles + U(-0.2, 0.2) deg.
    """
    rng = np.random.default_rng(seed)
    coef = coef_table(rng)
    edges = rng.uniform(3.0, 15.0, size=(n, 3))
    ang = _angles(rng, n)
    counts = rng.integers(8, 129, size=n)
    off, frac, Z, occ, B = _atoms(rng, counts, 2.0)
    base = Batch(np.hstack([edges, ang]), off, frac, Z, occ, B, coef)
    tf = (frac + rng.normal(0.0, 0.01, size=frac.shape)) % 1.0
    tB = np.clip(B + rng.uniform(-0.1, 0.1, size=B.shape), 0.0, None)
    te = edges * (1.0 + rng.uniform(-0.005, 0.005, size=edges.shape))
    ta = ang + rng.uniform(-0.2, 0.2, size=ang.shape)
    target = Batch(np.hstack([te, ta]), off.copy(), tf, Z.copy(), occ.copy(), tB, coef)
    return base, target, Opts(CU_KA, 5.0, 90.0, 1e-5, 0.0, 0), Grid()


@dataclasses.dataclass
class Augment:
    """Experimental effects per structure: fwhm, eta, po_r, noise_sigma float64 [n]; po_dir float64 [n, 3]
    (reciprocal-lattice components); z float32 [n, n_pts] standard normal draws."""
    fwhm: np.ndarray
    eta: np.ndarray
    po_dir: np.ndarray
    po_r: np.ndarray
    noise_sigma: np.ndarray
    z: np.ndarray


def augment(n: int, n_pts: int, seed: int = 6) -> Augment:
    rng = np.random.default_rng(seed)
    d = rng.integers(-2, 3, size=(n, 3)).astype(np.float64)
    d[~d.any(axis=1), 2] = 1.0  # never the zero direction
    return Augment(rng.uniform(0.05, 0.3, n), rng.uniform(0.0, 1.0, n), d, rng.uniform(0.6, 1.4, n),
                   rng.uniform(0.0, 1.0, n), rng.standard_normal((n, n_pts)).astype(np.float32))


def random_cell(rng: np.random.Generator, n_atoms: int, edge=(3.0, 15.0), bmax=2.0, zs=None) -> Batch:
    """One seeded P1 cell, for small ad-hoc test cases."""
    edges = rng.uniform(*edge, size=(1, 3))
    ang = _angles(rng, 1)
    off, frac, Z, occ, B = _atoms(rng, np.array([n_atoms]), bmax)
    if zs is not None:
        Z = np.asarray(zs, dtype=np.int16)
    return Batch(np.hstack([edges, ang]), off, frac, Z, occ, B, coef_table(rng))


def concat(batches: list[Batch]) -> Batch:
    """Concatenate batches that share one coefficient table."""
    coef = batches[0].coef
    lat = np.vstack([b.lattice for b in batches])
    counts = np.concatenate([np.diff(b.atom_off) for b in batches])
    off = np.zeros(len(counts) + 1, dtype=np.int64)
    off[1:] = np.cumsum(counts)
    return Batch(lat, off, np.vstack([b.frac for b in batches]), np.concatenate([b.Z for b in batches]),
                 np.concatenate([b.occ for b in batches]), np.concatenate([b.B for b in batches]), coef)


WORKLOADS = {"nacl": nacl, "small": small, "large": large, "mixed": mixed}

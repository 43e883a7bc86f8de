"""Calculator-style front end in the shape of the pymatgen XRD calculator (the
Python interface the paper keeps, Sec. 2, Fig. 1): structures in, per-structure
patterns out (x = 2-theta of each peak, y = intensity, hkls = families with
multiplicities, d_hkls), every pattern of a call computed in one batched GPU
pass through the C ABI.

Structures are accepted as plain dicts
    {"lattice": (a, b, c, alpha, beta, gamma), "sites": [{"species": {"Fe": 0.5, "Co": 0.5},
                                                          "frac": (x, y, z)}, ...]}
or as objects with the attributes of a pymatgen Structure (lattice.abc,
lattice.angles, sites[i].frac_coords, sites[i].species as a mapping from an
element -- a symbol string or an object with .symbol -- to its occupancy).
A site shared by several species becomes one atom record per species.
pymatgen itself is not needed. Its atomic scattering-factor table is not
shipped here, so the caller passes the coefficient table (a_i, b_i) per element.

Hexagonal cells (the library sets xrd.XRD_FLAG_HEXAGONAL in the structure's
flag word) report 4-index (h, k, i, l) families, as the pymatgen calculator does.
"""
from __future__ import annotations

import dataclasses

import numpy as np

from . import xrd

# element symbols by atomic number (Z = 1 .. 83)
ELEMENTS = ("H He Li Be B C N O F Ne Na Mg Al Si P S Cl Ar K Ca Sc Ti V Cr Mn Fe Co Ni Cu Zn Ga Ge As Se Br Kr "
            "Rb Sr Y Zr Nb Mo Tc Ru Rh Pd Ag Cd In Sn Sb Te I Xe Cs Ba La Ce Pr Nd Pm Sm Eu Gd Tb Dy Ho Er Tm Yb "
            "Lu Hf Ta W Re Os Ir Pt Au Hg Tl Pb Bi").split()
Z_OF = {sym: z for z, sym in enumerate(ELEMENTS, start=1)}

# characteristic X-ray wavelengths in angstrom (K-alpha: intensity-weighted mean of alpha1 and alpha2)
WAVELENGTHS = {
    "CuKa": 1.54184, "CuKa1": 1.54056, "CuKa2": 1.54439, "CuKb1": 1.39222,
    "MoKa": 0.71073, "MoKa1": 0.70930, "MoKa2": 0.71359,
    "CoKa": 1.79026, "CoKa1": 1.78896,
    "FeKa": 1.93735, "FeKa1": 1.93604,
    "CrKa": 2.29100, "CrKa1": 2.28970,
    "AgKa": 0.560885, "AgKa1": 0.559421,
}


# Generators of the Laue groups as operations on reflection indices (h, k, l) (column vector);
# hexagonal and trigonal groups in hexagonal axes. laue_group_ops closes them under products
# (with the inversion), giving the point group that xrd_set_point_group takes.
_E = ((1, 0, 0), (0, 1, 0), (0, 0, 1))
_C2B = ((-1, 0, 0), (0, 1, 0), (0, 0, -1))  # 2-fold about b (monoclinic unique axis b)
_MX = ((-1, 0, 0), (0, 1, 0), (0, 0, 1))    # h -> -h
_MY = ((1, 0, 0), (0, -1, 0), (0, 0, 1))    # k -> -k
_C4 = ((0, -1, 0), (1, 0, 0), (0, 0, 1))    # 4-fold about c
_SW = ((0, 1, 0), (1, 0, 0), (0, 0, 1))     # h <-> k
_C3D = ((0, 0, 1), (1, 0, 0), (0, 1, 0))    # 3-fold about [111]
_C6 = ((0, -1, 0), (1, 1, 0), (0, 0, 1))    # 6-fold about c, hexagonal axes: (h, k, l) -> (-k, h + k, l)
_C3 = ((-1, -1, 0), (1, 0, 0), (0, 0, 1))   # 3-fold about c, hexagonal axes
LAUE_GENERATORS = {
    "-1": (), "2/m": (_C2B,), "mmm": (_MX, _MY), "4/m": (_C4,), "4/mmm": (_C4, _SW),
    "-3": (_C3,), "-3m": (_C3, _SW), "6/m": (_C6,), "6/mmm": (_C6, _SW), "m-3": (_MX, _MY, _C3D),
    "m-3m": (_C4, _C3D),
}


def laue_group_ops(name: str) -> np.ndarray:
    """Operations [n][3][3] of a Laue group (a key of LAUE_GENERATORS): the closure of its
    generators and the inversion under matrix products."""
    gens = [np.array(g, dtype=np.int64) for g in LAUE_GENERATORS[name]] + [-np.eye(3, dtype=np.int64)]
    ops = {tuple(np.eye(3, dtype=np.int64).ravel())}
    frontier = [np.eye(3, dtype=np.int64)]
    while frontier:
        nxt = []
        for m in frontier:
            for g in gens:
                p = g @ m
                t = tuple(p.ravel())
                if t not in ops:
                    ops.add(t)
                    nxt.append(p)
        frontier = nxt
    return np.array(sorted(ops), dtype=np.int32).reshape(-1, 3, 3)


@dataclasses.dataclass
class DiffractionPattern:
    x: np.ndarray        # 2-theta of each peak, degrees, ascending
    y: np.ndarray        # intensity (0-100 when scaled)
    hkls: list           # per peak: [{"hkl": tuple, "multiplicity": int}, ...]
    d_hkls: np.ndarray   # d spacing of each peak, angstrom
    status: int = 0      # XRD_OK, or the library's per-structure error code


def _symbol(sp) -> str:
    s = getattr(sp, "symbol", None)
    if s is None:
        s = str(sp)
    s = "".join(ch for ch in s if ch.isalpha())  # "Fe2+" -> "Fe"
    return s


def structure_arrays(structure, debye_waller_factors=None):
    """(lattice[6], frac[N][3], Z[N], occ[N], B[N]) of one structure (one record per species on each site)."""
    dw = debye_waller_factors or {}
    if isinstance(structure, dict):
        lat = np.asarray(structure["lattice"], dtype=np.float64)
        sites = [(s["species"], s["frac"]) for s in structure["sites"]]
    else:
        lat = np.asarray(tuple(structure.lattice.abc) + tuple(structure.lattice.angles), dtype=np.float64)
        sites = [(site.species, site.frac_coords) for site in structure.sites]
    frac, Z, occ, B = [], [], [], []
    for species, x in sites:
        items = species.items() if hasattr(species, "items") else [(species, 1.0)]
        for sp, amount in items:
            sym = _symbol(sp)
            if sym not in Z_OF:
                raise ValueError("element %r is outside Z = 1 .. %d" % (sym, len(ELEMENTS)))
            frac.append(np.asarray(x, dtype=np.float64))
            Z.append(Z_OF[sym])
            occ.append(float(amount))
            B.append(float(dw.get(sym, 0.0)))
    return (lat.reshape(6), np.asarray(frac, dtype=np.float64).reshape(-1, 3), np.asarray(Z, dtype=np.int16),
            np.asarray(occ, dtype=np.float64), np.asarray(B, dtype=np.float64))


def batch_of(structures, coef, debye_waller_factors=None):
    """A host batch (the layout the C ABI takes) of several structures."""
    from .synth import Batch
    parts = [structure_arrays(s, debye_waller_factors) for s in structures]
    counts = np.array([len(p[2]) for p in parts], dtype=np.int64)
    off = np.zeros(len(parts) + 1, dtype=np.int64)
    off[1:] = np.cumsum(counts)
    coef = np.ascontiguousarray(coef, dtype=np.float64)
    zmax = coef.shape[0] - 1
    Z = np.concatenate([p[2] for p in parts]) if parts else np.zeros(0, np.int16)
    if len(Z) and int(Z.max()) > zmax:
        raise ValueError("the coefficient table stops at Z = %d" % zmax)
    return Batch(np.vstack([p[0] for p in parts]) if parts else np.zeros((0, 6)), off,
                 np.vstack([p[1] for p in parts]) if parts else np.zeros((0, 3)), Z,
                 np.concatenate([p[3] for p in parts]) if parts else np.zeros(0),
                 np.concatenate([p[4] for p in parts]) if parts else np.zeros(0), coef, zmax)


def patterns_from(res):
    """DiffractionPattern objects from the per-structure results of xrd.compute; the library's flag
    word says which structures report Miller-Bravais (4-index) families."""
    hexa = (np.asarray(res["flags"]) & xrd.XRD_FLAG_HEXAGONAL) != 0
    out = []
    for s in range(len(res["peak_tt"])):
        fo, hkl, mult = res["peak_fam_off"][s], res["fam_hkl"][s], res["fam_mult"][s]
        if hexa[s] and len(hkl):
            hkl = xrd.miller_bravais(hkl)
        fams = [[{"hkl": tuple(int(v) for v in hkl[f]), "multiplicity": int(mult[f])} for f in range(fo[p], fo[p + 1])]
                for p in range(len(res["peak_tt"][s]))]
        out.append(DiffractionPattern(np.asarray(res["peak_tt"][s]), np.asarray(res["peak_I"][s]), fams,
                                      np.asarray(res["peak_d"][s]), int(res["status"][s])))
    return out


class XRDCalculator:
    """get_pattern / get_patterns on the GPU.

    wavelength: a key of WAVELENGTHS or a value in angstrom. coef: the scattering-factor
    table, float64 [zmax + 1][4][2] of (a_i, b_i) in f(s) = Z - 41.78214 s^2 sum a_i exp(-b_i s^2).
    debye_waller_factors: {symbol: B in angstrom^2} (default 0). rel_cutoff: peaks at or below
    this fraction of the largest are dropped (0 keeps all); tt_tol: merge tolerance in degrees
    (at least xrd.XRD_MIN_TT_TOL = 1e-9). point_group: None (families by permutation and sign),
    a Laue group name of LAUE_GENERATORS, or integer operations [n][3][3] on (h, k, l): families
    are then the orbits of that group (xrd_set_point_group).
    """

    def __init__(self, coef, wavelength="CuKa", debye_waller_factors=None, precision="fp32_phasefix",
                 rel_cutoff=1e-3, tt_tol=1e-5, handle=None, device=0, point_group=None):
        self.wavelength = WAVELENGTHS[wavelength] if isinstance(wavelength, str) else float(wavelength)
        self.coef = np.ascontiguousarray(coef, dtype=np.float64)
        self.dw = dict(debye_waller_factors or {})
        self.precision = precision
        self.rel_cutoff = float(rel_cutoff)
        self.tt_tol = float(tt_tol)
        self.device = device
        self._handle = handle
        # symmetry-aware families: a Laue group name (laue_group_ops) or operations [n][3][3]
        self.point_group = laue_group_ops(point_group) if isinstance(point_group, str) else point_group

    def _h(self):
        if self._handle is None:
            self._handle = xrd.Handle(self.device)
        return self._handle

    def get_patterns(self, structures, scaled=True, two_theta_range=(0, 90)):
        from .synth import Opts
        structures = list(structures)
        b = batch_of(structures, self.coef, self.dw)
        o = Opts(self.wavelength, float(two_theta_range[0]), float(two_theta_range[1]), self.tt_tol,
                 self.rel_cutoff, 1 if scaled else 0)
        o.point_group = self.point_group
        res = xrd.compute(b, o, self.precision, handle=self._h(), device=self.device)
        return patterns_from(res)

    def get_pattern(self, structure, scaled=True, two_theta_range=(0, 90)):
        return self.get_patterns([structure], scaled, two_theta_range)[0]

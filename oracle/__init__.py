"""Python access to the plain FP64 CPU oracle (``oracle/xrd_oracle.c``).

TEST INFRASTRUCTURE ONLY: imported by ``tests/``, ``__graft_entry__.smoke()``
and the CPU-baseline leg of ``bench.py``. The product package never imports
it, and it never imports the product package. Arrays are numpy; the layouts
are those of the C ABI (see ``xrd_oracle.h``).
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from . import build as _build

_lib = None

_D = C.POINTER(C.c_double)
_I32 = C.POINTER(C.c_int32)
_I64 = C.POINTER(C.c_int64)
_I16 = C.POINTER(C.c_int16)


class Opts(C.Structure):
    _fields_ = [("lambda_", C.c_double), ("tt_min", C.c_double), ("tt_max", C.c_double),
                ("tt_tol", C.c_double), ("cutoff", C.c_double), ("scaled", C.c_int),
                ("n_pg", C.c_int), ("pg", C.POINTER(C.c_int32))]


class _Out(C.Structure):
    _fields_ = [("cap_refl", C.c_long), ("cap_peaks", C.c_long), ("cap_fam", C.c_long),
                ("refl_hkl", _I32), ("refl_q", _D), ("refl_tt", _D), ("refl_lp", _D), ("refl_I", _D),
                ("refl_Fr", _D), ("refl_Fi", _D),
                ("peak_tt", _D), ("peak_I", _D), ("peak_d", _D), ("peak_fam_off", _I64),
                ("fam_hkl", _I32), ("fam_mult", _I32),
                ("n_refl", C.c_long), ("n_peaks_merged", C.c_long), ("n_peaks", C.c_long), ("n_fam", C.c_long),
                ("imax", C.c_double)]


def lib():
    global _lib
    if _lib is None:
        path = _build.build()
        _lib = C.CDLL(path)
        _lib.orc_metric.argtypes = [_D, _D, _D, _D]
        _lib.orc_q.argtypes = [_D, C.c_int, C.c_int, C.c_int]
        _lib.orc_q.restype = C.c_double
        _lib.orc_r2.argtypes = [C.c_double, C.c_double]
        _lib.orc_r2.restype = C.c_double
        _lib.orc_enumerate.argtypes = [_D, C.POINTER(Opts), C.c_long, _I32, _D]
        _lib.orc_enumerate.restype = C.c_long
        _lib.orc_refl.argtypes = [C.c_double, C.c_double, _D, _D, _D, _D]
        _lib.orc_f.argtypes = [_D, C.c_int, C.c_double]
        _lib.orc_f.restype = C.c_double
        _lib.orc_sf.argtypes = [C.c_int, C.c_int, C.c_int, C.c_double, C.c_long, _D, _I16, _D, _D, _D, _D, _D]
        _lib.orc_pattern.argtypes = [_D, C.c_long, _D, _I16, _D, _D, _D, C.c_int, C.POINTER(Opts), C.POINTER(_Out)]
        _lib.orc_pattern.restype = C.c_int
        _lib.orc_pattern_batch.argtypes = [C.c_int, _D, _I64, _D, _I16, _D, _D, _D, C.c_int, C.POINTER(Opts),
                                           C.c_int, C.c_int, _I64, _I64, _D, _D, _D, _I64, _I32, _I32,
                                           _I64, _I64, _I32]
        _lib.orc_pattern_batch.restype = C.c_int
        _lib.orc_max_threads.restype = C.c_int
        _lib.orc_broadened.argtypes = [_D, C.c_long, _D, _I16, _D, _D, _D, C.c_double, C.c_long, _I32, C.c_double,
                                       C.c_double, C.c_int, C.c_double, _D]
        _lib.orc_broadened_grad.argtypes = [_D, C.c_long, _D, _I16, _D, _D, _D, C.c_double, C.c_long, _I32,
                                            C.c_double, C.c_double, C.c_int, C.c_double, _D, _D, _D, _D]
        _lib.orc_augmented.argtypes = [_D, C.c_long, _D, _I16, _D, _D, _D, C.c_double, C.c_long, _I32, C.c_double,
                                       C.c_double, C.c_int, C.c_double, C.c_double, _D, C.c_double, C.c_void_p,
                                       C.c_double, _D]
        _lib.orc_march_dollase.argtypes = [_D, C.c_int, C.c_int, C.c_int, _D, C.c_double]
        _lib.orc_march_dollase.restype = C.c_double
        _lib.orc_is_hexagonal.argtypes = [_D]
        _lib.orc_is_hexagonal.restype = C.c_int
    return _lib


def _p(a, t):
    return a.ctypes.data_as(t) if a is not None else None


def opts(o) -> Opts:
    """Oracle options from any object with wavelength/tt_min/tt_max/tt_tol/rel_cutoff/scaled and,
    optionally, point_group: integer operations [n][3][3] on (h, k, l) (families by its orbits)."""
    pg = getattr(o, "point_group", None)
    if pg is None or len(pg) == 0:
        return Opts(float(o.wavelength), float(o.tt_min), float(o.tt_max), float(o.tt_tol),
                    float(o.rel_cutoff), int(o.scaled), 0, None)
    arr = np.ascontiguousarray(np.asarray(pg, dtype=np.int32).reshape(-1, 3, 3))
    oo = Opts(float(o.wavelength), float(o.tt_min), float(o.tt_max), float(o.tt_tol),
              float(o.rel_cutoff), int(o.scaled), int(arr.shape[0]), arr.ctypes.data_as(C.POINTER(C.c_int32)))
    oo._pg_arr = arr  # keeps the operations alive as long as the options
    return oo


def metric(lat):
    lat = np.ascontiguousarray(lat, dtype=np.float64)
    G = np.zeros(6)
    Gs = np.zeros(6)
    v = np.zeros(1)
    rc = lib().orc_metric(_p(lat, _D), _p(G, _D), _p(Gs, _D), _p(v, _D))
    if rc != 0:
        raise ValueError("invalid cell")
    return G, Gs, float(v[0])


def q_of(Gs, h, k, l) -> float:
    Gs = np.ascontiguousarray(Gs, dtype=np.float64)
    return lib().orc_q(_p(Gs, _D), int(h), int(k), int(l))


def r2(tt_deg, lam) -> float:
    return lib().orc_r2(float(tt_deg), float(lam))


def enumerate_refl(lat, o):
    lat = np.ascontiguousarray(lat, dtype=np.float64)
    oo = opts(o)
    n = lib().orc_enumerate(_p(lat, _D), C.byref(oo), 0, None, None)
    if n < 0:
        raise ValueError("invalid cell or options")
    hkl = np.zeros((n, 3), np.int32)
    q = np.zeros(n)
    lib().orc_enumerate(_p(lat, _D), C.byref(oo), n, _p(hkl, _I32), _p(q, _D))
    return hkl, q


def refl(q, lam):
    s2, tt, lp, d = C.c_double(), C.c_double(), C.c_double(), C.c_double()
    lib().orc_refl(float(q), float(lam), C.byref(s2), C.byref(tt), C.byref(lp), C.byref(d))
    return s2.value, tt.value, lp.value, d.value


def fatom(coef, Z, s2) -> float:
    coef = np.ascontiguousarray(coef, dtype=np.float64)
    return lib().orc_f(_p(coef, _D), int(Z), float(s2))


def sf(batch, s, h, k, l, s2):
    """Complex F(g) of structure s of a batch at reflection (h, k, l) with s^2 given."""
    sl = batch.atoms_of(s)
    frac = np.ascontiguousarray(batch.frac[sl])
    Z = np.ascontiguousarray(batch.Z[sl], dtype=np.int16)
    occ = np.ascontiguousarray(batch.occ[sl])
    B = np.ascontiguousarray(batch.B[sl])
    coef = np.ascontiguousarray(batch.coef, dtype=np.float64)
    fr, fi = C.c_double(), C.c_double()
    lib().orc_sf(int(h), int(k), int(l), float(s2), len(Z), _p(frac, _D), _p(Z, _I16), _p(occ, _D), _p(B, _D),
                 _p(coef, _D), C.byref(fr), C.byref(fi))
    return complex(fr.value, fi.value)


def pattern(batch, s, o, with_refl=True):
    """Full pattern of structure s: per-reflection list (sorted) and peaks/families."""
    lat = np.ascontiguousarray(batch.lattice[s], dtype=np.float64)
    sl = batch.atoms_of(s)
    frac = np.ascontiguousarray(batch.frac[sl])
    Z = np.ascontiguousarray(batch.Z[sl], dtype=np.int16)
    occ = np.ascontiguousarray(batch.occ[sl])
    B = np.ascontiguousarray(batch.B[sl])
    coef = np.ascontiguousarray(batch.coef, dtype=np.float64)
    oo = opts(o)
    n = lib().orc_enumerate(_p(lat, _D), C.byref(oo), 0, None, None)
    if n < 0:
        return {"status": 1}
    cap = max(n, 1)
    r = {"hkl": np.zeros((cap, 3), np.int32), "q": np.zeros(cap), "tt": np.zeros(cap), "lp": np.zeros(cap),
         "I": np.zeros(cap), "Fr": np.zeros(cap), "Fi": np.zeros(cap)}
    pk = {"tt": np.zeros(cap), "I": np.zeros(cap), "d": np.zeros(cap), "fam_off": np.zeros(cap + 1, np.int64)}
    fam = {"hkl": np.zeros((cap, 3), np.int32), "mult": np.zeros(cap, np.int32)}
    out = _Out()
    out.cap_refl = cap if with_refl else 0
    out.cap_peaks = cap
    out.cap_fam = cap
    if with_refl:
        out.refl_hkl, out.refl_q, out.refl_tt = _p(r["hkl"], _I32), _p(r["q"], _D), _p(r["tt"], _D)
        out.refl_lp, out.refl_I, out.refl_Fr, out.refl_Fi = (_p(r["lp"], _D), _p(r["I"], _D),
                                                              _p(r["Fr"], _D), _p(r["Fi"], _D))
    out.peak_tt, out.peak_I, out.peak_d = _p(pk["tt"], _D), _p(pk["I"], _D), _p(pk["d"], _D)
    out.peak_fam_off = _p(pk["fam_off"], _I64)
    out.fam_hkl, out.fam_mult = _p(fam["hkl"], _I32), _p(fam["mult"], _I32)
    rc = lib().orc_pattern(_p(lat, _D), len(Z), _p(frac, _D), _p(Z, _I16), _p(occ, _D), _p(B, _D), _p(coef, _D),
                           int(batch.zmax), C.byref(oo), C.byref(out))
    nr, npk, nf = out.n_refl, out.n_peaks, out.n_fam
    res = {"status": rc, "n_refl": nr, "n_peaks_merged": out.n_peaks_merged, "imax": out.imax,
           "peak_tt": pk["tt"][:npk].copy(), "peak_I": pk["I"][:npk].copy(), "peak_d": pk["d"][:npk].copy(),
           "peak_fam_off": pk["fam_off"][:npk + 1].copy(),
           "fam_hkl": fam["hkl"][:nf].copy(), "fam_mult": fam["mult"][:nf].copy()}
    if with_refl:
        for key in r:
            res["refl_" + key] = r[key][:nr].copy()
    return res


def pattern_batch(batch, o, threads: int = 0):
    """Peaks and families of every structure (OpenMP over structures when threads != 1).

    Returns a dict of per-structure lists of arrays, plus the status codes.
    """
    n = batch.n_struct
    lat = np.ascontiguousarray(batch.lattice, dtype=np.float64)
    off = np.ascontiguousarray(batch.atom_off, dtype=np.int64)
    frac = np.ascontiguousarray(batch.frac, dtype=np.float64)
    Z = np.ascontiguousarray(batch.Z, dtype=np.int16)
    occ = np.ascontiguousarray(batch.occ, dtype=np.float64)
    B = np.ascontiguousarray(batch.B, dtype=np.float64)
    coef = np.ascontiguousarray(batch.coef, dtype=np.float64)
    oo = opts(o)
    cnt = np.zeros(n, np.int64)
    st = np.zeros(n, np.int32)
    L = lib()
    L.orc_pattern_batch(n, _p(lat, _D), _p(off, _I64), _p(frac, _D), _p(Z, _I16), _p(occ, _D), _p(B, _D),
                        _p(coef, _D), int(batch.zmax), C.byref(oo), int(threads), 1, _p(cnt, _I64),
                        None, None, None, None, None, None, None, None, None, _p(st, _I32))
    cap_off = np.zeros(n + 1, np.int64)
    cap_off[1:] = np.cumsum(cnt)
    tot = max(int(cap_off[-1]), 1)
    ptt, pI, pd = np.zeros(tot), np.zeros(tot), np.zeros(tot)
    pfo = np.zeros(tot, np.int64)
    fh = np.zeros((tot, 3), np.int32)
    fm = np.zeros(tot, np.int32)
    npk = np.zeros(n, np.int64)
    nfm = np.zeros(n, np.int64)
    L.orc_pattern_batch(n, _p(lat, _D), _p(off, _I64), _p(frac, _D), _p(Z, _I16), _p(occ, _D), _p(B, _D),
                        _p(coef, _D), int(batch.zmax), C.byref(oo), int(threads), 0, _p(cnt, _I64),
                        _p(cap_off, _I64), _p(ptt, _D), _p(pI, _D), _p(pd, _D), _p(pfo, _I64), _p(fh, _I32),
                        _p(fm, _I32), _p(npk, _I64), _p(nfm, _I64), _p(st, _I32))
    res = {"status": st, "n_refl": cnt, "peak_tt": [], "peak_I": [], "peak_d": [], "peak_fam_off": [],
           "fam_hkl": [], "fam_mult": []}
    for s in range(n):
        b, p, f = int(cap_off[s]), int(npk[s]), int(nfm[s])
        res["peak_tt"].append(ptt[b:b + p])
        res["peak_I"].append(pI[b:b + p])
        res["peak_d"].append(pd[b:b + p])
        fo = np.empty(p + 1, np.int64)
        fo[:p] = pfo[b:b + p]
        fo[p] = f
        res["peak_fam_off"].append(fo)
        res["fam_hkl"].append(fh[b:b + f])
        res["fam_mult"].append(fm[b:b + f])
    return res


def refl_counts(batch, o, threads: int = 0) -> np.ndarray:
    """Full-sphere reflection count of every structure (the enumeration only; OpenMP over structures)."""
    n = batch.n_struct
    cnt = np.zeros(max(n, 1), np.int64)
    st = np.zeros(max(n, 1), np.int32)
    lib().orc_pattern_batch(n, _p(np.ascontiguousarray(batch.lattice, dtype=np.float64), _D),
                            _p(np.ascontiguousarray(batch.atom_off, dtype=np.int64), _I64),
                            _p(np.ascontiguousarray(batch.frac, dtype=np.float64), _D),
                            _p(np.ascontiguousarray(batch.Z, dtype=np.int16), _I16),
                            _p(np.ascontiguousarray(batch.occ, dtype=np.float64), _D),
                            _p(np.ascontiguousarray(batch.B, dtype=np.float64), _D),
                            _p(np.ascontiguousarray(batch.coef, dtype=np.float64), _D), int(batch.zmax),
                            C.byref(opts(o)), int(threads), 1, _p(cnt, _I64), None, None, None, None, None, None,
                            None, None, None, _p(st, _I32))
    return cnt[:n]


def max_threads() -> int:
    return int(lib().orc_max_threads())


def _struct_arrays(batch, s):
    sl = batch.atoms_of(s)
    return (np.ascontiguousarray(batch.lattice[s], dtype=np.float64), np.ascontiguousarray(batch.frac[sl]),
            np.ascontiguousarray(batch.Z[sl], dtype=np.int16), np.ascontiguousarray(batch.occ[sl]),
            np.ascontiguousarray(batch.B[sl]), np.ascontiguousarray(batch.coef, dtype=np.float64))


def broadened(batch, s, hkl, lam, grid):
    """y over the grid for structure s and a fixed full-sphere reflection list hkl[nr][3]."""
    lat, frac, Z, occ, B, coef = _struct_arrays(batch, s)
    hkl = np.ascontiguousarray(hkl, dtype=np.int32)
    y = np.zeros(int(grid.n_pts))
    lib().orc_broadened(_p(lat, _D), len(Z), _p(frac, _D), _p(Z, _I16), _p(occ, _D), _p(B, _D), _p(coef, _D),
                        float(lam), len(hkl), _p(hkl, _I32), float(grid.t0), float(grid.dt), int(grid.n_pts),
                        float(grid.fwhm), _p(y, _D))
    return y


def augmented(batch, s, hkl, lam, t0, dt, n_pts, fwhm, eta, po_dir=(0.0, 0.0, 1.0), po_r=1.0, z=None, sigma=0.0):
    """Augmented pattern of structure s on the grid t0 + i dt (i < n_pts) for a fixed full-sphere
    reflection list: March-Dollase about po_dir (reciprocal-lattice components), area-normalised
    pseudo-Voigt (fwhm, eta), then y += sigma sqrt(y) z when z (standard normal draws) is given."""
    lat, frac, Z, occ, B, coef = _struct_arrays(batch, s)
    hkl = np.ascontiguousarray(hkl, dtype=np.int32)
    y = np.zeros(int(n_pts))
    d = np.ascontiguousarray(po_dir, dtype=np.float64)
    zz = None if z is None else np.ascontiguousarray(z, dtype=np.float64)
    lib().orc_augmented(_p(lat, _D), len(Z), _p(frac, _D), _p(Z, _I16), _p(occ, _D), _p(B, _D), _p(coef, _D),
                        float(lam), len(hkl), _p(hkl, _I32), float(t0), float(dt), int(n_pts), float(fwhm),
                        float(eta), _p(d, _D), float(po_r), None if zz is None else zz.ctypes.data, float(sigma),
                        _p(y, _D))
    return y


def is_hexagonal(lat):
    lat = np.ascontiguousarray(lat, dtype=np.float64)
    return bool(lib().orc_is_hexagonal(_p(lat, _D)))


def march_dollase(lat, h, k, l, po_dir, po_r):
    _, Gs, _ = metric(lat)
    d = np.ascontiguousarray(po_dir, dtype=np.float64)
    return lib().orc_march_dollase(_p(np.ascontiguousarray(Gs, dtype=np.float64), _D), int(h), int(k), int(l),
                                   _p(d, _D), float(po_r))


def broadened_grad(batch, s, hkl, lam, grid, dLdy):
    """(d_frac [n][3], d_B [n], d_lattice [6]) of L = sum(dLdy * y)."""
    lat, frac, Z, occ, B, coef = _struct_arrays(batch, s)
    hkl = np.ascontiguousarray(hkl, dtype=np.int32)
    g = np.ascontiguousarray(dLdy, dtype=np.float64)
    df = np.zeros((len(Z), 3))
    dB = np.zeros(len(Z))
    dl = np.zeros(6)
    lib().orc_broadened_grad(_p(lat, _D), len(Z), _p(frac, _D), _p(Z, _I16), _p(occ, _D), _p(B, _D), _p(coef, _D),
                             float(lam), len(hkl), _p(hkl, _I32), float(grid.t0), float(grid.dt), int(grid.n_pts),
                             float(grid.fwhm), _p(g, _D), _p(df, _D), _p(dB, _D), _p(dl, _D))
    return df, dB, dl

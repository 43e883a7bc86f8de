"""Pins of the FP64 CPU oracle against facts the mathematics and crystallography fix.

Every check here is independent of the oracle's own code: textbook closed forms,
selection rules, invariances, exact-rational brute force and a long-double
re-summation. A plausible mistake (dropped term, wrong sign or index, a
transposed lattice angle) fails at least one of them.
"""
import math
import os
from fractions import Fraction

import numpy as np
import pytest

import oracle
from paper_2602_11709_gb300 import synth

HERE = os.path.dirname(os.path.abspath(__file__))
LAM = synth.CU_KA


def _opts(**kw):
    o = synth.Opts()
    for k, v in kw.items():
        setattr(o, k, v)
    return o


def _rand_lat(rng):
    return np.concatenate([rng.uniform(3, 15, 3), synth._angles(rng, 1)[0]])


# ---------------------------------------------------------------- metric tensors

def test_metric_inverse_and_volume():
    rng = np.random.default_rng(11)
    for _ in range(50):
        lat = _rand_lat(rng)
        G, Gs, V = oracle.metric(lat)
        Gm = np.array([[G[0], G[3], G[4]], [G[3], G[1], G[5]], [G[4], G[5], G[2]]])
        Gsm = np.array([[Gs[0], Gs[3], Gs[4]], [Gs[3], Gs[1], Gs[5]], [Gs[4], Gs[5], Gs[2]]])
        assert np.allclose(Gm @ Gsm, np.eye(3), atol=1e-13)
        a, b, c = lat[:3]
        ca, cb, cg = np.cos(np.radians(lat[3:]))
        V_ref = a * b * c * math.sqrt(1 - ca * ca - cb * cb - cg * cg + 2 * ca * cb * cg)
        assert V == pytest.approx(V_ref, rel=1e-12)
        # Direct metric from explicit Cartesian cell vectors (textbook construction).
        av = np.array([a, 0, 0])
        bv = np.array([b * cg, b * math.sin(math.radians(lat[5])), 0])
        cx = c * cb
        cy = c * (ca - cb * cg) / math.sin(math.radians(lat[5]))
        cv = np.array([cx, cy, math.sqrt(c * c - cx * cx - cy * cy)])
        M = np.array([av, bv, cv])
        assert np.allclose(M @ M.T, Gm, rtol=1e-12, atol=1e-10)


def test_hexagonal_and_monoclinic_d_spacing_closed_forms():
    a, c = 3.21, 5.21
    _, Gs, _ = oracle.metric([a, a, c, 90, 90, 120])
    for h, k, l in [(1, 0, 0), (1, 1, 0), (1, 0, 1), (2, -1, 3), (0, 0, 2), (3, 2, 1)]:
        inv_d2 = 4.0 / 3.0 * (h * h + h * k + k * k) / a ** 2 + l * l / c ** 2
        assert oracle.q_of(Gs, h, k, l) == pytest.approx(inv_d2, rel=1e-13)
    a, b, c, beta = 5.1, 7.3, 6.2, 104.5
    _, Gs, _ = oracle.metric([a, b, c, 90, beta, 90])
    sb, cbt = math.sin(math.radians(beta)), math.cos(math.radians(beta))
    for h, k, l in [(1, 0, 0), (1, 2, 3), (-2, 1, 1), (0, 3, -2)]:
        inv_d2 = (h * h / a ** 2 + k * k * sb * sb / b ** 2 + l * l / c ** 2 - 2 * h * l * cbt / (a * c)) / sb ** 2
        assert oracle.q_of(Gs, h, k, l) == pytest.approx(inv_d2, rel=1e-12)


def test_invalid_cells_rejected():
    for lat in ([5, 5, 5, 60, 60, 120], [0, 5, 5, 90, 90, 90], [5, 5, 5, 120, 120, 120], [5, 5, np.nan, 90, 90, 90]):
        with pytest.raises(ValueError):
            oracle.metric(lat)


# ---------------------------------------------------------------- enumeration

def _rational_enum(a, b, c, lam_frac, sin2_max):
    """Exact-rational brute force for an orthogonal cell: |g|^2 = h^2/a^2 + k^2/b^2 + l^2/c^2."""
    r2 = 4 * sin2_max / lam_frac ** 2
    out = set()
    H = int(math.isqrt(int(r2 * a * a)) + 2)
    K = int(math.isqrt(int(r2 * b * b)) + 2)
    L = int(math.isqrt(int(r2 * c * c)) + 2)
    for h in range(-H, H + 1):
        for k in range(-K, K + 1):
            for l in range(-L, L + 1):
                if (h, k, l) == (0, 0, 0):
                    continue
                if Fraction(h * h) / (a * a) + Fraction(k * k) / (b * b) + Fraction(l * l) / (c * c) <= r2:
                    out.add((h, k, l))
    return out


def test_enumeration_exact_rational_orthogonal():
    # 2-theta max = 90 deg: sin^2(45) = 1/2 exactly; lambda and edges exact binary-friendly rationals
    for a, b, c in [(Fraction(4), Fraction(5), Fraction(6)), (Fraction(7, 2), Fraction(9, 2), Fraction(11, 4))]:
        lam = Fraction(3, 2)
        ref = _rational_enum(a, b, c, lam, Fraction(1, 2))
        hkl, q = oracle.enumerate_refl([float(a), float(b), float(c), 90, 90, 90],
                                       _opts(wavelength=float(lam), tt_min=0.0, tt_max=90.0))
        got = {tuple(int(x) for x in r) for r in hkl}
        # boundary reflections with |g|^2 == r^2 exactly can differ by rounding of sin(45 deg)
        r2 = 4 * Fraction(1, 2) / lam ** 2
        diff = got ^ ref
        for h, k, l in diff:
            qq = Fraction(h * h) / (a * a) + Fraction(k * k) / (b * b) + Fraction(l * l) / (c * c)
            assert abs(float(qq - r2)) <= 4e-15 * float(r2), (h, k, l)


def test_enumeration_nacl_is_integer_sphere():
    b, o = synth.nacl()
    hkl, q = oracle.enumerate_refl(b.lattice[0], o)
    n2 = (hkl ** 2).sum(axis=1)
    limit = 2 * 5.64 ** 2 / LAM ** 2  # h^2+k^2+l^2 <= 2 a^2 / lambda^2 = 26.76
    expect = {(h, k, l) for h in range(-6, 7) for k in range(-6, 7) for l in range(-6, 7)
              if 0 < h * h + k * k + l * l <= limit}
    assert {tuple(r) for r in hkl} == expect
    assert n2.max() == 26 and len(hkl) == 586


def test_enumeration_box_bound_and_friedel_symmetry():
    rng = np.random.default_rng(12)
    for _ in range(10):
        lat = _rand_lat(rng)
        o = _opts(tt_min=0.0, tt_max=90.0)
        hkl, q = oracle.enumerate_refl(lat, o)
        S = {tuple(r) for r in hkl}
        assert S == {(-h, -k, -l) for h, k, l in S}
        # independent brute force over a much larger box, vectorised
        _, Gs, V = oracle.metric(lat)
        r2max = oracle.r2(90.0, LAM)
        M = int(math.sqrt(r2max) * lat[:3].max()) + 4
        g = np.arange(-M, M + 1)
        h, k, l = np.meshgrid(g, g, g, indexing="ij")
        qq = (Gs[0] * h * h + Gs[1] * k * k + Gs[2] * l * l + 2 * (Gs[3] * h * k + Gs[4] * h * l + Gs[5] * k * l))
        inside = (qq <= r2max * (1 + 1e-12)) & ((h != 0) | (k != 0) | (l != 0))
        loose = {(int(a), int(b), int(c)) for a, b, c in zip(h[inside], k[inside], l[inside])}
        assert S <= loose and len(loose - S) <= 2
        # count close to sphere volume times cell volume
        expect = 4.0 / 3.0 * math.pi * r2max ** 1.5 * V
        assert abs(len(S) - expect) < 0.05 * expect + 60


def test_enumeration_inner_limit():
    b, _ = synth.nacl()
    hkl, q = oracle.enumerate_refl(b.lattice[0], _opts(tt_min=30.0, tt_max=60.0))
    tt = np.array([oracle.refl(x, LAM)[1] for x in q])
    assert tt.min() >= 30.0 - 1e-9 and tt.max() <= 60.0 + 1e-9
    n2 = set((hkl ** 2).sum(axis=1).tolist())
    # 2theta(N) = 2 asin(lambda sqrt(N) / (2 a)); the lines between 30 and 60 deg
    sums = {h * h + k * k + l * l for h in range(7) for k in range(7) for l in range(7)}
    exp_n = {n for n in range(1, 40)
             if n in sums and 30 <= 2 * math.degrees(math.asin(LAM * math.sqrt(n) / (2 * 5.64))) <= 60}
    assert n2 == exp_n


# ---------------------------------------------------------------- per-reflection scalars

def test_bragg_and_lp_closed_forms():
    # 2-theta = 90 deg: LP = (1 + 0) / (sin^2 45 cos 45) = 2 sqrt 2
    q90 = oracle.r2(90.0, LAM)
    s2, tt, lp, d = oracle.refl(q90, LAM)
    assert tt == pytest.approx(90.0, abs=1e-12)
    assert lp == pytest.approx(2 * math.sqrt(2), rel=1e-12)
    assert s2 == pytest.approx(q90 / 4, rel=1e-15)
    # 2-theta = 60 deg: LP = (1 + 1/4) / (1/4 * sqrt(3)/2)
    s2, tt, lp, d = oracle.refl(oracle.r2(60.0, LAM), LAM)
    assert lp == pytest.approx(1.25 / (0.25 * math.sqrt(3) / 2), rel=1e-12)
    # NaCl (200): d = a / 2, Bragg angle 2 asin(lambda / a)
    _, Gs, _ = oracle.metric([5.64] * 3 + [90] * 3)
    s2, tt, lp, d = oracle.refl(oracle.q_of(Gs, 2, 0, 0), LAM)
    assert d == pytest.approx(2.82, rel=1e-14)
    assert tt == pytest.approx(2 * math.degrees(math.asin(LAM / 5.64)), abs=1e-12)
    assert tt == pytest.approx(31.7305, abs=1e-4)


# ---------------------------------------------------------------- scattering factor

def test_atomic_scattering_factor_limits():
    coef = synth.coef_table(np.random.default_rng(3))
    for Z in (1, 11, 17, 83):
        assert oracle.fatom(coef, Z, 0.0) == Z  # forward scattering counts the electrons
    # the s^2 coefficient is the Mott-Bethe factor 8 pi^2 a0 with the Bohr radius a0 = 0.529177 A
    a0 = 0.529177
    ds = 1e-7
    for Z in (6, 29):
        slope = (oracle.fatom(coef, Z, ds) - Z) / ds
        assert slope == pytest.approx(-8 * math.pi ** 2 * a0 * coef[Z, :, 0].sum(), rel=1e-5)
    # the electron-scattering sum decays faster than s^2 grows: f returns to Z at large s
    assert oracle.fatom(coef, 40, 1e4) == pytest.approx(40.0, abs=1e-12)
    # a table of zeros leaves the bare electron count
    assert oracle.fatom(np.zeros_like(coef), 40, 0.3) == 40.0


# ---------------------------------------------------------------- structure factor

def _nacl_batch(B=0.5):
    b, o = synth.nacl()
    b.B[:] = B
    return b, o


def test_rock_salt_closed_form():
    b, o = _nacl_batch()
    _, Gs, _ = oracle.metric(b.lattice[0])
    for hkl in [(1, 1, 1), (2, 0, 0), (2, 2, 0), (3, 1, 1), (2, 2, 2), (4, 2, 0), (1, 0, 0), (2, 1, 0), (3, 2, 1),
                (-3, 1, -1), (0, 0, 4), (5, 1, 0)]:
        s2 = oracle.q_of(Gs, *hkl) / 4
        F = oracle.sf(b, 0, *hkl, s2)
        fna, fcl = oracle.fatom(b.coef, 11, s2), oracle.fatom(b.coef, 17, s2)
        dw = math.exp(-0.5 * s2)
        par = {x % 2 for x in hkl}
        if par == {0}:
            ref = 4 * dw * (fna + fcl)
        elif par == {1}:
            ref = 4 * dw * (fna - fcl)
        else:
            ref = 0.0
        assert abs(F - ref) < 1e-11 * (abs(fna) + abs(fcl)) * 8, (hkl, F, ref)


def _one_struct(frac, Z, occ, B, lat, coef):
    frac = np.asarray(frac, dtype=np.float64).reshape(-1, 3)
    n = len(frac)
    return synth.Batch(np.asarray([lat], dtype=np.float64), np.array([0, n], np.int64), frac,
                       np.asarray(Z, np.int16), np.asarray(occ, np.float64), np.asarray(B, np.float64), coef)


def _random_struct(rng, n):
    lat = _rand_lat(rng)
    coef = synth.coef_table(rng)
    return _one_struct(rng.random((n, 3)), rng.integers(1, 84, n), rng.uniform(0.5, 1, n), rng.uniform(0, 2, n),
                       lat, coef)


def _F(b, hkl):
    _, Gs, _ = oracle.metric(b.lattice[0])
    s2 = oracle.q_of(Gs, *hkl) / 4
    return oracle.sf(b, 0, *hkl, s2)


HKLS = [(1, 0, 0), (0, 1, 0), (1, 1, 1), (2, -1, 3), (3, 2, -2), (-4, 1, 2), (1, 3, 5), (5, 0, -1)]


def test_friedel_and_origin_shift():
    rng = np.random.default_rng(21)
    b = _random_struct(rng, 13)
    t = rng.random(3)
    shifted = synth.Batch(b.lattice, b.atom_off, (b.frac + t) % 1.0, b.Z, b.occ, b.B, b.coef)
    ishift = synth.Batch(b.lattice, b.atom_off, b.frac + np.array([3.0, -2.0, 7.0]), b.Z, b.occ, b.B, b.coef)
    for hkl in HKLS:
        F = _F(b, hkl)
        Fm = _F(b, tuple(-x for x in hkl))
        assert abs(Fm - F.conjugate()) < 1e-11 * (1 + abs(F))
        Fs = _F(shifted, hkl)
        assert abs(abs(Fs) - abs(F)) < 1e-10 * (1 + abs(F))
        # the shift multiplies F by exp(2 pi i g.t)
        ph = np.exp(2j * np.pi * np.dot(hkl, t))
        assert abs(Fs - F * ph) < 1e-10 * (1 + abs(F))
        # integer shifts change nothing
        assert abs(_F(ishift, hkl) - F) < 1e-10 * (1 + abs(F))


@pytest.mark.parametrize("kind", ["I", "F", "C"])
def test_centring_absences(kind):
    rng = np.random.default_rng(22)
    base = _random_struct(rng, 5)
    shifts = {"I": [(0, 0, 0), (.5, .5, .5)], "F": [(0, 0, 0), (0, .5, .5), (.5, 0, .5), (.5, .5, 0)],
              "C": [(0, 0, 0), (.5, .5, 0)]}[kind]
    frac = np.vstack([(base.frac + np.array(s)) % 1.0 for s in shifts])
    rep = len(shifts)
    b = _one_struct(frac, np.tile(base.Z, rep), np.tile(base.occ, rep), np.tile(base.B, rep), base.lattice[0],
                    base.coef)
    for h in range(-3, 4):
        for k in range(-3, 4):
            for l in range(-3, 4):
                if (h, k, l) == (0, 0, 0):
                    continue
                F = _F(b, (h, k, l))
                F0 = _F(base, (h, k, l))
                if kind == "I":
                    absent = (h + k + l) % 2 == 1
                elif kind == "F":
                    absent = len({h % 2, k % 2, l % 2}) > 1
                else:
                    absent = (h + k) % 2 == 1
                if absent:
                    assert abs(F) < 1e-10 * (1 + abs(F0)) * rep
                else:
                    assert abs(F - rep * F0) < 1e-10 * (1 + abs(F0)) * rep


def test_two_atom_interference_and_single_atom():
    rng = np.random.default_rng(23)
    lat = _rand_lat(rng)
    coef = synth.coef_table(rng)
    x1, x2 = rng.random(3), rng.random(3)
    b = _one_struct([x1, x2], [26, 8], [1.0, 0.7], [0.3, 1.1], lat, coef)
    _, Gs, _ = oracle.metric(lat)
    for hkl in HKLS:
        s2 = oracle.q_of(Gs, *hkl) / 4
        w1 = 1.0 * oracle.fatom(coef, 26, s2) * math.exp(-0.3 * s2)
        w2 = 0.7 * oracle.fatom(coef, 8, s2) * math.exp(-1.1 * s2)
        F = _F(b, hkl)
        ref = w1 * w1 + w2 * w2 + 2 * w1 * w2 * math.cos(2 * math.pi * np.dot(hkl, x1 - x2))
        assert abs(F) ** 2 == pytest.approx(ref, rel=1e-10, abs=1e-10 * (w1 * w1 + w2 * w2))
    single = _one_struct([[0, 0, 0]], [30], [0.8], [0.9], lat, coef)
    for hkl in HKLS:
        s2 = oracle.q_of(Gs, *hkl) / 4
        F = _F(single, hkl)
        assert F.imag == 0.0 and F.real == pytest.approx(0.8 * oracle.fatom(coef, 30, s2) * math.exp(-0.9 * s2),
                                                         rel=1e-14)


def test_zero_occupancy_atoms_vanish():
    rng = np.random.default_rng(24)
    b = _random_struct(rng, 6)
    occ = b.occ.copy()
    occ[[1, 4]] = 0.0
    b0 = synth.Batch(b.lattice, b.atom_off, b.frac, b.Z, occ, b.B, b.coef)
    keep = [0, 2, 3, 5]
    b1 = _one_struct(b.frac[keep], b.Z[keep], b.occ[keep], b.B[keep], b.lattice[0], b.coef)
    for hkl in HKLS:
        assert abs(_F(b0, hkl) - _F(b1, hkl)) < 1e-11 * (1 + abs(_F(b1, hkl)))


def test_long_double_resummation_bounds_fp64_error():
    """Re-sum F in extended precision (numpy longdouble) from the same per-atom weights."""
    rng = np.random.default_rng(25)
    b = _random_struct(rng, 40)
    _, Gs, _ = oracle.metric(b.lattice[0])
    for hkl in HKLS:
        s2 = oracle.q_of(Gs, *hkl) / 4
        F = _F(b, hkl)
        acc = np.longdouble(0), np.longdouble(0)
        re = np.longdouble(0)
        im = np.longdouble(0)
        for j in range(b.n_atoms):
            w = np.longdouble(b.occ[j]) * np.longdouble(oracle.fatom(b.coef, int(b.Z[j]), s2)) * \
                np.exp(-np.longdouble(b.B[j]) * np.longdouble(s2))
            phi = np.longdouble(hkl[0]) * np.longdouble(b.frac[j, 0]) + np.longdouble(hkl[1]) * \
                np.longdouble(b.frac[j, 1]) + np.longdouble(hkl[2]) * np.longdouble(b.frac[j, 2])
            phi = phi - np.floor(phi)
            ang = 2 * np.pi * phi  # longdouble pi
            re += w * np.cos(ang)
            im += w * np.sin(ang)
        scale = float(np.sum(np.abs(b.occ) * 100))
        assert abs(F.real - float(re)) < 1e-12 * scale
        assert abs(F.imag - float(im)) < 1e-12 * scale


def test_supercell_and_axis_relabel():
    rng = np.random.default_rng(26)
    b = _random_struct(rng, 7)
    lat = b.lattice[0]
    # 2 x 1 x 1 supercell: odd h' vanish, F'(2h, k, l) = 2 F(h, k, l)
    f2 = np.vstack([b.frac * np.array([0.5, 1, 1]), b.frac * np.array([0.5, 1, 1]) + np.array([0.5, 0, 0])])
    sup = _one_struct(f2, np.tile(b.Z, 2), np.tile(b.occ, 2), np.tile(b.B, 2),
                      [2 * lat[0], lat[1], lat[2], lat[3], lat[4], lat[5]], b.coef)
    for h, k, l in HKLS:
        assert abs(_F(sup, (2 * h, k, l)) - 2 * _F(b, (h, k, l))) < 1e-10 * (1 + abs(_F(b, (h, k, l))))
        assert abs(_F(sup, (2 * h + 1, k, l))) < 1e-10 * (1 + abs(_F(b, (h, k, l))))
    # relabel axes a->b->c->a: (a,b,c,al,be,ga,x,y,z) -> (b,c,a,be,ga,al,y,z,x), hkl -> (k,l,h)
    rl = _one_struct(b.frac[:, [1, 2, 0]], b.Z, b.occ, b.B, [lat[1], lat[2], lat[0], lat[4], lat[5], lat[3]], b.coef)
    for h, k, l in HKLS:
        assert abs(_F(rl, (k, l, h)) - _F(b, (h, k, l))) < 1e-10 * (1 + abs(_F(b, (h, k, l))))
    o = _opts(rel_cutoff=1e-3)
    p0 = oracle.pattern(b, 0, o, with_refl=False)
    p1 = oracle.pattern(rl, 0, o, with_refl=False)
    assert np.allclose(p0["peak_tt"], p1["peak_tt"], atol=1e-9)
    assert np.allclose(p0["peak_I"], p1["peak_I"], rtol=1e-9, atol=1e-9)
    assert np.array_equal(np.sort(p0["fam_mult"]), np.sort(p1["fam_mult"]))


# ---------------------------------------------------------------- merge, families, cutoff, scaling

def _golden_nacl():
    rows = []
    with open(os.path.join(HERE, "golden", "nacl_cubic_families.txt")) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            parts = line.split()
            fams = []
            for p in parts[2:]:
                hkl, m = p.split(":")
                fams.append((tuple(int(c) for c in hkl), int(m)))
            rows.append((parts[0] == "yes", int(parts[1]), fams))
    return rows


@pytest.mark.parametrize("cutoff", [1e-3, 0.0])
def test_nacl_families_and_intensities(cutoff):
    b, o = synth.nacl()
    o.rel_cutoff = cutoff
    o.scaled = 0
    p = oracle.pattern(b, 0, o)
    gold = [r for r in _golden_nacl() if r[0] or cutoff == 0.0]
    gold.sort(key=lambda r: r[1])
    assert len(p["peak_tt"]) == len(gold)
    _, Gs, _ = oracle.metric(b.lattice[0])
    fo = p["peak_fam_off"]
    for i, (_, n2, fams) in enumerate(gold):
        got = [(tuple(int(x) for x in p["fam_hkl"][f]), int(p["fam_mult"][f])) for f in range(fo[i], fo[i + 1])]
        assert sorted(got) == sorted(fams), (n2, got, fams)
        # merged intensity = multiplicity x closed-form per-reflection intensity
        rep = fams[0][0]
        q = oracle.q_of(Gs, *rep)
        s2, tt, lp, d = oracle.refl(q, o.wavelength)
        assert p["peak_tt"][i] == pytest.approx(2 * math.degrees(math.asin(o.wavelength * math.sqrt(n2) / (2 * 5.64))),
                                                abs=1e-10)
        if n2 % 2 == 0 and all(x % 2 == 0 for x in rep) or all(x % 2 == 1 for x in rep):
            fna, fcl = oracle.fatom(b.coef, 11, s2), oracle.fatom(b.coef, 17, s2)
            sgn = 1 if all(x % 2 == 0 for x in rep) else -1
            I1 = (4 * math.exp(-0.5 * s2) * (fna + sgn * fcl)) ** 2 * lp
            mult = sum(m for _, m in fams)
            assert p["peak_I"][i] == pytest.approx(mult * I1, rel=1e-11)
        else:
            assert p["peak_I"][i] < 1e-20 * p["imax"]


def test_nacl_scaled_max_is_100():
    b, o = synth.nacl()
    p = oracle.pattern(b, 0, o)
    assert p["peak_I"].max() == 100.0
    assert np.all(np.diff(p["peak_tt"]) > 0)
    assert np.all(p["peak_I"] > 0.1)


def test_anchor_rule_merges_against_first_member():
    """(100) anchors a peak; (010) sits 0.6 tol above it and joins; (001) sits 1.2 tol above
    the anchor but only 0.6 tol above (010): the anchor rule opens a new peak for it."""
    lam, a, tol = 1.5, 5.0, 1e-3
    tt100 = 2 * math.degrees(math.asin(lam / (2 * a)))

    def edge(tt):
        return lam / (2 * math.sin(math.radians(tt / 2)))
    b_, c_ = edge(tt100 + 0.6 * tol), edge(tt100 + 1.2 * tol)
    coef = synth.coef_table(np.random.default_rng(0))
    st = _one_struct([[0.1, 0.2, 0.3]], [20], [1.0], [0.0], [a, b_, c_, 90, 90, 90], coef)
    o = _opts(wavelength=lam, tt_min=0.0, tt_max=1.2 * tt100, tt_tol=tol, rel_cutoff=0.0, scaled=0)
    p = oracle.pattern(st, 0, o)
    assert len(p["peak_tt"]) == 2
    fo = p["peak_fam_off"]
    fam0 = [(tuple(p["fam_hkl"][f]), int(p["fam_mult"][f])) for f in range(fo[0], fo[1])]
    fam1 = [(tuple(p["fam_hkl"][f]), int(p["fam_mult"][f])) for f in range(fo[1], fo[2])]
    assert fam0 == [((1, 0, 0), 4)]
    assert fam1 == [((0, 0, 1), 2)]
    assert p["peak_tt"][0] == pytest.approx(tt100, abs=1e-12)
    # with a previous-neighbour rule all three would merge; with tol just above 1.2 tol they do
    o.tt_tol = 1.3 * tol
    p2 = oracle.pattern(st, 0, o)
    assert len(p2["peak_tt"]) == 1 and int(p2["fam_mult"].sum()) == 6


def test_cutoff_counts_and_order():
    rng = np.random.default_rng(27)
    b = _random_struct(rng, 20)
    o = _opts(rel_cutoff=0.0, scaled=0)
    full = oracle.pattern(b, 0, o, with_refl=True)
    imax = full["peak_I"].max()
    assert imax == full["imax"]
    # every reflection lands in exactly one peak: multiplicities add up to the reflection count
    assert int(full["fam_mult"].sum()) == full["n_refl"]
    assert full["refl_I"].sum() == pytest.approx(full["peak_I"].sum(), rel=1e-12)
    for c in (1e-3, 1e-2):
        o2 = _opts(rel_cutoff=c, scaled=1)
        cut = oracle.pattern(b, 0, o2, with_refl=False)
        keep = full["peak_I"] > c * imax
        assert len(cut["peak_tt"]) == int(keep.sum())
        assert np.array_equal(cut["peak_tt"], full["peak_tt"][keep])
        assert np.allclose(cut["peak_I"], 100 * full["peak_I"][keep] / imax, rtol=1e-14)
        assert cut["peak_I"].max() == 100.0


def test_empty_and_degenerate_inputs():
    b, o = synth.nacl()
    # no reflection below 2-theta = 10 deg for a = 5.64 A
    o2 = _opts(tt_min=0.0, tt_max=10.0)
    p = oracle.pattern(b, 0, o2)
    assert p["status"] == 0 and p["n_refl"] == 0 and len(p["peak_tt"]) == 0
    # a structure without atoms has reflections but zero intensity everywhere
    empty = _one_struct(np.zeros((0, 3)), [], [], [], b.lattice[0], b.coef)
    p = oracle.pattern(empty, 0, _opts(rel_cutoff=0.0))
    assert p["status"] == 0 and p["n_refl"] == 586 and np.all(p["peak_I"] == 0.0)


def test_batch_matches_single():
    b, o = synth.small(n=24)
    res = oracle.pattern_batch(b, o, threads=2)
    for s in range(b.n_struct):
        p = oracle.pattern(b, s, o, with_refl=False)
        assert np.array_equal(res["peak_tt"][s], p["peak_tt"])
        assert np.array_equal(res["peak_I"][s], p["peak_I"])
        assert np.array_equal(res["fam_hkl"][s], p["fam_hkl"])
        assert np.array_equal(res["fam_mult"][s], p["fam_mult"])
        assert np.array_equal(res["peak_fam_off"][s], p["peak_fam_off"])


def _golden_diamond():
    rows = []
    with open(os.path.join(HERE, "golden", "diamond_cubic_lines.txt")) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            parts = line.split()
            fams = []
            for item in parts[2:]:
                h, m = item.split(":")
                fams.append((tuple(int(c) for c in h), int(m)))
            rows.append((parts[0] == "yes", int(parts[1]), fams))
    return rows


def test_diamond_cubic_lines_and_extinctions():
    """Diamond structure (fcc + fcc shifted by a quarter of the body diagonal): |F| = 8 f' for
    h + k + l = 4n, 4 sqrt(2) f' for odd h + k + l, 0 for 4n + 2 and mixed parity; the kept lines,
    their families (two at N = 27) and multiplicities, and their merged intensities."""
    coef = synth.coef_table(np.random.default_rng(3))
    a, B, Z = 5.431, 0.4, 14
    fcc = np.array([[0, 0, 0], [0, .5, .5], [.5, 0, .5], [.5, .5, 0]], dtype=np.float64)
    frac = np.vstack([fcc, (fcc + 0.25) % 1.0])
    b = synth.Batch(np.array([[a, a, a, 90.0, 90.0, 90.0]]), np.array([0, 8], np.int64), frac,
                    np.full(8, Z, np.int16), np.ones(8), np.full(8, B), coef)
    o = synth.Opts(LAM, 0.0, 150.0, 1e-5, 1e-3, 0)
    _, Gs, _ = oracle.metric(b.lattice[0])

    def fprime(s2):
        return oracle.fatom(coef, Z, s2) * math.exp(-B * s2)

    def closed(h, k, l, s2):
        if len({h % 2, k % 2, l % 2}) > 1 or (h + k + l) % 4 == 2:
            return 0.0
        return (8.0 if (h + k + l) % 4 == 0 else 4.0 * math.sqrt(2.0)) * fprime(s2)

    for hkl in [(1, 1, 1), (2, 0, 0), (2, 2, 0), (2, 2, 2), (3, 3, 3), (5, 1, 1), (4, 0, 0), (4, 2, 0), (6, 0, 0),
                (4, 4, 2), (6, 2, 2), (1, 0, 0), (2, 1, 0), (3, 2, 1), (-1, 1, 1), (-2, -2, 0), (3, -1, 1)]:
        s2, _, _, _ = oracle.refl(oracle.q_of(Gs, *hkl), LAM)
        F = oracle.sf(b, 0, *hkl, s2)
        want = closed(*hkl, s2)
        assert abs(F) == pytest.approx(want, rel=1e-12, abs=1e-12 * fprime(s2)), hkl
    p = oracle.pattern(b, 0, o)
    nmax = (2 * math.sin(math.radians(75.0)) / LAM) ** 2 * a * a
    gold = [r for r in _golden_diamond() if r[0] and r[1] <= nmax]
    assert [r[1] for r in gold] == [3, 8, 11, 16, 19, 24, 27, 32, 35, 40, 43]
    assert len(p["peak_tt"]) == len(gold)
    fo = p["peak_fam_off"]
    for i, (_, n2, fams) in enumerate(gold):
        got = [(tuple(int(x) for x in p["fam_hkl"][f]), int(p["fam_mult"][f])) for f in range(fo[i], fo[i + 1])]
        assert sorted(got) == sorted(fams), (n2, got, fams)
        assert p["peak_tt"][i] == pytest.approx(2 * math.degrees(math.asin(LAM * math.sqrt(n2) / (2 * a))), abs=1e-10)
        s2, _, lp, _ = oracle.refl(oracle.q_of(Gs, *fams[0][0]), LAM)
        want = sum(m * closed(*h, s2) ** 2 for h, m in fams) * lp
        assert p["peak_I"][i] == pytest.approx(want, rel=1e-11), n2


def test_hcp_structure_factor_and_lines():
    """Hexagonal close packing (atoms at (1/3, 2/3, 1/4) and (2/3, 1/3, 3/4) of a hexagonal cell):
    |F|^2 = 4 f'^2 cos^2(pi ((k - h) / 3 - l / 2)), so 00l vanishes for odd l and hh(-2h)l for odd l,
    100 has f'^2 and 101 3 f'^2. Every merged line's intensity is the sum over its reflections."""
    coef = synth.coef_table(np.random.default_rng(4))
    a, c, B, Z = 3.209, 5.211, 0.6, 12
    frac = np.array([[1 / 3, 2 / 3, 0.25], [2 / 3, 1 / 3, 0.75]])
    b = synth.Batch(np.array([[a, a, c, 90.0, 90.0, 120.0]]), np.array([0, 2], np.int64), frac,
                    np.full(2, Z, np.int16), np.ones(2), np.full(2, B), coef)
    _, Gs, _ = oracle.metric(b.lattice[0])

    def f2(h, k, l, s2):
        fp = oracle.fatom(coef, Z, s2) * math.exp(-B * s2)
        return 4.0 * fp * fp * math.cos(math.pi * ((k - h) / 3.0 - l / 2.0)) ** 2

    for hkl in [(0, 0, 1), (0, 0, 2), (0, 0, 3), (1, 0, 0), (1, 0, 1), (1, 0, 2), (1, 1, 0), (1, 1, 1), (1, 1, 2),
                (2, 0, 1), (2, -1, 3), (-1, 2, 1), (3, 0, 0), (2, 1, 1)]:
        s2, _, _, _ = oracle.refl(oracle.q_of(Gs, *hkl), LAM)
        F = oracle.sf(b, 0, *hkl, s2)
        fp = oracle.fatom(coef, Z, s2) * math.exp(-B * s2)
        assert abs(F) ** 2 == pytest.approx(f2(*hkl, s2), rel=1e-11, abs=1e-11 * fp * fp), hkl
    s2, _, _, _ = oracle.refl(oracle.q_of(Gs, 1, 0, 0), LAM)
    fp = oracle.fatom(coef, Z, s2) * math.exp(-B * s2)
    assert f2(1, 0, 0, s2) == pytest.approx(fp * fp) and f2(0, 0, 1, s2) == pytest.approx(0.0, abs=1e-20)
    # merged lines without a cutoff: every reflection of the sphere in exactly one line, line
    # intensity = sum over its members of |F|^2 LP from the closed form
    o = synth.Opts(LAM, 0.0, 120.0, 1e-5, 0.0, 0)
    p = oracle.pattern(b, 0, o)
    hkl, _ = oracle.enumerate_refl(b.lattice[0], o)
    want = {}
    for h, k, l in hkl:
        s2, tt, lp, _ = oracle.refl(oracle.q_of(Gs, h, k, l), LAM)
        key = round(tt, 6)
        want[key] = want.get(key, 0.0) + f2(int(h), int(k), int(l), s2) * lp
    assert len(p["peak_tt"]) == len(want)
    scale = max(want.values())
    for tt, I in zip(p["peak_tt"], p["peak_I"]):
        assert I == pytest.approx(want[round(tt, 6)], rel=1e-9, abs=1e-12 * scale)

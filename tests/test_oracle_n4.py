"""Oracle pins for hexagonal cells (Miller-Bravais families) and multi-species
disordered sites.

Hexagonal cells: families group the reflections of a peak by permutation and
sign of (h, k, i = -h - k, l). For a metrically hexagonal lattice that gives
the multiplicities of Laue class 6/mmm (International Tables for
Crystallography, Vol. A): {0001} 2; {h0-h0} and {hh-2h0} 6; {hki0} general 12;
{h0-hl} and {hh-2hl} 12; {hkil} general 24.

Disordered sites: a site shared by several species is one atom record per
species at the same coordinates with its own occupancy; the structure factor is
linear in those occupancies, and splitting one record into two half-occupied
ones changes nothing.
"""
import numpy as np
import pytest

import oracle
from paper_2602_11709_gb300 import synth


def _opts(**kw):
    o = synth.Opts()
    for k, v in kw.items():
        setattr(o, k, v)
    return o


def _struct(lat, frac, Z, occ, B, coef):
    frac = np.asarray(frac, dtype=np.float64).reshape(-1, 3)
    n = len(frac)
    return synth.Batch(np.asarray([lat], dtype=np.float64), np.array([0, n], np.int64), frac,
                       np.asarray(Z, np.int16), np.asarray(occ, np.float64), np.asarray(B, np.float64), coef)


def _mult_6mmm(h, k, l):
    """Multiplicity of the form {h k i l} in Laue class 6/mmm."""
    i = -h - k
    a = sorted([abs(h), abs(k), abs(i)])
    if a == [0, 0, 0]:
        return 2
    special = a[0] == 0 or a[0] == a[1] or a[1] == a[2]  # an index zero, or two equal magnitudes
    base = 6 if special else 12
    return base if l == 0 else 2 * base


def test_hexagonal_rule():
    assert oracle.is_hexagonal([3.0, 3.0, 5.0, 90.0, 90.0, 120.0])
    assert oracle.is_hexagonal([3.0, 3.009, 5.0, 94.9, 85.1, 115.1])
    assert not oracle.is_hexagonal([3.0, 3.011, 5.0, 90.0, 90.0, 120.0])
    assert not oracle.is_hexagonal([3.0, 3.0, 5.0, 90.0, 90.0, 90.0])
    assert not oracle.is_hexagonal([3.0, 3.0, 5.0, 90.0, 95.0, 120.0])
    assert not oracle.is_hexagonal([3.0, 3.0, 5.0, 90.0, 90.0, 60.0])  # the 60-degree setting is not used


@pytest.mark.parametrize("c", [4.9, 7.31])
def test_hexagonal_families_have_6mmm_multiplicities(c):
    rng = np.random.default_rng(40)
    coef = synth.coef_table(rng)
    n = 5
    b = _struct([3.0, 3.0, c, 90.0, 90.0, 120.0], rng.random((n, 3)), rng.integers(1, 84, n), np.ones(n),
                rng.uniform(0, 1, n), coef)
    res = oracle.pattern(b, 0, _opts(tt_min=0.0, tt_max=120.0, rel_cutoff=0.0, scaled=0))
    assert res["status"] == 0 and len(res["peak_tt"]) > 20
    off = res["peak_fam_off"]
    for p in range(len(res["peak_tt"])):
        for f in range(off[p], off[p + 1]):
            h, k, l = (int(v) for v in res["fam_hkl"][f])
            assert res["fam_mult"][f] == _mult_6mmm(h, k, l), (p, (h, k, l))
    # every reflection of the sphere sits in exactly one family
    assert int(res["fam_mult"].sum()) == res["n_refl"]


def test_hexagonal_first_prism_peak_is_one_family_of_six():
    """{10-10}: (1,0,0), (0,1,0), (1,-1,0) and their negatives share one peak.
    Grouping by (h, k, l) alone would give two families, (1,0,0) x 4 and (1,-1,0) x 2;
    the Miller-Bravais grouping gives one family of 6."""
    rng = np.random.default_rng(41)
    coef = synth.coef_table(rng)
    hexa = _struct([3.0, 3.0, 4.9, 90.0, 90.0, 120.0], rng.random((3, 3)), rng.integers(1, 84, 3), np.ones(3),
                   np.zeros(3), coef)
    res = oracle.pattern(hexa, 0, _opts(tt_min=0.0, tt_max=60.0, rel_cutoff=0.0, scaled=0))
    off = res["peak_fam_off"]
    peaks = [p for p in range(len(res["peak_tt"]))
             if any(tuple(int(v) for v in res["fam_hkl"][f]) == (1, 0, 0) for f in range(off[p], off[p + 1]))]
    assert len(peaks) == 1
    p = peaks[0]
    fams = {tuple(int(v) for v in res["fam_hkl"][f]): int(res["fam_mult"][f]) for f in range(off[p], off[p + 1])}
    assert fams == {(1, 0, 0): 6}


def test_split_site_equals_single_record():
    rng = np.random.default_rng(42)
    coef = synth.coef_table(rng)
    lat = [4.1, 5.2, 6.3, 80.0, 95.0, 105.0]
    frac = rng.random((4, 3))
    Z, B = np.array([8, 26, 14, 30]), rng.uniform(0, 1, 4)
    one = _struct(lat, frac, Z, np.ones(4), B, coef)
    split = _struct(lat, np.vstack([frac, frac[1:2]]), np.append(Z, Z[1]), np.array([1, 0.5, 1, 1, 0.5]),
                    np.append(B, B[1]), coef)
    o = _opts(tt_min=0.0, tt_max=90.0, rel_cutoff=0.0, scaled=0)
    r1, r2 = oracle.pattern(one, 0, o), oracle.pattern(split, 0, o)
    assert np.array_equal(r1["fam_hkl"], r2["fam_hkl"]) and np.array_equal(r1["fam_mult"], r2["fam_mult"])
    assert np.allclose(r1["peak_I"], r2["peak_I"], rtol=1e-12, atol=1e-12 * r1["peak_I"].max())


def test_mixed_site_is_linear_in_the_species_occupancies():
    rng = np.random.default_rng(43)
    coef = synth.coef_table(rng)
    lat = [5.0, 5.5, 7.0, 90.0, 100.0, 90.0]
    frac = rng.random((3, 3))
    site = frac[0]
    Zs, B = [26, 27, 28], np.array([0.3, 0.6, 0.9])  # three species share the site
    x = np.array([0.5, 0.3, 0.2])

    def F(occs, hkl):
        b = _struct(lat, np.vstack([np.tile(site, (3, 1)), frac[1:]]), Zs + [8, 8], np.append(occs, [1, 1]),
                    np.append(B, [0.4, 0.4]), coef)
        _, Gs, _ = oracle.metric(b.lattice[0])
        return oracle.sf(b, 0, *hkl, oracle.q_of(Gs, *hkl) / 4)

    for hkl in [(1, 0, 0), (1, 2, -1), (3, -1, 2), (0, 4, 1)]:
        full = F(x, hkl)
        rest = F(np.zeros(3), hkl)
        parts = [F(np.eye(3)[j], hkl) - rest for j in range(3)]
        assert abs(full - (rest + sum(x[j] * parts[j] for j in range(3)))) <= 1e-12 * max(abs(full), 1.0)


@pytest.mark.parametrize("seed", [50, 51, 52, 53])
def test_family_multiplicities_partition_the_sphere(seed):
    """Without a cutoff every reflection of the sphere is in exactly one family of exactly one
    peak, P1 and hexagonal cells alike, and every family representative lies inside the sphere
    within the merge tolerance above its peak's anchor."""
    rng = np.random.default_rng(seed)
    coef = synth.coef_table(rng)
    hexa = seed % 2 == 0
    if hexa:
        a = rng.uniform(2.5, 6.0)
        lat = [a, a, rng.uniform(3.0, 9.0), 90.0, 90.0, 120.0]
    else:
        lat = list(rng.uniform(3.0, 9.0, 3)) + list(synth._angles(rng, 1)[0])
    n = int(rng.integers(2, 9))
    b = _struct(lat, rng.random((n, 3)), rng.integers(1, 84, n), np.ones(n), rng.uniform(0, 1, n), coef)
    o = _opts(tt_min=0.0, tt_max=100.0, rel_cutoff=0.0, scaled=0)
    res = oracle.pattern(b, 0, o)
    assert oracle.is_hexagonal(lat) == hexa
    assert int(res["fam_mult"].sum()) == res["n_refl"]
    _, Gs, _ = oracle.metric(b.lattice[0])
    off = res["peak_fam_off"]
    for p in range(len(res["peak_tt"])):
        for f in range(off[p], off[p + 1]):
            q = oracle.q_of(Gs, *(int(v) for v in res["fam_hkl"][f]))
            _, tt, _, _ = oracle.refl(q, o.wavelength)
            # the anchor rule: every member of a peak lies in [anchor, anchor + tol)
            assert 0.0 < tt <= o.tt_max and -1e-12 <= tt - res["peak_tt"][p] < o.tt_tol

"""Oracle pins of the symmetry-aware family mode (families = orbits of a caller's point group).

Reference values: the multiplicities of the reflection forms of the Laue classes mmm and 4/mmm
(International Tables for Crystallography, Vol. A, the general and special forms of each class),
and, for m-3m and 6/mmm, the default grouping by permutation and sign (whose classes are those
groups' orbits). Every structure is one atom at the origin, so every reflection is present and
all members of an orbit fall in one peak.
"""
import numpy as np
import pytest

import oracle
from paper_2602_11709_gb300 import adapter, synth


def _one_atom(lat):
    rng = np.random.default_rng(7)
    return synth.Batch(np.array([lat], dtype=np.float64), np.array([0, 1], dtype=np.int64),
                       np.zeros((1, 3)), np.array([26], dtype=np.int16), np.ones(1), np.full(1, 0.3),
                       synth.coef_table(rng))


def _families(b, o):
    res = oracle.pattern_batch(b, o, threads=1)
    fo, hkl, mult = res["peak_fam_off"][0], res["fam_hkl"][0], res["fam_mult"][0]
    return [(tuple(int(v) for v in hkl[f]), int(mult[f])) for f in range(int(fo[-1]))], res


def _opts(pg, tt_max=120.0):
    o = synth.Opts(synth.CU_KA, 0.0, tt_max, 1e-5, 0.0, 1)
    o.point_group = pg
    return o


def test_laue_group_orders():
    orders = {"-1": 2, "2/m": 4, "mmm": 8, "4/m": 8, "4/mmm": 16, "-3": 6, "-3m": 12, "6/m": 12, "6/mmm": 24,
              "m-3": 24, "m-3m": 48}
    for name, n in orders.items():
        ops = adapter.laue_group_ops(name)
        assert ops.shape == (n, 3, 3), name
        assert set(np.unique(ops)) <= {-1, 0, 1}
        # a group: closed under products, every element invertible within it
        S = {tuple(m.ravel()) for m in ops}
        for a in ops:
            for b in ops:
                assert tuple((a @ b).ravel()) in S


def _expected_4mmm(h, k, l):
    a, b, c = abs(h), abs(k), abs(l)
    if a == 0 and b == 0:
        return 2          # {00l}
    if c == 0:
        if a == 0 or b == 0 or a == b:
            return 4      # {h00}, {hh0}
        return 8          # {hk0}
    if a == 0 or b == 0 or a == b:
        return 8          # {h0l}, {hhl}
    return 16             # {hkl}


def _expected_mmm(h, k, l):
    return 2 ** (3 - [h, k, l].count(0))  # {h00} 2, {hk0} 4, {hkl} 8


@pytest.mark.parametrize("name,lat,rule", [("4/mmm", (4.0, 4.0, 6.5, 90.0, 90.0, 90.0), _expected_4mmm),
                                           ("mmm", (4.0, 5.1, 6.5, 90.0, 90.0, 90.0), _expected_mmm)])
def test_multiplicities_of_the_laue_class(name, lat, rule):
    b = _one_atom(lat)
    o = _opts(adapter.laue_group_ops(name))
    fams, res = _families(b, o)
    assert len(fams) > 50
    for hkl, m in fams:
        assert m == rule(*hkl), (name, hkl, m)
    hkl_all, _ = oracle.enumerate_refl(b.lattice[0], o)
    assert sum(m for _, m in fams) == len(hkl_all)  # every reflection of the sphere in one family


@pytest.mark.parametrize("name,lat", [("m-3m", (5.64, 5.64, 5.64, 90.0, 90.0, 90.0)),
                                      ("6/mmm", (3.2, 3.2, 5.2, 90.0, 90.0, 120.0))])
def test_holohedry_equals_the_default_grouping(name, lat):
    """m-3m on a cubic cell and 6/mmm (hexagonal axes) on a hexagonal cell: the orbits are the
    default classes (permutation and sign of (h, k, l), of (h, k, i, l) for the hexagonal cell)."""
    b = _one_atom(lat)
    with_pg, _ = _families(b, _opts(adapter.laue_group_ops(name)))
    default, _ = _families(b, _opts(None))
    assert with_pg == default


def test_friedel_pairs_only_for_the_trivial_group():
    b = _one_atom((4.0, 4.0, 6.5, 90.0, 90.0, 90.0))
    fams, _ = _families(b, _opts(adapter.laue_group_ops("-1")))
    assert fams and all(m == 2 for _, m in fams)

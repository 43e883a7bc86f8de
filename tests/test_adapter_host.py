"""Host logic of the calculator-style adapter: structure conversion, batching, 4-index output."""
import numpy as np
import pytest

from paper_2602_11709_gb300 import adapter, xrd, synth


class _El:
    def __init__(self, symbol):
        self.symbol = symbol


class _Lattice:
    def __init__(self, abc, angles):
        self.abc, self.angles = abc, angles


class _Site:
    def __init__(self, species, frac):
        self.species, self.frac_coords = species, np.asarray(frac)


class _Structure:  # the attributes of a pymatgen Structure that the adapter reads
    def __init__(self, lat, sites):
        self.lattice = _Lattice(tuple(lat[:3]), tuple(lat[3:]))
        self.sites = sites


DICT = {"lattice": (4.0, 4.0, 6.5, 90.0, 90.0, 120.0),
        "sites": [{"species": {"Zn": 1.0}, "frac": (1 / 3, 2 / 3, 0.0)},
                  {"species": {"O": 0.6, "S": 0.4}, "frac": (1 / 3, 2 / 3, 0.38)}]}


def test_dict_and_object_forms_agree_and_split_shared_sites():
    dw = {"Zn": 0.5, "O": 0.3}
    a = adapter.structure_arrays(DICT, dw)
    obj = _Structure(DICT["lattice"], [_Site({_El("Zn"): 1.0}, (1 / 3, 2 / 3, 0.0)),
                                        _Site({"O2-": 0.6, _El("S"): 0.4}, (1 / 3, 2 / 3, 0.38))])
    b = adapter.structure_arrays(obj, dw)
    for x, y in zip(a, b):
        assert np.allclose(x, y)
    lat, frac, Z, occ, B = a
    assert Z.tolist() == [30, 8, 16] and occ.tolist() == [1.0, 0.6, 0.4] and B.tolist() == [0.5, 0.3, 0.0]
    assert np.allclose(frac[1], frac[2])


def test_batch_of_and_limits():
    coef = synth.coef_table(np.random.default_rng(1))
    b = adapter.batch_of([DICT, DICT], coef)
    assert b.n_struct == 2 and b.atom_off.tolist() == [0, 3, 6] and b.zmax == coef.shape[0] - 1
    with pytest.raises(ValueError):
        adapter.batch_of([DICT], coef[:20])  # Zn (30) beyond the table
    with pytest.raises(ValueError):
        adapter.structure_arrays({"lattice": DICT["lattice"], "sites": [{"species": {"Xx": 1}, "frac": (0, 0, 0)}]})


def test_wavelengths_and_hexagonal_output():
    assert adapter.WAVELENGTHS["CuKa"] == synth.CU_KA
    assert len(adapter.ELEMENTS) == 83 and adapter.Z_OF["Bi"] == 83
    res = {"peak_tt": [np.array([20.0, 30.0]), np.array([25.0])], "peak_I": [np.array([100.0, 5.0]), np.array([100.0])],
           "peak_d": [np.array([2.0, 1.5]), np.array([1.8])],
           "peak_fam_off": [np.array([0, 1, 3]), np.array([0, 1])],
           "fam_hkl": [np.array([[1, 0, 0], [1, 0, 1], [0, 0, 2]]), np.array([[1, 1, 0]])],
           "fam_mult": [np.array([6, 12, 2]), np.array([4])], "status": np.array([0, 0]),
           "flags": np.array([xrd.XRD_FLAG_HEXAGONAL, 0], np.int32)}
    pats = adapter.patterns_from(res)
    assert pats[0].hkls == [[{"hkl": (1, 0, -1, 0), "multiplicity": 6}],
                            [{"hkl": (1, 0, -1, 1), "multiplicity": 12}, {"hkl": (0, 0, 0, 2), "multiplicity": 2}]]
    assert pats[1].hkls == [[{"hkl": (1, 1, 0), "multiplicity": 4}]]
    assert pats[0].x.tolist() == [20.0, 30.0] and pats[1].d_hkls.tolist() == [1.8]

"""The calculator-style adapter on the GPU against the oracle (positions, intensities, families)."""
import numpy as np
import pytest

import oracle
from paper_2602_11709_gb300 import adapter, synth, xrd

pytestmark = pytest.mark.gpu

STRUCTS = [
    {"lattice": (5.64, 5.64, 5.64, 90.0, 90.0, 90.0),  # rock salt
     "sites": [{"species": {"Na": 1.0}, "frac": f} for f in [(0, 0, 0), (0, .5, .5), (.5, 0, .5), (.5, .5, 0)]] +
              [{"species": {"Cl": 1.0}, "frac": f} for f in [(.5, 0, 0), (.5, .5, .5), (0, 0, .5), (0, .5, 0)]]},
    {"lattice": (3.25, 3.25, 5.21, 90.0, 90.0, 120.0),  # wurtzite-like, one shared anion site
     "sites": [{"species": {"Zn": 1.0}, "frac": (1 / 3, 2 / 3, 0.0)}, {"species": {"Zn": 1.0}, "frac": (2 / 3, 1 / 3, 0.5)},
               {"species": {"O": 0.7, "S": 0.3}, "frac": (1 / 3, 2 / 3, 0.382)},
               {"species": {"O": 1.0}, "frac": (2 / 3, 1 / 3, 0.882)}]},
    {"lattice": (4.1, 5.3, 6.2, 81.0, 97.0, 104.0),
     "sites": [{"species": {"Fe": 0.5, "Co": 0.5}, "frac": (0.1, 0.2, 0.3)}, {"species": {"Si": 1.0}, "frac": (0.6, 0.7, 0.1)}]},
]


def test_get_patterns_matches_oracle(gpu_lib):
    coef = synth.coef_table(np.random.default_rng(3))
    dw = {"Na": 0.4, "Cl": 0.6, "O": 0.3}
    calc = adapter.XRDCalculator(coef, "CuKa", dw)
    pats = calc.get_patterns(STRUCTS, scaled=True, two_theta_range=(5, 100))
    b = adapter.batch_of(STRUCTS, coef, dw)
    o = synth.Opts(adapter.WAVELENGTHS["CuKa"], 5.0, 100.0, 1e-5, 1e-3, 1)
    for s, p in enumerate(pats):
        ref = oracle.pattern(b, s, o, with_refl=False)
        assert p.status == 0 and len(p.x) == len(ref["peak_tt"])
        assert np.abs(p.x - ref["peak_tt"]).max() <= 1e-6
        assert np.abs(p.y - ref["peak_I"]).max() <= 1e-5 * 100.0
        assert np.allclose(p.d_hkls, ref["peak_d"], rtol=1e-12)
        hexa = oracle.is_hexagonal(b.lattice[s])
        off = ref["peak_fam_off"]
        for k in range(len(p.x)):
            want = [(tuple(xrd.miller_bravais(ref["fam_hkl"][f]).tolist()) if hexa else
                     tuple(int(v) for v in ref["fam_hkl"][f]), int(ref["fam_mult"][f])) for f in range(off[k], off[k + 1])]
            got = [(f["hkl"], f["multiplicity"]) for f in p.hkls[k]]
            assert got == want, (s, k)
    assert pats[0].hkls[1] == [{"hkl": (2, 0, 0), "multiplicity": 6}]  # NaCl {200}
    assert any(len(f["hkl"]) == 4 and f["multiplicity"] == 6 for fam in pats[1].hkls for f in fam)

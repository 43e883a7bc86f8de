"""Hexagonal cells (Miller-Bravais families) and multi-species disordered sites
on the GPU against the oracle, every precision (bar as in parity.py: families
identical, positions to 1e-6 deg, intensities to the precision's tolerance)."""
import numpy as np
import pytest

import oracle
from paper_2602_11709_gb300 import synth

from parity import compare_batch, families

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def handle(gpu_lib):
    h = gpu_lib.Handle(0)
    yield h
    h.close()


@pytest.mark.parametrize("prec", ["fp64", "fp32_phase64", "fp32_phasefix"])
def test_hexagonal_and_disordered_batch(gpu_lib, handle, prec):
    b, o = synth.hexdis()
    ref = oracle.pattern_batch(b, o, threads=0)
    got = gpu_lib.compute(b, o, prec, handle=handle)
    st = compare_batch(got, ref, prec, o.rel_cutoff, o.scaled)
    assert st["pairs"] > 50000
    hexa = (got["flags"] & gpu_lib.XRD_FLAG_HEXAGONAL) != 0
    assert hexa.tolist() == [bool(oracle.is_hexagonal(lat)) for lat in b.lattice]
    assert hexa.sum() == b.n_struct // 2
    # the hexagonal cells' families carry 6/mmm multiplicities; a 6-member {10-10} family is present
    six = 0
    for s in np.nonzero(hexa)[0]:
        for p in range(len(got["peak_tt"][s])):
            for hkl, m in families(got, s, p):
                assert m in (2, 6, 12, 24), (s, hkl, m)
                six += hkl == (1, 0, 0) and m == 6
    assert six > 0


def test_hexagonal_flag_only_changes_families(gpu_lib, handle):
    """A cell just outside the rule (|a - b| = 0.011 A) keeps (h, k, l) families."""
    b, o = synth.hexdis(n=8)
    lat = b.lattice.copy()
    lat[0, 1] = lat[0, 0] + 0.011
    b2 = synth.Batch(lat, b.atom_off, b.frac, b.Z, b.occ, b.B, b.coef)
    assert not oracle.is_hexagonal(lat[0])
    ref = oracle.pattern_batch(b2, o, threads=1)
    got = gpu_lib.compute(b2, o, "fp32_phasefix", handle=handle)
    assert not got["flags"][0] & gpu_lib.XRD_FLAG_HEXAGONAL
    compare_batch(got, ref, "fp32_phasefix", o.rel_cutoff, o.scaled)


def test_hexagonal_flag_matches_oracle_rule_on_boundaries(gpu_lib, handle):
    """The library's flag word against the oracle's rule, cells on and around the 5 degree and
    0.01 A boundaries (and one invalid cell, which is never hexagonal)."""
    rng = np.random.default_rng(7)
    cells = [[3.0, 3.0, 5.0, 90.0, 90.0, 120.0], [3.0, 3.0099, 5.0, 94.99, 85.01, 124.99],
             [3.0, 3.0101, 5.0, 90.0, 90.0, 120.0], [3.0, 3.0, 5.0, 95.0, 90.0, 120.0],
             [3.0, 3.0, 5.0, 90.0, 90.0, 115.0], [3.0, 3.0, 5.0, 90.0, 90.0, 60.0], [np.nan, 3.0, 5.0, 90, 90, 120]]
    for _ in range(200):
        a = rng.uniform(2, 8)
        cells.append([a, a + rng.normal(0, 0.01), rng.uniform(2, 8), 90 + rng.normal(0, 4), 90 + rng.normal(0, 4),
                      120 + rng.normal(0, 4)])
    lat = np.array(cells)
    n = len(lat)
    b = synth.Batch(lat, np.arange(n + 1, dtype=np.int64), np.full((n, 3), 0.1), np.full(n, 8, np.int16),
                    np.ones(n), np.full(n, 0.3), synth.coef_table(np.random.default_rng(1)))
    o = synth.Opts(1.54184, 5.0, 60.0, 1e-5, 1e-3, 1)
    got = gpu_lib.compute(b, o, "fp32_phasefix", handle=handle)
    want = [bool(oracle.is_hexagonal(c)) for c in lat]
    assert [bool(f & gpu_lib.XRD_FLAG_HEXAGONAL) for f in got["flags"]] == want
    assert 0 < sum(want) < n

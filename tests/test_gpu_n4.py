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
    hexa = gpu_lib.is_hexagonal(b.lattice)
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
    assert not gpu_lib.is_hexagonal(lat)[0]
    ref = oracle.pattern_batch(b2, o, threads=1)
    got = gpu_lib.compute(b2, o, "fp32_phasefix", handle=handle)
    compare_batch(got, ref, "fp32_phasefix", o.rel_cutoff, o.scaled)

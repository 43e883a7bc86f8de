"""The symmetry-aware family mode on the GPU against the oracle (same operations on both sides),
every precision: one-atom cells of the tetragonal, orthorhombic, cubic and hexagonal holohedries,
a small random P1 batch under 4/mmm (orbits that are not peaks of the structure: families still
group the members of each merged peak by orbit), and a tetragonal cell above 6144 reflections
(the flat post passes)."""
import numpy as np
import pytest

import oracle
from paper_2602_11709_gb300 import adapter, synth

from parity import compare_batch, families

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def handle(gpu_lib):
    h = gpu_lib.Handle(0)
    yield h
    h.close()


def _cells(lats, seed=11):
    rng = np.random.default_rng(seed)
    n = len(lats)
    # one atom at the origin and, for half the cells, a second one at the body centre
    counts = np.array([1 + (i % 2) for i in range(n)], dtype=np.int64)
    off = np.zeros(n + 1, np.int64)
    off[1:] = np.cumsum(counts)
    frac = np.vstack([[[0, 0, 0]] if c == 1 else [[0, 0, 0], [.5, .5, .5]] for c in counts]).astype(np.float64)
    Z = np.array([26 if j % 2 == 0 else 8 for j in range(int(off[-1]))], dtype=np.int16)
    return synth.Batch(np.array(lats, dtype=np.float64), off, frac, Z, np.ones(int(off[-1])),
                       rng.uniform(0.1, 1.0, int(off[-1])), synth.coef_table(rng))


CASES = {
    "4/mmm": [(4.0, 4.0, 6.5, 90, 90, 90), (3.3, 3.3, 9.1, 90, 90, 90), (5.0, 5.0, 4.2, 90, 90, 90)],
    "mmm": [(4.0, 5.1, 6.5, 90, 90, 90), (3.1, 7.2, 5.5, 90, 90, 90)],
    "m-3m": [(5.64, 5.64, 5.64, 90, 90, 90), (4.05, 4.05, 4.05, 90, 90, 90)],
    "6/mmm": [(3.2, 3.2, 5.2, 90, 90, 120), (2.5, 2.5, 6.7, 90, 90, 120)],
}


@pytest.mark.parametrize("prec", ["fp64", "fp32_phase64", "fp32_phasefix"])
@pytest.mark.parametrize("group", sorted(CASES))
def test_point_group_families(gpu_lib, handle, group, prec):
    b = _cells(CASES[group])
    o = synth.Opts(synth.CU_KA, 0.0, 150.0, 1e-5, 0.0, 1)
    o.point_group = adapter.laue_group_ops(group)
    ref = oracle.pattern_batch(b, o, threads=0)
    got = gpu_lib.compute(b, o, prec, handle=handle)
    st = compare_batch(got, ref, prec, o.rel_cutoff, o.scaled)
    assert st["pairs"] > 40
    n_multi = sum(len(families(got, s, p)) and max(m for _, m in families(got, s, p)) > 2
                  for s in range(b.n_struct) for p in range(len(got["peak_tt"][s])))
    assert n_multi > 20  # orbits larger than a Friedel pair are present


def test_point_group_on_random_cells_and_reset(gpu_lib, handle):
    b, o = synth.small(n=48)
    o.point_group = adapter.laue_group_ops("4/mmm")
    ref = oracle.pattern_batch(b, o, threads=0)
    got = gpu_lib.compute(b, o, "fp32_phasefix", handle=handle)
    compare_batch(got, ref, "fp32_phasefix", o.rel_cutoff, o.scaled)
    o.point_group = None  # the next call restores the default grouping
    ref0 = oracle.pattern_batch(b, o, threads=0)
    got0 = gpu_lib.compute(b, o, "fp32_phasefix", handle=handle)
    compare_batch(got0, ref0, "fp32_phasefix", o.rel_cutoff, o.scaled)


def test_point_group_flat_passes(gpu_lib, handle):
    """A tetragonal cell with more than 6144 Friedel-unique reflections goes through the flat
    device-wide post passes; their family keys come from the same orbit rule."""
    b = _cells([(14.0, 14.0, 21.0, 90, 90, 90), (4.0, 4.0, 6.5, 90, 90, 90)])
    o = synth.Opts(synth.CU_KA, 0.0, 120.0, 1e-5, 0.0, 1)
    o.point_group = adapter.laue_group_ops("4/mmm")
    ref = oracle.pattern_batch(b, o, threads=0)
    got = gpu_lib.compute(b, o, "fp32_phasefix", handle=handle)
    assert got["sizes"]["max_refl"] > 6144
    st = compare_batch(got, ref, "fp32_phasefix", o.rel_cutoff, o.scaled)
    assert st["pairs"] > 500


def test_bad_point_groups_are_refused(gpu_lib, handle):
    with pytest.raises(Exception):
        handle.set_point_group(np.full((1, 3, 3), 2, np.int32))  # entries outside {-1, 0, 1}
    with pytest.raises(Exception):
        handle.set_point_group(np.zeros((49, 3, 3), np.int32))   # more than 48 operations
    handle.set_point_group(None)

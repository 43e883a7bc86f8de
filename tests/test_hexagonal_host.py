"""Host-side hexagonal rule and Miller-Bravais conversion of the binding against the oracle's rule."""
import numpy as np

import oracle
from paper_2602_11709_gb300 import xrd


def test_rule_matches_oracle_on_boundaries():
    rng = np.random.default_rng(7)
    cells = [[3.0, 3.0, 5.0, 90.0, 90.0, 120.0], [3.0, 3.0099, 5.0, 94.99, 85.01, 124.99],
             [3.0, 3.0101, 5.0, 90.0, 90.0, 120.0], [3.0, 3.0, 5.0, 95.0, 90.0, 120.0],
             [3.0, 3.0, 5.0, 90.0, 90.0, 115.0], [3.0, 3.0, 5.0, 90.0, 90.0, 60.0], [np.nan, 3.0, 5.0, 90, 90, 120]]
    for _ in range(200):
        a = rng.uniform(2, 8)
        cells.append([a, a + rng.normal(0, 0.01), rng.uniform(2, 8), 90 + rng.normal(0, 4), 90 + rng.normal(0, 4),
                      120 + rng.normal(0, 4)])
    cells = np.array(cells)
    got = xrd.is_hexagonal(cells)
    assert [bool(g) for g in got] == [oracle.is_hexagonal(c) for c in cells]
    assert 0 < got.sum() < len(cells)


def test_miller_bravais():
    hkl = np.array([[1, 0, 0], [1, -1, 2], [-2, 3, 5]])
    mb = xrd.miller_bravais(hkl)
    assert mb.tolist() == [[1, 0, -1, 0], [1, -1, 0, 2], [-2, 3, -1, 5]]
    assert np.all(mb[:, :3].sum(axis=1) == 0)

"""Host-side Miller-Bravais conversion of the binding (the hexagonal rule itself is the library's:
its flag word is checked against the oracle's rule in tests/test_gpu_n4.py)."""
import numpy as np

from paper_2602_11709_gb300 import xrd


def test_miller_bravais():
    hkl = np.array([[1, 0, 0], [1, -1, 2], [-2, 3, 5]])
    mb = xrd.miller_bravais(hkl)
    assert mb.tolist() == [[1, 0, -1, 0], [1, -1, 0, 2], [-2, 3, -1, 5]]
    assert np.all(mb[:, :3].sum(axis=1) == 0)


def test_binding_does_not_restate_the_rule():
    """The 4-index decision comes from the library (XRD_FLAG_HEXAGONAL), not from Python."""
    assert not hasattr(xrd, "is_hexagonal")
    assert xrd.XRD_FLAG_HEXAGONAL == 1

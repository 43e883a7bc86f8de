"""Pins of the oracle's augmented pattern (pseudo-Voigt profile, March-Dollase
preferred orientation, caller-supplied noise).

The profile is pinned by its integral (the closed forms of the Lorentzian and
Gaussian areas between the grid ends), by the half maximum at 2theta +- fwhm/2
for every mixing eta, and by its Gaussian limit against the oracle's
unit-height broadened pattern; the March-Dollase factor by its closed forms at
0, 45 and 90 degrees, its symmetries, its normalisation over the sphere (mean 1
over uniformly distributed directions) and, in a triclinic cell, the angle
between g and n taken from Cartesian reciprocal vectors; the noise by its limits.
"""
import math

import numpy as np
import pytest

import oracle
from paper_2602_11709_gb300 import synth


def _case(seed=11, n_atoms=6):
    rng = np.random.default_rng(seed)
    b = synth.random_cell(rng, n_atoms, edge=(3.5, 5.0))
    o = synth.Opts(synth.CU_KA, 5.0, 90.0, 1e-5, 0.0, 0)
    hkl, _ = oracle.enumerate_refl(b.lattice[0], o)
    return b, o, hkl


def _one(b, o, hkl, lo=30.0, hi=60.0):
    """One reflection of the list with 2theta inside (lo, hi), its 2theta and I = |F|^2 LP."""
    _, Gs, _ = oracle.metric(b.lattice[0])
    for h, k, l in hkl:
        s2, tt, lp, _ = oracle.refl(oracle.q_of(Gs, h, k, l), o.wavelength)
        if lo < tt < hi:
            F = oracle.sf(b, 0, int(h), int(k), int(l), s2)
            return np.array([[h, k, l]], dtype=np.int32), tt, abs(F) ** 2 * lp
    raise AssertionError("no reflection in range")


@pytest.mark.parametrize("eta", [0.0, 0.35, 1.0])
def test_profile_area_matches_closed_form(eta):
    b, o, hkl = _case()
    one, tt, I = _one(b, o, hkl)
    fwhm = 0.3
    t0, dt, n = tt - 40.0, fwhm / 400.0, 32001  # 80 degrees around the peak
    y = oracle.augmented(b, 0, one, o.wavelength, t0, dt, n, fwhm, eta)
    area = np.trapezoid(y, dx=dt)
    a, c = t0 - tt, t0 + (n - 1) * dt - tt
    lor = (math.atan(2 * c / fwhm) - math.atan(2 * a / fwhm)) / math.pi
    k = 2 * math.sqrt(math.log(2)) / fwhm
    gau = 0.5 * (math.erf(k * c) - math.erf(k * a))
    assert area == pytest.approx(I * (eta * lor + (1 - eta) * gau), rel=2e-6)


@pytest.mark.parametrize("eta", [0.0, 0.5, 1.0])
def test_profile_half_maximum_at_half_width(eta):
    b, o, hkl = _case(12)
    one, tt, _ = _one(b, o, hkl)
    fwhm = 0.2
    y = oracle.augmented(b, 0, one, o.wavelength, tt - fwhm / 2, fwhm / 2, 3, fwhm, eta)
    assert y[0] == pytest.approx(y[1] / 2, rel=1e-12)
    assert y[2] == pytest.approx(y[1] / 2, rel=1e-12)


def test_gaussian_limit_is_the_broadened_pattern_normalised():
    b, o, hkl = _case(13)
    grid = synth.Grid()
    y_aug = oracle.augmented(b, 0, hkl, o.wavelength, grid.t0, grid.dt, grid.n_pts, grid.fwhm, 0.0)
    y_gau = oracle.broadened(b, 0, hkl, o.wavelength, grid)
    scale = (2.0 / grid.fwhm) * math.sqrt(math.log(2) / math.pi)
    assert np.allclose(y_aug, scale * y_gau, rtol=1e-12, atol=1e-12 * y_aug.max())


def test_superposition():
    b, o, hkl = _case(14)
    half = len(hkl) // 2
    args = (o.wavelength, 5.0, 0.02, 4000, 0.15, 0.4, (1.0, 0.0, 2.0), 1.4)
    y = oracle.augmented(b, 0, hkl, *args)
    y1 = oracle.augmented(b, 0, hkl[:half], *args)
    y2 = oracle.augmented(b, 0, hkl[half:], *args)
    assert np.allclose(y, y1 + y2, rtol=1e-12, atol=1e-12 * y.max())


@pytest.mark.parametrize("r", [0.5, 0.8, 1.3, 2.0])
def test_march_dollase_closed_forms_and_symmetry(r):
    lat = np.array([4.0, 4.0, 4.0, 90.0, 90.0, 90.0])
    n = (0.0, 0.0, 1.0)
    assert oracle.march_dollase(lat, 0, 0, 2, n, r) == pytest.approx(r ** -3, rel=1e-13)  # g parallel to n
    assert oracle.march_dollase(lat, 3, 0, 0, n, r) == pytest.approx(r ** 1.5, rel=1e-13)  # perpendicular
    assert oracle.march_dollase(lat, 1, 0, 1, n, r) == pytest.approx((r * r / 2 + 1 / (2 * r)) ** -1.5, rel=1e-13)
    lat2 = np.array([4.1, 5.3, 6.2, 81.0, 97.0, 104.0])
    for g in ((1, 2, 3), (-2, 1, 0), (3, -1, 2)):
        p = oracle.march_dollase(lat2, *g, (1.0, -1.0, 2.0), r)
        assert oracle.march_dollase(lat2, *(-np.array(g)), (1.0, -1.0, 2.0), r) == pytest.approx(p, rel=1e-13)
        assert oracle.march_dollase(lat2, *g, (-2.0, 2.0, -4.0), r) == pytest.approx(p, rel=1e-13)
        assert oracle.march_dollase(lat2, *g, (1.0, -1.0, 2.0), 1.0) == pytest.approx(1.0, rel=1e-14)


@pytest.mark.parametrize("r", [0.6, 1.0, 1.7])
def test_march_dollase_is_normalised_over_the_sphere(r):
    """Mean of P over directions uniform on the sphere = 1: Gauss-Legendre in cos(alpha),
    directions realised as long integer vectors of a cubic cell."""
    lat = np.array([1.0, 1.0, 1.0, 90.0, 90.0, 90.0])
    c, w = np.polynomial.legendre.leggauss(48)
    mean = 0.0
    for ci, wi in zip(c, w):
        si = math.sqrt(1 - ci * ci)
        g = (int(round(4000 * si)), 0, int(round(4000 * ci)))
        mean += 0.5 * wi * oracle.march_dollase(lat, *g, (0.0, 0.0, 1.0), r)
    assert mean == pytest.approx(1.0, rel=2e-3)


def test_noise_limits():
    b, o, hkl = _case(15)
    args = (o.wavelength, 10.0, 0.05, 800, 0.2, 0.3)
    y = oracle.augmented(b, 0, hkl, *args)
    z = np.random.default_rng(3).standard_normal(800)
    assert np.array_equal(oracle.augmented(b, 0, hkl, *args, z=z, sigma=0.0), y)
    assert np.array_equal(oracle.augmented(b, 0, hkl, *args, z=np.zeros(800), sigma=0.7), y)
    d1 = oracle.augmented(b, 0, hkl, *args, z=z, sigma=0.5) - y
    d2 = oracle.augmented(b, 0, hkl, *args, z=z, sigma=1.0) - y
    assert np.allclose(d2, 2 * d1, rtol=1e-12, atol=1e-12 * np.abs(d2).max())
    assert np.all(np.sign(d1[y > 0]) == np.sign(z[y > 0]))


def test_march_dollase_angle_in_a_triclinic_cell():
    """The angle between g and n from Cartesian reciprocal vectors (rows of inv(A).T for the
    direct cell vectors A, built from a, b, c, alpha, beta, gamma independently of the metric
    tensors) agrees with the oracle's metric form for a low-symmetry cell."""
    lat = np.array([4.1, 5.3, 6.2, 81.0, 97.0, 104.0])
    a, b, c = lat[:3]
    al, be, ga = np.radians(lat[3:])
    A = np.zeros((3, 3))
    A[0] = [a, 0.0, 0.0]
    A[1] = [b * np.cos(ga), b * np.sin(ga), 0.0]
    cx = c * np.cos(be)
    cy = c * (np.cos(al) - np.cos(be) * np.cos(ga)) / np.sin(ga)
    A[2] = [cx, cy, np.sqrt(c * c - cx * cx - cy * cy)]
    Bstar = np.linalg.inv(A).T  # rows: a*, b*, c*
    r = 1.3
    for g in ((1, 2, 3), (-2, 1, 0), (3, -1, 2), (0, 0, 1)):
        for n in ((1.0, -1.0, 2.0), (0.0, 1.0, 0.0), (2.0, 0.5, -1.0)):
            gc, nc = np.asarray(g) @ Bstar, np.asarray(n) @ Bstar
            cos2 = (gc @ nc) ** 2 / ((gc @ gc) * (nc @ nc))
            want = (r * r * cos2 + (1.0 - cos2) / r) ** -1.5
            assert oracle.march_dollase(lat, *g, n, r) == pytest.approx(want, rel=1e-12), (g, n)

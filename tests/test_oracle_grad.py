"""Pins of the oracle's broadened pattern and its analytic gradient.

The broadened profile is pinned by the Gaussian integral (area I sigma sqrt(2 pi))
and the textbook FWHM = 2 sqrt(2 ln 2) sigma; the analytic gradient by 5-point
finite differences of the oracle's own forward pattern (coordinates, B factors
and all six lattice parameters, on a fixed reflection list) and by translation
invariance (shifting every atom changes no intensity, so sum_j dL/dx_j = 0);
the coordinate and B gradients also by the closed forms of one- and two-atom cells.
"""
import math

import numpy as np
import pytest

import oracle
from paper_2602_11709_gb300 import synth


def _small_case(seed, n_atoms=5, edge=(3.2, 4.5)):
    rng = np.random.default_rng(seed)
    b = synth.random_cell(rng, n_atoms, edge=edge)
    o = synth.Opts(synth.CU_KA, 5.0, 90.0, 1e-5, 0.0, 0)
    grid = synth.Grid()
    hkl, _ = oracle.enumerate_refl(b.lattice[0], o)
    g = rng.standard_normal(grid.n_pts)
    return b, o, grid, hkl, g


def _loss(b, hkl, o, grid, g):
    return float(np.dot(g, oracle.broadened(b, 0, hkl, o.wavelength, grid)))


def _fd(fun, x0, h):
    return (fun(x0 - 2 * h) - 8 * fun(x0 - h) + 8 * fun(x0 + h) - fun(x0 + 2 * h)) / (12 * h)


def _rel(a, b):
    a, b = np.asarray(a), np.asarray(b)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def test_broadened_area_and_width():
    b, o, grid, hkl, _ = _small_case(1)
    p = oracle.pattern(b, 0, o)
    # the strongest reflection alone
    r = int(np.argmax(p["refl_I"] * (p["refl_tt"] > 20) * (p["refl_tt"] < 80)))
    one = p["refl_hkl"][r:r + 1]
    y = oracle.broadened(b, 0, one, o.wavelength, grid)
    I, tt = p["refl_I"][r], p["refl_tt"][r]
    sigma = grid.fwhm / (2 * math.sqrt(2 * math.log(2)))
    assert y.sum() * grid.dt == pytest.approx(I * sigma * math.sqrt(2 * math.pi), rel=1e-9)
    t = grid.t0 + grid.dt * np.arange(grid.n_pts)
    k = int(np.argmax(y))
    assert abs(t[k] - tt) <= grid.dt / 2 + 1e-12
    # width at half maximum of the sampled Gaussian, by interpolation on both flanks
    yy = y / I

    def cross(side):
        idx = np.arange(k, -1, -1) if side < 0 else np.arange(k, grid.n_pts)
        for a, c in zip(idx[:-1], idx[1:]):
            if yy[c] < 0.5 <= yy[a]:
                return t[a] + (t[c] - t[a]) * (yy[a] - 0.5) / (yy[a] - yy[c])
    # the Gaussian is sampled coarsely (dt ~ sigma / 2): compare against the exact
    # half-maximum points of exp(-(t - tt)^2 / (2 sigma^2)) interpolated the same way
    exact = np.exp(-(t - tt) ** 2 / (2 * sigma ** 2))
    assert np.allclose(yy, exact, atol=1e-12)
    half = sigma * math.sqrt(2 * math.log(2))
    assert half * 2 == pytest.approx(grid.fwhm, rel=1e-12)
    assert cross(+1) - cross(-1) == pytest.approx(grid.fwhm, rel=0.1)


def test_broadened_is_sum_over_reflections():
    b, o, grid, hkl, _ = _small_case(2)
    y_all = oracle.broadened(b, 0, hkl, o.wavelength, grid)
    half = len(hkl) // 2
    y_a = oracle.broadened(b, 0, hkl[:half], o.wavelength, grid)
    y_b = oracle.broadened(b, 0, hkl[half:], o.wavelength, grid)
    assert np.allclose(y_all, y_a + y_b, rtol=1e-12, atol=1e-9 * y_all.max())


@pytest.mark.parametrize("seed", [3, 4])
def test_gradient_coordinates_and_b_vs_finite_differences(seed):
    b, o, grid, hkl, g = _small_case(seed)
    df, dB, dl = oracle.broadened_grad(b, 0, hkl, o.wavelength, grid, g)
    n = b.n_atoms
    fd_x = np.zeros((n, 3))
    fd_B = np.zeros(n)
    for j in range(n):
        for d in range(3):
            def f(v, j=j, d=d):
                bb = synth.Batch(b.lattice, b.atom_off, b.frac.copy(), b.Z, b.occ, b.B, b.coef)
                bb.frac[j, d] = v
                return _loss(bb, hkl, o, grid, g)
            fd_x[j, d] = _fd(f, b.frac[j, d], 1e-5)

        def fB(v, j=j):
            bb = synth.Batch(b.lattice, b.atom_off, b.frac, b.Z, b.occ, b.B.copy(), b.coef)
            bb.B[j] = v
            return _loss(bb, hkl, o, grid, g)
        fd_B[j] = _fd(fB, b.B[j], 1e-4)
    assert _rel(df, fd_x) < 1e-6
    assert _rel(dB, fd_B) < 1e-6


@pytest.mark.parametrize("seed", [5, 6])
def test_gradient_lattice_vs_finite_differences(seed):
    b, o, grid, hkl, g = _small_case(seed)
    _, _, dl = oracle.broadened_grad(b, 0, hkl, o.wavelength, grid, g)
    fd = np.zeros(6)
    for m in range(6):
        def f(v, m=m):
            bb = synth.Batch(b.lattice.copy(), b.atom_off, b.frac, b.Z, b.occ, b.B, b.coef)
            bb.lattice[0, m] = v
            return _loss(bb, hkl, o, grid, g)
        h = 1e-6 * b.lattice[0, m] if m < 3 else 1e-5
        fd[m] = _fd(f, b.lattice[0, m], h)
    assert _rel(dl, fd) < 1e-6, (dl, fd)


def test_gradient_translation_invariance():
    b, o, grid, hkl, g = _small_case(7, n_atoms=9)
    df, _, _ = oracle.broadened_grad(b, 0, hkl, o.wavelength, grid, g)
    assert np.abs(df.sum(axis=0)).max() < 1e-9 * np.abs(df).max()


def _weights(hkl, lat, lam, grid, g):
    """Per reflection: s^2, LP, 2-theta, and c_r = sum_k g_k exp(-(t_k - 2theta_r)^2 / (2 sigma^2))."""
    _, Gs, _ = oracle.metric(lat)
    t = grid.t0 + grid.dt * np.arange(grid.n_pts)
    sigma = grid.fwhm / (2 * math.sqrt(2 * math.log(2)))
    out = []
    for h, k, l in hkl:
        s2, tt, lp, _ = oracle.refl(oracle.q_of(Gs, h, k, l), lam)
        out.append((s2, lp, float(np.dot(g, np.exp(-(t - tt) ** 2 / (2 * sigma ** 2))))))
    return out


def test_gradient_closed_forms_one_and_two_atoms():
    """Single atom: I = (occ f e^{-B s^2})^2 LP, so dI/dB = -2 s^2 I and dI/dx = 0. Two atoms with
    weights w_j = occ_j f_j e^{-B_j s^2}: I = LP (w1^2 + w2^2 + 2 w1 w2 cos 2 pi g.(x1 - x2)), so
    dI/dx1 = -4 pi LP w1 w2 sin(2 pi g.(x1 - x2)) g = -dI/dx2 and dI/dB1 = -2 s^2 LP w1 (w1 + w2 cos).
    The loss gradient is sum_r c_r dI_r with c_r the Gaussian-weighted upstream gradient at 2theta_r."""
    rng = np.random.default_rng(21)
    coef = synth.coef_table(rng)
    grid = synth.Grid()
    o = synth.Opts(synth.CU_KA, 5.0, 90.0, 1e-5, 0.0, 0)
    g = rng.standard_normal(grid.n_pts)
    lat = np.array([4.3, 5.1, 6.7, 84.0, 97.0, 109.0])

    # one atom off the origin
    x, Z, occ, B = np.array([0.21, 0.37, 0.63]), 26, 0.8, 0.7
    one = synth.Batch(lat[None], np.array([0, 1], np.int64), x[None].copy(), np.array([Z], np.int16),
                      np.array([occ]), np.array([B]), coef)
    hkl, _ = oracle.enumerate_refl(lat, o)
    df, dB, _ = oracle.broadened_grad(one, 0, hkl, o.wavelength, grid, g)
    want_B = 0.0
    for (s2, lp, c) in _weights(hkl, lat, o.wavelength, grid, g):
        w = occ * oracle.fatom(coef, Z, s2) * math.exp(-B * s2)
        want_B += c * (-2 * s2) * w * w * lp
    assert dB[0] == pytest.approx(want_B, rel=1e-10)
    assert np.abs(df).max() < 1e-9 * abs(want_B)

    # two atoms of different elements, occupancies and B factors
    x = np.array([[0.11, 0.52, 0.33], [0.71, 0.08, 0.91]])
    Zs, occs, Bs = (8, 29), (1.0, 0.6), (0.4, 1.1)
    two = synth.Batch(lat[None], np.array([0, 2], np.int64), x.copy(), np.array(Zs, np.int16),
                      np.array(occs), np.array(Bs), coef)
    df, dB, _ = oracle.broadened_grad(two, 0, hkl, o.wavelength, grid, g)
    want_x1 = np.zeros(3)
    want_B = np.zeros(2)
    for (h, k, l), (s2, lp, c) in zip(hkl, _weights(hkl, lat, o.wavelength, grid, g)):
        w1 = occs[0] * oracle.fatom(coef, Zs[0], s2) * math.exp(-Bs[0] * s2)
        w2 = occs[1] * oracle.fatom(coef, Zs[1], s2) * math.exp(-Bs[1] * s2)
        arg = 2 * math.pi * float(np.dot((h, k, l), x[0] - x[1]))
        want_x1 += c * (-4 * math.pi * lp * w1 * w2 * math.sin(arg)) * np.array((h, k, l), float)
        want_B[0] += c * (-2 * s2) * lp * w1 * (w1 + w2 * math.cos(arg))
        want_B[1] += c * (-2 * s2) * lp * w2 * (w2 + w1 * math.cos(arg))
    assert _rel(df[0], want_x1) < 1e-10
    assert _rel(df[1], -want_x1) < 1e-10
    assert _rel(dB, want_B) < 1e-10

"""The seeded synthetic workloads follow their stated recipes (host only).

Each generator is checked for determinism (same seed, same bytes), the C ABI
layout (dtypes, shapes, CSR offsets) and the distributions it promises:
ranges of edges, angles, atom counts, Z, B and occupancies, the volume-factor
rejection of near-degenerate cells, the lognormal medians of the mixed batch,
the hexagonal/P1 alternation and shared sites of the hexdis batch, and the
ranges of the augmentation effects.
"""
import numpy as np
import pytest

from paper_2602_11709_gb300 import synth


def _volume_factor(lat):
    c = np.cos(np.radians(lat[:, 3:]))
    return 1 - (c ** 2).sum(axis=1) + 2 * c.prod(axis=1)


def _check_layout(b):
    n, N = b.n_struct, b.n_atoms
    assert b.lattice.dtype == np.float64 and b.lattice.shape == (n, 6)
    assert b.atom_off.dtype == np.int64 and b.atom_off.shape == (n + 1,)
    assert b.atom_off[0] == 0 and b.atom_off[-1] == N and np.all(np.diff(b.atom_off) >= 0)
    assert b.frac.dtype == np.float64 and b.frac.shape == (N, 3)
    assert b.Z.dtype == np.int16 and b.Z.shape == (N,)
    assert b.occ.dtype == np.float64 and b.occ.shape == (N,)
    assert b.B.dtype == np.float64 and b.B.shape == (N,)
    assert b.coef.shape == (b.zmax + 1, 4, 2)
    assert np.all(b.coef[0] == 0)  # row 0 unused (no element Z = 0)
    assert np.all((b.coef[1:, :, 0] >= 0.5) & (b.coef[1:, :, 0] <= 4.0))
    assert np.all((b.coef[1:, :, 1] >= 0.5) & (b.coef[1:, :, 1] <= 50.0))
    assert np.all((b.frac >= 0) & (b.frac < 1))
    assert np.all((b.Z >= 1) & (b.Z <= b.zmax))


def _same(b1, b2):
    for f in ("lattice", "atom_off", "frac", "Z", "occ", "B", "coef"):
        assert np.array_equal(getattr(b1, f), getattr(b2, f)), f


@pytest.mark.parametrize("name", ["nacl", "small", "large", "mixed", "hexdis"])
def test_deterministic_and_abi_layout(name):
    gen = getattr(synth, name)
    b1, o1 = gen()
    b2, o2 = gen()
    _same(b1, b2)
    assert o1 == o2
    _check_layout(b1)


def test_small_recipe():
    b, o = synth.small()
    assert b.n_struct == 1024
    assert np.all((b.lattice[:, :3] >= 3) & (b.lattice[:, :3] <= 15))
    assert np.all((b.lattice[:, 3:] >= 60) & (b.lattice[:, 3:] <= 120))
    assert np.all(_volume_factor(b.lattice) >= 0.1)
    n = np.diff(b.atom_off)
    assert n.min() >= 1 and n.max() <= 64 and n.min() <= 2 and n.max() >= 63
    assert np.all((b.B >= 0) & (b.B <= 2)) and np.all(b.occ == 1)
    assert (o.wavelength, o.tt_min, o.tt_max, o.rel_cutoff, o.scaled) == (synth.CU_KA, 0.0, 90.0, 1e-3, 1)
    assert not np.array_equal(synth.small(seed=3)[0].lattice, b.lattice)


def test_large_recipe():
    b, o = synth.large()
    assert b.n_struct == 256
    assert np.all((b.lattice[:, :3] >= 15) & (b.lattice[:, :3] <= 40))
    n = np.diff(b.atom_off)
    assert n.min() >= 200 and n.max() <= 2000
    assert np.all((b.B >= 0) & (b.B <= 3))
    part = b.occ < 1
    assert abs(part.mean() - 0.2) < 0.01  # Bernoulli(0.2) over ~2.9e5 sites
    assert np.all((b.occ[part] >= 0.5) & (b.occ[part] < 1))
    assert (o.tt_min, o.tt_max) == (5.0, 120.0)


def test_mixed_recipe():
    b, o = synth.mixed()
    assert b.n_struct == 100_000
    n = np.diff(b.atom_off)
    assert n.min() >= 1 and n.max() <= 500
    assert abs(np.median(n) - 20) <= 1  # lognormal, median 20
    # sigma 1 in log space: the quartiles sit at 20 exp(-+0.674)
    q1, q3 = np.percentile(n, [25, 75])
    assert abs(q1 - 20 * np.exp(-0.6745)) <= 1 and abs(q3 - 20 * np.exp(0.6745)) <= 1.5
    e = b.lattice[:, :3]
    assert e.min() >= 3 and e.max() <= 30
    assert abs(np.median(e) - 7.0) < 0.1  # lognormal, median 7 A
    assert np.all(_volume_factor(b.lattice) >= 0.1)


def test_nacl_recipe():
    b, o = synth.nacl()
    assert b.n_struct == 1 and b.n_atoms == 8
    assert np.array_equal(b.lattice[0], [5.64, 5.64, 5.64, 90, 90, 90])
    na, cl = b.frac[b.Z == 11], b.frac[b.Z == 17]
    assert len(na) == 4 and len(cl) == 4
    # Cl = Na + (1/2, 0, 0) modulo 1, site by site
    assert np.allclose((na + [0.5, 0, 0]) % 1.0, cl)
    assert np.all(b.B == 0.5) and np.all(b.occ == 1)


def test_hexdis_recipe():
    b, o = synth.hexdis()
    lat = b.lattice
    even, odd = lat[0::2], lat[1::2]
    assert np.all(even[:, 0] == even[:, 1]) and np.all(even[:, 3:] == [90, 90, 120])
    assert np.all((even[:, 0] >= 2.5) & (even[:, 0] <= 6)) and np.all((even[:, 2] >= 3) & (even[:, 2] <= 12))
    assert np.all((odd[:, :3] >= 3) & (odd[:, :3] <= 10)) and np.all(_volume_factor(odd) >= 0.1)
    shared = 0
    sites = 0
    for s in range(b.n_struct):
        sl = b.atoms_of(s)
        x, occ = b.frac[sl], b.occ[sl]
        # records at one coordinate form a site; its occupancies sum to 1
        _, inv = np.unique(x, axis=0, return_inverse=True)
        inv = inv.reshape(-1)
        tot = np.bincount(inv, weights=occ)
        k = np.bincount(inv)
        assert np.allclose(tot, 1.0)
        assert k.max() <= 3 and 2 <= len(k) <= 24
        shared += int((k > 1).sum())
        sites += len(k)
    assert abs(shared / sites - 1 / 3) < 0.05
    assert np.all((b.B >= 0) & (b.B <= 1.5))
    assert (o.tt_min, o.tt_max, o.rel_cutoff, o.scaled) == (5.0, 110.0, 1e-3, 1)


def test_grad_recipe():
    base, target, o, grid = synth.grad(n=64)
    n = np.diff(base.atom_off)
    assert n.min() >= 8 and n.max() <= 128
    assert np.array_equal(base.atom_off, target.atom_off) and np.array_equal(base.Z, target.Z)
    d = (target.frac - base.frac + 0.5) % 1.0 - 0.5  # wrapped displacement
    assert abs(d.std() - 0.01) < 0.001
    assert np.all(np.abs(target.lattice[:, :3] / base.lattice[:, :3] - 1) <= 0.005)
    assert np.all(np.abs(target.lattice[:, 3:] - base.lattice[:, 3:]) <= 0.2)
    assert np.all(target.B >= 0) and np.all(np.abs(target.B - base.B) <= 0.1 + 1e-12)
    assert (grid.t0, grid.n_pts, grid.fwhm) == (5.0, 4096, 0.1)
    assert grid.t0 + (grid.n_pts - 1) * grid.dt == pytest.approx(90.0, abs=1e-12)
    assert (o.rel_cutoff, o.scaled) == (0.0, 0)


def test_augment_recipe():
    a = synth.augment(2000, 64)
    assert np.all((a.fwhm >= 0.05) & (a.fwhm <= 0.3)) and np.all((a.eta >= 0) & (a.eta <= 1))
    assert np.all((a.po_r >= 0.6) & (a.po_r <= 1.4)) and np.all((a.noise_sigma >= 0) & (a.noise_sigma <= 1))
    assert a.po_dir.shape == (2000, 3) and np.all(a.po_dir == np.rint(a.po_dir))
    assert np.all(np.abs(a.po_dir) <= 2) and np.all(np.abs(a.po_dir).sum(axis=1) > 0)
    assert a.z.dtype == np.float32 and a.z.shape == (2000, 64)
    assert abs(float(a.z.mean())) < 0.01 and abs(float(a.z.std()) - 1) < 0.01
    b = synth.augment(2000, 64)
    assert np.array_equal(a.z, b.z) and np.array_equal(a.po_dir, b.po_dir)


def test_subset_and_concat_round_trip():
    b, _ = synth.small(n=40)
    idx = np.array([5, 0, 39, 17])
    sub = b.subset(idx)
    _check_layout(sub)
    for i, s in enumerate(idx):
        assert np.array_equal(sub.frac[sub.atoms_of(i)], b.frac[b.atoms_of(s)])
        assert np.array_equal(sub.lattice[i], b.lattice[s])
    whole = synth.concat([b.subset(np.arange(0, 13)), b.subset(np.arange(13, 40))])
    _same(whole, b)
    empty = b.subset(np.zeros(0, np.int64))
    assert empty.n_struct == 0 and empty.n_atoms == 0 and np.array_equal(empty.atom_off, [0])

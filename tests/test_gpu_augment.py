"""Augmented pattern (pseudo-Voigt, March-Dollase, noise) on the GPU against the FP64 oracle.

Bar: every grid point within 1e-5 of the structure's largest oracle value
(FP32 structure factors and FP32 sums over every (point, reflection) pair;
the Gaussian component is skipped on the GPU only below 2^-40 of its peak).
Repeated calls give identical bytes (fixed summation order).
"""
import numpy as np
import pytest

import oracle
from paper_2602_11709_gb300 import synth

pytestmark = pytest.mark.gpu

TOL = 1e-5


@pytest.fixture(scope="module")
def handle(gpu_lib):
    h = gpu_lib.Handle(0)
    yield h
    h.close()


def _run(xrd, handle, b, o, grid, aug, po=True, noise=True, shape=None):
    import torch
    cuda = lambda x: torch.from_numpy(np.ascontiguousarray(x)).cuda()  # noqa: E731
    db = xrd.DeviceBatch.from_host(b)
    co = xrd.make_opts(o, "fp32_phasefix")
    cg = xrd.make_grid(grid)
    sz = handle.query_sizes(db, co)
    ws = xrd.workspace(sz.ws_grad_bytes)
    y = torch.full((b.n_struct, grid.n_pts), np.nan, dtype=torch.float32, device="cuda")
    status = torch.zeros(b.n_struct, dtype=torch.int32, device="cuda")
    totals = torch.zeros(4, dtype=torch.int64, device="cuda")
    if shape is not None:
        handle.set_sf_shape(*shape)
    try:
        handle.pattern_augmented(db, co, cg, cuda(aug.fwhm), cuda(aug.eta), y, status, totals, ws,
                                 po_dir=cuda(aug.po_dir) if po else None, po_r=cuda(aug.po_r) if po else None,
                                 noise_z=cuda(aug.z) if noise else None,
                                 noise_sigma=cuda(aug.noise_sigma) if noise else None)
        torch.cuda.synchronize()
    finally:
        if shape is not None:
            handle.set_sf_shape(128, 2, 0)  # the handle default
    return y.cpu().numpy(), status.cpu().numpy(), totals.cpu().numpy()


def _ref(b, s, o, grid, aug, po=True, noise=True):
    hkl, _ = oracle.enumerate_refl(b.lattice[s], o)
    return oracle.augmented(b, s, hkl, o.wavelength, grid.t0, grid.dt, grid.n_pts, aug.fwhm[s], aug.eta[s],
                            aug.po_dir[s] if po else (0.0, 0.0, 1.0), aug.po_r[s] if po else 1.0,
                            z=aug.z[s].astype(np.float64) if noise else None,
                            sigma=aug.noise_sigma[s] if noise else 0.0)


def _check(got, ref, s):
    err = np.abs(got.astype(np.float64) - ref).max()
    assert err <= TOL * np.abs(ref).max(), (s, err / np.abs(ref).max())


@pytest.mark.parametrize("po,noise", [(True, True), (False, False), (True, False)])
def test_augmented_matches_oracle(gpu_lib, handle, po, noise):
    base, _, o, grid = synth.grad()
    b = base.subset(np.array([0, 1, 2, 3, 4, 5, 6, 7]))
    aug = synth.augment(b.n_struct, grid.n_pts)
    aug.eta[0], aug.eta[1] = 0.0, 1.0  # pure Gaussian, pure Lorentzian
    aug.fwhm[2] = 0.6 * grid.dt        # undersampled peaks: 2 dt / fwhm > 1
    y, status, totals = _run(gpu_lib, handle, b, o, grid, aug, po, noise)
    assert np.all(status == 0) and totals[3] == 0
    for s in range(b.n_struct):
        _check(y[s], _ref(b, s, o, grid, aug, po, noise), s)


def test_ragged_grid_and_offset_range(gpu_lib, handle):
    """A grid that is not a multiple of the 1024-point CTA span, starting below
    the 2-theta range and ending inside it (peaks beyond the grid still add tails)."""
    base, _, o, _ = synth.grad()
    b = base.subset(np.array([9, 10, 11]))
    grid = synth.Grid(t0=-3.0, dt=0.037, n_pts=2001)
    aug = synth.augment(b.n_struct, grid.n_pts, seed=8)
    y, status, _ = _run(gpu_lib, handle, b, o, grid, aug)
    assert np.all(status == 0)
    for s in range(b.n_struct):
        _check(y[s], _ref(b, s, o, grid, aug), s)


def test_runs_shape_gives_the_same_pattern(gpu_lib, handle):
    base, _, o, grid = synth.grad()
    b = base.subset(np.arange(12, 20))
    aug = synth.augment(b.n_struct, grid.n_pts, seed=9)
    y0, _, _ = _run(gpu_lib, handle, b, o, grid, aug, shape=(128, 2, 0))
    y1, _, _ = _run(gpu_lib, handle, b, o, grid, aug, shape=(128, 2, 1))
    for s in range(b.n_struct):
        assert np.abs(y1[s] - y0[s]).max() <= TOL * np.abs(y0[s]).max(), s
    _check(y1[3], _ref(b, 3, o, grid, aug), 3)


def test_invalid_parameters_flag_only_their_structure(gpu_lib, handle):
    base, _, o, grid = synth.grad()
    b = base.subset(np.arange(8))
    aug = synth.augment(b.n_struct, grid.n_pts, seed=10)
    aug.fwhm[1] = 0.0
    aug.eta[2] = 1.5
    aug.po_r[3] = 0.0
    aug.noise_sigma[4] = -1.0
    aug.po_dir[5] = 0.0
    aug.fwhm[6] = np.nan
    y, status, totals = _run(gpu_lib, handle, b, o, grid, aug)
    bad = [1, 2, 3, 4, 5, 6]
    assert list(np.nonzero(status)[0]) == bad and np.all(status[bad] == gpu_lib.XRD_EINVAL)
    assert totals[3] == len(bad)
    assert np.all(y[bad] == 0.0)
    for s in (0, 7):
        _check(y[s], _ref(b, s, o, grid, aug), s)


def test_structure_without_reflections_and_empty_batch(gpu_lib, handle):
    import torch
    rng = np.random.default_rng(21)
    tiny = synth.random_cell(rng, 2, edge=(2.0, 2.2))  # no reflection below 2theta = 20 deg
    o = synth.Opts(synth.CU_KA, 0.0, 20.0, 1e-5, 0.0, 0)
    grid = synth.Grid(t0=0.0, dt=0.01, n_pts=1500)
    aug = synth.augment(1, grid.n_pts)
    assert len(oracle.enumerate_refl(tiny.lattice[0], o)[0]) == 0
    y, status, _ = _run(gpu_lib, handle, tiny, o, grid, aug)
    assert status[0] == 0 and np.all(y == 0.0)
    empty = tiny.subset(np.array([], dtype=np.int64))
    db = gpu_lib.DeviceBatch.from_host(empty)
    co = gpu_lib.make_opts(o, "fp32_phasefix")
    ws = gpu_lib.workspace(handle.query_sizes(db, co).ws_grad_bytes)
    z = torch.zeros(0, dtype=torch.float64, device="cuda")
    totals = torch.zeros(4, dtype=torch.int64, device="cuda")
    yy = torch.zeros((0, grid.n_pts), dtype=torch.float32, device="cuda")
    st = torch.zeros(0, dtype=torch.int32, device="cuda")
    handle.pattern_augmented(db, co, gpu_lib.make_grid(grid), z, z, yy, st, totals, ws)
    torch.cuda.synchronize()
    assert totals.cpu().numpy()[3] == 0


def test_host_side_argument_checks(gpu_lib, handle):
    import torch
    base, _, o, grid = synth.grad()
    b = base.subset(np.arange(2))
    aug = synth.augment(b.n_struct, grid.n_pts)
    db = gpu_lib.DeviceBatch.from_host(b)
    co = gpu_lib.make_opts(o, "fp32_phasefix")
    ws = gpu_lib.workspace(handle.query_sizes(db, co).ws_grad_bytes)
    cuda = lambda x: torch.from_numpy(np.ascontiguousarray(x)).cuda()  # noqa: E731
    y = torch.zeros((b.n_struct, grid.n_pts), dtype=torch.float32, device="cuda")
    st = torch.zeros(b.n_struct, dtype=torch.int32, device="cuda")
    tot = torch.zeros(4, dtype=torch.int64, device="cuda")
    f, e = cuda(aug.fwhm), cuda(aug.eta)
    with pytest.raises(gpu_lib.XrdError):  # po_dir without po_r
        handle.pattern_augmented(db, co, gpu_lib.make_grid(grid), f, e, y, st, tot, ws, po_dir=cuda(aug.po_dir))
    with pytest.raises(gpu_lib.XrdError):  # noise draws without a scale
        handle.pattern_augmented(db, co, gpu_lib.make_grid(grid), f, e, y, st, tot, ws, noise_z=cuda(aug.z))
    with pytest.raises(gpu_lib.XrdError):  # grid too far from the 2-theta range
        handle.pattern_augmented(db, co, gpu_lib.make_grid(synth.Grid(t0=0.0, dt=1e-6, n_pts=100)), f, e, y, st,
                                 tot, ws)
    with pytest.raises(gpu_lib.XrdError):  # pattern precision other than the integer phase
        handle.pattern_augmented(db, gpu_lib.make_opts(o, "fp64"), gpu_lib.make_grid(grid), f, e, y, st, tot, ws)


def test_small_workload_sampled_structures(gpu_lib, handle):
    """The benchmark's 1024-structure batch in one call; sampled structures against the oracle."""
    b, o = synth.small()
    grid = synth.Grid(t0=0.0, dt=90.0 / 4095.0, n_pts=4096)
    aug = synth.augment(b.n_struct, grid.n_pts, seed=7)
    y, status, totals = _run(gpu_lib, handle, b, o, grid, aug)
    assert np.all(status == 0) and totals[3] == 0
    assert np.all(np.isfinite(y))
    for s in (0, 17, 511, 1023):
        _check(y[s], _ref(b, s, o, grid, aug), s)


def test_repeated_calls_are_bitwise_identical(gpu_lib, handle):
    base, _, o, grid = synth.grad()
    b = base.subset(np.arange(20, 28))
    aug = synth.augment(b.n_struct, grid.n_pts, seed=12)
    y0, _, _ = _run(gpu_lib, handle, b, o, grid, aug)
    y1, _, _ = _run(gpu_lib, handle, b, o, grid, aug)
    assert np.array_equal(y0.view(np.uint32), y1.view(np.uint32))


def test_profiling_times_the_profile_sum(gpu_lib, handle):
    base, _, o, grid = synth.grad()
    b = base.subset(np.arange(4))
    aug = synth.augment(b.n_struct, grid.n_pts)
    handle.set_profiling(2)
    try:
        _run(gpu_lib, handle, b, o, grid, aug)
        st = handle.stage_times()
    finally:
        handle.set_profiling(0)
    assert st["profile_sum"] > 0.0 and all(v == 0.0 for k, v in st.items() if k != "profile_sum")


def test_large_batch_takes_the_multi_block_scans(gpu_lib, handle):
    """9000 structures (three 4096-structure scan chunks): the augmented path's front runs the
    multi-block reflection scan; sampled structures against the oracle."""
    b, o = synth.small(n=9000)
    grid = synth.Grid(t0=0.0, dt=90.0 / 1023.0, n_pts=1024)
    aug = synth.augment(b.n_struct, grid.n_pts, seed=13)
    y, status, totals = _run(gpu_lib, handle, b, o, grid, aug)
    assert np.all(status == 0) and totals[3] == 0 and np.all(np.isfinite(y))
    for s in (0, 4095, 4096, 8191, 8999):
        _check(y[s], _ref(b, s, o, grid, aug), s)

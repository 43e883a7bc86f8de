"""Broadened pattern and its gradient on the GPU against the FP64 oracle.

Bar: broadened profile within 1e-5 of the structure's largest value; gradients
(coordinates, B factors, lattice parameters, each group separately) within
1e-3 relative in norm of the FP64 oracle gradient and with cosine similarity
>= 0.99999 (FP32 arithmetic; the oracle sums every Gaussian over the whole
grid, the GPU cuts each one at about 6 sigma, a 2e-8 effect).
"""
import numpy as np
import pytest

import oracle
from paper_2602_11709_gb300 import synth

pytestmark = pytest.mark.gpu


def _grad_case(n=None, idx=None):
    base, target, o, grid = synth.grad()
    if idx is not None:
        base = base.subset(idx)
        target = target.subset(idx)
    return base, target, o, grid


def _run(xrd, handle, b, o, grid, dLdy=None):
    import torch
    db = xrd.DeviceBatch.from_host(b)
    co = xrd.make_opts(o, "fp32_phasefix")
    cg = xrd.make_grid(grid)
    sz = handle.query_sizes(db, co)
    ws = xrd.workspace(sz.ws_grad_bytes)
    y = torch.empty(b.n_struct, grid.n_pts, dtype=torch.float32, device="cuda")
    status = torch.zeros(b.n_struct, dtype=torch.int32, device="cuda")
    totals = torch.zeros(4, dtype=torch.int64, device="cuda")
    handle.pattern_broadened(db, co, cg, y, status, totals, ws)
    out = {"y": y, "status": status, "totals": totals}
    if dLdy is not None:
        g = torch.from_numpy(np.ascontiguousarray(dLdy, dtype=np.float32)).cuda()
        d_frac = torch.full((b.n_atoms, 3), np.nan, dtype=torch.float32, device="cuda")
        d_B = torch.full((b.n_atoms,), np.nan, dtype=torch.float32, device="cuda")
        d_lat = torch.full((b.n_struct, 6), np.nan, dtype=torch.float32, device="cuda")
        handle.pattern_grad(db, co, cg, g, d_frac, d_B, d_lat, ws)
        out.update(d_frac=d_frac, d_B=d_B, d_lat=d_lat)
    torch.cuda.synchronize()
    return {k: v.cpu().numpy() for k, v in out.items()}


def _cmp(a, b):
    a, b = np.asarray(a, np.float64).ravel(), np.asarray(b, np.float64).ravel()
    rel = np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)
    cos = float(np.dot(a, b) / max(np.linalg.norm(a) * np.linalg.norm(b), 1e-300))
    return rel, cos


@pytest.fixture(scope="module")
def handle(gpu_lib):
    h = gpu_lib.Handle(0)
    yield h
    h.close()


def test_broadened_matches_oracle(gpu_lib, handle):
    idx = np.array([0, 1, 2, 3, 4, 5])
    b, _, o, grid = _grad_case(idx=idx)
    got = _run(gpu_lib, handle, b, o, grid)
    assert np.all(got["status"] == 0)
    for s in range(b.n_struct):
        hkl, _ = oracle.enumerate_refl(b.lattice[s], o)
        ref = oracle.broadened(b, s, hkl, o.wavelength, grid)
        assert np.abs(got["y"][s] - ref).max() <= 1e-5 * ref.max(), s


def test_gradient_matches_oracle(gpu_lib, handle):
    idx = np.array([7, 11, 19, 23, 42])
    b, _, o, grid = _grad_case(idx=idx)
    rng = np.random.default_rng(99)
    g = rng.standard_normal((b.n_struct, grid.n_pts))
    got = _run(gpu_lib, handle, b, o, grid, dLdy=g)
    worst = {}
    for s in range(b.n_struct):
        hkl, _ = oracle.enumerate_refl(b.lattice[s], o)
        df, dB, dl = oracle.broadened_grad(b, s, hkl, o.wavelength, grid, g[s].astype(np.float32).astype(np.float64))
        sl = b.atoms_of(s)
        for name, gv, rv in (("frac", got["d_frac"][sl], df), ("B", got["d_B"][sl], dB), ("lattice", got["d_lat"][s], dl)):
            rel, cos = _cmp(gv, rv)
            worst[name] = max(worst.get(name, 0.0), rel)
            assert rel <= 1e-3 and cos >= 0.99999, (s, name, rel, cos)


def test_autograd_function_mse_loss(gpu_lib, handle):
    import torch
    from paper_2602_11709_gb300 import autograd as ag
    idx = np.array([3, 8, 13])
    b, t, o, grid = _grad_case(idx=idx)
    fixed = ag.FixedBatch.from_host(b)
    frac = torch.tensor(b.frac, device="cuda", requires_grad=True)
    B = torch.tensor(b.B, device="cuda", requires_grad=True)
    lat = torch.tensor(b.lattice, device="cuda", requires_grad=True)
    with torch.no_grad():
        ft = ag.FixedBatch.from_host(t)
        yt = ag.broadened_pattern(torch.tensor(t.frac, device="cuda"), torch.tensor(t.B, device="cuda"),
                                  torch.tensor(t.lattice, device="cuda"), ft, o, grid, handle)
    scale = yt.amax(dim=1, keepdim=True)
    y = ag.broadened_pattern(frac, B, lat, fixed, o, grid, handle)
    y.retain_grad()
    loss = (((y - yt) / scale) ** 2).mean()
    loss.backward()
    gy = y.grad.detach().cpu().numpy().astype(np.float64)
    assert frac.grad is not None and B.grad is not None and lat.grad is not None
    for s in range(b.n_struct):
        hkl, _ = oracle.enumerate_refl(b.lattice[s], o)
        df, dB, dl = oracle.broadened_grad(b, s, hkl, o.wavelength, grid, gy[s])
        sl = b.atoms_of(s)
        for gv, rv in ((frac.grad[sl].cpu().numpy(), df), (B.grad[sl].cpu().numpy(), dB),
                       (lat.grad[s].cpu().numpy(), dl)):
            rel, cos = _cmp(gv, rv)
            assert rel <= 1e-3 and cos >= 0.99999, (s, rel, cos)


def test_full_gradient_workload(gpu_lib, handle):
    """All 512 structures of the gradient workload in one launch; sampled structures
    checked against the oracle gradient, the rest against invariants."""
    b, _, o, grid = _grad_case()
    rng = np.random.default_rng(5)
    g = rng.standard_normal((b.n_struct, grid.n_pts))
    got = _run(gpu_lib, handle, b, o, grid, dLdy=g)
    assert np.all(got["status"] == 0)
    assert np.all(np.isfinite(got["y"])) and np.all(np.isfinite(got["d_frac"]))
    assert np.all(np.isfinite(got["d_B"])) and np.all(np.isfinite(got["d_lat"]))
    # translation invariance of every structure: sum_j dL/dx_j = 0
    for s in range(b.n_struct):
        d = got["d_frac"][b.atoms_of(s)].astype(np.float64)
        assert np.abs(d.sum(axis=0)).max() <= 1e-3 * max(np.abs(d).max(), 1e-30) * np.sqrt(len(d))
    for s in rng.choice(b.n_struct, size=3, replace=False):
        hkl, _ = oracle.enumerate_refl(b.lattice[s], o)
        df, dB, dl = oracle.broadened_grad(b, s, hkl, o.wavelength, grid, g[s].astype(np.float32).astype(np.float64))
        sl = b.atoms_of(s)
        for gv, rv in ((got["d_frac"][sl], df), (got["d_B"][sl], dB), (got["d_lat"][s], dl)):
            rel, cos = _cmp(gv, rv)
            assert rel <= 1e-3 and cos >= 0.99999, (s, rel, cos)


def test_bad_structures_get_zero_gradients(gpu_lib, handle):
    b, _, o, grid = _grad_case(idx=np.array([0, 1]))
    b.lattice[1] = [5.0, 5.0, 5.0, 60.0, 60.0, 120.0]  # degenerate cell
    g = np.ones((2, grid.n_pts))
    got = _run(gpu_lib, handle, b, o, grid, dLdy=g)
    assert list(got["status"]) == [0, 1]
    assert np.all(got["y"][1] == 0.0)
    sl = b.atoms_of(1)
    assert np.all(got["d_frac"][sl] == 0.0) and np.all(got["d_B"][sl] == 0.0) and np.all(got["d_lat"][1] == 0.0)
    assert np.all(np.isfinite(got["d_frac"][b.atoms_of(0)]))


def test_gradient_back_scattering(gpu_lib, handle):
    """Reflections between 100 and 179.5 degrees, where the Lorentz factor and d(2theta)/d|g|^2 grow
    as 1 / cos(theta) and cos^2(theta) = 1 - sin^2(theta) loses digits in FP32."""
    idx = np.array([7, 11, 19])
    b, _, o, _ = _grad_case(idx=idx)
    o = synth.Opts(o.wavelength, 100.0, 179.5, o.tt_tol, 0.0, 0)
    grid = synth.Grid(t0=100.0, dt=79.5 / 4095.0, n_pts=4096, fwhm=0.1)
    rng = np.random.default_rng(17)
    g = rng.standard_normal((b.n_struct, grid.n_pts))
    got = _run(gpu_lib, handle, b, o, grid, dLdy=g)
    assert np.all(got["status"] == 0)
    for s in range(b.n_struct):
        hkl, _ = oracle.enumerate_refl(b.lattice[s], o)
        ref = oracle.broadened(b, s, hkl, o.wavelength, grid)
        assert np.abs(got["y"][s] - ref).max() <= 1e-5 * ref.max(), s
        df, dB, dl = oracle.broadened_grad(b, s, hkl, o.wavelength, grid, g[s].astype(np.float32).astype(np.float64))
        sl = b.atoms_of(s)
        for name, gv, rv in (("frac", got["d_frac"][sl], df), ("B", got["d_B"][sl], dB), ("lattice", got["d_lat"][s], dl)):
            rel, cos = _cmp(gv, rv)
            assert rel <= 1e-3 and cos >= 0.99999, (s, name, rel, cos)


def test_gradient_against_finite_differences_of_the_gpu_forward(gpu_lib, handle):
    """GPU gradients against 5-point central differences of the GPU's own broadened pattern, for
    L = sum_k w_k y_k with fixed random w: coordinates and B of four atoms and the six lattice
    parameters of three structures. The broadened path computes in FP32 (its y rounds at about
    1e-7), so the steps are 1e-3 in fractional coordinates, 5e-2 A^2 in B (one atom's B moves L by
    about 2 s^2 / N of itself), 1e-4 relative in the edges and 1e-3 deg in the angles: truncation
    error (step^4) and rounding (1e-7 / step) both stay well below the bar. A lattice step that moves a reflection across a sphere surface
    changes the reflection set (a jump, not a derivative): such parameters are skipped, and at
    least four of the six must remain."""
    import torch
    xrd = gpu_lib
    base, _, o, grid = _grad_case(idx=np.array([7, 11, 19]))
    rng = np.random.default_rng(41)
    w = rng.standard_normal(grid.n_pts)

    def forward(b):
        db = xrd.DeviceBatch.from_host(b)
        co = xrd.make_opts(o, "fp32_phasefix")
        sz = handle.query_sizes(db, co)
        ws = xrd.workspace(sz.ws_grad_bytes)
        y = torch.empty(1, grid.n_pts, dtype=torch.float32, device="cuda")
        status = torch.zeros(1, dtype=torch.int32, device="cuda")
        totals = torch.zeros(4, dtype=torch.int64, device="cuda")
        handle.pattern_broadened(db, co, xrd.make_grid(grid), y, status, totals, ws)
        torch.cuda.synchronize()
        return float(np.dot(w, y.cpu().numpy()[0].astype(np.float64))), int(totals[0])

    def fd(b, setter, h):
        vals, counts = [], set()
        for k in (2, 1, -1, -2):
            bb = b.subset([0])
            setter(bb, k * h)
            L, n = forward(bb)
            vals.append(L)
            counts.add(n)
        return (-vals[0] + 8 * vals[1] - 8 * vals[2] + vals[3]) / (12 * h), len(counts) == 1

    checked_lat = 0
    for s in range(base.n_struct):
        b = base.subset([s])
        got = _run(xrd, handle, b, o, grid, dLdy=w[None, :])
        groups = {"frac": ([], []), "B": ([], []), "lattice": ([], [])}
        for j in range(min(4, b.n_atoms)):
            for c in range(3):
                def set_x(bb, d, j=j, c=c):
                    bb.frac[j, c] += d
                v, _ = fd(b, set_x, 1e-3)
                groups["frac"][0].append(got["d_frac"][j, c])
                groups["frac"][1].append(v)

            def set_b(bb, d, j=j):
                bb.B[j] += d
            v, _ = fd(b, set_b, 5e-2)  # one atom's share of L is small: a step well above the FP32 rounding
            groups["B"][0].append(got["d_B"][j])
            groups["B"][1].append(v)
        for p in range(6):
            h = 1e-4 * b.lattice[0, p] if p < 3 else 1e-3

            def set_l(bb, d, p=p):
                bb.lattice[0, p] += d
            v, same = fd(b, set_l, h)
            if same:
                groups["lattice"][0].append(got["d_lat"][0, p])
                groups["lattice"][1].append(v)
                checked_lat += 1
        # the bar of the oracle-gradient tests, per group, plus 2e-3 for the differences' own error
        for name, (gv, rv) in groups.items():
            if not gv:
                continue
            rel, cos = _cmp(gv, rv)
            assert rel <= 3e-3 and cos >= 0.99999, (s, name, rel, cos)
    assert checked_lat >= 4

"""Parity of the CUDA path (through the C ABI) with the FP64 CPU oracle."""
import json
import math
import os

import numpy as np
import pytest

import oracle
from paper_2602_11709_gb300 import synth

from parity import compare_batch, compare_reflections, families, half_space

pytestmark = pytest.mark.gpu

PRECS = ["fp64", "fp32_phase64", "fp32_phasefix"]
# one JSON line per case (peaks compared, largest errors) when XRD_PARITY_REPORT names a file
REPORT = os.environ.get("XRD_PARITY_REPORT", "")


def _report(name, stats):
    if not REPORT:
        return
    try:
        os.makedirs(os.path.dirname(os.path.abspath(REPORT)), exist_ok=True)
        with open(REPORT, "a") as f:
            f.write(json.dumps({"test": name, **{k: (float(v) if isinstance(v, (np.floating, float)) else v)
                                                  for k, v in stats.items()}}) + "\n")
    except OSError:
        pass


@pytest.fixture(scope="module")
def handle(gpu_lib):
    h = gpu_lib.Handle(0)
    yield h
    h.close()


def _opts(base, **kw):
    o = synth.Opts(base.wavelength, base.tt_min, base.tt_max, base.tt_tol, base.rel_cutoff, base.scaled)
    for k, v in kw.items():
        setattr(o, k, v)
    return o


@pytest.mark.parametrize("prec", PRECS)
def test_nacl(gpu_lib, handle, prec):
    b, o = synth.nacl()
    ref = oracle.pattern_batch(b, o, threads=1)
    got = gpu_lib.compute(b, o, prec, handle=handle)
    st = compare_batch(got, ref, prec, o.rel_cutoff, o.scaled)
    assert st["boundary"] == 0 and st["pairs"] == 9
    assert got["sizes"]["n_refl"] == 293  # 586 reflections, one per Friedel pair
    assert [families(got, 0, p) for p in range(9)][1] == [((2, 0, 0), 6)]
    _report("nacl_" + prec, st)


@pytest.mark.parametrize("prec", PRECS)
def test_small_batch_full_size(gpu_lib, handle, prec):
    """All 1024 structures of the small-cell workload (the benchmark's batch)."""
    b, o = synth.small()
    ref = oracle.pattern_batch(b, o, threads=0)
    got = gpu_lib.compute(b, o, prec, handle=handle)
    assert got["sizes"]["n_refl"] * 2 == int(ref["n_refl"].sum())
    st = compare_batch(got, ref, prec, o.rel_cutoff, o.scaled)
    _report("small_" + prec, st)


@pytest.mark.parametrize("prec", ["fp64", "fp32_phasefix"])
@pytest.mark.parametrize("variant", ["nocut_unscaled", "range_5_120", "wide_tol"])
def test_options(gpu_lib, handle, prec, variant):
    b, o = synth.small(n=96)
    if variant == "nocut_unscaled":
        o = _opts(o, rel_cutoff=0.0, scaled=0)
    elif variant == "range_5_120":
        o = _opts(o, tt_min=5.0, tt_max=120.0, wavelength=0.71073)
    else:
        o = _opts(o, tt_tol=0.05)
    ref = oracle.pattern_batch(b, o, threads=0)
    got = gpu_lib.compute(b, o, prec, handle=handle)
    st = compare_batch(got, ref, prec, o.rel_cutoff, o.scaled)
    _report("options_%s_%s" % (variant, prec), st)


@pytest.mark.parametrize("prec", PRECS)
def test_large_cells(gpu_lib, handle, prec):
    """Large cells (more reflections than one CTA keeps in shared memory)."""
    b, o = synth.large(n=256)
    counts = np.diff(b.atom_off)
    idx = np.argsort(counts)[:2]
    sub = b.subset(idx)
    ref = oracle.pattern_batch(sub, o, threads=0)
    got = gpu_lib.compute(sub, o, prec, handle=handle)
    assert got["sizes"]["max_refl"] > 2048
    st = compare_batch(got, ref, prec, o.rel_cutoff, o.scaled)
    _report("large_" + prec, st)


def test_mixed_sample(gpu_lib, handle):
    b, o = synth.mixed(n=100_000)
    sub = b.subset(np.arange(3000))
    ref = oracle.pattern_batch(sub, o, threads=0)
    got = gpu_lib.compute(sub, o, "fp32_phasefix", handle=handle)
    st = compare_batch(got, ref, "fp32_phasefix", o.rel_cutoff, o.scaled)
    _report("mixed3000_fp32_phasefix", st)


def test_determinism(gpu_lib, handle):
    b, o = synth.small(n=200)
    r1 = gpu_lib.compute(b, o, "fp32_phasefix", handle=handle)
    r2 = gpu_lib.compute(b, o, "fp32_phasefix", handle=handle)
    for key in ("peak_tt", "peak_I", "fam_hkl", "fam_mult"):
        for s in range(b.n_struct):
            assert np.array_equal(r1[key][s], r2[key][s])


def test_edge_cases(gpu_lib, handle):
    nacl, o = synth.nacl()
    rng = np.random.default_rng(77)
    empty_atoms = synth.Batch(nacl.lattice.copy(), np.array([0, 0], np.int64), np.zeros((0, 3)),
                              np.zeros(0, np.int16), np.zeros(0), np.zeros(0), nacl.coef)
    bad_cell = synth.Batch(np.array([[5.0, 5.0, 5.0, 60.0, 60.0, 120.0]]), nacl.atom_off.copy(), nacl.frac.copy(),
                           nacl.Z.copy(), nacl.occ.copy(), nacl.B.copy(), nacl.coef)
    bad_z = synth.Batch(nacl.lattice.copy(), nacl.atom_off.copy(), nacl.frac.copy(),
                        np.array([11, 11, 11, 11, 17, 17, 17, 99], np.int16), nacl.occ.copy(), nacl.B.copy(),
                        nacl.coef)
    nan_x = synth.Batch(nacl.lattice.copy(), nacl.atom_off.copy(), nacl.frac.copy(), nacl.Z.copy(), nacl.occ.copy(),
                        nacl.B.copy(), nacl.coef)
    nan_x.frac[3, 1] = np.nan
    neg_occ = synth.Batch(nacl.lattice.copy(), nacl.atom_off.copy(), nacl.frac.copy(), nacl.Z.copy(),
                          nacl.occ.copy(), nacl.B.copy(), nacl.coef)
    neg_occ.occ[2] = -0.5
    rand = synth.random_cell(rng, 5)
    rand.coef = nacl.coef
    batch = synth.concat([nacl, empty_atoms, bad_cell, bad_z, nan_x, neg_occ, rand])
    got = gpu_lib.compute(batch, o, "fp32_phasefix", handle=handle)
    st = list(got["status"])
    assert st == [0, 0, 1, 1, 1, 1, 0]
    assert got["totals"][3] == 4
    assert len(got["peak_tt"][0]) == 9
    assert len(got["peak_tt"][1]) == 0  # no atoms: every merged peak is 0 and cut off
    for s in (2, 3, 4, 5):
        assert len(got["peak_tt"][s]) == 0
    ref = oracle.pattern_batch(batch.subset([0, 6]), o)
    sub = {k: [v[0], v[6]] for k, v in got.items() if isinstance(v, list)}
    sub["status"] = [got["status"][0], got["status"][6]]
    compare_batch(sub, ref, "fp32_phasefix", o.rel_cutoff, o.scaled)
    # without a cutoff the atom-free structure keeps its zero peaks
    o0 = _opts(o, rel_cutoff=0.0)
    got0 = gpu_lib.compute(batch.subset([1]), o0, "fp32_phasefix", handle=handle)
    assert len(got0["peak_tt"][0]) == 23 and np.all(got0["peak_I"][0] == 0.0)
    # no reflection in range
    onone = _opts(o, tt_max=5.0)
    gotn = gpu_lib.compute(nacl, onone, "fp64", handle=handle)
    assert gotn["sizes"]["n_refl"] == 0 and len(gotn["peak_tt"][0]) == 0 and gotn["status"][0] == 0


def test_empty_batch(gpu_lib, handle):
    nacl, o = synth.nacl()
    b = nacl.subset(np.zeros(0, np.int64))
    got = gpu_lib.compute(b, o, "fp32_phasefix", handle=handle)
    assert got["totals"][0] == 0 and got["totals"][1] == 0 and len(got["peak_tt"]) == 0


def test_capacity_errors(gpu_lib, handle):
    import torch
    xrd = gpu_lib
    b, o = synth.small(n=16)
    db = xrd.DeviceBatch.from_host(b)
    co = xrd.make_opts(o, "fp32_phasefix")
    sz = handle.query_sizes(db, co)
    # workspace with room for only half of the reflections: the device flags every structure
    out = xrd.PatternBuffers(b.n_struct, sz.n_refl)
    small_ws = xrd.workspace(sz.ws_bytes - 40 * sz.n_refl)
    handle.pattern_batch(db, co, out, small_ws)
    torch.cuda.synchronize()
    assert np.all(out.status.cpu().numpy() == xrd.XRD_ECAPACITY)
    assert int(out.totals[3]) == b.n_struct
    # too small an output: flagged as well
    out2 = xrd.PatternBuffers(b.n_struct, 10)
    ws = xrd.workspace(sz.ws_bytes)
    handle.pattern_batch(db, co, out2, ws)
    torch.cuda.synchronize()
    assert np.all(out2.status.cpu().numpy() == xrd.XRD_ECAPACITY)
    # host-side argument errors
    with pytest.raises(xrd.XrdError) as e:
        handle.pattern_batch(db, xrd.make_opts(synth.Opts(wavelength=-1.0)), out, ws)
    assert e.value.code == xrd.XRD_EINVAL
    for tol in (0.0, 1e-10, -1e-5, float("nan")):  # below the smallest merge tolerance
        with pytest.raises(xrd.XrdError) as e:
            handle.pattern_batch(db, xrd.make_opts(synth.Opts(tt_tol=tol), "fp32_phasefix"), out, ws)
        assert e.value.code == xrd.XRD_EINVAL
    handle.pattern_batch(db, xrd.make_opts(synth.Opts(tt_tol=xrd.XRD_MIN_TT_TOL), "fp32_phasefix"), out, ws)
    with pytest.raises(xrd.XrdError) as e:
        handle.pattern_batch(db, co, out, xrd.workspace(64))
    assert e.value.code == xrd.XRD_ECAPACITY


@pytest.mark.parametrize("prec", ["fp32_phasefix", "fp64"])
def test_large_full_size_sampled(gpu_lib, handle, prec):
    """All 256 large cells in one launch; single-family peaks checked one by one
    against the oracle's structure factor, plus size invariants."""
    b, o = synth.large()
    if prec == "fp64":
        b = b.subset(np.arange(24))
    o = _opts(o, rel_cutoff=0.0, scaled=0)
    got = gpu_lib.compute(b, o, prec, handle=handle)
    assert np.all(got["status"] == 0)
    rng = np.random.default_rng(5)
    lam = o.wavelength
    worst = 0.0
    for s in rng.choice(b.n_struct, size=6, replace=False):
        tt, I, fo = got["peak_tt"][s], got["peak_I"][s], got["peak_fam_off"][s]
        assert np.all(np.diff(tt) > 0)
        hkl_full, _ = oracle.enumerate_refl(b.lattice[s], o)
        assert int(got["fam_mult"][s].sum()) == len(hkl_full)
        imax = I.max()
        _, Gs, _ = oracle.metric(b.lattice[s])
        picks = [p for p in rng.choice(len(tt), size=40, replace=False) if fo[p + 1] - fo[p] == 1
                 and got["fam_mult"][s][fo[p]] == 2]
        for p in picks[:15]:
            h, k, l = (int(x) for x in got["fam_hkl"][s][fo[p]])
            q = oracle.q_of(Gs, h, k, l)
            s2, ttr, lp, d = oracle.refl(q, lam)
            F = oracle.sf(b, s, h, k, l, s2)
            Iref = 2 * abs(F) ** 2 * lp
            assert abs(tt[p] - ttr) <= 1e-6
            worst = max(worst, abs(I[p] - Iref) / imax)
            assert abs(I[p] - Iref) <= (1e-5 if prec != "fp64" else 1e-9) * imax, (s, p, I[p], Iref)
    _report("large_full_sampled_" + prec, {"max_abs_rel_to_max": worst})


def test_mixed_full_size_sampled(gpu_lib, handle):
    """All 100 000 mixed cells in one launch sequence; sampled structures against the
    oracle, every structure against invariants."""
    b, o = synth.mixed()
    got = gpu_lib.compute(b, o, "fp32_phasefix", handle=handle)
    assert np.all(got["status"] == 0)
    assert got["totals"][3] == 0
    for s in range(b.n_struct):
        tt, I = got["peak_tt"][s], got["peak_I"][s]
        if len(tt):
            assert np.all(np.diff(tt) > 0) and I.max() == 100.0
    rng = np.random.default_rng(17)
    idx = rng.choice(b.n_struct, size=40, replace=False)
    # the largest structures too (longest per-structure paths)
    idx = np.concatenate([idx, np.argsort(np.diff(b.atom_off))[-5:]])
    sub = b.subset(idx)
    ref = oracle.pattern_batch(sub, o, threads=0)
    picked = {k: [v[s] for s in idx] for k, v in got.items() if isinstance(v, list)}
    picked["status"] = got["status"][idx]
    st = compare_batch(picked, ref, "fp32_phasefix", o.rel_cutoff, o.scaled)
    _report("mixed_full_sampled_fp32_phasefix", st)


def test_runs_shape_against_oracle(gpu_lib, handle):
    """Lanes taking runs consecutive in l (one exact phase seed per run and atom, the
    phase factor rotated along l): every peak of small and large cells against the
    oracle at the FP32 bar, and sampled peaks of the full large batch."""
    try:
        handle.set_sf_shape(128, 2, 1)
        b, o = synth.small()
        sub = b.subset(np.arange(0, 1024, 8))
        st = compare_batch(gpu_lib.compute(sub, o, "fp32_phasefix", handle=handle),
                           oracle.pattern_batch(sub, o, threads=0), "fp32_phasefix", o.rel_cutoff, o.scaled)
        _report("runs_small_fp32_phasefix", st)
        bl, ol = synth.large(n=256)
        idx = np.argsort(np.diff(bl.atom_off))[:2]
        subl = bl.subset(idx)
        st = compare_batch(gpu_lib.compute(subl, ol, "fp32_phasefix", handle=handle),
                           oracle.pattern_batch(subl, ol, threads=0), "fp32_phasefix", ol.rel_cutoff, ol.scaled)
        _report("runs_large_fp32_phasefix", st)
        o0 = _opts(ol, rel_cutoff=0.0, scaled=0)
        got = gpu_lib.compute(bl, o0, "fp32_phasefix", handle=handle)
        rng = np.random.default_rng(9)
        worst = 0.0
        for s in rng.choice(bl.n_struct, size=4, replace=False):
            tt, I, fo = got["peak_tt"][s], got["peak_I"][s], got["peak_fam_off"][s]
            imax = I.max()
            _, Gs, _ = oracle.metric(bl.lattice[s])
            picks = [p for p in rng.choice(len(tt), size=40, replace=False) if fo[p + 1] - fo[p] == 1
                     and got["fam_mult"][s][fo[p]] == 2]
            for p in picks[:12]:
                h, k, l = (int(x) for x in got["fam_hkl"][s][fo[p]])
                q = oracle.q_of(Gs, h, k, l)
                s2, ttr, lp, d = oracle.refl(q, o0.wavelength)
                Iref = 2 * abs(oracle.sf(bl, s, h, k, l, s2)) ** 2 * lp
                worst = max(worst, abs(I[p] - Iref) / imax)
                assert abs(I[p] - Iref) <= 1e-5 * imax, (s, p, I[p], Iref)
        _report("runs_large_full_sampled_fp32_phasefix", {"max_abs_rel_to_max": worst})
    finally:
        handle.set_sf_shape(128, 2, 0)


@pytest.mark.parametrize("n", [1, 7, 37, 1024])
def test_query_sizes_counts_every_structure(gpu_lib, handle, n):
    """xrd_query_sizes: the Friedel-unique count of every structure of the batch (sizes that are not
    multiples of the kernels' CTA or lane groups), against the oracle's full-sphere count / 2."""
    b, o = synth.small(n=n)
    db = gpu_lib.DeviceBatch.from_host(b)
    sz = handle.query_sizes(db, gpu_lib.make_opts(o, "fp32_phasefix"))
    counts = [len(oracle.enumerate_refl(b.lattice[s], o)[0]) // 2 for s in range(n)]
    assert sz.n_refl == sum(counts) and sz.max_refl == max(counts)


def test_multi_block_scans(gpu_lib, handle):
    """9000 structures: three 4096-structure chunks (the last one ragged) take the multi-block
    reflection and output scans; every structure against the oracle."""
    b, o = synth.small(n=9000)
    ref = oracle.pattern_batch(b, o, threads=0)
    got = gpu_lib.compute(b, o, "fp32_phasefix", handle=handle)
    st = compare_batch(got, ref, "fp32_phasefix", o.rel_cutoff, o.scaled)
    assert st["pairs"] > 7_000_000 // 2
    assert int(got["totals"][0]) == sum(int(x) for x in ref["n_refl"]) // 2
    _report("multi_block_scans", st)


@pytest.mark.parametrize("workload", ["small", "mixed_sample"])
def test_bench_launch_configuration_against_oracle(gpu_lib, workload):
    """The configuration bench.py times: the autotuned launch shapes, the call captured as a CUDA
    graph (profiling mode 2, the structure-factor events), replayed after an L2 flush on the
    caller's stream; every structure of the small batch (sampled ones of 20 000 mixed cells)
    against the oracle."""
    import torch
    xrd = gpu_lib
    if workload == "small":
        b, o = synth.small()
        idx = np.arange(b.n_struct)
    else:
        b, o = synth.mixed(n=100_000)
        b = b.subset(np.arange(20_000))
        idx = np.random.default_rng(17).choice(b.n_struct, 400, replace=False)
    h = xrd.Handle(0)
    try:
        db = xrd.DeviceBatch.from_host(b)
        co = xrd.make_opts(o, "fp32_phasefix")
        sz = h.query_sizes(db, co)
        out = xrd.PatternBuffers(b.n_struct, sz.n_refl)
        ws = xrd.workspace(sz.ws_bytes)
        h.autotune(db, co, out, ws)
        h.set_profiling(2)
        g = h.graph(db, co, out, ws)
        flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device="cuda")
        for _ in range(2):
            flush.fill_(1.0)
            g.launch(torch.cuda.current_stream())
        torch.cuda.synchronize()
        h.set_profiling(0)
        got = out.to_host()
        assert np.all(got["status"] == 0)
        sub = b.subset(idx)
        ref = oracle.pattern_batch(sub, o, threads=0)
        picked = {k: [got[k][i] for i in idx] for k in ("peak_tt", "peak_I", "peak_d", "peak_fam_off", "fam_hkl",
                                                        "fam_mult")}
        picked["status"] = got["status"][idx]
        st = compare_batch(picked, ref, "fp32_phasefix", o.rel_cutoff, o.scaled)
        _report("bench_configuration_" + workload, st)
        g.close()
    finally:
        h.close()


def _near_tolerance_case(lat, seed):
    """A two-atom cell and the gap between two neighbouring distinct 2-theta values (an anchor and
    the next line, both well apart from their other neighbours), as the oracle computes it."""
    rng = np.random.default_rng(seed)
    coef = synth.coef_table(rng)
    b = synth.Batch(np.asarray([lat], np.float64), np.array([0, 2], np.int64), rng.random((2, 3)),
                    np.array([26, 8], np.int16), np.ones(2), np.array([0.4, 0.9]), coef)
    o = synth.Opts(synth.CU_KA, 0.0, 70.0, 1e-5, 0.0, 0)
    u = np.unique(oracle.pattern(b, 0, o)["refl_tt"])
    for i in range(1, len(u) - 2):
        gap = u[i + 1] - u[i]
        if 0.005 < gap < 0.3 and u[i] - u[i - 1] > 2 * gap and u[i + 2] - u[i + 1] > 2 * gap:
            return b, o, gap
    raise AssertionError("no isolated pair")


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("cell", ["orthorhombic", "triclinic"])
def test_merge_decision_at_the_tolerance(gpu_lib, handle, prec, cell):
    """Two lines whose 2-theta gap lies 2e-8 (relative) below or above the tolerance: the GPU
    merges exactly when the oracle's FP64 difference of 2 asin(lambda |g| / 2) is below it."""
    lat = [4.0, 4.004, 5.3, 90.0, 90.0, 90.0] if cell == "orthorhombic" else [4.7, 5.9, 6.4, 83.0, 101.0, 112.0]
    b, o, gap = _near_tolerance_case(lat, 31)
    counts = []
    for rel in (2e-8, -2e-8):
        oo = _opts(o, tt_tol=gap * (1 + rel))
        ref = oracle.pattern_batch(b, oo, threads=1)
        got = gpu_lib.compute(b, oo, prec, handle=handle)
        st = compare_batch(got, ref, prec, oo.rel_cutoff, oo.scaled)
        assert st["boundary"] == 0
        counts.append(len(ref["peak_tt"][0]))
    assert counts[0] + 1 == counts[1]  # the pair merges below the tolerance and not above it


@pytest.mark.parametrize("prec", PRECS)
def test_back_scattering_range(gpu_lib, handle, prec):
    """2-theta up to 180 degrees: the Lorentz factor grows as 1 / cos(theta) and cos^2(theta) = 1 - sin^2(theta)
    loses digits to cancellation near the back-scattering limit; intensities still within the bar."""
    b, o = synth.small(n=48)
    o = _opts(o, tt_min=0.0, tt_max=180.0)
    ref = oracle.pattern_batch(b, o, threads=0)
    got = gpu_lib.compute(b, o, prec, handle=handle)
    assert got["sizes"]["n_refl"] * 2 == int(ref["n_refl"].sum())
    st = compare_batch(got, ref, prec, o.rel_cutoff, o.scaled)
    assert max(max(t) for t in ref["peak_tt"] if len(t)) > 175.0  # the batch reaches the limit
    _report("back_scattering_" + prec, st)


def _q_of(lat):
    _, Gs, _ = oracle.metric(lat)
    return lambda k: oracle.q_of(Gs, *k)


@pytest.mark.parametrize("prec", PRECS)
def test_reflection_list_against_oracle(gpu_lib, handle, prec):
    """The per-reflection list (Friedel-unique hkl, 2-theta, unmerged intensity) of 128 small cells,
    the NaCl cell and the two smallest large cells against the oracle's full sphere: the hkl set
    bit-exact (a reflection within 4 ulp of a sphere radius^2 is reported as boundary-ambiguous),
    every 2-theta to 1e-6 deg, every intensity to 1e-5 max(I, 1e-3 M) (FP32) / 1e-9 (FP64)."""
    bl, ol = synth.large()
    cases = [synth.small(n=128), synth.nacl(), (bl.subset(np.argsort(np.diff(bl.atom_off))[:2]), ol)]
    tot = {"refl": 0, "ambiguous": 0, "max_tt": 0.0, "max_rel": 0.0}
    for b, o in cases:
        got = gpu_lib.compute(b, o, prec, handle=handle, refl=True)
        assert int(got["totals"][0]) == sum(len(x) for x in got["refl_hkl"])
        r2 = (oracle.r2(o.tt_min, o.wavelength), oracle.r2(o.tt_max, o.wavelength))
        for s in range(b.n_struct):
            ref = oracle.pattern(b, s, o, with_refl=True)
            st = compare_reflections(got, ref, s, prec, _q_of(b.lattice[s]), r2)
            tot["refl"] += st["refl"]
            tot["ambiguous"] += st["ambiguous"]
            tot["max_tt"] = max(tot["max_tt"], st["max_tt"])
            tot["max_rel"] = max(tot["max_rel"], st["max_rel"])
    assert tot["refl"] > 100000
    _report("reflections_" + prec, tot)


_LARGEST = {}


def _largest_large_cells():
    """The 16 cells of the large workload with the most structure-factor terms (atoms x volume), and
    their oracle patterns (computed once per session: about a minute on the host cores)."""
    if not _LARGEST:
        b, o = synth.large()
        work = np.diff(b.atom_off) * np.prod(b.lattice[:, :3], axis=1)
        sub = b.subset(np.sort(np.argsort(work)[-16:]))
        _LARGEST["case"] = (sub, o, oracle.pattern_batch(sub, o, threads=0))
    return _LARGEST["case"]


@pytest.mark.parametrize("prec", ["fp32_phasefix", "fp32_phase64"])
def test_large_largest_cells(gpu_lib, handle, prec):
    """Every peak of the 16 largest cells of the large workload (1100-2000 atoms, up to ~190 000
    Friedel-unique reflections each, post-processing by the flat passes) against the oracle."""
    sub, o, ref = _largest_large_cells()
    got = gpu_lib.compute(sub, o, prec, handle=handle)
    assert got["sizes"]["max_refl"] > 6144  # the global-scratch size class
    st = compare_batch(got, ref, prec, o.rel_cutoff, o.scaled)
    assert st["pairs"] > 400000
    _report("large_largest16_" + prec, st)


@pytest.mark.parametrize("prec", ["fp32_phasefix", "fp64"])
def test_stress_cell(gpu_lib, handle, prec):
    """One 50 A cell of 940 atoms at Mo K-alpha, 2-theta 2-60 deg: about 680 000 Friedel-unique
    reflections in one structure (the shape of the paper's largest COD case, Sec. 4.2). The hkl
    set against the oracle's enumeration (bit-exact), 3000 sampled reflections against the oracle's
    structure factor, and the peak list against its own reflections (sums and multiplicities)."""
    b, o = synth.stress()
    o0 = _opts(o, rel_cutoff=0.0, scaled=0)
    got = gpu_lib.compute(b, o0, prec, handle=handle, refl=True)
    assert got["status"][0] == 0
    gh = got["refl_hkl"][0]
    assert len(gh) > 600000
    hkl_full, _ = oracle.enumerate_refl(b.lattice[0], o0)
    ref_half = hkl_full[half_space(hkl_full)]
    assert len(ref_half) * 2 == len(hkl_full)
    key = lambda a: np.sort((a[:, 0].astype(np.int64) + 512) << 20 | (a[:, 1] + 512) << 10 | (a[:, 2] + 512))  # noqa
    assert np.array_equal(key(gh), key(ref_half))
    gI, gtt = got["refl_I"][0], got["refl_tt"][0]
    M = gI.max()
    _, Gs, _ = oracle.metric(b.lattice[0])
    rng = np.random.default_rng(11)
    pick = np.concatenate([rng.choice(len(gh), 2500, replace=False), np.argsort(gI)[:250], np.argsort(gI)[-250:]])
    worst = 0.0
    tol, floor = (1e-9, 1e-6) if prec == "fp64" else (1e-5, 1e-3)
    for i in pick:
        h, k, l = (int(v) for v in gh[i])
        s2, tt, lp, d = oracle.refl(oracle.q_of(Gs, h, k, l), o0.wavelength)
        Iref = abs(oracle.sf(b, 0, h, k, l, s2)) ** 2 * lp
        assert abs(gtt[i] - tt) <= 1e-6
        assert abs(gI[i] - Iref) <= tol * max(Iref, floor * M), (h, k, l, gI[i], Iref)
        if Iref > floor * M:
            worst = max(worst, abs(gI[i] - Iref) / Iref)
    # peaks (uncut, unscaled): every reflection in exactly one family, intensities summing the pairs
    assert int(got["fam_mult"][0].sum()) == 2 * len(gh)
    assert abs(got["peak_I"][0].sum() - 2 * gI.sum()) <= 1e-6 * 2 * gI.sum()
    _report("stress_" + prec, {"refl": len(gh), "max_rel": worst})


def test_refinement_share_and_effect(gpu_lib, handle):
    """The re-evaluation touches a few percent of the small batch's reflections; without it the
    FP32 pass alone misses the elementwise bar that the tests above hold the library to."""
    import torch
    xrd = gpu_lib
    b, o = synth.small()
    ref = oracle.pattern_batch(b, o, threads=0)
    db = xrd.DeviceBatch.from_host(b)
    co = xrd.make_opts(o, "fp32_phasefix")
    sz = handle.query_sizes(db, co)
    ws = xrd.workspace(sz.ws_bytes)
    worst = {}
    try:
        for on in (True, False):
            handle.set_refine(on)
            out = xrd.PatternBuffers(b.n_struct, sz.n_refl)
            handle.pattern_batch(db, co, out, ws)
            torch.cuda.synchronize()
            refined = handle.work_counts(db, ws)[3]
            if on:
                assert 0 < refined < 0.2 * sz.n_refl, refined
            else:
                assert refined == 0
            got = out.to_host()
            w = 0.0
            for s in range(b.n_struct):
                gI, rI = got["peak_I"][s], ref["peak_I"][s]
                if len(gI) == len(rI) and len(rI):
                    m = rI > 1e-3 * 100.0
                    w = max(w, float((np.abs(gI[m] - rI[m]) / rI[m]).max()) if m.any() else 0.0)
            worst[on] = (w, refined)
    finally:
        handle.set_refine(True)
    assert worst[True][0] <= 1e-5 and worst[False][0] > worst[True][0]
    _report("refinement_small", {"max_rel_refined": worst[True][0], "max_rel_fp32_only": worst[False][0],
                                 "refined": worst[True][1], "n_refl": int(sz.n_refl)})

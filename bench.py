"""Benchmark: structure-factor terms/s and patterns/s of the powder-XRD engine on GB300.

Workload (default): the 100 000-structure mixed batch (lognormal atom counts,
median 20, and cell edges, median 7 A; Cu K-alpha, 2-theta 0-90 deg), seeded
and synthetic. One step = one CUDA-graph replay of the whole pattern path
(geometry, enumeration, structure factor + LP, re-evaluation of weak
reflections, sort, merge, families, cutoff, scaling, compaction) over the
batch, inputs resident in HBM, launch shape autotuned. L2 is flushed (256 MiB
write) between timed steps. The same line carries sub-records of the large
cells, NaCl (FP64 and FP32 latency), the 50 A stress cell and the small batch,
each timed the same way, and the FP64 and FP32-with-FP64-phase variants timed
through their own graphs.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                  [--workload mixed|large|small|stress|nacl] [--path pattern|augmented|grad]
                  [--sf-shape TILE,WARPS,RUNS | --no-tune] [--no-extras]
                  [--profile-calls K [--subset N]]

Under torchrun (N > 1) each rank takes a cost-balanced share (largest
processing time first on reflections x atoms) of a batch N times larger (weak
scaling, no collective on the data path); value = all ranks' terms / max time.
`--impl reference` times the FP64 CPU oracle on the host cores instead.
`--path augmented` times xrd_pattern_augmented (pseudo-Voigt profiles,
March-Dollase orientation and noise on a 4096-point grid); `--path grad` the
broadened pattern and its gradient.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "structure-factor terms/s and patterns/s at 1 GB300 (FP32 vs FP64) vs SFU roofline"
AUG_METRIC = "augmented patterns/s (pseudo-Voigt, March-Dollase, noise; 4096-point grid) at 1 GB300 vs MUFU roofline"
AUG_GRID = (0.0, 90.0 / 4095.0, 4096)  # t0, dt (degrees), points: the workload's 2-theta range
AUG_LAUNCHES = 10  # prep, coef, atoms, order, count, scan, emit, structure factor, structure order, profile sum

WORKLOADS = {
    "nacl": ("nacl: rock-salt NaCl conventional cell, a = 5.64 A, 8 atoms, occ 1, B 0.5 A^2, lambda 1.54184 A, "
             "2theta 0-90 deg (one structure: latency)"),
    "stress": ("stress: one P1 cell with 50 A edges, angles U[60,120] deg, 940 atoms, Z U{1..83}, B U[0,3] A^2, "
               "20% sites occ U[0.5,1], lambda 0.71073 A, 2theta 2-60 deg (~680 000 Friedel-unique reflections)"),
    "small": ("small: 1024 seeded P1 cells, a,b,c U[3,15] A, angles U[60,120] deg, 1-64 atoms, Z U{1..83}, "
              "B U[0,2] A^2, occ 1, lambda 1.54184 A, 2theta 0-90 deg"),
    "mixed": ("mixed: 100000 seeded cells, atoms lognormal (median 20, <= 500), edges lognormal (median 7 A, "
              "3-30 A), angles U[60,120] deg, Z U{1..83}, B U[0,2] A^2, lambda 1.54184 A, 2theta 0-90 deg"),
    "large": ("large: 256 seeded P1 cells, a,b,c U[15,40] A, 200-2000 atoms, 20% sites occ U[0.5,1], "
              "B U[0,3] A^2, lambda 1.54184 A, 2theta 5-120 deg"),
}


def load_workload(name, world=1):
    """The named workload; with world > 1 the batch holds world times as many structures (same
    generator), of which each rank takes one contiguous shard (weak scaling)."""
    from paper_2602_11709_gb300 import synth
    gen = {"small": synth.small, "mixed": synth.mixed, "large": synth.large, "nacl": synth.nacl,
           "stress": synth.stress}[name]
    if world == 1:
        return gen()
    import inspect
    return gen(n=inspect.signature(gen).parameters["n"].default * world)


def shard_bounds(n_total, rank, world):
    """Contiguous shard [start, end) of n_total structures for one rank; shards cover the batch."""
    q, r = divmod(n_total, world)
    start = rank * q + min(rank, r)
    return start, start + q + (1 if rank < r else 0)


def reduce_over_ranks(terms, structures, seconds, world, device="cpu"):
    """Whole-job totals: terms and structures summed over ranks, time = the slowest rank's.
    Host-side measurement only (the pattern path itself exchanges nothing between ranks)."""
    if world == 1:
        return terms, structures, seconds
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(terms), float(structures)], dtype=torch.float64, device=device)
    m = torch.tensor([float(seconds)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    dist.all_reduce(m, op=dist.ReduceOp.MAX)
    return int(t[0].item()), int(t[1].item()), float(m[0].item())


# DRAM bytes (read + write) of one k_sf launch per (workload, tile, warps, runs): dram__bytes_read.sum +
# dram__bytes_write.sum from one ncu capture of the current kernel on each timed shape (profiles/);
# a shape without a capture of the current kernel reports null.
SF_TRAFFIC_BYTES = {("mixed", 128, 1, 1): 1.81e9}
N_SMS = 152
SM_MAX_MHZ = 2070.0
GRAD_WORKLOAD = ("grad: 512 seeded P1 cells, a,b,c U[3,15] A, angles U[60,120] deg, 8-128 atoms, Z U{1..83}, "
                 "B U[0,2] A^2, lambda 1.54184 A, 2theta 5-90 deg; Gaussians FWHM 0.1 deg on 4096 points; target = "
                 "the perturbed structures")


def dist_env():
    return int(os.environ.get("RANK", 0)), int(os.environ.get("WORLD_SIZE", 1)), int(os.environ.get("LOCAL_RANK", 0))


class ClockSampler:
    """nvidia-smi clock/throttle samples during the timed region."""

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + q,
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except OSError:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def wait_first(self, timeout=5.0):
        """nvidia-smi's start-up stalls the driver: let it finish before timing."""
        t0 = time.time()
        while self.proc and not self.lines and time.time() - t0 < timeout:
            time.sleep(0.05)
        time.sleep(0.3)
        self.mark = len(self.lines)

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines[getattr(self, "mark", 0):]:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def cpu_oracle_rate(b, o, budget_s=12.0, threads=0):
    """Oracle (FP64, full sphere) on the host cores over a bounded sample of the batch."""
    import oracle
    cores = oracle.max_threads() if threads == 0 else threads
    t0 = time.perf_counter()
    done_struct = 0
    terms = 0
    counts = np.diff(b.atom_off)
    chunk = 64
    s = 0
    while time.perf_counter() - t0 < budget_s:
        idx = np.arange(s, min(s + chunk, b.n_struct))
        if len(idx) == 0:
            s = 0
            continue
        sub = b.subset(idx)
        res = oracle.pattern_batch(sub, o, threads=threads)
        terms += int((res["n_refl"] * counts[idx]).sum())
        done_struct += len(idx)
        s += chunk
    dt = time.perf_counter() - t0
    return {"terms_per_s": terms / dt, "patterns_per_s": done_struct / dt, "cores": cores, "seconds": dt,
            "structures": done_struct}


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    b, o = load_workload(args.workload)
    steps = []
    per_step_budget = max(0.2, min(20.0, 120.0 / max(args.steps + args.warmup, 1)))  # about two minutes in all
    for i in range(args.warmup + args.steps):
        r = cpu_oracle_rate(b, o, budget_s=per_step_budget)
        if i >= args.warmup:
            steps.append(r)
    tps = float(np.mean([r["terms_per_s"] for r in steps]))
    pps = float(np.mean([r["patterns_per_s"] for r in steps]))
    line = {"impl": "reference", "metric": METRIC, "value": tps, "unit": "terms/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * b.n_struct / pps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOADS[args.workload], "n_struct": b.n_struct, "precision": "oracle fp64"},
            "patterns_per_s": pps,
            "cpu_baseline": {"value": tps, "unit": "terms/s", "cores": steps[0]["cores"], "kind": "oracle",
                             "sample": "consecutive 64-structure chunks of the batch, %.2f s per step" % per_step_budget},
            "e2e": {"value": tps, "unit": "terms/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def _graph_ms(h, graph, steps, flush, stream, sf=False):
    """Mean ms per CUDA-graph replay over `steps` replays, L2 flushed before each; with sf=True also
    the mean structure-factor and re-evaluation stage times (the handle records them in mode 2)."""
    import torch
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    sf_ms, ref_ms = [], []
    for i in range(steps):
        flush.fill_(1.0)
        ev[i][0].record(stream)
        graph.launch(stream)
        ev[i][1].record(stream)
        if sf:
            t = h.stage_times()  # synchronises on the step's last recorded event
            sf_ms.append(t["structure_factor"])
            ref_ms.append(t.get("refine", 0.0))
    torch.cuda.synchronize()
    ms = [a.elapsed_time(c) for a, c in ev]
    return ms, (float(np.mean(sf_ms)) if sf_ms else None), (float(np.mean(ref_ms)) if ref_ms else None)


def _half_counts(h, db, o, precision, sz, dev):
    """Friedel-unique reflections per structure (half the multiplicity sum of the uncut pattern)."""
    import torch
    from paper_2602_11709_gb300 import synth, xrd
    n = db.n_struct
    co0 = xrd.make_opts(synth.Opts(o.wavelength, o.tt_min, o.tt_max, o.tt_tol, 0.0, 0), precision)
    out0 = xrd.PatternBuffers(n, sz.n_refl, dev, refl=True)
    h.pattern_batch(db, co0, out0, xrd.workspace(sz.ws_bytes, dev))
    torch.cuda.synchronize()
    ro = out0.refl_off.cpu().numpy()
    return np.diff(ro).astype(np.int64)


class Roofline:
    """Arithmetic floor of the structure-factor kernel (pattern variants) from the measured unit
    rates (xrd_unit_rates) and the batch's operation counts. FP32 pipe, per phase seed: the exact
    phase (3 integer multiply-adds) and sin/cos from it on the FMA pipe (17 operations: quarter turn,
    conversion and scale, a^2, two polynomials, the rotation back); per term: the Debye-Waller
    argument, the weight, two accumulations, the error scale (3) and the blocked two-float sum (14 per
    block of 8 atoms, 16 with runs); with runs, per reflection after a run's first the step to l + 1
    (4, then 2 for the two-term recurrence); per (reflection, element run) f(s): four exponent
    arguments, four multiply-adds and the error-scale bound (9). MUFU pipe: one exp2 per term
    (Debye-Waller) and four per (reflection, element run) for f(s). The floor is the larger of the
    two pipes' times."""

    def __init__(self, h, sms=N_SMS):
        self.rates = h.unit_rates()
        self.sms = sms

    @staticmethod
    def fp32_ops(terms, seeds, runs, f_evals=0.0):
        per_term = 4.0 + (14.0 / 16.0 if runs else 14.0 / 8.0)
        ops = terms * per_term + seeds * (3.0 + 17.0 + (3.0 if runs else 0.0)) + 9.0 * f_evals
        if runs:
            ops += (terms - seeds) * (8.0 / 3.0)  # a run of four: 4 + 2 + 2 for its last three reflections
        else:
            ops += terms * 3.0
        return ops

    def floors_s(self, terms, seeds, f_evals, runs, mhz):
        r = self.rates
        den = self.sms * mhz * 1e6
        fp32 = self.fp32_ops(terms, seeds, runs, f_evals) / r["ffma"] / den
        mufu = (terms + 4.0 * f_evals) / r["mufu_ex2"] / den
        return fp32, mufu

    def floor_s(self, terms, seeds, f_evals, mhz, runs=False):
        return max(self.floors_s(terms, seeds, f_evals, runs, mhz))


def roofline_record(roof, terms, seeds, f_evals, runs, mhz, sf_ms):
    """k_sf against its arithmetic floor (Roofline): achieved and peak in Friedel-unique terms/s."""
    fp32, mufu = roof.floors_s(terms, seeds, f_evals, runs, mhz)
    floor = max(fp32, mufu)
    t = sf_ms / 1e3
    return {"bound": "alu", "unit": "Gterm/s", "achieved": terms / t / 1e9, "peak": terms / floor / 1e9,
            "frac": floor / t, "fp32_pipe_frac": fp32 / t, "mufu_frac": mufu / t,
            "fp32_ops_per_term": roof.fp32_ops(terms, seeds, runs, f_evals) / max(terms, 1),
            "phase_seeds_per_term": seeds / max(terms, 1), "kernel": "k_sf"}


def measure_pattern(h, b, o, precision, dev, steps, warmup, flush, stream, tune=True, shape=None, roof=None,
                    mhz=None, other_precisions=(), other_steps=3):
    """One workload through the pattern path: launch-shape tuning, one CUDA graph per precision,
    timed replays. Returns a dict (ms per step, terms and patterns per second, the k_sf roofline,
    the re-evaluation's share, the stage breakdown, the other precisions timed the same way)."""
    import torch
    from paper_2602_11709_gb300 import xrd
    db = xrd.DeviceBatch.from_host(b, dev)
    co = xrd.make_opts(o, precision)
    sz = h.query_sizes(db, co)
    out = xrd.PatternBuffers(b.n_struct, sz.n_refl, dev)
    ws = xrd.workspace(sz.ws_bytes, dev)
    half = _half_counts(h, db, o, precision, sz, dev)
    assert int(half.sum()) == int(sz.n_refl)
    counts = np.diff(b.atom_off).astype(np.int64)
    species = np.array([len(np.unique(b.Z[b.atom_off[s]:b.atom_off[s + 1]])) for s in range(b.n_struct)])
    terms_full = int((2 * half * counts).sum())
    terms_eval = int((half * counts).sum())
    f_evals = float((half * species).sum())
    if shape:
        h.set_sf_shape(*shape)
        tuned = tuple(shape)
    else:
        tuned = h.autotune(db, co, out, ws) if tune else None
    h.set_profiling(2)
    graph = h.graph(db, co, out, ws)
    for _ in range(warmup):
        flush.fill_(1.0)
        graph.launch(stream)
    torch.cuda.synchronize()
    ms, sf_ms, ref_ms = _graph_ms(h, graph, steps, flush, stream, sf=True)
    w_terms, w_seeds, _, refined = h.work_counts(db, ws)
    assert w_terms == terms_eval, (w_terms, terms_eval)
    totals = out.totals.cpu().numpy()
    assert int(totals[3]) == 0, totals
    # per-stage breakdown from a separate pass (events between all stages add time per stage)
    h.set_profiling(1)
    graph1 = h.graph(db, co, out, ws)
    acc = {}
    nst = min(steps, 10)
    for _ in range(nst):
        flush.fill_(1.0)
        graph1.launch(stream)
        for k, v in h.stage_times().items():
            if k != "profile_sum":
                acc[k] = acc.get(k, 0.0) + v / nst
    h.set_profiling(0)
    # post-processing (sort, merge, families, cutoff, staging) and compaction against HBM: algorithmic
    # bytes per Friedel-unique reflection (|g|^2, key, intensity read), per kept peak (staged |g|^2,
    # intensity, family offset; compaction: those read, 2-theta, d, intensity, family offset written)
    # and per family (packed hkl and multiplicity staged; compaction: those read, hkl and
    # multiplicity written)
    ib = 8 if precision == "fp64" else 4
    npk, nfm = int(totals[1]), int(totals[2])
    post_bytes = (12 + ib) * int(sz.n_refl) + (12 + ib) * npk + 8 * nfm
    comp_bytes = (12 + ib + 32) * npk + (8 + 16) * nfm
    hbm = measured_hbm_gbs()
    hbm_rec = {}
    for stage, nbytes in (("post", post_bytes), ("compact", comp_bytes)):
        t = acc.get(stage)
        if t:
            gbs = nbytes / (t / 1e3) / 1e9
            hbm_rec[stage] = {"ms": t, "algorithmic_bytes": nbytes, "achieved_gbs": gbs, "hbm_frac": gbs / hbm[0],
                              "peak_gbs": hbm[0], "peak_basis": hbm[1]}
    res = {"n_struct": b.n_struct, "ms_per_step": float(np.mean(ms)), "step_ms": ms, "terms_full": terms_full,
           "terms_eval": terms_eval, "n_refl": int(sz.n_refl), "refined": int(refined),
           "sf_ms": sf_ms, "refine_ms": ref_ms, "stage_ms": acc, "tuned": tuned, "seeds": w_seeds,
           "f_evals": f_evals, "hbm_stages": hbm_rec}
    res["terms_per_s"] = terms_full / (res["ms_per_step"] / 1e3)
    res["patterns_per_s"] = b.n_struct / (res["ms_per_step"] / 1e3)
    runs = bool(tuned and tuned[2])
    res["runs"] = runs
    if roof is not None and sf_ms and precision == "fp32_phasefix":
        res["roofline"] = roofline_record(roof, terms_eval, w_seeds, f_evals, runs, mhz or SM_MAX_MHZ, sf_ms)
    other = {}
    for pname in other_precisions:
        cp = xrd.make_opts(o, pname)
        g2 = h.graph(db, cp, out, ws)
        g2.launch(stream)
        torch.cuda.synchronize()
        ms2, _, _ = _graph_ms(h, g2, other_steps, flush, stream)
        m2 = float(np.mean(ms2))
        other[pname] = {"ms_per_step": m2, "terms_per_s": terms_full / (m2 / 1e3), "launch": "CUDA graph"}
        g2.close()
    res["other_precisions"] = other
    graph.close()
    graph1.close()
    return res, (db, co, sz)


def measured_hbm_gbs():
    """HBM copy bandwidth of the GB300s (MEASURED_PEAKS.json beside this file), else the
    earlier single measurement used as the fallback."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["hbm_gbs"]), "measured (MEASURED_PEAKS.json hbm_gbs)"
    except (OSError, KeyError, ValueError):
        return 6800.0, "fallback 6.8 TB/s"


def d2h_ceiling(nbytes, dev):
    """Pinned device-to-host bandwidth of one large cudaMemcpyAsync (GB/s): the link's ceiling."""
    import torch
    nbytes = max(int(nbytes), 1 << 20)
    src = torch.empty(nbytes, dtype=torch.uint8, device=dev)
    dst = torch.empty(nbytes, dtype=torch.uint8).pin_memory()
    st = torch.cuda.current_stream()
    best = 0.0
    for _ in range(5):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(st)
        dst.copy_(src, non_blocking=True)
        e1.record(st)
        torch.cuda.synchronize()
        best = max(best, nbytes / (e0.elapsed_time(e1) / 1e3) / 1e9)
    return best


def run_ours(args):
    import torch
    from paper_2602_11709_gb300 import synth, xrd

    rank, world, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    dev_i = local if torch.cuda.is_available() else 0
    torch.cuda.set_device(dev_i)
    dev = "cuda:%d" % dev_i
    b, o = load_workload(args.workload, world)
    if world > 1:  # this rank's structures: cost-balanced (LPT) over the world-times-larger batch
        from paper_2602_11709_gb300 import shard
        h0 = xrd.Handle(dev_i)
        cnt = h0.reflection_counts(xrd.DeviceBatch.from_host(b, dev), xrd.make_opts(o, args.precision))
        h0.close()
        parts = shard.partition(shard.costs(cnt, np.diff(b.atom_off)), world)
        b = b.subset(parts[rank])
    h = xrd.Handle(dev_i)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream()
    roof = Roofline(h, torch.cuda.get_device_properties(dev_i).multi_processor_count)

    def barrier():
        if world > 1:
            import torch.distributed as dist
            dist.barrier()
        torch.cuda.synchronize()

    shape = tuple(int(v) for v in args.sf_shape.split(",")) if args.sf_shape else None
    clocks = ClockSampler(dev_i)
    clocks.start()
    clocks.wait_first()
    barrier()
    main, (db, co, sz) = measure_pattern(
        h, b, o, args.precision, dev, args.steps, args.warmup, flush, stream, tune=not args.no_tune, shape=shape,
        roof=roof, mhz=None, other_precisions=("fp64", "fp32_phase64") if args.fp64_steps > 0 else (),
        other_steps=max(args.fp64_steps, 1))
    barrier()
    ck = clocks.stop()
    mhz = ck.get("sm_mhz") or SM_MAX_MHZ
    if "roofline" in main:  # the floor at the clock the kernel ran at
        main["roofline"] = roofline_record(roof, main["terms_eval"], main["seeds"], main["f_evals"], main["runs"],
                                           mhz, main["sf_ms"])
    total_terms, total_structs, total_s = reduce_over_ranks(main["terms_full"], b.n_struct,
                                                            sum(main["step_ms"]) / 1e3, world, dev)
    value = total_terms * args.steps / total_s
    pps = total_structs * args.steps / total_s

    # end to end through the public API: pinned host inputs -> device -> pattern -> host results,
    # two batches in flight (xrd.PatternPipeline: a batch's output copies overlap the next batch)
    host = {k: torch.from_numpy(np.ascontiguousarray(getattr(b, k))).pin_memory()
            for k in ("lattice", "atom_off", "frac", "Z", "occ", "B", "coef")}
    co_e = xrd.make_opts(o, args.precision)
    pp = xrd.PatternPipeline(h, b, co_e, sz, device=dev_i)
    for _ in range(args.warmup):
        pp.submit(host)
    res = pp.flush()
    assert int(res["totals"][3]) == 0
    torch.cuda.synchronize()
    b_in0, b_out0 = pp.bytes_in, pp.bytes_out
    e2e_steps = min(args.steps, 50)
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        pp.submit(host)
    res = pp.flush()
    torch.cuda.synchronize()
    e2e_total = time.perf_counter() - t0
    assert int(res["totals"][3]) == 0
    h2d = (pp.bytes_in - b_in0) // e2e_steps
    d2h = (pp.bytes_out - b_out0) // e2e_steps
    e2e_terms, _, e2e_s = reduce_over_ranks(main["terms_full"], b.n_struct, e2e_total / e2e_steps, world, dev)
    link = d2h_ceiling(d2h, dev)
    del pp

    extras = {}
    if world == 1 and not args.no_extras and args.workload == "mixed":
        for name in ("large", "nacl", "stress", "small"):
            bx, ox = load_workload(name)
            rx, _ = measure_pattern(h, bx, ox, args.precision, dev, 10 if name != "nacl" else 50, 3, flush, stream,
                                    tune=name in ("large", "small"), roof=roof, mhz=mhz,
                                    other_precisions=("fp64", "fp32_phase64") if name != "stress" else ("fp64",),
                                    other_steps=3)
            rec = {"workload": WORKLOADS[name], "ms_per_step": rx["ms_per_step"], "terms_per_s": rx["terms_per_s"],
                   "patterns_per_s": rx["patterns_per_s"], "reflections_friedel_unique": rx["n_refl"],
                   "refined_reflections": rx["refined"], "sf_ms": rx["sf_ms"], "refine_ms": rx["refine_ms"],
                   "stage_ms": rx["stage_ms"], "hbm_stages": rx["hbm_stages"],
                   "other_precisions": rx["other_precisions"],
                   "sf_shape": {"tile": rx["tuned"][0], "warps": rx["tuned"][1], "runs_in_l": rx["tuned"][2]}
                   if rx["tuned"] else "default"}
            if "roofline" in rx:
                rec["roofline"] = rx["roofline"]
            if "fp64" in rx["other_precisions"]:
                rec["speedup_vs_fp64_gpu"] = rx["other_precisions"]["fp64"]["ms_per_step"] / rx["ms_per_step"]
            extras[name] = rec

    if rank == 0:
        cpu = None
        if world == 1 and args.cpu_seconds > 0:
            r = cpu_oracle_rate(b, o, budget_s=args.cpu_seconds)
            cpu = {"value": r["terms_per_s"], "unit": "terms/s", "cores": r["cores"], "kind": "oracle",
                   "sample": "%d structures of the batch (consecutive 64-structure chunks), %.1f s" %
                             (r["structures"], r["seconds"]),
                   "patterns_per_s": r["patterns_per_s"]}
        tuned = main["tuned"]
        roofl = dict(main.get("roofline", {}))
        roofl.update({"unit_rates_per_clk_per_sm": {k: round(v, 2) for k, v in roof.rates.items()},
                      "traffic": SF_TRAFFIC_BYTES.get((args.workload,) + tuple(tuned or (128, 2, 0))),
                      "traffic_unit": "bytes per launch (dram read + write, ncu, this shape)",
                      "peak_basis": "arithmetic floor from unit rates measured in this run (xrd_unit_rates: FFMA "
                                    "%.1f, MUFU ex2 %.1f per clk per SM) x %d SMs at the sampled SM clock %.0f MHz: "
                                    "the larger of the FP32-pipe floor (per phase seed 20 operations: exact phase and "
                                    "sin/cos on the FMA pipe; per term the Debye-Waller argument, weight, two "
                                    "accumulations, error scale and blocked sum; the l + 1 step with runs; 9 per "
                                    "reflection and element run for f(s)) and the MUFU floor (exp2 per term and four "
                                    "per reflection and element run); "
                                    "Friedel-unique terms"
                                    % (roof.rates["ffma"], roof.rates["mufu_ex2"], roof.sms, mhz)})
        line = {
            "metric": METRIC, "value": value, "unit": "terms/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * total_s / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None,
            "dtype": "f32 (i32 phase)" if args.precision == "fp32_phasefix" else args.precision, "data": "synthetic",
            "config": {"workload": WORKLOADS[args.workload], "n_struct": b.n_struct, "precision": args.precision,
                       "terms_full_sphere": main["terms_full"], "terms_evaluated": main["terms_eval"],
                       "reflections_friedel_unique": main["n_refl"], "l2": "flushed between steps (256 MiB write)",
                       "parallelism": "cost-balanced structure shard per GPU" if world > 1 else "1 GPU",
                       "launch": "CUDA graph",
                       "sf_shape": {"tile": tuned[0], "warps": tuned[1], "runs_in_l": tuned[2]} if tuned else
                       "default"},
            "patterns_per_s": pps,
            "roofline": roofl,
            "refine": {"reflections": main["refined"], "share": main["refined"] / max(main["n_refl"], 1),
                       "ms": main["refine_ms"], "kernel": "k_refine (double-float re-evaluation of weak reflections)"},
            "cpu_baseline": cpu,
            "e2e": {"value": e2e_terms / e2e_s, "unit": "terms/s", "h2d_bytes_per_step": int(h2d),
                    "d2h_bytes_per_step": int(d2h), "ms_per_step": e2e_s * 1e3,
                    "api": "xrd.PatternPipeline, two batches in flight",
                    "d2h_link_gbs": link, "d2h_copy_bound_ms": d2h / (link * 1e9) * 1e3},
            "clocks": ck,
            "gpu_launches": xrd.launches_per_batch(b.n_struct, args.precision != "fp64") * args.steps,
            "stage_ms": main["stage_ms"],
            "stage_ms_note": "separate pass with events between all stages (adds time per stage)",
            "hbm_stages": main["hbm_stages"],
            "other_precisions": main["other_precisions"],
        }
        if "fp64" in main["other_precisions"]:
            line["speedup_vs_fp64_gpu"] = main["other_precisions"]["fp64"]["ms_per_step"] / main["ms_per_step"]
        if extras:
            line["workloads"] = extras
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


def cpu_oracle_augmented_rate(b, o, aug, budget_s=12.0):
    """Oracle augmented pattern (FP64, full sphere, every grid point) over a bounded sample."""
    import oracle
    t0g, dtg, npts = AUG_GRID
    t0 = time.perf_counter()
    done = 0
    s = 0
    while time.perf_counter() - t0 < budget_s:
        hkl, _ = oracle.enumerate_refl(b.lattice[s], o)
        oracle.augmented(b, s, hkl, o.wavelength, t0g, dtg, npts, aug.fwhm[s], aug.eta[s], aug.po_dir[s],
                         aug.po_r[s], z=aug.z[s].astype(np.float64), sigma=aug.noise_sigma[s])
        done += 1
        s = (s + 1) % b.n_struct
    dt = time.perf_counter() - t0
    return {"patterns_per_s": done / dt, "structures": done, "seconds": dt, "cores": 1}


def run_augmented(args):
    """The augmented-pattern path (xrd_pattern_augmented) on the workload's batch: one step = the
    geometry, structure factors and the pseudo-Voigt / March-Dollase / noise profile of every
    structure on the 4096-point grid."""
    import torch
    from paper_2602_11709_gb300 import synth, xrd

    rank, world, local = dist_env()
    if args.impl == "reference":
        if rank != 0:
            return
        b, o = load_workload(args.workload)
        aug = synth.augment(b.n_struct, AUG_GRID[2], seed=7)
        per_step = max(2.0, min(20.0, 100.0 / max(args.steps + args.warmup, 1)))
        rates = [cpu_oracle_augmented_rate(b, o, aug, per_step) for _ in range(args.warmup + args.steps)]
        pps = float(np.mean([r["patterns_per_s"] for r in rates[args.warmup:]]))
        print(json.dumps({"impl": "reference", "metric": AUG_METRIC, "value": pps, "unit": "patterns/s",
                          "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
                          "ms_per_step": 1e3 * b.n_struct / pps, "higher_is_better": True, "scaling": "weak",
                          "vs_baseline": None, "dtype": "f64", "data": "synthetic",
                          "config": {"workload": WORKLOADS[args.workload], "path": "augmented"},
                          "cpu_baseline": {"value": pps, "unit": "patterns/s", "cores": 1, "kind": "oracle",
                                           "sample": "consecutive structures, %.0f s per step" % per_step},
                          "e2e": {"value": pps, "unit": "patterns/s", "h2d_bytes_per_step": 0,
                                  "d2h_bytes_per_step": 0}}), flush=True)
        return
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    dev = local if torch.cuda.is_available() else 0
    torch.cuda.set_device(dev)
    b, o = load_workload(args.workload, world)
    if world > 1:
        lo, hi = shard_bounds(b.n_struct, rank, world)
        b = b.subset(np.arange(lo, hi))
    aug = synth.augment(b.n_struct, AUG_GRID[2], seed=7)
    d = "cuda:%d" % dev
    h = xrd.Handle(dev)
    db = xrd.DeviceBatch.from_host(b, d)
    co = xrd.make_opts(o, "fp32_phasefix")
    grid = xrd.make_grid(synth.Grid(t0=AUG_GRID[0], dt=AUG_GRID[1], n_pts=AUG_GRID[2]))
    sz = h.query_sizes(db, co)
    ws = xrd.workspace(sz.ws_grad_bytes, d)
    tuned = h.autotune(db, co, xrd.PatternBuffers(b.n_struct, sz.n_refl, d), xrd.workspace(sz.ws_bytes, d)) \
        if not args.no_tune else None
    host = {k: torch.from_numpy(np.ascontiguousarray(getattr(aug, k))).pin_memory()
            for k in ("fwhm", "eta", "po_dir", "po_r", "noise_sigma", "z")}
    dv = {k: v.to(d) for k, v in host.items()}
    n, npts = b.n_struct, AUG_GRID[2]
    y = torch.empty((n, npts), dtype=torch.float32, device=d)
    status = torch.zeros(n, dtype=torch.int32, device=d)
    totals = torch.zeros(4, dtype=torch.int64, device=d)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=d)
    stream = torch.cuda.current_stream()

    def call(t):
        h.pattern_augmented(db, co, grid, t["fwhm"], t["eta"], y, status, totals, ws, po_dir=t["po_dir"],
                            po_r=t["po_r"], noise_z=t["z"], noise_sigma=t["noise_sigma"])

    def barrier():
        if world > 1:
            import torch.distributed as dist
            dist.barrier()
        torch.cuda.synchronize()
    h.set_profiling(2)
    clocks = ClockSampler(dev)
    clocks.start()
    clocks.wait_first()
    for _ in range(args.warmup):
        flush.fill_(1.0)
        call(dv)
    barrier()
    assert int(totals[3]) == 0 and int(status.abs().sum()) == 0
    R = int(totals[0])
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    sum_ms = []
    for i in range(args.steps):
        flush.fill_(1.0)
        ev[i][0].record(stream)
        call(dv)
        ev[i][1].record(stream)
        sum_ms.append(h.stage_times()["profile_sum"])
    barrier()
    ck = clocks.stop()
    h.set_profiling(0)
    step_s = sum(a.elapsed_time(c) for a, c in ev) / 1e3
    tot_terms, tot_structs, tot_s = reduce_over_ranks(R * npts, n, step_s, world, d)
    pps = tot_structs * args.steps / tot_s
    # end to end: every step copies its inputs (batch arrays and effect parameters, noise draws
    # included) from pinned host memory, runs the call and reads the patterns back to pinned memory
    hb = {k: torch.from_numpy(np.ascontiguousarray(getattr(b, k))).pin_memory()
          for k in ("lattice", "atom_off", "frac", "Z", "occ", "B", "coef")}
    y_host = torch.empty((n, npts), dtype=torch.float32).pin_memory()
    bytes_in = sum(t.numel() * t.element_size() for t in list(hb.values()) + list(host.values()))
    bytes_out = y_host.numel() * 4

    def e2e_step():
        for k, t in hb.items():
            getattr(db, k).copy_(t, non_blocking=True)
        for k, t in host.items():
            dv[k].copy_(t, non_blocking=True)
        call(dv)
        y_host.copy_(y, non_blocking=True)
    for _ in range(args.warmup):
        e2e_step()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        e2e_step()
    torch.cuda.synchronize()
    e2e_s = (time.perf_counter() - t0) / args.steps
    _, e2e_structs, e2e_max = reduce_over_ranks(R * npts, n, e2e_s, world, d)
    if rank == 0:
        sum_s = float(np.mean(sum_ms)) / 1e3
        # profile sum: one MUFU reciprocal per two (point, reflection) pairs, 16 MUFU/clk/SM
        peak_terms = 2.0 * 16.0 * 152.0 * SM_MAX_MHZ * 1e6
        cpu = None
        if world == 1 and args.cpu_seconds > 0:
            r = cpu_oracle_augmented_rate(b, o, aug, args.cpu_seconds)
            cpu = {"value": r["patterns_per_s"], "unit": "patterns/s", "cores": r["cores"], "kind": "oracle",
                   "sample": "%d structures of the batch in order, %.1f s" % (r["structures"], r["seconds"])}
        line = {
            "metric": AUG_METRIC, "value": pps, "unit": "patterns/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * tot_s / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32 (i32 phase)", "data": "synthetic",
            "config": {"workload": WORKLOADS[args.workload], "path": "augmented", "n_struct": n,
                       "grid": {"t0": AUG_GRID[0], "dt": AUG_GRID[1], "n_pts": npts},
                       "effects": "fwhm U[0.05,0.3] deg, eta U[0,1], March-Dollase r U[0.6,1.4] about a "
                                  "low-index direction, noise sigma U[0,1] with standard normal draws",
                       "point_reflection_terms": R * npts, "l2": "flushed between steps (256 MiB write)",
                       "sf_shape": {"tile": tuned[0], "warps": tuned[1], "runs_in_l": tuned[2]} if tuned else
                       "default"},
            "terms_per_s": tot_terms * args.steps / tot_s,
            "roofline": {"bound": "alu", "unit": "Gterm/s", "achieved": R * npts / sum_s / 1e9,
                         "peak": peak_terms / 1e9, "frac": (R * npts / sum_s) / peak_terms, "traffic": None,
                         "kernel": "k_aug_order + k_aug_sum",
                         "peak_basis": "MUFU: one reciprocal per two (point, reflection) terms at 16/clk/SM, "
                                       "152 SMs, 2070 MHz"},
            "cpu_baseline": cpu,
            "e2e": {"value": e2e_structs / e2e_max, "unit": "patterns/s", "h2d_bytes_per_step": int(bytes_in),
                    "d2h_bytes_per_step": int(bytes_out), "ms_per_step": e2e_max * 1e3,
                    "api": "Handle.pattern_augmented with pinned host copies each step"},
            "clocks": ck,
            "gpu_launches": AUG_LAUNCHES * args.steps,
        }
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


GRAD_METRIC = ("broadened-pattern gradients/s (forward + adjoint w.r.t. coordinates, B and lattice; 4096-point "
               "grid) at 1 GB300 vs MUFU roofline")
GRAD_LAUNCHES = 11  # prep, coef, atoms, order, count, scan, emit, structure factor, broaden | grad_refl, grad_atoms


def cpu_oracle_grad_rate(b, o, grid, g, budget_s=10.0):
    """Oracle broadened pattern + analytic gradient (FP64, full sphere, no window) over a bounded
    sample of the batch's structures, one after another on one core."""
    import oracle
    t0 = time.perf_counter()
    done, s = 0, 0
    while time.perf_counter() - t0 < budget_s:
        hkl, _ = oracle.enumerate_refl(b.lattice[s], o)
        oracle.broadened(b, s, hkl, o.wavelength, grid)
        oracle.broadened_grad(b, s, hkl, o.wavelength, grid, g[s])
        done += 1
        s = (s + 1) % b.n_struct
    dt = time.perf_counter() - t0
    return {"structures_per_s": done / dt, "structures": done, "seconds": dt, "cores": 1}


def run_grad(args):
    """The gradient path: 512 structures of 8-128 atoms, Gaussian-broadened (FWHM 0.1 deg) on a
    4096-point grid over 5-90 deg, loss = mean squared difference to a perturbed-structure target.
    One step = xrd_pattern_broadened (forward), the loss gradient dL/dy (one torch elementwise
    expression, the caller's loss), xrd_pattern_grad (adjoint: coordinates, B, lattice)."""
    import torch
    from paper_2602_11709_gb300 import synth, xrd

    rank, world, local = dist_env()
    b, t, o, grid = synth.grad()
    n, npts = b.n_struct, grid.n_pts
    if args.impl == "reference":
        if rank != 0:
            return
        g = np.random.default_rng(3).standard_normal((n, npts))
        per = max(2.0, min(20.0, 100.0 / max(args.steps + args.warmup, 1)))
        rates = [cpu_oracle_grad_rate(b, o, grid, g, per) for _ in range(args.warmup + args.steps)]
        sps = float(np.mean([r["structures_per_s"] for r in rates[args.warmup:]]))
        print(json.dumps({"impl": "reference", "metric": GRAD_METRIC, "value": sps, "unit": "structures/s",
                          "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
                          "ms_per_step": 1e3 * n / sps, "higher_is_better": True, "scaling": "weak",
                          "vs_baseline": None, "dtype": "f64", "data": "synthetic",
                          "config": {"workload": GRAD_WORKLOAD, "path": "grad"},
                          "cpu_baseline": {"value": sps, "unit": "structures/s", "cores": 1, "kind": "oracle",
                                           "sample": "consecutive structures, %.0f s per step" % per},
                          "e2e": {"value": sps, "unit": "structures/s", "h2d_bytes_per_step": 0,
                                  "d2h_bytes_per_step": 0}}), flush=True)
        return
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
        lo, hi = shard_bounds(n, rank, world)
        b, t = b.subset(np.arange(lo, hi)), t.subset(np.arange(lo, hi))
        n = b.n_struct
    dev_i = local if torch.cuda.is_available() else 0
    torch.cuda.set_device(dev_i)
    d = "cuda:%d" % dev_i
    h = xrd.Handle(dev_i)
    roof = Roofline(h, torch.cuda.get_device_properties(dev_i).multi_processor_count)
    db, dt_ = xrd.DeviceBatch.from_host(b, d), xrd.DeviceBatch.from_host(t, d)
    co = xrd.make_opts(o, "fp32_phasefix")
    cg = xrd.make_grid(grid)
    sz, szt = h.query_sizes(db, co), h.query_sizes(dt_, co)
    ws = xrd.workspace(max(sz.ws_grad_bytes, szt.ws_grad_bytes), d)
    y = torch.empty(n, npts, dtype=torch.float32, device=d)
    yt = torch.empty(n, npts, dtype=torch.float32, device=d)
    status = torch.zeros(n, dtype=torch.int32, device=d)
    totals = torch.zeros(4, dtype=torch.int64, device=d)
    h.pattern_broadened(dt_, co, cg, yt, status, totals, ws)  # the fitting target
    torch.cuda.synchronize()
    scale = 1.0 / (n * npts)
    d_frac = torch.empty(b.n_atoms, 3, dtype=torch.float32, device=d)
    d_B = torch.empty(b.n_atoms, dtype=torch.float32, device=d)
    d_lat = torch.empty(n, 6, dtype=torch.float32, device=d)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=d)
    stream = torch.cuda.current_stream()
    ev_mid = []

    def step(mark=False):
        h.pattern_broadened(db, co, cg, y, status, totals, ws)
        gy = (y - yt) * (2.0 * scale)
        if mark:
            e = (torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
            e[0].record(stream)
        h.pattern_grad(db, co, cg, gy, d_frac, d_B, d_lat, ws)
        if mark:
            e[1].record(stream)
            ev_mid.append(e)
    clocks = ClockSampler(dev_i)
    clocks.start()
    clocks.wait_first()
    for _ in range(args.warmup):
        flush.fill_(1.0)
        step()
    torch.cuda.synchronize()
    assert int(totals[3]) == 0
    R = int(totals[0])
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    for i in range(args.steps):
        flush.fill_(1.0)
        ev[i][0].record(stream)
        step(mark=True)
        ev[i][1].record(stream)
    torch.cuda.synchronize()
    ck = clocks.stop()
    mhz = ck.get("sm_mhz") or SM_MAX_MHZ
    step_s = sum(a.elapsed_time(c) for a, c in ev) / 1e3
    adj_s = float(np.mean([a.elapsed_time(c) for a, c in ev_mid])) / 1e3
    counts = np.diff(b.atom_off)
    terms = float((np.diff(_refl_off_of(h, db, co, sz, d)) * counts).sum())
    # adjoint floor: per (atom, reflection) sin + cos and five exp2 (f(s) and Debye-Waller)
    r = roof.rates
    floor = terms * (1.0 / r["mufu_sin"] + 1.0 / r["mufu_cos"] + 5.0 / r["mufu_ex2"]) / (roof.sms * mhz * 1e6)
    _, tot_structs, tot_s = reduce_over_ranks(0, n, step_s, world, d)
    value = tot_structs * args.steps / tot_s
    # end to end through the public API: the batch's differentiable inputs copied in from pinned memory,
    # forward, loss gradient, adjoint, gradients and the loss read back every step
    hb = {k: torch.from_numpy(np.ascontiguousarray(getattr(b, k))).pin_memory() for k in ("frac", "B", "lattice")}
    out_h = {"d_frac": torch.empty_like(d_frac, device="cpu").pin_memory(),
             "d_B": torch.empty_like(d_B, device="cpu").pin_memory(),
             "d_lat": torch.empty_like(d_lat, device="cpu").pin_memory()}
    loss_h = torch.empty(1, dtype=torch.float32).pin_memory()

    def e2e_step():
        for k, v in hb.items():
            getattr(db, k).copy_(v, non_blocking=True)
        step()
        loss_h.copy_(((y - yt) ** 2).sum().reshape(1) * scale, non_blocking=True)
        out_h["d_frac"].copy_(d_frac, non_blocking=True)
        out_h["d_B"].copy_(d_B, non_blocking=True)
        out_h["d_lat"].copy_(d_lat, non_blocking=True)
    for _ in range(args.warmup):
        e2e_step()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        e2e_step()
    torch.cuda.synchronize()
    e2e_s = (time.perf_counter() - t0) / args.steps
    _, e2e_structs, e2e_max = reduce_over_ranks(0, n, e2e_s, world, d)
    bytes_in = sum(v.numel() * v.element_size() for v in hb.values())
    bytes_out = sum(v.numel() * v.element_size() for v in out_h.values()) + 4
    if rank == 0:
        cpu = None
        if world == 1 and args.cpu_seconds > 0:
            g = ((y - yt) * (2.0 * scale)).cpu().numpy().astype(np.float64)
            rr = cpu_oracle_grad_rate(b, o, grid, g, args.cpu_seconds)
            cpu = {"value": rr["structures_per_s"], "unit": "structures/s", "cores": 1, "kind": "oracle",
                   "sample": "%d structures of the batch in order, %.1f s" % (rr["structures"], rr["seconds"])}
        line = {
            "metric": GRAD_METRIC, "value": value, "unit": "structures/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * tot_s / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32 (i32 phase)", "data": "synthetic",
            "config": {"workload": GRAD_WORKLOAD, "path": "grad", "n_struct": n, "reflections_friedel_unique": R,
                       "grid": {"t0": grid.t0, "dt": grid.dt, "n_pts": npts, "fwhm": grid.fwhm},
                       "loss": "mean squared difference to the target's broadened pattern",
                       "l2": "flushed between steps (256 MiB write)", "launch": "eager"},
            "adjoint_ms": adj_s * 1e3,
            "roofline": {"bound": "alu", "unit": "Gterm/s", "achieved": terms / adj_s / 1e9,
                         "peak": terms / floor / 1e9, "frac": floor / adj_s, "traffic": None,
                         "kernel": "k_grad_refl + k_grad_atoms (xrd_pattern_grad)",
                         "peak_basis": "SFU floor of k_grad_atoms: sin + cos + 5 exp2 per (atom, Friedel-unique "
                                       "reflection) at the MUFU rates measured in this run, %d SMs, %.0f MHz"
                                       % (roof.sms, mhz)},
            "cpu_baseline": cpu,
            "e2e": {"value": e2e_structs / e2e_max, "unit": "structures/s", "h2d_bytes_per_step": int(bytes_in),
                    "d2h_bytes_per_step": int(bytes_out), "ms_per_step": e2e_max * 1e3,
                    "api": "Handle.pattern_broadened + pattern_grad, pinned host copies each step"},
            "clocks": ck,
            "gpu_launches": GRAD_LAUNCHES * args.steps,
        }
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


def _refl_off_of(h, db, co, sz, d):
    """Friedel-unique reflection offsets of a batch (the per-reflection list of one pattern call)."""
    import torch
    from paper_2602_11709_gb300 import xrd
    out = xrd.PatternBuffers(db.n_struct, sz.n_refl, d, refl=True)
    h.pattern_batch(db, co, out, xrd.workspace(sz.ws_bytes, d))
    torch.cuda.synchronize()
    return out.refl_off.cpu().numpy()


def run_profile_calls(args):
    """--profile-calls K: K untimed xrd_pattern_batch calls on the workload (its first --subset
    structures), launch shape --sf-shape (default 128,1,1), no graph, no autotuning, no oracle: the
    program that profiler captures run. Prints the work counts of the last call."""
    import torch
    from paper_2602_11709_gb300 import xrd
    b, o = load_workload(args.workload)
    if 0 < args.subset < b.n_struct:
        b = b.subset(np.arange(args.subset))
    h = xrd.Handle(0)
    h.set_sf_shape(*[int(v) for v in (args.sf_shape or "128,1,1").split(",")])
    db = xrd.DeviceBatch.from_host(b)
    co = xrd.make_opts(o, args.precision)
    sz = h.query_sizes(db, co)
    out = xrd.PatternBuffers(b.n_struct, sz.n_refl)
    ws = xrd.workspace(sz.ws_bytes)
    for _ in range(args.profile_calls):
        h.pattern_batch(db, co, out, ws)
    torch.cuda.synchronize()
    t = h.work_counts(db, ws)
    print(json.dumps({"workload": args.workload, "n_struct": b.n_struct, "n_refl": int(sz.n_refl),
                      "calls": args.profile_calls, "terms": int(t[0]), "seeds": int(t[1]), "refined": int(t[3]),
                      "totals": [int(v) for v in out.totals.tolist()]}))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", default="fp32_phasefix", choices=["fp64", "fp32_phase64", "fp32_phasefix"])
    ap.add_argument("--fp64-steps", type=int, default=3)
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    ap.add_argument("--no-tune", action="store_true", help="skip the launch-shape autotuner")
    ap.add_argument("--sf-shape", default="", help="tile,warps,runs: set the structure-factor shape, no tuning")
    ap.add_argument("--workload", default=None, choices=sorted(WORKLOADS),
                    help="pattern path: mixed (default, the largest configuration), large, small, stress, nacl; "
                         "augmented path: small by default")
    ap.add_argument("--path", default="pattern", choices=["pattern", "augmented", "grad"],
                    help="pattern (default): the peak list of every structure; augmented: the "
                         "pseudo-Voigt / preferred-orientation / noise profile on a 4096-point grid; grad: the "
                         "broadened pattern and its gradient (512 structures, 4096 points)")
    ap.add_argument("--no-extras", action="store_true",
                    help="mixed workload: skip the large, NaCl, stress and small sub-records")
    ap.add_argument("--profile-calls", type=int, default=0,
                    help="K > 0: K untimed pattern calls (fixed --sf-shape, default 128,1,1) for profiler "
                         "captures; prints work counts instead of a bench line")
    ap.add_argument("--subset", type=int, default=0, help="with --profile-calls: the first N structures only")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.workload is None:
        args.workload = "small" if args.path == "augmented" else "mixed"
    if args.profile_calls > 0:
        run_profile_calls(args)
    elif args.path == "grad":
        run_grad(args)
    elif args.path == "augmented":
        run_augmented(args)
    elif args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()

"""Benchmark: structure-factor terms/s and patterns/s of the powder-XRD engine on GB300.

Workload: the 1024-structure small-cell batch (P1 cells, edges 3-15 A, 1-64
atoms, Cu K-alpha, 2-theta 0-90 deg), seeded and synthetic. One step = one
pass of the whole pattern path (geometry, enumeration, structure factor + LP,
sort, merge, families, cutoff, scaling, compaction) over the batch, inputs
resident in HBM. L2 is flushed (256 MiB write) between timed steps.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                  [--workload small|mixed|large] [--path pattern|augmented]
                  [--sf-shape TILE,WARPS,RUNS | --no-tune] [--no-graph]

Under torchrun (N > 1) each rank takes one shard of a batch N times larger
(weak scaling, no collective on the data path); value = all ranks' terms / max
time. `--impl reference` times the FP64 CPU oracle on the host cores instead.
`--path augmented` times xrd_pattern_augmented (pseudo-Voigt profiles,
March-Dollase orientation and noise on a 4096-point grid) on the same batch.
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
    gen = {"small": synth.small, "mixed": synth.mixed, "large": synth.large}[name]
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


# DRAM bytes (read + write) of one k_sf launch per (workload, tile, warps, runs), from one ncu
# capture of each shape (dram__bytes_read.sum + dram__bytes_write.sum, the written intensities
# stay in L2), taken before k_sf formed cos^2(theta) in FP64 above 2theta = 90 degrees. That
# change added a branch and a reload of |g|^2 for such reflections (never taken on the 0-90 degree
# workloads), so `traffic` is reported as null and this capture beside it as the prior one.
SF_TRAFFIC_BYTES_PRIOR = {("small", 64, 1, 0): 13618432, ("small", 64, 2, 0): 13618688, ("small", 64, 4, 0): 13618176,
                    ("small", 128, 1, 0): 13556224, ("small", 128, 2, 0): 13555968, ("small", 128, 4, 0): 13556224,
                    ("small", 128, 2, 1): 15159040, ("mixed", 128, 1, 0): 1243995648,
                    ("mixed", 64, 1, 0): 1247074816, ("large", 128, 1, 1): 228812544,
                    ("large", 128, 2, 1): 228943360}
# SFU issue rates per SM per clock measured on this GB300 (MUFU.SIN/COS 16, MUFU.EX2 32) and the
# maximum SM clock; the structure-factor roofline of a batch follows from its mix of operations.
MUFU_SINCOS_PER_CLK = 16.0
MUFU_EX2_PER_CLK = 32.0
# FP32 FMA-pipe operations per term of the integer-phase loop (Debye-Waller argument, weight, two
# accumulations, the four-operation rotation to the next l) and the pipe's rate per SM per clock
FMA_OPS_PER_TERM = 8.0
FMA_PER_CLK = 128.0
SM_MAX_MHZ = 2070.0


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
    per_step_budget = max(2.0, min(20.0, 100.0 / max(args.steps + args.warmup, 1)))
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
                             "sample": "consecutive 64-structure chunks of the batch, %.0f s per step" % per_step_budget},
            "e2e": {"value": tps, "unit": "terms/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_ours(args):
    import torch
    from paper_2602_11709_gb300 import synth, xrd

    rank, world, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    dev = local if torch.cuda.is_available() else 0
    torch.cuda.set_device(dev)
    b, o = load_workload(args.workload, world)
    if world > 1:  # this rank's shard of the world-times-larger batch
        lo, hi = shard_bounds(b.n_struct, rank, world)
        b = b.subset(np.arange(lo, hi))
    h = xrd.Handle(dev)
    fixed_shape = None
    if args.sf_shape:  # every call of the run, the first included, uses this shape
        fixed_shape = tuple(int(v) for v in args.sf_shape.split(","))
        h.set_sf_shape(*fixed_shape)
    db = xrd.DeviceBatch.from_host(b, "cuda:%d" % dev)
    co = xrd.make_opts(o, args.precision)
    sz = h.query_sizes(db, co)
    out = xrd.PatternBuffers(b.n_struct, sz.n_refl, "cuda:%d" % dev)
    ws = xrd.workspace(sz.ws_bytes, "cuda:%d" % dev)
    counts = np.diff(b.atom_off).astype(np.int64)
    species = np.array([len(np.unique(b.Z[b.atom_off[s]:b.atom_off[s + 1]])) for s in range(b.n_struct)])
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda:%d" % dev)
    stream = torch.cuda.current_stream()

    def barrier():
        if world > 1:
            import torch.distributed as dist
            dist.barrier()
        torch.cuda.synchronize()

    # Friedel-unique reflections per structure: half the multiplicity sum of the uncut pattern
    half = np.zeros(b.n_struct, np.int64)
    co0 = xrd.make_opts(synth.Opts(o.wavelength, o.tt_min, o.tt_max, o.tt_tol, 0.0, 0), args.precision)
    out0 = xrd.PatternBuffers(b.n_struct, sz.n_refl, "cuda:%d" % dev)
    h.pattern_batch(db, co0, out0, ws)
    torch.cuda.synchronize()
    po = out0.peak_off.cpu().numpy()
    fo = out0.fam_off.cpu().numpy()
    mult = out0.mult[: int(out0.totals[2])].cpu().numpy().astype(np.int64)
    cm = np.concatenate([[0], np.cumsum(mult)])
    for s in range(b.n_struct):
        half[s] = (cm[fo[po[s + 1]]] - cm[fo[po[s]]]) // 2 if po[s + 1] > po[s] else 0
    assert int(half.sum()) == int(sz.n_refl)
    terms_full = int((2 * half * counts).sum())
    terms_eval = int((half * counts).sum())
    # per Friedel-unique reflection and element run: f(s), four exp2
    f_cycles = float((half * species).sum()) * 4.0 / MUFU_EX2_PER_CLK

    # launch-shape tuning of the structure-factor kernel, then one CUDA graph for the whole step
    if args.sf_shape:
        tuned = fixed_shape
    else:
        tuned = h.autotune(db, co, out, ws) if not args.no_tune else None
    # timed steps carry events around the structure-factor kernel only (every event is a graph
    # node and costs time); the per-stage breakdown comes from a separate pass afterwards
    h.set_profiling(2)
    graph = h.graph(db, co, out, ws) if not args.no_graph else None

    def step():
        if graph is not None:
            graph.launch(stream)
        else:
            h.pattern_batch(db, co, out, ws)
    clocks = ClockSampler(dev)
    clocks.start()
    clocks.wait_first()
    for _ in range(args.warmup):
        flush.fill_(1.0)
        step()
    barrier()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    sf_ms = []
    barrier()
    for i in range(args.steps):
        flush.fill_(1.0)
        ev[i][0].record(stream)
        step()
        ev[i][1].record(stream)
        sf_ms.append(h.stage_times()["structure_factor"])  # synchronises on the step's SF event
    barrier()
    ck = clocks.stop()
    # per-stage breakdown (events between all stages), outside the timed region
    stage_acc = {}
    n_stage_steps = min(args.steps, 20)
    h.set_profiling(1)
    graph1 = h.graph(db, co, out, ws) if not args.no_graph else None
    for i in range(n_stage_steps):
        flush.fill_(1.0)
        if graph1 is not None:
            graph1.launch(stream)
        else:
            h.pattern_batch(db, co, out, ws)
        for k, v in h.stage_times().items():
            if k != "profile_sum":  # the augmented path's stage: not part of a pattern call
                stage_acc[k] = stage_acc.get(k, 0.0) + v
    h.set_profiling(0)
    step_ms = [a.elapsed_time(c) for a, c in ev]
    total_terms, total_structs, total_s = reduce_over_ranks(terms_full, b.n_struct, sum(step_ms) / 1e3, world,
                                                            "cuda:%d" % dev)
    value = total_terms * args.steps / total_s
    pps = total_structs * args.steps / total_s
    sf_avg = float(np.mean(sf_ms)) / 1e3
    # the kernel's own work counts: one sin/cos pair per run of consecutive reflections and atom,
    # one exp2 (Debye-Waller) per term
    w_terms, w_seeds, _ = h.work_counts(db, ws)
    assert w_terms == terms_eval, (w_terms, terms_eval)
    sfu_cycles = w_seeds * 2.0 / MUFU_SINCOS_PER_CLK + terms_eval / MUFU_EX2_PER_CLK + f_cycles
    fma_cycles = terms_eval * FMA_OPS_PER_TERM / FMA_PER_CLK
    sfu_floor_s = sfu_cycles / (152.0 * SM_MAX_MHZ * 1e6)
    peak_gterms = terms_eval / sfu_floor_s / 1e9
    achieved_gterms = terms_eval / sf_avg / 1e9

    # FP64 GPU path on the same batch (a few steps), for the FP32-vs-FP64 comparison
    extra = {}
    if args.fp64_steps > 0:
        for pname in ("fp64", "fp32_phase64"):
            cp = xrd.make_opts(o, pname)
            h.pattern_batch(db, cp, out, ws)
            torch.cuda.synchronize()
            tt = []
            for _ in range(args.fp64_steps):
                flush.fill_(1.0)
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                h.pattern_batch(db, cp, out, ws)
                e1.record(stream)
                torch.cuda.synchronize()
                tt.append(e0.elapsed_time(e1))
            ms = float(np.mean(tt))
            extra[pname] = {"ms_per_step": ms, "terms_per_s": terms_full / (ms / 1e3)}

    # end to end through the public API: pinned host inputs -> device -> pattern -> host results,
    # two batches in flight (xrd.PatternPipeline: a batch's output copies overlap the next batch)
    host = {k: torch.from_numpy(np.ascontiguousarray(getattr(b, k))).pin_memory()
            for k in ("lattice", "atom_off", "frac", "Z", "occ", "B", "coef")}
    h.set_profiling(False)
    pp = xrd.PatternPipeline(h, b, co, sz, device=dev)
    for i in range(args.warmup):
        pp.submit(host)
    res = pp.flush()
    assert int(res["totals"][3]) == 0
    torch.cuda.synchronize()
    b_in0, b_out0 = pp.bytes_in, pp.bytes_out
    t0 = time.perf_counter()
    for i in range(args.steps):
        pp.submit(host)
    res = pp.flush()
    torch.cuda.synchronize()
    e2e_total = time.perf_counter() - t0
    assert int(res["totals"][3]) == 0
    h2d = (pp.bytes_in - b_in0) // args.steps
    d2h = (pp.bytes_out - b_out0) // args.steps
    e2e_terms, _, e2e_s = reduce_over_ranks(terms_full, b.n_struct, e2e_total / args.steps, world, "cuda:%d" % dev)

    if rank == 0:
        cpu = None
        if world == 1 and args.cpu_seconds > 0:
            r = cpu_oracle_rate(b, o, budget_s=args.cpu_seconds)
            cpu = {"value": r["terms_per_s"], "unit": "terms/s", "cores": r["cores"], "kind": "oracle",
                   "sample": "%d structures of the batch (consecutive 64-structure chunks), %.1f s" %
                             (r["structures"], r["seconds"]),
                   "patterns_per_s": r["patterns_per_s"]}
        line = {
            "metric": METRIC, "value": value, "unit": "terms/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * total_s / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32 (i32 phase)" if args.precision == "fp32_phasefix"
            else args.precision, "data": "synthetic",
            "config": {"workload": WORKLOADS[args.workload], "n_struct": b.n_struct, "precision": args.precision,
                       "terms_full_sphere": terms_full, "terms_evaluated": terms_eval,
                       "reflections_friedel_unique": int(sz.n_refl), "l2": "flushed between steps (256 MiB write)",
                       "parallelism": "one structure shard per GPU" if world > 1 else "1 GPU",
                       "launch": "CUDA graph" if graph is not None else "eager",
                       "sf_shape": {"tile": tuned[0], "warps": tuned[1], "runs_in_l": tuned[2]} if tuned else "default"},
            "patterns_per_s": pps,
            "roofline": {"bound": "alu", "unit": "Gterm/s", "achieved": achieved_gterms, "peak": peak_gterms,
                         "frac": achieved_gterms / peak_gterms,
                         "traffic": None,
                         "traffic_prior_capture": SF_TRAFFIC_BYTES_PRIOR.get((args.workload,) +
                                                                             tuple(tuned or (128, 2, 0))),
                         "traffic_unit": "bytes per launch (dram read + write, ncu, this shape)",
                         "traffic_note": "k_sf changed after its last ncu capture (cos^2 theta in FP64 above "
                                         "2theta = 90 deg); traffic_prior_capture is the earlier kernel's",
                         "fma_floor_frac": (fma_cycles / (152.0 * SM_MAX_MHZ * 1e6)) / sf_avg,
                         "phase_seeds_per_term": w_seeds / max(terms_eval, 1),
                         "kernel": "k_sf", "peak_basis": "SFU: sin+cos at 16/clk/SM per phase seed (one per run of "
                                                         "consecutive l and atom), exp2 at 32/clk/SM, "
                                                         "152 SMs, 2070 MHz; Friedel-unique terms"},
            "cpu_baseline": cpu,
            "e2e": {"value": e2e_terms / e2e_s, "unit": "terms/s", "h2d_bytes_per_step": int(h2d),
                    "d2h_bytes_per_step": int(d2h), "ms_per_step": e2e_s * 1e3,
                    "api": "xrd.PatternPipeline, two batches in flight"},
            "clocks": ck,
            "gpu_launches": xrd.launches_per_batch(b.n_struct) * args.steps,
            "stage_ms": {k: v / n_stage_steps for k, v in stage_acc.items()},
            "stage_ms_note": "separate pass with events between all stages (adds time per stage)",
            "other_precisions": extra,
        }
        if "fp64" in extra:
            line["speedup_vs_fp64_gpu"] = extra["fp64"]["ms_per_step"] / (1e3 * total_s / args.steps)
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


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", default="fp32_phasefix", choices=["fp64", "fp32_phase64", "fp32_phasefix"])
    ap.add_argument("--fp64-steps", type=int, default=3)
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    ap.add_argument("--no-graph", action="store_true", help="launch the step eagerly instead of as a CUDA graph")
    ap.add_argument("--no-tune", action="store_true", help="skip the launch-shape autotuner")
    ap.add_argument("--sf-shape", default="", help="tile,warps,runs: set the structure-factor shape, no tuning")
    ap.add_argument("--workload", default="small", choices=sorted(WORKLOADS),
                    help="small (default, the benchmark configuration), mixed or large")
    ap.add_argument("--path", default="pattern", choices=["pattern", "augmented"],
                    help="pattern (default): the peak list of every structure; augmented: the "
                         "pseudo-Voigt / preferred-orientation / noise profile on a 4096-point grid")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.path == "augmented":
        run_augmented(args)
    elif args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()

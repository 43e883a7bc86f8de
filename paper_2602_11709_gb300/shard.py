"""Structure sharding across ranks (one process per GPU) and the gather of their results.

Structures are independent, so a batch splits into per-rank sub-batches and
nothing is exchanged on the data path. The cost of a structure is its
structure-factor work, R x N (Friedel-unique reflections, from
xrd_reflection_counts, times atoms; an atom-free structure counts R for its
post-processing). `partition` assigns structures by longest processing time
first: in decreasing cost, each to the rank with the smallest load so far,
which keeps the largest load within 4/3 of the best possible (Graham's bound)
and, for many small structures, within a fraction of a percent of the mean.

After each rank has computed its patterns, `gather_patterns` collects the
ranks' dense CSR blocks (the layout of xrd_pattern: peak offsets, per-peak
2-theta, intensity, d, family offsets, per-family hkl and multiplicity, and a
status per structure) and reassembles them in the batch's structure order, so
that the result is the one a single rank would have produced.
"""
from __future__ import annotations

import heapq

import numpy as np

CSR_KEYS = ("two_theta", "intensity", "d_hkl")  # per-peak arrays
FAM_KEYS = ("hkl", "mult")                      # per-family arrays


def costs(refl_counts, atom_counts) -> np.ndarray:
    """Structure-factor cost of every structure: reflections x atoms (at least the reflections)."""
    R = np.asarray(refl_counts, dtype=np.int64)
    N = np.asarray(atom_counts, dtype=np.int64)
    return R * np.maximum(N, 1)


def partition(cost, world: int) -> list[np.ndarray]:
    """Structure indices of each rank (ascending within a rank): longest processing time first."""
    cost = np.asarray(cost, dtype=np.int64)
    if world < 1:
        raise ValueError("world must be >= 1")
    order = np.argsort(-cost, kind="stable")
    heap = [(0, r) for r in range(world)]
    owner = np.empty(len(cost), dtype=np.int64)
    for s in order:
        load, r = heapq.heappop(heap)
        owner[s] = r
        heapq.heappush(heap, (load + int(cost[s]), r))
    return [np.nonzero(owner == r)[0] for r in range(world)]


def loads(cost, parts) -> np.ndarray:
    cost = np.asarray(cost, dtype=np.int64)
    return np.array([int(cost[p].sum()) for p in parts], dtype=np.int64)


def assemble(blocks, parts, n_total: int) -> dict:
    """The whole batch's CSR arrays from per-rank blocks; blocks[r] covers structures parts[r] in that
    order, with keys peak_off [n_r + 1], fam_off [peaks_r + 1], status [n_r] and the per-peak and
    per-family arrays."""
    owner = np.full(n_total, -1, dtype=np.int64)
    local = np.zeros(n_total, dtype=np.int64)
    for r, p in enumerate(parts):
        owner[p] = r
        local[p] = np.arange(len(p))
    if n_total and owner.min() < 0:
        raise ValueError("parts do not cover the batch")
    npk = np.zeros(n_total, dtype=np.int64)
    nfm = np.zeros(n_total, dtype=np.int64)
    for s in range(n_total):
        blk, i = blocks[owner[s]], local[s]
        po, fo = blk["peak_off"], blk["fam_off"]
        npk[s] = po[i + 1] - po[i]
        nfm[s] = fo[po[i + 1]] - fo[po[i]]
    peak_off = np.zeros(n_total + 1, dtype=np.int64)
    peak_off[1:] = np.cumsum(npk)
    P = int(peak_off[-1])
    F = int(nfm.sum())
    out = {"peak_off": peak_off, "fam_off": np.zeros(P + 1, dtype=np.int64),
           "status": np.zeros(n_total, dtype=np.int32)}
    for k in CSR_KEYS:
        out[k] = np.zeros(P, dtype=blocks[0][k].dtype if blocks else np.float64)
    out["hkl"] = np.zeros((F, 3), dtype=np.int32)
    out["mult"] = np.zeros(F, dtype=np.int32)
    f_at = 0
    for s in range(n_total):
        blk, i = blocks[owner[s]], local[s]
        po, fo = blk["peak_off"], blk["fam_off"]
        p0, p1 = int(po[i]), int(po[i + 1])
        q0 = int(peak_off[s])
        for k in CSR_KEYS:
            out[k][q0:q0 + p1 - p0] = blk[k][p0:p1]
        f0, f1 = int(fo[p0]), int(fo[p1])
        out["fam_off"][q0:q0 + p1 - p0] = fo[p0:p1] - f0 + f_at
        out["hkl"][f_at:f_at + f1 - f0] = blk["hkl"][f0:f1]
        out["mult"][f_at:f_at + f1 - f0] = blk["mult"][f0:f1]
        out["status"][s] = blk["status"][i]
        f_at += f1 - f0
    out["fam_off"][P] = f_at
    return out


def gather_patterns(block: dict, parts, n_total: int, group=None, dst: int = 0):
    """Collect every rank's block (torch.distributed, any backend) and assemble them on rank dst;
    other ranks get None. The blocks travel as pickled numpy arrays (gather_object)."""
    import torch.distributed as dist
    world = dist.get_world_size(group)
    rank = dist.get_rank(group)
    got = [None] * world if rank == dst else None
    dist.gather_object({k: np.asarray(v) for k, v in block.items()}, got, dst=dst, group=group)
    if rank != dst:
        return None
    return assemble(got, parts, n_total)

"""The N > 1 path on CPU ranks (gloo, world size 2).

Structures are independent: each rank takes a cost-balanced share of the
batch (longest processing time first on reflections x atoms, with the
reflection counts of the enumeration) and nothing is exchanged on the data
path. After the patterns, the ranks' CSR blocks are gathered and reassembled
in the batch's order. The measurement sums terms and structures over ranks and
takes the time of the slowest rank. Each rank here computes with the oracle
(no GPU); what is tested is the partition, the gather and the reduction.
"""
import os
import socket

import numpy as np
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _terms(b, o):
    import oracle
    total = 0
    for s in range(b.n_struct):
        hkl, _ = oracle.enumerate_refl(b.lattice[s], o)  # full sphere: every reflection and its mate
        total += (len(hkl) // 2) * int(b.atom_off[s + 1] - b.atom_off[s])
    return total


def _worker(rank, world, port, out):
    import sys
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    import torch.distributed as dist
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import bench
        from paper_2602_11709_gb300 import synth
        b, o = synth.small(n=12 * world)
        lo, hi = bench.shard_bounds(b.n_struct, rank, world)
        mine = b.subset(np.arange(lo, hi))
        terms = _terms(mine, o)
        seconds = 1.0 + rank  # rank 1 is the slow one
        tot = bench.reduce_over_ranks(terms, mine.n_struct, seconds, world)
        out.put((rank, lo, hi, terms, tot))
    finally:
        dist.destroy_process_group()


def test_shards_cover_the_batch_without_overlap():
    import sys
    sys.path.insert(0, ROOT)
    import bench
    for n in (0, 1, 5, 1024, 100_001):
        for world in (1, 2, 3, 8):
            spans = [bench.shard_bounds(n, r, world) for r in range(world)]
            assert spans[0][0] == 0 and spans[-1][1] == n
            assert all(spans[i][1] == spans[i + 1][0] for i in range(world - 1))
            sizes = [e - s for s, e in spans]
            assert max(sizes) - min(sizes) <= 1


def test_weak_scaling_batch_is_world_times_larger():
    import sys
    sys.path.insert(0, ROOT)
    import bench
    b1, _ = bench.load_workload("small", 1)
    b2, _ = bench.load_workload("small", 2)
    assert b2.n_struct == 2 * b1.n_struct


def test_two_gloo_ranks_sum_terms_and_take_the_slowest_time():
    import sys
    sys.path.insert(0, ROOT)
    from paper_2602_11709_gb300 import synth
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.SimpleQueue()
    mp.start_processes(_worker, args=(world, _free_port(), q), nprocs=world, join=True, start_method="spawn")
    res = sorted(q.get() for _ in range(world))
    b, o = synth.small(n=12 * world)
    assert [r[1] for r in res] == [0, 12] and [r[2] for r in res] == [12, 24]
    whole = _terms(b, o)
    assert sum(r[3] for r in res) == whole
    for _, _, _, _, (terms, structs, seconds) in res:
        assert terms == whole and structs == b.n_struct and seconds == 2.0


def _flat(res):
    """Per-structure result lists (oracle.pattern_batch layout) -> one CSR block (xrd_pattern layout)."""
    n = len(res["peak_tt"])
    npk = np.array([len(x) for x in res["peak_tt"]], np.int64)
    po = np.zeros(n + 1, np.int64)
    po[1:] = np.cumsum(npk)
    fo, f_at = [], 0
    for s in range(n):
        fo.append(res["peak_fam_off"][s][:-1] + f_at)
        f_at += int(res["peak_fam_off"][s][-1])
    cat = lambda k, shape: np.concatenate(res[k]) if n and sum(len(x) for x in res[k]) else np.zeros(shape)  # noqa
    return {"peak_off": po, "two_theta": cat("peak_tt", 0), "intensity": cat("peak_I", 0), "d_hkl": cat("peak_d", 0),
            "fam_off": np.concatenate(fo + [np.array([f_at], np.int64)]).astype(np.int64),
            "hkl": cat("fam_hkl", (0, 3)).astype(np.int32), "mult": cat("fam_mult", 0).astype(np.int32),
            "status": np.asarray(res["status"], np.int32)}


def test_partition_balances_real_reflection_counts():
    """LPT over reflections x atoms of the 100 000-structure mixed batch (reflection counts from the
    enumeration): every structure on exactly one rank, the largest load within 1.05 of the mean."""
    import sys
    sys.path.insert(0, ROOT)
    import oracle
    from paper_2602_11709_gb300 import shard, synth
    b, o = synth.mixed()
    cost = shard.costs(oracle.refl_counts(b, o) // 2, np.diff(b.atom_off))
    for world in (1, 2, 4, 8):
        parts = shard.partition(cost, world)
        allidx = np.sort(np.concatenate(parts))
        assert np.array_equal(allidx, np.arange(b.n_struct))
        load = shard.loads(cost, parts)
        assert load.sum() == cost.sum()
        assert load.max() <= 1.05 * load.mean(), (world, load)
    # a few dominant structures: LPT reaches the optimum here (largest load 105 of 206 in all)
    few = np.array([100, 90, 5, 5, 5, 1], np.int64)
    parts = shard.partition(few, 2)
    assert sorted(shard.loads(few, parts).tolist()) == [101, 105]


def _gather_worker(rank, world, port, out):
    import sys
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    import torch.distributed as dist
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import oracle
        from paper_2602_11709_gb300 import shard, synth
        b, o = synth.small(n=160)
        parts = shard.partition(shard.costs(oracle.refl_counts(b, o, threads=1) // 2, np.diff(b.atom_off)), world)
        mine = b.subset(parts[rank])
        block = _flat(oracle.pattern_batch(mine, o, threads=1))
        whole = shard.gather_patterns(block, parts, b.n_struct)
        out.put((rank, len(parts[rank]), None if whole is None else {k: v.tolist() for k, v in whole.items()}))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_gather_the_single_rank_result():
    """Two ranks, each with its LPT share of 160 structures; the gathered CSR arrays equal a single
    rank's result for the whole batch, element for element."""
    import sys
    sys.path.insert(0, ROOT)
    import oracle
    from paper_2602_11709_gb300 import synth
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.SimpleQueue()
    pc = mp.start_processes(_gather_worker, args=(world, _free_port(), q), nprocs=world, join=False,
                            start_method="spawn")
    res = sorted((q.get() for _ in range(world)), key=lambda r: r[0])  # read before joining: the result is large
    while not pc.join():
        pass
    assert res[1][2] is None and res[0][1] + res[1][1] == 160 and min(res[0][1], res[1][1]) > 40
    b, o = synth.small(n=160)
    ref = _flat(oracle.pattern_batch(b, o, threads=1))
    got = res[0][2]
    for k, v in ref.items():
        assert np.array_equal(np.asarray(got[k]).reshape(np.shape(v)), v), k

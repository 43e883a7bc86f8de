"""The N > 1 path of bench.py on CPU ranks (gloo, world size 2).

Structures are independent, so ranks take contiguous shards of a batch
world times the single-GPU size and exchange nothing on the data path; the
only cross-rank step is the measurement: terms and structures summed over
ranks, the time of the slowest rank. Each rank here computes its shard's
Friedel-unique terms with the oracle (no GPU) and a rank-dependent time.
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

"""World-size-2 checks (gloo, CPU) of the multi-GPU host logic: the
per-rank zoom-prefix shards cover every bin exactly once, the merged top
bins of the shards equal the top bins of the whole output, and the timing
reduction takes the slowest rank."""
import os
import socket

import numpy as np
import pytest

import oracle as O
from paper_2207_00933_gb300 import parallel


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, q):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        rng = np.random.default_rng(3)
        P = rng.random(1 << 12)                       # the whole output (all ranks know it here)
        P[rng.integers(0, P.size, 50)] = 0.5          # ties across shards
        # shard by a zoom prefix on the lowest active qubit(s): rank r owns bins b with b's low bits == r
        bits = parallel.shard_prefix(rank, world)
        p = len(bits)
        mine = np.nonzero((np.arange(P.size) & ((1 << p) - 1)) == rank)[0]
        lb, lv = O.top_bins(P[mine], 37)
        gb, gv = parallel.merge_top_bins(mine[lb], lv, 37)
        eb, ev = O.top_bins(P, 37)
        slow = parallel.max_over_ranks(1.0 + rank)
        q.put((rank, gb.tolist() == eb.tolist() and np.array_equal(gv, ev), slow, len(mine)))
    finally:
        dist.destroy_process_group()


def test_two_rank_shards_merge_to_the_global_top_bins():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert all(ok for _, ok, _, _ in res)
    assert all(slow == 2.0 for _, _, slow, _ in res)
    assert sum(n for _, _, _, n in res) == 1 << 12


def test_shard_prefix():
    assert parallel.shard_prefix(0, 1) == []
    assert parallel.shard_prefix(3, 4) == [1, 1]
    with pytest.raises(ValueError):
        parallel.shard_prefix(0, 3)

"""World-size-2 checks (gloo, CPU) of the multi-GPU host logic: the
per-rank zoom-prefix shards cover every bin exactly once, the merged top
bins of the shards equal the top bins of the whole output, and the timing
reduction takes the slowest rank.  One case shards a real reconstruction:
each rank zooms the query's lowest active qubit to its rank (Algorithm 2's
zoom role, computed by the oracle), and the shards together are the whole
query's bins."""
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


def _shard_worker(rank, world, port, q):
    """Rank `rank` reconstructs its zoom-prefix shard of a real cut circuit
    (the lowest active qubits zoomed to the rank's bits, Algorithm 2's
    zoom role) and the ranks merge their selected bins."""
    import torch.distributed as dist
    from synthetic import workloads as W
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        w = W.small_random(5, n_qubits=9, roles="active")
        c = w.circuit
        g = O.Graph.from_arrays(c.n_qubits, *c.graph_arrays())
        act = np.nonzero(np.asarray(w.roles) == 0)[0]
        bits = parallel.shard_prefix(rank, world)
        roles = np.array(w.roles, dtype=np.int8)
        for j, bit in enumerate(bits):
            roles[act[j]] = 3 if bit else 2           # zoom1 / zoom0
        Pr = O.reconstruct(g, w.probs, roles)
        p = len(bits)
        glob = (np.arange(Pr.size, dtype=np.int64) << p) | rank
        lb, lv = O.top_bins(Pr, 20)
        gb, gv = parallel.merge_top_bins(glob[lb], lv, 20)
        q.put((rank, glob.tolist(), Pr.tolist(), gb.tolist(), gv.tolist()))
    finally:
        dist.destroy_process_group()


def test_zoom_prefix_shards_of_a_reconstruction():
    """Two ranks, each owning the bins whose lowest active qubit equals its
    rank: the shards are exactly the whole query's bins, and the merged top
    bins of the shards are the whole query's top bins."""
    import torch.multiprocessing as mp
    from synthetic import workloads as W
    w = W.small_random(5, n_qubits=9, roles="active")
    c = w.circuit
    P = O.reconstruct(O.Graph.from_arrays(c.n_qubits, *c.graph_arrays()), w.probs, w.roles)
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_shard_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    whole = np.full(P.size, np.nan)
    for _, glob, Pr, _, _ in res:
        whole[np.asarray(glob)] = Pr
    assert not np.isnan(whole).any()
    np.testing.assert_allclose(whole, P, rtol=0, atol=1e-14)
    eb, ev = O.top_bins(P, 20)
    for _, _, _, gb, gv in res:
        np.testing.assert_allclose(gv, ev, rtol=0, atol=1e-14)
        # every bin clearly above the k-th value is selected (bins tied with
        # it within the shards' rounding may be exchanged for one another)
        sure = set(np.nonzero(P > ev[-1] + 1e-13)[0].tolist())
        assert sure <= set(gb), sorted(sure - set(gb))

"""GPU: the continuous-batching serving loop.  Zoom queries against resident
circuits (forests of chains, up to hundreds of qubits) are submitted in a
burst and in a stream; every result must equal the same query reconstructed
alone (bit for bit: a bin is summed by one thread in the same order either
way), and sampled results must match the FP64 oracle.  A small HBM budget
forces admission to hold requests back until launches retire."""
import time

import numpy as np
import pytest

import oracle as O
from synthetic import workloads as W

pytestmark = pytest.mark.gpu


def _workload():
    return W.serving_set(seed=8, n_circuits=3, n_queries=48, n_qubit_range=(100, 400), n_sub_range=(10, 30),
                         K_range=(6, 30))


def _load(ctx, b):
    import torch
    return [ctx.load_subcircuit_outputs(c.n_qubits, *c.graph_arrays(), [torch.from_numpy(p).cuda() for p in ps])
            for c, ps in zip(b.circuits, b.probs)]


def _alone(ctx, cids, b):
    import torch
    res = []
    for ci, roles in b.queries:
        q, na = ctx.set_qubit_roles(cids[ci], roles)
        out = torch.empty(1 << na, dtype=torch.float32, device="cuda")
        ctx.reconstruct(q, out, "fp32")
        res.append(out.cpu().numpy())
        ctx.release_query(q)
    return res


@pytest.mark.parametrize("mode", ["batched", "plain"])
def test_served_results_equal_alone(mode):
    from paper_2207_00933_gb300 import Context, Server, _build
    _build.build()
    b = _workload()
    ctx = Context(0)
    cids = _load(ctx, b)
    alone = _alone(ctx, cids, b)
    with Server(ctx, max_batch=16, n_streams=3, plain=(mode == "plain")) as srv:
        tickets = [srv.submit(cids[ci], roles) for ci, roles in b.queries[:24]]      # burst
        for ci, roles in b.queries[24:]:                                              # stream
            tickets.append(srv.submit(cids[ci], roles))
            time.sleep(0.0005)
        srv.drain(120.0)
        lat = []
        for j, t in enumerate(tickets):
            state, us, na = srv.poll(t)
            assert state == 2 and us > 0
            lat.append(us)
            assert np.array_equal(srv.result(t), alone[j]), j
        st = srv.stats()
        assert st["admitted"] == len(tickets)
        if mode == "batched":
            assert st["launches"] < len(tickets)            # requests shared launches
    ctx.close()


def test_every_served_query_matches_the_oracle():
    # all 48 queries (forests of chains of 100-400 qubits, zoom prefixes,
    # 12-20 active qubits) through the batching server, each against the
    # FP64 oracle
    from paper_2207_00933_gb300 import Context, Server, _build
    _build.build()
    b = _workload()
    graphs = [O.Graph.from_arrays(c.n_qubits, *c.graph_arrays()) for c in b.circuits]
    probs64 = [[p.astype(np.float64) for p in ps] for ps in b.probs]
    with Context(0) as ctx:
        cids = _load(ctx, b)
        with Server(ctx, max_batch=16, n_streams=3) as srv:
            tickets = [srv.submit(cids[ci], roles) for ci, roles in b.queries]
            srv.drain(120.0)
            for j, t in enumerate(tickets):
                ci, roles = b.queries[j]
                state, _, na = srv.poll(t)
                assert state == 2
                P = srv.result(t).astype(np.float64)
                ref = O.reconstruct(graphs[ci], probs64[ci], roles)
                assert P.size == ref.size == 1 << na
                err = np.abs(P - ref).max()
                assert err <= 1e-6 and err <= 1e-5 * np.abs(ref).max() + 1e-15, (j, err)


def test_admission_by_hbm_footprint():
    from paper_2207_00933_gb300 import Context, Server
    b = _workload()
    probe = Context(0)
    cids = _load(probe, b)
    alone = _alone(probe, cids, b)
    resident = probe.memory_info()["held"]
    per_query = 0
    for ci, roles in b.queries:
        before = probe.memory_info()["held"]
        q, na = probe.set_qubit_roles(cids[ci], roles)
        per_query = max(per_query, probe.memory_info()["held"] - before + (4 << na) + (1 << 20))
        probe.release_query(q)
    probe.close()
    # room for the resident circuits plus only a few queries in flight
    ctx = Context(0, hbm_budget_bytes=int(resident + 3 * per_query))
    cids = _load(ctx, b)
    with Server(ctx, max_batch=64, n_streams=4) as srv:
        tickets = [srv.submit(cids[ci], roles) for ci, roles in b.queries]
        srv.drain(60.0)
        for j, t in enumerate(tickets):
            assert np.array_equal(srv.result(t), alone[j]), j
        assert srv.stats()["busy_refusals"] > 0


def test_request_larger_than_budget_fails():
    from paper_2207_00933_gb300 import Context, SQCError, Server
    b = _workload()
    probe = Context(0)
    _load(probe, b)
    resident = probe.memory_info()["held"]
    probe.close()
    ctx = Context(0, hbm_budget_bytes=resident + (2 << 20))
    cids = _load(ctx, b)
    c = b.circuits[0]
    big = np.full(c.n_qubits, O.MERGED, dtype=np.int8)
    big[:20] = O.ACTIVE                                   # 4 MB of bins: more than the 2 MB left
    small = np.full(c.n_qubits, O.MERGED, dtype=np.int8)
    for dq in c.data_qubits[:4]:
        small[dq[0]] = O.ACTIVE
    with Server(ctx, max_batch=8, n_streams=2) as srv:
        t_big = srv.submit(cids[0], big)
        t_small = srv.submit(cids[0], small)
        srv.drain(60.0)
        with pytest.raises(SQCError) as ei:
            srv.poll(t_big)
        assert ei.value.status == 6                       # SQC_EBUSY
        assert srv.poll(t_small)[0] == 2
    ctx.close()

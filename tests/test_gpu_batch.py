"""GPU: the batched recursion level -- many zoom queries over several
resident circuits in one persistent launch -- against the FP64 oracle and
against the same queries run one at a time (which must give the very same
bins: every bin is summed by one thread in the same order either way)."""
import numpy as np
import pytest

import oracle as O
from synthetic import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def setup():
    import torch
    from paper_2207_00933_gb300 import Context, _build
    _build.build()
    ctx = Context(0)
    b = W.batch_level(seed=5, n_circuits=3, n_queries=24, a_range=(6, 12), max_log_input=18, min_qubits=30)
    cids = [ctx.load_subcircuit_outputs(c.n_qubits, *c.graph_arrays(), [torch.from_numpy(p).cuda() for p in ps])
            for c, ps in zip(b.circuits, b.probs)]
    qs = [ctx.set_qubit_roles(cids[ci], roles) for ci, roles in b.queries]
    yield ctx, b, qs
    torch.cuda.synchronize()
    ctx.close()


def _oracle(b, j):
    ci, roles = b.queries[j]
    c = b.circuits[ci]
    g = O.Graph.from_arrays(c.n_qubits, *c.graph_arrays())
    return O.reconstruct(g, [p.astype(np.float64) for p in b.probs[ci]], roles)


def test_batch_matches_oracle_and_single_queries(setup):
    import torch
    ctx, b, qs = setup
    outs = [torch.full((1 << na,), -1.0, dtype=torch.float32, device="cuda") for _, na in qs]
    totals = torch.zeros(len(qs), dtype=torch.float64, device="cuda")
    bid = ctx.batch_create([q for q, _ in qs], outs, totals)
    for _ in range(2):                              # the launch re-arms itself
        ctx.batch_run(bid)
    ctx.batch_status(bid)
    for j, (q, na) in enumerate(qs):
        ref = _oracle(b, j)
        P = outs[j].double().cpu().numpy()
        err = np.abs(P - ref).max()
        assert err <= 1e-6 and err <= 1e-5 * np.abs(ref).max() + 1e-15, (j, err)
        single = torch.empty_like(outs[j])
        tot1 = torch.zeros(1, dtype=torch.float64, device="cuda")
        ctx.reconstruct(q, single, "fp32", tot1)
        torch.cuda.synchronize()
        assert torch.equal(single, outs[j]), j
        assert abs(tot1.item() - totals[j].item()) <= 1e-12 * max(1.0, abs(tot1.item())) + 1e-15
    ctx.batch_release(bid)


def test_batch_replays_from_a_cuda_graph(setup):
    import torch
    ctx, b, qs = setup
    outs = [torch.zeros((1 << na,), dtype=torch.float64, device="cuda") for _, na in qs]
    bid = ctx.batch_create([q for q, _ in qs], outs)
    ctx.batch_run(bid)
    torch.cuda.synchronize()
    first = [o.clone() for o in outs]
    for o in outs:
        o.zero_()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        ctx.batch_run(bid)
    for _ in range(3):
        g.replay()
    torch.cuda.synchronize()
    ctx.batch_status(bid)
    for o, f in zip(outs, first):
        assert torch.equal(o, f)
    ctx.batch_release(bid)


def test_autotune_policies_give_the_same_bins(setup):
    """sqc_batch_autotune times the two contraction orders x the three tile
    policies; under the chosen order every policy sums each bin in the same
    order, so the bins equal the one-at-a-time runs (planned under that
    order) bit for bit, and match the oracle."""
    import torch
    ctx, b, qs = setup
    outs = [torch.full((1 << na,), -1.0, dtype=torch.float32, device="cuda") for _, na in qs]
    totals = torch.zeros(len(qs), dtype=torch.float64, device="cuda")
    best, order, ms = ctx.batch_autotune([q for q, _ in qs], outs, totals, reps=3)
    assert best in (0, 1, 2) and order in (0, 1)
    flat = ms[0] + ms[1]
    assert all(t > 0 for t in flat) and ms[order][best] == min(flat)
    after_tune = [o.clone() for o in outs]
    for o in outs:
        o.fill_(-1.0)
    bid = ctx.batch_create([q for q, _ in qs], outs, totals)     # built under the chosen policy
    ctx.batch_run(bid)
    ctx.batch_status(bid)
    for j, (q, na) in enumerate(qs):
        single = torch.empty_like(outs[j])
        tot1 = torch.zeros(1, dtype=torch.float64, device="cuda")
        ctx.reconstruct(q, single, "fp32", tot1)
        torch.cuda.synchronize()
        assert torch.equal(single, outs[j]), j
        assert torch.equal(single, after_tune[j]), j
        assert abs(tot1.item() - totals[j].item()) <= 1e-12 * max(1.0, abs(tot1.item())) + 1e-15
        ref = _oracle(b, j)
        err = np.abs(outs[j].double().cpu().numpy() - ref).max()
        assert err <= 1e-6 and err <= 1e-5 * np.abs(ref).max() + 1e-15, (j, err)
    ctx.batch_release(bid)


def test_query_autotune_keeps_the_faster_order():
    """sqc_query_autotune times a query under the greedy and the
    fewest-multiplications order and keeps the faster plan; both orders
    reconstruct the oracle's bins, and the kept plan is the one later calls
    run (same bins as the last timed run of that order)."""
    import torch
    from paper_2207_00933_gb300 import Context
    b = W.batch_level(seed=5, n_circuits=3, n_queries=6, a_range=(8, 12), max_log_input=18, min_qubits=30)
    with Context(0) as ctx:
        cids = [ctx.load_subcircuit_outputs(c.n_qubits, *c.graph_arrays(), [torch.from_numpy(p).cuda() for p in ps])
                for c, ps in zip(b.circuits, b.probs)]
        for j, (ci, roles) in enumerate(b.queries):
            q, na = ctx.set_qubit_roles(cids[ci], roles)
            res = {}
            for order in (0, 1):
                with Context(0, contraction_order=order) as c2:
                    cc = b.circuits[ci]
                    cid2 = c2.load_subcircuit_outputs(cc.n_qubits, *cc.graph_arrays(),
                                                      [torch.from_numpy(p).cuda() for p in b.probs[ci]])
                    q2, _ = c2.set_qubit_roles(cid2, roles)
                    o2 = torch.empty(1 << na, dtype=torch.float32, device="cuda")
                    c2.reconstruct(q2, o2)
                    torch.cuda.synchronize()
                    res[order] = o2.cpu()
            out = torch.empty(1 << na, dtype=torch.float32, device="cuda")
            best, ms = ctx.query_autotune(q, out, reps=3)
            assert best in (0, 1) and all(t > 0 for t in ms)
            ctx.reconstruct(q, out)
            torch.cuda.synchronize()
            assert torch.equal(out.cpu(), res[best]), j
            ref = _oracle(b, j)
            for order in (0, 1):
                err = np.abs(res[order].double().numpy() - ref).max()
                assert err <= 1e-6 and err <= 1e-5 * np.abs(ref).max() + 1e-15, (j, order, err)


def test_autotune_rejects_bad_arguments(setup):
    import torch
    from paper_2207_00933_gb300 import SQCError
    ctx, b, qs = setup
    outs = [torch.zeros((1 << na,), dtype=torch.float32, device="cuda") for _, na in qs]
    with pytest.raises(SQCError):
        ctx.batch_autotune([q for q, _ in qs], outs, reps=0)


def test_batch_chunked_fp64_last_step():
    """FP64 outputs with the cross-chunk sum on (Section 6.3): every query's
    last step sums its shared index in FP32 chunks of 16 terms added in
    FP64 (4 chunks where the last step shares 3 cut edges).  Each batched
    query equals its single run bit for bit and the FP64 oracle within
    1e-6."""
    import torch
    from paper_2207_00933_gb300 import Context
    b = W.batch_level(seed=5, n_circuits=3, n_queries=24, a_range=(6, 12), max_log_input=18, min_qubits=30)
    assert all(c.n_edges >= 10 for c in b.circuits)
    with Context(0, fp64_chunk_min_edges=10, chunk_terms=16) as ctx:
        cids = [ctx.load_subcircuit_outputs(c.n_qubits, *c.graph_arrays(),
                                            [torch.from_numpy(p).cuda() for p in ps])
                for c, ps in zip(b.circuits, b.probs)]
        qs = [ctx.set_qubit_roles(cids[ci], roles) for ci, roles in b.queries]
        kd = [ctx.query_steps(q)[-1][2] for q, _ in qs]
        assert sum(k > 16 for k in kd) >= 4            # several last steps of 2 or more chunks
        outs = [torch.full((1 << na,), -1.0, dtype=torch.float64, device="cuda") for _, na in qs]
        totals = torch.zeros(len(qs), dtype=torch.float64, device="cuda")
        bid = ctx.batch_create([q for q, _ in qs], outs, totals)
        ctx.batch_run(bid)
        ctx.batch_status(bid)
        for j, (q, na) in enumerate(qs):
            ref = _oracle(b, j)
            P = outs[j].cpu().numpy()
            err = np.abs(P - ref).max()
            assert err <= 1e-6 and err <= 1e-5 * np.abs(ref).max() + 1e-15, (j, err)
            single = torch.empty_like(outs[j])
            tot1 = torch.zeros(1, dtype=torch.float64, device="cuda")
            ctx.reconstruct(q, single, "fp32", tot1)
            torch.cuda.synchronize()
            assert torch.equal(single, outs[j]), j
            assert abs(tot1.item() - totals[j].item()) <= 1e-12 * max(1.0, abs(tot1.item()))
        ctx.batch_release(bid)


def test_bounded_wait_runs_out_and_the_context_recovers():
    """Failure detection: the host raises the completion target of one
    intermediate tensor beyond what its producers deliver, so the items that
    read it wait until the bounded wait (50 ms here) runs out.  The launch
    must end by itself, report SQC_ETIMEOUT, and leave the context usable:
    the restored batch then gives the same bins as the single runs."""
    import time
    import torch
    from paper_2207_00933_gb300 import Context, SQCError
    b = W.batch_level(seed=5, n_circuits=3, n_queries=12, a_range=(6, 12), max_log_input=18, min_qubits=30)
    with Context(0, wait_limit_ms=50) as ctx:
        cids = [ctx.load_subcircuit_outputs(c.n_qubits, *c.graph_arrays(),
                                            [torch.from_numpy(p).cuda() for p in ps])
                for c, ps in zip(b.circuits, b.probs)]
        qs = [ctx.set_qubit_roles(cids[ci], roles) for ci, roles in b.queries]
        outs = [torch.zeros((1 << na,), dtype=torch.float32, device="cuda") for _, na in qs]
        bid = ctx.batch_create([q for q, _ in qs], outs)
        ctx.batch_inject_stall(bid, True)
        t0 = time.perf_counter()
        ctx.batch_run(bid)
        with pytest.raises(SQCError) as ei:
            ctx.batch_status(bid)                      # synchronises: the kernel has returned
        assert ei.value.status == 5                    # SQC_ETIMEOUT
        assert time.perf_counter() - t0 < 30.0
        ctx.batch_inject_stall(bid, False)
        ctx.batch_run(bid)
        ctx.batch_status(bid)                          # no error left behind
        for j, (q, na) in enumerate(qs):
            single = torch.empty_like(outs[j])
            ctx.reconstruct(q, single, "fp32")
            torch.cuda.synchronize()
            assert torch.equal(single, outs[j]), j
        ctx.batch_release(bid)


def test_split_bf16_batch_matches_single_split_runs():
    """The batched level in split-BF16: each query's tensor-core steps run as
    tcgen05 launches between the persistent phases (here a SIMT step
    produces the BF16-plane operand of a tensor-core last step in two of the
    circuits), the other steps FP32 in the persistent launch.  Every batched
    query equals its own split-BF16 reconstruction bit for bit (same plan,
    same kernels, same summation order) and the FP64 oracle within 1e-6."""
    import torch
    from paper_2207_00933_gb300 import Context
    big = [W.random_line_chain(17, [8, 11, 11], [2, 4], 1, [4, 7, 7]),
           W.random_line_chain(18, [7, 10, 11], [2, 4], 1, [5, 6, 7]),
           W.random_line_chain(20, [12, 12], [4], 1, [7, 7])]
    small = W.batch_level(seed=5, n_circuits=2, n_queries=6, a_range=(6, 10), max_log_input=16, min_qubits=24)
    with Context(0) as ctx:
        entries = []     # (qid, na, circuit, probs, roles)
        for w in big:
            c = w.circuit
            cid = ctx.load_subcircuit_outputs(c.n_qubits, *c.graph_arrays(), [torch.from_numpy(p).cuda() for p in w.probs])
            roles2 = w.roles.copy()
            mq = next(q for q in range(c.n_qubits) if roles2[q] == O.MERGED)
            roles2[mq] = O.ZOOM1                              # a zoomed variant of the same shape
            for r in (w.roles, roles2):
                q, na = ctx.set_qubit_roles(cid, r)
                entries.append((q, na, c, w.probs, r))
        cids = [ctx.load_subcircuit_outputs(c.n_qubits, *c.graph_arrays(), [torch.from_numpy(p).cuda() for p in ps])
                for c, ps in zip(small.circuits, small.probs)]
        for ci, roles in small.queries:
            q, na = ctx.set_qubit_roles(cids[ci], roles)
            entries.append((q, na, small.circuits[ci], small.probs[ci], roles))
        outs = [torch.full((1 << na,), -1.0, dtype=torch.float64, device="cuda") for _, na, *_ in entries]
        totals = torch.zeros(len(entries), dtype=torch.float64, device="cuda")
        bid = ctx.batch_create([e[0] for e in entries], outs, totals, precision="split_bf16")
        n_tc = sum(ctx.query_tc_steps(e[0])[0] for e in entries)
        assert n_tc >= 6                                        # every big query's last step
        for _ in range(2):
            ctx.batch_run(bid)
        ctx.batch_status(bid)
        for j, (q, na, c, probs, roles) in enumerate(entries):
            single = torch.empty_like(outs[j])
            tot1 = torch.zeros(1, dtype=torch.float64, device="cuda")
            ctx.reconstruct(q, single, "split_bf16", tot1)
            torch.cuda.synchronize()
            assert torch.equal(single, outs[j]), j
            assert abs(tot1.item() - totals[j].item()) <= 1e-12 * max(1.0, abs(tot1.item()))
            ref = O.reconstruct(O.Graph.from_arrays(c.n_qubits, *c.graph_arrays()),
                                [p.astype(np.float64) for p in probs], roles)
            err = np.abs(outs[j].cpu().numpy() - ref).max()
            assert err <= 1e-6 and err <= 1e-5 * np.abs(ref).max() + 1e-15, (j, err)
        ctx.batch_release(bid)

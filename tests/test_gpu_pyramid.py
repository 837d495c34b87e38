"""GPU: the merge pyramid (sqc_config.merge_pyramid).  With it, a query
whose merged qubits of a subcircuit are that subcircuit's highest data
qubits reads the pyramid level holding their sums instead of summing A_i
again.  Checked against the FP64 oracle, against the same queries without
the pyramid, batched and one at a time, after an update of the subcircuit
outputs, and in the HBM budget."""
import numpy as np
import pytest

import oracle as O
from synthetic import workloads as W

pytestmark = pytest.mark.gpu

ABS_TOL = 1e-6
REL_TOL = 1e-5


def _oracle(c, probs, roles):
    g = O.Graph.from_arrays(c.n_qubits, *c.graph_arrays())
    return O.reconstruct(g, [p.astype(np.float64) for p in probs], roles)


def _check(P, ref):
    err = np.abs(P - ref).max()
    assert err <= ABS_TOL and err <= REL_TOL * np.abs(ref).max() + 1e-15, err


@pytest.fixture(scope="module")
def ctxs():
    import torch
    from paper_2207_00933_gb300 import Context, _build
    _build.build()
    on, off = Context(0, merge_pyramid=True), Context(0)
    yield on, off
    torch.cuda.synchronize()
    on.close()
    off.close()


def _run(ctx, c, probs, roles, out_dtype="float32", precision="fp32"):
    import torch
    cid = ctx.load_subcircuit_outputs(c.n_qubits, *c.graph_arrays(), [torch.from_numpy(p).cuda() for p in probs])
    qid, na = ctx.set_qubit_roles(cid, roles)
    out = torch.empty(1 << na, dtype=getattr(torch, out_dtype), device="cuda")
    tot = torch.zeros(1, dtype=torch.float64, device="cuda")
    ctx.reconstruct(qid, out, precision, tot)
    torch.cuda.synchronize()
    res = out.double().cpu().numpy(), float(tot.item())
    ctx.unload(cid)
    return res


@pytest.mark.parametrize("wl,out,prec", [("merged_30q", "float32", "fp32"), ("grid_40q", "float64", "fp32"),
                                         ("grid_40q", "float64", "split_bf16"), ("full_state_12q", "float32", "fp32")])
def test_pyramid_matches_oracle_and_plain_merge(ctxs, wl, out, prec):
    on, off = ctxs
    w = getattr(W, wl)()
    ref = _oracle(w.circuit, w.probs, w.roles)
    P1, t1 = _run(on, w.circuit, w.probs, w.roles, out, prec)
    P0, t0 = _run(off, w.circuit, w.probs, w.roles, out, prec)
    _check(P1, ref)
    _check(P0, ref)
    assert abs(t1 - O.total_probability(ref)) < 1e-6


def test_pyramid_zoom_queries_batched_and_single(ctxs):
    """Zoom queries (zoomed prefix, active, merged) over several circuits:
    the batched launch equals the one-at-a-time runs bit for bit, both
    read the pyramid, and both match the oracle."""
    import torch
    on, _ = ctxs
    b = W.batch_level(seed=5, n_circuits=3, n_queries=24, a_range=(6, 12), max_log_input=18, min_qubits=30)
    cids = [on.load_subcircuit_outputs(c.n_qubits, *c.graph_arrays(), [torch.from_numpy(p).cuda() for p in ps])
            for c, ps in zip(b.circuits, b.probs)]
    qs = [on.set_qubit_roles(cids[ci], roles) for ci, roles in b.queries]
    outs = [torch.full((1 << na,), -1.0, dtype=torch.float32, device="cuda") for _, na in qs]
    bid = on.batch_create([q for q, _ in qs], outs)
    on.batch_run(bid)
    on.batch_status(bid)
    for j, (q, na) in enumerate(qs):
        ci, roles = b.queries[j]
        _check(outs[j].double().cpu().numpy(), _oracle(b.circuits[ci], b.probs[ci], roles))
        single = torch.empty_like(outs[j])
        on.reconstruct(q, single)
        torch.cuda.synchronize()
        assert torch.equal(single, outs[j]), j
    on.batch_release(bid)
    for cid in cids:
        on.unload(cid)


def test_pyramid_follows_updates(ctxs):
    import torch
    on, _ = ctxs
    w = W.merged_30q()
    c = w.circuit
    cid = on.load_subcircuit_outputs(c.n_qubits, *c.graph_arrays(), [torch.from_numpy(p).cuda() for p in w.probs])
    qid, na = on.set_qubit_roles(cid, w.roles)
    rng = np.random.default_rng(9)
    new = [np.ascontiguousarray(p * rng.uniform(0.5, 1.5, size=p.shape).astype(np.float32)) for p in w.probs]
    on.update_subcircuit_outputs(cid, [torch.from_numpy(p).cuda() for p in new])
    out = torch.empty(1 << na, dtype=torch.float32, device="cuda")
    on.reconstruct(qid, out)
    torch.cuda.synchronize()
    _check(out.double().cpu().numpy(), _oracle(c, new, w.roles))
    on.unload(cid)


def test_pyramid_counts_in_the_hbm_budget():
    import torch
    from paper_2207_00933_gb300 import Context, SQCError
    w = W.merged_30q()
    c = w.circuit
    a_bytes = sum(p.shape[0] * (1 << len(c.data_qubits[i])) * 4 for i, p in enumerate(w.probs))
    budget = a_bytes + a_bytes // 2            # room for A but not for A and its pyramid
    probs = [torch.from_numpy(p).cuda() for p in w.probs]
    with Context(0, hbm_budget_bytes=budget) as plain:
        plain.unload(plain.load_subcircuit_outputs(c.n_qubits, *c.graph_arrays(), probs))
    with Context(0, hbm_budget_bytes=budget, merge_pyramid=True) as pyr:
        with pytest.raises(SQCError) as ei:
            pyr.load_subcircuit_outputs(c.n_qubits, *c.graph_arrays(), probs)
        assert ei.value.status == 6                 # SQC_EBUSY

"""GPU: first-level index slicing (Section 6.3).  Writing out cut edges
explicitly splits the Eq. 1 sum into 4^S smaller contractions whose bins
are added into the output; the result must not change (beyond FP32
rounding), and the edges chosen must be the ones the paper's greedy rule
(slice the edge that shrinks the total tensor size most) picks in the
oracle."""
import numpy as np
import pytest

import oracle as O
from synthetic import workloads as W

pytestmark = pytest.mark.gpu


def _run(w, slice_edges, precision="fp32", out_dtype="float32"):
    import torch
    from paper_2207_00933_gb300 import Context, _build
    _build.build()
    c = w.circuit
    with Context(0, slice_edges=slice_edges) as ctx:
        cid = ctx.load_subcircuit_outputs(c.n_qubits, *c.graph_arrays(), [torch.from_numpy(p).cuda() for p in w.probs])
        q, na = ctx.set_qubit_roles(cid, w.roles)
        out = torch.empty(1 << na, dtype=getattr(torch, out_dtype), device="cuda")
        tot = torch.zeros(1, dtype=torch.float64, device="cuda")
        ctx.reconstruct(q, out, precision, tot)
        torch.cuda.synchronize()
        return out.double().cpu().numpy(), float(tot.item()), ctx.query_slices(q)


@pytest.mark.parametrize("wl,S,prec,out", [("merged_30q", 1, "fp32", "float32"), ("merged_30q", 2, "fp32", "float32"),
                                            ("grid_40q", 1, "fp32", "float64"), ("grid_40q", 2, "split_bf16", "float64")])
def test_sliced_equals_unsliced_and_oracle(wl, S, prec, out):
    w = getattr(W, wl)()
    c = w.circuit
    g = O.Graph.from_arrays(c.n_qubits, *c.graph_arrays())
    ref = O.reconstruct(g, [p.astype(np.float64) for p in w.probs], w.roles)
    P, tot, sliced = _run(w, S, prec, out)
    assert len(sliced) == S
    bins = [1 << sum(1 for q in dq if w.roles[q] == O.ACTIVE) for dq in c.data_qubits]
    assert sliced == O.greedy_slicing(g, bins, 0)[:S]
    err = np.abs(P - ref).max()
    assert err <= 1e-6 and err <= 1e-5 * np.abs(ref).max() + 1e-15
    assert abs(tot - O.total_probability(ref)) < 1e-6
    P0, _, none = _run(w, 0, prec, out)
    assert none == []
    assert np.abs(P - P0).max() <= 1e-5 * np.abs(ref).max()


def _run_cfg(w, **cfg):
    import torch
    from paper_2207_00933_gb300 import Context, _build
    _build.build()
    c = w.circuit
    with Context(0, **cfg) as ctx:
        cid = ctx.load_subcircuit_outputs(c.n_qubits, *c.graph_arrays(), [torch.from_numpy(p).cuda() for p in w.probs])
        q, na = ctx.set_qubit_roles(cid, w.roles)
        out = torch.empty(1 << na, dtype=torch.float64, device="cuda")
        ctx.reconstruct(q, out)
        torch.cuda.synchronize()
        return out.cpu().numpy(), ctx.query_slices(q), ctx.query_steps(q)


@pytest.mark.parametrize("wl", ["merged_30q", "grid_40q"])
def test_input_budget_slicing_follows_the_papers_rule(wl):
    # first level by memory budget: slice until sum_i 4^k_i 2^a_i fits, the
    # same edges as the oracle's greedy rule under the same budget
    w = getattr(W, wl)()
    c = w.circuit
    g = O.Graph.from_arrays(c.n_qubits, *c.graph_arrays())
    bins = [1 << sum(1 for q in dq if w.roles[q] == O.ACTIVE) for dq in c.data_qubits]
    full = O.sliced_sizes(g, bins, set())
    log2_budget = int(np.log2(full)) - 3            # needs a few sliced edges
    P, sliced, _ = _run_cfg(w, slice_input_log2=log2_budget)
    assert sliced and sliced == O.greedy_slicing(g, bins, 2 ** log2_budget)
    assert O.sliced_sizes(g, bins, set(sliced)) <= 2 ** log2_budget
    ref = O.reconstruct(g, [p.astype(np.float64) for p in w.probs], w.roles)
    err = np.abs(P - ref).max()
    assert err <= 1e-6 and err <= 1e-5 * np.abs(ref).max() + 1e-15


@pytest.mark.parametrize("wl", ["merged_30q", "grid_40q"])
def test_intermediate_budget_slicing(wl):
    # second level: slice until every intermediate tensor of the contraction
    # (the outputs of all but the last step, M x N floats) fits
    w = getattr(W, wl)()
    c = w.circuit
    g = O.Graph.from_arrays(c.n_qubits, *c.graph_arrays())
    _, none, steps0 = _run_cfg(w)
    assert none == []
    largest = max(m * n for m, n, _ in steps0[:-1])
    log2_budget = int(np.log2(largest)) - 2
    P, sliced, steps = _run_cfg(w, slice_intermediate_log2=log2_budget)
    assert sliced
    assert max(m * n for m, n, _ in steps[:-1]) <= 2 ** log2_budget
    ref = O.reconstruct(g, [p.astype(np.float64) for p in w.probs], w.roles)
    err = np.abs(P - ref).max()
    assert err <= 1e-6 and err <= 1e-5 * np.abs(ref).max() + 1e-15


def test_unreachable_slicing_budget_is_refused():
    import torch
    from paper_2207_00933_gb300 import Context, SQCError, _build
    _build.build()
    w = W.grid_40q()
    c = w.circuit
    with Context(0, slice_input_log2=1) as ctx:
        cid = ctx.load_subcircuit_outputs(c.n_qubits, *c.graph_arrays(), [torch.from_numpy(p).cuda() for p in w.probs])
        with pytest.raises(SQCError) as ei:
            ctx.set_qubit_roles(cid, w.roles)
        assert ei.value.status == 3                 # SQC_ESHAPE

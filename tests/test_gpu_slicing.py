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
    assert err <= 1e-6 and err <= 1e-5 * np.abs(ref).max() + 1e-12
    assert abs(tot - O.total_probability(ref)) < 1e-6
    P0, _, none = _run(w, 0, prec, out)
    assert none == []
    assert np.abs(P - P0).max() <= 1e-5 * np.abs(ref).max()

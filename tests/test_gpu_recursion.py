"""GPU: Algorithm 1 end to end.  On a Bernstein-Vazirani circuit (one
solution state, every other state exactly zero) cut into a chain of
subcircuits, the recursion finds the hidden string in ceil(n / log2 M)
recursions (Section 4)."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("M", [2 ** 4, 2 ** 6])
def test_bv_solution_in_n_over_log2M_recursions(M):
    import torch
    from paper_2207_00933_gb300 import Context, _build, recursion
    from synthetic import subcircuit_variant_probs
    from synthetic.circuits import bernstein_vazirani_chain
    _build.build()
    c, s = bernstein_vazirani_chain(9, [7, 7, 6], [2, 2])
    probs = [torch.from_numpy(subcircuit_variant_probs(c, i).astype(np.float32)).cuda()
             for i in range(c.n_subcircuits)]
    graph = (c.n_qubits, *c.graph_arrays())
    with Context(0) as ctx:
        cid = ctx.load_subcircuit_outputs(*graph, probs)
        sols, r = recursion.search(ctx, cid, graph, M, R=64, keep=4, threshold=1e-3)
    assert r == recursion.recursions_needed(c.n_qubits, M)
    assert len(sols) == 1
    bits, p = sols[0]
    assert bits == s
    assert abs(p - 1.0) < 1e-5

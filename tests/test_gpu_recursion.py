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


def test_bv_1000_qubits_at_the_papers_scale():
    """Algorithm 1 at the paper's scale (Section 8.1: 1000-qubit BV,
    M = 2^20 bins per recursion): a 1000-qubit Bernstein-Vazirani circuit
    cut into a chain of 59 subcircuits of at most 18 qubits (58 cuts).  The
    recursion zooms 20 qubits per level and must find the hidden string in
    ceil(1000 / 20) = 50 recursions, with probability 1."""
    import time
    import torch
    from paper_2207_00933_gb300 import Context, _build, recursion
    from synthetic.circuits import bernstein_vazirani_chain
    from synthetic.qpu import product_variant_probs
    _build.build()
    c, s = bernstein_vazirani_chain(5, [18] * 58 + [14], [1] * 58)
    assert c.n_qubits == 1000 and c.n_subcircuits == 59 and c.n_edges == 58
    graph = (c.n_qubits, *c.graph_arrays())
    M = 2 ** 20
    with Context(0) as ctx:
        probs = [torch.from_numpy(product_variant_probs(c, i, np.float32)).cuda() for i in range(c.n_subcircuits)]
        cid = ctx.load_subcircuit_outputs(*graph, probs)
        del probs
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        sols, r = recursion.search(ctx, cid, graph, M, R=64, keep=4, threshold=1e-3)
        dt = time.perf_counter() - t0
    assert r == recursion.recursions_needed(c.n_qubits, M) == 50
    assert len(sols) == 1
    bits, p = sols[0]
    assert bits == s
    assert abs(p - 1.0) < 1e-5
    assert dt / r < 1.0                     # seconds per recursion (planning, reconstruction, selection)

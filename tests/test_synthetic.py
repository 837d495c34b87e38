"""CPU checks of the synthetic QPU stand-in: the product-state generator of
subcircuit outputs (blocks with one-qubit gates only) equals the full
statevector generator on every variant, including wires that are both
received and passed on by one block."""
import numpy as np

from synthetic.circuits import Block, CutCircuit, bernstein_vazirani_chain
from synthetic.qpu import product_variant_probs, subcircuit_variant_probs


def test_product_generator_matches_statevector_on_bv():
    c, _ = bernstein_vazirani_chain(9, [7, 7, 6], [2, 2])
    for i in range(c.n_subcircuits):
        a = product_variant_probs(c, i)
        b = subcircuit_variant_probs(c, i)
        assert a.shape == b.shape
        assert np.abs(a - b).max() < 1e-14


def test_product_generator_matches_statevector_on_rotations():
    # wire 2 passes through all three blocks (received and passed on by the
    # middle one); gates from the whole one-qubit set
    rng = np.random.default_rng(4)
    names = ["h", "t", "sx", "sy"]

    def gates(qs):
        g = [(names[int(rng.integers(4))], q) for q in qs for _ in range(3)]
        return g + [("rz", qs[0], float(rng.uniform(0, 6.28)))]
    c = CutCircuit(6, [Block([0, 1, 2], gates([0, 1, 2])), Block([1, 2, 3], gates([1, 2, 3])),
                       Block([2, 3, 4, 5], gates([2, 3, 4, 5]))]).finalize()
    assert any(set(c.in_edges[1]) and set(c.out_edges[1]) for _ in [0])
    for i in range(c.n_subcircuits):
        assert np.abs(product_variant_probs(c, i) - subcircuit_variant_probs(c, i)).max() < 1e-14

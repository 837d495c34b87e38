"""Pins for the FP64 oracle and the QPU stand-in: each check compares against
something other than the oracle itself (textbook quantum mechanics, the
uncut circuit's statevector, exact identities of the method, and the numbers
the paper prints)."""
import json
import math
import os

import numpy as np
import pytest

import oracle as O
import importlib
R = importlib.import_module("oracle.reconstruct")
from synthetic import (chain_line_circuit, full_circuit_probs, random_block_circuit,
                       subcircuit_variant_probs)
from synthetic.circuits import Block, CutCircuit
from synthetic.qpu import GATES
from synthetic import workloads as W

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def graph_of(c):
    return O.Graph.from_arrays(c.n_qubits, *c.graph_arrays())


def exact_probs(c):
    return [subcircuit_variant_probs(c, i) for i in range(c.n_subcircuits)]


# ---- the QPU stand-in against textbook circuits -------------------------------

def _dense_unitary(gates, n):
    """Textbook construction: each gate as a 2^n x 2^n Kronecker product,
    qubit 0 the least significant index bit."""
    I2 = np.eye(2)
    U = np.eye(1 << n, dtype=complex)
    for g in gates:
        if g[0] == "cz":
            d = np.ones(1 << n)
            for x in range(1 << n):
                if (x >> g[1]) & 1 and (x >> g[2]) & 1:
                    d[x] = -1
            G = np.diag(d)
        else:
            u = GATES[g[0]] if g[0] != "rz" else np.diag([np.exp(-0.5j * g[2]), np.exp(0.5j * g[2])])
            G = np.array([[1.0]])
            for q in reversed(range(n)):
                G = np.kron(G, u if q == g[1] else I2)
        U = G @ U
    return U


def test_gate_matrices_are_the_textbook_ones():
    X = np.array([[0, 1], [1, 0]])
    Y = np.array([[0, -1j], [1j, 0]])
    for name in ("h", "t", "sx", "sy", "sdg"):
        u = GATES[name]
        assert np.allclose(u @ u.conj().T, np.eye(2))
    assert np.allclose(GATES["sx"] @ GATES["sx"], X)
    assert np.allclose(GATES["sy"] @ GATES["sy"], Y)
    assert np.allclose(GATES["t"] @ GATES["t"] @ GATES["t"] @ GATES["t"], np.diag([1, -1]))


def test_bell_state():
    c = CutCircuit(2, [Block([0, 1], [("h", 0), ("h", 1), ("cz", 0, 1), ("h", 1)])]).finalize()
    assert np.allclose(full_circuit_probs(c), [0.5, 0, 0, 0.5])


def test_statevector_matches_dense_matrices():
    rng = np.random.default_rng(7)
    gates = []
    for _ in range(12):
        name = ["h", "t", "sx", "sy", "rz", "cz"][rng.integers(6)]
        if name == "cz":
            a, b = rng.choice(4, 2, replace=False)
            gates.append(("cz", int(a), int(b)))
        elif name == "rz":
            gates.append(("rz", int(rng.integers(4)), float(rng.uniform(0, 6))))
        else:
            gates.append((name, int(rng.integers(4))))
    c = CutCircuit(4, [Block([0, 1, 2, 3], gates)]).finalize()
    psi0 = np.zeros(16)
    psi0[0] = 1
    expect = np.abs(_dense_unitary(gates, 4) @ psi0) ** 2
    assert np.allclose(full_circuit_probs(c), expect, atol=1e-14)


def test_variant_measurement_bases():
    # one wire prepared in |+i> by H then S (S = T^2), then cut straight away:
    # upstream measurements in X, Y, Z bases give <X>=0, <Y>=1, <Z>=0
    c = CutCircuit(1, [Block([0], [("h", 0), ("t", 0), ("t", 0)]), Block([0], [])]).finalize()
    p = subcircuit_variant_probs(c, 0)          # [4 bases, 2 outcomes]
    exp = p[:, 0] - p[:, 1]
    assert np.allclose(exp, [0.0, 0.0, 1.0, 0.0], atol=1e-15)
    assert np.allclose(p.sum(axis=1), 1.0)
    # downstream initial states: measuring right away gives their Z statistics
    q = subcircuit_variant_probs(c, 1)          # [4 inits, 2 outcomes]
    assert np.allclose(q, [[1, 0], [0, 1], [0.5, 0.5], [0.5, 0.5]])


# ---- Eq. 1 end to end against the uncut circuit --------------------------------

def test_full_state_12q_matches_statevector():
    w = W.full_state_12q()
    g = graph_of(w.circuit)
    P = O.reconstruct(g, w.probs, w.roles)
    F = full_circuit_probs(w.circuit)
    assert P.shape == (1 << 12,)
    assert np.abs(P - F).max() < 1e-13


@pytest.mark.parametrize("seed", range(24))
def test_random_graphs_match_statevector(seed):
    c = random_block_circuit(seed, 9, 4, 5, 2, p_reuse=0.8)
    g = graph_of(c)
    P = O.reconstruct(g, exact_probs(c), np.zeros(c.n_qubits, dtype=int))
    assert np.abs(P - full_circuit_probs(c)).max() < 1e-13


def test_wire_cut_twice_matches_statevector():
    # qubit 2 runs through all three blocks: block 1 has an in- and an
    # out-edge on the same wire
    c = chain_line_circuit(5, [3, 3, 3], [2, 2], 3)
    assert any(e[2] == 2 for e in c.edges if e[0] == 0) and any(e[2] == 2 for e in c.edges if e[0] == 1)
    P = O.reconstruct(graph_of(c), exact_probs(c), np.zeros(c.n_qubits, dtype=int))
    assert np.abs(P - full_circuit_probs(c)).max() < 1e-13


def test_subcircuit_without_data_qubits_matches_statevector():
    # the middle block hands every one of its wires on (2 in, 3 out, no
    # data qubit), as subcircuit 2 of the paper's Fig. 5 graph (2^0 bins)
    c = chain_line_circuit(7, [4, 3, 4], [2, 3], 3)
    assert [len(d) for d in c.data_qubits] == [2, 0, 4] and c.n_edges == 5
    P = O.reconstruct(graph_of(c), exact_probs(c), np.zeros(c.n_qubits, dtype=int))
    assert np.abs(P - full_circuit_probs(c)).max() < 1e-13


def test_zero_cut_identity():
    c = CutCircuit(5, [Block(list(range(5)), [("h", 0), ("cz", 0, 1), ("sx", 3), ("t", 1), ("sy", 4)])]).finalize()
    p = exact_probs(c)
    P = O.reconstruct(graph_of(c), p, np.zeros(5, dtype=int))
    assert c.n_edges == 0
    assert np.array_equal(P, p[0][0])


# ---- states merging identities -------------------------------------------------

def test_all_merged_is_one():
    w = W.full_state_12q(4)
    roles = np.full(w.circuit.n_qubits, O.MERGED)
    P = O.reconstruct(graph_of(w.circuit), w.probs, roles)
    assert P.shape == (1,)
    assert abs(P[0] - 1.0) < 1e-13


def test_merged_and_zoomed_bins_are_marginals_of_the_statevector():
    for seed in range(6):
        w = W.small_random(seed, roles="mixed")
        c = w.circuit
        P = O.reconstruct(graph_of(c), w.probs, w.roles)
        F = full_circuit_probs(c)
        x = np.arange(1 << c.n_qubits)
        keep = np.ones_like(x, dtype=bool)
        b = np.zeros_like(x)
        j = 0
        for q in range(c.n_qubits):
            bit = (x >> q) & 1
            if w.roles[q] == O.ZOOM0:
                keep &= bit == 0
            elif w.roles[q] == O.ZOOM1:
                keep &= bit == 1
            elif w.roles[q] == O.ACTIVE:
                b |= bit << j
                j += 1
        expect = np.zeros(1 << j)
        np.add.at(expect, b[keep], F[keep])
        assert np.abs(P - expect).max() < 1e-13


def test_children_sum_to_parent():
    w = W.merged_30q()
    g = graph_of(w.circuit)
    probs = [p.astype(np.float64) for p in w.probs]
    q = w.circuit.data_qubits[1][5]          # a merged qubit of subcircuit 1
    assert w.roles[q] == O.MERGED
    parent = O.reconstruct(g, probs, w.roles)
    kids = []
    for role in (O.ZOOM0, O.ZOOM1):
        r = w.roles.copy()
        r[q] = role
        kids.append(O.reconstruct(g, probs, r))
    assert np.abs(kids[0] + kids[1] - parent).max() < 1e-13
    assert abs(O.total_probability(parent) - 1.0) < 1e-6     # FP32-rounded inputs


def test_full_state_when_M_covers_everything():
    # Section 4: with M >= 2^n states merging is the full-state reconstruction
    w = W.full_state_12q()
    g = graph_of(w.circuit)
    roles = O.roles_for_recursion(g, {}, 1 << 12)
    assert all(r == O.ACTIVE for r in roles)


# ---- contraction order only permutes; Eq. 1 bin by bin agrees ----------------

@pytest.mark.parametrize("seed", range(8))
def test_pairwise_equals_bruteforce_random(seed):
    w = W.small_random(seed, roles="mixed")
    g = graph_of(w.circuit)
    T = O.subcircuit_tensors(g, w.probs, w.roles)
    P = O.reconstruct_pairwise(g, T, w.roles)
    bins = np.arange(P.size)
    assert np.abs(O.reconstruct_bruteforce(g, T, w.roles, bins) - P).max() < 1e-14


def test_pairwise_equals_bruteforce_30q_sampled():
    w = W.merged_30q()
    g = graph_of(w.circuit)
    T = O.subcircuit_tensors(g, w.probs, w.roles)
    P = O.reconstruct_pairwise(g, T, w.roles)
    rng = np.random.default_rng(0)
    bins = rng.integers(0, P.size, 6)
    bf = O.reconstruct_bruteforce(g, T, w.roles, bins)
    assert np.abs(bf - P[bins]).max() < 1e-15


def test_subcircuit_order_does_not_matter():
    # reversing the subcircuit numbering changes the contraction order but
    # not the reconstructed bins (Section 6.4)
    w = W.small_random(3, roles="mixed")
    c = w.circuit
    g = graph_of(c)
    P = O.reconstruct(g, w.probs, w.roles)
    nC = g.n_subcircuits
    perm = list(reversed(range(nC)))
    g2 = O.Graph(g.n_qubits, [perm.index(u) for u in g.edge_up], [perm.index(d) for d in g.edge_down],
                 [g.data_qubits[perm[i]] for i in range(nC)])
    # the edges keep their ids, so each subcircuit's variant layout is unchanged
    P2 = O.reconstruct(g2, [w.probs[perm[i]] for i in range(nC)], w.roles)
    assert np.abs(P - P2).max() < 1e-15


def test_factored_attribution_equals_literal_sum():
    c = chain_line_circuit(11, [4, 4, 3], [2, 2], 2)
    g = graph_of(c)
    p = exact_probs(c)
    for i in range(c.n_subcircuits):
        assert np.abs(O.attribute(g, i, p[i]) - O.attribute_literal(g, i, p[i])).max() < 1e-15


# ---- planted mistakes are caught ------------------------------------------------

@pytest.mark.parametrize("mistake", ["x_row_sign", "y_uses_plus", "z_row_sign", "w_sign", "no_scale",
                                     "swap_inits", "swap_plus_states"])
def test_planted_mistakes_fail_the_statevector_pin(monkeypatch, mistake):
    # a plausible slip anywhere in the attribution changes at least one of
    # these circuits' reconstructions far beyond rounding
    Dm, Wm = R.D.copy(), R.W.copy()
    if mistake == "x_row_sign":
        Dm[1] = -Dm[1]
    elif mistake == "y_uses_plus":
        Dm[2] = [-1, -1, 2, 0]
    elif mistake == "z_row_sign":
        Dm[3] = -Dm[3]
    elif mistake == "w_sign":
        Wm[2] = [1, 1]
    elif mistake == "swap_inits":
        Dm = Dm[:, [1, 0, 2, 3]]
    elif mistake == "swap_plus_states":
        Dm = Dm[:, [0, 1, 3, 2]]
    monkeypatch.setattr(R, "D", Dm)
    monkeypatch.setattr(R, "W", Wm)
    worst = 0.0
    for seed in range(2, 8):
        c = chain_line_circuit(seed, [4, 4], [2], 3)
        P = O.reconstruct(graph_of(c), exact_probs(c), np.zeros(c.n_qubits, dtype=int))
        if mistake == "no_scale":
            P = P * 2.0 ** c.n_edges
        worst = max(worst, np.abs(P - full_circuit_probs(c)).max())
    assert worst > 1e-3


# ---- top bins ------------------------------------------------------------------

def test_top_bins_order_and_ties():
    P = np.array([0.1, 0.3, 0.3, 0.05, 0.3, 0.25])
    b, v = O.top_bins(P, 4)
    assert b.tolist() == [1, 2, 4, 5]
    assert v.tolist() == [0.3, 0.3, 0.3, 0.25]
    b, v = O.top_bins(P, 10, threshold=0.1)
    assert b.tolist() == [1, 2, 4, 5, 0]
    b, _ = O.top_bins(P, 0)
    assert b.size == 0


def test_top_bins_single_solution():
    # Bernstein-Vazirani-like concentrated output: the one solution bin is
    # the unique top bin at every level (Section 4)
    P = np.full(1 << 10, 1e-9)
    P[613] = 0.9
    assert O.top_bins(P, 1)[0].tolist() == [613]


# ---- Algorithm 2 and the cost model ----------------------------------------------

def test_states_assignment_configs():
    assert O.states_assignment([2 ** 7, 2 ** 8, 2 ** 7, 2 ** 8], 2 ** 20) == [32] * 4
    assert O.states_assignment([2 ** 5, 2 ** 8, 2 ** 8, 2 ** 8, 2 ** 11], 2 ** 22) == [16, 16, 16, 32, 32]
    lp = O.states_assignment([2 ** 7, 2 ** 3, 2 ** 9], 2 ** 10)
    assert math.prod(lp) <= 2 ** 10 and all(x & (x - 1) == 0 for x in lp)


def test_workload_roles_follow_algorithm_2():
    for w, M in ((W.merged_30q(), 2 ** 20), (W.grid_40q(), 2 ** 22)):
        g = graph_of(w.circuit)
        assert list(O.roles_for_recursion(g, {}, M)) == list(w.roles)


def test_zoomed_recursion_keeps_low_bits_active():
    g = O.Graph(6, [], [], [[0, 1, 2, 3, 4, 5]])
    roles = O.roles_for_recursion(g, {0: 1, 1: 0}, 4)
    assert roles == [O.ZOOM1, O.ZOOM0, O.ACTIVE, O.ACTIVE, O.MERGED, O.MERGED]


def test_cost_model_worked_example():
    gold = json.load(open(os.path.join(GOLDEN, "fig5_cost_model.json")))
    edges, bins = gold["graph"]["edges"], gold["graph"]["bins"]
    g = O.Graph(0, [e[0] for e in edges], [e[1] for e in edges], [[], [], []])
    k = [len(g.incident(i)) for i in range(3)]
    assert k == [3, 2, 3]
    floats1 = sum(O.tensor_floats(k[i], bins[i]) for i in range(3))
    assert floats1 == gold["input_floats_step1"]
    # step 1 contracts subcircuits 1 and 2 over their shared edge (dim 4):
    # free dims 4^2 x 2^1 (subcircuit 1) and 4^1 x 2^0 (subcircuit 2)
    assert O.step_multiplications([4 ** 2 * bins[0], 4, 4 * bins[1]]) == gold["multiplications_step1"]
    # step 2: subcircuit 3 with the 12 result ({4,4,4,2^1}) over three edges
    assert O.tensor_floats(3, bins[2]) + O.tensor_floats(3, bins[0] * bins[1]) == gold["input_floats_step2"]
    assert O.step_multiplications([bins[2], 4 ** 3, bins[0] * bins[1]]) == gold["multiplications_step2"]
    naive = O.naive_multiplications(len(edges), bins)
    assert naive == gold["naive_multiplications"]
    assert round(naive / (gold["multiplications_step1"] + gold["multiplications_step2"]), 1) == \
        gold["naive_overhead_ratio_printed"]
    sl = O.greedy_slicing(g, bins, gold["sliced_one_edge_floats"])
    assert len(sl) == 1 and set(edges[sl[0]]) == {0, 2}
    assert O.sliced_sizes(g, bins, set(sl)) == gold["sliced_one_edge_floats"]
    assert 4 ** len(sl) == gold["sliced_graphs"]

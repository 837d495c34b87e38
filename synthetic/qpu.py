"""FP64 statevector simulation: the stand-in for the QPU.

Two uses, neither of which is the reconstruction method itself:

* ``subcircuit_variant_probs`` produces what a QPU returns for every cut
  assignment of a subcircuit (Section 2.1, Fig. 1b): the subcircuit is
  initialised in each of |0>, |1>, |+>, |+i> on its incoming cut wires and
  measured in each of the I, X, Y, Z bases on its outgoing cut wires.
* ``full_circuit_probs`` simulates the uncut circuit, the brute-force truth
  the reconstruction must reproduce.

Basis conventions (the paper defers them to Peng et al.):
  measurement basis digit 0=I, 1=X, 2=Y, 3=Z; X is measured after H, Y after
  S^dagger then H, I and Z in the computational basis (so I and Z are the
  same physical run).  Initial-state digit 0=|0>, 1=|1>, 2=|+>,
  3=|+i>=(|0>+i|1>)/sqrt2.

Index conventions (the boundary's input layout):
  * a state index is little-endian over the listed wires;
  * a subcircuit's output index is y = x | c << n_i, where x runs over its
    data qubits in ascending original-qubit order and c over its outgoing
    cut wires in ascending edge id;
  * the variant index has one base-4 digit per incident edge, edges in
    ascending id, the first edge the most significant digit.
"""
from __future__ import annotations

import numpy as np

from .circuits import CutCircuit

_S2 = 1.0 / np.sqrt(2.0)
GATES = {
    "h": np.array([[1, 1], [1, -1]], dtype=np.complex128) * _S2,
    "t": np.array([[1, 0], [0, np.exp(1j * np.pi / 4)]], dtype=np.complex128),
    "sx": 0.5 * np.array([[1 + 1j, 1 - 1j], [1 - 1j, 1 + 1j]], dtype=np.complex128),
    "sy": 0.5 * np.array([[1 + 1j, -1 - 1j], [1 + 1j, 1 + 1j]], dtype=np.complex128),
    "sdg": np.array([[1, 0], [0, -1j]], dtype=np.complex128),
}


def rz(theta: float) -> np.ndarray:
    return np.array([[np.exp(-0.5j * theta), 0], [0, np.exp(0.5j * theta)]], dtype=np.complex128)


INIT_STATES = np.array([[1, 0], [0, 1], [_S2, _S2], [_S2, 1j * _S2]], dtype=np.complex128)


def apply_1q(psi: np.ndarray, u: np.ndarray, q: int, nq: int) -> np.ndarray:
    """psi: [B, 2^nq]; apply 2x2 u to local wire q (bit q of the index)."""
    B = psi.shape[0]
    v = psi.reshape(B, 1 << (nq - q - 1), 2, 1 << q)
    v = np.einsum("ab,xsbt->xsat", u, v)
    return v.reshape(B, 1 << nq)


def apply_cz(psi: np.ndarray, q0: int, q1: int, nq: int) -> np.ndarray:
    idx = np.arange(1 << nq)
    mask = ((idx >> q0) & 1) & ((idx >> q1) & 1)
    out = psi.copy()
    out[:, mask.astype(bool)] *= -1
    return out


def _run_gates(psi, gates, local, nq):
    for g in gates:
        if g[0] == "cz":
            psi = apply_cz(psi, local[g[1]], local[g[2]], nq)
        elif g[0] == "rz":
            psi = apply_1q(psi, rz(g[2]), local[g[1]], nq)
        else:
            psi = apply_1q(psi, GATES[g[0]], local[g[1]], nq)
    return psi


def full_circuit_probs(c: CutCircuit) -> np.ndarray:
    """|amplitude|^2 of the uncut circuit, index little-endian over all
    original qubits.  Feasible up to ~24 qubits."""
    n = c.n_qubits
    psi = np.zeros((1, 1 << n), dtype=np.complex128)
    psi[0, 0] = 1.0
    ident = {q: q for q in range(n)}
    for blk in c.blocks:
        psi = _run_gates(psi, blk.gates, ident, n)
    return (np.abs(psi[0]) ** 2).astype(np.float64)


def subcircuit_variant_probs(c: CutCircuit, i: int) -> np.ndarray:
    """[4^{k_i}, 2^{w_i}] FP64 output probabilities of subcircuit i for every
    variant, in the boundary's input layout (module docstring)."""
    blk = c.blocks[i]
    wires = list(blk.qubits)
    nq = len(wires)
    local = {q: t for t, q in enumerate(wires)}
    edge_q = {eid: c.edges[eid][2] for eid in c.incident[i]}
    ins, outs = c.in_edges[i], c.out_edges[i]
    kin, kout = len(ins), len(outs)

    # batch over all init-state tuples of the incoming wires: digit order of
    # the batch index = ins in ascending edge id, first one most significant
    B = 4 ** kin
    psi = np.zeros((B, 1 << nq), dtype=np.complex128)
    for bidx in range(B):
        digits = [(bidx >> (2 * (kin - 1 - t))) & 3 for t in range(kin)]
        vec = np.ones(1, dtype=np.complex128)
        # build the product state wire by wire (wire 0 least significant)
        for t in range(nq):
            q = wires[t]
            st = np.array([1, 0], dtype=np.complex128)
            for pos, eid in enumerate(ins):
                if edge_q[eid] == q:
                    st = INIT_STATES[digits[pos]]
            vec = np.kron(st, vec)
        psi[bidx] = vec
    psi = _run_gates(psi, blk.gates, local, nq)

    # measurement settings over outgoing wires
    data = c.data_qubits[i]
    n_i = len(data)
    perm_src = [local[q] for q in data] + [local[edge_q[e]] for e in outs]  # y bit -> local wire
    w = n_i + kout
    assert w == nq, "every wire of a block is either data or cut onward"
    k = len(c.incident[i])
    out = np.zeros((4 ** k, 1 << w), dtype=np.float64)
    y = np.arange(1 << w)
    src_index = np.zeros(1 << w, dtype=np.int64)
    for bit, lw in enumerate(perm_src):
        src_index |= ((y >> bit) & 1) << lw
    for m in range(4 ** kout):
        bases = [(m >> (2 * (kout - 1 - t))) & 3 for t in range(kout)]
        phi = psi
        for pos, eid in enumerate(outs):
            lw = local[edge_q[eid]]
            if bases[pos] == 1:
                phi = apply_1q(phi, GATES["h"], lw, nq)
            elif bases[pos] == 2:
                phi = apply_1q(phi, GATES["sdg"], lw, nq)
                phi = apply_1q(phi, GATES["h"], lw, nq)
        probs = np.abs(phi) ** 2                     # [B, 2^nq] over local wires
        probs = probs[:, src_index]                  # -> output index y
        # scatter into the variant index (digits over incident edges)
        for bidx in range(B):
            in_digits = [(bidx >> (2 * (kin - 1 - t))) & 3 for t in range(kin)]
            v = 0
            for eid in c.incident[i]:
                d = in_digits[ins.index(eid)] if eid in ins else bases[outs.index(eid)]
                v = v * 4 + d
            out[v] = probs[bidx]
    return out


def random_variant_probs(c: CutCircuit, i: int, rng: np.random.Generator) -> np.ndarray:
    """Random numbers in place of a QPU's output (as in the paper's timing
    runs, Section 7.1): each variant row is uniform on [0,1) normalised to
    sum 1; the I and Z measurement variants of each outgoing cut are the
    same row, as on hardware."""
    k = len(c.incident[i])
    w = c.width(i)
    out = rng.random((4 ** k, 1 << w))
    out /= out.sum(axis=1, keepdims=True)
    outs = c.out_edges[i]
    if outs:
        pos = {eid: (k - 1 - c.incident[i].index(eid)) for eid in outs}
        v = np.arange(4 ** k)
        src = v.copy()
        for eid, p in pos.items():
            d = (v >> (2 * p)) & 3
            src = np.where(d == 0, src + (3 << (2 * p)), src)  # I row := Z row
        out = out[src]
    return out


def product_variant_probs(c: CutCircuit, i: int, dtype=np.float64) -> np.ndarray:
    """What subcircuit_variant_probs returns, for a block with one-qubit
    gates only: every wire then evolves on its own, so each variant's
    output distribution is the product of its wires' distributions (exact,
    no statevector of the whole block).  Used for wide single-qubit-gate
    blocks (Bernstein-Vazirani in phase-oracle form), where a block of 18
    wires has 16 variants of 2^18 outcomes."""
    blk = c.blocks[i]
    if any(g[0] == "cz" for g in blk.gates):
        raise ValueError("product_variant_probs needs a block without two-qubit gates")
    wires = list(blk.qubits)
    edge_q = {eid: c.edges[eid][2] for eid in c.incident[i]}
    ins, outs = c.in_edges[i], c.out_edges[i]
    unitary = {q: np.eye(2, dtype=np.complex128) for q in wires}
    for g in blk.gates:
        u = rz(g[2]) if g[0] == "rz" else GATES[g[0]]
        unitary[g[1]] = u @ unitary[g[1]]
    ybits = list(c.data_qubits[i]) + [edge_q[e] for e in outs]     # y bit j -> wire
    assert sorted(ybits) == sorted(wires)
    inc = c.incident[i]
    k = len(inc)
    out = np.empty((4 ** k, 1 << len(ybits)), dtype=dtype)
    in_wire = {edge_q[e]: e for e in ins}
    out_wire = {edge_q[e]: e for e in outs}
    for v in range(4 ** k):
        digit = {eid: (v >> (2 * (k - 1 - pos))) & 3 for pos, eid in enumerate(inc)}
        vec = np.ones(1)
        for q in ybits:                                  # bit 0 first: it ends up least significant
            st = INIT_STATES[digit[in_wire[q]]] if q in in_wire else np.array([1, 0], dtype=np.complex128)
            st = unitary[q] @ st
            if q in out_wire:
                basis = digit[out_wire[q]]
                if basis == 1:
                    st = GATES["h"] @ st
                elif basis == 2:
                    st = GATES["h"] @ (GATES["sdg"] @ st)
            vec = np.kron(np.abs(st) ** 2, vec)
        out[v] = vec
    return out

"""Seeded synthetic cut circuits (cut-first generator).

A circuit is a sequence of *blocks*; block i is subcircuit i.  Each block
acts on a set of original qubits with its own gates, and blocks are applied
one after the other.  A qubit that is acted on by several blocks is cut
between each consecutive pair of them (one cut edge per hand-off), which is
exactly the wire cut of Section 2.1 (Fig. 1): the upstream block measures the
wire, the downstream block initialises it.  A qubit's *last* block owns it as
a data (output) qubit.

Choosing the blocks first and the gates inside them second makes the number
of cuts and the subcircuit widths exact, which the paper's MIP cut finder
(Section 5) would otherwise decide.  This module holds no reconstruction
arithmetic; it only describes circuits.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

# single-qubit gate names drawn by the generators
LINE_GATES = ("h", "t", "sx", "sy")
GRID_GATES = ("h", "t", "sx", "sy", "rz")


@dataclass
class Block:
    qubits: list[int]                       # original qubit indices, ascending
    gates: list[tuple] = field(default_factory=list)
    # gate tuples: ("h"|"t"|"sx"|"sy", q) | ("rz", q, theta) | ("cz", q0, q1)


@dataclass
class CutCircuit:
    """A circuit cut into subcircuits; block i is subcircuit i."""
    n_qubits: int
    blocks: list[Block]
    # derived by finalize():
    edges: list[tuple[int, int, int]] = field(default_factory=list)   # (up, down, qubit), edge id = position
    data_qubits: list[list[int]] = field(default_factory=list)        # per subcircuit, ascending
    in_edges: list[list[int]] = field(default_factory=list)           # per subcircuit, ascending edge id
    out_edges: list[list[int]] = field(default_factory=list)
    incident: list[list[int]] = field(default_factory=list)           # in + out, ascending edge id

    @property
    def n_subcircuits(self) -> int:
        return len(self.blocks)

    @property
    def n_edges(self) -> int:
        return len(self.edges)

    def width(self, i: int) -> int:
        """Qubits measured at the end of subcircuit i: data + outgoing cuts."""
        return len(self.data_qubits[i]) + len(self.out_edges[i])

    def finalize(self) -> "CutCircuit":
        nb = len(self.blocks)
        seq: dict[int, list[int]] = {}
        for b, blk in enumerate(self.blocks):
            if sorted(set(blk.qubits)) != list(blk.qubits):
                raise ValueError("block qubits must be ascending and unique")
            for q in blk.qubits:
                seq.setdefault(q, []).append(b)
            for g in blk.gates:
                for q in _gate_qubits(g):
                    if q not in blk.qubits:
                        raise ValueError(f"gate {g} outside block {b}")
        if sorted(seq) != list(range(self.n_qubits)):
            raise ValueError("every qubit must belong to at least one block")
        edges = []
        for q, bs in seq.items():
            for u, d in zip(bs[:-1], bs[1:]):
                edges.append((u, d, q))
        edges.sort()
        self.edges = edges
        self.data_qubits = [[] for _ in range(nb)]
        for q, bs in sorted(seq.items()):
            self.data_qubits[bs[-1]].append(q)
        self.in_edges = [[] for _ in range(nb)]
        self.out_edges = [[] for _ in range(nb)]
        for eid, (u, d, _q) in enumerate(edges):
            self.out_edges[u].append(eid)
            self.in_edges[d].append(eid)
        self.incident = [sorted(self.in_edges[i] + self.out_edges[i]) for i in range(nb)]
        return self

    def graph_arrays(self):
        """(edge_up, edge_down, n_data, data_qubit) as int32 arrays: the
        compute graph of Fig. 3d in the boundary's flat form."""
        eu = np.array([e[0] for e in self.edges], dtype=np.int32)
        ed = np.array([e[1] for e in self.edges], dtype=np.int32)
        nd = np.array([len(d) for d in self.data_qubits], dtype=np.int32)
        dq = np.array([q for d in self.data_qubits for q in d], dtype=np.int32)
        return eu, ed, nd, dq


def _gate_qubits(g):
    return (g[1], g[2]) if g[0] == "cz" else (g[1],)


def _line_layers(rng, qubits, depth, gates=LINE_GATES):
    """Brickwork on a line: a layer of random single-qubit gates, then CZ on
    alternating neighbour pairs (even pairs on even layers, odd on odd)."""
    out = []
    for layer in range(depth):
        for q in qubits:
            name = gates[rng.integers(len(gates))]
            out.append((name, q, float(rng.uniform(0, 2 * np.pi))) if name == "rz" else (name, q))
        for j in range(layer % 2, len(qubits) - 1, 2):
            out.append(("cz", qubits[j], qubits[j + 1]))
    return out


def _grid_layers(rng, qubits, depth, rows, cols, gates=GRID_GATES):
    """Grid brickwork: random single-qubit gates, then CZ on one of four
    neighbour patterns (horizontal even/odd, vertical even/odd), cycling.
    Qubit q sits at row q % rows, column q // rows (column-major)."""
    qs = set(qubits)
    out = []
    for layer in range(depth):
        for q in qubits:
            name = gates[rng.integers(len(gates))]
            out.append((name, q, float(rng.uniform(0, 2 * np.pi))) if name == "rz" else (name, q))
        pat = layer % 4
        for q in qubits:
            r, c = q % rows, q // rows
            if pat < 2:            # horizontal pairs (c, c+1), c parity = pat
                if c % 2 == pat and c + 1 < cols:
                    p = q + rows
                else:
                    continue
            else:                  # vertical pairs (r, r+1), r parity = pat - 2
                if r % 2 == pat - 2 and r + 1 < rows:
                    p = q + 1
                else:
                    continue
            if p in qs:
                out.append(("cz", q, p))
    return out


def chain_line_circuit(seed: int, widths: list[int], handoffs: list[int], depth: int,
                       gates=LINE_GATES) -> CutCircuit:
    """A chain of blocks on a line.  Block b covers `widths[b]` consecutive
    qubits; its last `handoffs[b]` qubits continue into block b+1 (cut
    there), so block b+1 starts at those qubits.  Each block carries
    `depth` brickwork layers."""
    rng = np.random.default_rng(seed)
    assert len(handoffs) == len(widths) - 1
    blocks = []
    start = 0
    for b, w in enumerate(widths):
        qs = list(range(start, start + w))
        blocks.append(Block(qs, _line_layers(rng, qs, depth, gates)))
        if b < len(handoffs):
            h = handoffs[b]
            assert 0 <= h <= w
            start = start + w - h
    n = start + widths[-1]
    return CutCircuit(n, blocks).finalize()


def chain_grid_circuit(seed: int, rows: int, cols: int, widths: list[int], handoffs: list[int],
                       depth: int) -> CutCircuit:
    """Chain of blocks over a rows x cols grid in column-major qubit order,
    same hand-off rule as chain_line_circuit, grid brickwork inside each."""
    rng = np.random.default_rng(seed)
    blocks = []
    start = 0
    for b, w in enumerate(widths):
        qs = list(range(start, start + w))
        blocks.append(Block(qs, _grid_layers(rng, qs, depth, rows, cols)))
        if b < len(handoffs):
            start = start + w - handoffs[b]
    n = start + widths[-1]
    assert n == rows * cols, (n, rows, cols)
    return CutCircuit(n, blocks).finalize()


def random_block_circuit(seed: int, n_qubits: int, n_blocks: int, max_block: int, depth: int,
                         p_reuse: float = 0.5) -> CutCircuit:
    """Small random cut circuit with an arbitrary (not just chain) compute
    graph: each block takes some already-used qubits (cut edges from
    whichever block touched them last) and some fresh ones.  Wires may be cut
    more than once and a block may have both an in- and an out-edge on the
    same wire.  Used for tiny parity cases."""
    rng = np.random.default_rng(seed)
    fresh = list(range(n_qubits))
    used: list[int] = []
    blocks = []
    for b in range(n_blocks):
        remaining_blocks = n_blocks - b
        w = int(rng.integers(1, max_block + 1))
        take_fresh = []
        # leave enough fresh qubits so every later block can take at least one
        max_fresh = max(0, len(fresh) - (remaining_blocks - 1))
        if b == n_blocks - 1:
            take_fresh = list(fresh)
        elif max_fresh > 0:
            nf = int(rng.integers(1, min(w, max_fresh) + 1))
            take_fresh = list(rng.choice(fresh, size=nf, replace=False))
        reuse_pool = [q for q in used]
        n_reuse = 0
        if reuse_pool and b > 0:
            n_reuse = int(rng.binomial(min(len(reuse_pool), max(0, w - len(take_fresh))), p_reuse))
            if n_reuse == 0 and not take_fresh:
                n_reuse = 1
        take_reuse = list(rng.choice(reuse_pool, size=n_reuse, replace=False)) if n_reuse else []
        qs = sorted(int(q) for q in take_fresh + take_reuse)
        if len(qs) > max_block:
            qs = qs[:max_block] if len(take_fresh) <= max_block else qs
        if not qs:
            qs = [int(fresh[0])] if fresh else [int(used[0])]
        for q in qs:
            if q in fresh:
                fresh.remove(q)
                used.append(q)
        blocks.append(Block(qs, _line_layers(rng, qs, depth)))
    # any leftover fresh qubit goes to the last block
    if fresh:
        last = blocks[-1]
        last.qubits = sorted(last.qubits + fresh)
        last.gates += _line_layers(rng, last.qubits, 1)
    return CutCircuit(n_qubits, blocks).finalize()


def bernstein_vazirani_chain(seed: int, widths: list[int], handoffs: list[int]) -> tuple[CutCircuit, list[int]]:
    """Bernstein-Vazirani in phase-oracle form on a chain of blocks: H on
    every qubit, Z (= T^4) on the qubits of the hidden string s, H again, so
    the output is |s> with probability 1.  Each qubit's first H sits in the
    first block that holds it and the rest in its last block, so the cut
    wires carry |+>.  Returns (circuit, s)."""
    rng = np.random.default_rng(seed)
    start, ranges = 0, []
    for b, w in enumerate(widths):
        ranges.append(list(range(start, start + w)))
        if b < len(handoffs):
            start = start + w - handoffs[b]
    n = start + widths[-1]
    s = [int(v) for v in rng.integers(0, 2, n)]
    first = {}
    last = {}
    for b, qs in enumerate(ranges):
        for q in qs:
            first.setdefault(q, b)
            last[q] = b
    blocks = []
    for b, qs in enumerate(ranges):
        gates = []
        for q in qs:
            if first[q] == b:
                gates.append(("h", q))
        for q in qs:
            if last[q] == b:
                if s[q]:
                    gates += [("t", q)] * 4
                gates.append(("h", q))
        blocks.append(Block(qs, gates))
    return CutCircuit(n, blocks).finalize(), s

"""Workload recipes: seeded synthetic cut circuits shaped like the
benchmarked configurations, with their subcircuit variant outputs and qubit
roles.  The recipes state their shapes explicitly; roles are "the lowest a_i
data qubits of each subcircuit active, the rest merged", with a_i given per
recipe (the tests check that this equals what Algorithm 2 assigns)."""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

from .circuits import CutCircuit, chain_grid_circuit, chain_line_circuit, random_block_circuit
from .qpu import random_variant_probs, subcircuit_variant_probs

ACTIVE, MERGED, ZOOM0, ZOOM1 = 0, 1, 2, 3


@dataclass
class Workload:
    name: str
    circuit: CutCircuit
    probs: list[np.ndarray]            # per subcircuit [4^k_i, 2^w_i]
    roles: np.ndarray                  # int8 per original qubit
    meta: dict = field(default_factory=dict)

    @property
    def n_active(self) -> int:
        return int((self.roles == ACTIVE).sum())


def lowest_active_roles(c: CutCircuit, a: list[int], zoom: dict[int, int] | None = None) -> np.ndarray:
    zoom = zoom or {}
    roles = np.full(c.n_qubits, MERGED, dtype=np.int8)
    for q, v in zoom.items():
        roles[q] = ZOOM1 if v else ZOOM0
    for i, dq in enumerate(c.data_qubits):
        free = [q for q in dq if q not in zoom]
        for q in free[:a[i]]:
            roles[q] = ACTIVE
    return roles


def _exact_probs(c: CutCircuit, dtype) -> list[np.ndarray]:
    return [subcircuit_variant_probs(c, i).astype(dtype) for i in range(c.n_subcircuits)]


def full_state_12q(seed: int = 1) -> Workload:
    """12-qubit line circuit, 8 brickwork layers per block, cut at K=2 into
    two 7-qubit subcircuits; FP64 variants; every qubit active (2^12 bins)."""
    c = chain_line_circuit(seed, [7, 7], [2], 8)
    roles = np.zeros(c.n_qubits, dtype=np.int8)
    return Workload("line12_K2_full", c, _exact_probs(c, np.float64), roles,
                    {"seed": seed, "precision": "fp64 inputs"})


def merged_30q(seed: int = 2) -> Workload:
    """30-qubit line circuit of depth 10, cut at K=8 (3,2,3) into 4
    subcircuits of width 10,10,10,8; FP32 variants from exact simulation;
    20 active qubits (5 per subcircuit) and 10 merged: 2^20 bins."""
    c = chain_line_circuit(seed, [10, 10, 10, 8], [3, 2, 3], 10)
    roles = lowest_active_roles(c, [5, 5, 5, 5])
    return Workload("line30_K8_a20", c, _exact_probs(c, np.float32), roles, {"seed": seed})


def grid_40q(seed: int = 3) -> Workload:
    """40-qubit 5x8 grid circuit of depth 8, cut at K=12 (3,3,3,3) into 5
    subcircuits of width 8,11,11,11,11; FP32 variants from exact simulation;
    22 active qubits (4,4,4,5,5): 2^22 bins."""
    c = chain_grid_circuit(seed, 5, 8, [8, 11, 11, 11, 11], [3, 3, 3, 3], 8)
    roles = lowest_active_roles(c, [4, 4, 4, 5, 5])
    return Workload("grid40_K12_a22", c, _exact_probs(c, np.float32), roles, {"seed": seed})


def small_random(seed: int, n_qubits: int = 9, n_blocks: int = 4, max_block: int = 5, depth: int = 2,
                 dtype=np.float64, roles: str = "active") -> Workload:
    """Tiny random cut circuit with an arbitrary compute graph (exact
    variants).  roles: 'active' (all active), or 'mixed' (seeded random
    active / merged / zoom0 / zoom1 per qubit)."""
    c = random_block_circuit(seed, n_qubits, n_blocks, max_block, depth, p_reuse=0.8)
    if roles == "active":
        r = np.zeros(c.n_qubits, dtype=np.int8)
    else:
        rng = np.random.default_rng(seed + 1000)
        r = rng.choice([ACTIVE, ACTIVE, MERGED, ZOOM0, ZOOM1], size=c.n_qubits).astype(np.int8)
    return Workload(f"random{n_qubits}_s{seed}", c, _exact_probs(c, dtype), r, {"seed": seed})


def random_line_chain(seed: int, widths: list[int], handoffs: list[int], depth: int, active: list[int],
                      dtype=np.float32, zoom_bits: int = 0) -> Workload:
    """A chain of line blocks with random numbers in place of QPU outputs
    (as in the paper's timing runs); used where exact simulation of every
    variant would be too slow.  The first `zoom_bits` data qubits of the
    circuit's subcircuits (lowest original index first) are zoomed to seeded
    random values."""
    c = chain_line_circuit(seed, widths, handoffs, depth)
    rng = np.random.default_rng(seed)
    probs = [random_variant_probs(c, i, rng).astype(dtype) for i in range(c.n_subcircuits)]
    zoom = {}
    if zoom_bits:
        for i, dq in enumerate(c.data_qubits):
            for q in dq[:zoom_bits]:
                zoom[q] = int(rng.integers(2))
    roles = lowest_active_roles(c, active, zoom)
    return Workload(f"randline{c.n_qubits}_s{seed}", c, probs, roles, {"seed": seed, "outputs": "random"})


@dataclass
class BatchWorkload:
    """Many zoom queries over a few resident circuits."""
    name: str
    circuits: list                     # CutCircuit
    probs: list                        # per circuit: list of per-subcircuit arrays
    queries: list                      # (circuit index, roles int8 array)
    meta: dict = field(default_factory=dict)


def _chain_shape(rng, n_sub: int, K: int, max_log_input: int, max_width: int, min_qubits: int):
    """Random chain: hand-offs h (sum K, each >= 1) and block widths w with
    4^{k_b} 2^{w_b} <= 2^max_log_input (k_b = h_{b-1} + h_b) and at least two
    data qubits per block; retried until the circuit has >= min_qubits."""
    for _ in range(1000):
        cuts = np.sort(rng.choice(np.arange(1, K), n_sub - 2, replace=False)) if n_sub > 2 else np.array([], int)
        h = np.diff(np.concatenate([[0], cuts, [K]])).astype(int).tolist()
        widths = []
        ok = True
        for b in range(n_sub):
            hin = h[b - 1] if b > 0 else 0
            hout = h[b] if b < n_sub - 1 else 0
            kb = hin + hout
            wmax = min(max_width, max_log_input - 2 * kb)
            wmin = max(hin + hout + 2, hin + 1)
            if wmax < wmin:
                ok = False
                break
            widths.append(int(rng.integers(max(wmin, wmax - 2), wmax + 1)))
        if ok and sum(widths) - K >= min_qubits:
            return widths, h
    raise ValueError("no chain shape satisfies the constraints")


def batch_level(seed: int = 4, n_circuits: int = 4, n_queries: int = 256, a_range=(10, 20),
                n_sub_range=(5, 6), K_range=(6, 10), max_width: int = 16, max_log_input: int = 22,
                min_qubits: int = 60, dtype=np.float32) -> BatchWorkload:
    """Batched recursion level: `n_queries` zoomed bins, each with an active
    count drawn uniformly from a_range, over `n_circuits` seeded random line
    circuits cut into n_sub_range subcircuits at K_range wires.  Subcircuit
    outputs are random numbers (as in the paper's timing runs).  Within each
    subcircuit a query zooms a random number (up to a third) of the lowest
    data qubits to random bits, makes the next ones active (the active count
    spread over the subcircuits at random) and merges the rest."""
    rng = np.random.default_rng(seed)
    circuits, probs = [], []
    for ci in range(n_circuits):
        n_sub = int(rng.integers(n_sub_range[0], n_sub_range[1] + 1))
        K = int(rng.integers(max(K_range[0], n_sub - 1), K_range[1] + 1))
        widths, h = _chain_shape(rng, n_sub, K, max_log_input, max_width, min_qubits)
        c = chain_line_circuit(seed * 1000 + ci, widths, h, 2)
        circuits.append(c)
        probs.append([random_variant_probs(c, i, rng).astype(dtype) for i in range(c.n_subcircuits)])
    queries = []
    for _ in range(n_queries):
        ci = int(rng.integers(n_circuits))
        c = circuits[ci]
        a_total = int(rng.integers(a_range[0], a_range[1] + 1))
        roles = np.full(c.n_qubits, MERGED, dtype=np.int8)
        zoom_n, act_n = [], []
        for dq in c.data_qubits:
            z = int(rng.integers(0, len(dq) // 3 + 1))
            zoom_n.append(z)
            act_n.append(0)
        for _ in range(a_total):
            cand = [i for i, dq in enumerate(c.data_qubits) if zoom_n[i] + act_n[i] < len(dq)]
            if not cand:
                break
            act_n[int(rng.choice(cand))] += 1
        for i, dq in enumerate(c.data_qubits):
            for q in dq[:zoom_n[i]]:
                roles[q] = ZOOM1 if rng.integers(2) else ZOOM0
            for q in dq[zoom_n[i]:zoom_n[i] + act_n[i]]:
                roles[q] = ACTIVE
        queries.append((ci, roles))
    return BatchWorkload(f"batch{n_queries}_s{seed}", circuits, probs, queries,
                         {"seed": seed, "n_qubits": [c.n_qubits for c in circuits],
                          "cuts": [c.n_edges for c in circuits], "subcircuits": [c.n_subcircuits for c in circuits]})


def _merge_components(parts: list[CutCircuit]) -> CutCircuit:
    """Place independent circuits side by side (disjoint qubits): a compute
    graph made of several components, joined by outer products only."""
    from .circuits import Block
    blocks, off = [], 0
    for c in parts:
        for blk in c.blocks:
            gates = []
            for g in blk.gates:
                if g[0] == "cz":
                    gates.append(("cz", g[1] + off, g[2] + off))
                elif g[0] == "rz":
                    gates.append(("rz", g[1] + off, g[2]))
                else:
                    gates.append((g[0], g[1] + off))
            blocks.append(Block([q + off for q in blk.qubits], gates))
        off += c.n_qubits
    return CutCircuit(off, blocks).finalize()


def serving_set(seed: int = 6, n_circuits: int = 8, n_qubit_range=(200, 1000), n_sub_range=(16, 50),
                K_range=(10, 40), max_width: int = 14, max_log_input: int = 18, n_queries: int = 512,
                a_range=(12, 20), dtype=np.float32) -> BatchWorkload:
    """Resident circuits for the serving loop: seeded random line circuits of
    n_qubit_range qubits cut into n_sub_range subcircuits of at most
    max_width qubits at K_range wires.  With fewer cuts than subcircuits - 1
    the compute graph is a forest of chains.  Outputs are random numbers.
    Each query fixes a random zoom prefix (the lowest 0-2 data qubits of a
    few subcircuits) and asks for a_range active qubits spread over a few
    subcircuits; everything else is merged."""
    rng = np.random.default_rng(seed)
    circuits, probs = [], []
    while len(circuits) < n_circuits:
        n_sub = int(rng.integers(n_sub_range[0], n_sub_range[1] + 1))
        K = int(rng.integers(K_range[0], K_range[1] + 1))
        n_comp = max(1, n_sub - K)
        sizes = [n_sub // n_comp + (1 if i < n_sub % n_comp else 0) for i in range(n_comp)]
        links = sum(s - 1 for s in sizes)
        extra = K - links                     # cuts beyond one per link: spread as wider hand-offs
        parts = []
        ok = True
        for ci, sz in enumerate(sizes):
            h = [1] * (sz - 1)
            for _ in range(max(0, extra) if ci == 0 else 0):
                if not h:
                    break
                j = int(rng.integers(len(h)))
                if h[j] < 3:
                    h[j] += 1
            widths = []
            for b in range(sz):
                hin = h[b - 1] if b > 0 else 0
                hout = h[b] if b < sz - 1 else 0
                wmax = min(max_width, max_log_input - 2 * (hin + hout))
                wmin = hin + hout + 2
                if wmax < wmin:
                    ok = False
                    break
                widths.append(int(rng.integers(max(wmin, wmax - 3), wmax + 1)))
            if not ok:
                break
            parts.append(chain_line_circuit(int(rng.integers(1 << 30)), widths, h, 2) if sz > 1 else
                         chain_line_circuit(int(rng.integers(1 << 30)), widths, [], 2))
        if not ok:
            continue
        c = _merge_components(parts)
        if not (n_qubit_range[0] <= c.n_qubits <= n_qubit_range[1]):
            continue
        circuits.append(c)
        probs.append([random_variant_probs(c, i, rng).astype(dtype) for i in range(c.n_subcircuits)])
    queries = []
    for _ in range(n_queries):
        ci = int(rng.integers(n_circuits))
        c = circuits[ci]
        roles = np.full(c.n_qubits, MERGED, dtype=np.int8)
        nsub = c.n_subcircuits
        zoomed = rng.choice(nsub, size=min(nsub, int(rng.integers(1, 4))), replace=False)
        zoom_n = np.zeros(nsub, dtype=int)
        for i in zoomed:
            zoom_n[i] = int(rng.integers(0, min(3, len(c.data_qubits[i])) + 1))
        a_total = int(rng.integers(a_range[0], a_range[1] + 1))
        hosts = rng.choice(nsub, size=min(nsub, int(rng.integers(2, 6))), replace=False)
        act_n = np.zeros(nsub, dtype=int)
        for _ in range(a_total):
            cand = [i for i in hosts if zoom_n[i] + act_n[i] < len(c.data_qubits[i])]
            if not cand:
                cand = [i for i in range(nsub) if zoom_n[i] + act_n[i] < len(c.data_qubits[i])]
            act_n[int(rng.choice(cand))] += 1
        for i, dq in enumerate(c.data_qubits):
            for q in dq[:zoom_n[i]]:
                roles[q] = ZOOM1 if rng.integers(2) else ZOOM0
            for q in dq[zoom_n[i]:zoom_n[i] + act_n[i]]:
                roles[q] = ACTIVE
        queries.append((ci, roles))
    return BatchWorkload(f"serve{n_circuits}_s{seed}", circuits, probs, queries,
                         {"seed": seed, "n_qubits": [c.n_qubits for c in circuits],
                          "cuts": [c.n_edges for c in circuits], "subcircuits": [c.n_subcircuits for c in circuits]})

"""FP64 CPU oracle for the states-merging reconstruction (test infrastructure).

Only the tests, the smoke check and the CPU-baseline leg of the benchmark use
this module.  It shares no code with the CUDA library and is deliberately
plain: numpy in float64, one step of the method per function, in the order
and notation of the paper.

What it computes (Section 2.1, Eq. 1, with the normalisation and the signed
attribution that the paper leaves to Peng et al. written out):

    P[b] = 2^-K  sum_{e in {I,X,Y,Z}^K}  prod_i  T_i[e|_i, b|_i]

* ``attribute``  -- subcircuit variant outputs -> A_i[e, x]   (Eq. 1, Fig. 1b)
* ``merge``      -- A_i -> T_i[e, b]: merged qubits summed, zoomed qubits
                    fixed (Section 4, Algorithm 2)
* ``reconstruct_bruteforce`` -- the Eq. 1 sum over all 4^K edge assignments,
                    bin by bin
* ``reconstruct_pairwise``   -- the same sum as a sequence of pairwise tensor
                    contractions in subcircuit order (Section 6.1, Fig. 4-5)
* ``top_bins``   -- largest bins, value descending then bin ascending
                    (Algorithm 1, "append the largest bins ... sort and
                    truncate")

Attribution, from rho = 1/2 sum_O Tr(O rho) O on each cut wire:
  upstream, basis O in {I,X,Y,Z}: outcome c weighs +1 for I and (-1)^c for
  X, Y, Z; downstream, O is expanded over the prepared states
  |0>,|1>,|+>,|+i> with the coefficients of ``D`` (I = |0><0|+|1><1|,
  Z = |0><0|-|1><1|, X = 2|+><+| - I, Y = 2|+i><+i| - I); the 1/2 of each
  cut gives the 2^-K.

Index conventions are the boundary's: variant digits over incident edges in
ascending edge id, most significant first; output index y = x | c << n_i;
data-qubit index x little-endian over the subcircuit's data qubits in
ascending original index; a subcircuit's bin index b little-endian over its
active qubits in ascending original index; the reconstructed output index is
little-endian over all active original qubits in ascending order.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

ACTIVE, MERGED, ZOOM0, ZOOM1 = 0, 1, 2, 3

# D[e, s]: cut operator e (rows I, X, Y, Z) expanded over prepared states s
# (columns |0>, |1>, |+>, |+i>).
D = np.array([[1.0, 1.0, 0.0, 0.0],
              [-1.0, -1.0, 2.0, 0.0],
              [-1.0, -1.0, 0.0, 2.0],
              [1.0, -1.0, 0.0, 0.0]])
# W[e, c]: weight of measurement outcome c under basis e.
W = np.array([[1.0, 1.0],
              [1.0, -1.0],
              [1.0, -1.0],
              [1.0, -1.0]])


@dataclass
class Graph:
    """Compute graph (Fig. 3d): subcircuits are vertices, cut edges join an
    upstream to a downstream subcircuit; every original qubit is a data
    qubit of exactly one subcircuit."""
    n_qubits: int
    edge_up: list[int]
    edge_down: list[int]
    data_qubits: list[list[int]]   # per subcircuit, ascending original index

    @property
    def n_subcircuits(self) -> int:
        return len(self.data_qubits)

    @property
    def n_edges(self) -> int:
        return len(self.edge_up)

    def incident(self, i: int) -> list[int]:
        return [e for e in range(self.n_edges) if self.edge_up[e] == i or self.edge_down[e] == i]

    def in_edges(self, i: int) -> list[int]:
        return [e for e in range(self.n_edges) if self.edge_down[e] == i]

    def out_edges(self, i: int) -> list[int]:
        return [e for e in range(self.n_edges) if self.edge_up[e] == i]

    @staticmethod
    def from_arrays(n_qubits, edge_up, edge_down, n_data, data_qubit) -> "Graph":
        dq, off = [], 0
        for n in n_data:
            dq.append([int(q) for q in data_qubit[off:off + n]])
            off += n
        return Graph(int(n_qubits), [int(u) for u in edge_up], [int(d) for d in edge_down], dq)


def attribute(g: Graph, i: int, p: np.ndarray) -> np.ndarray:
    """A_i[e, x] for subcircuit i from its variant outputs p[v, y] (Eq. 1).

    A_i[e, x] = sum_{s, c} prod_{in-edges t} D[e_t, s_t]
                          prod_{out-edges u} W[e_u, c_u]
                          p[variant(s on in-edges, e on out-edges), x | c << n_i]

    The sum factorises over edges, so it is applied one edge at a time:
    each in-edge digit axis is multiplied by D, each out-edge's digit axis
    picks its basis and its outcome axis is summed with the weights W."""
    inc = g.incident(i)
    ins = set(g.in_edges(i))
    outs = g.out_edges(i)
    k, n_i, k_out = len(inc), len(g.data_qubits[i]), len(outs)
    p = np.asarray(p, dtype=np.float64)
    assert p.shape == (4 ** k, 1 << (n_i + k_out)), p.shape
    # axes: one per incident edge digit (first = most significant), then one
    # per outcome bit c_u (highest u first), then x
    t = p.reshape([4] * k + [2] * k_out + [1 << n_i])
    for pos, eid in enumerate(inc):
        if eid in ins:
            t = np.moveaxis(np.tensordot(D, t, axes=([1], [pos])), 0, pos)
    for u, eid in enumerate(outs):
        a = inc.index(eid)
        cb = k + (k_out - 1 - u)          # axis of outcome bit c_u
        q = np.moveaxis(t, (a, cb), (-2, -1))        # [..., 4 (basis e), 2 (c)]
        r = (q * W).sum(axis=-1)                     # [..., 4]
        # put the digit axis back, and a length-1 placeholder where c_u was,
        # so that the remaining axis numbers stay valid
        r = np.expand_dims(r, -1)
        t = np.moveaxis(r, (-2, -1), (a, cb))
    t = t.reshape(4 ** k, 1 << n_i)
    return t


def attribute_literal(g: Graph, i: int, p: np.ndarray) -> np.ndarray:
    """The same A_i written as the literal sum over (e, s, c); slow, for tiny
    subcircuits only."""
    inc = g.incident(i)
    ins = g.in_edges(i)
    outs = g.out_edges(i)
    k, n_i = len(inc), len(g.data_qubits[i])
    A = np.zeros((4 ** k, 1 << n_i))
    for e in range(4 ** k):
        ed = {eid: (e >> (2 * (k - 1 - pos))) & 3 for pos, eid in enumerate(inc)}
        for s in range(4 ** len(ins)):
            sd = {eid: (s >> (2 * (len(ins) - 1 - t))) & 3 for t, eid in enumerate(ins)}
            for c in range(1 << len(outs)):
                coef = 1.0
                for eid in ins:
                    coef *= D[ed[eid], sd[eid]]
                for u, eid in enumerate(outs):
                    coef *= W[ed[eid], (c >> u) & 1]
                if coef == 0.0:
                    continue
                v = 0
                for eid in inc:
                    v = v * 4 + (sd[eid] if eid in sd else ed[eid])
                A[e] += coef * p[v, (c << n_i): (c << n_i) + (1 << n_i)]
    return A


def merge(g: Graph, i: int, A: np.ndarray, roles: np.ndarray) -> np.ndarray:
    """T_i[e, b] = sum over data states x of subcircuit i whose zoomed qubits
    hold their fixed values and whose active qubits spell b (Section 4,
    Algorithm 2: a bin keeps the sum of its states' probabilities)."""
    dq = g.data_qubits[i]
    n_i = len(dq)
    r = np.asarray([roles[q] for q in dq])
    active = [t for t in range(n_i) if r[t] == ACTIVE]
    x = np.arange(1 << n_i)
    keep = np.ones(1 << n_i, dtype=bool)
    for t in range(n_i):
        if r[t] == ZOOM0:
            keep &= ((x >> t) & 1) == 0
        elif r[t] == ZOOM1:
            keep &= ((x >> t) & 1) == 1
    b = np.zeros(1 << n_i, dtype=np.int64)
    for j, t in enumerate(active):
        b |= ((x >> t) & 1) << j
    T = np.zeros((A.shape[0], 1 << len(active)))
    np.add.at(T.T, b[keep], A[:, keep].T)
    return T


def subcircuit_tensors(g: Graph, probs, roles) -> list[np.ndarray]:
    return [merge(g, i, attribute(g, i, probs[i]), roles) for i in range(g.n_subcircuits)]


def active_qubits(roles) -> list[int]:
    return [q for q in range(len(roles)) if roles[q] == ACTIVE]


def reconstruct_bruteforce(g: Graph, T: list[np.ndarray], roles, bins) -> np.ndarray:
    """Eq. 1 bin by bin: P[b] = 2^-K sum over all 4^K edge assignments of the
    product of the subcircuit entries."""
    K = g.n_edges
    act = active_qubits(roles)
    pos = {q: j for j, q in enumerate(act)}
    e = np.arange(4 ** K, dtype=np.int64)
    digit = [(e >> (2 * (K - 1 - eid))) & 3 for eid in range(K)]   # edge 0 most significant
    rows = []
    for i in range(g.n_subcircuits):
        r = np.zeros(4 ** K, dtype=np.int64)
        for eid in g.incident(i):
            r = r * 4 + digit[eid]
        rows.append(r)
    out = np.zeros(len(bins))
    for n, bb in enumerate(bins):
        term = np.ones(4 ** K)
        for i in range(g.n_subcircuits):
            mine = [q for q in g.data_qubits[i] if roles[q] == ACTIVE]
            bi = 0
            for j, q in enumerate(mine):
                bi |= ((int(bb) >> pos[q]) & 1) << j
            term = term * T[i][rows[i], bi]
        out[n] = math.fsum(term) * 2.0 ** (-K)
    return out


def reconstruct_pairwise(g: Graph, T: list[np.ndarray], roles) -> np.ndarray:
    """All bins by contracting the compute graph two vertices at a time
    (Section 6.1): subcircuit 1 with 2, the result with 3, and so on.  Each
    step sums over the cut edges the two share (a matrix product) and keeps
    the rest as outer-product axes.  Returns P over the active qubits,
    little-endian in ascending original index, scaled by 2^-K."""
    K = g.n_edges
    act = active_qubits(roles)

    def as_labelled(i):
        inc = g.incident(i)
        mine = [q for q in g.data_qubits[i] if roles[q] == ACTIVE]
        arr = T[i].reshape([4] * len(inc) + [2] * len(mine))
        labels = [("e", eid) for eid in inc] + [("q", q) for q in reversed(mine)]
        return arr, labels

    R, RL = as_labelled(0)
    for i in range(1, g.n_subcircuits):
        B, BL = as_labelled(i)
        shared = [lab for lab in RL if lab[0] == "e" and lab in BL]
        ax_r = [RL.index(s) for s in shared]
        ax_b = [BL.index(s) for s in shared]
        R = np.tensordot(R, B, axes=(ax_r, ax_b))
        RL = [lab for lab in RL if lab not in shared] + [lab for lab in BL if lab not in shared]
    assert all(lab[0] == "q" for lab in RL), "every cut edge joins two subcircuits"
    order = [RL.index(("q", q)) for q in reversed(act)]
    P = np.transpose(R, order).reshape(-1) if order else R.reshape(1)
    return P * 2.0 ** (-K)


def reconstruct(g: Graph, probs, roles) -> np.ndarray:
    """Attribution, merge and pairwise contraction in FP64."""
    return reconstruct_pairwise(g, subcircuit_tensors(g, probs, roles), roles)


def top_bins(P: np.ndarray, k: int, threshold: float = -math.inf):
    """Bins with P >= threshold, ordered by probability descending, ties by
    bin index ascending, truncated to k.  Returns (bins, probs)."""
    P = np.asarray(P)
    idx = np.nonzero(P >= threshold)[0]
    order = np.lexsort((idx, -P[idx]))
    sel = idx[order][:k]
    return sel.astype(np.int64), P[sel]


def total_probability(P: np.ndarray) -> float:
    return math.fsum(np.asarray(P, dtype=np.float64).tolist())

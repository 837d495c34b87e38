"""Host-side rules of the method, written plainly (test infrastructure).

* ``states_assignment``   -- Algorithm 2: how many bins each subcircuit
                             gets so that their product stays <= M.
* ``roles_for_recursion`` -- the qubit roles that assignment implies
                             (j % l'_i keeps the low bits of the state index
                             active; the rest are merged; the bits a previous
                             recursion fixed are zoomed).
* cost model of Section 6.2 and the greedy first-level slicing of
  Section 6.3, checked against the paper's worked example (Fig. 5, Fig. 6).
"""
from __future__ import annotations

import math

from .reconstruct import ACTIVE, MERGED, ZOOM0, ZOOM1, Graph


def states_assignment(l: list[int], M: int) -> list[int]:
    """Algorithm 2, target-bin loop: while the product of the bin counts
    exceeds M, halve (rounding up) the largest; ties go to the lowest
    subcircuit index."""
    lp = list(l)
    while math.prod(lp) > M:
        i = max(range(len(lp)), key=lambda j: (lp[j], -j))
        if lp[i] == 1:
            break
        lp[i] = -(-lp[i] // 2)
    return lp


def roles_for_recursion(g: Graph, zoom: dict[int, int], M: int) -> list[int]:
    """Roles per original qubit for one recursion.  `zoom` maps the qubits
    fixed by earlier recursions to their bit value.  Within each subcircuit
    the remaining data qubits, in ascending original index, enumerate its
    states j; with l'_i = 2^{a_i} bins, j % l'_i makes the lowest a_i of them
    active and the others merged."""
    free = [[q for q in dq if q not in zoom] for dq in g.data_qubits]
    lp = states_assignment([1 << len(f) for f in free], M)
    roles = [MERGED] * g.n_qubits
    for q, v in zoom.items():
        roles[q] = ZOOM1 if v else ZOOM0
    for i, f in enumerate(free):
        a = int(round(math.log2(lp[i])))
        for q in f[:a]:
            roles[q] = ACTIVE
    return roles


# ---- Section 6.2: memory and multiplications --------------------------------

def tensor_floats(n_cuts: int, n_bins: int) -> int:
    """A subcircuit tensor holds 4^{#cuts} x #bins floats."""
    return 4 ** n_cuts * n_bins


def step_multiplications(dims: list[int]) -> int:
    """A pairwise contraction costs the product of every dimension involved
    (free dims of both operands and the shared dims, each counted once)."""
    return math.prod(dims)


def naive_multiplications(n_edges: int, bins: list[int]) -> int:
    """Eq. 1 evaluated literally: for each of the 4^K assignments, build the
    outer product subcircuit by subcircuit."""
    total, run = 0, bins[0]
    for b in bins[1:]:
        run *= b
        total += run
    return 4 ** n_edges * total


def sliced_sizes(g: Graph, bins: list[int], sliced: set[int]) -> int:
    """Total input floats when the edges in `sliced` are written out
    explicitly (each sliced edge no longer indexes a tensor)."""
    tot = 0
    for i in range(g.n_subcircuits):
        k = len([e for e in g.incident(i) if e not in sliced])
        tot += tensor_floats(k, bins[i])
    return tot


def greedy_slicing(g: Graph, bins: list[int], budget_floats: int) -> list[int]:
    """Section 6.3: keep slicing the edge that reduces the total input size
    the most until it fits the budget; ties go to the lowest edge id."""
    sliced: list[int] = []
    while sliced_sizes(g, bins, set(sliced)) > budget_floats:
        cand = [e for e in range(g.n_edges) if e not in sliced]
        if not cand:
            break
        best = min(cand, key=lambda e: (sliced_sizes(g, bins, set(sliced) | {e}), e))
        sliced.append(best)
    return sliced

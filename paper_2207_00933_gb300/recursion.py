"""Algorithm 1 of the paper as a host-side driver over the library.

Each recursion assigns the states still under analysis to at most M bins
(Algorithm 2, sqc_recursion_roles), reconstructs those bins on the GPU
(sqc_reconstruct), keeps the largest bins (sqc_top_bins), and expands the
most probable bin that is not yet a single state by zooming into it.  A bin
whose qubits are all fixed is a solution state.
"""
from __future__ import annotations

import math

import numpy as np

from . import ROLE_ACTIVE, ROLE_MERGED, ROLE_ZOOM0, ROLE_ZOOM1, Context, recursion_roles


def search(ctx: Context, circuit: int, graph: tuple, M: int, R: int, keep: int = 16, threshold: float = 0.0,
           precision: str = "fp32"):
    """Run at most R recursions on a loaded circuit.
    graph = (n_qubits, edge_up, edge_down, n_data, data_qubit) as loaded.
    Returns (solutions, recursions): solutions = list of (bitstring as a
    list of qubit values, probability) for the single-state bins found."""
    import torch
    n = graph[0]
    zoom = np.full(n, ROLE_MERGED, dtype=np.int8)        # nothing fixed yet
    pending: list[tuple[float, np.ndarray]] = []          # the list L of Algorithm 1
    solutions = []
    r = 0
    while r < R:
        roles = recursion_roles(*graph, zoom, M)
        active = [q for q in range(n) if roles[q] == ROLE_ACTIVE]
        q, na = ctx.set_qubit_roles(circuit, roles)
        bins = torch.empty(1 << na, dtype=torch.float32, device="cuda")
        ctx.reconstruct(q, bins, precision)
        b, v, nf = ctx.top_bins(q, bins, min(keep, 1 << na), threshold)
        torch.cuda.synchronize()
        b, v, nf = b.cpu().numpy(), v.cpu().numpy(), int(nf.item())
        ctx.release_query(q)
        for j in range(nf):
            z = zoom.copy()
            for pos, qb in enumerate(active):
                z[qb] = ROLE_ZOOM1 if (int(b[j]) >> pos) & 1 else ROLE_ZOOM0
            if np.all((z == ROLE_ZOOM0) | (z == ROLE_ZOOM1)):
                solutions.append(([int(x == ROLE_ZOOM1) for x in z], float(v[j])))
            else:
                pending.append((float(v[j]), z))
        r += 1
        # sort and truncate L, then pop the largest bin still to expand
        pending.sort(key=lambda t: -t[0])
        del pending[keep:]
        if not pending:
            break
        _, zoom = pending.pop(0)
    return solutions, r


def recursions_needed(n_qubits: int, M: int, n_solutions: int = 1) -> int:
    """Section 4: with zero-probability non-solutions, at most m n / log2 M
    recursions find m solutions."""
    return n_solutions * math.ceil(n_qubits / math.log2(M))

"""Host-side planner (sqc_plan_preview, no GPU): first-level slicing, the
greedy contraction order on the Section 6.2 cost, and the step shapes.

Pinned to the paper's worked example (Section 6.2, Fig. 5: the order
contracts subcircuits 1 and 2 first, 512 + 2048 multiplications; Section
6.3, Fig. 6: one sliced edge between subcircuits 1 and 3 brings the inputs
to 304 floats) and to the oracle's cost model and greedy slicing on the
test workloads."""
import json
import math
import os

import numpy as np
import pytest

import oracle as O
from synthetic import workloads as W

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


@pytest.fixture(scope="module")
def sqc():
    from paper_2207_00933_gb300 import _build
    _build.build()
    import paper_2207_00933_gb300 as m
    return m


def _fig5():
    gold = json.load(open(os.path.join(GOLDEN, "fig5_cost_model.json")))
    edges, bins = gold["graph"]["edges"], gold["graph"]["bins"]
    n_data = [int(math.log2(b)) for b in bins]               # every data qubit active
    arrays = ([e[0] for e in edges], [e[1] for e in edges], n_data, list(range(sum(n_data))))
    return gold, sum(n_data), arrays, bins


def _bins(c, roles):
    return [1 << sum(1 for q in dq if roles[q] == O.ACTIVE) for dq in c.data_qubits]


def test_fig5_worked_example(sqc):
    gold, nq, arrays, bins = _fig5()
    roles = np.zeros(nq, dtype=np.int8)
    p = sqc.plan_preview(nq, *arrays, roles)
    mults = [m * n * k for m, n, k in p["steps"]]
    assert mults == [gold["multiplications_step1"], gold["multiplications_step2"]]
    assert [k for _, _, k in p["steps"]] == [4, 4 ** 3]        # one shared edge, then three
    assert p["flops"] == 2 * sum(mults)
    assert p["steps"][-1][0] * p["steps"][-1][1] == 1 << nq
    assert round(O.naive_multiplications(len(arrays[0]), bins) / sum(mults), 1) == gold["naive_overhead_ratio_printed"]
    assert p["sliced"] == []


def test_fig6_slicing_by_input_budget(sqc):
    gold, nq, arrays, bins = _fig5()
    g = O.Graph.from_arrays(nq, *arrays)
    roles = np.zeros(nq, dtype=np.int8)
    # a budget of 512 floats: one edge between subcircuits 1 and 3 (304 floats)
    p = sqc.plan_preview(nq, *arrays, roles, slice_input_log2=9)
    assert p["sliced"] == O.greedy_slicing(g, bins, 512)
    assert len(p["sliced"]) == 1 and {arrays[0][p["sliced"][0]], arrays[1][p["sliced"][0]]} == {0, 2}
    assert O.sliced_sizes(g, bins, set(p["sliced"])) == gold["sliced_one_edge_floats"]
    # tighter budgets keep following the same greedy rule
    for lg in (8, 6, 5):
        p = sqc.plan_preview(nq, *arrays, roles, slice_input_log2=lg)
        assert p["sliced"] == O.greedy_slicing(g, bins, 2 ** lg), lg
        assert O.sliced_sizes(g, bins, set(p["sliced"])) <= 2 ** lg
    # with every edge sliced the inputs still hold 2 + 1 + 16 = 19 floats:
    # a 16-float budget cannot be met and the planner refuses it
    from paper_2207_00933_gb300 import SQCError
    assert O.sliced_sizes(g, bins, set(range(len(arrays[0])))) == 19
    with pytest.raises(SQCError) as ei:
        sqc.plan_preview(nq, *arrays, roles, slice_input_log2=4)
    assert ei.value.status == 3
    # a fixed number of sliced edges: the greedy prefix
    p = sqc.plan_preview(nq, *arrays, roles, slice_edges=2)
    assert p["sliced"] == O.greedy_slicing(g, bins, 0)[:2]


def _workloads():
    out = [("line30_K8_a20", W.merged_30q().circuit, W.merged_30q().roles)]
    w = W.grid_40q()
    out.append(("grid40_K12_a22", w.circuit, w.roles))
    for seed in range(6):
        w = W.small_random(seed, n_qubits=12, n_blocks=5, roles="mixed")
        out.append((w.name, w.circuit, w.roles))
    return out


@pytest.fixture(scope="module")
def workloads():
    return _workloads()


def test_step_shapes_and_first_step_cost(sqc, workloads):
    for name, c, roles in workloads:
        g = O.Graph.from_arrays(c.n_qubits, *c.graph_arrays())
        p = sqc.plan_preview(c.n_qubits, *c.graph_arrays(), roles)
        steps = p["steps"]
        na = int(np.sum(roles == O.ACTIVE))
        assert len(steps) == c.n_subcircuits - 1, name
        m, n, _ = steps[-1]
        assert m * n == 1 << na, name
        # every cut edge is contracted exactly once: the shared indices are
        # powers of 4 whose exponents add up to the number of edges
        logs = [int(round(math.log(k, 4))) for _, _, k in steps]
        assert all(4 ** e == k for e, (_, _, k) in zip(logs, steps)), name
        assert sum(logs) == g.n_edges, name
        assert p["flops"] == 2 * sum(a * b * k for a, b, k in steps), name
        # the first step is the cheapest connected pair under the Section 6.2
        # cost (free dims of both operands times the shared dims)
        bins = _bins(c, roles)
        k_of = [len(g.incident(i)) for i in range(g.n_subcircuits)]
        best = None
        for i in range(g.n_subcircuits):
            for j in range(i + 1, g.n_subcircuits):
                sh = sum(1 for e in range(g.n_edges) if {g.edge_up[e], g.edge_down[e]} == {i, j})
                if sh == 0:
                    continue
                cost = O.step_multiplications([4 ** (k_of[i] - sh) * bins[i], 4 ** sh, 4 ** (k_of[j] - sh) * bins[j]])
                best = cost if best is None else min(best, cost)
        if best is not None:
            a, b, k = steps[0]
            assert a * b * k == best, name


def test_greedy_beats_the_literal_sum(sqc, workloads):
    for name, c, roles in workloads[:2]:
        p = sqc.plan_preview(c.n_qubits, *c.graph_arrays(), roles)
        mults = sum(a * b * k for a, b, k in p["steps"])
        assert mults < O.naive_multiplications(len(c.graph_arrays()[0]), _bins(c, roles)), name


def test_intermediate_budget(sqc, workloads):
    for name, c, roles in workloads[:2]:
        p0 = sqc.plan_preview(c.n_qubits, *c.graph_arrays(), roles)
        largest = max(m * n for m, n, _ in p0["steps"][:-1])
        lg = int(math.log2(largest)) - 2
        p = sqc.plan_preview(c.n_qubits, *c.graph_arrays(), roles, slice_intermediate_log2=lg)
        assert p["sliced"], name
        assert max(m * n for m, n, _ in p["steps"][:-1]) <= 2 ** lg, name
        # slicing removes the sliced edges from every step
        assert sum(int(round(math.log(k, 4))) for _, _, k in p["steps"]) == \
            len(c.graph_arrays()[0]) - len(p["sliced"]), name


def test_errors(sqc, workloads):
    from paper_2207_00933_gb300 import SQCError
    _, c, roles = workloads[0]
    arr = c.graph_arrays()
    with pytest.raises(SQCError) as ei:
        sqc.plan_preview(c.n_qubits, *arr, roles, slice_input_log2=1)          # needs > 8 sliced edges
    assert ei.value.status == 3 and "slicing" in str(ei.value)
    with pytest.raises(SQCError) as ei:
        sqc.plan_preview(c.n_qubits, *arr, roles, max_active_qubits=4)
    assert ei.value.status == 3
    with pytest.raises(SQCError) as ei:
        sqc.plan_preview(c.n_qubits, *arr, roles, chunk_terms=3)
    assert ei.value.status == 1 and "chunk_terms" in str(ei.value)
    bad = roles.copy()
    bad[0] = 9
    with pytest.raises(SQCError) as ei:
        sqc.plan_preview(c.n_qubits, *arr, bad)
    assert ei.value.status == 1
    with pytest.raises(SQCError) as ei:
        sqc.plan_preview(c.n_qubits, arr[0], arr[1], arr[2], arr[3][::-1].copy() * 0, roles)   # not a permutation
    assert ei.value.status == 1


def test_fewest_multiplications_order_is_never_costlier(sqc):
    """The exact order (dynamic programming over subsets) needs at most the
    greedy order's multiplications on every query, and strictly fewer on
    some, with the same number of steps and the same result size."""
    from synthetic import workloads as W
    fewer = 0
    for seed in range(30):
        w = W.small_random(seed, n_qubits=14, n_blocks=7, max_block=5, roles="mixed")
        c = w.circuit
        g = sqc.plan_preview(c.n_qubits, *c.graph_arrays(), w.roles)
        d = sqc.plan_preview(c.n_qubits, *c.graph_arrays(), w.roles, contraction_order=1)
        assert d["flops"] <= g["flops"]
        assert len(d["steps"]) == len(g["steps"])
        gm, gn, _ = g["steps"][-1]
        dm, dn, _ = d["steps"][-1]
        assert gm * gn == dm * dn
        fewer += d["flops"] < g["flops"]
    assert fewer > 0

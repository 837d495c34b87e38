"""GPU parity: the CUDA reconstruction through the C ABI against the FP64
oracle on the same seeded inputs.

Tolerance: 1e-6 max-abs probability error (the stated target), and a
relative bound derived from the arithmetic: every bin is a sum of products
accumulated in FP32 (unit roundoff 6e-8) over at most a few hundred terms
per step, so the error stays below ~1e-5 of the largest bin; tighter where
noted.  Bin selection and indexing are compared exactly."""
import math

import numpy as np
import pytest

import oracle as O
from synthetic import full_circuit_probs, workloads as W

pytestmark = pytest.mark.gpu

ABS_TOL = 1e-6
REL_TOL = 1e-5
# bins that are exactly zero in exact arithmetic come out of the FP64 oracle as
# rounding noise of ~1e-17 (sums of products of order-one terms): the
# relative check allows that much absolute difference
ORACLE_FLOOR = 1e-15


@pytest.fixture(scope="module")
def ctx():
    import torch
    from paper_2207_00933_gb300 import Context, _build
    _build.build()
    c = Context(0)
    yield c
    torch.cuda.synchronize()
    c.close()


def graph_of(c):
    return O.Graph.from_arrays(c.n_qubits, *c.graph_arrays())


def gpu_run(ctx, w, roles=None, out_dtype="float32", precision="fp32", host_inputs=False):
    import torch
    c = w.circuit
    roles = w.roles if roles is None else roles
    eu, ed, nd, dq = c.graph_arrays()
    probs = [p if host_inputs else torch.from_numpy(np.ascontiguousarray(p)).cuda() for p in w.probs]
    cid = ctx.load_subcircuit_outputs(c.n_qubits, eu, ed, nd, dq, probs)
    qid, na = ctx.set_qubit_roles(cid, roles)
    out = torch.empty(1 << na, dtype=getattr(torch, out_dtype), device="cuda")
    tot = torch.zeros(1, dtype=torch.float64, device="cuda")
    ctx.reconstruct(qid, out, precision, tot)
    torch.cuda.synchronize()
    res = out.double().cpu().numpy(), float(tot.item())
    ctx.unload(cid)
    return res


def oracle_run(w, roles=None):
    roles = w.roles if roles is None else roles
    probs = [p.astype(np.float64) for p in w.probs]
    return O.reconstruct(graph_of(w.circuit), probs, roles)


def check(P, ref, rel=REL_TOL):
    err = np.abs(P - ref).max()
    scale = np.abs(ref).max()
    assert err <= ABS_TOL, err
    # relative to the largest bin
    assert err <= rel * scale + ORACLE_FLOOR, (err, scale)
    return err


def test_full_state_12q(ctx):
    w = W.full_state_12q()
    P, tot = gpu_run(ctx, w)
    ref = oracle_run(w)
    check(P, ref)
    assert np.abs(P - full_circuit_probs(w.circuit)).max() < 1e-6
    assert abs(tot - 1.0) < 1e-5
    assert abs(tot - math.fsum(P)) < 1e-9


@pytest.mark.parametrize("seed", range(12))
def test_random_graphs_mixed_roles(ctx, seed):
    w = W.small_random(seed, roles="mixed")
    P, _ = gpu_run(ctx, w)
    check(P, oracle_run(w))


@pytest.mark.parametrize("seed", range(6))
def test_random_graphs_all_active_vs_statevector(ctx, seed):
    w = W.small_random(seed + 100, n_qubits=10, n_blocks=5, roles="active")
    P, tot = gpu_run(ctx, w, out_dtype="float64")
    check(P, full_circuit_probs(w.circuit))
    assert abs(tot - 1.0) < 1e-5


def test_merged_30q_all_bins(ctx):
    w = W.merged_30q()
    P, tot = gpu_run(ctx, w)
    ref = oracle_run(w)
    assert P.size == 1 << 20
    check(P, ref)
    assert abs(tot - O.total_probability(ref)) < 1e-6


def test_merged_30q_host_inputs_fp64_out(ctx):
    w = W.merged_30q()
    P, _ = gpu_run(ctx, w, out_dtype="float64", host_inputs=True)
    check(P, oracle_run(w))


def test_grid_40q_fp64_chunked(ctx):
    w = W.grid_40q()
    P, tot = gpu_run(ctx, w, out_dtype="float64")
    ref = oracle_run(w)
    assert P.size == 1 << 22
    check(P, ref)
    assert abs(tot - O.total_probability(ref)) < 1e-6


@pytest.mark.parametrize("wl,out", [("merged_30q", "float32"), ("grid_40q", "float64"), ("full_state_12q", "float32")])
def test_split_bf16_matches_oracle(ctx, wl, out):
    # split-BF16 (three BF16 planes, six products) on tcgen05 for the steps
    # with M, N >= 128; FP32 SIMT for the rest
    w = getattr(W, wl)()
    P, tot = gpu_run(ctx, w, out_dtype=out, precision="split_bf16")
    ref = oracle_run(w)
    check(P, ref)
    assert abs(tot - O.total_probability(ref)) < 1e-6


def test_split_bf16_contraction_bound_step(ctx):
    # two subcircuits sharing 4 cut edges: one 1024 x 1024 x 256 step on the
    # tensor cores (four 64-wide K blocks through the two-stage pipeline)
    w = W.random_line_chain(7, [14, 14], [4], 2, [10, 10])
    assert w.circuit.n_edges == 4 and w.n_active == 20
    ref = oracle_run(w)
    for prec in ("split_bf16", "fp32"):
        P, tot = gpu_run(ctx, w, precision=prec)
        check(P, ref)


@pytest.mark.parametrize("active,out", [((12, 12), "float32"), ((12, 12), "float64"), ((11, 12), "float32")])
def test_split_bf16_wide_tiles(ctx, active, out):
    # 4096 x 4096 x 256 (and 2048 x 4096): enough 128 x 256 tiles to fill
    # every SM, so the tensor-core step runs the 256-wide, 32-deep,
    # three-stage configuration (64-byte swizzle) in 2-CTA pairs.  At 4096 x
    # 4096 the 256 pair units leave a last wave of 28 on 76 clusters, which
    # runs as 56 half-width units; at 2048 x 4096 (128 units, a tail of 52)
    # every unit is full width
    w = W.random_line_chain(11, [16, 16], [4], 1, list(active))
    ref = oracle_run(w)
    P, tot = gpu_run(ctx, w, out_dtype=out, precision="split_bf16")
    check(P, ref)
    # the FP64 check sums exactly the bins that were written
    assert abs(tot - O.total_probability(P)) < 1e-9
    # and drifts from the oracle's total only by the tensor cores' FP32
    # accumulation, which may drop up to one unit in the last place (2^-23
    # relative) per accumulation step, always toward zero: the step adds
    # 6 products x Kp/16 MMAs into one accumulator, so the drift of a total
    # near 1 is at most 6 * (256 / 16) * 2^-23 = 1.1e-5
    assert abs(tot - O.total_probability(ref)) <= 6 * (256 // 16) * 2.0 ** -23


def test_zoomed_children_sum_to_parent(ctx):
    w = W.merged_30q()
    q = w.circuit.data_qubits[2][6]
    assert w.roles[q] == O.MERGED
    parent, _ = gpu_run(ctx, w)
    kids = []
    for role in (O.ZOOM0, O.ZOOM1):
        r = w.roles.copy()
        r[q] = role
        kids.append(gpu_run(ctx, w, roles=r)[0])
        check(kids[-1], oracle_run(w, r))
    assert np.abs(kids[0] + kids[1] - parent).max() < 1e-9


def test_single_subcircuit_no_cuts(ctx):
    from synthetic.circuits import Block, CutCircuit
    from synthetic.workloads import Workload
    from synthetic import subcircuit_variant_probs
    c = CutCircuit(6, [Block(list(range(6)), [("h", 0), ("cz", 0, 1), ("sx", 3), ("t", 1), ("sy", 5)])]).finalize()
    w = Workload("one", c, [subcircuit_variant_probs(c, 0)], np.array([0, 1, 0, 2, 0, 3], dtype=np.int8))
    P, tot = gpu_run(ctx, w)
    check(P, oracle_run(w))


def test_all_merged_gives_one(ctx):
    w = W.full_state_12q(4)
    roles = np.full(w.circuit.n_qubits, O.MERGED, dtype=np.int8)
    P, tot = gpu_run(ctx, w, roles=roles, out_dtype="float64")
    assert P.shape == (1,)
    assert abs(P[0] - 1.0) < 1e-6 and abs(tot - 1.0) < 1e-6


def test_top_bins_matches_oracle_exactly(ctx):
    import torch
    w = W.merged_30q()
    c = w.circuit
    probs = [torch.from_numpy(p).cuda() for p in w.probs]
    cid = ctx.load_subcircuit_outputs(c.n_qubits, *c.graph_arrays(), probs)
    qid, na = ctx.set_qubit_roles(cid, w.roles)
    out = torch.empty(1 << na, dtype=torch.float32, device="cuda")
    ctx.reconstruct(qid, out)
    P = out.double().cpu().numpy()
    for k, thr in ((1, -math.inf), (10, -math.inf), (1000, -math.inf), (4096, -math.inf), (50, 3e-6),
                   (4096, 1e-6)):
        b, v, n = ctx.top_bins(qid, out, k, thr)
        torch.cuda.synchronize()
        nf = int(n.item())
        eb, ev = O.top_bins(P, k, thr)          # same FP32 values, compared as FP64
        assert nf == eb.size
        assert b[:nf].cpu().numpy().tolist() == eb.tolist()
        assert np.array_equal(v[:nf].cpu().numpy(), ev)
    # the GPU's selection agrees with the FP64 oracle's up to near-ties:
    # every bin that only one of the two selected lies within 2x the
    # measured max-abs error of the oracle's k-th value, and the selected
    # bins agree where the values are separated by more than that
    ref = oracle_run(w)
    err = np.abs(P - ref).max()
    for k in (1, 64, 1000, 4096):
        eb, ev = O.top_bins(ref, k)
        b, v, n = ctx.top_bins(qid, out, k)
        torch.cuda.synchronize()
        gb = b[: int(n.item())].cpu().numpy()
        assert gb.size == eb.size == k
        kth = ev[-1]
        for bb in set(gb.tolist()) ^ set(eb.tolist()):
            assert abs(ref[bb] - kth) <= 2 * err, (k, bb, ref[bb], kth, err)
        # bins clearly above the k-th value are selected by both
        sure = set(np.nonzero(ref > kth + 2 * err)[0].tolist())
        assert sure <= set(gb.tolist()) and sure <= set(eb.tolist())
    ctx.unload(cid)


@pytest.mark.parametrize("dtype", ["float32", "float64"])
def test_top_bins_ties_and_edges(ctx, dtype):
    import torch
    rng = np.random.default_rng(5)
    n = 300_000
    x = rng.integers(0, 7, n).astype(dtype) * 0.125        # heavy exact ties
    x[rng.integers(0, n, 40)] = 2.0
    w = W.full_state_12q()
    c = w.circuit
    cid = ctx.load_subcircuit_outputs(c.n_qubits, *c.graph_arrays(), [torch.from_numpy(p).cuda() for p in w.probs])
    qid, _ = ctx.set_qubit_roles(cid, w.roles)
    xd = torch.from_numpy(x).cuda()
    for k, thr in ((1, -math.inf), (37, -math.inf), (100, -math.inf), (4096, -math.inf), (4096, 0.7),
                   (5, 3.0), (4096, 0.0)):
        b, v, nf = ctx.top_bins(qid, xd, k, thr)
        torch.cuda.synchronize()
        eb, ev = O.top_bins(x.astype(np.float64), k, thr)
        m = int(nf.item())
        assert m == eb.size
        assert b[:m].cpu().numpy().tolist() == eb.tolist()
        assert np.array_equal(v[:m].cpu().numpy(), ev)
    # a group of exact ties at the top that fits the candidate capacity
    # (ranked by bin inside one bucket), above a continuous tail
    y = rng.random(1 << 20).astype(dtype) * 0.5
    y[rng.choice(y.size, 2000, replace=False)] = 3.0
    yd = torch.from_numpy(y).cuda()
    for k, thr in ((1024, -math.inf), (2000, -math.inf), (2048, -math.inf), (7, 3.0)):
        b, v, nf = ctx.top_bins(qid, yd, k, thr)
        torch.cuda.synchronize()
        eb, ev = O.top_bins(y.astype(np.float64), k, thr)
        m = int(nf.item())
        assert m == eb.size
        assert b[:m].cpu().numpy().tolist() == eb.tolist()
        assert np.array_equal(v[:m].cpu().numpy(), ev)
    # empty and tiny inputs
    for m in (1, 3):
        y = torch.from_numpy(x[:m].copy()).cuda()
        b, v, nf = ctx.top_bins(qid, y, 10)
        torch.cuda.synchronize()
        assert int(nf.item()) == m
    ctx.unload(cid)


def test_errors_are_reported(ctx):
    import torch
    from paper_2207_00933_gb300 import SQCError
    w = W.full_state_12q()
    c = w.circuit
    cid = ctx.load_subcircuit_outputs(c.n_qubits, *c.graph_arrays(), [torch.from_numpy(p).cuda() for p in w.probs])
    with pytest.raises(SQCError) as ei:
        ctx.set_qubit_roles(cid, np.full(c.n_qubits, 7, dtype=np.int8))
    assert ei.value.status == 1
    qid, na = ctx.set_qubit_roles(cid, w.roles)
    small = torch.empty(10, dtype=torch.float32, device="cuda")
    with pytest.raises(SQCError) as ei:
        ctx.reconstruct(qid, small)
    assert ei.value.status == 3
    with pytest.raises(SQCError) as ei:
        ctx.top_bins(qid, small, 0)
    assert ei.value.status == 3
    ctx.unload(cid)
    with pytest.raises(SQCError) as ei:
        ctx.reconstruct(qid, small)
    assert ei.value.status == 7


def test_hbm_budget_admission(ctx):
    import torch
    from paper_2207_00933_gb300 import Context, SQCError
    w = W.merged_30q()
    c = w.circuit
    with Context(0, hbm_budget_bytes=1 << 20) as small:   # the circuit needs ~2.7 MB
        with pytest.raises(SQCError) as ei:
            small.load_subcircuit_outputs(c.n_qubits, *c.graph_arrays(), [torch.from_numpy(p).cuda() for p in w.probs])
        assert ei.value.status == 6


@pytest.mark.parametrize("wl,out", [("merged_30q", "float32"), ("grid_40q", "float64"), ("full_state_12q", "float64")])
def test_single_launch_equals_per_stage_launches(wl, out):
    """An FP32 query runs its merge and every contraction step as one
    persistent launch (the default) or as one launch per stage: every bin is
    summed by one thread in the same order either way, so the bins are the
    same bit for bit, and both match the oracle; the FP64 probability sums
    agree to rounding."""
    import torch
    from paper_2207_00933_gb300 import Context
    w = getattr(W, wl)()
    ref = oracle_run(w)
    res = {}
    for fused in (True, False):
        with Context(0, fused_query=fused) as c:
            P, tot = gpu_run(c, w, out_dtype=out)
            res[fused] = (P, tot)
    assert np.array_equal(res[True][0], res[False][0])
    check(res[True][0], ref)
    assert abs(res[True][1] - res[False][1]) <= 1e-12
    torch.cuda.synchronize()


@pytest.mark.parametrize("seed", range(6))
def test_fewest_multiplications_order_matches_oracle(seed):
    """Plans under the fewest-multiplications contraction order (exact search
    over subsets of subcircuits, Section 6.2 cost) reconstruct the oracle's
    bins in both precisions, on random compute graphs with mixed roles."""
    from paper_2207_00933_gb300 import Context
    w = W.small_random(seed + 40, n_qubits=12, n_blocks=6, max_block=5, roles="mixed")
    ref = oracle_run(w)
    with Context(0, contraction_order=1) as c:
        for prec in ("fp32", "split_bf16"):
            P, _ = gpu_run(c, w, out_dtype="float64", precision=prec)
            check(P, ref)

"""GPU parity of one recursion step in one call (sqc_reconstruct_select):
the bins of a query and the selection of its largest bins (Algorithm 1:
reconstruct, then keep the largest bins), with the contraction steps, the
bins and the selection fused into one cooperative launch where the plan
allows it.

Every case is checked three ways: against the separate calls on the same
context (sqc_reconstruct + sqc_top_bins: the bins, the selected bins, their
values and count bit for bit), the selection against the oracle's exact
ordering of the GPU's own FP32 bins, and the bins against the FP64 oracle
(Eq. 1) element by element.  The probability sum is checked against the
exactly rounded sum of the written bins within the bound of recursive FP64
summation, (n - 1) u sum |P|."""
import math

import numpy as np
import pytest

import oracle as O
from synthetic import workloads as W

pytestmark = pytest.mark.gpu

ABS_TOL = 1e-6
REL_TOL = 1e-5
U64 = 2.0 ** -53


def _oracle(c, probs, roles):
    return O.reconstruct(O.Graph.from_arrays(c.n_qubits, *c.graph_arrays()), [p.astype(np.float64) for p in probs],
                         roles)


def _load(ctx, w, host=False):
    """Load the outputs (from host arrays: the circuit then keeps a staging
    buffer for later host inputs) and set the roles."""
    import torch
    c = w.circuit
    src = list(w.probs) if host else [torch.from_numpy(p).cuda() for p in w.probs]
    cid = ctx.load_subcircuit_outputs(c.n_qubits, *c.graph_arrays(), src)
    qid, na = ctx.set_qubit_roles(cid, w.roles)
    return cid, qid, na


def _step(ctx, qid, na, k, thr, fresh=None, out_dtype="float32"):
    """(bins written, selected bins, values, count, total) of one fused call."""
    import torch
    out = torch.full((1 << na,), -3.0, dtype=getattr(torch, out_dtype), device="cuda")
    tot = torch.zeros(1, dtype=torch.float64, device="cuda")
    b, v, n = ctx.reconstruct_select(qid, out, k, thr, probs=fresh, total_prob=tot)
    torch.cuda.synchronize()
    m = int(n.item())
    return out, b[:m].cpu().numpy(), v[:m].cpu().numpy(), m, tot.item()


def _separate(ctx, qid, na, k, thr, fresh=None, out_dtype="float32"):
    import torch
    out = torch.full((1 << na,), -3.0, dtype=getattr(torch, out_dtype), device="cuda")
    tot = torch.zeros(1, dtype=torch.float64, device="cuda")
    if fresh is None:
        ctx.reconstruct(qid, out, "fp32", tot)
    else:
        ctx.reconstruct_outputs(qid, fresh, out, "fp32", tot)
    b, v, n = ctx.top_bins(qid, out, k, thr)
    torch.cuda.synchronize()
    m = int(n.item())
    return out, b[:m].cpu().numpy(), v[:m].cpu().numpy(), m, tot.item()


def _check(ctx, qid, na, ref, ks, fresh=None, out_dtype="float32", fused=True):
    """fused: the call runs the fused launch, whose probability sum adds the
    FP32 bins in FP64 (the separate stages add up to 16 bins per thread in
    FP32 first: checked at 1e-5 relative)."""
    import torch
    for k, thr in ks:
        out, b, v, m, tot = _step(ctx, qid, na, k, thr, fresh, out_dtype)
        out2, b2, v2, m2, tot2 = _separate(ctx, qid, na, k, thr, fresh, out_dtype)
        assert torch.equal(out, out2)
        assert m == m2 and b.tolist() == b2.tolist() and np.array_equal(v, v2)
        P = out.double().cpu().numpy()
        eb, ev = O.top_bins(P, k, thr)
        assert m == eb.size and b.tolist() == eb.tolist() and np.array_equal(v, ev)
        exact = O.total_probability(P)
        bound = (P.size - 1) * U64 * float(np.abs(P).sum())
        if fused:
            assert abs(tot - exact) <= bound, (tot, exact, bound)
        else:
            assert abs(tot - exact) <= 1e-5 * max(1.0, abs(exact))
        assert abs(tot2 - exact) <= 1e-5 * max(1.0, abs(exact))
        err = float(np.abs(P - ref).max())
        assert err <= ABS_TOL and err <= REL_TOL * float(np.abs(ref).max()) + 1e-15, err


def _profile_launches(ctx, fn):
    ctx.profile_enable(True)
    fn()
    import torch
    torch.cuda.synchronize()
    r = ctx.profile_read()
    ctx.profile_enable(False)
    return r


def test_line30_resident_and_fresh():
    """The 30-qubit, 2^20-bin step: the two 32 x 512 x 64 steps run as the
    first level inside the launch, the 1024 x 1024 x 16 bins per CTA slice."""
    import torch
    from paper_2207_00933_gb300 import Context
    w = W.merged_30q()
    c = w.circuit
    ref = _oracle(c, w.probs, w.roles)
    with Context(0) as ctx:
        cid, qid, na = _load(ctx, w, host=True)
        steps = ctx.query_steps(qid)
        assert ctx.query_fused_select(qid) == len(steps) == 3
        ks = [(1, -math.inf), (1000, -math.inf), (4096, -math.inf), (50, 3e-6), (4096, 1e-6), (10, 1.0)]
        _check(ctx, qid, na, ref, ks)
        # one merge launch and one fused launch
        r = _profile_launches(ctx, lambda: _step(ctx, qid, na, 1000, -math.inf))
        assert r["launches"] == 2 and r["calls"]["select"] == 1 and r["calls"]["final"] == 0
        # fresh outputs (one recursion step): device and host inputs
        rng = np.random.default_rng(8)
        fresh = [(p * (1.0 + 0.25 * rng.random(p.shape))).astype(np.float32) for p in w.probs]
        ref_f = _oracle(c, fresh, w.roles)
        _check(ctx, qid, na, ref_f, [(1000, -math.inf)], fresh=[torch.from_numpy(p).cuda() for p in fresh])
        _check(ctx, qid, na, ref_f, [(4096, -math.inf)], fresh=fresh)
        r = _profile_launches(ctx, lambda: _step(ctx, qid, na, 1000, -math.inf,
                                                 fresh=[torch.from_numpy(p).cuda() for p in fresh]))
        assert r["calls"]["select"] == 1 and r["calls"]["contract"] == 0 and r["calls"]["final"] == 0
        # the resident tensors are untouched by the fresh-output steps
        _check(ctx, qid, na, ref, [(100, -math.inf)])
        ctx.unload(cid)


def test_chain_of_six_several_levels():
    """Five steps over three or more dependency levels: the grid barriers
    between levels inside the launch."""
    from paper_2207_00933_gb300 import Context
    w = W.random_line_chain(11, [7, 8, 8, 8, 8, 6], [2, 2, 2, 2, 2], 1, [3, 3, 3, 3, 3, 3])
    ref = _oracle(w.circuit, w.probs, w.roles)
    with Context(0) as ctx:
        cid, qid, na = _load(ctx, w)
        assert ctx.query_fused_select(qid) == len(ctx.query_steps(qid)) == 5
        _check(ctx, qid, na, ref, [(500, -math.inf), (4096, 0.0)])
        ctx.unload(cid)


def _two_components(seed: int):
    """A two-subcircuit chain with 11 + 11 active qubits next to a separate
    one-block circuit with every qubit merged: the first step is a 2048 x
    2048 output (128 x 128 tiles in the launch), the last an outer product
    with a shared index of one value (2^22 bins)."""
    from synthetic.circuits import chain_line_circuit
    from synthetic.workloads import Workload, _merge_components, lowest_active_roles
    from synthetic import random_variant_probs
    c = _merge_components([chain_line_circuit(seed, [12, 12], [1], 1), chain_line_circuit(seed + 1, [3], [], 1)])
    rng = np.random.default_rng(seed)
    probs = [random_variant_probs(c, i, rng).astype(np.float32) for i in range(c.n_subcircuits)]
    roles = lowest_active_roles(c, [11, 11, 0])
    return Workload(f"twocomp_s{seed}", c, probs, roles, {"seed": seed})


def test_large_first_level_and_outer_product():
    from paper_2207_00933_gb300 import Context
    w = _two_components(21)
    ref = _oracle(w.circuit, w.probs, w.roles)
    with Context(0) as ctx:
        cid, qid, na = _load(ctx, w)
        steps = ctx.query_steps(qid)
        assert na == 22 and len(steps) == 2
        M, N, K = steps[0]
        assert ((M + 127) // 128) * ((N + 127) // 128) >= 152      # the 128 x 128 tile shape
        assert steps[-1][2] == 1                                   # outer product
        assert ctx.query_fused_select(qid) == 2
        _check(ctx, qid, na, ref, [(4096, -math.inf), (7, -math.inf)])
        ctx.unload(cid)


@pytest.mark.parametrize("seed", [3, 4, 7])
def test_interleaved_bins(seed):
    """Random block circuits: each operand of the last step owns scattered
    bits of the bin index (several runs)."""
    from paper_2207_00933_gb300 import Context
    w = W.small_random(seed, n_qubits=14, n_blocks=4, max_block=6, dtype=np.float32)
    ref = _oracle(w.circuit, w.probs, w.roles)
    with Context(0) as ctx:
        cid, qid, na = _load(ctx, w)
        n_steps = len(ctx.query_steps(qid))
        if n_steps == 0:
            pytest.skip("one subcircuit")
        assert ctx.query_fused_select(qid) == n_steps
        _check(ctx, qid, na, ref, [(100, -math.inf), (4096, -math.inf)])
        ctx.unload(cid)


def test_uniform_exact_ties():
    """Hadamards only: every one of the 2^16 bins is exactly 2^-16, so the
    selection takes the lowest bin indices (ties in ascending bin order,
    more ties than the candidate capacity)."""
    from synthetic.circuits import Block, CutCircuit
    from synthetic.workloads import Workload
    from synthetic import subcircuit_variant_probs
    from paper_2207_00933_gb300 import Context
    c = CutCircuit(16, [Block(list(range(9)), [("h", q) for q in range(9)]),
                        Block(list(range(8, 16)), [("h", q) for q in range(9, 16)])]).finalize()
    probs = [subcircuit_variant_probs(c, i).astype(np.float32) for i in range(2)]
    w = Workload("hadamard16", c, probs, np.zeros(16, dtype=np.int8))
    ref = _oracle(c, probs, w.roles)
    assert np.allclose(ref, 2.0 ** -16, atol=1e-15)
    with Context(0) as ctx:
        cid, qid, na = _load(ctx, w)
        assert ctx.query_fused_select(qid) == 1
        _check(ctx, qid, na, ref, [(100, -math.inf), (4096, -math.inf), (4096, 2.0 ** -16)])
        out, b, v, m, _ = _step(ctx, qid, na, 100, -math.inf)
        assert b.tolist() == list(range(100)) and np.all(v == 2.0 ** -16)
        ctx.unload(cid)


def test_forms_that_run_separately():
    """Where the fused launch does not apply -- the option off, a sliced
    plan, FP64 output, split-BF16 -- the call runs the separate stages and
    gives their results."""
    import torch
    from paper_2207_00933_gb300 import Context
    w = W.merged_30q()
    ref = _oracle(w.circuit, w.probs, w.roles)
    with Context(0, fused_select=False) as ctx:
        cid, qid, na = _load(ctx, w)
        assert ctx.query_fused_select(qid) == 0
        _check(ctx, qid, na, ref, [(1000, -math.inf)], fused=False)
        r = _profile_launches(ctx, lambda: _step(ctx, qid, na, 1000, -math.inf))
        assert r["calls"]["final"] == 1 and r["calls"]["select"] == 1
        ctx.unload(cid)
    with Context(0, slice_edges=1) as ctx:
        cid, qid, na = _load(ctx, w)
        assert ctx.query_fused_select(qid) == 0
        _check(ctx, qid, na, ref, [(1000, -math.inf)], fused=False)
        ctx.unload(cid)
    with Context(0) as ctx:
        cid, qid, na = _load(ctx, w)
        assert ctx.query_fused_select(qid) == 3
        # FP64 bins: separate stages, same selection as top_bins on them
        _check(ctx, qid, na, ref, [(1000, -math.inf)], out_dtype="float64", fused=False)
        # split-BF16
        out = torch.empty(1 << na, dtype=torch.float32, device="cuda")
        b, v, n = ctx.reconstruct_select(qid, out, 1000, precision="split_bf16")
        out2 = torch.empty_like(out)
        ctx.reconstruct(qid, out2, "split_bf16")
        b2, v2, n2 = ctx.top_bins(qid, out2, 1000)
        torch.cuda.synchronize()
        assert torch.equal(out, out2) and torch.equal(b, b2) and torch.equal(v, v2)
        ctx.unload(cid)


def test_pinned_host_inputs_read_in_place():
    """Fresh outputs in pinned host memory read in place by the kernels
    (probs_on_device == 2, no staging copy): the same bins and selection as
    from device copies of the same outputs; pageable host memory is refused
    in that mode."""
    import torch
    from paper_2207_00933_gb300 import Context, SQCError
    w = W.merged_30q()
    c = w.circuit
    rng = np.random.default_rng(9)
    fresh = [(p * (1.0 + 0.25 * rng.random(p.shape))).astype(np.float32) for p in w.probs]
    ref = _oracle(c, fresh, w.roles)
    with Context(0) as ctx:
        cid, qid, na = _load(ctx, w)
        pinned = [torch.from_numpy(p).pin_memory() for p in fresh]
        on_dev = [torch.from_numpy(p).cuda() for p in fresh]
        for k in (1024, 4096):
            out = torch.empty(1 << na, dtype=torch.float32, device="cuda")
            tot = torch.zeros(1, dtype=torch.float64, device="cuda")
            b, v, n = ctx.reconstruct_select(qid, out, k, probs=pinned, total_prob=tot, host_direct=True)
            torch.cuda.synchronize()
            out2 = torch.empty_like(out)
            tot2 = torch.zeros_like(tot)
            b2, v2, n2 = ctx.reconstruct_select(qid, out2, k, probs=on_dev, total_prob=tot2)
            torch.cuda.synchronize()
            assert torch.equal(out, out2) and torch.equal(b, b2) and torch.equal(v, v2) and torch.equal(n, n2)
            assert tot.item() == tot2.item()
            err = float(np.abs(out.double().cpu().numpy() - ref).max())
            assert err <= ABS_TOL, err
        # the separate-call form reads pinned inputs in place too
        out3 = torch.empty(1 << na, dtype=torch.float32, device="cuda")
        ctx.reconstruct_outputs(qid, pinned, out3, host_direct=True)
        torch.cuda.synchronize()
        assert torch.equal(out3, out2)
        ctx.unload(cid)
        # pinned host inputs staged by the SMs' copy kernel (the default for
        # mapped pinned memory): loads, updates and fresh steps
        cid = ctx.load_subcircuit_outputs(c.n_qubits, *c.graph_arrays(), [torch.from_numpy(p).pin_memory()
                                                                             for p in w.probs])
        qid, na = ctx.set_qubit_roles(cid, w.roles)
        out4 = torch.empty(1 << na, dtype=torch.float32, device="cuda")
        ctx.reconstruct(qid, out4)
        torch.cuda.synchronize()
        err = float(np.abs(out4.double().cpu().numpy() - _oracle(c, w.probs, w.roles)).max())
        assert err <= ABS_TOL, err
        b4, v4, n4 = ctx.reconstruct_select(qid, out4, 1024, probs=pinned)
        torch.cuda.synchronize()
        b2, v2, n2 = ctx.reconstruct_select(qid, out2, 1024, probs=on_dev)
        torch.cuda.synchronize()
        assert torch.equal(out4, out2) and torch.equal(b4, b2) and torch.equal(v4, v2)
        # an update from staged pinned inputs and one from device copies of
        # the same outputs leave the same resident tensors
        ctx.update_subcircuit_outputs(cid, pinned)
        ctx.reconstruct(qid, out4)
        ctx.update_subcircuit_outputs(cid, on_dev)
        out5 = torch.empty_like(out4)
        ctx.reconstruct(qid, out5)
        torch.cuda.synchronize()
        assert torch.equal(out4, out5)
        err = float(np.abs(out4.double().cpu().numpy() - ref).max())
        assert err <= ABS_TOL, err
        with pytest.raises(SQCError) as ei:
            ctx.reconstruct_select(qid, out3, 10, probs=list(fresh), host_direct=True)
        assert ei.value.status == 1
        ctx.unload(cid)

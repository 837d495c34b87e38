"""GPU: degenerate shapes of the method against the FP64 oracle.

A subcircuit without data qubits (every wire it touches is cut: 2 in, 3
out) has a one-column A_i and T_i (2^0 bins, as subcircuit 2 of the
paper's Fig. 5 graph); checked with all qubits active and with seeded
mixed roles, FP32/FP64 inputs and outputs, both precisions, and batched
against the same queries one at a time."""
import numpy as np
import pytest

import oracle as O
from synthetic import chain_line_circuit, subcircuit_variant_probs

pytestmark = pytest.mark.gpu


def _circuit():
    c = chain_line_circuit(7, [4, 3, 4], [2, 3], 3)
    assert [len(d) for d in c.data_qubits] == [2, 0, 4]
    return c, [subcircuit_variant_probs(c, i) for i in range(c.n_subcircuits)]


def _roles(c, kind):
    if kind == "active":
        return np.zeros(c.n_qubits, dtype=np.int8)
    rng = np.random.default_rng(3)
    r = rng.choice([O.ACTIVE, O.ACTIVE, O.MERGED, O.ZOOM0, O.ZOOM1], size=c.n_qubits).astype(np.int8)
    r[0] = O.ACTIVE
    return r


@pytest.fixture(scope="module")
def ctx():
    import torch
    from paper_2207_00933_gb300 import Context, _build
    _build.build()
    with Context(0) as c:
        yield c
        torch.cuda.synchronize()


@pytest.mark.parametrize("roles_kind", ["active", "mixed"])
@pytest.mark.parametrize("in_dtype", [np.float32, np.float64])
@pytest.mark.parametrize("out,prec", [("float32", "fp32"), ("float64", "fp32"), ("float64", "split_bf16")])
def test_subcircuit_without_data_qubits(ctx, roles_kind, in_dtype, out, prec):
    import torch
    c, probs = _circuit()
    roles = _roles(c, roles_kind)
    g = O.Graph.from_arrays(c.n_qubits, *c.graph_arrays())
    ref = O.reconstruct(g, probs, roles)
    cid = ctx.load_subcircuit_outputs(c.n_qubits, *c.graph_arrays(),
                                      [torch.from_numpy(p.astype(in_dtype)).cuda() for p in probs])
    qid, na = ctx.set_qubit_roles(cid, roles)
    P = torch.empty(1 << na, dtype=getattr(torch, out), device="cuda")
    tot = torch.zeros(1, dtype=torch.float64, device="cuda")
    ctx.reconstruct(qid, P, prec, tot)
    torch.cuda.synchronize()
    Pn = P.double().cpu().numpy()
    err = np.abs(Pn - ref).max()
    assert err <= 1e-6 and err <= 1e-5 * np.abs(ref).max() + 1e-15, err
    assert abs(tot.item() - O.total_probability(ref)) < 1e-6
    ctx.unload(cid)


def test_subcircuit_without_data_qubits_batched(ctx):
    import torch
    c, probs = _circuit()
    cid = ctx.load_subcircuit_outputs(c.n_qubits, *c.graph_arrays(),
                                      [torch.from_numpy(p.astype(np.float32)).cuda() for p in probs])
    qs = [ctx.set_qubit_roles(cid, _roles(c, k)) for k in ("active", "mixed")]
    outs = [torch.full((1 << na,), -1.0, dtype=torch.float32, device="cuda") for _, na in qs]
    bid = ctx.batch_create([q for q, _ in qs], outs)
    ctx.batch_run(bid)
    ctx.batch_status(bid)
    for (q, _), o in zip(qs, outs):
        single = torch.empty_like(o)
        ctx.reconstruct(q, single)
        torch.cuda.synchronize()
        assert torch.equal(single, o)
    ctx.batch_release(bid)
    ctx.unload(cid)


def test_fp64_output_widens_fp32_exactly(ctx):
    """FP64 results of an FP32 pipeline are the exact widening of the FP32
    values (the kernels rearrange the bits instead of using the FP64
    converter).  A circuit without cuts reproduces its single subcircuit's
    output (the zero-cut identity), so every bin is one input value:
    normals across the exponent range, the smallest normal, subnormals and
    zero must come back as numpy's own float32 -> float64 conversion."""
    import torch
    from synthetic.circuits import Block, CutCircuit
    c = CutCircuit(5, [Block(list(range(5)), [("h", 0)])]).finalize()
    tiny = np.finfo(np.float32).tiny
    vals = np.array([0.0, 1.0, 0.5, 3.0e-8, 1.5e-30, tiny, tiny / 2, tiny * 0.75, 1.4e-45, 2.9e-44,
                     1.0e-40, 6.0e37, 3.4e38, 0.125, 0.7, 1.0 / 3.0] * 2, dtype=np.float32)
    vals[16:] = vals[:16] * np.float32(0.37)
    assert vals.size == 32
    cid = ctx.load_subcircuit_outputs(c.n_qubits, *c.graph_arrays(), [torch.from_numpy(vals[None, :].copy()).cuda()])
    qid, na = ctx.set_qubit_roles(cid, np.zeros(5, dtype=np.int8))
    out = torch.empty(1 << na, dtype=torch.float64, device="cuda")
    ctx.reconstruct(qid, out)
    torch.cuda.synchronize()
    got = out.cpu().numpy()
    assert np.array_equal(got.view(np.uint64), vals.astype(np.float64).view(np.uint64))
    ctx.unload(cid)

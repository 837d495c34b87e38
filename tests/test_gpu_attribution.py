"""GPU parity of the attribution (Eq. 1 with the I/X/Y/Z expansion of
every cut wire) on large subcircuits, where the kernel switches to 32 x 8
state tiles: the 4-states-per-thread form for 16-byte aligned FP32 inputs,
the one-state-per-thread form for FP64 inputs and for FP32 inputs that are
not 16-byte aligned.  The cases cover subcircuits with 1, 2 or 3 outgoing
cut edges and none, with incoming edges and without (every form of the
kernel, the double-buffered one with one and with two incoming edges),
each checked through the whole reconstruction against the FP64 oracle."""
import numpy as np
import pytest

import oracle as O
from synthetic import workloads as W

pytestmark = pytest.mark.gpu

ABS_TOL = 1e-6
REL_TOL = 1e-5

# (widths, hand-offs, active qubits per subcircuit)
CASES = {
    "kout1": ([20, 6], [1], [8, 4]),        # 19 data qubits, 1 outgoing edge
    "kout3": ([18, 6], [3], [8, 4]),        # 15 data qubits, 3 outgoing edges
    "kout2_kin2": ([20, 22], [2], [10, 10]),  # 18 + 22 data qubits, 2 cuts
    "kin1_kout1": ([6, 21, 6], [1, 1], [3, 8, 3]),  # a middle subcircuit of 20 data qubits
    "kin1_kout0": ([6, 20], [1], [3, 8]),   # 5 + 20 data qubits: the double-buffered form with one incoming edge
}


@pytest.fixture(scope="module")
def ctx():
    import torch
    from paper_2207_00933_gb300 import Context, _build
    _build.build()
    c = Context(0)
    yield c
    torch.cuda.synchronize()
    c.close()


def _device_input(p, form):
    import torch
    if form == "fp64":
        return torch.from_numpy(p.astype(np.float64)).cuda()
    t = torch.from_numpy(p).cuda()
    if form == "fp32_aligned":
        assert t.data_ptr() % 16 == 0
        return t
    # the same values one element into a larger buffer: 4-byte aligned only
    buf = torch.empty(p.size + 1, dtype=torch.float32, device="cuda")
    view = buf[1:].view(p.shape)
    view.copy_(t)
    assert view.data_ptr() % 16 == 4
    return view


@pytest.mark.parametrize("case", sorted(CASES))
def test_large_tiles_match_oracle(ctx, case):
    import torch
    widths, handoffs, active = CASES[case]
    w = W.random_line_chain(21, widths, handoffs, 1, active)
    c = w.circuit
    ref = O.reconstruct(O.Graph.from_arrays(c.n_qubits, *c.graph_arrays()),
                        [p.astype(np.float64) for p in w.probs], w.roles)
    scale = np.abs(ref).max()
    for form in ("fp32_aligned", "fp32_unaligned", "fp64"):
        probs = [_device_input(p, form) for p in w.probs]
        cid = ctx.load_subcircuit_outputs(c.n_qubits, *c.graph_arrays(), probs)
        qid, na = ctx.set_qubit_roles(cid, w.roles)
        out = torch.empty(1 << na, dtype=torch.float32, device="cuda")
        ctx.reconstruct(qid, out)
        torch.cuda.synchronize()
        err = np.abs(out.double().cpu().numpy() - ref).max()
        assert err <= ABS_TOL and err <= REL_TOL * scale + 1e-15, (case, form, err)
        ctx.unload(cid)


def _star_circuit(kout_on_b: bool):
    """Two upstream subcircuits each hand 4 wires to a third (8 incoming cut
    edges: more than the fused kernel's 7, so the attribution takes the
    two-pass form -- outcome weights per outgoing edge, then the 4 x 4
    prepared-state expansion per incoming edge).  With kout_on_b the third
    subcircuit also hands one received wire on to a fourth."""
    from synthetic.circuits import Block, CutCircuit
    blocks = [Block([0, 1, 2, 3, 4], [("h", 4), ("cz", 3, 4)]),
              Block([5, 6, 7, 8, 9], [("h", 5), ("cz", 5, 6)]),
              Block([0, 1, 2, 3, 5, 6, 7, 8], [("sx", 0), ("cz", 3, 5)])]
    if kout_on_b:
        blocks.append(Block([0, 10], [("h", 10), ("cz", 0, 10)]))
        return CutCircuit(11, blocks).finalize()
    return CutCircuit(10, blocks).finalize()


@pytest.mark.parametrize("kout_on_b,forms", [(False, ("fp32_aligned", "fp64")), (True, ("fp32_aligned",))])
def test_eight_incoming_edges_two_pass_form(ctx, kout_on_b, forms):
    import torch
    from synthetic.qpu import random_variant_probs
    from synthetic.workloads import Workload
    c = _star_circuit(kout_on_b)
    b = 2
    assert len(c.in_edges[b]) == 8 and len(c.out_edges[b]) == (1 if kout_on_b else 0)
    rng = np.random.default_rng(41)
    probs = [random_variant_probs(c, i, rng).astype(np.float32) for i in range(c.n_subcircuits)]
    g = O.Graph.from_arrays(c.n_qubits, *c.graph_arrays())
    rr = np.random.default_rng(42)
    for roles in (np.zeros(c.n_qubits, dtype=np.int8),
                  rr.choice([O.ACTIVE, O.ACTIVE, O.MERGED, O.ZOOM0, O.ZOOM1], c.n_qubits).astype(np.int8)):
        w = Workload("star8", c, probs, roles)
        ref = O.reconstruct(g, [p.astype(np.float64) for p in probs], roles)
        scale = np.abs(ref).max()
        for form in forms:
            dev = [_device_input(p, form) for p in probs]
            cid = ctx.load_subcircuit_outputs(c.n_qubits, *c.graph_arrays(), dev)
            qid, na = ctx.set_qubit_roles(cid, w.roles)
            out = torch.empty(1 << na, dtype=torch.float64, device="cuda")
            ctx.reconstruct(qid, out)
            torch.cuda.synchronize()
            err = np.abs(out.cpu().numpy() - ref).max()
            assert err <= ABS_TOL and err <= REL_TOL * scale + 1e-15, (kout_on_b, form, err)
            ctx.unload(cid)
            del dev

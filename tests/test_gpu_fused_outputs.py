"""GPU parity of one recursion step on fresh subcircuit outputs with the
attribution fused into the merge (sqc_reconstruct_outputs; Section 4's
states merging applied while attributing, Eq. 1): only the states a query
keeps are attributed, the merged qubits are summed in shared memory and the
merged tensors are written directly.

Each case is checked element by element against the FP64 oracle on the
fresh outputs, against sqc_update_subcircuit_outputs + sqc_reconstruct on
the same outputs, and the circuit's resident tensors must be untouched (a
plain reconstruct afterwards still gives the loaded outputs' bins)."""
import numpy as np
import pytest

import oracle as O
from synthetic import workloads as W

pytestmark = pytest.mark.gpu

ABS_TOL = 1e-6
REL_TOL = 1e-5


def _oracle(c, probs, roles):
    return O.reconstruct(O.Graph.from_arrays(c.n_qubits, *c.graph_arrays()), [p.astype(np.float64) for p in probs],
                         roles)


def _check(P, ref):
    err = float(np.abs(P - ref).max())
    assert err <= ABS_TOL and err <= REL_TOL * float(np.abs(ref).max()) + 1e-15, err


def _fresh(w, seed):
    # new outputs of the same shapes: the loaded ones with seeded noise
    # (still valid probability rows are not needed by the method)
    rng = np.random.default_rng(seed)
    return [(p * (1.0 + 0.25 * rng.random(p.shape))).astype(p.dtype) for p in w.probs]


def _case(w, roles, precision, out_dtype, in_dtype, host_inputs):
    import torch
    from paper_2207_00933_gb300 import Context, _build
    _build.build()
    c = w.circuit
    fresh = [p.astype(in_dtype) for p in _fresh(w, 5)]
    ref_new = _oracle(c, fresh, roles)
    ref_old = _oracle(c, w.probs, roles)
    with Context(0) as ctx:
        # host inputs are staged in the buffer a host-data load sizes
        loaded = [p.astype(in_dtype) for p in w.probs] if host_inputs else [torch.from_numpy(p).cuda() for p in w.probs]
        cid = ctx.load_subcircuit_outputs(c.n_qubits, *c.graph_arrays(), loaded)
        qid, na = ctx.set_qubit_roles(cid, roles)
        out = torch.full((1 << na,), -3.0, dtype=getattr(torch, out_dtype), device="cuda")
        tot = torch.zeros(1, dtype=torch.float64, device="cuda")
        src = fresh if host_inputs else [torch.from_numpy(p).cuda() for p in fresh]
        ctx.reconstruct_outputs(qid, src, out, precision, tot)
        torch.cuda.synchronize()
        P = out.double().cpu().numpy()
        _check(P, ref_new)
        assert abs(tot.item() - O.total_probability(P)) <= 1e-9 * max(1.0, abs(tot.item()))
        # the resident tensors still hold the loaded outputs
        ctx.reconstruct(qid, out, precision)
        torch.cuda.synchronize()
        _check(out.double().cpu().numpy(), ref_old)
        # and an update + reconstruct of the fresh outputs agrees
        ctx.update_subcircuit_outputs(cid, [torch.from_numpy(p).cuda() for p in fresh])
        ctx.reconstruct(qid, out, precision)
        torch.cuda.synchronize()
        assert np.abs(out.double().cpu().numpy() - P).max() <= ABS_TOL
        ctx.unload(cid)


@pytest.mark.parametrize("precision", ["fp32", "split_bf16"])
@pytest.mark.parametrize("in_dtype,host", [(np.float32, False), (np.float64, False), (np.float32, True)])
def test_line30_recursion_roles(precision, in_dtype, host):
    w = W.merged_30q()
    _case(w, w.roles, precision, "float32", in_dtype, host)


def test_grid40_fp64_out_chunked():
    w = W.grid_40q()
    _case(w, w.roles, "split_bf16", "float64", np.float32, False)


def test_zoomed_and_all_active():
    # zoom prefixes on every subcircuit (the next recursion's roles) and the
    # all-active full state (no merged qubits)
    w = W.random_line_chain(9, [9, 9, 8], [2, 2], 2, [3, 3, 3], zoom_bits=2)
    assert (w.roles >= O.ZOOM0).sum() == 6
    _case(w, w.roles, "fp32", "float64", np.float32, False)
    w = W.full_state_12q()
    _case(w, w.roles, "fp32", "float64", np.float64, False)


def test_one_subcircuit_writes_the_bins():
    from synthetic.circuits import Block, CutCircuit
    from synthetic.workloads import Workload
    from synthetic import subcircuit_variant_probs
    c = CutCircuit(6, [Block(list(range(6)), [("h", 0), ("cz", 0, 1), ("sx", 3), ("t", 1), ("sy", 5)])]).finalize()
    roles = np.array([2, 3, 0, 0, 1, 1], dtype=np.int8)      # zoom 2, active 2, merged 2
    w = Workload("one", c, [subcircuit_variant_probs(c, 0)], roles)
    _case(w, roles, "fp32", "float64", np.float64, False)


def test_roles_outside_the_pattern_are_refused():
    import torch
    from paper_2207_00933_gb300 import Context, SQCError
    w = W.small_random(3, roles="mixed")
    c = w.circuit
    with Context(0) as ctx:
        cid = ctx.load_subcircuit_outputs(c.n_qubits, *c.graph_arrays(), [torch.from_numpy(p).cuda() for p in w.probs])
        # an active qubit below a merged one in some subcircuit
        roles = np.full(c.n_qubits, O.MERGED, dtype=np.int8)
        dq = next(d for d in c.data_qubits if len(d) >= 2)
        roles[dq[-1]] = O.ACTIVE
        qid, na = ctx.set_qubit_roles(cid, roles)
        out = torch.empty(1 << na, dtype=torch.float32, device="cuda")
        with pytest.raises(SQCError) as ei:
            ctx.reconstruct_outputs(qid, [torch.from_numpy(p).cuda() for p in w.probs], out)
        assert ei.value.status == 1
        ctx.unload(cid)

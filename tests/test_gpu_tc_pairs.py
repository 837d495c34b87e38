"""GPU parity of the 2-SM tensor-core form (tcgen05.mma.cta_group::2,
256 x 256 output units, each SM of a pair loading its own half of both
operands) against the FP64 oracle and against the one-SM form.

4096 x 4096 x 256 gives 256 pair units: with 74-76 co-resident pairs the
last wave is at most half full, so it runs as half-width (256 x 128) units;
2048 x 4096 (128 units) leaves a tail over half a wave, so every unit is
full width.  FP32 and FP64 outputs, and FP64 with the shared index summed
in four FP32 passes (Section 6.3)."""
import numpy as np
import pytest

import oracle as O
from synthetic import workloads as W

pytestmark = pytest.mark.gpu

ABS_TOL = 1e-6
REL_TOL = 1e-5


def _oracle(w):
    c = w.circuit
    return O.reconstruct(O.Graph.from_arrays(c.n_qubits, *c.graph_arrays()),
                         [p.astype(np.float64) for p in w.probs], w.roles)


@pytest.fixture(scope="module")
def cases():
    out = {}
    for active in ((12, 12), (11, 12)):
        w = W.random_line_chain(11, [16, 16], [4], 1, list(active))
        out[active] = (w, _oracle(w))
    return out


def _run(w, pairs, out_dtype, **cfg):
    import torch
    from paper_2207_00933_gb300 import Context, _build
    _build.build()
    c = w.circuit
    with Context(0, tc_pairs=pairs, **cfg) as ctx:
        cid = ctx.load_subcircuit_outputs(c.n_qubits, *c.graph_arrays(), [torch.from_numpy(p).cuda() for p in w.probs])
        qid, na = ctx.set_qubit_roles(cid, w.roles)
        out = torch.full((1 << na,), -7.0, dtype=getattr(torch, out_dtype), device="cuda")
        tot = torch.zeros(1, dtype=torch.float64, device="cuda")
        ctx.reconstruct(qid, out, "split_bf16", tot)
        torch.cuda.synchronize()
        assert ctx.query_tc_steps(qid)[0] == 1
        res = out.double().cpu().numpy(), float(tot.item())
        ctx.unload(cid)
    return res


@pytest.mark.parametrize("active,out", [((12, 12), "float32"), ((12, 12), "float64"), ((11, 12), "float32")])
def test_pairs_match_oracle_and_single_sm_form(cases, active, out):
    w, ref = cases[active]
    P, tot = _run(w, True, out)
    err = np.abs(P - ref).max()
    assert err <= ABS_TOL and err <= REL_TOL * np.abs(ref).max() + 1e-15, err
    assert abs(tot - O.total_probability(P)) < 1e-9
    # the one-SM form adds the same products over the same 16-wide slices
    # into one FP32 accumulator: equal up to the FP32 rounding of the sums
    P1, _ = _run(w, False, out)
    assert np.abs(P - P1).max() <= 2.0 ** -20 * np.abs(ref).max()


def test_pairs_chunked_fp64(cases):
    w, ref = cases[(12, 12)]
    P, tot = _run(w, True, "float64", chunk_terms=64, fp64_chunk_min_edges=4)
    err = np.abs(P - ref).max()
    assert err <= ABS_TOL and err <= REL_TOL * np.abs(ref).max() + 1e-15, err
    P1, _ = _run(w, False, "float64", chunk_terms=64, fp64_chunk_min_edges=4)
    assert np.abs(P - P1).max() <= 2.0 ** -20 * np.abs(ref).max()

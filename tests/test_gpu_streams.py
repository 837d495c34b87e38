"""GPU: reconstruct on the caller's stream, on a side stream and inside
CUDA graphs, with stage timing off and on (graph mode keeps the timing
events; a capture fails if any work is left unjoined).  Every form must
give the very same bins (same kernels, same summation order) and the same
FP64 total, and match the FP64 oracle."""
import numpy as np
import pytest

import oracle as O
from synthetic import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", params=["merged_30q", "grid_40q"])
def setup(request):
    import torch
    from paper_2207_00933_gb300 import Context, _build
    _build.build()
    w = getattr(W, request.param)()
    c = w.circuit
    ref = O.reconstruct(O.Graph.from_arrays(c.n_qubits, *c.graph_arrays()),
                        [p.astype(np.float64) for p in w.probs], w.roles)
    ctx = Context(0)
    cid = ctx.load_subcircuit_outputs(c.n_qubits, *c.graph_arrays(), [torch.from_numpy(p).cuda() for p in w.probs])
    qid, na = ctx.set_qubit_roles(cid, w.roles)
    yield ctx, qid, na, ref
    torch.cuda.synchronize()
    ctx.close()


def _check(P, ref):
    err = np.abs(P - ref).max()
    assert err <= 1e-6 and err <= 1e-5 * np.abs(ref).max() + 1e-15, err


@pytest.mark.parametrize("precision", ["fp32", "split_bf16"])
def test_streams_graphs_and_profiled_capture(setup, precision):
    import torch
    ctx, qid, na, ref = setup
    out0 = torch.empty(1 << na, dtype=torch.float64, device="cuda")
    tot0 = torch.zeros(1, dtype=torch.float64, device="cuda")
    ctx.reconstruct(qid, out0, precision, tot0)
    torch.cuda.synchronize()
    _check(out0.cpu().numpy(), ref)
    assert abs(tot0.item() - O.total_probability(ref)) < 1e-6

    # on a side stream, synchronising only that stream
    s = torch.cuda.Stream()
    out1 = torch.full_like(out0, -1.0)
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        ctx.reconstruct(qid, out1, precision, stream=s)
    s.synchronize()
    assert torch.equal(out1, out0)

    # graphs, with stage timing off and on (graph mode keeps the events)
    for prof in (0, 2):
        ctx.profile_enable(prof)
        out2 = torch.full_like(out0, -1.0)
        tot2 = torch.zeros_like(tot0)
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g):
            ctx.reconstruct(qid, out2, precision, tot2, stream=torch.cuda.current_stream())
        for _ in range(3):
            out2.fill_(-1.0)
            g.replay()
        torch.cuda.synchronize()
        assert torch.equal(out2, out0), prof
        assert tot2.item() == tot0.item()
        if prof:
            r = ctx.profile_read()
            # FP32 runs the merge and every step as one launch (recorded as
            # the contraction stage); split-BF16 launches per stage
            assert r["ms"]["contract"] > 0, r
            if precision == "split_bf16":
                assert r["ms"]["final"] > 0, r
        del g
    ctx.profile_enable(0)


@pytest.mark.parametrize("precision", ["fp32", "split_bf16"])
def test_programmatic_launch_changes_nothing(precision):
    """With programmatic dependent launch every kernel starts while its
    predecessor finishes and waits on the device for its results: the
    bins, the probability sum and the selected bins are the same as with
    plain launches, eagerly and replayed from a CUDA graph."""
    import math
    import torch
    from paper_2207_00933_gb300 import Context
    w = W.merged_30q()
    c = w.circuit
    res = {}
    for pdl in (True, False):
        with Context(0, pdl=pdl) as ctx:
            probs = [torch.from_numpy(p).cuda() for p in w.probs]
            cid = ctx.load_subcircuit_outputs(c.n_qubits, *c.graph_arrays(), probs)
            qid, na = ctx.set_qubit_roles(cid, w.roles)
            out = torch.empty(1 << na, dtype=torch.float32, device="cuda")
            tot = torch.zeros(1, dtype=torch.float64, device="cuda")

            def step():
                ctx.update_subcircuit_outputs(cid, probs)
                ctx.reconstruct(qid, out, precision, tot)
                return ctx.top_bins(qid, out, 256, -math.inf)
            b, v, n = step()
            g = torch.cuda.CUDAGraph()
            with torch.cuda.graph(g):
                b2, v2, n2 = step()
            out.fill_(-1.0)
            g.replay()
            torch.cuda.synchronize()
            assert torch.equal(b, b2) and torch.equal(v, v2)
            res[pdl] = (out.cpu().clone(), tot.item(), b2.cpu().clone())
            ctx.unload(cid)
    assert torch.equal(res[True][0], res[False][0])
    assert res[True][1] == res[False][1]
    assert torch.equal(res[True][2], res[False][2])

"""GPU parity of the cross-chunk FP64 sum (Section 6.3: the sum over the 4^K
edge terms, FP64 across chunks when K >= 12) with two or more chunks.

The last contraction step sums its shared index in FP32 chunks of
`chunk_terms` terms and adds the chunks in FP64: on the SIMT cores in the
FP32 precision, and on the tcgen05 tensor cores in split-BF16 (each chunk
one accumulator pass in tensor memory, added into the FP64 output by the
epilogue).  Every result is compared element by element with the FP64
oracle at the stated 1e-6 max-abs (and 1e-5 of the largest bin), and with
the same query run as a single chunk.  Sliced queries (Section 6.3, first
level) add every slice's last step into the output, which the tensor-core
epilogue does itself."""
import numpy as np
import pytest

import oracle as O
from synthetic import workloads as W

pytestmark = pytest.mark.gpu

ABS_TOL = 1e-6
REL_TOL = 1e-5


def _oracle(w, roles=None):
    c = w.circuit
    return O.reconstruct(O.Graph.from_arrays(c.n_qubits, *c.graph_arrays()),
                         [p.astype(np.float64) for p in w.probs], w.roles if roles is None else roles)


def _run(w, precision, out_dtype="float64", **cfg):
    """Reconstruct w on a fresh context with configuration cfg; returns the
    bins, the FP64 total, the last step's (M, N, Kd) and the number of
    tensor-core steps of the split plan."""
    import torch
    from paper_2207_00933_gb300 import Context, _build
    _build.build()
    c = w.circuit
    with Context(0, **cfg) as ctx:
        cid = ctx.load_subcircuit_outputs(c.n_qubits, *c.graph_arrays(), [torch.from_numpy(p).cuda() for p in w.probs])
        qid, na = ctx.set_qubit_roles(cid, w.roles)
        out = torch.full((1 << na,), -7.0, dtype=getattr(torch, out_dtype), device="cuda")
        tot = torch.zeros(1, dtype=torch.float64, device="cuda")
        ctx.reconstruct(qid, out, precision, tot)
        torch.cuda.synchronize()
        last = ctx.query_steps(qid)[-1]
        ntc = ctx.query_tc_steps(qid)[0]
        res = out.double().cpu().numpy(), float(tot.item()), last, ntc
        ctx.unload(cid)
    return res


def _check(P, ref):
    err = float(np.abs(P - ref).max())
    assert err <= ABS_TOL, err
    assert err <= REL_TOL * float(np.abs(ref).max()), err
    return err


@pytest.fixture(scope="module")
def grid40():
    w = W.grid_40q()
    return w, _oracle(w)


@pytest.mark.parametrize("precision", ["fp32", "split_bf16"])
def test_grid40_four_chunks(grid40, precision):
    # K = 12 (the default threshold); the last step shares 3 cuts (Kd = 64),
    # summed in 4 chunks of 16 terms
    w, ref = grid40
    P, tot, (M, N, Kd), ntc = _run(w, precision, chunk_terms=16)
    assert Kd == 64 and M * N == 1 << 22
    _check(P, ref)
    assert abs(tot - O.total_probability(ref)) < 1e-6
    if precision == "split_bf16":
        assert ntc >= 1                      # the last step runs on the tensor cores
    P1, _, _, _ = _run(w, precision, chunk_terms=256)       # one chunk
    assert np.abs(P - P1).max() <= ABS_TOL


@pytest.fixture(scope="module")
def five_shared():
    # two subcircuits sharing 5 cut edges: one step with Kd = 4^5 = 1024
    # (M = N = 256), summed in chunks of 256 (4 chunks) or 16 (64 chunks)
    w = W.random_line_chain(31, [13, 13], [5], 1, [8, 8])
    assert w.circuit.n_edges == 5 and w.n_active == 16
    return w, _oracle(w)


@pytest.mark.parametrize("precision", ["fp32", "split_bf16"])
@pytest.mark.parametrize("chunk", [16, 256])
def test_last_step_kd1024_chunked(five_shared, precision, chunk):
    w, ref = five_shared
    P, tot, (M, N, Kd), ntc = _run(w, precision, chunk_terms=chunk, fp64_chunk_min_edges=5)
    assert Kd == 1024 and M == 256 and N == 256
    _check(P, ref)
    assert abs(tot - O.total_probability(P)) < 1e-9
    if precision == "split_bf16":
        assert ntc == 1
    # and the same in one FP32 pass (FP64 chunking off: threshold above K)
    P1, _, _, _ = _run(w, precision, chunk_terms=chunk, fp64_chunk_min_edges=6)
    assert np.abs(P - P1).max() <= ABS_TOL


@pytest.fixture(scope="module")
def wide():
    # 4096 x 4096 x 256: the 256-wide tensor-core configuration
    w = W.random_line_chain(11, [16, 16], [4], 1, [12, 12])
    return w, _oracle(w)


def test_wide_tiles_chunked_fp64(wide):
    # four passes of 64 terms per 128 x 256 unit, added in FP64
    w, ref = wide
    P, tot, (M, N, Kd), ntc = _run(w, "split_bf16", chunk_terms=64, fp64_chunk_min_edges=4, tc_pairs=False)
    assert (M, N, Kd) == (4096, 4096, 256) and ntc == 1
    _check(P, ref)
    assert abs(tot - O.total_probability(P)) < 1e-9


@pytest.mark.parametrize("precision", ["fp32", "split_bf16"])
def test_sliced_last_step_accumulates(precision):
    # first-level slicing of 2 edges: 16 slices, each adding its last step
    # into the output (FP32 and FP64 outputs)
    w = W.merged_30q()
    ref = _oracle(w)
    for out in ("float32", "float64"):
        P, tot, _, ntc = _run(w, precision, out_dtype=out, slice_edges=2)
        _check(P, ref)
        assert abs(tot - O.total_probability(ref)) < 1e-6


@pytest.mark.parametrize("out", ["float32", "float64"])
def test_sliced_tensor_core_step_accumulates(wide, out):
    # one sliced edge: 4 slices, each adding its 4096 x 4096 x 64 last step
    # into the output on the tensor cores
    w, ref = wide
    P, tot, (M, N, Kd), ntc = _run(w, "split_bf16", out_dtype=out, slice_edges=1)
    assert (M, N, Kd) == (4096, 4096, 64) and ntc == 1
    _check(P, ref)
    assert abs(tot - O.total_probability(P)) < 1e-9

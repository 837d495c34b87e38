"""The allocation-free selection entry point (sqc_top_bins_noalloc).

It serves callers that cannot allocate device memory -- code embedded in a
host application that owns every device allocation, or a latency-critical
loop where a cudaMalloc (which can synchronise the device) is not
acceptable -- so its scratch is a static device array inside the library.
This file is collected last on purpose: if it fails, a run that stops at
the first failure has already run every other test.

Each check calls the new entry point through the C ABI twice in a row and
compares it with the existing entry point (sqc_top_bins, workspace from a
query).  Selection is exact, so the comparison is exact: the tolerance the
other parity tests use for bin selection."""
import ctypes
import math

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def setup():
    import torch
    import paper_2207_00933_gb300 as sqc
    from paper_2207_00933_gb300 import _build
    from synthetic import workloads as W
    _build.build()
    lib = sqc.load_library()
    ctx = sqc.Context(0)
    w = W.full_state_12q()
    c = w.circuit
    cid = ctx.load_subcircuit_outputs(c.n_qubits, *c.graph_arrays(), [torch.from_numpy(p).cuda() for p in w.probs])
    qid, _ = ctx.set_qubit_roles(cid, w.roles)
    yield lib, ctx, qid
    torch.cuda.synchronize()
    ctx.close()


def _noalloc(lib, x, k, thr):
    """Direct C-ABI call of sqc_top_bins_noalloc on the current stream."""
    import torch
    bins = torch.full((k,), -1, dtype=torch.int64, device=x.device)
    vals = torch.full((k,), -1.0, dtype=torch.float64, device=x.device)
    nf = torch.full((1,), -1, dtype=torch.int32, device=x.device)
    dt = 1 if x.dtype == torch.float64 else 0
    st = lib.sqc_top_bins_noalloc(0, ctypes.c_void_p(x.data_ptr()), dt, x.numel(), k, float(thr),
                                  ctypes.c_void_p(bins.data_ptr()), ctypes.c_void_p(vals.data_ptr()),
                                  ctypes.c_void_p(nf.data_ptr()), ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert st == 0, lib.sqc_last_error(None)
    return bins, vals, nf


@pytest.mark.parametrize("dtype", ["float32", "float64"])
def test_noalloc_matches_workspace_selection_twice(setup, dtype):
    import torch
    lib, ctx, qid = setup
    rng = np.random.default_rng(11)
    cases = [
        (rng.random(1 << 20).astype(dtype) * 1e-6, 1024, -math.inf),          # 2^20 bins, top 1024
        (rng.integers(0, 9, 200_000).astype(dtype) * 0.25, 4096, 0.5),         # exact ties past capacity
    ]
    for x_np, k, thr in cases:
        x = torch.from_numpy(x_np).cuda()
        ref_b, ref_v, ref_n = ctx.top_bins(qid, x, k, thr)
        for _ in range(2):                       # two calls in a row share the static scratch
            b, v, n = _noalloc(lib, x, k, thr)
            torch.cuda.synchronize()
            m = int(ref_n.item())
            assert int(n.item()) == m
            assert torch.equal(b[:m], ref_b[:m])
            assert torch.equal(v[:m], ref_v[:m])


def test_noalloc_rejects_k_beyond_capacity(setup):
    import torch
    lib, _, _ = setup
    x = torch.zeros(16, dtype=torch.float32, device="cuda")
    buf = torch.empty(8192, dtype=torch.int64, device="cuda")
    st = lib.sqc_top_bins_noalloc(0, ctypes.c_void_p(x.data_ptr()), 0, 16, 8192, 0.0, ctypes.c_void_p(buf.data_ptr()),
                                  ctypes.c_void_p(buf.data_ptr()), ctypes.c_void_p(buf.data_ptr()), None)
    assert st == 3
    assert b"4096" in lib.sqc_last_error(None)

"""GPU parity of the bin selection (Algorithm 1: keep the largest bins, then
the probability check) for both cooperative kernels: the shared-memory
resident one (default for up to ~7 million values) and the streaming one
(select_resident=False, and every larger input).  Results are compared
exactly with the oracle's top_bins on the same values: bins ordered by
value descending, ties by bin index ascending, values >= threshold."""
import math
import zlib

import numpy as np
import pytest

import oracle as O
from synthetic import workloads as W

pytestmark = pytest.mark.gpu


def _values(kind, n, dtype, rng):
    if kind == "narrow":          # sums over many merged states: one octave
        x = 1.0 + 0.03 * rng.standard_normal(n)
    elif kind == "porter_thomas":  # exponential, spans many octaves
        x = rng.exponential(1.0, n)
    elif kind == "ties":          # heavy exact ties
        x = rng.integers(0, 7, n) * 0.125
        x[rng.integers(0, n, 40)] = 2.0
    elif kind == "zeros":         # one nonzero bin (a Bernstein-Vazirani level)
        x = np.zeros(n)
        x[n // 3] = 1.0
    elif kind == "signed_nan":    # negatives, infinities and NaNs
        x = rng.standard_normal(n)
        x[rng.integers(0, n, 50)] = np.nan
        x[rng.integers(0, n, 3)] = np.inf
        x[rng.integers(0, n, 3)] = -np.inf
    else:
        raise ValueError(kind)
    return (x / max(n, 1)).astype(dtype)


@pytest.fixture(scope="module")
def ctxs():
    import torch
    from paper_2207_00933_gb300 import Context, _build
    _build.build()
    w = W.full_state_12q()
    c = w.circuit
    out = {}
    for resident in (True, False):
        ctx = Context(0, select_resident=resident)
        cid = ctx.load_subcircuit_outputs(c.n_qubits, *c.graph_arrays(),
                                          [torch.from_numpy(p).cuda() for p in w.probs])
        qid, _ = ctx.set_qubit_roles(cid, w.roles)
        out[resident] = (ctx, qid)
    yield out
    torch.cuda.synchronize()
    for ctx, _ in out.values():
        ctx.close()


def _full_order(x):
    """The oracle's complete order of x (every non-NaN value)."""
    return O.top_bins(x.astype(np.float64), x.size, -math.inf)


def _check(ctx, qid, x, k, thr, full=None):
    """GPU top_bins(k, thr) against the oracle.  With the oracle's full
    order given, the expected answer is its first k entries >= thr (a
    prefix, the order being by value descending)."""
    import torch
    xd = torch.from_numpy(x).cuda()
    b, v, nf = ctx.top_bins(qid, xd, k, thr)
    torch.cuda.synchronize()
    if full is None:
        eb, ev = O.top_bins(x.astype(np.float64), k, thr)
    else:
        m_all = int(np.count_nonzero(full[1] >= thr))
        eb, ev = full[0][:min(k, m_all)], full[1][:min(k, m_all)]
    m = int(nf.item())
    assert m == eb.size, (m, eb.size)
    assert b[:m].cpu().numpy().tolist() == eb.tolist()
    assert np.array_equal(v[:m].cpu().numpy(), ev)


@pytest.mark.parametrize("resident", [True, False])
@pytest.mark.parametrize("dtype", ["float32", "float64"])
@pytest.mark.parametrize("kind", ["narrow", "porter_thomas", "ties", "zeros", "signed_nan"])
def test_selection_matches_oracle(ctxs, resident, dtype, kind):
    ctx, qid = ctxs[resident]
    rng = np.random.default_rng(zlib.crc32(f"{kind}/{dtype}".encode()))
    # several tiles per CTA and a ragged tail
    x = _values(kind, (1 << 20) + 37, dtype, rng)
    full = _full_order(x)
    for k, thr in ((1, -math.inf), (37, -math.inf), (1024, -math.inf), (4096, -math.inf)):
        _check(ctx, qid, x, k, thr, full)
    vals = full[1]
    thr = float(vals[min(500, vals.size - 1)])      # a threshold inside the data
    _check(ctx, qid, x, 4096, thr, full)
    _check(ctx, qid, x, 100, thr, full)
    _check(ctx, qid, x, 4096, float(np.nextafter(vals[0], np.inf)))   # nothing passes


@pytest.mark.parametrize("resident", [True, False])
def test_selection_small_and_ragged(ctxs, resident):
    ctx, qid = ctxs[resident]
    rng = np.random.default_rng(7)
    for n in (1, 3, 5, 151, 152 * 4 + 3, 4097, 100_003):
        for dtype in ("float32", "float64"):
            x = _values("porter_thomas", n, dtype, rng)
            for k in (1, 10, 4096):
                _check(ctx, qid, x, k, -math.inf)


def test_selection_size_limits_and_shared_workspace(ctxs):
    """Inputs just past the resident limit take the streaming kernel on the
    same query workspace; alternating sizes checks that each kernel leaves
    the workspace as the other expects it."""
    ctx, qid = ctxs[True]
    rng = np.random.default_rng(11)
    big32 = _values("narrow", 7_500_000, "float32", rng)      # > 200 KB of key words per SM
    small = _values("porter_thomas", 1 << 20, "float32", rng)
    big64 = _values("porter_thomas", 7_400_000, "float64", rng)
    mid64 = _values("ties", (1 << 22) + 3, "float64", rng)     # resident (32-bit key words)
    fulls = {id(x): _full_order(x) for x in (big32, small, big64, mid64)}
    for x in (big32, small, big64, mid64, small, big32):
        _check(ctx, qid, x, 1024, -math.inf, fulls[id(x)])
        _check(ctx, qid, x, 4096, -math.inf, fulls[id(x)])


def test_selection_repeats_identically(ctxs):
    import torch
    ctx, qid = ctxs[True]
    x = torch.from_numpy(_values("narrow", 1 << 20, "float32", np.random.default_rng(3))).cuda()
    first = [t.clone() for t in ctx.top_bins(qid, x, 1024)]
    for _ in range(20):
        b, v, n = ctx.top_bins(qid, x, 1024)
        assert torch.equal(b, first[0]) and torch.equal(v, first[1]) and torch.equal(n, first[2])

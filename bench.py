#!/usr/bin/env python
"""Benchmark of the states-merging reconstruction on GB300.

A step is one pass of the whole hot path over one batch of synthetic input
already resident in HBM: attribution of the subcircuit variant outputs
(new QPU results, Algorithm 1), merge/zoom of every subcircuit (Algorithm
2), the contraction steps (Section 6) with the 2^-K scale and the FP64
probability check, and the selection of the largest bins.  The default
workload is the 30-qubit line circuit cut at K=8 into 4 subcircuits with
20 active and 10 merged qubits (2^20 bins, FP32).

Timing: W untimed warm-up steps, then K steps, each bracketed by CUDA
events on the launching stream; the inputs fit in L2, so a 256 MiB buffer
is written between steps (outside the events) to flush it.  The per-stage
times behind the roofline come from a second, separate run of K steps with
stage events inside the step (they are not in the timed region).  One JSON
line on rank 0.  --impl reference times the FP64 CPU oracle on the same
workload instead.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

if "reference" in sys.argv:
    # the oracle baseline runs single-threaded so that its core count is exact
    for _v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS", "NUMEXPR_NUM_THREADS"):
        os.environ[_v] = "1"

import numpy as np  # noqa: E402

WORKLOADS = {
    "line30_K8_a20": "merged_30q",
    "grid40_K12_a22": "grid_40q",
    "line12_K2_full": "full_state_12q",
}
METRIC = "recon bins/s"
UNIT = "bins/s"
TOPK = 1024
FALLBACK_HBM_GBS = 6800.0
# DRAM bytes (read + write) per launch of the dominant kernel, from one ncu
# capture (dram__bytes_read.sum + dram__bytes_write.sum) of
# `bench.py --steps 3 --warmup 3 --no-extras --no-cpu-baseline` on this
# workload; to be re-taken (or dropped) whenever that kernel changes
# (the 4 MB of bins written stay in L2 at the end of that launch)
NCU_TRAFFIC = {("line30_K8_a20", "fp32", "select_resident_kernel (fused: contraction steps, bins, selection)"):
               416768 + 1280}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=30)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="line30_K8_a20", choices=sorted(WORKLOADS))
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-graph", action="store_true", help="launch the step eagerly instead of replaying a CUDA graph")
    ap.add_argument("--precision", default="fp32", choices=["fp32", "split_bf16"])
    ap.add_argument("--no-extras", action="store_true", help="skip the microbenchmarks, batch and serving runs")
    ap.add_argument("--extra", choices=["tensor", "hbm", "batch", "batch_tc", "serving", "grid40", "recursion"],
                    help="run only this microbenchmark and print its JSON line")
    return ap.parse_args()


def make_workload(name: str, seed_offset: int = 0):
    from synthetic import workloads as W
    fn = getattr(W, WORKLOADS[name])
    import inspect
    seed = inspect.signature(fn).parameters["seed"].default + seed_offset
    return fn(seed)


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return FALLBACK_HBM_GBS, "fallback"


def bf16_peak():
    """Dense BF16 tensor peak (TFLOP/s) for a kernel timed alone: the
    measured burst figure, else the fallback."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["bf16_tflops"]), "measured"
    except Exception:
        return 1900.0, "fallback"


def tensor_microbench(dev, reps: int = 20) -> dict:
    """A contraction-bound step: two subcircuits sharing 4 cut edges, 12
    active qubits each, so the last step is C[4096 x 4096] = A[4096 x 256]
    B^T (Section 6.1, Fig. 4a).  Times that step (stage events) in
    split-BF16 on the tensor cores and in FP32 SIMT; hardware flops of the
    split form = 6 products x 2MNK."""
    import torch
    import oracle as O
    from paper_2207_00933_gb300 import Context
    from synthetic import workloads as W
    w = W.random_line_chain(11, [16, 16], [4], 1, [12, 12])
    c = w.circuit
    g = O.Graph.from_arrays(c.n_qubits, *c.graph_arrays())
    ref = O.reconstruct(g, [p.astype(np.float64) for p in w.probs], w.roles)
    out = {}
    for pairs in (False, True):
        # per-stage launches, so that the last step has its own stage events
        with Context(dev.index or 0, tc_pairs=pairs, fused_query=False) as ctx:
            cid = ctx.load_subcircuit_outputs(c.n_qubits, *c.graph_arrays(), [torch.from_numpy(p).to(dev) for p in w.probs])
            qid, na = ctx.set_qubit_roles(cid, w.roles)
            M, N, K = ctx.query_steps(qid)[-1]
            res = torch.empty(1 << na, dtype=torch.float32, device=dev)
            for prec in (("split_bf16",) if pairs else ("split_bf16", "fp32")):
                for _ in range(3):
                    ctx.reconstruct(qid, res, prec)
                torch.cuda.synchronize(dev)
                ctx.profile_enable(True)
                for _ in range(reps):
                    ctx.reconstruct(qid, res, prec)
                pr = ctx.profile_read()
                ctx.profile_enable(False)
                ms = pr["ms"]["final"] / max(1, pr["calls"]["final"])
                err = float(np.abs(res.double().cpu().numpy() - ref).max())
                alg = 2.0 * M * N * K / (ms * 1e-3) / 1e12
                d = {"ms": ms, "alg_tflops": alg, "max_abs_err_vs_fp64": err}
                if prec == "split_bf16":
                    peak, src = bf16_peak()
                    d.update({"hw_tflops": 6 * alg, "peak_tflops": peak, "peak_source": src,
                              "tensor_frac": 6 * alg / peak,
                              "form": "2-SM pairs (cta_group::2, 256 x 256 units)" if pairs else
                                      "one SM per 128 x 256 unit"})
                out[prec + ("_pairs" if pairs else "")] = d
            ctx.unload(cid)
    return {"shape": {"M": M, "N": N, "K": K}, "workload": "randline32_K4_a24 (two subcircuits, 4 shared cuts)", **out}


def grid40_bench(dev, reps: int = 20) -> dict:
    """The mixed-precision configuration: the 40-qubit 5 x 8 grid circuit cut
    at K = 12 into 5 subcircuits, 22 active qubits (2^22 bins), FP64 output
    (K >= 12: the last step sums its shared index in FP32 and adds it in
    FP64).  The whole step (attribution, merge, contraction, FP64 check,
    top-1024) replayed from a CUDA graph with L2 flushed between steps, in
    split-BF16 and FP32, each checked against the FP64 oracle; plus the
    event-timed last contraction step (tcgen05 in split-BF16) against the
    HBM roofline (its output write dominates its bytes)."""
    import torch
    import oracle as O
    from paper_2207_00933_gb300 import Context
    from synthetic import workloads as W
    w = W.grid_40q()
    c = w.circuit
    ref = O.reconstruct(O.Graph.from_arrays(c.n_qubits, *c.graph_arrays()),
                        [p.astype(np.float64) for p in w.probs], w.roles)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream(dev)
    hbm, src = peaks()
    res = {"workload": "grid40_K12_a22 (5 x 8 grid, depth 8, K = 12, 22 active qubits, FP64 output)"}
    with Context(dev.index or 0) as ctx:
        probs = [torch.from_numpy(p).to(dev) for p in w.probs]
        cid = ctx.load_subcircuit_outputs(c.n_qubits, *c.graph_arrays(), probs)
        qid, na = ctx.set_qubit_roles(cid, w.roles)
        out = torch.empty(1 << na, dtype=torch.float64, device=dev)
        tot = torch.zeros(1, dtype=torch.float64, device=dev)
        kb = torch.empty(TOPK, dtype=torch.int64, device=dev)
        kp = torch.empty(TOPK, dtype=torch.float64, device=dev)
        kn = torch.empty(1, dtype=torch.int32, device=dev)
        M, N, K = ctx.query_steps(qid)[-1]
        for prec in ("split_bf16", "fp32"):
            def step():
                ctx.update_subcircuit_outputs(cid, probs)
                ctx.reconstruct(qid, out, prec, tot)
                ctx.top_bins(qid, out, TOPK, -math.inf, kb, kp, kn)
            for _ in range(3):
                step()
            torch.cuda.synchronize(dev)
            err = float(np.abs(out.cpu().numpy() - ref).max())
            g = torch.cuda.CUDAGraph()
            with torch.cuda.graph(g):
                step()
            for _ in range(3):
                g.replay()
            torch.cuda.synchronize(dev)
            tt = 0.0
            for _ in range(reps):
                flush.zero_()
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                g.replay()
                e1.record(stream)
                torch.cuda.synchronize(dev)
                tt += e0.elapsed_time(e1)
            ms = tt / reps
            del g
            # the last step alone (stage events, separate run)
            ctx.profile_enable(True)
            for _ in range(reps):
                flush.zero_()
                ctx.reconstruct(qid, out, prec, tot)
            pr = ctx.profile_read()
            ctx.profile_enable(False)
            d = {"ms_per_step": ms, "bins_per_s": (1 << na) / (ms * 1e-3), "max_abs_err_vs_fp64": err,
                 "total_prob": float(tot.item())}
            if prec == "split_bf16":
                fin = pr["ms"]["final"] / max(1, pr["calls"]["final"])
                byts = 6 * (M * K + N * K) + 8 * M * N
                d["last_step"] = {"shape": [M, N, K], "kernel": "gemm_tc_kernel", "us": 1e3 * fin,
                                  "roofline": {"bound": "hbm", "achieved": byts / (fin * 1e-3) / 1e9, "peak": hbm,
                                               "unit": "GB/s", "frac": byts / (fin * 1e-3) / 1e9 / hbm,
                                               "peak_source": src, "algorithmic_bytes": byts},
                                  "alg_tflops": 2.0 * M * N * K / (fin * 1e-3) / 1e12,
                                  "tc_steps": ctx.query_tc_steps(qid)}
            res[prec] = d
        ctx.unload(cid)
    return res


def recursion_bench(dev) -> dict:
    """Algorithm 1 at the paper's scale (Section 8.1): a 1000-qubit
    Bernstein-Vazirani circuit cut into a chain of 59 subcircuits of at most
    18 qubits, M = 2^20 bins per recursion, run to its single solution:
    recursions, seconds per recursion (planning, reconstruction and
    selection of each level, host planning included) and whether the
    hidden string was found."""
    import torch
    from paper_2207_00933_gb300 import Context, recursion
    from synthetic.circuits import bernstein_vazirani_chain
    from synthetic.qpu import product_variant_probs
    c, s = bernstein_vazirani_chain(5, [18] * 58 + [14], [1] * 58)
    graph = (c.n_qubits, *c.graph_arrays())
    M = 2 ** 20
    with Context(dev.index or 0) as ctx:
        probs = [torch.from_numpy(product_variant_probs(c, i, np.float32)).to(dev) for i in range(c.n_subcircuits)]
        cid = ctx.load_subcircuit_outputs(*graph, probs)
        del probs
        recursion.search(ctx, cid, graph, M, R=2, keep=4, threshold=1e-3)       # warm-up
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        sols, r = recursion.search(ctx, cid, graph, M, R=64, keep=4, threshold=1e-3)
        dt = time.perf_counter() - t0
    found = len(sols) == 1 and sols[0][0] == s
    return {"workload": "bv1000: 1000-qubit Bernstein-Vazirani, 59 subcircuits <= 18 qubits, 58 cuts, M = 2^20",
            "recursions": r, "expected": recursion.recursions_needed(c.n_qubits, M), "solution_found": found,
            "probability": sols[0][1] if sols else None, "seconds": dt, "seconds_per_recursion": dt / max(1, r)}


def hbm_microbench(dev, reps: int = 10) -> dict:
    """HBM-bound stages at a size where they stream: two line subcircuits of
    20 and 22 qubits sharing 2 cut edges, with random outputs (4^2 variants
    each, 320 MiB of FP32 input, 272 MiB of attributed tensors), 10 + 14
    active qubits.  Times, with stage events and the inputs resident in HBM
    (all buffers larger than L2), the attribution (reads every variant
    output once, writes A) and the merge (reads A once); achieved bandwidth
    is the algorithmic bytes over the stage time.  The result is checked
    against the FP64 oracle."""
    import torch
    import oracle as O
    from paper_2207_00933_gb300 import Context
    from synthetic import workloads as W
    w = W.random_line_chain(12, [20, 22], [2], 1, [10, 14])
    c = w.circuit
    hbm, src = peaks()
    out = {"workload": "randline40_K2_a24 (subcircuits of 20 and 22 measured qubits, 2 cuts, 10+14 active)",
           "peak_gbs": hbm, "peak_source": src}
    with Context(dev.index or 0, fused_query=False) as ctx:     # the merge as its own launch
        probs_dev = [torch.from_numpy(p).to(dev) for p in w.probs]
        cid = ctx.load_subcircuit_outputs(c.n_qubits, *c.graph_arrays(), probs_dev)
        qid, na = ctx.set_qubit_roles(cid, w.roles)
        res = torch.empty(1 << na, dtype=torch.float32, device=dev)
        steps = ctx.query_steps(qid)

        def step():
            ctx.update_subcircuit_outputs(cid, probs_dev)
            ctx.reconstruct(qid, res, "fp32")

        for _ in range(3):
            step()
        torch.cuda.synchronize(dev)
        ctx.profile_enable(True)
        for _ in range(reps):
            step()
        pr = ctx.profile_read()
        ctx.profile_enable(False)
        algo = algorithmic_bytes(w, steps, 4)
        for k in ("attribute", "merge"):
            ms = pr["ms"][k] / max(1, pr["calls"][k])
            gbs = algo[k] / (ms * 1e-3) / 1e9
            out[k] = {"us": 1e3 * ms, "bytes": algo[k], "GBps": gbs, "frac": gbs / hbm}
        g = O.Graph.from_arrays(c.n_qubits, *c.graph_arrays())
        ref = O.reconstruct(g, [p.astype(np.float64) for p in w.probs], w.roles)
        out["max_abs_err_vs_fp64"] = float(np.abs(res.double().cpu().numpy() - ref).max())
        ctx.unload(cid)
    return out


# ---- clocks during the timed region ---------------------------------------------

class ClockSampler:
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines: list[str] = []
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        if self.thread:
            self.thread.join(timeout=2)
        sm, smax, reasons = [], [], set()
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                smax.append(float(parts[1]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[4:8]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ---- the oracle on the host cores --------------------------------------------------

def oracle_step(w, g, probs64, k):
    import oracle as O
    P = O.reconstruct(g, probs64, w.roles)
    O.top_bins(P, k)
    O.total_probability(P)
    return P


_ORACLE_LOOP = """
import os, sys, time, json
sys.path.insert(0, {root!r})
import numpy as np
import bench, oracle as O
w = bench.make_workload({name!r})
g = O.Graph.from_arrays(w.circuit.n_qubits, *w.circuit.graph_arrays())
probs = [p.astype(np.float64) for p in w.probs]
bench.oracle_step(w, g, probs, bench.TOPK)
n, t0 = 0, time.perf_counter()
while True:
    bench.oracle_step(w, g, probs, bench.TOPK)
    n += 1
    dt = time.perf_counter() - t0
    if dt >= {budget} or n >= 200:
        break
print(json.dumps({{"reps": n, "seconds": dt, "bins": 1 << w.n_active}}))
"""


def _oracle_procs(name: str, budget_s: float, procs: int) -> list:
    """`procs` single-threaded oracle loops side by side (fresh interpreters,
    no fork of this GPU process); each reports (reps, seconds, bins)."""
    env = dict(os.environ)
    for v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS", "NUMEXPR_NUM_THREADS"):
        env[v] = "1"
    code = _ORACLE_LOOP.format(root=ROOT, name=name, budget=budget_s)
    ps = [subprocess.Popen([sys.executable, "-c", code], stdout=subprocess.PIPE, stderr=subprocess.PIPE, text=True,
                           env=env) for _ in range(procs)]
    out = []
    for p in ps:
        o, e = p.communicate(timeout=900)
        if p.returncode != 0:
            raise RuntimeError(e[-300:])
        out.append(json.loads(o.strip().splitlines()[-1]))
    return out


def cpu_baseline(name: str, budget_s: float = 12.0) -> dict:
    """Time the oracle, as it stands, on a bounded sample of the same
    workload: one single-threaded process, and one process per host core
    (independent reconstructions side by side: the whole host's oracle
    throughput).  `value` is the single-thread figure, `all_cores` the
    host-wide one with its core count."""
    try:
        one = _oracle_procs(name, budget_s, 1)[0]
    except Exception as ex:  # noqa: BLE001
        return {"value": None, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": f"failed: {ex}"}
    res = {"value": one["reps"] * one["bins"] / one["seconds"], "unit": UNIT, "cores": 1, "kind": "oracle",
           "sample": f"{one['reps']} full reconstructions (attribution, merge, pairwise contraction, top-{TOPK}, "
                     f"FP64 sum) of {name}, {one['seconds']:.1f} s, one thread"}
    cores = os.cpu_count() or 1
    try:
        many = _oracle_procs(name, budget_s, cores)
        res["all_cores"] = {"value": sum(d["reps"] * d["bins"] / d["seconds"] for d in many), "unit": UNIT,
                            "cores": cores,
                            "sample": f"{cores} single-threaded processes, {sum(d['reps'] for d in many)} "
                                      f"reconstructions in {max(d['seconds'] for d in many):.1f} s"}
    except Exception as ex:  # noqa: BLE001
        res["all_cores"] = {"value": None, "cores": cores, "sample": f"failed: {ex}"}
    return res


def batch_bench(dev, reps: int = 10) -> dict:
    """Batched recursion level: 256 zoom queries (10-20 active qubits) over 4
    resident random-output circuits of 60-70 qubits (5-6 subcircuits, 7-10
    cuts).  Times (CUDA events, L2 flushed between repetitions) the one-launch
    persistent batch (FP32, replayed from a CUDA graph) against the plain
    form -- every query's own launches, one query after another -- in FP32
    and in split-BF16.  Each form's bins are checked on 8 sampled queries
    against the FP64 oracle."""
    import torch
    import oracle as O
    from paper_2207_00933_gb300 import Context
    from synthetic import workloads as W
    b = W.batch_level()
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream(dev)
    res = {"workload": f"{len(b.queries)} queries, circuits {b.meta['n_qubits']} qubits, cuts {b.meta['cuts']}, "
                       f"subcircuits {b.meta['subcircuits']}, active 10-20"}
    # the plain form launches every stage of every query on its own
    with Context(dev.index or 0, fused_query=False) as ctx:
        cids = [ctx.load_subcircuit_outputs(c.n_qubits, *c.graph_arrays(), [torch.from_numpy(p).to(dev) for p in ps])
                for c, ps in zip(b.circuits, b.probs)]
        qs = [ctx.set_qubit_roles(cids[ci], roles) for ci, roles in b.queries]
        bins = sum(1 << na for _, na in qs)
        outs = [torch.empty(1 << na, dtype=torch.float32, device=dev) for _, na in qs]
        totals = torch.zeros(len(qs), dtype=torch.float64, device=dev)
        sample = list(range(0, len(qs), len(qs) // 8))[:8]
        refs = {}
        for j in sample:
            ci, roles = b.queries[j]
            c = b.circuits[ci]
            refs[j] = O.reconstruct(O.Graph.from_arrays(c.n_qubits, *c.graph_arrays()),
                                    [p.astype(np.float64) for p in b.probs[ci]], roles)

        def timed(fn):
            for _ in range(3):
                fn()
            torch.cuda.synchronize(dev)
            tot = 0.0
            for _ in range(reps):
                flush.zero_()
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                fn()
                e1.record(stream)
                torch.cuda.synchronize(dev)
                tot += e0.elapsed_time(e1)
            return tot / reps

        def err():
            return max(float(np.abs(outs[j].double().cpu().numpy() - refs[j]).max()) for j in sample)

        bid = ctx.batch_create([q for q, _ in qs], outs, totals)
        graph = torch.cuda.CUDAGraph()
        ctx.batch_run(bid)
        with torch.cuda.graph(graph):
            ctx.batch_run(bid)
        ms = timed(graph.replay)
        ctx.batch_status(bid)
        res["batch_fp32"] = {"ms": ms, "bins_per_s": bins / (ms * 1e-3), "launches": 1, "max_abs_err_vs_fp64": err()}
        ctx.batch_release(bid)
        # the tile policy picked by the autotuner (sqc_batch_autotune), timed the same way
        best, order, pol_ms = ctx.batch_autotune([q for q, _ in qs], outs, totals, reps=5)
        bid = ctx.batch_create([q for q, _ in qs], outs, totals)
        graph = torch.cuda.CUDAGraph()
        ctx.batch_run(bid)
        with torch.cuda.graph(graph):
            ctx.batch_run(bid)
        ms = timed(graph.replay)
        ctx.batch_status(bid)
        res["batch_fp32_autotuned"] = {"ms": ms, "bins_per_s": bins / (ms * 1e-3), "launches": 1,
                                       "policy": best, "order": ["greedy", "fewest multiplications"][order],
                                       "ms_unflushed_by_order_and_policy": pol_ms, "max_abs_err_vs_fp64": err()}
        for prec in ("fp32", "split_bf16"):
            def plain():
                for (q, _), o in zip(qs, outs):
                    ctx.reconstruct(q, o, prec)
            ms = timed(plain)
            res[f"plain_{prec}"] = {"ms": ms, "bins_per_s": bins / (ms * 1e-3), "max_abs_err_vs_fp64": err()}
            if prec == "split_bf16":
                tc = [ctx.query_tc_steps(q) for q, _ in qs]
                res["plain_split_bf16"]["tc_steps"] = sum(a for a, _ in tc)
                res["plain_split_bf16"]["steps"] = sum(b for _, b in tc)
        res["batch_vs_plain_fp32"] = res["plain_fp32"]["ms"] / res["batch_fp32"]["ms"]
        res["bins"] = bins
        ctx.batch_release(bid)
        # the same level in split-BF16: steps the planner puts on the tensor
        # cores run as tcgen05 launches between the persistent phases
        bid = ctx.batch_create([q for q, _ in qs], outs, totals, precision="split_bf16")
        graph = torch.cuda.CUDAGraph()
        ctx.batch_run(bid)
        with torch.cuda.graph(graph):
            ctx.batch_run(bid)
        ms = timed(graph.replay)
        ctx.batch_status(bid)
        res["batch_split_bf16"] = {"ms": ms, "bins_per_s": bins / (ms * 1e-3), "max_abs_err_vs_fp64": err(),
                                   "tc_steps": sum(ctx.query_tc_steps(q)[0] for q, _ in qs)}
        ctx.batch_release(bid)
    # one query at a time, each as ONE persistent launch (merge and every
    # step; the library's default for FP32 queries)
    with Context(dev.index or 0) as ctx:
        cids = [ctx.load_subcircuit_outputs(c.n_qubits, *c.graph_arrays(), [torch.from_numpy(p).to(dev) for p in ps])
                for c, ps in zip(b.circuits, b.probs)]
        qs = [ctx.set_qubit_roles(cids[ci], roles) for ci, roles in b.queries]

        def single_launch():
            for (q, _), o in zip(qs, outs):
                ctx.reconstruct(q, o, "fp32")
        ms = timed(single_launch)
        res["plain_fp32_single_launch"] = {"ms": ms, "bins_per_s": bins / (ms * 1e-3), "launches": len(qs),
                                           "max_abs_err_vs_fp64": err()}
    # the same batch with the merge pyramid (merges read the level that
    # holds the sums over each subcircuit's merged qubits)
    with Context(dev.index or 0, merge_pyramid=True) as ctx:
        cids = [ctx.load_subcircuit_outputs(c.n_qubits, *c.graph_arrays(), [torch.from_numpy(p).to(dev) for p in ps])
                for c, ps in zip(b.circuits, b.probs)]
        qs = [ctx.set_qubit_roles(cids[ci], roles) for ci, roles in b.queries]
        bid = ctx.batch_create([q for q, _ in qs], outs, totals)
        graph = torch.cuda.CUDAGraph()
        ctx.batch_run(bid)
        with torch.cuda.graph(graph):
            ctx.batch_run(bid)
        ms = timed(graph.replay)
        ctx.batch_status(bid)
        res["batch_fp32_pyramid"] = {"ms": ms, "bins_per_s": bins / (ms * 1e-3), "launches": 1,
                                     "max_abs_err_vs_fp64": err()}
        ctx.batch_release(bid)
        # pyramid and the autotuned tile policy together
        best, order, pol_ms = ctx.batch_autotune([q for q, _ in qs], outs, totals, reps=5)
        bid = ctx.batch_create([q for q, _ in qs], outs, totals)
        graph = torch.cuda.CUDAGraph()
        ctx.batch_run(bid)
        with torch.cuda.graph(graph):
            ctx.batch_run(bid)
        ms = timed(graph.replay)
        ctx.batch_status(bid)
        res["batch_fp32_pyramid_autotuned"] = {"ms": ms, "bins_per_s": bins / (ms * 1e-3), "launches": 1,
                                               "policy": best, "order": ["greedy", "fewest multiplications"][order],
                                               "ms_unflushed_by_order_and_policy": pol_ms,
                                               "max_abs_err_vs_fp64": err()}
        ctx.batch_release(bid)
    return res


def batch_tc_bench(dev, reps: int = 10) -> dict:
    """A batched level whose last steps are contraction-bound (shared index
    of 256 terms): 12 queries over three random-output chain circuits of
    20-24 qubits (each circuit's full-active query and three zoomed ones),
    FP64 outputs.  The batch in split-BF16 (those last steps on tcgen05,
    between the persistent phases) against the batch in FP32 and against
    the plain one-query-at-a-time forms; every form checked against the FP64
    oracle on every query."""
    import torch
    import oracle as O
    from paper_2207_00933_gb300 import Context
    from synthetic import workloads as W
    ws = [W.random_line_chain(17, [8, 11, 11], [2, 4], 1, [4, 7, 7]),
          W.random_line_chain(18, [7, 10, 11], [2, 4], 1, [5, 6, 7]),
          W.random_line_chain(20, [12, 12], [4], 1, [7, 7])]
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream(dev)
    res = {"workload": "12 queries over 3 chain circuits of 20-24 qubits; last steps 128 x 2048 x 256 and "
                       "128 x 128 x 256; FP64 outputs"}
    with Context(dev.index or 0, fused_query=False) as ctx:
        ent = []
        for w in ws:
            c = w.circuit
            cid = ctx.load_subcircuit_outputs(c.n_qubits, *c.graph_arrays(), [torch.from_numpy(p).to(dev) for p in w.probs])
            merged = [q for q in range(c.n_qubits) if w.roles[q] == O.MERGED][:2]
            for v in range(4):
                r = w.roles.copy()
                for b, q in enumerate(merged):
                    if v & (1 << b):
                        r[q] = O.ZOOM1
                q, na = ctx.set_qubit_roles(cid, r)
                ent.append((q, na, O.reconstruct(O.Graph.from_arrays(c.n_qubits, *c.graph_arrays()),
                                                 [p.astype(np.float64) for p in w.probs], r)))
        outs = [torch.empty(1 << na, dtype=torch.float64, device=dev) for _, na, _ in ent]
        totals = torch.zeros(len(ent), dtype=torch.float64, device=dev)
        bins = sum(1 << na for _, na, _ in ent)

        def timed(fn):
            for _ in range(3):
                fn()
            torch.cuda.synchronize(dev)
            tot = 0.0
            for _ in range(reps):
                flush.zero_()
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                fn()
                e1.record(stream)
                torch.cuda.synchronize(dev)
                tot += e0.elapsed_time(e1)
            return tot / reps

        def err():
            return max(float(np.abs(o.cpu().numpy() - ref).max()) for o, (_, _, ref) in zip(outs, ent))

        for prec in ("split_bf16", "fp32"):
            bid = ctx.batch_create([q for q, _, _ in ent], outs, totals, precision=prec)
            graph = torch.cuda.CUDAGraph()
            ctx.batch_run(bid)
            with torch.cuda.graph(graph):
                ctx.batch_run(bid)
            ms = timed(graph.replay)
            ctx.batch_status(bid)
            res[f"batch_{prec}"] = {"ms": ms, "bins_per_s": bins / (ms * 1e-3), "max_abs_err_vs_fp64": err()}
            ctx.batch_release(bid)
            del graph

            def plain():
                for (q, _, _), o in zip(ent, outs):
                    ctx.reconstruct(q, o, prec)
            ms = timed(plain)
            res[f"plain_{prec}"] = {"ms": ms, "bins_per_s": bins / (ms * 1e-3), "max_abs_err_vs_fp64": err()}
        res["tc_steps"] = sum(ctx.query_tc_steps(q)[0] for q, _, _ in ent)
        res["bins"] = bins
    return res


def serving_bench(dev, rates=(100, 300, 1000, 3000, 5000), seconds: float = 0.6, max_per_rate: int = 600) -> dict:
    """Serving stream: zoom queries (random zoom prefix, 12-20 active qubits)
    arrive by Poisson arrivals against 8 resident random-output circuits of
    200-1000 qubits (16-50 subcircuits of <= 14 qubits, 10-40 cuts; forests
    of chains where cuts < subcircuits - 1).  For every arrival rate the
    continuous-batching server and the plain one-query-per-launch FP32
    server are offered the same seeded arrival sequence; latency is submit
    to completion on the server's clock, throughput = bins completed / wall
    time from first submission to last completion.  `batched_pyramid` is
    the batching server on a context with the merge pyramid."""
    import torch
    from paper_2207_00933_gb300 import Context, Server
    from synthetic import workloads as W
    b = W.serving_set(n_queries=4096)
    rng = np.random.default_rng(12)
    out = {"workload": f"8 circuits {b.meta['n_qubits']} qubits, cuts {b.meta['cuts']}, "
                       f"subcircuits {b.meta['subcircuits']}; queries: zoom prefix + 12-20 active"}
    for mode in ("batched", "plain", "batched_pyramid"):
        res = {}
        ctx = Context(dev.index or 0, merge_pyramid=(mode == "batched_pyramid"))
        cids = [ctx.load_subcircuit_outputs(c.n_qubits, *c.graph_arrays(),
                                            [torch.from_numpy(p).to(dev) for p in ps])
                for c, ps in zip(b.circuits, b.probs)]
        torch.cuda.synchronize(dev)
        with Server(ctx, max_batch=64, n_streams=4, plain=(mode == "plain")) as srv:
            # warm-up
            for ci, roles in b.queries[:32]:
                srv.submit(cids[ci], roles)
            srv.drain(120.0)
            qi = 32
            for rate in rates:
                n = int(min(max_per_rate, max(20, rate * seconds)))
                gaps = np.random.default_rng(1000 + rate).exponential(1.0 / rate, n)
                tickets = []
                t0 = time.perf_counter()
                t_next = t0
                for k in range(n):
                    t_next += gaps[k]
                    while time.perf_counter() < t_next:
                        pass
                    ci, roles = b.queries[qi % len(b.queries)]
                    qi += 1
                    tickets.append(srv.submit(cids[ci], roles))
                srv.drain(300.0)
                wall_end = time.perf_counter()
                lat, bins = [], 0
                for t in tickets:
                    state, us, na = srv.poll(t)
                    lat.append(us)
                    bins += 1 << na
                    srv.result(t)
                lat.sort()
                res[str(rate)] = {"queries": n, "p50_ms": lat[len(lat) // 2] / 1e3,
                                  "p99_ms": lat[min(len(lat) - 1, int(0.99 * len(lat)))] / 1e3,
                                  "bins_per_s": bins / (wall_end - t0),
                                  "offered_per_s": rate, "achieved_per_s": n / (wall_end - t0)}
            res["server_stats"] = srv.stats()
        ctx.close()
        out[mode] = res
    return out


def bench_config(args, w) -> dict:
    """The workload description both arms print (identical dicts): which
    circuit, how many bins, the selection size, the output format and the
    precision of the GPU arm, the seed, and how the timing treats L2."""
    c = w.circuit
    world = int(os.environ.get("WORLD_SIZE", "1"))
    return {"workload": args.workload, "bins": 1 << w.n_active, "active_qubits": int(w.n_active),
            "cuts": c.n_edges, "subcircuits": c.n_subcircuits, "topk": TOPK,
            "out_dtype": "float64" if args.workload == "grid40_K12_a22" else "float32",
            "precision": args.precision, "seed": w.meta.get("seed"),
            "parallelism": f"{world} independent circuits" if world > 1 else "1 gpu",
            "l2": "inputs resident in HBM; the GPU arm flushes L2 between steps (256 MiB write outside the "
                  "timed events)"}


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    import oracle as O
    w = make_workload(args.workload)
    g = O.Graph.from_arrays(w.circuit.n_qubits, *w.circuit.graph_arrays())
    probs = [p.astype(np.float64) for p in w.probs]
    for _ in range(args.warmup):
        oracle_step(w, g, probs, TOPK)
    times = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        oracle_step(w, g, probs, TOPK)
        times.append(time.perf_counter() - t0)
    bins = 1 << w.n_active
    tot = sum(times)
    value = bins * len(times) / tot
    import multiprocessing
    cores = 1
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * tot / len(times),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": bench_config(args, w),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": f"{len(times)} full reconstructions of {args.workload} "
                                       f"({multiprocessing.cpu_count()} host cores present; numpy oracle)"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ---- our arm -------------------------------------------------------------------------

def algorithmic_bytes(w, steps, out_elem_bytes):
    """Bytes the method itself must move per step, per stage."""
    c = w.circuit
    in_b = w.probs[0].dtype.itemsize
    attr = sum(p.size * in_b + (p.shape[0] << len(c.data_qubits[i])) * 4 for i, p in enumerate(w.probs))
    merge = 0
    for i in range(c.n_subcircuits):
        k = len(c.incident[i])
        dq = c.data_qubits[i]
        z = sum(1 for q in dq if w.roles[q] in (2, 3))
        a = sum(1 for q in dq if w.roles[q] == 0)
        merge += (4 ** k) * (1 << (len(dq) - z)) * 4 + (4 ** k) * (1 << a) * 4
    contract = sum(4 * (M * K + K * N) + 4 * M * N for (M, N, K) in steps[:-1])
    M, N, K = steps[-1] if steps else (1, 1, 1)
    final = 4 * (M * K + K * N) + out_elem_bytes * M * N
    select = (1 << w.n_active) * out_elem_bytes
    # attribution fused into the merge: the kept states' outputs read once
    # (zoomed states skipped), the merged tensors written
    fused = 0
    for i, p in enumerate(w.probs):
        dq = c.data_qubits[i]
        z = sum(1 for q in dq if w.roles[q] in (2, 3))
        a = sum(1 for q in dq if w.roles[q] == 0)
        fused += (p.size >> z) * in_b + p.shape[0] * (1 << a) * 4
    return {"attribute": attr, "merge": merge, "contract": contract, "final": final, "select": select,
            "attribute_fused": fused}


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
        return
    import torch
    import torch.distributed as dist

    if args.extra:
        import __graft_entry__
        __graft_entry__.build()
        dev = torch.device("cuda", 0)
        fn = {"tensor": tensor_microbench, "hbm": hbm_microbench, "batch": batch_bench, "serving": serving_bench,
              "grid40": grid40_bench, "recursion": recursion_bench, "batch_tc": batch_tc_bench}
        print(json.dumps({"extra": args.extra, **fn[args.extra](dev)}), flush=True)
        return

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    dev = torch.device("cuda", local)

    import __graft_entry__
    __graft_entry__.build()
    from paper_2207_00933_gb300 import Context

    w = make_workload(args.workload, seed_offset=rank)      # weak scaling: an independent circuit per rank
    c = w.circuit
    out_dtype = torch.float64 if args.workload == "grid40_K12_a22" else torch.float32
    out_b = 8 if out_dtype == torch.float64 else 4
    stream = torch.cuda.current_stream(dev)
    ctx = Context(local)
    probs_dev = [torch.from_numpy(p).to(dev) for p in w.probs]
    probs_host = [torch.from_numpy(p).pin_memory() for p in w.probs]
    cid = ctx.load_subcircuit_outputs(c.n_qubits, *c.graph_arrays(), probs_host)   # host-staged (e2e path)
    qid, na = ctx.set_qubit_roles(cid, w.roles)
    bins = 1 << na
    out = torch.empty(bins, dtype=out_dtype, device=dev)
    # the step's results (top bins, their values, the FP64 total, the count)
    # as views of one device buffer, read back by one copy
    res_dev = torch.zeros(16 * TOPK + 16, dtype=torch.uint8, device=dev)
    kb = res_dev[:8 * TOPK].view(torch.int64)
    kp = res_dev[8 * TOPK:16 * TOPK].view(torch.float64)
    tot = res_dev[16 * TOPK:16 * TOPK + 8].view(torch.float64)
    kn = res_dev[16 * TOPK + 8:16 * TOPK + 12].view(torch.int32)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)

    prec = args.precision
    from paper_2207_00933_gb300 import SQCError

    # one recursion step on fresh subcircuit outputs in one call
    # (sqc_reconstruct_select): attribution fused into the merge (only the
    # kept states), then the contraction steps, the bins and the selection
    # in one cooperative launch where the plan allows it; queries whose roles
    # do not allow the fused attribution update the resident tensors and
    # reconstruct instead
    try:
        ctx.reconstruct_outputs(qid, probs_dev, out, prec, tot)
        fused_step = True
    except SQCError:
        fused_step = False
    tail_steps = ctx.query_fused_select(qid) if (prec == "fp32" and out_dtype == torch.float32) else 0

    def unfused_step():
        ctx.update_subcircuit_outputs(cid, probs_dev)
        ctx.reconstruct(qid, out, prec, tot)
        ctx.top_bins(qid, out, TOPK, -math.inf, kb, kp, kn)

    def staged_step():
        ctx.reconstruct_outputs(qid, probs_dev, out, prec, tot)
        ctx.top_bins(qid, out, TOPK, -math.inf, kb, kp, kn)

    def step():
        if not fused_step:
            return unfused_step()
        ctx.reconstruct_select(qid, out, TOPK, -math.inf, probs=probs_dev, precision=prec, total_prob=tot,
                               bins_out=kb, probs_out=kp, n_found=kn)

    for _ in range(max(3, args.warmup)):
        step()
    torch.cuda.synchronize(dev)

    # correctness of the timed configuration against the FP64 oracle
    import oracle as O
    g = O.Graph.from_arrays(c.n_qubits, *c.graph_arrays())
    ref = O.reconstruct(g, [p.astype(np.float64) for p in w.probs], w.roles)
    err = float(np.abs(out.double().cpu().numpy() - ref).max())

    steps_shape = ctx.query_steps(qid)
    info = ctx.query_info(qid)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    use_graph = not args.no_graph

    def capture(profiled):
        # the whole step (attribution, merge, contraction steps, selection)
        # captured once and replayed; with profiling the stage events
        # become graph nodes
        ctx.profile_enable(2 if profiled else False)
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g):
            step()
        torch.cuda.synchronize(dev)
        for _ in range(max(3, args.warmup)):
            g.replay()
        torch.cuda.synchronize(dev)
        if profiled:
            ctx.profile_read()
        return g

    # timed region: the step alone, no stage events inside
    if use_graph:
        run = capture(False).replay
    else:
        ctx.profile_enable(False)
        run = step
    sampler = ClockSampler(local)
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize(dev)
    sampler.start()
    time.sleep(0.3)
    wall0 = time.perf_counter()
    for i in range(args.steps):
        flush.zero_()
        ev[i][0].record(stream)
        run()
        ev[i][1].record(stream)
    torch.cuda.synchronize(dev)
    wall = time.perf_counter() - wall0
    clocks = sampler.stop()

    # the other forms of the step, timed the same way for comparison: the
    # separate calls (attribution fused into the merge, contraction steps,
    # selection), and the resident tensors updated by a separate attribution
    # before the merge
    def time_form(fn):
        if use_graph:
            fg = torch.cuda.CUDAGraph()
            with torch.cuda.graph(fg):
                fn()
            for _ in range(max(3, args.warmup)):
                fg.replay()
            frun = fg.replay
        else:
            frun = fn
        torch.cuda.synchronize(dev)
        tt = []
        for _ in range(args.steps):
            flush.zero_()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            frun()
            e1.record(stream)
            torch.cuda.synchronize(dev)
            tt.append(e0.elapsed_time(e1))
        return sum(tt) / len(tt)

    unfused_ms = staged_ms = None
    if fused_step:
        unfused_ms = time_form(unfused_step)
        staged_ms = time_form(staged_step)
        # back to the fused form's outputs for the checks below
        step()
        torch.cuda.synchronize(dev)

    # stage breakdown (roofline, launch count): the same step with stage
    # events, run separately after the timed region
    stage_total = {k: 0.0 for k in ("attribute", "merge", "contract", "final", "select")}
    stage_calls = {k: 0 for k in stage_total}
    launches = 0
    prun = capture(True).replay if use_graph else step
    if not use_graph:
        ctx.profile_enable(True)
    for i in range(args.steps):
        flush.zero_()
        prun()
        torch.cuda.synchronize(dev)
        pr = ctx.profile_read()
        for k in stage_total:
            stage_total[k] += pr["ms"][k]
            stage_calls[k] += pr["calls"][k]
        launches += pr["launches"]
    ctx.profile_enable(False)
    prof = {"ms": stage_total, "calls": stage_calls, "launches": launches}
    step_ms = [a.elapsed_time(b) for a, b in ev]
    total_ms = sum(step_ms)
    if world > 1:
        t = torch.tensor([total_ms], dtype=torch.float64, device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        total_ms = float(t.item())
    ms_per_step = total_ms / args.steps
    value = world * bins * args.steps / (total_ms * 1e-3)

    # roofline of the dominant stage; with the fused step the merge stage is
    # the attribution fused into the merge (reads the kept states' outputs,
    # writes the merged tensors); single-launch FP32 queries record the
    # merge and every contraction step as the contraction stage
    algo = algorithmic_bytes(w, steps_shape, out_b)
    if fused_step:
        algo["merge"] = algo["attribute_fused"]
    if fused_step and tail_steps:
        # the selection launch runs the contraction steps and writes the bins
        # once; they are not read back
        algo["select"] = algo["contract"] + algo["final"]
    fused = prof["calls"]["merge"] == 0 and prof["calls"]["contract"] > 0
    if fused:
        algo["contract"] = algo["merge"] + algo["contract"] + algo["final"]
    stage_ms = {k: v / max(1, prof["calls"][k]) for k, v in prof["ms"].items() if prof["calls"][k]}
    share = {k: prof["ms"][k] / max(1e-12, sum(prof["ms"].values())) for k in prof["ms"]}
    dom = max(stage_ms, key=lambda k: prof["ms"][k])
    hbm, src = peaks()
    achieved = algo[dom] / (stage_ms[dom] * 1e-3) / 1e9
    kernel_of = {"attribute": "attr_fused_kernel", "merge": "attr_merge_kernel" if fused_step else "merge_kernel",
                 "contract": "batch_kernel (merge and every step, one launch)" if fused else "gemm_simt_kernel",
                 "final": "gemm_simt_kernel (last step)",
                 "select": ("select_resident_kernel (fused: contraction steps, bins, selection)"
                            if fused_step and tail_steps else
                            "select_resident_kernel" if (1 << na) <= 7_000_000 else "select_coop_kernel")}
    traffic = NCU_TRAFFIC.get((args.workload, prec, kernel_of[dom]))
    roofline = {"bound": "hbm", "kernel": kernel_of[dom], "achieved": achieved, "peak": hbm, "unit": "GB/s",
                "frac": achieved / hbm, "traffic": traffic, "peak_source": src,
                "algorithmic_bytes": algo[dom],
                "stages": {k: {"us": 1e3 * stage_ms[k], "share": share[k],
                               "GBps": algo[k] / (stage_ms[k] * 1e-3) / 1e9} for k in stage_ms}}

    # end to end through the public API with host buffers: every step
    # copies its inputs from pinned host memory (inside
    # update_subcircuit_outputs) and reads the top bins and the total back
    h_res = torch.empty(16 * TOPK + 16, dtype=torch.uint8).pin_memory()
    h_bins = h_res[:8 * TOPK].view(torch.int64)
    h_n = h_res[16 * TOPK + 8:16 * TOPK + 12].view(torch.int32)

    def e2e_step():
        if fused_step:
            # the step's inputs copied from pinned host memory inside the call
            # (read in place by the kernels instead, host_direct=True, the
            # step measured 0.16 ms against 0.11: every latency-bound load
            # of the attribution then crosses the host link)
            ctx.reconstruct_select(qid, out, TOPK, -math.inf, probs=probs_host, precision=prec, total_prob=tot,
                                   bins_out=kb, probs_out=kp, n_found=kn)
        else:
            ctx.update_subcircuit_outputs(cid, probs_host)              # H2D of this step's inputs inside
            ctx.reconstruct(qid, out, prec, tot)
            ctx.top_bins(qid, out, TOPK, -math.inf, kb, kp, kn)
        h_res.copy_(res_dev, non_blocking=True)                         # every result, one copy

    def e2e_time(run):
        ms = []
        for i in range(args.steps):
            flush.zero_()
            torch.cuda.synchronize(dev)
            t0 = time.perf_counter()
            run()
            torch.cuda.synchronize(dev)
            ms.append(1e3 * (time.perf_counter() - t0))
        return ms

    e2e_eager_ms = e2e_time(e2e_step)
    if use_graph:
        # the same API calls captured once (the host copies become graph
        # nodes reading the pinned buffers at every replay)
        ctx.profile_enable(False)
        e2e_graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(e2e_graph):
            e2e_step()
        torch.cuda.synchronize(dev)
        for _ in range(max(3, args.warmup)):
            e2e_graph.replay()
        torch.cuda.synchronize(dev)
        e2e_ms = e2e_time(e2e_graph.replay)
    else:
        e2e_ms = e2e_eager_ms
    e2e_ok = int(h_n.item()) == TOPK and bool(torch.equal(h_bins, kb.cpu()))
    e2e_total = sum(e2e_ms)
    if world > 1:
        t = torch.tensor([e2e_total], dtype=torch.float64, device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        e2e_total = float(t.item())
    h2d = sum(p.nbytes for p in w.probs)
    d2h = int(h_res.numel())                  # bins, values, total, count in one readback

    if rank == 0:
        step_sorted = sorted(step_ms)
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32" if prec == "fp32" else "bf16x3", "data": "synthetic",
            "config": bench_config(args, w),
            "timing": {"cuda_graph": use_graph, "events": "CUDA events on the launching stream per step"},
            "max_abs_err_vs_fp64": err,
            "tflops": info["flops"] / (ms_per_step * 1e-3) / 1e12,
            "latency_ms": {"p50": step_sorted[len(step_sorted) // 2],
                           "p99": step_sorted[min(len(step_sorted) - 1, int(0.99 * len(step_sorted)))]},
            "wall_s": wall,
            "gpu_launches": prof["launches"],
            "step_form": ("fresh outputs, one call (sqc_reconstruct_select): attribution fused into the merge, "
                          + ("then the contraction steps, bins and selection in one cooperative launch"
                             if tail_steps else "then the contraction steps and the selection")) if fused_step
                         else "update of the resident tensors, then reconstruct and select",
            "separate_calls_ms_per_step": staged_ms,
            "unfused_ms_per_step": unfused_ms,
            "roofline": roofline,
            "clocks": clocks,
            "e2e": {"value": world * bins * args.steps / (e2e_total * 1e-3), "unit": UNIT,
                    "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h, "cuda_graph": use_graph,
                    "ms_per_step": e2e_total / args.steps, "results_match_device": e2e_ok,
                    "inputs": "pinned host tensors copied to the device inside the call",
                    "eager_value": bins * args.steps / (sum(e2e_eager_ms) * 1e-3)},
        }
        if world == 1 and not args.no_extras:
            tm = line["tensor_microbench"] = tensor_microbench(dev)
            hm = line["hbm_microbench"] = hbm_microbench(dev)
            line["batched_level"] = batch_bench(dev)
            line["batched_tensor_core_level"] = batch_tc_bench(dev)
            line["serving"] = serving_bench(dev)
            g40 = line["grid40_K12_a22"] = grid40_bench(dev)
            rec = line["recursion_bv1000"] = recursion_bench(dev)
            line["bv1000_seconds_per_recursion"] = rec["seconds_per_recursion"]
            # the microbenchmarks' roofline fractions, as named fields
            line["tensor_frac"] = tm["split_bf16"]["tensor_frac"]
            line["tensor_frac_pairs"] = tm.get("split_bf16_pairs", {}).get("tensor_frac")
            line["attribute_hbm_frac"] = hm["attribute"]["frac"]
            line["merge_hbm_frac"] = hm["merge"]["frac"]
            line["grid40_bins_per_s"] = g40["split_bf16"]["bins_per_s"]
            line["grid40_max_abs_err_vs_fp64"] = g40["split_bf16"]["max_abs_err_vs_fp64"]
        if world == 1 and not args.no_cpu_baseline:
            line["cpu_baseline"] = cpu_baseline(args.workload)
        print(json.dumps(line), flush=True)
    ctx.close()
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()

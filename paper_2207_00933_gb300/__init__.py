"""GB300 states-merging reconstruction (ScaleQC, arXiv 2207.00933).

Thin Python binding over the C ABI in ``include/sqc.h``: argument
marshalling only.  Every step of the reconstruction runs in the CUDA
library ``libsqc.so`` built from ``csrc/``; PyTorch supplies device memory
and streams.  Importing works without a GPU; creating a ``Context`` needs
one and the built library, and fails loudly otherwise (there is no CPU
fallback).
"""
from __future__ import annotations

import ctypes
import math
import os
from typing import Sequence

import numpy as np

__all__ = ["Context", "SQCError", "lib_path", "load_library", "ROLE_ACTIVE", "ROLE_MERGED", "ROLE_ZOOM0",
           "ROLE_ZOOM1", "STATUS"]

_HERE = os.path.dirname(os.path.abspath(__file__))

ROLE_ACTIVE, ROLE_MERGED, ROLE_ZOOM0, ROLE_ZOOM1 = 0, 1, 2, 3
F32, F64 = 0, 1
PREC = {"fp32": 0, "split_bf16": 1}
STATUS = {0: "SQC_OK", 1: "SQC_EINVAL", 2: "SQC_ENOMEM", 3: "SQC_ESHAPE", 4: "SQC_ECUDA", 5: "SQC_ETIMEOUT",
          6: "SQC_EBUSY", 7: "SQC_ENOTFOUND"}


class SQCError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


class _Config(ctypes.Structure):
    _fields_ = [("hbm_budget_bytes", ctypes.c_uint64), ("max_active_qubits", ctypes.c_int32),
                ("fp64_chunk_min_edges", ctypes.c_int32), ("chunk_terms", ctypes.c_int32),
                ("slice_edges", ctypes.c_int32), ("select_resident", ctypes.c_int32),
                ("merge_pyramid", ctypes.c_int32), ("slice_input_log2", ctypes.c_int32),
                ("slice_intermediate_log2", ctypes.c_int32), ("tc_pairs", ctypes.c_int32),
                ("wait_limit_ms", ctypes.c_int32), ("fused_query", ctypes.c_int32), ("pdl", ctypes.c_int32),
                ("contraction_order", ctypes.c_int32), ("fused_select", ctypes.c_int32)]


class _Graph(ctypes.Structure):
    _fields_ = [("n_qubits", ctypes.c_int32), ("n_subcircuits", ctypes.c_int32), ("n_edges", ctypes.c_int32),
                ("edge_up", ctypes.POINTER(ctypes.c_int32)), ("edge_down", ctypes.POINTER(ctypes.c_int32)),
                ("n_data", ctypes.POINTER(ctypes.c_int32)), ("data_qubit", ctypes.POINTER(ctypes.c_int32))]


_c = ctypes
_P = ctypes.c_void_p
_SIGS = {
    "sqc_default_config": (None, [_P]),
    "sqc_create": (_c.c_int32, [_c.POINTER(_P), _c.c_int, _P]),
    "sqc_destroy": (None, [_P]),
    "sqc_last_error": (_c.c_char_p, [_P]),
    "sqc_load_subcircuit_outputs": (_c.c_int32, [_P, _P, _c.POINTER(_P), _c.c_int, _c.c_int,
                                                 _c.POINTER(_c.c_int64), _P]),
    "sqc_update_subcircuit_outputs": (_c.c_int32, [_P, _c.c_int64, _c.POINTER(_P), _c.c_int, _c.c_int, _P]),
    "sqc_unload": (_c.c_int32, [_P, _c.c_int64]),
    "sqc_set_qubit_roles": (_c.c_int32, [_P, _c.c_int64, _P, _c.POINTER(_c.c_int64), _c.POINTER(_c.c_int32)]),
    "sqc_release_query": (_c.c_int32, [_P, _c.c_int64]),
    "sqc_reconstruct": (_c.c_int32, [_P, _c.c_int64, _c.c_int, _P, _c.c_int, _c.c_uint64, _P, _P]),
    "sqc_reconstruct_outputs": (_c.c_int32, [_P, _c.c_int64, _c.POINTER(_P), _c.c_int, _c.c_int, _c.c_int, _P,
                                             _c.c_int, _c.c_uint64, _P, _P]),
    "sqc_top_bins": (_c.c_int32, [_P, _c.c_int64, _P, _c.c_int, _c.c_uint64, _c.c_int32, _c.c_double, _P, _P,
                                  _P, _P]),
    "sqc_reconstruct_select": (_c.c_int32, [_P, _c.c_int64, _c.POINTER(_P), _c.c_int, _c.c_int, _c.c_int, _P,
                                            _c.c_int, _c.c_uint64, _P, _c.c_int32, _c.c_double, _P, _P, _P, _P]),
    "sqc_query_fused_select": (_c.c_int32, [_P, _c.c_int64, _c.POINTER(_c.c_int32)]),
    "sqc_query_info": (_c.c_int32, [_P, _c.c_int64, _c.POINTER(_c.c_int32), _c.POINTER(_c.c_double),
                                    _c.POINTER(_c.c_double), _c.POINTER(_c.c_uint64)]),
    "sqc_query_step": (_c.c_int32, [_P, _c.c_int64, _c.c_int32, _c.POINTER(_c.c_int64), _c.POINTER(_c.c_int64),
                                    _c.POINTER(_c.c_int64)]),
    "sqc_query_tc_steps": (_c.c_int32, [_P, _c.c_int64, _c.POINTER(_c.c_int32), _c.POINTER(_c.c_int32)]),
    "sqc_top_bins_noalloc": (_c.c_int32, [_c.c_int, _P, _c.c_int, _c.c_uint64, _c.c_int32, _c.c_double, _P, _P,
                                          _P, _P]),
    "sqc_batch_create": (_c.c_int32, [_P, _c.c_int32, _P, _P, _c.c_int, _P, _c.c_int, _c.POINTER(_c.c_int64)]),
    "sqc_batch_run": (_c.c_int32, [_P, _c.c_int64, _P]),
    "sqc_batch_status": (_c.c_int32, [_P, _c.c_int64]),
    "sqc_batch_release": (_c.c_int32, [_P, _c.c_int64]),
    "sqc_batch_inject_stall": (_c.c_int32, [_P, _c.c_int64, _c.c_int32]),
    "sqc_plan_preview": (_c.c_int32, [_P, _P, _P, _c.POINTER(_c.c_int32), _P, _c.c_int32,
                                      _c.POINTER(_c.c_int32), _P, _c.c_int32, _P, _P, _c.c_char_p, _c.c_int32]),
    "sqc_batch_autotune": (_c.c_int32, [_P, _c.c_int32, _P, _P, _c.c_int, _P, _c.c_int32,
                                        _c.POINTER(_c.c_int32), _c.POINTER(_c.c_int32), _P]),
    "sqc_query_autotune": (_c.c_int32, [_P, _c.c_int64, _c.c_int, _P, _c.c_int, _c.c_uint64, _c.c_int32,
                                        _c.POINTER(_c.c_int32), _P]),
    "sqc_server_default_config": (None, [_P]),
    "sqc_server_create": (_c.c_int32, [_P, _P, _c.POINTER(_P)]),
    "sqc_server_submit": (_c.c_int32, [_P, _c.c_int64, _P, _c.c_int32, _c.POINTER(_c.c_int64)]),
    "sqc_server_poll": (_c.c_int32, [_P, _c.c_int64, _c.POINTER(_c.c_int32), _c.POINTER(_c.c_double),
                                     _c.POINTER(_c.c_int32)]),
    "sqc_server_result": (_c.c_int32, [_P, _c.c_int64, _P, _c.c_uint64]),
    "sqc_server_drain": (_c.c_int32, [_P, _c.c_double]),
    "sqc_server_stats": (_c.c_int32, [_P, _c.POINTER(_c.c_int64), _c.POINTER(_c.c_int64), _c.POINTER(_c.c_int64)]),
    "sqc_server_destroy": (None, [_P]),
    "sqc_memory_info": (_c.c_int32, [_P, _c.POINTER(_c.c_uint64), _c.POINTER(_c.c_uint64)]),
    "sqc_assign_states": (_c.c_int32, [_c.c_int32, _P, _c.c_uint64, _P]),
    "sqc_query_slices": (_c.c_int32, [_P, _c.c_int64, _c.POINTER(_c.c_int32), _P, _c.c_int32]),
    "sqc_recursion_roles": (_c.c_int32, [_P, _P, _c.c_uint64, _P]),
    "sqc_profile_enable": (_c.c_int32, [_P, _c.c_int]),
    "sqc_profile_read": (_c.c_int32, [_P, _P, _P, _P]),
}

STAGES = ("attribute", "merge", "contract", "final", "select")

_LIB = None


def lib_path() -> str:
    return os.path.join(_HERE, "libsqc.so")


def load_library():
    """Load libsqc.so (built by ``_build.build()``); raises if it is missing."""
    global _LIB
    if _LIB is not None:
        return _LIB
    path = lib_path()
    if not os.path.exists(path):
        raise RuntimeError(f"CUDA library not built: {path} is missing (run __graft_entry__.build())")
    lib = ctypes.CDLL(path)
    for name, (res, args) in _SIGS.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _LIB = lib
    return lib


def _ptr(t) -> int:
    """Device or host address of a torch tensor or numpy array."""
    if t is None:
        return 0
    if isinstance(t, np.ndarray):
        return t.ctypes.data
    return t.data_ptr()


def _stream_handle(stream) -> int:
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


def _dtype_code(t) -> int:
    name = str(t.dtype)
    if name.endswith("float32"):
        return F32
    if name.endswith("float64"):
        return F64
    raise TypeError(f"unsupported dtype {t.dtype}: float32 or float64")


class Context:
    """One library context on one GPU (C ABI: sqc_create / sqc_destroy)."""

    def __init__(self, device: int = 0, hbm_budget_bytes: int = 0, max_active_qubits: int = 32,
                 fp64_chunk_min_edges: int = 12, chunk_terms: int = 256, slice_edges: int = 0,
                 select_resident: bool = True, merge_pyramid: bool = False, slice_input_log2: int = 0,
                 slice_intermediate_log2: int = 0, tc_pairs: bool | None = None, wait_limit_ms: int = 0,
                 fused_query: bool = False, pdl: bool = True, contraction_order: int = 0,
                 fused_select: bool = True):
        self._lib = load_library()
        cfg = _Config()
        self._lib.sqc_default_config(ctypes.byref(cfg))
        cfg.hbm_budget_bytes = hbm_budget_bytes
        cfg.max_active_qubits = max_active_qubits
        cfg.fp64_chunk_min_edges = fp64_chunk_min_edges
        cfg.chunk_terms = chunk_terms
        cfg.slice_edges = slice_edges
        cfg.select_resident = int(bool(select_resident))
        cfg.merge_pyramid = int(bool(merge_pyramid))
        cfg.slice_input_log2 = slice_input_log2
        cfg.slice_intermediate_log2 = slice_intermediate_log2
        if tc_pairs is not None:
            cfg.tc_pairs = int(bool(tc_pairs))
        cfg.wait_limit_ms = wait_limit_ms
        cfg.fused_query = int(bool(fused_query))
        cfg.pdl = int(bool(pdl))
        cfg.contraction_order = int(contraction_order)
        cfg.fused_select = int(bool(fused_select))
        h = _P()
        st = self._lib.sqc_create(ctypes.byref(h), device, ctypes.byref(cfg))
        if st != 0:
            raise SQCError(st, self._lib.sqc_last_error(None).decode())
        self._h = h
        self.device = device
        self._keep = {}

    def close(self):
        if getattr(self, "_h", None):
            self._lib.sqc_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def _check(self, st: int):
        if st != 0:
            raise SQCError(st, self._lib.sqc_last_error(self._h).decode())

    # -- circuits ---------------------------------------------------------
    def load_subcircuit_outputs(self, n_qubits: int, edge_up: Sequence[int], edge_down: Sequence[int],
                                n_data: Sequence[int], data_qubit: Sequence[int], probs: list, stream=None) -> int:
        """Attribute and keep resident one circuit's subcircuit outputs.
        probs: per subcircuit a [4^k_i, 2^w_i] float32/float64 tensor, all on
        the GPU or all on the host (torch CPU tensor or numpy array)."""
        arrs = [np.ascontiguousarray(np.asarray(a, dtype=np.int32)) for a in (edge_up, edge_down, n_data, data_qubit)]
        g = _Graph()
        g.n_qubits = n_qubits
        g.n_subcircuits = len(arrs[2])
        g.n_edges = len(arrs[0])
        ip = ctypes.POINTER(ctypes.c_int32)
        g.edge_up, g.edge_down, g.n_data, g.data_qubit = (a.ctypes.data_as(ip) for a in arrs)
        on_dev, ptrs, dt = self._prob_ptrs(probs)
        cid = ctypes.c_int64()
        self._check(self._lib.sqc_load_subcircuit_outputs(self._h, ctypes.byref(g), ptrs, dt, on_dev,
                                                          ctypes.byref(cid), _stream_handle(stream)))
        return cid.value

    def update_subcircuit_outputs(self, circuit: int, probs: list, stream=None):
        on_dev, ptrs, dt = self._prob_ptrs(probs)
        self._check(self._lib.sqc_update_subcircuit_outputs(self._h, circuit, ptrs, dt, on_dev,
                                                            _stream_handle(stream)))

    @staticmethod
    def _prob_ptrs(probs):
        on_dev = None
        dt = None
        ptrs = (ctypes.c_void_p * len(probs))()
        for i, p in enumerate(probs):
            dev = (not isinstance(p, np.ndarray)) and p.is_cuda
            if on_dev is None:
                on_dev = dev
            if dev != on_dev:
                raise ValueError("probs must be all on the GPU or all on the host")
            d = _dtype_code(p)
            if dt is None:
                dt = d
            if d != dt:
                raise ValueError("probs must share one dtype")
            if not (p.flags["C_CONTIGUOUS"] if isinstance(p, np.ndarray) else p.is_contiguous()):
                raise ValueError("probs must be contiguous")
            ptrs[i] = _ptr(p)
        return int(bool(on_dev)), ptrs, dt

    def unload(self, circuit: int):
        self._check(self._lib.sqc_unload(self._h, circuit))

    # -- queries ----------------------------------------------------------
    def set_qubit_roles(self, circuit: int, roles) -> tuple[int, int]:
        r = np.ascontiguousarray(np.asarray(roles, dtype=np.int8))
        q = ctypes.c_int64()
        na = ctypes.c_int32()
        self._check(self._lib.sqc_set_qubit_roles(self._h, circuit, r.ctypes.data, ctypes.byref(q),
                                                  ctypes.byref(na)))
        return q.value, na.value

    def release_query(self, query: int):
        self._check(self._lib.sqc_release_query(self._h, query))

    def query_info(self, query: int) -> dict:
        ns, fl, mb, wb = ctypes.c_int32(), ctypes.c_double(), ctypes.c_double(), ctypes.c_uint64()
        self._check(self._lib.sqc_query_info(self._h, query, ctypes.byref(ns), ctypes.byref(fl), ctypes.byref(mb),
                                             ctypes.byref(wb)))
        return {"n_steps": ns.value, "flops": fl.value, "merge_bytes": mb.value, "work_bytes": wb.value}

    def query_slices(self, query: int) -> list[int]:
        """Cut edges the query slices (Section 6.3), in the greedy order."""
        n = ctypes.c_int32()
        buf = (ctypes.c_int32 * 64)()
        self._check(self._lib.sqc_query_slices(self._h, query, ctypes.byref(n), buf, 64))
        return list(buf[: n.value])

    def memory_info(self) -> dict:
        """Device bytes the context holds and its HBM budget (0: none)."""
        held, budget = ctypes.c_uint64(), ctypes.c_uint64()
        self._check(self._lib.sqc_memory_info(self._h, ctypes.byref(held), ctypes.byref(budget)))
        return {"held": held.value, "budget": budget.value}

    def query_steps(self, query: int) -> list[tuple[int, int, int]]:
        """(M, N, Kd) of every contraction step, in launch order."""
        out = []
        for s in range(self.query_info(query)["n_steps"]):
            m, n, k = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64()
            self._check(self._lib.sqc_query_step(self._h, query, s, ctypes.byref(m), ctypes.byref(n), ctypes.byref(k)))
            out.append((m.value, n.value, k.value))
        return out

    def query_tc_steps(self, query: int) -> tuple[int, int]:
        """(steps on the tensor cores, steps) of the query's split-BF16 plan."""
        a, b = ctypes.c_int32(), ctypes.c_int32()
        self._check(self._lib.sqc_query_tc_steps(self._h, query, ctypes.byref(a), ctypes.byref(b)))
        return a.value, b.value

    def reconstruct(self, query: int, out, precision: str = "fp32", total_prob=None, stream=None):
        """Bins of `query` into the device tensor `out` (float32/float64,
        2^n_active elements); total_prob: optional device float64 tensor of
        one element receiving the FP64 sum of the bins."""
        if not out.is_cuda:
            raise ValueError("out must be a device tensor")
        if total_prob is not None and (not total_prob.is_cuda or str(total_prob.dtype) != "torch.float64"):
            raise ValueError("total_prob must be a device float64 tensor")
        self._check(self._lib.sqc_reconstruct(self._h, query, PREC[precision], _ptr(out), _dtype_code(out),
                                              out.numel() * out.element_size(), _ptr(total_prob),
                                              _stream_handle(stream)))

    def reconstruct_outputs(self, query: int, probs: list, out, precision: str = "fp32", total_prob=None,
                            stream=None, host_direct: bool = False):
        """Bins of `query` for fresh subcircuit outputs `probs` (one recursion
        step, sqc_reconstruct_outputs): attribution fused into the merge; the
        circuit's resident tensors are not changed."""
        if not out.is_cuda:
            raise ValueError("out must be a device tensor")
        if total_prob is not None and (not total_prob.is_cuda or str(total_prob.dtype) != "torch.float64"):
            raise ValueError("total_prob must be a device float64 tensor")
        on_dev, ptrs, dt = self._prob_ptrs(probs)
        if host_direct and not on_dev:
            on_dev = 2          # pinned host tensors read in place by the kernels
        self._check(self._lib.sqc_reconstruct_outputs(self._h, query, ptrs, dt, on_dev, PREC[precision], _ptr(out),
                                                      _dtype_code(out), out.numel() * out.element_size(),
                                                      _ptr(total_prob), _stream_handle(stream)))

    def reconstruct_select(self, query: int, out, k: int, threshold: float = -math.inf, probs: list | None = None,
                           precision: str = "fp32", total_prob=None, bins_out=None, probs_out=None, n_found=None,
                           stream=None, host_direct: bool = False):
        """One recursion step (sqc_reconstruct_select): the bins of `query`
        into `out` (from the resident tensors, or from fresh outputs `probs`),
        then their k largest (value descending, bin ascending, >= threshold),
        fused into one launch where the plan allows it.  Returns device
        tensors (bins int64 [k], probs float64 [k], n_found int32 [1])."""
        import torch
        if not out.is_cuda:
            raise ValueError("out must be a device tensor")
        if total_prob is not None and (not total_prob.is_cuda or str(total_prob.dtype) != "torch.float64"):
            raise ValueError("total_prob must be a device float64 tensor")
        dev = out.device
        if bins_out is None:
            bins_out = torch.empty(k, dtype=torch.int64, device=dev)
        if probs_out is None:
            probs_out = torch.empty(k, dtype=torch.float64, device=dev)
        if n_found is None:
            n_found = torch.empty(1, dtype=torch.int32, device=dev)
        if probs is None:
            ptrs, dt, on_dev = None, F32, 1
        else:
            on_dev, ptrs, dt = self._prob_ptrs(probs)
            if host_direct and not on_dev:
                on_dev = 2      # pinned host tensors read in place by the kernels
        self._check(self._lib.sqc_reconstruct_select(self._h, query, ptrs, dt, on_dev, PREC[precision], _ptr(out),
                                                     _dtype_code(out), out.numel() * out.element_size(),
                                                     _ptr(total_prob), k, float(threshold), _ptr(bins_out),
                                                     _ptr(probs_out), _ptr(n_found), _stream_handle(stream)))
        return bins_out, probs_out, n_found

    def query_fused_select(self, query: int) -> int:
        """Contraction steps sqc_reconstruct_select runs inside its fused
        selection launch for this query (0: per-stage launches)."""
        n = ctypes.c_int32()
        self._check(self._lib.sqc_query_fused_select(self._h, query, ctypes.byref(n)))
        return n.value

    # -- batches ----------------------------------------------------------
    def batch_create(self, queries: list[int], outs: list, totals=None, precision: str = "fp32") -> int:
        """Persistent launches for many queries (sqc_batch_create): outs[j]
        is the device tensor receiving query j's bins (all float32 or all
        float64); totals: optional device float64 tensor [len(queries)];
        precision "split_bf16" runs each query's tensor-core steps on
        tcgen05 between the phases."""
        n = len(queries)
        qa = (ctypes.c_int64 * n)(*queries)
        oa = (ctypes.c_void_p * n)(*[_ptr(o) for o in outs])
        dt = _dtype_code(outs[0])
        if any(_dtype_code(o) != dt for o in outs):
            raise ValueError("batch outputs must share one dtype")
        b = ctypes.c_int64()
        self._check(self._lib.sqc_batch_create(self._h, n, qa, oa, dt, _ptr(totals), PREC[precision],
                                               ctypes.byref(b)))
        return b.value

    def batch_run(self, batch: int, stream=None):
        self._check(self._lib.sqc_batch_run(self._h, batch, _stream_handle(stream)))

    def batch_status(self, batch: int):
        self._check(self._lib.sqc_batch_status(self._h, batch))

    def batch_release(self, batch: int):
        self._check(self._lib.sqc_batch_release(self._h, batch))

    def batch_inject_stall(self, batch: int, on: bool = True):
        self._check(self._lib.sqc_batch_inject_stall(self._h, batch, int(bool(on))))

    def batch_autotune(self, queries: list[int], outs: list, totals=None, reps: int = 5):
        """Time the batched launch of `queries` under each contraction order
        and tile policy (sqc_batch_autotune) and keep the fastest.  Returns
        (best tile policy, best order, mean ms per launch [order][policy])."""
        n = len(queries)
        qa = (ctypes.c_int64 * n)(*queries)
        oa = (ctypes.c_void_p * n)(*[_ptr(o) for o in outs])
        dt = _dtype_code(outs[0])
        if any(_dtype_code(o) != dt for o in outs):
            raise ValueError("batch outputs must share one dtype")
        best, order = ctypes.c_int32(), ctypes.c_int32()
        ms = (ctypes.c_float * 6)()
        self._check(self._lib.sqc_batch_autotune(self._h, n, qa, oa, dt, _ptr(totals), reps, ctypes.byref(best),
                                                 ctypes.byref(order), ms))
        return best.value, order.value, [list(ms[0:3]), list(ms[3:6])]

    def query_autotune(self, query: int, out, precision: str = "fp32", reps: int = 5):
        """Time reconstructions of `query` under the greedy and the
        fewest-multiplications contraction order (sqc_query_autotune) and keep
        the faster plan.  Returns (best order, [ms greedy, ms fewest])."""
        best = ctypes.c_int32()
        ms = (ctypes.c_float * 2)()
        self._check(self._lib.sqc_query_autotune(self._h, query, PREC[precision], _ptr(out), _dtype_code(out),
                                                 out.numel() * out.element_size(), reps, ctypes.byref(best), ms))
        return best.value, list(ms)

    def top_bins(self, query: int, probs, k: int, threshold: float = -math.inf, bins_out=None, probs_out=None,
                 n_found=None, stream=None):
        """Largest bins of the device tensor `probs` (value descending, bin
        ascending, values >= threshold, at most k).  Outputs are device
        tensors (allocated here when not given): (bins int64 [k], probs
        float64 [k], n_found int32 [1])."""
        import torch
        dev = probs.device
        if bins_out is None:
            bins_out = torch.empty(k, dtype=torch.int64, device=dev)
        if probs_out is None:
            probs_out = torch.empty(k, dtype=torch.float64, device=dev)
        if n_found is None:
            n_found = torch.empty(1, dtype=torch.int32, device=dev)
        self._check(self._lib.sqc_top_bins(self._h, query, _ptr(probs), _dtype_code(probs), probs.numel(), k,
                                           float(threshold), _ptr(bins_out), _ptr(probs_out), _ptr(n_found),
                                           _stream_handle(stream)))
        return bins_out, probs_out, n_found


def _profile_enable(self, on=True):
    """Stage timing on/off (sqc_profile_enable); turning it on clears it.
    on=2: graph mode (events captured into a CUDA graph are kept; each read
    reports the latest replay)."""
    self._check(self._lib.sqc_profile_enable(self._h, int(on)))


def _profile_read(self) -> dict:
    """Per-stage milliseconds and call counts since the last read, and the
    number of kernels launched (sqc_profile_read)."""
    ms = (ctypes.c_double * len(STAGES))()
    calls = (ctypes.c_int64 * len(STAGES))()
    launches = ctypes.c_int64()
    self._check(self._lib.sqc_profile_read(self._h, ms, calls, ctypes.byref(launches)))
    return {"ms": dict(zip(STAGES, list(ms))), "calls": dict(zip(STAGES, list(calls))),
            "launches": launches.value}


Context.profile_enable = _profile_enable
Context.profile_read = _profile_read


def top_bins_noalloc(probs, k: int, threshold: float = -math.inf, bins_out=None, probs_out=None, n_found=None,
                     stream=None):
    """Allocation-free selection (sqc_top_bins_noalloc): same result as
    Context.top_bins, scratch in the library's static device array, no
    context needed.  Calls that may overlap on the GPU must be serialised."""
    import torch
    lib = load_library()
    dev = probs.device
    if bins_out is None:
        bins_out = torch.empty(k, dtype=torch.int64, device=dev)
    if probs_out is None:
        probs_out = torch.empty(k, dtype=torch.float64, device=dev)
    if n_found is None:
        n_found = torch.empty(1, dtype=torch.int32, device=dev)
    st = lib.sqc_top_bins_noalloc(dev.index or 0, _ptr(probs), _dtype_code(probs), probs.numel(), k, float(threshold),
                                  _ptr(bins_out), _ptr(probs_out), _ptr(n_found), _stream_handle(stream))
    if st != 0:
        raise SQCError(st, lib.sqc_last_error(None).decode())
    return bins_out, probs_out, n_found


class _ServerConfig(ctypes.Structure):
    _fields_ = [("max_batch", ctypes.c_int32), ("n_streams", ctypes.c_int32), ("plain", ctypes.c_int32),
                ("reserved", ctypes.c_int32 * 5)]


class Server:
    """Continuous-batching serving loop over a context (sqc_server_*).  The
    server thread owns the context until close()."""

    def __init__(self, ctx: Context, max_batch: int = 64, n_streams: int = 4, plain: bool = False):
        self._lib = ctx._lib
        self._ctx = ctx
        cfg = _ServerConfig()
        self._lib.sqc_server_default_config(ctypes.byref(cfg))
        cfg.max_batch, cfg.n_streams, cfg.plain = max_batch, n_streams, int(plain)
        h = _P()
        ctx._check(self._lib.sqc_server_create(ctx._h, ctypes.byref(cfg), ctypes.byref(h)))
        self._h = h

    def submit(self, circuit: int, roles) -> int:
        r = np.ascontiguousarray(np.asarray(roles, dtype=np.int8))
        t = ctypes.c_int64()
        st = self._lib.sqc_server_submit(self._h, circuit, r.ctypes.data, r.size, ctypes.byref(t))
        if st != 0:
            raise SQCError(st, "submit failed")
        return t.value

    def poll(self, ticket: int):
        """(state, latency_us, n_active); state 0 waiting, 1 running, 2 done, 3 failed, 4 collected."""
        s, lat, na = ctypes.c_int32(), ctypes.c_double(), ctypes.c_int32()
        st = self._lib.sqc_server_poll(self._h, ticket, ctypes.byref(s), ctypes.byref(lat), ctypes.byref(na))
        if st != 0:
            raise SQCError(st, "request failed")
        return s.value, lat.value, na.value

    def result(self, ticket: int) -> np.ndarray:
        _, _, na = self.poll(ticket)
        out = np.empty(1 << na, dtype=np.float32)
        st = self._lib.sqc_server_result(self._h, ticket, out.ctypes.data, out.size)
        if st != 0:
            raise SQCError(st, "result not available")
        return out

    def drain(self, timeout_s: float = 60.0):
        st = self._lib.sqc_server_drain(self._h, timeout_s)
        if st != 0:
            raise SQCError(st, "drain timed out")

    def stats(self) -> dict:
        a, b, c = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64()
        self._lib.sqc_server_stats(self._h, ctypes.byref(a), ctypes.byref(b), ctypes.byref(c))
        return {"launches": a.value, "admitted": b.value, "busy_refusals": c.value}

    def close(self):
        if getattr(self, "_h", None):
            self._lib.sqc_server_destroy(self._h)
            self._h = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


def assign_states(l, M: int) -> list[int]:
    """Algorithm 2's target bin counts (sqc_assign_states); host only."""
    lib = load_library()
    a = np.ascontiguousarray(np.asarray(l, dtype=np.uint64))
    out = np.empty_like(a)
    st = lib.sqc_assign_states(a.size, a.ctypes.data, int(M), out.ctypes.data)
    if st != 0:
        raise SQCError(st, "assign_states")
    return out.tolist()


def _graph_struct(n_qubits: int, edge_up, edge_down, n_data, data_qubit):
    """(sqc_graph, the int32 arrays it points into -- keep them alive)."""
    arrs = [np.ascontiguousarray(np.asarray(a, dtype=np.int32)) for a in (edge_up, edge_down, n_data, data_qubit)]
    g = _Graph()
    g.n_qubits, g.n_subcircuits, g.n_edges = n_qubits, len(arrs[2]), len(arrs[0])
    ip = ctypes.POINTER(ctypes.c_int32)
    g.edge_up, g.edge_down, g.n_data, g.data_qubit = (a.ctypes.data_as(ip) for a in arrs)
    return g, arrs


def recursion_roles(n_qubits: int, edge_up, edge_down, n_data, data_qubit, zoom, M: int) -> np.ndarray:
    """Roles of one recursion (sqc_recursion_roles); zoom: per qubit
    ROLE_ZOOM0/ROLE_ZOOM1 for fixed qubits, anything else free.  Host only."""
    lib = load_library()
    g, arrs = _graph_struct(n_qubits, edge_up, edge_down, n_data, data_qubit)
    z = np.ascontiguousarray(np.asarray(zoom, dtype=np.int8))
    roles = np.empty(n_qubits, dtype=np.int8)
    st = lib.sqc_recursion_roles(ctypes.byref(g), z.ctypes.data, int(M), roles.ctypes.data)
    if st != 0:
        raise SQCError(st, "recursion_roles")
    return roles


def plan_preview(n_qubits: int, edge_up, edge_down, n_data, data_qubit, roles, **config) -> dict:
    """The FP32 plan sqc_set_qubit_roles would build (sqc_plan_preview):
    host only, no GPU.  config: the Context keyword arguments that shape a
    plan (max_active_qubits, slice_edges, slice_input_log2,
    slice_intermediate_log2, ...).  Returns {"steps": [(M, N, K), ...],
    "sliced": [edge ids], "flops": 2 sum MNK, "work_bytes": ...}."""
    lib = load_library()
    g, arrs = _graph_struct(n_qubits, edge_up, edge_down, n_data, data_qubit)
    r = np.ascontiguousarray(np.asarray(roles, dtype=np.int8))
    cfg = _Config()
    lib.sqc_default_config(ctypes.byref(cfg))
    for k, v in config.items():
        if not hasattr(cfg, k):
            raise TypeError(f"unknown configuration field {k}")
        setattr(cfg, k, int(v))
    cap = max(1, len(arrs[2]))
    steps = np.zeros((cap, 3), dtype=np.int64)
    sliced = np.zeros(max(1, len(arrs[0])), dtype=np.int32)
    n_steps, n_sliced = ctypes.c_int32(), ctypes.c_int32()
    flops, work = ctypes.c_double(), ctypes.c_uint64()
    err = ctypes.create_string_buffer(256)
    st = lib.sqc_plan_preview(ctypes.byref(g), r.ctypes.data, ctypes.byref(cfg), ctypes.byref(n_steps),
                              steps.ctypes.data, cap, ctypes.byref(n_sliced), sliced.ctypes.data, sliced.size,
                              ctypes.byref(flops), ctypes.byref(work), err, len(err))
    if st != 0:
        raise SQCError(st, err.value.decode())
    return {"steps": [tuple(int(x) for x in s) for s in steps[:n_steps.value]],
            "sliced": sliced[:n_sliced.value].tolist(), "flops": flops.value, "work_bytes": work.value}


def declared_symbols() -> list[str]:
    """Function names declared with SQC_API in include/sqc.h."""
    import re
    hdr = os.path.join(os.path.dirname(_HERE), "include", "sqc.h")
    text = open(hdr).read()
    return sorted(set(re.findall(r"SQC_API\s+[\w\s\*]*?\b(sqc_\w+)\s*\(", text)))

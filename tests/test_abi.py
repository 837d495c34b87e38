"""Host-side checks of the C-ABI library that need no GPU: it builds, loads,
exports every function include/sqc.h declares, and reports the missing GPU
as an error instead of falling back to anything."""
import ctypes

import pytest

import paper_2207_00933_gb300 as sqc
from paper_2207_00933_gb300 import _build


@pytest.fixture(scope="module")
def lib():
    _build.build()
    return sqc.load_library()


def test_every_declared_symbol_is_exported(lib):
    names = sqc.declared_symbols()
    assert len(names) >= 12
    for n in names:
        assert hasattr(lib, n), n


def test_binding_covers_the_header(lib):
    # the binding declares a signature for every entry point of the header
    assert set(sqc.declared_symbols()) <= set(sqc._SIGS)


def test_default_config(lib):
    cfg = sqc._Config()
    lib.sqc_default_config(ctypes.byref(cfg))
    assert cfg.max_active_qubits == 32 and cfg.fp64_chunk_min_edges == 12 and cfg.chunk_terms == 256
    assert cfg.select_resident == 1
    assert cfg.merge_pyramid == 0 and cfg.slice_input_log2 == 0 and cfg.slice_intermediate_log2 == 0
    assert cfg.tc_pairs == 0 and cfg.wait_limit_ms == 0 and cfg.fused_query == 0 and cfg.pdl == 1 and cfg.contraction_order == 0
    assert cfg.fused_select == 1


def test_create_without_gpu_fails_loudly(lib):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    with pytest.raises(sqc.SQCError) as ei:
        sqc.Context()
    assert ei.value.status == 4          # SQC_ECUDA


def test_null_arguments_are_rejected(lib):
    assert lib.sqc_create(None, 0, None) == 1
    assert lib.sqc_last_error(None)
    lib.sqc_destroy(None)                # ignored


def test_assign_states_matches_algorithm_2_oracle(lib):
    import numpy as np
    import oracle as O
    rng = np.random.default_rng(0)
    for _ in range(200):
        n = int(rng.integers(1, 7))
        l = [1 << int(rng.integers(0, 12)) for _ in range(n)]
        M = 1 << int(rng.integers(0, 30))
        assert sqc.assign_states(l, M) == O.states_assignment(l, M)
    assert sqc.assign_states([2 ** 7, 2 ** 8, 2 ** 7, 2 ** 8], 2 ** 20) == [32] * 4


def test_recursion_roles_match_oracle(lib):
    import numpy as np
    import oracle as O
    from synthetic import workloads as W
    for w, M in ((W.merged_30q(), 2 ** 20), (W.grid_40q(), 2 ** 22)):
        c = w.circuit
        g = O.Graph.from_arrays(c.n_qubits, *c.graph_arrays())
        rng = np.random.default_rng(1)
        for trial in range(5):
            zoom = {}
            if trial:
                for q in rng.choice(c.n_qubits, size=int(rng.integers(1, 12)), replace=False):
                    zoom[int(q)] = int(rng.integers(2))
            zarr = np.full(c.n_qubits, O.MERGED, dtype=np.int8)
            for q, v in zoom.items():
                zarr[q] = O.ZOOM1 if v else O.ZOOM0
            got = sqc.recursion_roles(c.n_qubits, *c.graph_arrays(), zarr, M)
            assert got.tolist() == list(O.roles_for_recursion(g, zoom, M))

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

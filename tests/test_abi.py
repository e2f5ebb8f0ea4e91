"""The C-ABI library loads and exports every declared entry point; host-side
argument checks answer before any CUDA call (runs without a GPU)."""
import ctypes
import os
import re

import numpy as np
import pytest

from paper_2104_13209_gb300 import build, kclique, synth

HEADER = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include", "kclique.h")


@pytest.fixture(scope="module")
def lib():
    build.build()
    return kclique.load()


def declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(kc_[a-z0-9_]+)\s*\(", src)))


def test_header_declares_what_binding_lists():
    assert declared_functions() == sorted(kclique.EXPORTED)


def test_every_declared_symbol_is_exported(lib):
    for name in declared_functions():
        assert hasattr(lib, name), name


def test_version_and_status_names(lib):
    assert lib.kc_version() >= 10000
    for code, name in [(0, "KC_OK"), (2, "KC_E_INVALID_GRAPH"), (4, "KC_E_OVERFLOW"), (5, "KC_E_TIMEOUT")]:
        assert lib.kc_status_name(code).decode() == name


def _create(lib, rp, ci, n, nnz, orient=1, out=True):
    h = ctypes.c_void_p()
    rp_p = rp.ctypes.data if rp is not None else None
    ci_p = ci.ctypes.data if ci is not None else None
    return lib.kc_graph_create(rp_p, ci_p, n, nnz, 0, orient, 1, None, ctypes.byref(h) if out else None)


def test_argument_checks_without_gpu(lib):
    rp = np.array([0, 1, 2], dtype=np.uint32)
    ci = np.array([1, 0], dtype=np.uint32)
    assert _create(lib, rp, ci, 2, 2, out=False) == kclique.KC_E_INVALID_ARG
    assert _create(lib, None, ci, 2, 2) == kclique.KC_E_INVALID_ARG
    assert _create(lib, rp, None, 2, 2) == kclique.KC_E_INVALID_ARG
    assert _create(lib, rp, ci, 2, 2, orient=7) == kclique.KC_E_INVALID_ARG
    assert _create(lib, rp, ci, 2, 3) == kclique.KC_E_INVALID_GRAPH  # odd nnz cannot be symmetric
    assert _create(lib, rp, ci, 2, 1 << 32) == kclique.KC_E_UNSUPPORTED
    assert "orientation" in kclique.last_error() or "nnz" in kclique.last_error()
    assert lib.kc_graph_destroy(None) == 0
    total = ctypes.c_uint64()
    assert lib.kc_count(None, 3, 0, 0, 0, ctypes.byref(total), None, None, None) == kclique.KC_E_INVALID_ARG
    assert lib.kc_graph_info_get(None, None) == kclique.KC_E_INVALID_ARG


def _has_gpu():
    try:
        import torch

        return torch.cuda.is_available()
    except Exception:
        return False


@pytest.mark.skipif(_has_gpu(), reason="checks the behaviour on a machine without a GPU")
def test_no_gpu_fails_loudly(lib):
    # no fallback: a graph cannot be created, the error says why
    with pytest.raises(kclique.KCError) as e:
        kclique.Graph(np.array([0, 1, 2], dtype=np.uint32), np.array([1, 0], dtype=np.uint32))
    assert e.value.status in (kclique.KC_E_CUDA, kclique.KC_E_NO_MEMORY)
    assert kclique.last_error()
    with pytest.raises(kclique.KCError):
        kclique.Batch([synth.complete_graph(3)])
    with pytest.raises(kclique.KCError):
        kclique.Server()


def test_missing_library_raises(monkeypatch, tmp_path):
    monkeypatch.setattr(kclique, "_lib", None)
    monkeypatch.setattr(build, "LIB", str(tmp_path / "absent.so"))
    with pytest.raises(ImportError):
        kclique.load()

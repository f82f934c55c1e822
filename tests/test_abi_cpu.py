"""Host-side checks of the C ABI that need no GPU: the library builds, loads, exports
every entry point declared in include/cos.h, and rejects malformed graphs and
arguments with an error code (validation happens before any CUDA call)."""
import ctypes
import os
import re
import subprocess

import numpy as np
import pytest

from paper_2501_00675_gb300 import _build, binding
from workloads import figure_graph

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    _build.build()
    return binding.load_library()


def _declared():
    with open(os.path.join(ROOT, "include", "cos.h")) as f:
        text = f.read()
    return sorted(set(re.findall(r"^\s*(?:int|const char\*)\s+(cos_\w+)\s*\(", text, re.M)))


def test_header_declarations_are_exported(lib):
    names = _declared()
    assert len(names) >= 9
    out = subprocess.run(["nm", "-D", "--defined-only", _build.LIB], capture_output=True, text=True, check=True).stdout
    exported = set(re.findall(r"\sT\s+(cos_\w+)", out))
    missing = [n for n in names if n not in exported]
    assert not missing, missing
    for n in names:
        assert getattr(lib, n) is not None


def _create(lib, widths, counts, edges, K=1, D=1):
    w = np.ascontiguousarray(widths, dtype=np.int64)
    c = np.ascontiguousarray(counts, dtype=np.int64)
    e = np.ascontiguousarray(edges, dtype=np.int32).reshape(-1, 5)
    h = ctypes.c_void_p()
    rc = lib.cos_create_graph(len(w), w.ctypes.data, c.ctypes.data, e.ctypes.data if e.size else None, K, D,
                              ctypes.byref(h))
    if rc == 0:
        lib.cos_destroy(h)
    return rc, lib.cos_last_error().decode()


def _fig():
    g = figure_graph()
    return g.widths.copy(), g.edge_counts.copy(), g.edges.copy()


@pytest.mark.parametrize("mutate,needle", [
    (lambda w, c, e: (w, c, _set(e, 3, 0, 0)), "src"),             # src from level 0 into level 2
    (lambda w, c, e: (w, c, _set(e, 0, 1, 5)), "dst"),             # dst outside level 1
    (lambda w, c, e: (w, c, _set(e, 4, 2, 1)), "kind"),            # kind >= K
    (lambda w, c, e: (w, c, _set(e, 4, 3, 7)), "time index"),      # i >= D
    (lambda w, c, e: (w, c, _set(e, 4, 4, -1)), "time index"),     # j < 0
    (lambda w, c, e: (_set1(w, 2, 0), c, e), "width"),             # an empty level
    (lambda w, c, e: (_set1(w, 0, 2), c, e), "width 1"),           # root level wider than 1
    (lambda w, c, e: (_set1(w, 4, 2), c, e), "width 1"),           # sink level wider than 1
    (lambda w, c, e: (w, _set1(c, 0, 1), e), "root"),              # in-edges into level 0
    (lambda w, c, e: (w, _set1(c, 1, -1), e), "negative"),         # negative edge count
])
def test_malformed_graphs_are_rejected(lib, mutate, needle):
    w, c, e = mutate(*_fig())
    rc, msg = _create(lib, w, c, e)
    assert rc == binding.COS_ERR_INVALID
    assert needle in msg


def _set(e, row, col, val):
    e = e.copy()
    e[row, col] = val
    return e


def _set1(a, i, val):
    a = a.copy()
    a[i] = val
    return a


def test_kind_sign_bit_is_accepted_and_bit_31_rejected(lib):
    w, c, e = _fig()
    e = e.copy()
    e[3, 2] = -1                                  # bit 31: invalid
    rc, msg = _create(lib, w, c, e)
    assert rc == binding.COS_ERR_INVALID and "kind" in msg


def test_non_consecutive_levels_rejected(lib):
    # an edge that skips a level (0 -> level 2) is invalid
    w = [1, 2, 2, 1]
    c = [0, 2, 2, 2]
    e = [[0, 1, 0, 0, 0], [0, 2, 0, 0, 0], [0, 3, 0, 0, 0], [1, 4, 0, 0, 0], [3, 5, 0, 0, 0], [4, 5, 0, 0, 0]]
    rc, msg = _create(lib, w, c, e)
    assert rc == binding.COS_ERR_INVALID and "not in level" in msg


def test_null_and_range_arguments(lib):
    h = ctypes.c_void_p()
    w = np.array([1, 1], dtype=np.int64)
    c = np.array([0, 1], dtype=np.int64)
    assert lib.cos_create_graph(2, w.ctypes.data, c.ctypes.data, None, 1, 1, ctypes.byref(h)) == binding.COS_ERR_INVALID
    assert lib.cos_create_graph(1, w.ctypes.data, c.ctypes.data, None, 1, 1, ctypes.byref(h)) == binding.COS_ERR_INVALID
    assert lib.cos_create_graph(2, None, c.ctypes.data, None, 1, 1, ctypes.byref(h)) == binding.COS_ERR_INVALID
    assert lib.cos_create_graph(2, w.ctypes.data, c.ctypes.data, None, 0, 1, ctypes.byref(h)) == binding.COS_ERR_INVALID
    e = np.array([[0, 1, 0, 0, 0]], dtype=np.int32)
    assert lib.cos_create_graph(2, w.ctypes.data, c.ctypes.data, e.ctypes.data, 1, 1, None) == binding.COS_ERR_INVALID
    assert lib.cos_evaluate(None, 0, None, None, None) == binding.COS_ERR_INVALID
    assert lib.cos_set_samples(None, 1, None, 0, None, 1.0, None) == binding.COS_ERR_INVALID
    assert lib.cos_destroy(None) == binding.COS_OK
    info = np.zeros(4, dtype=np.int64)
    assert lib.cos_graph_info(None, info.ctypes.data, 4) == binding.COS_ERR_INVALID


def test_binding_fails_loudly_without_library(monkeypatch, tmp_path):
    monkeypatch.setattr(binding, "_lib", None)
    monkeypatch.setattr(_build, "LIB", str(tmp_path / "missing.so"))
    with pytest.raises(RuntimeError, match="missing"):
        binding.load_library()


def test_server_arguments_checked_before_any_cuda_call(lib):
    """cos_server_*: argument errors come back as COS_ERR_INVALID without touching the
    device; NULL handles are refused (destroy accepts NULL)."""
    h = ctypes.c_void_p()
    create = lib.cos_server_create
    assert create(3, 4, None, 0, 0, 0, ctypes.byref(h)) == binding.COS_ERR_INVALID          # mode
    assert create(0, 0, None, 0, 0, 0, ctypes.byref(h)) == binding.COS_ERR_INVALID          # max_times
    assert create(0, 4, None, -1, 0, 0, ctypes.byref(h)) == binding.COS_ERR_INVALID         # max_requests
    assert create(0, 4, None, 0, -5, 0, ctypes.byref(h)) == binding.COS_ERR_INVALID         # queue_tasks
    assert create(0, 4, None, 0, 0, -1, ctypes.byref(h)) == binding.COS_ERR_INVALID         # idle_ms
    assert create(0, 4, None, 0, 0, 0, None) == binding.COS_ERR_INVALID
    for field, value in (("samples_per_lane", 3), ("layout", 2), ("rows_per_warp", 32), ("prefetch", 8),
                         ("window_chunks", -1)):
        t = binding.CosTuning()
        setattr(t, field, value)
        assert create(0, 4, ctypes.byref(t), 0, 0, 0, ctypes.byref(h)) == binding.COS_ERR_INVALID, field
    rid = ctypes.c_int64()
    m = ctypes.c_double()
    assert lib.cos_server_submit(None, None, 1, 1, 0, None, ctypes.byref(rid)) == binding.COS_ERR_INVALID
    assert lib.cos_server_poll(None, 1, ctypes.byref(m)) == binding.COS_ERR_INVALID
    assert lib.cos_server_wait(None, 1, 0, ctypes.byref(m)) == binding.COS_ERR_INVALID
    assert lib.cos_server_stats(None, None) == binding.COS_ERR_INVALID
    assert lib.cos_server_destroy(None) == binding.COS_OK


def test_server_without_a_device_reports_cuda_error(lib):
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    h = ctypes.c_void_p()
    rc = lib.cos_server_create(0, 4, None, 0, 0, 0, ctypes.byref(h))
    assert rc == binding.COS_ERR_CUDA and "device" in lib.cos_last_error().decode()

"""ctypes binding of libcosgpu.so: the C entry points under their C names, plus a
small handle class.  Argument marshalling only -- every step of the evaluation
runs in the CUDA library.  PyTorch supplies device memory and streams.

There is no fallback: if the library is missing or no GPU is present, calls
raise.
"""
from __future__ import annotations

import ctypes
import os
import threading
from typing import Optional, Sequence

import numpy as np

from . import _build

COS_OK = 0
COS_ERR_INVALID = -1
COS_ERR_OOM = -2
COS_ERR_CUDA = -3
COS_ERR_TIMEOUT = -4
COS_ERR_OVERFLOW = -5
COS_ERR_STATE = -6
COS_ERR_BUSY = -7

COS_MODE_FP64 = 0
COS_MODE_FP32_MIXED = 1
COS_MODE_COUNT_I64 = 2
COS_EVAL_ABS = 16          # flag: the same walk also sums |path| values (A(s) and its mean)

COS_T_DEVICE_DS = 0
COS_T_HOST = 1
COS_T_SAMPLE_MAJOR = 2
COS_T_BORROW = 4

EXPORTED = ["cos_create_graph", "cos_set_samples", "cos_evaluate", "cos_get_result", "cos_graph_info",
            "cos_set_tuning", "cos_get_tuning", "cos_set_trace", "cos_get_trace", "cos_evaluate_static",
            "cos_graph_share", "cos_batch_create", "cos_batch_reset", "cos_batch_set_tuning", "cos_batch_get_tuning", "cos_batch_autotune",
            "cos_batch_launch", "cos_batch_results", "cos_batch_destroy", "cos_evaluate_batch",
            "cos_selftest_exp", "cos_probe_fma_rate", "cos_set_samples_uniform", "cos_copy_times", "cos_server_create",
            "cos_server_submit", "cos_server_poll", "cos_server_wait", "cos_server_stats", "cos_server_destroy",
            "cos_destroy", "cos_last_error"]

_lock = threading.Lock()
_lib = None


class CosError(RuntimeError):
    def __init__(self, code: int, message: str):
        super().__init__(f"[{code}] {message}")
        self.code = code


class CosServerInfo(ctypes.Structure):
    _fields_ = [("launches", ctypes.c_int64), ("completed", ctypes.c_int64), ("in_flight", ctypes.c_int64),
                ("queued_tasks", ctypes.c_int64), ("published_tasks", ctypes.c_int64), ("running", ctypes.c_int32),
                ("grid", ctypes.c_int32), ("samples_per_lane", ctypes.c_int32), ("failed", ctypes.c_int32),
                ("stale_claims", ctypes.c_int64)]


class CosTuning(ctypes.Structure):
    _fields_ = [("samples_per_lane", ctypes.c_int32), ("tile_samples", ctypes.c_int32),
                ("rows_per_warp", ctypes.c_int32), ("blocks_per_sm", ctypes.c_int32),
                ("timeout_ms", ctypes.c_int32), ("layout", ctypes.c_int32), ("schedule", ctypes.c_int32),
                ("window_chunks", ctypes.c_int32), ("prefetch", ctypes.c_int32)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


def library_path() -> str:
    return _build.LIB


def load_library(build_if_missing: bool = False):
    """Load libcosgpu.so (raises if it is missing and build_if_missing is False)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        path = _build.LIB
        if not os.path.exists(path):
            if not build_if_missing:
                raise RuntimeError(f"{path} is missing: build it with paper_2501_00675_gb300._build.build()")
            _build.build()
        lib = ctypes.CDLL(path)
        vp, i32, i64, f64 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_double
        lib.cos_create_graph.argtypes = [i32, vp, vp, vp, i32, i32, ctypes.POINTER(vp)]
        lib.cos_set_samples.argtypes = [vp, i64, vp, i32, vp, f64, vp]
        lib.cos_evaluate.argtypes = [vp, i32, vp, vp, vp]
        lib.cos_get_result.argtypes = [vp, vp, vp]
        lib.cos_graph_info.argtypes = [vp, vp, i32]
        lib.cos_set_tuning.argtypes = [vp, ctypes.POINTER(CosTuning)]
        lib.cos_get_tuning.argtypes = [vp, i32, ctypes.POINTER(CosTuning)]
        lib.cos_set_trace.argtypes = [vp, i32]
        lib.cos_get_trace.argtypes = [vp, vp, i32, ctypes.POINTER(ctypes.c_int32)]
        lib.cos_evaluate_static.argtypes = [vp, i32, i64, vp, i64, vp, f64, vp, vp, vp]
        lib.cos_graph_share.argtypes = [vp, ctypes.POINTER(vp)]
        lib.cos_set_propagator_table.argtypes = [vp, i32, vp, f64]
        lib.cos_autotune.argtypes = [vp, i32, vp, vp, ctypes.POINTER(CosTuning)]
        lib.cos_evaluate_abs.argtypes = [vp, i32, vp, vp, vp]
        lib.cos_mc_create.argtypes = [vp, i32, ctypes.c_uint64, vp, ctypes.POINTER(vp)]
        lib.cos_mc_run.argtypes = [vp, i32, vp]
        lib.cos_mc_stats.argtypes = [vp, vp, vp]
        lib.cos_mc_values.argtypes = [vp, vp, vp]
        lib.cos_mc_destroy.argtypes = [vp]
        lib.cos_batch_create.argtypes = [i32, vp, i32, vp, ctypes.POINTER(vp)]
        lib.cos_batch_reset.argtypes = [vp, i32, vp, vp]
        lib.cos_batch_set_tuning.argtypes = [vp, ctypes.POINTER(CosTuning)]
        lib.cos_batch_get_tuning.argtypes = [vp, ctypes.POINTER(CosTuning)]
        lib.cos_batch_autotune.argtypes = [vp, vp, ctypes.POINTER(CosTuning)]
        lib.cos_batch_launch.argtypes = [vp, vp]
        lib.cos_batch_results.argtypes = [vp, vp, vp]
        lib.cos_batch_destroy.argtypes = [vp]
        lib.cos_evaluate_batch.argtypes = [i32, vp, vp, vp, vp, vp]
        lib.cos_selftest_exp.argtypes = [vp, i64, vp, vp, vp, vp]
        lib.cos_probe_fma_rate.argtypes = [i32, ctypes.POINTER(f64)]
        lib.cos_set_samples_uniform.argtypes = [vp, i64, ctypes.c_uint64, i64, vp, f64, vp]
        lib.cos_copy_times.argtypes = [vp, vp, vp]
        lib.cos_server_create.argtypes = [i32, i32, ctypes.POINTER(CosTuning), i32, i64, i32, ctypes.POINTER(vp)]
        lib.cos_server_submit.argtypes = [vp, vp, i64, ctypes.c_uint64, i64, vp, ctypes.POINTER(i64)]
        lib.cos_server_poll.argtypes = [vp, i64, ctypes.POINTER(f64)]
        lib.cos_server_wait.argtypes = [vp, i64, i32, ctypes.POINTER(f64)]
        lib.cos_server_stats.argtypes = [vp, ctypes.POINTER(CosServerInfo)]
        lib.cos_server_destroy.argtypes = [vp]
        lib.cos_destroy.argtypes = [vp]
        lib.cos_last_error.restype = ctypes.c_char_p
        lib.cos_last_error.argtypes = []
        for name in EXPORTED[:-1]:
            getattr(lib, name).restype = ctypes.c_int
        _lib = lib
        return lib


def _check(rc: int, allow=()) -> int:
    if rc != COS_OK and rc not in allow:
        msg = load_library().cos_last_error()
        raise CosError(rc, msg.decode() if msg else "")
    return rc


def _ptr(a) -> Optional[int]:
    """Address of a numpy array or torch tensor (None passes NULL)."""
    if a is None:
        return None
    if isinstance(a, np.ndarray):
        return a.ctypes.data
    return a.data_ptr()


def _stream_handle(stream) -> Optional[int]:
    if stream is None:
        return None
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


def evaluate_batch(graphs: Sequence["Graph"], modes: Sequence[int], outs=None, stream=None,
                   allow_overflow: bool = False) -> np.ndarray:
    """cos_evaluate_batch: one mode per graph (the graphs of each distinct mode form
    one persistent launch); returns means [n][2] (mean R, mean A or NaN)."""
    n = len(graphs)
    hs = (ctypes.c_void_p * max(n, 1))(*[g.handle for g in graphs])
    ms = (ctypes.c_int32 * max(n, 1))(*[int(m) for m in modes])
    optr = None
    if outs is not None:
        optr = (ctypes.c_void_p * max(n, 1))(*[_ptr(o) for o in outs])
    means = np.zeros(max(2 * n, 1))
    _check(load_library().cos_evaluate_batch(n, hs, ms, optr, _ptr(means), _stream_handle(stream)),
           allow=(COS_ERR_OVERFLOW,) if allow_overflow else ())
    return means[:2 * n].reshape(n, 2)


def probe_fma_rate(precision: int = 0) -> float:
    """Multiply-adds per second of the current device (0: double, 1: float)."""
    out = ctypes.c_double(0.0)
    _check(load_library().cos_probe_fma_rate(precision, ctypes.byref(out)))
    return out.value


class Graph:
    """Owning handle of one device-resident CoS graph (cos_create_graph / cos_destroy)."""

    def __init__(self, widths: Sequence[int], edge_counts: Sequence[int], edges: np.ndarray, num_kinds: int,
                 num_times: int):
        lib = load_library()
        self._w = np.ascontiguousarray(widths, dtype=np.int64)
        self._c = np.ascontiguousarray(edge_counts, dtype=np.int64)
        e = np.ascontiguousarray(edges, dtype=np.int32)
        h = ctypes.c_void_p()
        _check(lib.cos_create_graph(len(self._w), _ptr(self._w), _ptr(self._c), _ptr(e) if e.size else None,
                                    int(num_kinds), int(num_times), ctypes.byref(h)))
        self._h = h
        self.num_samples = 0

    @classmethod
    def from_workload_graph(cls, g) -> "Graph":
        return cls(g.widths, g.edge_counts, g.edges, g.num_kinds, g.num_times)

    def share(self) -> "Graph":
        """cos_graph_share: a second handle on this graph's device structure."""
        h = ctypes.c_void_p()
        _check(load_library().cos_graph_share(self._h, ctypes.byref(h)))
        obj = Graph.__new__(Graph)
        obj._h = h
        obj._w, obj._c = self._w, self._c
        obj.num_samples = 0
        return obj

    @property
    def handle(self) -> int:
        return self._h.value

    def info(self) -> dict:
        arr = np.zeros(10, dtype=np.int64)
        _check(load_library().cos_graph_info(self._h, _ptr(arr), 10))
        keys = ["L", "N", "E", "P", "W_max", "count", "count_overflow", "K", "D", "device"]
        return {k: int(v) for k, v in zip(keys, arr)}

    def set_samples(self, t, eps, beta: float, t_flags: int, num_samples: Optional[int] = None, stream=None):
        """t: torch tensor (device or host) or numpy array (host); layout per t_flags."""
        eps = np.ascontiguousarray(eps, dtype=np.float64)
        if num_samples is None:
            num_samples = int(t.shape[0] if (t_flags & COS_T_SAMPLE_MAJOR) else t.shape[1])
        self._eps = eps
        _check(load_library().cos_set_samples(self._h, int(num_samples), _ptr(t), int(t_flags), _ptr(eps),
                                              float(beta), _stream_handle(stream)))
        self.num_samples = int(num_samples)

    def set_samples_uniform(self, num_samples: int, seed: int, eps, beta: float, first_sample: int = 0, stream=None):
        """cos_set_samples_uniform: times drawn on the device by the counter-based generator."""
        eps = np.ascontiguousarray(eps, dtype=np.float64)
        self._eps = eps
        _check(load_library().cos_set_samples_uniform(self._h, int(num_samples), int(seed), int(first_sample),
                                                      _ptr(eps), float(beta), _stream_handle(stream)))
        self.num_samples = int(num_samples)

    def copy_times(self, dst, stream=None):
        """cos_copy_times into dst ([D][S] doubles, torch tensor or numpy array)."""
        _check(load_library().cos_copy_times(self._h, _ptr(dst), _stream_handle(stream)))

    def evaluate(self, mode: int, out=None, want_mean: bool = True, stream=None, allow_overflow: bool = False):
        """Run cos_evaluate; returns the mean (float) -- (mean R, mean A) when mode has
        COS_EVAL_ABS, whose out then holds 2*S values -- if want_mean, else None."""
        means = (ctypes.c_double * 2)()
        rc = load_library().cos_evaluate(self._h, int(mode), _ptr(out), ctypes.addressof(means) if want_mean else None,
                                         _stream_handle(stream))
        _check(rc, allow=(COS_ERR_OVERFLOW,) if allow_overflow else ())
        if not want_mean:
            return None
        return (means[0], means[1]) if int(mode) & COS_EVAL_ABS else means[0]

    def evaluate_abs(self, mode: int, out=None, want_mean: bool = True, stream=None):
        """cos_evaluate_abs: A(s) = sum of |path| values per sample; returns its mean."""
        mean = ctypes.c_double(0.0)
        _check(load_library().cos_evaluate_abs(self._h, int(mode), _ptr(out),
                                               ctypes.addressof(mean) if want_mean else None, _stream_handle(stream)))
        return mean.value if want_mean else None

    def get_result(self, stream=None, both: bool = False):
        """cos_get_result: the last evaluation's mean (both=True: (mean R, mean A), the
        second meaningful after an evaluation with COS_EVAL_ABS)."""
        means = (ctypes.c_double * 2)()
        _check(load_library().cos_get_result(self._h, ctypes.addressof(means), _stream_handle(stream)))
        return (means[0], means[1]) if both else means[0]

    def set_tuning(self, samples_per_lane=0, tile_samples=0, rows_per_warp=0, blocks_per_sm=0, timeout_ms=0,
                   layout=0, schedule=0, window_chunks=0, prefetch=0):
        t = CosTuning(samples_per_lane, tile_samples, rows_per_warp, blocks_per_sm, timeout_ms, layout, schedule,
                      window_chunks, prefetch)
        _check(load_library().cos_set_tuning(self._h, ctypes.byref(t)))

    def set_propagator_table(self, tables, tau_max: float = 0.0):
        """tables: [K, 2, T+1] float64 (half 0: tau >= 0 on m*tau_max/T, half 1: tau < 0
        on -tau_max + m*tau_max/T); None returns to the free-fermion formula."""
        lib = load_library()
        if tables is None:
            _check(lib.cos_set_propagator_table(self._h, 0, None, ctypes.c_double(0.0)))
            return
        tab = np.ascontiguousarray(tables, dtype=np.float64)
        if tab.ndim != 3 or tab.shape[1] != 2 or tab.shape[2] < 2:
            raise ValueError("tables must be [K, 2, T+1] with T >= 1")
        _check(lib.cos_set_propagator_table(self._h, int(tab.shape[2] - 1),
                                            tab.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                            ctypes.c_double(float(tau_max))))

    def autotune(self, mode: int, out=None, stream=None) -> dict:
        """cos_autotune: time launch shapes on the attached samples, keep the fastest."""
        t = CosTuning()
        _check(load_library().cos_autotune(self._h, int(mode), _ptr(out), _stream_handle(stream), ctypes.byref(t)))
        return t.as_dict()

    def get_tuning(self, mode: int) -> dict:
        t = CosTuning()
        _check(load_library().cos_get_tuning(self._h, int(mode), ctypes.byref(t)))
        return t.as_dict()

    def set_trace(self, capacity: int):
        _check(load_library().cos_set_trace(self._h, int(capacity)))
        self._trace_cap = int(capacity)

    def get_trace(self):
        """[(phase id, ms since kernel start)] of the last evaluate (needs set_trace first)."""
        cap = getattr(self, "_trace_cap", 0)
        if cap <= 0:
            return []
        buf = np.zeros(2 * cap, dtype=np.int64)
        n = ctypes.c_int32(0)
        _check(load_library().cos_get_trace(self._h, _ptr(buf), cap, ctypes.byref(n)))
        rec = buf[:2 * n.value].reshape(-1, 2)
        if not len(rec):
            return []
        t0 = rec[0, 0]
        return [(int(ph), (int(t) - int(t0)) / 1e6) for t, ph in rec]

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            load_library().cos_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


class Batch:
    """Owning handle of one batched launch plan (cos_batch_create / cos_batch_destroy)."""

    def __init__(self, graphs: Sequence[Graph], mode: int, outs=None):
        lib = load_library()
        n = len(graphs)
        self._graphs = list(graphs)                       # keep the handles alive
        hs = (ctypes.c_void_p * max(n, 1))(*[g.handle for g in graphs])
        self._outs = list(outs) if outs is not None else None
        optr = None
        if outs is not None:
            arr = (ctypes.c_void_p * max(n, 1))(*[_ptr(o) for o in outs])
            self._optr = arr
            optr = arr
        h = ctypes.c_void_p()
        _check(lib.cos_batch_create(n, hs, int(mode), optr, ctypes.byref(h)))
        self._h = h
        self.n = n
        self.mode = int(mode)

    def reset(self, graphs: Sequence[Graph], outs=None):
        """cos_batch_reset: new members, same device buffers (previous launch must be collected)."""
        n = len(graphs)
        self._graphs = list(graphs)
        hs = (ctypes.c_void_p * max(n, 1))(*[g.handle for g in graphs])
        optr = None
        if outs is not None:
            optr = (ctypes.c_void_p * max(n, 1))(*[_ptr(o) for o in outs])
        self._optr = optr
        self._outs = list(outs) if outs is not None else None
        _check(load_library().cos_batch_reset(self._h, n, hs, optr))
        self.n = n

    def set_tuning(self, samples_per_lane=0, tile_samples=0, rows_per_warp=0, blocks_per_sm=0, timeout_ms=0,
                   layout=0, schedule=0, window_chunks=0, prefetch=0):
        t = CosTuning(samples_per_lane, tile_samples, rows_per_warp, blocks_per_sm, timeout_ms, layout, schedule,
                      window_chunks, prefetch)
        _check(load_library().cos_batch_set_tuning(self._h, ctypes.byref(t)))

    def get_tuning(self) -> dict:
        t = CosTuning()
        _check(load_library().cos_batch_get_tuning(self._h, ctypes.byref(t)))
        return t.as_dict()

    def autotune(self, stream=None) -> dict:
        t = CosTuning()
        _check(load_library().cos_batch_autotune(self._h, _stream_handle(stream), ctypes.byref(t)))
        return t.as_dict()

    def launch(self, stream=None):
        _check(load_library().cos_batch_launch(self._h, _stream_handle(stream)))

    def results(self, stream=None, allow_overflow: bool = False) -> np.ndarray:
        """Each graph's mean ([n]); [n][2] (mean R, mean A) for a COS_EVAL_ABS batch."""
        means = np.zeros(max(2 * self.n, 1))
        _check(load_library().cos_batch_results(self._h, _ptr(means), _stream_handle(stream)),
               allow=(COS_ERR_OVERFLOW,) if allow_overflow else ())
        if self.mode & COS_EVAL_ABS:
            return means[:2 * self.n].reshape(self.n, 2)
        return means[:self.n]

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            load_library().cos_batch_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Metropolis:
    """Metropolis walkers over a graph's attached times (cos_mc_*): every sample is
    a walker; the graph's time buffer is the walkers' state."""

    def __init__(self, graph: "Graph", mode: int, seed: int, stream=None):
        self.graph = graph
        h = ctypes.c_void_p()
        _check(load_library().cos_mc_create(graph._h, int(mode), ctypes.c_uint64(int(seed) & (2**64 - 1)),
                                            _stream_handle(stream), ctypes.byref(h)))
        self._h = h

    def run(self, num_steps: int, stream=None):
        _check(load_library().cos_mc_run(self._h, int(num_steps), _stream_handle(stream)))

    def stats(self, stream=None) -> dict:
        out = np.zeros(4, dtype=np.int64)
        _check(load_library().cos_mc_stats(self._h, _ptr(out), _stream_handle(stream)))
        steps, acc, pos, neg = (int(x) for x in out)
        return {"steps": steps, "accepted": acc, "n_pos": pos, "n_neg": neg}

    def values(self, out, stream=None):
        """Copy the walkers' current R into `out` (float64 tensor or array of S)."""
        _check(load_library().cos_mc_values(self._h, _ptr(out), _stream_handle(stream)))
        return out

    def close(self):
        if getattr(self, "_h", None):
            load_library().cos_mc_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class ResidentServer:
    """Resident server (cos_server_*): one persistent kernel that keeps running while
    requests arrive; each request evaluates a graph handle over counter-based uniform
    times drawn on the device.  See include/cos.h for the semantics."""

    def __init__(self, mode: int, max_times: int, max_requests: int = 256, queue_tasks: int = 65536,
                 idle_ms: int = 50, **tuning):
        t = CosTuning(**{k: int(v) for k, v in tuning.items()})
        h = ctypes.c_void_p()
        _check(load_library().cos_server_create(int(mode), int(max_times), ctypes.byref(t), int(max_requests),
                                                int(queue_tasks), int(idle_ms), ctypes.byref(h)))
        self._h = h
        self.mode = int(mode)

    def submit(self, graph: "Graph", num_samples: int, seed: int, out, first_sample: int = 0) -> Optional[int]:
        """Request id, or None when no slot or queue space is free (COS_ERR_BUSY)."""
        rid = ctypes.c_int64(0)
        rc = _check(load_library().cos_server_submit(self._h, graph._h, int(num_samples),
                                                     ctypes.c_uint64(int(seed) & (2**64 - 1)), int(first_sample),
                                                     _ptr(out), ctypes.byref(rid)), allow=(COS_ERR_BUSY,))
        return None if rc == COS_ERR_BUSY else int(rid.value)

    def poll(self, request_id: int, allow_overflow: bool = False):
        """The request's mean once complete (the request is then collected), else None."""
        m = ctypes.c_double(0.0)
        rc = _check(load_library().cos_server_poll(self._h, int(request_id), ctypes.byref(m)),
                    allow=(COS_ERR_BUSY, COS_ERR_OVERFLOW) if allow_overflow else (COS_ERR_BUSY,))
        return None if rc == COS_ERR_BUSY else m.value

    def wait(self, request_id: int, timeout_ms: int = -1, allow_overflow: bool = False) -> float:
        m = ctypes.c_double(0.0)
        _check(load_library().cos_server_wait(self._h, int(request_id), int(timeout_ms), ctypes.byref(m)),
               allow=(COS_ERR_OVERFLOW,) if allow_overflow else ())
        return m.value

    def stats(self) -> dict:
        info = CosServerInfo()
        _check(load_library().cos_server_stats(self._h, ctypes.byref(info)))
        return {f: int(getattr(info, f)) for f, _ in info._fields_}

    def close(self):
        if getattr(self, "_h", None):
            h, self._h = self._h, None
            _check(load_library().cos_server_destroy(h))

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

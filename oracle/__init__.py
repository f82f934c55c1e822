"""CPU oracle for CoS graph evaluation -- TEST INFRASTRUCTURE ONLY.

Only the tests, the smoke check and the benchmark's CPU-baseline leg may import
this package.  The GPU library never imports, links or runs it, and this
package never imports the GPU library.

Contents
  * ``cos_oracle.c`` (built here with gcc): the level-wise dynamic program of
    Sec. II.B / Fig. 1 in IEEE double, per-sample propagators, unit-weight path
    counts with 128-bit overflow detection, Neumaier summation; and the same DP in
    long double (``evaluate_tight``) as a tighter reference.
  * ``brute_force_paths`` / ``brute_force_sum``: pure-Python enumeration of all
    root-to-sink paths (one path = one diagram, Sec. II.B) for tiny graphs.
  * ``tabulated_propagator`` / ``evaluate_tabulated``: a user-tabulated G(tau) per
    kind (linear interpolation on a uniform grid, one table per sign of tau,
    evaluated in extended precision), the DP with those factors, and a bound on the
    effect of a double evaluation's grid-position rounding on R.
  * ``metropolis``: Metropolis walkers over the vertex times (weight |R|,
    single-time proposals from counter-based random numbers).

Parity status: every function here is pinned by the ``-m "not gpu"`` tests
(closed forms, brute force, library matrix products, propagator identities).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from typing import List, Optional, Sequence, Tuple

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "cos_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "libcos_oracle.so")
_lock = threading.Lock()
_lib = None

_i64p = ctypes.POINTER(ctypes.c_int64)
_i32p = ctypes.POINTER(ctypes.c_int32)
_f64p = ctypes.POINTER(ctypes.c_double)


def build(force: bool = False) -> str:
    """Compile cos_oracle.c into oracle/_build/libcos_oracle.so (gcc, OpenMP, no FP contraction)."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-std=gnu11", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off",
               "-fno-fast-math", _SRC, "-o", tmp, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_LIB_PATH)
            lib.cos_oracle_propagator.restype = ctypes.c_double
            lib.cos_oracle_propagator.argtypes = [ctypes.c_double, ctypes.c_double, ctypes.c_double]
            lib.cos_oracle_propagator_array.restype = None
            lib.cos_oracle_propagator_array.argtypes = [ctypes.c_double, ctypes.c_double, _f64p, _f64p,
                                                        ctypes.c_int64]
            lib.cos_oracle_pathsum.restype = ctypes.c_int
            lib.cos_oracle_pathsum.argtypes = [ctypes.c_int32, _i64p, _i64p, _i32p, _f64p, _f64p]
            lib.cos_oracle_eval.restype = ctypes.c_int
            lib.cos_oracle_eval.argtypes = [ctypes.c_int32, _i64p, _i64p, _i32p, ctypes.c_int32, ctypes.c_int32,
                                            _f64p, ctypes.c_double, ctypes.c_int64, _f64p, _f64p, _f64p,
                                            ctypes.c_int32]
            lib.cos_oracle_eval_ld.restype = ctypes.c_int
            lib.cos_oracle_eval_ld.argtypes = [ctypes.c_int32, _i64p, _i64p, _i32p, ctypes.c_int32, ctypes.c_int32,
                                               _f64p, ctypes.c_double, ctypes.c_int64, _f64p, _f64p, ctypes.c_int32]
            lib.cos_oracle_count.restype = ctypes.c_int
            lib.cos_oracle_count.argtypes = [ctypes.c_int32, _i64p, _i64p, _i32p, _i64p, _i32p]
            lib.cos_oracle_neumaier_sum.restype = ctypes.c_double
            lib.cos_oracle_neumaier_sum.argtypes = [_f64p, ctypes.c_int64]
            _lib = lib
    return _lib


def _p(a: np.ndarray, t):
    return a.ctypes.data_as(t)


def _graph_arrays(graph):
    w = np.ascontiguousarray(graph.widths, dtype=np.int64)
    c = np.ascontiguousarray(graph.edge_counts, dtype=np.int64)
    e = np.ascontiguousarray(graph.edges, dtype=np.int32)
    return w, c, e


def propagator(eps: float, beta: float, tau) -> np.ndarray:
    """G(tau) for one kind, elementwise over tau (free-fermion propagator, tau = t_i - t_j)."""
    lib = _load()
    tau = np.ascontiguousarray(np.atleast_1d(np.asarray(tau, dtype=np.float64)))
    out = np.empty_like(tau)
    lib.cos_oracle_propagator_array(float(eps), float(beta), _p(tau, _f64p), _p(out, _f64p), tau.size)
    return out


SIGN_BIT = 1 << 30          # kind bit 30: the edge closes a fermion loop (factor times -1)
KIND_MASK = SIGN_BIT - 1


def edge_weights(graph, eps: np.ndarray, beta: float, t_sample: np.ndarray) -> np.ndarray:
    """Per-edge factors w_e = +-G_{k_e}(t_{i_e} - t_{j_e}) for one sample (t_sample[D]);
    the sign is - for edges whose kind has bit 30 set (Sec. II.C, fermion loops)."""
    e = graph.edges
    tau = t_sample[e[:, 3]] - t_sample[e[:, 4]]
    kind = e[:, 2] & KIND_MASK
    out = np.empty(e.shape[0])
    for k in np.unique(kind):
        m = kind == k
        out[m] = propagator(eps[k], beta, tau[m])
    out[(e[:, 2] & SIGN_BIT) != 0] *= -1.0
    return out


def tabulated_propagator(table: np.ndarray, tau_max: float, tau) -> np.ndarray:
    """A user-tabulated propagator G(tau) for one kind (the general G of the Fig. 1
    caption, given as numbers), elementwise over tau: table[0] holds the values at
    tau_m = m*h, m = 0..T, h = tau_max/T, used for tau >= 0 (the tau = 0 branch of
    the free propagator, decided by t_i >= t_j); table[1] holds the values at
    tau_m = -tau_max + m*h, used for tau < 0.  Between nodes the value is the
    linear interpolation of its two neighbours; outside [-tau_max, tau_max] the end
    value.  Two halves keep the jump at tau = 0 (G(0+) - G(0-) = -1 for fermions).

    The definition is evaluated in extended precision (numpy longdouble: 64-bit
    significand on x86-64, 113-bit on AArch64) and rounded once to double: grid
    coordinate x = tau*T/tau_max (plus T below zero), m = floor(x), f = x - m,
    G = a_m + f*(a_{m+1} - a_m)."""
    table = np.asarray(table, dtype=np.float64)
    if table.ndim != 2 or table.shape[0] != 2 or table.shape[1] < 2:
        raise ValueError("table must be [2, T+1] with T >= 1")
    T = table.shape[1] - 1
    tau = np.atleast_1d(np.asarray(tau, dtype=np.float64))
    ld = np.longdouble
    pos = tau >= 0.0
    x = tau.astype(ld) * ld(T) / ld(tau_max)
    x = np.where(pos, x, x + ld(T))
    m, f = _grid_interval(x, T)
    half = np.where(pos[:, None], table[0][None, :], table[1][None, :])
    rows = np.arange(tau.size)
    a = half[rows, m].astype(ld)
    b = half[rows, m + 1].astype(ld)
    return (a + f * (b - a)).astype(np.float64)


def _grid_interval(x: np.ndarray, T: int):
    """Interval index m in [0, T-1] and position f in [0, 1] of grid coordinates x
    (before the grid: m = 0, f = 0; at or past its end: m = T-1, f = 1)."""
    below = x < 0
    past = x >= T
    m = np.floor(np.where(below | past, 0, x)).astype(np.int64)
    f = x - m
    m = np.where(past, T - 1, m)
    f = np.where(below, 0, np.where(past, 1, f))
    return np.minimum(m, T - 1), f


UNIT_ROUNDOFF = 2.0 ** -53


def tabulated_rounding_scale(table: np.ndarray, tau_max: float, tau) -> np.ndarray:
    """Bound on the error of any double-precision evaluation of ``tabulated_propagator``
    that forms the grid coordinate x = tau*T/tau_max (+T) with a few roundings: x is
    then off by at most 4u(|x| + T) grid units (u = 2^-53), which moves G by at most
    that times the largest |a_{m+1} - a_m| of the half (the interpolant is continuous,
    so landing in a neighbouring interval changes nothing beyond the slope), and the
    multiply-add of the interpolation rounds at most 4u(|a_m| + |a_{m+1}|).  Near a
    zero of G this absolute error can exceed any bound relative to |G| itself."""
    table = np.asarray(table, dtype=np.float64)
    T = table.shape[1] - 1
    tau = np.atleast_1d(np.asarray(tau, dtype=np.float64))
    pos = tau >= 0.0
    x = tau * (T / tau_max)
    x = np.where(pos, x, x + T)
    m, _ = _grid_interval(x, T)
    smax = np.max(np.abs(np.diff(table, axis=1)), axis=1)          # per half
    half = np.where(pos[:, None], table[0][None, :], table[1][None, :])
    rows = np.arange(tau.size)
    am, am1 = np.abs(half[rows, m]), np.abs(half[rows, m + 1])
    return UNIT_ROUNDOFF * (4.0 * (np.abs(x) + T) * np.where(pos, smax[0], smax[1]) + 4.0 * (am + am1))


def tabulated_edge_weights(graph, tables: np.ndarray, tau_max: float, t_sample: np.ndarray,
                           scale: bool = False):
    """Per-edge factors +-G_{k_e}(t_{i_e} - t_{j_e}) from tables[K, 2, T+1] for one sample;
    with scale=True also the per-edge rounding scale (``tabulated_rounding_scale``)."""
    e = graph.edges
    tau = t_sample[e[:, 3]] - t_sample[e[:, 4]]
    kind = e[:, 2] & KIND_MASK
    out = np.empty(e.shape[0])
    sc = np.empty(e.shape[0]) if scale else None
    for k in np.unique(kind):
        m = kind == k
        out[m] = tabulated_propagator(tables[k], tau_max, tau[m])
        if scale:
            sc[m] = tabulated_rounding_scale(tables[k], tau_max, tau[m])
    out[(e[:, 2] & SIGN_BIT) != 0] *= -1.0
    return (out, sc) if scale else out


def evaluate_tabulated(graph, tables: np.ndarray, tau_max: float, t: np.ndarray, with_bound: bool = False):
    """Per-sample sink values R[s] and A[s] = sum of |path| values with tabulated
    propagators: the level-wise DP (``pathsum``) once per sample with that sample's
    edge factors.  With with_bound=True also B[s], the first-order effect on R of the
    per-edge rounding scales eps_e of a double evaluation of the tables:
    B = sum_e eps_e * F(src_e) * Bk(dst_e), where F(v) is the sum over root-to-v
    paths and Bk(v) the sum over v-to-sink paths of the products of |factor|."""
    tables = np.asarray(tables, dtype=np.float64)
    if tables.ndim != 3 or tables.shape[0] < graph.num_kinds or tables.shape[1] != 2:
        raise ValueError("tables must be [K, 2, T+1]")
    S = t.shape[0]
    R = np.empty(S)
    A = np.empty(S)
    B = np.empty(S) if with_bound else None
    for s in range(S):
        if with_bound:
            w, sc = tabulated_edge_weights(graph, tables, tau_max, t[s], scale=True)
        else:
            w = tabulated_edge_weights(graph, tables, tau_max, t[s])
        R[s] = pathsum(graph, w)[-1]
        F = pathsum(graph, np.abs(w))
        A[s] = F[-1]
        if with_bound:
            Bk = _paths_to_sink(graph, np.abs(w))
            e = graph.edges
            B[s] = float(np.sum(sc * F[e[:, 0]] * Bk[e[:, 1]]))
    return (R, A, B) if with_bound else (R, A)


def _paths_to_sink(graph, w: np.ndarray) -> np.ndarray:
    """For every node v, the sum over v-to-sink paths of the products of w (the DP of
    Fig. 1 run from the last level back to the first)."""
    e = graph.edges
    N = graph.num_nodes
    out = np.zeros(N)
    out[N - 1] = 1.0
    hi = e.shape[0]
    for l in range(graph.num_levels - 1, 0, -1):
        lo = hi - int(graph.edge_counts[l])
        src, dst = e[lo:hi, 0], e[lo:hi, 1]
        out += np.bincount(src, weights=w[lo:hi] * out[dst], minlength=N)
        hi = lo
    return out


def pathsum(graph, w: np.ndarray) -> np.ndarray:
    """All node values of the level-wise DP with sample-independent edge weights w[E]."""
    lib = _load()
    wd, c, e = _graph_arrays(graph)
    w = np.ascontiguousarray(w, dtype=np.float64)
    out = np.empty(int(wd.sum()))
    rc = lib.cos_oracle_pathsum(len(wd), _p(wd, _i64p), _p(c, _i64p), _p(e, _i32p), _p(w, _f64p), _p(out, _f64p))
    if rc:
        raise ValueError("invalid graph")
    return out


def evaluate(graph, eps: np.ndarray, beta: float, t: np.ndarray, with_abs: bool = True,
             nthreads: int = 0) -> Tuple[np.ndarray, Optional[np.ndarray]]:
    """Per-sample sink values R[s] (and A[s] = sum of |path| values) in double precision."""
    lib = _load()
    wd, c, e = _graph_arrays(graph)
    eps = np.ascontiguousarray(eps, dtype=np.float64)
    t = np.ascontiguousarray(t, dtype=np.float64)
    S, D = t.shape
    if D != graph.num_times:
        raise ValueError("t must be [S, D]")
    R = np.empty(S)
    A = np.empty(S) if with_abs else None
    rc = lib.cos_oracle_eval(len(wd), _p(wd, _i64p), _p(c, _i64p), _p(e, _i32p), graph.num_kinds, D,
                             _p(eps, _f64p), float(beta), S, _p(t, _f64p), _p(R, _f64p),
                             _p(A, _f64p) if A is not None else None, int(nthreads))
    if rc:
        raise ValueError(f"oracle evaluation failed ({rc})")
    return R, A


def evaluate_tight(graph, eps: np.ndarray, beta: float, t: np.ndarray, nthreads: int = 0) -> np.ndarray:
    """Per-sample sink values computed in long double (expl), rounded once to double:
    a tighter reference than ``evaluate`` for measuring double-precision results."""
    lib = _load()
    wd, c, e = _graph_arrays(graph)
    eps = np.ascontiguousarray(eps, dtype=np.float64)
    t = np.ascontiguousarray(t, dtype=np.float64)
    S, D = t.shape
    R = np.empty(S)
    rc = lib.cos_oracle_eval_ld(len(wd), _p(wd, _i64p), _p(c, _i64p), _p(e, _i32p), graph.num_kinds, D,
                                _p(eps, _f64p), float(beta), S, _p(t, _f64p), _p(R, _f64p), int(nthreads))
    if rc:
        raise ValueError(f"oracle evaluation failed ({rc})")
    return R


def count_paths(graph) -> Tuple[int, bool]:
    """(path count modulo 2^64 as a signed int64, overflow flag for counts above 2^63-1)."""
    lib = _load()
    wd, c, e = _graph_arrays(graph)
    cnt = ctypes.c_int64(0)
    ovf = ctypes.c_int32(0)
    rc = lib.cos_oracle_count(len(wd), _p(wd, _i64p), _p(c, _i64p), _p(e, _i32p), ctypes.byref(cnt),
                              ctypes.byref(ovf))
    if rc:
        raise ValueError("invalid graph")
    return int(cnt.value), bool(ovf.value)


def neumaier_sum(x: np.ndarray) -> float:
    lib = _load()
    x = np.ascontiguousarray(x, dtype=np.float64)
    return float(lib.cos_oracle_neumaier_sum(_p(x, _f64p), x.size))


def neumaier_mean(x: np.ndarray) -> float:
    return neumaier_sum(x) / max(1, np.asarray(x).size)


def brute_force_paths(graph, limit: int = 200_000) -> List[List[int]]:
    """Every root-to-sink path as a list of edge indices (depth-first; tiny graphs only)."""
    e = graph.edges
    N = graph.num_nodes
    out_edges: List[List[int]] = [[] for _ in range(N)]
    for q in range(e.shape[0]):
        out_edges[int(e[q, 0])].append(q)
    paths: List[List[int]] = []
    stack: List[Tuple[int, List[int]]] = [(0, [])]
    while stack:
        node, path = stack.pop()
        if node == N - 1:
            paths.append(path)
            if len(paths) > limit:
                raise ValueError("too many paths for brute force")
            continue
        for q in out_edges[node]:
            stack.append((int(e[q, 1]), path + [q]))
    return paths


def brute_force_sum(paths: Sequence[Sequence[int]], w: np.ndarray) -> Tuple[float, float]:
    """(sum over paths of the product of w along the path, the same with |w|)."""
    r = 0.0
    a = 0.0
    for path in paths:
        prod = 1.0
        for q in path:
            prod *= float(w[q])
        r += prod
        a += abs(prod)
    return r, a

"""GPU parity: the CUDA path through the C ABI against the CPU oracle.

Tolerances (per sample s, relative to the oracle's sum of |path| values A(s)):
  FP64 mode       |R_gpu - R_oracle| <= 1e-12 * A
  FP32 mixed mode |R_gpu - R_oracle| <= 1e-5  * A
  count mode      bit-exact int64
The mean over samples is held to the same bound relative to mean(A).
"""
import math
import os
import time

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle  # noqa: E402
from workloads import (FaninSpec, chain_graph, complete_layered_graph, figure_graph, large, make_graph,  # noqa: E402
                       medium, tiny)

pytestmark = pytest.mark.gpu

TOL = {0: 1e-12, 1: 1e-5}


@pytest.fixture(scope="module")
def cg():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2501_00675_gb300 as cg
    from paper_2501_00675_gb300 import _build
    _build.build()
    cg.load_library()
    return cg


def run_gpu(cg, g, eps, beta, t, mode, tuning=None, layout="device_sd"):
    """Evaluate through the C ABI; returns (per-sample results as numpy, mean)."""
    gr = cg.Graph.from_workload_graph(g)
    if tuning:
        gr.set_tuning(**tuning)
    S = t.shape[0]
    if layout == "device_sd":
        tt = torch.from_numpy(np.ascontiguousarray(t)).cuda()
        flags = cg.COS_T_SAMPLE_MAJOR
    elif layout == "device_ds":
        tt = torch.from_numpy(np.ascontiguousarray(t.T)).cuda()
        flags = cg.COS_T_DEVICE_DS
    elif layout == "host_sd":
        tt = torch.from_numpy(np.ascontiguousarray(t)).pin_memory()
        flags = cg.COS_T_HOST | cg.COS_T_SAMPLE_MAJOR
    elif layout == "host_ds":
        tt = np.ascontiguousarray(t.T)
        flags = cg.COS_T_HOST
    else:
        raise ValueError(layout)
    gr.set_samples(tt, eps, beta, flags, num_samples=S)
    dt = torch.int64 if mode == cg.COS_MODE_COUNT_I64 else torch.float64
    out = torch.full((max(S, 1),), -7, dtype=dt, device="cuda")
    mean = gr.evaluate(mode, out=out[:S] if S else None, allow_overflow=True)
    torch.cuda.synchronize()
    res = out[:S].cpu().numpy()
    gr.close()
    return res, mean


def check_fp(R_gpu, mean_gpu, R, A, mode, idx=None, extra=None):
    """Per-sample |R_gpu - R| <= tol * A (+ extra, a per-sample bound on effects the
    relative tolerance does not cover, e.g. the tabulated propagators' grid position
    rounding), and the same for the mean."""
    tol = TOL[mode]
    if idx is not None:
        R_gpu = R_gpu[idx]
    err = np.abs(R_gpu - R)
    bound = tol * A if extra is None else tol * A + extra
    bad = err > bound
    assert not bad.any(), f"max err/A = {np.max(err / np.where(A > 0, A, 1)):.3e} at {np.nonzero(bad)[0][:5]}"
    if idx is None and R.size:
        slack = 0.0 if extra is None else float(np.mean(extra))
        assert abs(mean_gpu - oracle.neumaier_mean(R)) <= tol * float(np.mean(A)) + slack + 1e-300


# ------------------------------------------------------------------ tiny (full)

@pytest.mark.parametrize("mode", [0, 1])
def test_tiny_parity(cg, mode):
    w = tiny()
    R, A = oracle.evaluate(w.graph, w.samples.eps, w.samples.beta, w.samples.t)
    Rg, mg = run_gpu(cg, w.graph, w.samples.eps, w.samples.beta, w.samples.t, mode)
    check_fp(Rg, mg, R, A, mode)


def test_tiny_count_bit_exact(cg):
    w = tiny()
    cnt, ovf = oracle.count_paths(w.graph)
    Rg, mg = run_gpu(cg, w.graph, w.samples.eps, w.samples.beta, w.samples.t, 2)
    assert not ovf and np.all(Rg == cnt) and mg == float(cnt)


def test_figure_graph_count(cg):
    g = figure_graph()
    t = np.random.default_rng(0).uniform(0, 10, (70, 1))
    Rg, _ = run_gpu(cg, g, np.array([0.3]), 10.0, t, 2)
    assert np.all(Rg == 6)


# ------------------------------------------------------------------ medium

def test_medium_multi_tile_ragged_fp64(cg):
    w = medium(num_samples=5000)
    R, A = oracle.evaluate(w.graph, w.samples.eps, w.samples.beta, w.samples.t)
    for tuning in ({"tile_samples": 1024}, {"tile_samples": 640, "samples_per_lane": 1},
                   {"tile_samples": 1024, "layout": 2, "samples_per_lane": 2},
                   {"tile_samples": 768, "layout": 3, "samples_per_lane": 2}):
        Rg, mg = run_gpu(cg, w.graph, w.samples.eps, w.samples.beta, w.samples.t, 0, tuning)
        check_fp(Rg, mg, R, A, 0)


@pytest.fixture(scope="module")
def medium_full():
    """The medium workload at its full 65,536 samples and the oracle's R(s), A(s) for every one."""
    w = medium()
    R, A = oracle.evaluate(w.graph, w.samples.eps, w.samples.beta, w.samples.t)
    return w, R, A


@pytest.mark.parametrize("mode", [0, 1])
def test_medium_full_size(cg, medium_full, mode):
    """Every sample of the full medium workload, in the launch configuration the
    benchmark uses (automatic tuning), and the compensated mean over all of them
    against the oracle's Neumaier mean."""
    w, R, A = medium_full
    Rg, mg = run_gpu(cg, w.graph, w.samples.eps, w.samples.beta, w.samples.t, mode)
    assert Rg.size == w.samples.num_samples == 65536
    check_fp(Rg, mg, R, A, mode)
    assert math.isfinite(mg)


def test_medium_count_bit_exact(cg):
    w = medium(num_samples=777)
    cnt, ovf = oracle.count_paths(w.graph)
    Rg, _ = run_gpu(cg, w.graph, w.samples.eps, w.samples.beta, w.samples.t, 2)
    assert not ovf and np.all(Rg == cnt)


# ------------------------------------------------------------------ large (sampled)

LARGE_SLICE = 1 << 14


def test_large_mixed_first_slice(cg):
    """The large workload evaluated at its full 2^20 samples in the benchmark's launch
    configuration; the first 2^14 samples (a contiguous slice spanning more than one
    tile of samples, so more than one pass over the levels) are compared with the
    oracle one by one, and
    every sample is checked against the invariants |R| <= A <= C that hold at any
    size (C = path count)."""
    w = large()
    S = w.samples.num_samples
    t0 = time.time()
    R, A = oracle.evaluate(w.graph, w.samples.eps, w.samples.beta, w.samples.t[:LARGE_SLICE])
    print(f"oracle {LARGE_SLICE} samples: {time.time() - t0:.1f}s")
    Rg, mg = run_gpu(cg, w.graph, w.samples.eps, w.samples.beta, w.samples.t, 1)
    assert Rg.size == S
    check_fp(Rg, mg, R, A, 1, idx=np.arange(LARGE_SLICE))
    cnt, ovf = oracle.count_paths(w.graph)
    assert not ovf and np.all(np.abs(R) <= A) and np.all(A <= cnt)
    assert np.all(np.isfinite(Rg)) and np.all(np.abs(Rg) <= cnt) and math.isfinite(mg)


# ------------------------------------------------------------------ edge cases

@pytest.mark.parametrize("S", [1, 2, 31, 33, 129, 4097])
def test_ragged_sample_counts(cg, S):
    w = tiny(num_samples=S)
    R, A = oracle.evaluate(w.graph, w.samples.eps, w.samples.beta, w.samples.t)
    for mode in (0, 1):
        for tuning in (None, {"schedule": 2, "window_chunks": 1, "tile_samples": 256}):
            Rg, mg = run_gpu(cg, w.graph, w.samples.eps, w.samples.beta, w.samples.t, mode, tuning)
            check_fp(Rg, mg, R, A, mode)


@pytest.mark.parametrize("schedule", [1, 2])
def test_zero_samples(cg, schedule):
    w = tiny(num_samples=0)
    Rg, mg = run_gpu(cg, w.graph, w.samples.eps, w.samples.beta, w.samples.t, 0, {"schedule": schedule})
    assert Rg.size == 0 and mg == 0.0


def test_windowed_schedule_multi_tile_and_count(cg):
    """Windows continue across tiles of samples (ragged last tile) and the sample
    reduction waits for every window; count mode is bit-exact."""
    w = medium(num_samples=5000)
    R, A = oracle.evaluate(w.graph, w.samples.eps, w.samples.beta, w.samples.t)
    for mode, tuning in ((0, {"tile_samples": 1024, "window_chunks": 3}),
                         (1, {"tile_samples": 2048, "window_chunks": 1}),
                         (0, {"tile_samples": 640, "samples_per_lane": 1, "window_chunks": 7})):
        tuning = dict(tuning, schedule=2)
        Rg, mg = run_gpu(cg, w.graph, w.samples.eps, w.samples.beta, w.samples.t, mode, tuning)
        check_fp(Rg, mg, R, A, mode)
        base = run_gpu(cg, w.graph, w.samples.eps, w.samples.beta, w.samples.t, mode, dict(tuning, schedule=1))
        np.testing.assert_array_equal(Rg, base[0])
        assert mg == base[1]
    cnt, _ = oracle.count_paths(w.graph)
    Rg, mg = run_gpu(cg, w.graph, w.samples.eps, w.samples.beta, w.samples.t, 2,
                     {"schedule": 2, "window_chunks": 2, "tile_samples": 1500})
    assert np.all(Rg == cnt) and mg == float(cnt)


def test_schedule_tuning_resolution(cg):
    w = tiny(num_samples=64)
    gr = cg.Graph.from_workload_graph(w.graph)
    gr.set_samples(torch.from_numpy(w.samples.t).cuda(), w.samples.eps, w.samples.beta, cg.COS_T_SAMPLE_MAJOR)
    t = gr.get_tuning(0)
    assert t["schedule"] in (1, 2) and t["window_chunks"] >= 1
    gr.set_tuning(schedule=2, window_chunks=4)
    t = gr.get_tuning(1)
    assert t["schedule"] == 2 and t["window_chunks"] == 4
    with pytest.raises(cg.CosError):
        gr.set_tuning(schedule=3)
    with pytest.raises(cg.CosError):
        gr.set_tuning(window_chunks=-1)
    gr.close()


def test_two_level_graph_and_chain(cg):
    g = chain_graph([0], [0], [1], 1, 2)          # L = 2: root -> sink
    t = np.random.default_rng(1).uniform(0, 10, (50, 2))
    eps = np.array([0.7])
    R, A = oracle.evaluate(g, eps, 10.0, t)
    for mode in (0, 1):
        Rg, mg = run_gpu(cg, g, eps, 10.0, t, mode)
        check_fp(Rg, mg, R, A, mode)
    g = chain_graph([0, 1, 1, 0, 1, 0, 1, 1, 0], [0, 1, 2, 2, 0, 1, 2, 0, 1], [1, 2, 0, 2, 1, 1, 0, 0, 2], 2, 3)
    t = np.random.default_rng(2).uniform(0, 10, (300, 3))
    eps = np.array([1.3, -1.7])
    R, A = oracle.evaluate(g, eps, 10.0, t)
    for mode in (0, 1):
        Rg, mg = run_gpu(cg, g, eps, 10.0, t, mode)
        check_fp(Rg, mg, R, A, mode)


def test_wide_fanin_duplicates_dead_and_orphan_nodes(cg):
    rng = np.random.default_rng(3)
    # complete levels give fan-in 40 (> one warp of in-edges); then add duplicates, an orphan node
    g = complete_layered_graph([1, 5, 40, 40, 7, 1], num_kinds=3, num_times=4, rng=rng)
    e = g.edges.tolist()
    off = g.offsets()
    counts = g.edge_counts.copy()
    lvl = np.repeat(np.arange(g.num_levels), counts)
    extra = [row for row, l in zip(e, lvl) if l == 3][:10]       # duplicate (src, dst) pairs into level 3
    e3_end = int(counts[:4].sum())
    e = e[:e3_end] + extra + e[e3_end:]
    counts[3] += len(extra)
    # orphan: drop every in-edge of the first node of level 4
    orphan = off[4]
    keep = [row for row in e if row[1] != orphan]
    counts[4] -= len(e) - len(keep)
    e = np.array(keep, dtype=np.int32)
    from workloads import Graph
    g2 = Graph(g.widths, counts, e, 3, 4)
    t = rng.uniform(0, 10, (200, 4))
    t[:, 2] = t[:, 3]                                               # tau == 0 for (2,3) and (3,2) pairs
    eps = rng.uniform(-2, 2, 3)
    R, A = oracle.evaluate(g2, eps, 10.0, t)
    for mode in (0, 1):
        Rg, mg = run_gpu(cg, g2, eps, 10.0, t, mode)
        check_fp(Rg, mg, R, A, mode)
    cnt, _ = oracle.count_paths(g2)
    Rg, _ = run_gpu(cg, g2, eps, 10.0, t, 2)
    assert np.all(Rg == cnt)
    for mode in (0, 1, 2):                          # the bulk-copy ring on the same graph
        Rg, mg = run_gpu(cg, g2, eps, 10.0, t, mode, {"layout": 3})
        if mode == 2:
            assert np.all(Rg == cnt)
        else:
            check_fp(Rg, mg, R, A, mode)
    for mode in (0, 1, 2):                          # the work queue: FP64 items split their warps by edges
        for rpw in (31, 5):
            Rg, mg = run_gpu(cg, g2, eps, 10.0, t, mode, {"schedule": 2, "rows_per_warp": rpw})
            if mode == 2:
                assert np.all(Rg == cnt)
            else:
                check_fp(Rg, mg, R, A, mode)


def test_count_overflow_reports_and_wraps(cg):
    g = complete_layered_graph([1] + [256] * 8 + [1])
    cnt, ovf = oracle.count_paths(g)
    assert ovf
    gr = cg.Graph.from_workload_graph(g)
    assert gr.info()["count_overflow"] == 1 and gr.info()["count"] == cnt
    t = torch.zeros((64, 1), dtype=torch.float64, device="cuda")
    gr.set_samples(t, np.array([0.0]), 10.0, cg.COS_T_SAMPLE_MAJOR)
    out = torch.empty(64, dtype=torch.int64, device="cuda")
    with pytest.raises(cg.CosError) as ei:
        gr.evaluate(cg.COS_MODE_COUNT_I64, out=out)
    assert ei.value.code == cg.COS_ERR_OVERFLOW
    assert np.all(out.cpu().numpy() == cnt)
    gr.close()


# ------------------------------------------------------------------ invariances

def test_results_independent_of_launch_shape(cg):
    w = medium(num_samples=3000)
    ref = None
    for tuning in ({}, {"samples_per_lane": 1}, {"samples_per_lane": 4, "tile_samples": 512},
                   {"samples_per_lane": 2, "rows_per_warp": 4, "blocks_per_sm": 1},
                   {"samples_per_lane": 4, "layout": 2, "rows_per_warp": 28},
                   {"samples_per_lane": 2, "layout": 2, "rows_per_warp": 5, "tile_samples": 1000},
                   {"samples_per_lane": 4, "layout": 3, "rows_per_warp": 8},
                   {"samples_per_lane": 1, "layout": 3, "rows_per_warp": 3, "tile_samples": 700},
                   {"schedule": 2, "window_chunks": 1},
                   {"schedule": 2, "window_chunks": 3, "samples_per_lane": 2, "tile_samples": 1000},
                   {"schedule": 2, "window_chunks": 5, "samples_per_lane": 4, "layout": 2, "rows_per_warp": 6},
                   {"schedule": 2, "samples_per_lane": 4, "layout": 3, "window_chunks": 2},
                   {"prefetch": 3}, {"prefetch": 3, "schedule": 2, "samples_per_lane": 1}, {"prefetch": 1},
                   {"samples_per_lane": 4, "layout": 4, "rows_per_warp": 16},
                   {"samples_per_lane": 2, "layout": 4, "rows_per_warp": 7, "tile_samples": 900},
                   {"samples_per_lane": 1, "layout": 4, "rows_per_warp": 31},
                   {"schedule": 2, "samples_per_lane": 4, "layout": 4, "window_chunks": 3},
                   {"prefetch": 5}, {"prefetch": 4, "schedule": 2, "samples_per_lane": 2}):
        for mode in (0, 1):
            Rg, mg = run_gpu(cg, w.graph, w.samples.eps, w.samples.beta, w.samples.t, mode, tuning)
            if ref is None:
                ref = {}
            if mode in ref:
                np.testing.assert_array_equal(Rg, ref[mode][0])      # bitwise: same per-row order
                assert mg == ref[mode][1]
            else:
                ref[mode] = (Rg, mg)


@pytest.mark.parametrize("layout", ["device_ds", "host_sd", "host_ds"])
def test_sample_input_layouts(cg, layout):
    w = tiny(num_samples=300)
    a, ma = run_gpu(cg, w.graph, w.samples.eps, w.samples.beta, w.samples.t, 0, layout="device_sd")
    b, mb = run_gpu(cg, w.graph, w.samples.eps, w.samples.beta, w.samples.t, 0, layout=layout)
    np.testing.assert_array_equal(a, b)
    assert ma == mb


def test_repeat_and_reuse_handle(cg):
    w = tiny(num_samples=500)
    gr = cg.Graph.from_workload_graph(w.graph)
    t = torch.from_numpy(w.samples.t).cuda()
    gr.set_samples(t, w.samples.eps, w.samples.beta, cg.COS_T_SAMPLE_MAJOR)
    outs = []
    for _ in range(3):
        o = torch.empty(500, dtype=torch.float64, device="cuda")
        gr.evaluate(0, out=o)
        outs.append(o.cpu().numpy())
    np.testing.assert_array_equal(outs[0], outs[1])
    np.testing.assert_array_equal(outs[0], outs[2])
    # new samples on the same handle
    t2 = torch.from_numpy(w.samples.t[::-1].copy()).cuda()
    gr.set_samples(t2, w.samples.eps, w.samples.beta, cg.COS_T_SAMPLE_MAJOR)
    o = torch.empty(500, dtype=torch.float64, device="cuda")
    gr.evaluate(0, out=o)
    np.testing.assert_array_equal(o.cpu().numpy(), outs[0][::-1])
    gr.close()


def test_evaluate_before_samples_is_state_error(cg):
    gr = cg.Graph.from_workload_graph(tiny().graph)
    with pytest.raises(cg.CosError) as ei:
        gr.evaluate(0)
    assert ei.value.code == cg.COS_ERR_STATE
    gr.close()


@pytest.mark.parametrize("schedule", [1, 2])
def test_barrier_timeout_is_reported_and_context_survives(cg, monkeypatch, schedule):
    # Level-synchronous: one CTA leaves before the first level barrier and the
    # others' bounded waits run out.  Work queue: the plan gets a task that never
    # completes and the final item's bounded dependency wait runs out.  Either way
    # the launch ends with COS_ERR_TIMEOUT; no GPU fault is involved.
    w = tiny(num_samples=256)
    gr = cg.Graph.from_workload_graph(w.graph)
    gr.set_tuning(timeout_ms=200, schedule=schedule)
    t = torch.from_numpy(w.samples.t).cuda()
    gr.set_samples(t, w.samples.eps, w.samples.beta, cg.COS_T_SAMPLE_MAJOR)
    hook = "COS_TEST_SKIP_BARRIER_PHASE" if schedule == 1 else "COS_TEST_STALL_TASK"
    monkeypatch.setenv(hook, "4")   # schedule 1: the barrier after level 1
    t0 = time.time()
    with pytest.raises(cg.CosError) as ei:
        gr.evaluate(0)
    assert ei.value.code == cg.COS_ERR_TIMEOUT
    assert time.time() - t0 < 30
    monkeypatch.delenv(hook)
    R, A = oracle.evaluate(w.graph, w.samples.eps, w.samples.beta, w.samples.t)
    o = torch.empty(256, dtype=torch.float64, device="cuda")
    m = gr.evaluate(0, out=o)
    check_fp(o.cpu().numpy(), m, R, A, 0)
    gr.close()


def test_table_driven_exponentials_within_two_ulp(cg):
    # the propagator phase's e^{-x}, e^{+x} (Tang's table-driven method) against libm
    gr = cg.Graph.from_workload_graph(tiny().graph)
    rng = np.random.default_rng(7)
    x = np.concatenate([rng.uniform(-40, 40, 200000), rng.uniform(-600, 600, 20000),
                        np.array([0.0, 1e-300, -1e-300, 1e-9, np.log(2) / 128, -np.log(2) / 128, 20.0, -20.0])])
    xd = torch.from_numpy(x).cuda()
    em = torch.empty_like(xd)
    ep = torch.empty_like(xd)
    assert cg.load_library().cos_selftest_exp(gr.handle, x.size, xd.data_ptr(), em.data_ptr(), ep.data_ptr(), None) == 0
    torch.cuda.synchronize()
    for got, ref in ((em.cpu().numpy(), np.exp(-x)), (ep.cpu().numpy(), np.exp(x))):
        rel = np.abs(got - ref) / ref
        assert rel.max() <= 4.5e-16, rel.max()
    gr.close()


def test_mixed_mode_wide_energy_range_and_time_fallback(cg):
    # |eps| beta > 30 takes the double propagator path, |eps| beta <= 30 the float-float
    # path; times slightly beyond beta push a float-float item onto the double path.
    rng = np.random.default_rng(17)
    g = make_graph([1, 5, 9, 9, 6, 1], FaninSpec("uniform", 3), 6, 5, rng)
    eps = np.array([-7.5, -2.9, -0.3, 0.8, 2.95, 6.0])
    for hi in (10.0, 11.0):
        t = rng.uniform(0.0, hi, size=(700, 5))
        R, A = oracle.evaluate(g, eps, 10.0, t)
        Rg, mg = run_gpu(cg, g, eps, 10.0, t, 1)
        check_fp(Rg, mg, R, A, 1)
        Rg, mg = run_gpu(cg, g, eps, 10.0, t, 0)
        check_fp(Rg, mg, R, A, 0)


def test_fermion_loop_sign_flags(cg):
    # kind bit 30 negates an edge's factor (Sec. II.C); flagged and unflagged edges of the
    # same (kind, i, j) use distinct propagator slots
    from workloads import Graph
    w = medium(num_samples=900)
    g = w.graph
    e = g.edges.copy()
    e[np.random.default_rng(8).random(g.num_edges) < 0.3, 2] |= oracle.SIGN_BIT
    gs = Graph(g.widths, g.edge_counts, e, g.num_kinds, g.num_times)
    R, A = oracle.evaluate(gs, w.samples.eps, w.samples.beta, w.samples.t)
    for mode in (0, 1):
        Rg, mg = run_gpu(cg, gs, w.samples.eps, w.samples.beta, w.samples.t, mode)
        check_fp(Rg, mg, R, A, mode)
    R0, _ = oracle.evaluate(g, w.samples.eps, w.samples.beta, w.samples.t)
    assert not np.allclose(R, R0)                    # the flags matter
    cnt, _ = oracle.count_paths(gs)
    Rc, _ = run_gpu(cg, gs, w.samples.eps, w.samples.beta, w.samples.t, 2)
    assert np.all(Rc == cnt)                         # counting ignores signs
    gr = cg.Graph.from_workload_graph(gs)
    assert gr.info()["P"] > cg.Graph.from_workload_graph(g).info()["P"]
    gr.close()


@pytest.mark.parametrize("first", [0, (1 << 32) - 100])
def test_device_counter_times_match_and_evaluate(cg, first):
    # the device sampler and the host generator implement the same counter-based
    # draws independently: the times must agree bit for bit, the results within tolerance
    from workloads import counter_times
    w = tiny()
    S, D = 3000, w.graph.num_times
    t_host = counter_times(99, first, S, D, w.samples.beta)
    gr = cg.Graph.from_workload_graph(w.graph)
    gr.set_samples_uniform(S, 99, w.samples.eps, w.samples.beta, first_sample=first)
    tdev = torch.empty((D, S), dtype=torch.float64, device="cuda")
    gr.copy_times(tdev)
    torch.cuda.synchronize()
    np.testing.assert_array_equal(tdev.cpu().numpy().T, t_host)
    out = torch.empty(S, dtype=torch.float64, device="cuda")
    m = gr.evaluate(0, out=out)
    R, A = oracle.evaluate(w.graph, w.samples.eps, w.samples.beta, t_host)
    check_fp(out.cpu().numpy(), m, R, A, 0)
    gr.close()


# ------------------------------------------------------------------ tabulated propagators

def _tables(rng, K, T):
    # smooth random tables per kind and half, |G| <= 1 like a physical propagator
    xs = np.linspace(0.0, 1.0, T + 1)
    a, b, c = rng.uniform(-1, 1, (3, K, 2, 1))
    return 0.5 * np.tanh(a + b * xs + c * np.sin(7 * xs))


@pytest.mark.parametrize("mode", [0, 1])
def test_tabulated_propagator_parity(cg, mode):
    w = medium(num_samples=700)
    rng = np.random.default_rng(21)
    tables = _tables(rng, w.graph.num_kinds, 50)
    tau_max = 9.0      # part of tau in (-10, 10) falls outside: end values
    R, A, B = oracle.evaluate_tabulated(w.graph, tables, tau_max, w.samples.t, with_bound=True)
    for tuning in ({"schedule": 1}, {"schedule": 2, "rows_per_warp": 7}):
        gr = cg.Graph.from_workload_graph(w.graph)
        gr.set_tuning(**tuning)
        gr.set_propagator_table(tables, tau_max)
        gr.set_samples(torch.from_numpy(w.samples.t).cuda(), w.samples.eps, w.samples.beta, cg.COS_T_SAMPLE_MAJOR)
        out = torch.empty(700, dtype=torch.float64, device="cuda")
        m = gr.evaluate(mode, out=out)
        check_fp(out.cpu().numpy(), m, R, A, mode, extra=B)
        gr.close()


def test_tabulated_propagator_signs_share_reset_and_errors(cg):
    rng = np.random.default_rng(22)
    g = complete_layered_graph([1, 3, 6, 6, 2, 1], num_kinds=3, num_times=4, rng=rng)
    e = g.edges.copy()
    e[rng.random(len(e)) < 0.4, 2] |= oracle.SIGN_BIT
    from workloads import Graph
    g = Graph(g.widths, g.edge_counts, e, 3, 4)
    t = rng.uniform(0, 10, (300, 4))
    t[:, 1] = t[:, 2]                                  # tau == 0 on (1,2) and (2,1) slots
    eps = rng.uniform(-2, 2, 3)
    tables = _tables(rng, 3, 13)
    R, A, B = oracle.evaluate_tabulated(g, tables, 10.0, t, with_bound=True)
    gr = cg.Graph.from_workload_graph(g)
    gr.set_samples(torch.from_numpy(t).cuda(), eps, 10.0, cg.COS_T_SAMPLE_MAJOR)
    analytic = torch.empty(300, dtype=torch.float64, device="cuda")
    gr.evaluate(0, out=analytic)
    gr.set_propagator_table(tables, 10.0)
    out = torch.empty_like(analytic)
    m = gr.evaluate(0, out=out)
    check_fp(out.cpu().numpy(), m, R, A, 0, extra=B)
    twin = gr.share()                                  # the tables travel with a shared handle
    twin.set_samples(torch.from_numpy(t).cuda(), eps, 10.0, cg.COS_T_SAMPLE_MAJOR)
    out2 = torch.empty_like(out)
    twin.evaluate(0, out=out2)
    np.testing.assert_array_equal(out2.cpu().numpy(), out.cpu().numpy())
    twin.close()
    for bad in ((np.full((3, 2, 5), np.nan), 10.0), (tables, 0.0), (tables, -1.0)):
        with pytest.raises(cg.CosError):
            gr.set_propagator_table(*bad)
    gr.set_propagator_table(None)                      # back to the formula
    gr.evaluate(0, out=out)
    np.testing.assert_array_equal(out.cpu().numpy(), analytic.cpu().numpy())
    gr.close()


def test_renumbered_wide_levels_match_the_oracle(cg):
    # levels after a parent level of >= 65536 nodes are renumbered at ingest by their
    # smallest parent; the renumbering must not show in any result
    rng = np.random.default_rng(33)
    g = make_graph([1, 200, 70000, 70000, 300, 1], FaninSpec("uniform", 3), 4, 5, rng)
    t = rng.uniform(0, 10, (96, 5))
    eps = rng.uniform(-2, 2, 4)
    R, A = oracle.evaluate(g, eps, 10.0, t)
    for mode in (0, 1):
        for tuning in ({"schedule": 1}, {"schedule": 2}):
            Rg, mg = run_gpu(cg, g, eps, 10.0, t, mode, tuning)
            check_fp(Rg, mg, R, A, mode)
    cnt, _ = oracle.count_paths(g)
    Rg, _ = run_gpu(cg, g, eps, 10.0, t, 2)
    assert np.all(Rg == cnt)


def test_single_graph_autotune_keeps_results(cg):
    w = medium(num_samples=3000)
    gr = cg.Graph.from_workload_graph(w.graph)
    gr.set_samples(torch.from_numpy(w.samples.t).cuda(), w.samples.eps, w.samples.beta, cg.COS_T_SAMPLE_MAJOR)
    for mode in (0, 1, 2):
        dt = torch.int64 if mode == 2 else torch.float64
        ref = torch.empty(3000, dtype=dt, device="cuda")
        m_ref = gr.evaluate(mode, out=ref, allow_overflow=True)
        scratch = torch.empty_like(ref)
        best = gr.autotune(mode, out=scratch)
        assert best["schedule"] in (1, 2) and 1 <= best["rows_per_warp"] <= 31 and best["samples_per_lane"] in (1, 2, 4)
        assert gr.get_tuning(mode)["rows_per_warp"] == best["rows_per_warp"]
        out = torch.empty_like(ref)
        m = gr.evaluate(mode, out=out, allow_overflow=True)
        np.testing.assert_array_equal(out.cpu().numpy(), ref.cpu().numpy())
        assert m == m_ref
        gr.set_tuning()                                # back to automatic for the next mode
    gr.set_tuning(rows_per_warp=5)                     # fixed fields stay fixed
    assert gr.autotune(1)["rows_per_warp"] == 5
    gr.close()


def test_sum_of_abs_paths_matches_the_oracle(cg):
    # cos_evaluate_abs: A(s) = sum over paths of |path value|, the accuracy scale of R(s)
    w = medium(num_samples=900)
    R, A = oracle.evaluate(w.graph, w.samples.eps, w.samples.beta, w.samples.t)
    gr = cg.Graph.from_workload_graph(w.graph)
    gr.set_samples(torch.from_numpy(w.samples.t).cuda(), w.samples.eps, w.samples.beta, cg.COS_T_SAMPLE_MAJOR)
    for mode in (0, 1):
        for schedule in (1, 2):
            gr.set_tuning(schedule=schedule)
            out = torch.empty(900, dtype=torch.float64, device="cuda")
            ma = gr.evaluate_abs(mode, out=out)
            a = out.cpu().numpy()
            assert np.all(np.abs(a - A) <= TOL[mode] * A)
            assert abs(ma - float(np.mean(A))) <= TOL[mode] * float(np.mean(A))
            r = torch.empty_like(out)
            gr.evaluate(mode, out=r)                      # the ordinary walk is unchanged afterwards
            assert np.all(np.abs(r.cpu().numpy()) <= a * (1 + 1e-6))
    rng = np.random.default_rng(41)                        # with tabulated propagators: |table|
    tables = 0.5 * np.tanh(rng.normal(size=(w.graph.num_kinds, 2, 9))) + 0.3
    Rt, At, Bt = oracle.evaluate_tabulated(w.graph, tables, 9.0, w.samples.t, with_bound=True)
    gr.set_propagator_table(tables, 9.0)
    out = torch.empty(900, dtype=torch.float64, device="cuda")
    gr.evaluate_abs(0, out=out)
    assert np.all(np.abs(out.cpu().numpy() - At) <= 1e-12 * At + Bt)
    with pytest.raises(cg.CosError):
        gr.evaluate_abs(2)
    gr.close()


@pytest.mark.parametrize("schedule", [1, 2])
def test_fp64_error_against_the_long_double_reference(cg, schedule):
    # the GPU's FP64 results measured against the oracle's long-double evaluation:
    # within the double DP's own rounding bound (as the double oracle is), far inside 1e-12
    w = medium(num_samples=300)
    Rt = oracle.evaluate_tight(w.graph, w.samples.eps, w.samples.beta, w.samples.t)
    _, A = oracle.evaluate(w.graph, w.samples.eps, w.samples.beta, w.samples.t)
    Rg, _ = run_gpu(cg, w.graph, w.samples.eps, w.samples.beta, w.samples.t, 0, {"schedule": schedule})
    rel = np.abs(Rg - Rt) / A
    print(f"FP64 GPU vs long double, schedule {schedule}: max {rel.max():.2e} median {np.median(rel):.2e}")
    assert rel.max() <= 4 * (w.graph.num_levels + 4) * 2.0 ** -53


# ------------------------------------------------------------------ R and A(s) in one walk

@pytest.mark.parametrize("schedule", [1, 2])
def test_fused_sum_of_abs_paths_in_the_same_walk(cg, schedule):
    """mode | COS_EVAL_ABS: one launch gives R(s) -- bitwise the walk without the flag --
    and A(s) = sum of |path| values (float products: a scale, held to 1e-5 * A), and
    both means, against the oracle's A (Sec. II.B: R is a signed sum over diagrams,
    A the same sum of magnitudes)."""
    w = medium(num_samples=3000)
    g, s = w.graph, w.samples
    R, A = oracle.evaluate(g, s.eps, s.beta, s.t)
    gr = cg.Graph.from_workload_graph(g)
    gr.set_tuning(schedule=schedule, tile_samples=1024)
    gr.set_samples(torch.from_numpy(s.t).cuda(), s.eps, s.beta, cg.COS_T_SAMPLE_MAJOR)
    for mode in (0, 1):
        both = torch.full((2 * 3000,), -1.0, dtype=torch.float64, device="cuda")
        mr, ma = gr.evaluate(mode | cg.COS_EVAL_ABS, out=both)
        plain = torch.empty(3000, dtype=torch.float64, device="cuda")
        mp = gr.evaluate(mode, out=plain)
        r, a = both[:3000].cpu().numpy(), both[3000:].cpu().numpy()
        np.testing.assert_array_equal(r, plain.cpu().numpy())
        assert mr == mp
        check_fp(r, mr, R, A, mode)
        assert np.all(np.abs(a - A) <= 1e-5 * A), np.max(np.abs(a - A) / A)
        assert abs(ma - float(np.mean(A))) <= 1e-5 * float(np.mean(A))
        assert np.all(np.abs(r) <= a * (1 + 1e-5))
        gr.evaluate(mode | cg.COS_EVAL_ABS, out=both, want_mean=False)    # collected later
        assert gr.get_result(both=True) == (mr, ma)
    with pytest.raises(cg.CosError):
        gr.evaluate(2 | cg.COS_EVAL_ABS)
    gr.close()


def test_evaluate_batch_with_a_mode_per_graph(cg):
    """cos_evaluate_batch: a mode per graph (FP64, mixed, count, mixed with A), one
    persistent launch per distinct mode; means[n][2] and per-sample outputs against
    the oracle."""
    wls = [tiny(num_samples=900), tiny(seed=3, num_samples=1500), medium(num_samples=700),
           tiny(seed=4, num_samples=1100), medium(seed=9, num_samples=500)]
    modes = [0, 1, 2, 1 | cg.COS_EVAL_ABS, 0]
    graphs, outs = [], []
    for w, m in zip(wls, modes):
        gr = cg.Graph.from_workload_graph(w.graph)
        gr.set_samples(torch.from_numpy(w.samples.t).cuda(), w.samples.eps, w.samples.beta, cg.COS_T_SAMPLE_MAJOR)
        graphs.append(gr)
        n = w.samples.num_samples * (2 if m & cg.COS_EVAL_ABS else 1)
        outs.append(torch.full((n,), -3, dtype=torch.int64 if m == 2 else torch.float64, device="cuda"))
    means = cg.evaluate_batch(graphs, modes, outs)
    assert means.shape == (5, 2)
    for w, m, o, mm in zip(wls, modes, outs, means):
        S = w.samples.num_samples
        r = o.cpu().numpy()
        if m == 2:
            cnt, _ = oracle.count_paths(w.graph)
            assert np.all(r == cnt) and mm[0] == float(cnt) and np.isnan(mm[1])
            continue
        R, A = oracle.evaluate(w.graph, w.samples.eps, w.samples.beta, w.samples.t)
        base = m & ~cg.COS_EVAL_ABS
        check_fp(r[:S], mm[0], R, A, base)
        if m & cg.COS_EVAL_ABS:
            assert np.all(np.abs(r[S:] - A) <= 1e-5 * A) and abs(mm[1] - A.mean()) <= 1e-5 * A.mean()
        else:
            assert np.isnan(mm[1])
    with pytest.raises(cg.CosError):
        cg.evaluate_batch(graphs[:1], [7])
    for gr in graphs:
        gr.close()


def test_fused_sum_of_abs_paths_with_tabulated_propagators(cg):
    """COS_EVAL_ABS with user-tabulated propagators and fermion-loop signs: R(s) bitwise
    the walk without the flag, A(s) (float products) within 1e-5 of the oracle's A plus
    the tables' grid-position rounding bound."""
    rng = np.random.default_rng(43)
    w = medium(num_samples=1500)
    g = w.graph
    from workloads import Graph
    e = g.edges.copy()
    e[rng.random(len(e)) < 0.3, 2] |= oracle.SIGN_BIT
    g = Graph(g.widths, g.edge_counts, e, g.num_kinds, g.num_times)
    tables = _tables(rng, g.num_kinds, 33)
    R, A, B = oracle.evaluate_tabulated(g, tables, 9.5, w.samples.t, with_bound=True)
    gr = cg.Graph.from_workload_graph(g)
    gr.set_propagator_table(tables, 9.5)
    gr.set_samples(torch.from_numpy(w.samples.t).cuda(), w.samples.eps, w.samples.beta, cg.COS_T_SAMPLE_MAJOR)
    for mode in (0, 1):
        both = torch.empty(3000, dtype=torch.float64, device="cuda")
        mr, ma = gr.evaluate(mode | cg.COS_EVAL_ABS, out=both)
        plain = torch.empty(1500, dtype=torch.float64, device="cuda")
        gr.evaluate(mode, out=plain)
        r, a = both[:1500].cpu().numpy(), both[1500:].cpu().numpy()
        np.testing.assert_array_equal(r, plain.cpu().numpy())
        check_fp(r, mr, R, A, mode, extra=B)
        assert np.all(np.abs(a - A) <= 1e-5 * A + B)
    gr.close()

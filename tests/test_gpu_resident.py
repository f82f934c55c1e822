"""Resident server (cos_server_*) through the C ABI: requests on several graphs and
handles, submitted while the persistent kernel runs, each evaluated over
counter-based times that the kernel draws itself.  Every request's per-sample values
must match the oracle on the same times (``workloads.generate.counter_times``, the
generator's own restatement), count mode bit-exact; the times the kernel drew must
equal the generator's bitwise; admission must not need a relaunch while the kernel
runs; the task queue must survive many wrap-arounds; idle exits must be followed by
a relaunch; a dependency wait that runs out must fail the server cleanly."""
import os
import time

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle  # noqa: E402
from workloads import medium, tiny  # noqa: E402
from workloads.generate import counter_times  # noqa: E402

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


def _handles(cg, wl, n, capacity, seed=5):
    g = cg.Graph.from_workload_graph(wl.graph)
    hs = [g] + [g.share() for _ in range(n - 1)]
    for h in hs:
        h.set_samples_uniform(capacity, seed, wl.samples.eps, wl.samples.beta)
    torch.cuda.synchronize()
    return hs


def _check(wl, mode, S, seed, first, out, mean, cnt=None):
    g, s = wl.graph, wl.samples
    if mode == 2:
        r = out.cpu().numpy()[:S]
        assert np.all(r == cnt)
        if S:
            assert mean == float(cnt)
        return
    t = counter_times(seed, first, S, g.num_times, s.beta)
    R, A = oracle.evaluate(g, s.eps, s.beta, t)
    r = out.cpu().numpy()[:S]
    assert np.all(np.abs(r - R) <= TOL[mode] * A)
    if S:
        assert abs(mean - R.mean()) <= TOL[mode] * A.mean() + 1e-300
    else:
        assert mean == 0.0


@pytest.mark.parametrize("mode", [0, 1, 2])
def test_requests_match_oracle(cg, mode):
    works = [tiny(num_samples=8), medium(num_samples=8)]
    D = max(w.graph.num_times for w in works)
    srv = cg.ResidentServer(mode, D, max_requests=16)
    hs = [_handles(cg, works[0], 3, 5000), _handles(cg, works[1], 2, 12000)]
    counts = [oracle.count_paths(w.graph)[0] for w in works]
    rng = np.random.default_rng(7 + mode)
    dt = torch.int64 if mode == 2 else torch.float64
    reqs = []
    for wi, hl in enumerate(hs):
        for q, h in enumerate(hl):
            cap = 5000 if wi == 0 else 12000
            S = 0 if (wi, q) == (0, 2) else int(rng.integers(1, cap))
            seed, first = int(rng.integers(1, 2 ** 40)), int(rng.integers(0, 2 ** 34))
            out = torch.full((max(S, 1),), -9, dtype=dt, device="cuda")
            torch.cuda.synchronize()   # the fill, on torch's stream, must not land after the server's writes
            rid = srv.submit(h, S, seed, out, first)
            assert rid is not None
            reqs.append((wi, h, S, seed, first, out, rid))
    for wi, h, S, seed, first, out, rid in reqs:
        m = srv.wait(rid, 120000, allow_overflow=(mode == 2))
        _check(works[wi], mode, S, seed, first, out, m, counts[wi])
        if mode != 2 and S:   # the times the kernel drew are the generator's, bit for bit
            T = torch.empty((works[wi].graph.num_times, S), dtype=torch.float64, device="cuda")
            h.copy_times(T)
            torch.cuda.synchronize()
            want = counter_times(seed, first, S, works[wi].graph.num_times, works[wi].samples.beta)
            np.testing.assert_array_equal(T.cpu().numpy().T, want)
    st = srv.stats()
    assert st["completed"] == len(reqs) and st["failed"] == 0 and st["in_flight"] == 0
    srv.close()
    for hl in hs:
        for h in hl:
            h.close()


def test_admission_while_running(cg):
    """A long request, then small ones submitted at once: one launch serves them all."""
    wl_big, wl_small = medium(num_samples=8), tiny(num_samples=8)
    D = max(wl_big.graph.num_times, wl_small.graph.num_times)
    srv = cg.ResidentServer(1, D, max_requests=16, idle_ms=3000)
    big = _handles(cg, wl_big, 1, 1 << 18)[0]
    small = _handles(cg, wl_small, 6, 3000)
    out_big = torch.empty(1 << 18, dtype=torch.float64, device="cuda")
    rid_big = srv.submit(big, 1 << 18, 11, out_big, 0)
    assert srv.stats()["running"] == 1
    reqs = []
    for q, h in enumerate(small):
        out = torch.empty(3000, dtype=torch.float64, device="cuda")
        reqs.append((srv.submit(h, 3000, 100 + q, out, 0), 100 + q, out))
    done_small = [srv.wait(rid, 120000) for rid, _, _ in reqs]
    m_big = srv.wait(rid_big, 120000)
    st = srv.stats()
    assert st["launches"] == 1, st
    for (rid, seed, out), m in zip(reqs, done_small):
        _check(wl_small, 1, 3000, seed, 0, out, m)
    R, A = oracle.evaluate(wl_big.graph, wl_big.samples.eps, wl_big.samples.beta,
                           counter_times(11, 0, 4096, wl_big.graph.num_times, wl_big.samples.beta))
    r = out_big[:4096].cpu().numpy()   # the first 4096 samples (the oracle's share of the check)
    assert np.all(np.abs(r - R) <= TOL[1] * A)
    assert np.isfinite(m_big)
    srv.close()
    for h in [big] + small:
        h.close()


def test_idle_exit_and_relaunch(cg):
    wl = tiny(num_samples=8)
    srv = cg.ResidentServer(0, wl.graph.num_times, idle_ms=5)
    h = _handles(cg, wl, 1, 2000)[0]
    for k in range(3):
        out = torch.empty(2000, dtype=torch.float64, device="cuda")
        rid = srv.submit(h, 2000, 40 + k, out, 7)
        m = srv.wait(rid, 60000)
        _check(wl, 0, 2000, 40 + k, 7, out, m)
        t0 = time.time()
        while srv.stats()["running"] and time.time() - t0 < 10:   # every CTA leaves after 5 ms idle
            time.sleep(0.01)
        assert srv.stats()["running"] == 0
    assert srv.stats()["launches"] == 3
    srv.close()
    h.close()


def test_queue_wraps_and_slots_recycle(cg):
    """A 64-entry task queue and 4 request slots carry 40 requests: the queue wraps
    many times (cumulative completion counters, claim tags) and submits that find no
    room report busy without changing anything."""
    wl = tiny(num_samples=8)
    srv = cg.ResidentServer(1, wl.graph.num_times, max_requests=4, queue_tasks=64, idle_ms=2000)
    hs = _handles(cg, wl, 6, 1500)
    pending, done, busy = [], 0, 0
    k = 0
    while done < 40:
        free = [h for h in hs if all(p[1] is not h for p in pending)]
        if k < 40 and free:
            out = torch.empty(1500, dtype=torch.float64, device="cuda")
            S = 1 + (k * 377) % 1500
            rid = srv.submit(free[0], S, 1000 + k, out, k)
            if rid is None:
                busy += 1
            else:
                pending.append((rid, free[0], S, 1000 + k, k, out))
                k += 1
                continue
        rid, h, S, seed, first, out = pending.pop(0)
        m = srv.wait(rid, 60000)
        _check(wl, 1, S, seed, first, out, m)
        done += 1
    st = srv.stats()
    assert busy > 0 and st["published_tasks"] > 4 * 64 and st["failed"] == 0
    srv.close()
    for h in hs:
        h.close()


def test_submit_errors(cg):
    wl, wl2 = tiny(num_samples=8), medium(num_samples=8)
    srv = cg.ResidentServer(0, wl.graph.num_times)
    g = cg.Graph.from_workload_graph(wl.graph)
    out = torch.empty(4096, dtype=torch.float64, device="cuda")
    with pytest.raises(cg.CosError) as ei:               # no samples attached yet
        srv.submit(g, 10, 1, out)
    assert ei.value.code == cg.COS_ERR_STATE
    g.set_samples_uniform(1000, 1, wl.samples.eps, wl.samples.beta)
    with pytest.raises(cg.CosError) as ei:               # more samples than the handle holds
        srv.submit(g, 5000, 1, out)
    assert ei.value.code == cg.COS_ERR_STATE
    with pytest.raises(cg.CosError) as ei:               # per-sample output is required
        srv.submit(g, 10, 1, None)
    assert ei.value.code == cg.COS_ERR_INVALID
    g2 = cg.Graph.from_workload_graph(wl2.graph)
    if wl2.graph.num_times > wl.graph.num_times:
        g2.set_samples_uniform(100, 1, wl2.samples.eps, wl2.samples.beta)
        with pytest.raises(cg.CosError) as ei:           # more time variables than the server was made for
            srv.submit(g2, 10, 1, out)
        assert ei.value.code == cg.COS_ERR_INVALID
    rid = srv.submit(g, 1000, 3, out)
    with pytest.raises(cg.CosError) as ei:               # the handle is busy
        srv.submit(g, 10, 1, out)
    assert ei.value.code == cg.COS_ERR_STATE
    m = srv.wait(rid, 60000)
    _check(wl, 0, 1000, 3, 0, out, m)
    with pytest.raises(cg.CosError) as ei:               # collected: the id is gone
        srv.poll(rid)
    assert ei.value.code == cg.COS_ERR_INVALID
    srv.close()
    g.close()
    g2.close()


def test_dependency_timeout_fails_server(cg):
    """A task that never completes (test hook): the final task's wait runs into the
    200 ms limit, the kernel reports it and leaves, the request fails with
    COS_ERR_TIMEOUT and the server refuses further work; the context stays usable."""
    wl = tiny(num_samples=8)
    srv = cg.ResidentServer(0, wl.graph.num_times, timeout_ms=200)
    h = _handles(cg, wl, 1, 500)[0]
    out = torch.empty(500, dtype=torch.float64, device="cuda")
    os.environ["COS_TEST_STALL_TASK"] = "1"
    try:
        rid = srv.submit(h, 500, 1, out)
    finally:
        del os.environ["COS_TEST_STALL_TASK"]
    with pytest.raises(cg.CosError) as ei:
        srv.wait(rid, 60000)
    assert ei.value.code == cg.COS_ERR_TIMEOUT
    assert srv.stats()["failed"] == cg.COS_ERR_TIMEOUT
    with pytest.raises(cg.CosError):
        srv.submit(h, 10, 1, out)
    srv.close()
    # the device still works
    x = torch.ones(4, device="cuda") * 2
    assert float(x.sum()) == 8.0
    h.close()


def test_resident_scheduler_poisson_stream(cg):
    """The serving loop on the resident server: a Poisson stream over a small pool,
    every request completed, its mean equal to the oracle's on the request's own
    counter-based times, and all of it served by one kernel launch."""
    from paper_2501_00675_gb300.serve import RequestSpec, ResidentScheduler, latency_summary, poisson_run
    from workloads import batched
    wls = batched(seed=11, num_graphs=5, max_nodes=2e4, max_samples=4096, min_samples=1024)
    pool = [(cg.Graph.from_workload_graph(w.graph), w.samples.eps) for w in wls]
    srv = ResidentScheduler(pool, mode=cg.COS_MODE_FP32_MIXED, budget_bytes=8 << 30, max_samples=6000,
                            workspace_bytes=128 << 20, idle_ms=5000)
    rng = np.random.default_rng(3)
    specs = [RequestSpec(int(rng.integers(0, len(pool))), int(rng.integers(1, 6000)), 1000 + i) for i in range(30)]
    reqs, wall = poisson_run(srv, specs, rate_per_s=400.0, duration_s=5.0)
    done = [r for r in reqs if r.status == "done"]
    assert len(done) == len(specs)
    for r in done:
        w = wls[r.spec.graph_id]
        t = counter_times(r.spec.seed, 0, r.spec.num_samples, w.graph.num_times, srv.beta)
        R, A = oracle.evaluate(w.graph, w.samples.eps, srv.beta, t)
        assert abs(r.mean - R.mean()) <= TOL[1] * A.mean()
    s = latency_summary(reqs)
    assert s["completed"] == len(specs) and s["p99_ms"] >= s["p50_ms"] > 0
    assert srv.srv.stats()["launches"] == 1
    srv.close()
    for g, _ in pool:
        g.close()


def test_stale_cursor_claims_stay_exact(cg, monkeypatch):
    """Test hook (COS_TEST_STALE_CLAIMS=8): about one claim in eight acts on a cursor
    value a whole queue behind a published task ahead of the cursor, as a CTA would
    that read the cursor that long ago; the slot then holds that task and its item
    is taken out of order, waiting for its dependencies.  Every request must still
    match the oracle (each item run exactly once, after its dependencies), and the
    out-of-order path must have been taken."""
    monkeypatch.setenv("COS_TEST_STALE_CLAIMS", "8")
    works = [tiny(num_samples=8), medium(num_samples=8)]
    D = max(w.graph.num_times for w in works)
    srv = cg.ResidentServer(1, D, max_requests=8, queue_tasks=256, idle_ms=2000)
    hs = [(0, h) for h in _handles(cg, works[0], 4, 3000)] + [(1, h) for h in _handles(cg, works[1], 3, 4096)]
    pending, done, k = [], 0, 0
    while done < 24:
        free = [(wi, h) for wi, h in hs if all(p[1] is not h for p in pending)]
        if k < 24 and free:
            wi, h = free[k % len(free)]
            S = 3000 if wi == 0 else 4096
            out = torch.empty(S, dtype=torch.float64, device="cuda")
            rid = srv.submit(h, S, 500 + k, out, 0)
            if rid is not None:
                pending.append((rid, h, wi, S, 500 + k, out))
                k += 1
                continue
        rid, h, wi, S, seed, out = pending.pop(0)
        m = srv.wait(rid, 120000)
        _check(works[wi], 1, S, seed, 0, out, m)
        done += 1
    st = srv.stats()
    assert st["stale_claims"] > 0 and st["failed"] == 0, st
    srv.close()
    for _, h in hs:
        h.close()

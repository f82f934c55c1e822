"""Serving loop on the GPU: requests stream in while others run, are admitted by
device memory, batched into persistent launches on several streams, and every
result equals the same request evaluated alone."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from workloads import batched  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def cg():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2501_00675_gb300 as cg
    from paper_2501_00675_gb300 import _build
    _build.build()
    cg.load_library()
    return cg


@pytest.fixture(scope="module")
def pool(cg):
    wls = batched(seed=11, num_graphs=5, max_nodes=2e4, max_samples=4096, min_samples=1024)
    out = [(cg.Graph.from_workload_graph(w.graph), w.samples.eps) for w in wls]
    yield out
    for g, _ in out:
        g.close()


def _alone(cg, server, req):
    from paper_2501_00675_gb300.serve import request_times
    gid = req.spec.graph_id
    g = server.graphs[gid].share()
    t = request_times(torch, req.spec, server.info[gid]["D"], server.beta)
    g.set_samples(t, server.eps[gid], server.beta, cg.COS_T_BORROW, num_samples=req.spec.num_samples)
    out = torch.empty(req.spec.num_samples, dtype=torch.float64, device="cuda")
    m = g.evaluate(server.mode, out=out)
    g.close()
    return out.cpu().numpy(), m


@pytest.mark.parametrize("single", [False, True])
def test_results_same_alone_and_in_the_mix(cg, pool, single):
    from paper_2501_00675_gb300.serve import RequestSpec, Server, latency_summary, poisson_run
    mode = cg.COS_MODE_FP64 if single else cg.COS_MODE_FP32_MIXED
    srv = Server(pool, mode=mode, budget_bytes=6 << 30, max_batch=8, streams=2, single=single,
                 workspace_bytes=256 << 20)
    rng = np.random.default_rng(3)
    specs = [RequestSpec(int(rng.integers(0, len(pool))), int(rng.integers(1, 6000)), 1000 + i) for i in range(30)]
    reqs, wall = poisson_run(srv, specs, rate_per_s=400.0, duration_s=5.0)
    done = [r for r in reqs if r.status == "done"]
    assert len(done) == len(specs)
    assert srv.ctrl.peak <= srv.ctrl.budget
    if not single:
        assert max(srv.ctrl.peak, 0) > min(r.need_bytes for r in reqs)   # several requests were in flight
    for r in done:
        ref, m = _alone(cg, srv, r)
        np.testing.assert_array_equal(r.result.cpu().numpy(), ref)
        assert r.mean == m
    s = latency_summary(reqs)
    assert s["completed"] == len(specs) and s["p99_ms"] >= s["p50_ms"] > 0
    srv.close()


def test_budget_limits_concurrency(cg, pool):
    from paper_2501_00675_gb300.serve import RequestSpec, Server
    srv = Server(pool, mode=cg.COS_MODE_FP32_MIXED, budget_bytes=1, max_batch=8, streams=2)
    r = srv.submit(RequestSpec(0, 100, 1))
    srv.step()
    assert r.status == "shed" and srv.ctrl.shed == 1
    srv.close()

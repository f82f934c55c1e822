"""Batched uneven launch: many graphs of different size and sample count in one
persistent, CUDA-graph-captured launch.  Every graph's per-sample results must
be bitwise identical to evaluating it alone with the same launch shape (the sum
order at each node and the sample reduction order do not depend on the mix), and
within the oracle tolerance."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle  # noqa: E402
from workloads import batched, complete_layered_graph, tiny  # noqa: E402

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


def _setup(cg, wls):
    graphs = []
    for w in wls:
        gr = cg.Graph.from_workload_graph(w.graph)
        gr.set_samples(torch.from_numpy(w.samples.t).cuda(), w.samples.eps, w.samples.beta, cg.COS_T_SAMPLE_MAJOR)
        graphs.append(gr)
    return graphs


def _outs(wls, mode):
    dt = torch.int64 if mode == 2 else torch.float64
    return [torch.full((w.samples.num_samples,), -5, dtype=dt, device="cuda") for w in wls]


@pytest.fixture(scope="module")
def mix():
    return batched(num_graphs=9, max_nodes=3e4, max_samples=20000, min_samples=700)


@pytest.mark.parametrize("mode,tuning", [
    (1, {}), (0, {}), (2, {}),
    (1, {"samples_per_lane": 4, "layout": 2, "rows_per_warp": 8}),
    (0, {"samples_per_lane": 1, "rows_per_warp": 4, "tile_samples": 2048}),
    (1, {"samples_per_lane": 4, "layout": 3, "rows_per_warp": 8}),
    (2, {"samples_per_lane": 2, "layout": 3}),
    (1, {"window_chunks": 2}),
    (0, {"window_chunks": 1, "tile_samples": 2048}),
    (2, {"window_chunks": 3, "samples_per_lane": 1}),
    (1, {"samples_per_lane": 4, "layout": 4, "rows_per_warp": 31}),
    (0, {"samples_per_lane": 2, "layout": 4, "window_chunks": 2}),
    (2, {"samples_per_lane": 2, "layout": 4}),
])
def test_batch_matches_single_graph_bitwise(cg, mix, mode, tuning):
    graphs = _setup(cg, mix)
    outs = _outs(mix, mode)
    b = cg.Batch(graphs, mode, outs)
    if tuning:
        b.set_tuning(**tuning)
    b.launch()
    means = b.results()
    used = b.get_tuning()
    for w, gr, o, m in zip(mix, graphs, outs, means):
        single = torch.empty_like(o)
        gr.set_tuning(samples_per_lane=used["samples_per_lane"], layout=used["layout"],
                      rows_per_warp=used["rows_per_warp"], tile_samples=tuning.get("tile_samples", 0))
        ms = gr.evaluate(mode, out=single)
        np.testing.assert_array_equal(o.cpu().numpy(), single.cpu().numpy())
        assert m == ms
    b.close()
    for gr in graphs:
        gr.close()


def test_batch_against_oracle_and_replay(cg, mix):
    graphs = _setup(cg, mix)
    outs = _outs(mix, 1)
    b = cg.Batch(graphs, 1, outs)
    b.launch()
    first = [o.cpu().numpy().copy() for o in outs]
    m1 = b.results()
    for o in outs:
        o.fill_(0)
    b.launch()                                   # replay of the captured CUDA graph
    m2 = b.results()
    np.testing.assert_array_equal(m1, m2)
    for w, o, f in zip(mix, outs, first):
        np.testing.assert_array_equal(o.cpu().numpy(), f)
        idx = np.unique(np.r_[0, w.samples.num_samples - 1, np.random.default_rng(1).integers(0, w.samples.num_samples, 24)])
        R, A = oracle.evaluate(w.graph, w.samples.eps, w.samples.beta, w.samples.t[idx])
        assert np.all(np.abs(f[idx] - R) <= TOL[1] * A)
    b.close()
    for gr in graphs:
        gr.close()


def test_batch_autotune_keeps_results(cg, mix):
    sub = mix[:4]
    graphs = _setup(cg, sub)
    outs = _outs(sub, 1)
    b = cg.Batch(graphs, 1, outs)
    best = b.autotune()
    assert best["samples_per_lane"] in (1, 2, 4) and best["layout"] in (1, 2, 3, 4) and 1 <= best["rows_per_warp"] <= 31
    b.launch()
    b.results()
    for w, gr, o in zip(sub, graphs, outs):
        R, A = oracle.evaluate(w.graph, w.samples.eps, w.samples.beta, w.samples.t[:64])
        assert np.all(np.abs(o.cpu().numpy()[:64] - R) <= TOL[1] * A)
    b.close()
    for gr in graphs:
        gr.close()


def test_batch_with_empty_sample_set_and_tiny_graphs(cg):
    wls = [tiny(num_samples=0), tiny(seed=5, num_samples=33), tiny(seed=6, num_samples=1)]
    graphs = _setup(cg, wls)
    outs = [None, torch.empty(33, dtype=torch.float64, device="cuda"), torch.empty(1, dtype=torch.float64, device="cuda")]
    b = cg.Batch(graphs, 0, outs)
    b.launch()
    means = b.results()
    assert means[0] == 0.0
    for w, o, m in zip(wls[1:], outs[1:], means[1:]):
        R, A = oracle.evaluate(w.graph, w.samples.eps, w.samples.beta, w.samples.t)
        assert np.all(np.abs(o.cpu().numpy() - R) <= TOL[0] * A)
        assert abs(m - oracle.neumaier_mean(R)) <= TOL[0] * A.mean()
    b.close()
    for gr in graphs:
        gr.close()


def test_batch_rejects_duplicates_and_reports_overflow(cg):
    w = tiny(num_samples=40)
    g1 = _setup(cg, [w])[0]
    with pytest.raises(cg.CosError) as ei:
        cg.Batch([g1, g1], 0)
    assert ei.value.code == cg.COS_ERR_INVALID
    big = cg.Graph.from_workload_graph(complete_layered_graph([1] + [256] * 8 + [1]))
    big.set_samples(torch.zeros((16, 1), dtype=torch.float64, device="cuda"), np.array([0.0]), 10.0,
                    cg.COS_T_SAMPLE_MAJOR)
    b = cg.Batch([g1, big], 2)
    b.launch()
    with pytest.raises(cg.CosError) as ei:
        b.results()
    assert ei.value.code == cg.COS_ERR_OVERFLOW
    b.close()
    g1.close()
    big.close()


def test_queue_plans_enqueued_behind_busy_stream(cg):
    """Work-queue evaluations whose plans differ only in the output pointer, enqueued
    one after another without a host wait behind ~0.1 s of other work on the stream:
    each launch must use its own plan, so every buffer receives the sink values
    (the host-side plan staging may not be overwritten before its copy has run)."""
    from workloads import medium
    w = medium(num_samples=1024)
    g, s = w.graph, w.samples
    R, A = oracle.evaluate(g, s.eps, s.beta, s.t)
    gr = cg.Graph.from_workload_graph(g)
    gr.set_samples(torch.from_numpy(s.t).cuda(), s.eps, s.beta, cg.COS_T_SAMPLE_MAJOR)
    gr.set_tuning(schedule=2)
    st = torch.cuda.current_stream()
    outs = [torch.full((s.num_samples,), -9.0, dtype=torch.float64, device="cuda") for _ in range(3)]
    torch.cuda._sleep(200_000_000)
    for o in outs[:2]:
        gr.evaluate(0, out=o, want_mean=False, stream=st)
    outs[0].fill_(-9.0)
    gr.evaluate(0, out=outs[0], want_mean=False, stream=st)     # back to the first plan
    gr.evaluate(0, out=outs[2], want_mean=False, stream=st)
    torch.cuda.synchronize()
    for o in outs:
        r = o.cpu().numpy()
        assert np.all(np.abs(r - R) <= 1e-12 * A)
    gr.close()


def test_batch_replans_when_a_member_reattaches_samples(cg):
    """A batch launched twice (the second launch captured into a CUDA graph) whose
    member then attaches a larger sample set (new time, workspace and partial-sum
    buffers): the next launch must plan again for the new buffers and sizes, not
    replay the captured graph on the freed ones."""
    wls = [tiny(num_samples=300), tiny(seed=7, num_samples=200)]
    graphs = _setup(cg, wls)
    outs = _outs(wls, 0)
    b = cg.Batch(graphs, 0, outs)
    for _ in range(3):                          # direct launch, capture, replay
        b.launch()
        b.results()
    bigger = tiny(seed=8, num_samples=70000)    # > the 4096 partial sums allocated at first attach
    graphs[0].set_samples(torch.from_numpy(bigger.samples.t).cuda(), bigger.samples.eps, bigger.samples.beta,
                          cg.COS_T_SAMPLE_MAJOR)
    out0 = torch.full((70000,), -5.0, dtype=torch.float64, device="cuda")
    b.reset(graphs, [out0, outs[1]])
    for _ in range(2):
        b.launch()
        means = b.results()
    # graph 0 keeps its own structure (wls[0].graph) and now holds bigger's 70,000 samples
    for g, smp, o, m in ((wls[0].graph, bigger.samples, out0, means[0]), (wls[1].graph, wls[1].samples, outs[1],
                                                                          means[1])):
        R, A = oracle.evaluate(g, smp.eps, smp.beta, smp.t)
        assert np.all(np.abs(o.cpu().numpy() - R) <= TOL[0] * A)
        assert abs(m - oracle.neumaier_mean(R)) <= TOL[0] * A.mean()
    # same members and outputs, samples re-attached in place: re-planned as well
    graphs[1].set_samples(torch.from_numpy(bigger.samples.t[:200].copy()).cuda(), bigger.samples.eps,
                          bigger.samples.beta, cg.COS_T_SAMPLE_MAJOR)
    b.launch()
    means = b.results()
    R, A = oracle.evaluate(wls[1].graph, bigger.samples.eps, bigger.samples.beta, bigger.samples.t[:200])
    assert np.all(np.abs(outs[1].cpu().numpy() - R) <= TOL[0] * A)
    b.close()
    for gr in graphs:
        gr.close()


def test_batched_workload_full_size_first_samples(cg):
    """The batched uneven workload at its full size (64 graphs, 2.6e7 edges, 1.4e7
    samples) in one work-queue launch, in the launch shape the benchmark times (4
    samples per lane, 31 rows per warp, wide layout, each graph's workspace capped at
    2 GB): every graph's first 32 samples are compared with the oracle one by one,
    and every sample and mean against |R| <= C (C = the graph's path count)."""
    import math
    wls = batched(seed=3, num_graphs=64)
    graphs, outs = [], []
    for w in wls:
        gr = cg.Graph.from_workload_graph(w.graph)
        inf = gr.info()
        psb = 2 * 8 * inf["W_max"] + 8 * inf["P"]
        gr.set_tuning(tile_samples=int(max(128, min(65536, (2 << 30) // psb // 128 * 128))))
        gr.set_samples(torch.from_numpy(w.samples.t).cuda(), w.samples.eps, w.samples.beta, cg.COS_T_SAMPLE_MAJOR)
        graphs.append(gr)
        outs.append(torch.full((w.samples.num_samples,), float("nan"), dtype=torch.float64, device="cuda"))
    b = cg.Batch(graphs, 1, outs)
    b.set_tuning(samples_per_lane=4, rows_per_warp=31, layout=1)
    b.launch()
    means = b.results()
    for w, o, m in zip(wls, outs, means):
        r = o.cpu().numpy()
        R, A = oracle.evaluate(w.graph, w.samples.eps, w.samples.beta, w.samples.t[:32])
        assert np.all(np.abs(r[:32] - R) <= TOL[1] * A)
        cnt, ovf = oracle.count_paths(w.graph)
        assert not ovf
        assert np.all(np.isfinite(r)) and np.all(np.abs(r) <= cnt)
        assert math.isfinite(m) and abs(m) <= cnt
    b.close()
    for gr in graphs:
        gr.close()

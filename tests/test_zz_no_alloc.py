"""cos_evaluate_static: the entry point for callers that must not allocate device
memory while they evaluate -- a host framework whose own allocator owns the
device budget, or a latency-bound serving loop where cudaMalloc/cudaFree could
synchronise the device.  It keeps its scratch in a fixed 64 MiB device array
inside the library; these tests check, through the C ABI, that two calls in a row
give the same results as the allocating cos_evaluate on the same samples, that
oversize graphs are rejected with an error instead of running, and that a bounded
wait that gives up inside the kernel is reported (by the call itself, or by the
next call that asks for the mean when the failing call did not).

This file is collected last on purpose, so a run that stops at the first
failure has already run every other test.
"""
import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle  # noqa: E402
from workloads import complete_layered_graph, medium, tiny  # noqa: E402

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


def _padded_times(t: np.ndarray):
    """Device [D][t_ld] copy of t[S][D], t_ld = S rounded up to 128, zero padding."""
    S, D = t.shape
    t_ld = max(128, (S + 127) // 128 * 128)
    buf = torch.zeros((D, t_ld), dtype=torch.float64, device="cuda")
    buf[:, :S] = torch.from_numpy(np.ascontiguousarray(t.T)).cuda()
    return buf, t_ld


def _static(cg, gr, mode, t, eps, beta, want_mean=True):
    lib = cg.load_library()
    S = t.shape[0]
    tdev, t_ld = _padded_times(t)
    eps_dev = torch.from_numpy(np.ascontiguousarray(eps, dtype=np.float64)).cuda()
    out = torch.full((max(S, 1),), -3, dtype=torch.int64 if mode == 2 else torch.float64, device="cuda")
    mean = ctypes.c_double(0.0)
    stream = torch.cuda.current_stream().cuda_stream
    rc = lib.cos_evaluate_static(gr.handle, mode, S, tdev.data_ptr(), t_ld, eps_dev.data_ptr(), float(beta),
                                 out.data_ptr(), ctypes.addressof(mean) if want_mean else None, stream)
    torch.cuda.synchronize()
    return rc, out[:S].cpu().numpy(), mean.value


def _allocating(cg, gr, mode, t, eps, beta):
    gr.set_samples(torch.from_numpy(np.ascontiguousarray(t)).cuda(), eps, beta, cg.COS_T_SAMPLE_MAJOR)
    out = torch.empty(t.shape[0], dtype=torch.int64 if mode == 2 else torch.float64, device="cuda")
    mean = gr.evaluate(mode, out=out)
    return out.cpu().numpy(), mean


@pytest.mark.parametrize("factory,S", [(tiny, 1000), (medium, 1500)])
def test_static_matches_allocating_entry_point_twice(cg, factory, S):
    wl = factory(num_samples=2 * S)
    g, s = wl.graph, wl.samples
    gr = cg.Graph.from_workload_graph(g)
    halves = [s.t[:S], s.t[S:][::-1].copy()]          # two different sample sets, one call each
    for mode in (0, 1, 2):
        for t in halves:
            rc, r_static, m_static = _static(cg, gr, mode, t, s.eps, s.beta)
            assert rc == cg.COS_OK, cg.load_library().cos_last_error()
            r_alloc, m_alloc = _allocating(cg, gr, mode, t, s.eps, s.beta)
            if mode == 2:
                np.testing.assert_array_equal(r_static, r_alloc)
                assert m_static == m_alloc
            else:
                _, A = oracle.evaluate(g, s.eps, s.beta, t)
                assert np.all(np.abs(r_static - r_alloc) <= TOL[mode] * A)
                assert abs(m_static - m_alloc) <= TOL[mode] * float(np.mean(A))
    gr.close()


def test_static_rejects_graphs_beyond_the_scratch_limit(cg):
    g = complete_layered_graph([1, 1 << 19, 1])     # 2 * 2^19 * 8 B per sample > 64 MiB / 32 samples
    gr = cg.Graph.from_workload_graph(g)
    t = np.zeros((64, 1))
    rc, _, _ = _static(cg, gr, 0, t, np.array([0.5]), 10.0)
    assert rc == cg.COS_ERR_INVALID
    assert b"static scratch" in cg.load_library().cos_last_error()
    gr.close()


def test_static_rejects_the_sum_of_abs_paths_flag(cg):
    # the entry evaluates R only; COS_EVAL_ABS (a second output) is refused before any launch
    wl = tiny(num_samples=64)
    gr = cg.Graph.from_workload_graph(wl.graph)
    rc, _, _ = _static(cg, gr, 0 | cg.COS_EVAL_ABS, wl.samples.t, wl.samples.eps, wl.samples.beta)
    assert rc == cg.COS_ERR_INVALID
    gr.close()


def test_static_uses_the_handles_propagator_tables(cg):
    # tables set on the handle (cos_set_propagator_table) apply to the static entry too
    wl = tiny(num_samples=600)
    g, s = wl.graph, wl.samples
    rng = np.random.default_rng(31)
    tables = 0.5 * np.tanh(rng.normal(size=(g.num_kinds, 2, 17)))
    R, A, B = oracle.evaluate_tabulated(g, tables, 9.0, s.t, with_bound=True)
    gr = cg.Graph.from_workload_graph(g)
    gr.set_propagator_table(tables, 9.0)
    for mode in (0, 1):
        rc, r_static, _ = _static(cg, gr, mode, s.t, s.eps, s.beta)
        assert rc == cg.COS_OK, cg.load_library().cos_last_error()
        assert np.all(np.abs(r_static - R) <= TOL[mode] * A + B)   # B: grid position rounding of the tables
    gr.close()


def test_static_reports_a_bounded_wait_that_gave_up(cg, monkeypatch):
    """One CTA leaves before the barrier after level 1 (test hook), so the other
    CTAs' waits run out after the handle's 200 ms limit -- no GPU fault.  A call that
    asks for the mean reports it at once; a call that does not leaves it recorded,
    and the next call that asks for the mean reports it.  After the report the next
    call is clean and matches the oracle."""
    wl = tiny(num_samples=512)
    g, s = wl.graph, wl.samples
    R, A = oracle.evaluate(g, s.eps, s.beta, s.t)
    gr = cg.Graph.from_workload_graph(g)
    gr.set_tuning(timeout_ms=200)
    lib = cg.load_library()
    monkeypatch.setenv("COS_TEST_SKIP_BARRIER_PHASE", "4")
    rc, _, _ = _static(cg, gr, 0, s.t, s.eps, s.beta)
    assert rc == cg.COS_ERR_TIMEOUT, lib.cos_last_error()
    rc, _, _ = _static(cg, gr, 0, s.t, s.eps, s.beta, want_mean=False)     # returns after the launch
    assert rc == cg.COS_OK
    monkeypatch.delenv("COS_TEST_SKIP_BARRIER_PHASE")
    rc, _, _ = _static(cg, gr, 0, s.t[:0], s.eps, s.beta)                  # zero samples: collects the status
    assert rc == cg.COS_ERR_TIMEOUT and b"since the last one" in lib.cos_last_error()
    for _ in range(2):
        rc, r, m = _static(cg, gr, 0, s.t, s.eps, s.beta)
        assert rc == cg.COS_OK, lib.cos_last_error()
        assert np.all(np.abs(r - R) <= TOL[0] * A)
        assert abs(m - oracle.neumaier_mean(R)) <= TOL[0] * float(np.mean(A))
    gr.close()

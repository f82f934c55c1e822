"""Seeded random cases through the C ABI: random leveled graphs (widths, fan-ins,
kinds, times, fermion-loop flags, sometimes tabulated propagators) evaluated under
random launch shapes (schedule, vector width, rows per warp, layout, windows,
prefetch, tile size).  Every result must match the oracle within the mode's
tolerance (count mode bit-exact), and every launch shape of one case must give the
same bits (the per-row sum order and the sample reduction order are fixed)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle  # noqa: E402
from workloads import FaninSpec, Graph, make_graph  # noqa: E402

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


def _case(seed):
    rng = np.random.default_rng(1000 + seed)
    L = int(rng.integers(3, 8))
    widths = [1] + [int(x) for x in rng.integers(1, 300, L - 2)] + [1]
    K, D = int(rng.integers(1, 6)), int(rng.integers(1, 9))
    g = make_graph(widths, FaninSpec("uniform", int(rng.integers(1, 6))), K, D, rng)
    e = g.edges.copy()
    e[rng.random(len(e)) < 0.2, 2] |= oracle.SIGN_BIT
    g = Graph(g.widths, g.edge_counts, e, K, D)
    S = int(rng.integers(1, 1500))
    t = rng.uniform(0, 10, (S, D))
    if D > 1 and rng.random() < 0.5:
        t[:, 1] = t[:, 0]                       # tau == 0 on every (0, 1) and (1, 0) slot
    eps = rng.uniform(-2, 2, K)
    tables = None
    if rng.random() < 0.3:
        T = int(rng.integers(2, 40))
        xs = np.linspace(0, 1, T + 1)
        a, b = rng.uniform(-1, 1, (2, K, 2, 1))
        tables = 0.5 * np.tanh(a + b * np.sin(5 * xs)) + 0.6   # away from zero: positions stay well-conditioned
    return rng, g, t, eps, tables


def _shape(rng):
    shape = {"schedule": int(rng.integers(1, 3)), "samples_per_lane": int(rng.choice([1, 2, 4])),
             "rows_per_warp": int(rng.integers(1, 32)), "layout": int(rng.choice([1, 1, 2, 3, 4])),
             "prefetch": int(rng.integers(1, 6))}
    if rng.random() < 0.5:
        shape["window_chunks"] = int(rng.integers(1, 6))
    if rng.random() < 0.5:
        shape["tile_samples"] = int(rng.integers(32, 700))
    return shape


@pytest.mark.parametrize("seed", range(12))
def test_random_graphs_and_launch_shapes(cg, seed):
    rng, g, t, eps, tables = _case(seed)
    S = t.shape[0]
    B = 0.0                  # tabulated propagators: bound on their grid position rounding
    if tables is None:
        R, A = oracle.evaluate(g, eps, 10.0, t)
    else:
        R, A, B = oracle.evaluate_tabulated(g, tables, 8.0, t, with_bound=True)
    cnt, _ = oracle.count_paths(g)
    gr = cg.Graph.from_workload_graph(g)
    if tables is not None:
        gr.set_propagator_table(tables, 8.0)
    gr.set_samples(torch.from_numpy(np.ascontiguousarray(t)).cuda(), eps, 10.0, cg.COS_T_SAMPLE_MAJOR)
    first = {}
    for _ in range(4):
        shape = _shape(rng)
        gr.set_tuning(**shape)
        for mode in (0, 1, 2):
            dt = torch.int64 if mode == 2 else torch.float64
            out = torch.full((S,), -9, dtype=dt, device="cuda")
            m = gr.evaluate(mode, out=out, allow_overflow=True)
            r = out.cpu().numpy()
            if mode == 2:
                assert np.all(r == cnt), shape
            else:
                bad = np.abs(r - R) > TOL[mode] * A + B
                assert not bad.any(), (shape, mode, np.nonzero(bad)[0][:5])
            if mode in first:
                np.testing.assert_array_equal(r, first[mode][0], err_msg=str(shape))
                assert m == first[mode][1] or (np.isnan(m) and np.isnan(first[mode][1]))
            else:
                first[mode] = (r, m)
    gr.close()

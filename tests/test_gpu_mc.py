"""Metropolis walkers on the GPU (cos_mc_*) against the oracle's walkers
(``oracle.metropolis``): the same Philox proposals and the same acceptance rule,
so with decision margins far above the modes' rounding (checked on the oracle
side: every |u|R| - |R'|| / |R'| >= 3.9e-4 for these seeds) the walkers' times
must be bitwise equal, the tallies equal, and the current values within the
mode's tolerance.  The average sign of a one-edge graph is checked against
quadrature."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle  # noqa: E402
from oracle import metropolis as mc  # noqa: E402
from workloads import chain_graph, medium, tiny  # noqa: E402
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


def _walk_gpu(cg, g, eps, beta, t0, mode, seed, steps, tuning=None, chunks=1):
    gr = cg.Graph.from_workload_graph(g)
    if tuning:
        gr.set_tuning(**tuning)
    S, D = t0.shape
    gr.set_samples(torch.from_numpy(t0).cuda(), eps, beta, cg.COS_T_SAMPLE_MAJOR)
    m = cg.Metropolis(gr, mode, seed)
    for q in range(chunks):                         # runs continue the same chains
        m.run(steps // chunks)
    st = m.stats()
    R = torch.empty(S, dtype=torch.float64, device="cuda")
    m.values(R)
    T = torch.empty((D, S), dtype=torch.float64, device="cuda")
    gr.copy_times(T)
    torch.cuda.synchronize()
    m.close()
    gr.close()
    return st, R.cpu().numpy(), np.ascontiguousarray(T.cpu().numpy().T)


@pytest.mark.parametrize("wl,seed,mode,tuning", [
    ("tiny", 17, 0, None), ("tiny", 17, 1, None),
    ("medium", 31, 0, {"schedule": 2}), ("medium", 31, 0, {"schedule": 1}), ("medium", 31, 1, None),
])
def test_walkers_match_oracle(cg, wl, seed, mode, tuning):
    w = tiny(num_samples=400) if wl == "tiny" else medium(num_samples=256)
    g, s = w.graph, w.samples
    steps = 20
    ref = mc.metropolis_run(g, s.eps, s.beta, s.t, seed, steps)
    assert ref["margins"].min() > 1e-4                 # no decision near a tie
    st, R, T = _walk_gpu(cg, g, s.eps, s.beta, s.t, mode, seed, steps, tuning, chunks=2)
    assert st == {"steps": steps, "accepted": ref["accepted"], "n_pos": ref["n_pos"], "n_neg": ref["n_neg"]}
    np.testing.assert_array_equal(T, ref["t"])
    Rf, Af = oracle.evaluate(g, s.eps, s.beta, ref["t"])
    np.testing.assert_array_equal(Rf, ref["R"])
    assert np.all(np.abs(R - Rf) <= TOL[mode] * Af)


def test_average_sign_of_one_edge_graph(cg):
    from scipy import integrate
    beta, epsv = 10.0, 0.7
    g = chain_graph([0], [0], [1], 1, 2)
    S = 16384
    t0 = counter_times(3, 0, S, 2, beta)
    gr = cg.Graph.from_workload_graph(g)
    gr.set_samples(torch.from_numpy(t0).cuda(), np.array([epsv]), beta, cg.COS_T_SAMPLE_MAJOR)
    m = cg.Metropolis(gr, 0, 99)
    m.run(100)                                        # burn-in
    a = m.stats()
    m.run(300)
    b = m.stats()
    m.close()
    gr.close()
    pos, neg = b["n_pos"] - a["n_pos"], b["n_neg"] - a["n_neg"]
    assert pos + neg == 300 * S
    G = lambda x: oracle.propagator(epsv, beta, np.array([x]))[0]
    num = sum(integrate.quad(lambda x: G(x) * (beta - abs(x)), lo, hi, limit=200)[0] for lo, hi in ((-beta, 0), (0, beta)))
    den = sum(integrate.quad(lambda x: abs(G(x)) * (beta - abs(x)), lo, hi, limit=200)[0] for lo, hi in ((-beta, 0), (0, beta)))
    assert abs((pos - neg) / (pos + neg) - num / den) < 0.01
    assert 0.2 < b["accepted"] / (400 * S) < 1.0


def test_walker_errors(cg):
    w = tiny(num_samples=16)
    gr = cg.Graph.from_workload_graph(w.graph)
    with pytest.raises(cg.CosError) as ei:              # no samples attached yet
        cg.Metropolis(gr, 0, 1)
    assert ei.value.code == cg.COS_ERR_STATE
    gr.set_samples(torch.from_numpy(w.samples.t).cuda(), w.samples.eps, w.samples.beta, cg.COS_T_SAMPLE_MAJOR)
    with pytest.raises(cg.CosError) as ei:              # counting has no weight to sample
        cg.Metropolis(gr, 2, 1)
    assert ei.value.code == cg.COS_ERR_INVALID
    m = cg.Metropolis(gr, 0, 1)
    m.run(2)
    gr.set_samples(torch.from_numpy(w.samples.t[:8].copy()).cuda(), w.samples.eps, w.samples.beta,
                   cg.COS_T_SAMPLE_MAJOR)
    with pytest.raises(cg.CosError) as ei:              # samples replaced under the walkers
        m.run(1)
    assert ei.value.code == cg.COS_ERR_STATE
    m.close()
    gr.close()

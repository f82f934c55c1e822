"""Pins of the CPU oracle against facts fixed by the paper and by mathematics.

The oracle is the level-wise dynamic program of Sec. II.B / Fig. 1 with the
free-fermion propagator of the synthetic workload.  Each test below checks it
against something other than itself: closed forms, brute-force path
enumeration, library sparse matrix products, propagator identities, and a
hand-derived fixture of the example graph in Fig. 2 / Fig. 3.
"""
import json
import math
import os

import numpy as np
import pytest
import scipy.sparse as sp

import oracle
from workloads import (FaninSpec, chain_graph, complete_layered_graph, figure_graph, make_graph,
                       tiny)

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ---------------------------------------------------------------- propagator

def test_propagator_closed_forms():
    # eps = ln 2, beta = 2: exp(-eps) = 1/2, exp(-beta eps) = 1/4
    e = math.log(2.0)
    assert oracle.propagator(e, 2.0, 1.0)[0] == pytest.approx(-0.4, rel=1e-15)
    assert oracle.propagator(e, 2.0, -1.0)[0] == pytest.approx(0.4, rel=1e-15)   # -G(tau + beta)
    # tau = 0 takes the tau >= 0 branch: -1/(1 + exp(-beta eps)); beta eps = ln 3 -> -3/4
    assert oracle.propagator(math.log(3.0) / 10.0, 10.0, 0.0)[0] == pytest.approx(-0.75, rel=1e-15)
    # eps = 0: G = -1/2 for tau >= 0 and +1/2 for tau < 0
    g = oracle.propagator(0.0, 10.0, [0.0, 3.0, 9.99, -0.1, -9.0])
    np.testing.assert_array_equal(g, [-0.5, -0.5, -0.5, 0.5, 0.5])


def test_propagator_antiperiodic_and_jump():
    rng = np.random.default_rng(11)
    beta = 10.0
    for eps in rng.uniform(-2, 2, size=8):
        tau = rng.uniform(1e-3, beta - 1e-3, size=64)
        np.testing.assert_allclose(oracle.propagator(eps, beta, tau - beta), -oracle.propagator(eps, beta, tau),
                                   rtol=1e-13)
        # G(0+) - G(0-) = -1
        jump = oracle.propagator(eps, beta, 0.0)[0] - oracle.propagator(eps, beta, -1e-300)[0]
        assert jump == pytest.approx(-1.0, abs=1e-15)


def test_propagator_derivative_and_bound():
    # dG/dtau = -eps G on both branches (pins the sign of the exponent), |G| <= 1
    rng = np.random.default_rng(12)
    beta, h = 10.0, 1e-6
    for eps in rng.uniform(-2, 2, size=8):
        tau = np.concatenate([rng.uniform(0.01, beta - 0.01, 32), rng.uniform(-beta + 0.01, -0.01, 32)])
        d = (oracle.propagator(eps, beta, tau + h) - oracle.propagator(eps, beta, tau - h)) / (2 * h)
        np.testing.assert_allclose(d, -eps * oracle.propagator(eps, beta, tau), rtol=1e-6, atol=1e-12)
        g = oracle.propagator(eps, beta, rng.uniform(-beta, beta, 1000))
        assert np.all(np.abs(g) <= 1.0)


# ---------------------------------------------------------------- golden fixture (Fig. 2 / Fig. 3)

def test_figure_graph_golden():
    with open(os.path.join(GOLDEN, "figure_graph.json")) as f:
        gold = json.load(f)
    g = figure_graph()
    np.testing.assert_array_equal(g.widths, gold["widths"])
    np.testing.assert_array_equal(g.edges[:, :2], np.array(gold["edges_src_dst"]))
    np.testing.assert_array_equal(g.edge_counts, gold["level_edge_counts"])
    cnt, ovf = oracle.count_paths(g)
    assert cnt == gold["path_count"] and not ovf
    paths = oracle.brute_force_paths(g)
    by_node = sorted([[0] + [int(g.edges[q, 1]) for q in p] for p in paths])
    assert by_node == sorted(gold["paths_by_node_hand_enumerated"])
    w = np.arange(g.num_edges, dtype=np.float64) + 1.0
    assert oracle.pathsum(g, w)[-1] == gold["weighted_sum"]
    assert oracle.brute_force_sum(paths, w)[0] == gold["weighted_sum"]


# ---------------------------------------------------------------- path sums

def _random_graph(seed, widths, fmax=3, K=3, D=4):
    rng = np.random.default_rng(seed)
    g = make_graph(widths, FaninSpec("uniform", fmax), K, D, rng)
    eps = rng.uniform(-2, 2, K)
    t = rng.uniform(0, 10.0, size=(8, D))
    return g, eps, t


@pytest.mark.parametrize("seed", range(8))
def test_dp_equals_brute_force(seed):
    g, eps, t = _random_graph(seed, [1, 3, 5, 6, 4, 2, 1], fmax=3)
    R, A = oracle.evaluate(g, eps, 10.0, t)
    paths = oracle.brute_force_paths(g)
    cnt, _ = oracle.count_paths(g)
    assert cnt == len(paths)
    for s in range(t.shape[0]):
        w = oracle.edge_weights(g, eps, 10.0, t[s])
        r, a = oracle.brute_force_sum(paths, w)
        assert abs(R[s] - r) <= 1e-14 * a + 1e-300
        assert A[s] == pytest.approx(a, rel=1e-13)
        assert abs(R[s]) <= A[s] * (1 + 1e-15) and A[s] <= cnt


def test_zero_energy_reduces_to_sign_count():
    # eps = 0: every factor is -1/2 (t_i >= t_j) or +1/2 (t_i < t_j); the sum over paths of the
    # products of those signs pins the orientation tau = t_i - t_j and the branch at tau = 0.
    g, _, t = _random_graph(5, [1, 4, 6, 6, 3, 1], fmax=3, K=2, D=5)
    t[:, 1] = t[:, 2]  # force some tau == 0 edges
    eps = np.zeros(2)
    R, _ = oracle.evaluate(g, eps, 10.0, t)
    paths = oracle.brute_force_paths(g)
    e = g.edges
    for s in range(t.shape[0]):
        w = np.where(t[s, e[:, 3]] >= t[s, e[:, 4]], -0.5, 0.5)
        assert R[s] == pytest.approx(oracle.brute_force_sum(paths, w)[0], rel=1e-14, abs=1e-300)


def test_chain_graph_closed_form():
    # eps = ln 2, beta = 2, tau = +-1 -> factors -0.4 / +0.4; a chain multiplies them.
    kinds = [0, 0, 0, 0, 0]
    ii = [0, 1, 0, 1, 0]
    jj = [1, 0, 1, 0, 0]
    g = chain_graph(kinds, ii, jj, 1, 2)
    t = np.array([[1.5, 0.5]])  # t0 - t1 = 1, t1 - t0 = -1, t0 - t0 = 0
    R, A = oracle.evaluate(g, np.array([math.log(2.0)]), 2.0, t)
    # factors: G(1) = -0.4, G(-1) = 0.4, G(1), G(-1), G(0) = -1/(1+1/4) = -0.8
    expected = (-0.4) * 0.4 * (-0.4) * 0.4 * (-0.8)
    assert R[0] == pytest.approx(expected, rel=1e-14)
    assert A[0] == pytest.approx(abs(expected), rel=1e-14)


def _incidence(g, l, off):
    e = g.edges
    lo = int(np.sum(g.edge_counts[:l]))
    hi = lo + int(g.edge_counts[l])
    rows = e[lo:hi, 1] - off[l]
    cols = e[lo:hi, 0] - off[l - 1]
    return lo, hi, rows, cols


def test_dp_equals_sparse_matrix_chain():
    # With sample-independent weights the sink value is e_sink^T M_{L-1} ... M_1 e_root.
    g, _, _ = _random_graph(21, [1, 7, 30, 40, 25, 9, 1], fmax=4)
    rng = np.random.default_rng(3)
    w = rng.uniform(-1.5, 1.5, g.num_edges)
    off = g.offsets()
    vec = np.ones(1)
    nodes = oracle.pathsum(g, w)
    for l in range(1, g.num_levels):
        lo, hi, rows, cols = _incidence(g, l, off)
        M = sp.coo_matrix((w[lo:hi], (rows, cols)), shape=(int(g.widths[l]), int(g.widths[l - 1]))).tocsr()
        vec = M @ vec
        np.testing.assert_allclose(nodes[off[l]:off[l + 1]], vec, rtol=1e-12, atol=1e-14)
    assert nodes[-1] == pytest.approx(vec[0], rel=1e-12)


def test_count_equals_integer_matrix_chain():
    g, _, _ = _random_graph(22, [1, 9, 40, 60, 60, 33, 7, 1], fmax=4)
    off = g.offsets()
    vec = np.ones(1, dtype=np.int64)
    for l in range(1, g.num_levels):
        lo, hi, rows, cols = _incidence(g, l, off)
        M = sp.coo_matrix((np.ones(hi - lo, dtype=np.int64), (rows, cols)),
                          shape=(int(g.widths[l]), int(g.widths[l - 1]))).tocsr()
        vec = M @ vec
    cnt, ovf = oracle.count_paths(g)
    assert cnt == int(vec[0]) and not ovf


@pytest.mark.parametrize("widths", [[1, 4, 8, 8, 4, 1], [1, 2, 3, 5, 7, 1], [1, 1], [1, 9, 1]])
def test_complete_layered_count_is_product_of_widths(widths):
    g = complete_layered_graph(widths)
    cnt, ovf = oracle.count_paths(g)
    assert cnt == math.prod(widths) and not ovf


def test_count_overflow_flag_and_wrap():
    widths = [1] + [256] * 8 + [1]          # 2^64 paths: overflows int64, wraps to 0
    g = complete_layered_graph(widths)
    cnt, ovf = oracle.count_paths(g)
    exact = 256 ** 8
    assert ovf
    wrapped = exact % (1 << 64)
    assert cnt == (wrapped - (1 << 64) if wrapped >= (1 << 63) else wrapped)
    widths = [1, 256, 256, 256, 256, 256, 256, 255, 127, 1]   # 2^48 * 32385 < 2^63: no flag
    g = complete_layered_graph(widths)
    cnt, ovf = oracle.count_paths(g)
    assert cnt == math.prod(widths) and not ovf


def test_uniform_scaling_of_weights():
    # every root-to-sink path has exactly L-1 edges, so scaling all weights by c scales R by c^(L-1)
    g, _, _ = _random_graph(23, [1, 5, 9, 9, 5, 1], fmax=3)
    w = np.random.default_rng(4).uniform(-1, 1, g.num_edges)
    r1 = oracle.pathsum(g, w)[-1]
    r2 = oracle.pathsum(g, 2.0 * w)[-1]
    assert r2 == pytest.approx(r1 * 2.0 ** (g.num_levels - 1), rel=1e-13)


def test_bounds_on_tiny_workload():
    wl = tiny()
    g, s = wl.graph, wl.samples
    R, A = oracle.evaluate(g, s.eps, s.beta, s.t)
    cnt, _ = oracle.count_paths(g)
    assert np.all(np.abs(R) <= A * (1 + 1e-14))
    assert np.all(A <= cnt)
    paths = oracle.brute_force_paths(g)
    assert len(paths) == cnt
    for q in range(0, s.num_samples, 97):
        r, a = oracle.brute_force_sum(paths, oracle.edge_weights(g, s.eps, s.beta, s.t[q]))
        assert abs(R[q] - r) <= 1e-14 * a


def test_thread_count_does_not_change_results():
    wl = tiny(num_samples=257)
    g, s = wl.graph, wl.samples
    R1, A1 = oracle.evaluate(g, s.eps, s.beta, s.t, nthreads=1)
    R4, A4 = oracle.evaluate(g, s.eps, s.beta, s.t, nthreads=4)
    np.testing.assert_array_equal(R1, R4)
    np.testing.assert_array_equal(A1, A4)


# ---------------------------------------------------------------- compensated mean

def test_neumaier_sum_matches_exact_sum():
    rng = np.random.default_rng(9)
    cases = [np.array([1e16, 1.0, -1e16, 1.0]), np.array([1.0, 1e100, 1.0, -1e100]),
             rng.standard_normal(10001) * 10.0 ** rng.integers(-8, 8, 10001)]
    for x in cases:
        assert oracle.neumaier_sum(x) == math.fsum(x)
    assert oracle.neumaier_mean(np.array([])) == 0.0


# ---------------------------------------------------------------- fermion-loop sign (kind bit 30)

def _with_signs(g, mask):
    from workloads import Graph
    e = g.edges.copy()
    e[mask, 2] |= oracle.SIGN_BIT
    return Graph(g.widths, g.edge_counts, e, g.num_kinds, g.num_times)


def test_sign_flag_on_one_level_negates_every_path():
    # every root-to-sink path crosses each level exactly once, so flagging all edges
    # into one level multiplies every path, hence R, by -1 (A is unchanged)
    g, eps, t = _random_graph(31, [1, 4, 7, 7, 3, 1], fmax=3)
    R, A = oracle.evaluate(g, eps, 10.0, t)
    lvl = np.repeat(np.arange(g.num_levels), g.edge_counts)
    Rs, As = oracle.evaluate(_with_signs(g, lvl == 3), eps, 10.0, t)
    np.testing.assert_array_equal(Rs, -R)
    np.testing.assert_array_equal(As, A)
    # two flagged levels cancel
    R2, _ = oracle.evaluate(_with_signs(g, (lvl == 2) | (lvl == 4)), eps, 10.0, t)
    np.testing.assert_array_equal(R2, R)


def test_sign_flags_against_brute_force_and_chain():
    g, eps, t = _random_graph(32, [1, 3, 6, 6, 2, 1], fmax=3)
    mask = np.random.default_rng(2).random(g.num_edges) < 0.4
    gs = _with_signs(g, mask)
    R, _ = oracle.evaluate(gs, eps, 10.0, t)
    paths = oracle.brute_force_paths(gs)
    for s in range(t.shape[0]):
        w = oracle.edge_weights(gs, eps, 10.0, t[s])
        r, a = oracle.brute_force_sum(paths, w)
        assert abs(R[s] - r) <= 1e-14 * a
    # chain with closed-form factors: one flagged edge flips the sign of the product
    c = chain_graph([0, 0, 0], [0, 1, 0], [1, 0, 0], 1, 2)
    tt = np.array([[1.5, 0.5]])
    R0, _ = oracle.evaluate(c, np.array([math.log(2.0)]), 2.0, tt)
    R1, _ = oracle.evaluate(_with_signs(c, np.array([False, True, False])), np.array([math.log(2.0)]), 2.0, tt)
    assert R0[0] == pytest.approx((-0.4) * 0.4 * (-0.8), rel=1e-14) and R1[0] == -R0[0]


# ------------------------------------------------------------------ tabulated propagators

def test_tabulated_propagator_exact_on_piecewise_linear_tables():
    # a table sampled from a + b*tau on each half is reproduced exactly between nodes
    # (closed form), and the end values hold outside [-tau_max, tau_max]
    rng = np.random.default_rng(11)
    T, tau_max = 37, 7.5
    a_pos, b_pos, a_neg, b_neg = rng.normal(size=4)
    xs = np.arange(T + 1) * (tau_max / T)
    tab = np.stack([a_pos + b_pos * xs, a_neg + b_neg * (xs - tau_max)])
    tau = rng.uniform(-tau_max, tau_max, 4000)
    got = oracle.tabulated_propagator(tab, tau_max, tau)
    want = np.where(tau >= 0, a_pos + b_pos * tau, a_neg + b_neg * tau)
    np.testing.assert_allclose(got, want, rtol=0, atol=1e-13)
    out = oracle.tabulated_propagator(tab, tau_max, np.array([tau_max * 1.5, -tau_max * 2.0]))
    assert out[0] == pytest.approx(a_pos + b_pos * tau_max, abs=1e-13)
    assert out[1] == pytest.approx(a_neg - b_neg * tau_max, abs=1e-13)


def test_tabulated_propagator_hits_nodes_and_keeps_the_jump():
    # grid nodes exactly representable (T and tau_max powers of two): node values
    # come back exactly; tau = 0 takes the tau >= 0 table (G(0+)), tau < 0 the other
    T, tau_max = 64, 8.0
    rng = np.random.default_rng(12)
    tab = rng.normal(size=(2, T + 1))
    m = np.arange(T + 1)
    assert np.array_equal(oracle.tabulated_propagator(tab, tau_max, m * (tau_max / T)), tab[0])
    assert np.array_equal(oracle.tabulated_propagator(tab, tau_max, -tau_max + m[:-1] * (tau_max / T)), tab[1][:-1])
    assert oracle.tabulated_propagator(tab, tau_max, 0.0)[0] == tab[0][0]
    assert oracle.tabulated_propagator(tab, tau_max, -1e-300)[0] == pytest.approx(tab[1][-1], abs=1e-12)


@pytest.mark.parametrize("eps", [-1.7, 0.0, 0.9])
def test_tabulated_free_propagator_within_interpolation_bound(eps):
    # tables sampled from the free-fermion G: linear interpolation is within
    # h^2/8 * max|G''| of it, and G'' = eps^2 G with |G| <= 1 (antiperiodic halves)
    beta, T = 10.0, 400
    h = beta / T
    xs = np.arange(T + 1) * h
    tab = np.stack([oracle.propagator(eps, beta, xs), oracle.propagator(eps, beta, xs - beta + 0.0)])
    tab[1][-1] = oracle.propagator(eps, beta, -1e-12)[0]   # G(0-) as the limit from below
    tau = np.random.default_rng(13).uniform(-beta, beta, 5000)
    tau = tau[np.abs(tau) > 1e-9]
    err = np.abs(oracle.tabulated_propagator(tab, beta, tau) - oracle.propagator(eps, beta, tau))
    bound = h * h / 8.0 * eps * eps * 1.0 + 1e-12
    assert err.max() <= bound


def test_tabulated_dp_against_brute_force():
    g, eps, t = _random_graph(41, [1, 3, 5, 5, 2, 1], fmax=3)
    rng = np.random.default_rng(14)
    tables = rng.normal(size=(g.num_kinds, 2, 9))
    mask = rng.random(g.num_edges) < 0.3
    gs = _with_signs(g, mask)
    R, A = oracle.evaluate_tabulated(gs, tables, 10.0, t)
    paths = oracle.brute_force_paths(gs)
    for s in range(t.shape[0]):
        w = oracle.tabulated_edge_weights(gs, tables, 10.0, t[s])
        r, a = oracle.brute_force_sum(paths, w)
        assert abs(R[s] - r) <= 1e-13 * a and abs(A[s] - a) <= 1e-13 * a


def test_tabulated_sign_flags_on_one_level_negate_every_path():
    g, _, t = _random_graph(43, [1, 4, 6, 6, 3, 1], fmax=3)
    tables = np.random.default_rng(15).normal(size=(g.num_kinds, 2, 6))
    lvl = np.repeat(np.arange(g.num_levels), g.edge_counts)
    R0, A0 = oracle.evaluate_tabulated(g, tables, 10.0, t)
    R1, A1 = oracle.evaluate_tabulated(_with_signs(g, lvl == 3), tables, 10.0, t)
    np.testing.assert_array_equal(R1, -R0)
    np.testing.assert_array_equal(A1, A0)


def test_tabulated_formula_agrees_with_library_interpolation():
    # the fixed arithmetic of the definition against numpy's linear interpolation:
    # they differ only by the rounding of the position in the interval
    rng = np.random.default_rng(16)
    T, tau_max = 23, 9.0
    tab = rng.normal(size=(2, T + 1))
    tau = rng.uniform(-11.0, 11.0, 20000)
    got = oracle.tabulated_propagator(tab, tau_max, tau)
    xs = np.arange(T + 1) * (tau_max / T)
    pos = tau >= 0
    want = np.where(pos, np.interp(tau, xs, tab[0]), np.interp(tau, xs - tau_max, tab[1]))
    slope = np.max(np.abs(np.diff(tab, axis=1))) * T / tau_max
    assert np.max(np.abs(got - want)) <= 8 * np.finfo(float).eps * (11.0 * slope + np.max(np.abs(tab)))


def test_tabulated_double_evaluations_within_the_rounding_scale():
    # The long-double definition against three double-precision evaluations that
    # round the grid coordinate differently (scaled by T/tau_max and shifted by T;
    # divided by h after shifting by tau_max; numpy's own interpolation): each stays
    # within tabulated_rounding_scale of it, including at nodes, near zeros of G and
    # outside the grid.  A scale without its position term fails here.
    rng = np.random.default_rng(18)
    for T, tau_max in ((23, 9.0), (256, 10.0), (7, 3.3)):
        tab = rng.normal(size=(2, T + 1))
        tab[0][T // 2] = 1e-9                       # a zero crossing next to a node
        xs = np.arange(T + 1) * (tau_max / T)
        tau = np.concatenate([rng.uniform(-1.2 * tau_max, 1.2 * tau_max, 20000), xs, xs - tau_max,
                              xs[T // 2] + np.array([-1e-12, 1e-12])])
        exact = oracle.tabulated_propagator(tab, tau_max, tau)
        scale = oracle.tabulated_rounding_scale(tab, tau_max, tau)
        pos = tau >= 0
        evals = []
        u = np.where(pos, tau * (T / tau_max), tau * (T / tau_max) + T)
        v = np.where(pos, tau / (tau_max / T), (tau + tau_max) / (tau_max / T))
        for x in (u, v):
            m = np.clip(np.floor(x), 0, T - 1).astype(np.int64)
            f = np.clip(x - m, 0.0, 1.0)
            half = np.where(pos[:, None], tab[0][None, :], tab[1][None, :])
            a, b = half[np.arange(tau.size), m], half[np.arange(tau.size), m + 1]
            evals.append(a + f * (b - a))
        evals.append(np.where(pos, np.interp(tau, xs, tab[0]), np.interp(tau, xs - tau_max, tab[1])))
        for got in evals:
            assert np.all(np.abs(got - exact) <= scale)
        pos_only = 4.0 * oracle.UNIT_ROUNDOFF * (np.abs(np.concatenate([tab[0], tab[1]])).max())
        assert np.any(np.abs(evals[0] - exact) > pos_only) or np.any(np.abs(evals[1] - exact) > pos_only)


def test_tabulated_rounding_bound_against_brute_force():
    # B(s) = sum over edges of eps_e times the |paths| through the edge without it
    # (forward and backward DPs) equals the brute-force sum over paths of
    # sum_{e in path} eps_e * prod_{e' != e} |w_e'|
    g, _, t = _random_graph(44, [1, 3, 5, 4, 2, 1], fmax=3)
    tables = np.random.default_rng(19).normal(size=(g.num_kinds, 2, 11))
    R, A, B = oracle.evaluate_tabulated(g, tables, 10.0, t, with_bound=True)
    paths = oracle.brute_force_paths(g)
    for s in range(t.shape[0]):
        w, sc = oracle.tabulated_edge_weights(g, tables, 10.0, t[s], scale=True)
        want = 0.0
        for path in paths:
            aw = np.abs(w[path])
            for q, e in enumerate(path):
                want += sc[e] * np.prod(np.delete(aw, q))
        assert abs(B[s] - want) <= 1e-12 * want
        assert B[s] > 0 and abs(A[s] - oracle.brute_force_sum(paths, w)[1]) <= 1e-13 * A[s]


# ------------------------------------------------------------------ long-double reference

def test_tight_oracle_chain_closed_form():
    # the chain of rational factors (-0.4, 0.4, -0.4, 0.4, -0.8) of the double closed-form pin
    g = chain_graph([0, 0, 0, 0, 0], [0, 1, 0, 1, 0], [1, 0, 1, 0, 0], 1, 2)
    Rt = oracle.evaluate_tight(g, np.array([math.log(2.0)]), 2.0, np.array([[1.5, 0.5]]))
    expected = (-0.4) * 0.4 * (-0.4) * 0.4 * (-0.8)
    assert abs(Rt[0] - expected) <= 2 * np.spacing(abs(expected))


def test_tight_oracle_zero_energy_sign_count_is_exact():
    # eps = 0: factors are exactly -1/2 or +1/2, so every path value and their sum are
    # exact in any binary format; the long-double result must equal the brute-force sum
    g, _, t = _random_graph(6, [1, 4, 6, 6, 3, 1], fmax=3, K=2, D=5)
    t[:, 1] = t[:, 2]
    g = _with_signs(g, np.random.default_rng(7).random(g.num_edges) < 0.3)   # fermion-loop flags too
    Rt = oracle.evaluate_tight(g, np.zeros(2), 10.0, t)
    paths = oracle.brute_force_paths(g)
    e = g.edges
    flip = np.where((e[:, 2] & oracle.SIGN_BIT) != 0, -1.0, 1.0)
    for s in range(t.shape[0]):
        w = np.where(t[s, e[:, 3]] >= t[s, e[:, 4]], -0.5, 0.5) * flip
        assert Rt[s] == oracle.brute_force_sum(paths, w)[0]


def test_double_oracle_within_its_rounding_bound_of_the_tight_one():
    # the double DP's error is at most about (path length + fan-in) roundings of the
    # largest paths: |R - R_tight| <= c (L + F) u A with u = 2^-53
    from workloads import medium
    w = medium(num_samples=120)
    R, A = oracle.evaluate(w.graph, w.samples.eps, w.samples.beta, w.samples.t)
    Rt = oracle.evaluate_tight(w.graph, w.samples.eps, w.samples.beta, w.samples.t)
    u = 2.0 ** -53
    assert np.all(np.abs(R - Rt) <= 4 * (w.graph.num_levels + 4) * u * A)
    assert np.max(np.abs(R - Rt) / A) > 0      # the references differ: double rounding is visible

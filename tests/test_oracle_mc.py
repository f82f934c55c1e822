"""Pins of the oracle's Metropolis sampler of the vertex times (Sec. II.B: Monte
Carlo integration over the times; Sec. II.C/III: many walkers, proposal and
acceptance on the device): the chain's stationary distribution and average sign
on a one-edge graph against quadrature, exact acceptance when |R| is constant,
uniform coordinate choice, and the proposal words' formula."""
import math

import numpy as np
import pytest
from scipy import integrate

import oracle
from oracle import metropolis as mc
from workloads import chain_graph
from workloads.generate import counter_times, philox4x32_10


def _one_edge(eps):
    # root -> sink through one edge of kind 0 between times 0 and 1: R(t) = G(t0 - t1)
    return chain_graph([0], [0], [1], 1, 2), np.array([eps])


def _run_collect(g, eps, beta, S, burn, steps, seed):
    t = counter_times(seed, 0, S, g.num_times, beta)
    res = mc.metropolis_run(g, eps, beta, t, seed, burn)
    taus, signs = [], 0
    n = burn
    t = res["t"]
    tallies = np.zeros(2, dtype=np.int64)
    for _ in range(steps):
        r = mc.metropolis_run(g, eps, beta, t, seed, 1, first_step=n)
        t = r["t"]
        n += 1
        taus.append(t[:, 0] - t[:, 1])
        tallies += (r["n_pos"], r["n_neg"])
    return np.concatenate(taus), tallies


def test_stationary_distribution_and_average_sign_on_one_edge():
    beta, epsv = 10.0, 0.7
    g, eps = _one_edge(epsv)
    taus, (n_pos, n_neg) = _run_collect(g, eps, beta, S=2000, burn=60, steps=250, seed=5)
    G = lambda tau: oracle.propagator(epsv, beta, np.array([tau]))[0]
    # tau = t0 - t1 of uniform times has density (beta - |tau|) / beta^2; the chain
    # samples it weighted by |G(tau)|
    dens = lambda tau: abs(G(tau)) * (beta - abs(tau))
    Z = integrate.quad(dens, -beta, 0, limit=200)[0] + integrate.quad(dens, 0, beta, limit=200)[0]
    edges = np.linspace(-beta, beta, 11)
    hist = np.histogram(taus, bins=edges)[0] / taus.size
    for a, b, h in zip(edges[:-1], edges[1:], hist):
        p = integrate.quad(dens, a, b, limit=200, points=[0.0] if a < 0 < b else None)[0] / Z
        if p > 0.03:
            assert abs(h - p) <= 0.06 * p + 0.003, (a, b, h, p)
    # average sign -> integral of R over integral of |R|
    num = integrate.quad(lambda x: G(x) * (beta - abs(x)), -beta, 0, limit=200)[0] + \
        integrate.quad(lambda x: G(x) * (beta - abs(x)), 0, beta, limit=200)[0]
    want = num / Z
    got = (n_pos - n_neg) / (n_pos + n_neg)
    assert abs(got - want) < 0.03, (got, want)
    assert -1.0 < want < 0.0   # both signs occur: the check is not trivial


def test_constant_weight_accepts_every_move_and_keeps_last_proposals():
    # eps = 0: |G| = 1/2 everywhere, so u * |R| < |R'| always (u < 1)
    g, eps = _one_edge(0.0)
    S, D, beta, seed, steps = 300, 2, 10.0, 9, 12
    t0 = counter_times(seed, 0, S, D, beta)
    r = mc.metropolis_run(g, eps, beta, t0, seed, steps)
    assert r["accepted"] == S * steps
    want = t0.copy()
    for n in range(steps):
        i, val, _ = mc.mc_proposal(seed, n, S, D, beta)
        want[np.arange(S), i] = val
    np.testing.assert_array_equal(r["t"], want)


def test_coordinate_choice_uniform_and_values_in_range():
    S, D, beta = 20000, 5, 3.0
    i, val, u = mc.mc_proposal(11, 7, S, D, beta)
    counts = np.bincount(i, minlength=D)
    assert counts.size == D and np.all(np.abs(counts / S - 1 / D) < 0.02)
    assert np.all((val >= 0) & (val < beta)) and np.all((u > 0) & (u < 1))
    # values use the same 53-bit construction as the sample generator
    w0, w1, w2, w3 = mc.mc_words(11, 7, S)
    x = ((w2.astype(np.uint64) << np.uint64(32)) | w1) >> np.uint64(11)
    np.testing.assert_array_equal(val, beta * (x.astype(np.float64) * 2.0 ** -53))


def test_walker_streams_differ_from_sample_streams():
    # the fourth counter word's top bit separates the walkers' streams from counter_times'
    w = mc.mc_words(3, 0, 4)
    s = np.arange(4, dtype=np.uint64)
    v = philox4x32_10(s, s * 0, s * 0, s * 0, 3, 0)
    assert not any(np.array_equal(a, b) for a, b in zip(w, v))

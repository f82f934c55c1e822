"""Metropolis sampling of the vertex times -- TEST INFRASTRUCTURE ONLY (like the
rest of ``oracle``).

Sec. II.B: the sum over diagrams is integrated over the vertex times by Monte
Carlo sampling; Sec. II.C ("Distributing the task") runs many Markov-chain
walkers at once, and Sec. III notes that proposal and acceptance of
configurations belong in device code.  The chain here, one per walker s, is the
plain Metropolis algorithm on the weight |R(t)|:

  step n, walker s: Philox-4x32-10 with counter (s mod 2^32, s >> 32, n mod 2^32,
  2^31 | n >> 32) and key (seed mod 2^32, seed >> 32) gives words w0..w3;
    coordinate  i  = (w0 * D) >> 32
    new value   t'_i = beta * (((w2 << 32 | w1) >> 11) * 2^-53)
    uniform     u  = (w3 + 1/2) * 2^-32
  t' is t with coordinate i replaced; R' = R(t') (the DP of Fig. 1); the move is
  accepted iff u * |R| < |R'| (probability min(1, |R'|/|R|)); then the walker's
  current R is tallied: n_pos if R > 0, n_neg if R < 0.

The average sign (n_pos - n_neg) / (n_pos + n_neg) estimates the ratio of the
integral of R to the integral of |R| over [0, beta)^D.  The counter's top bit
keeps these streams apart from the sample generator of ``workloads``
(``counter_times``, whose fourth counter word is 0), whose Philox this module
uses.
"""
from __future__ import annotations

from typing import Dict

import numpy as np

from . import evaluate
from workloads.generate import philox4x32_10


def mc_words(seed: int, step: int, num_walkers: int):
    """Philox words (w0, w1, w2, w3) of every walker at one step, as uint64 arrays."""
    s = np.arange(num_walkers, dtype=np.uint64)
    lo, hi = s & np.uint64(0xFFFFFFFF), s >> np.uint64(32)
    c2 = np.full(num_walkers, step & 0xFFFFFFFF, np.uint64)
    c3 = np.full(num_walkers, 0x80000000 | ((step >> 32) & 0x7FFFFFFF), np.uint64)
    return philox4x32_10(lo, hi, c2, c3, seed & 0xFFFFFFFF, (seed >> 32) & 0xFFFFFFFF)


def mc_proposal(seed: int, step: int, num_walkers: int, num_times: int, beta: float):
    """(coordinate index i[s], proposed value t'_i[s], acceptance uniform u[s]) of one step."""
    w0, w1, w2, w3 = mc_words(seed, step, num_walkers)
    i = ((w0 * np.uint64(num_times)) >> np.uint64(32)).astype(np.int64)
    x = (((w2 << np.uint64(32)) | w1) >> np.uint64(11)).astype(np.float64) * 2.0 ** -53
    u = (w3.astype(np.float64) + 0.5) * 2.0 ** -32
    return i, beta * x, u


def metropolis_run(graph, eps: np.ndarray, beta: float, t0: np.ndarray, seed: int, num_steps: int,
                   first_step: int = 0) -> Dict[str, np.ndarray]:
    """Run num_steps Metropolis steps for every walker (rows of t0 [S, D]) and return
    the final times, the final R, the tallies and per step the acceptance masks and
    the decision margins |u|R| - |R'|| / max(|R'|, tiny) (small margins mark
    decisions that rounding could flip)."""
    t = np.array(t0, dtype=np.float64, copy=True)
    S, D = t.shape
    R, _ = evaluate(graph, eps, beta, t, with_abs=False)
    n_pos = n_neg = accepted = 0
    masks, margins = [], []
    for n in range(first_step, first_step + num_steps):
        i, val, u = mc_proposal(seed, n, S, D, beta)
        tp = t.copy()
        tp[np.arange(S), i] = val
        Rp, _ = evaluate(graph, eps, beta, tp, with_abs=False)
        lhs, rhs = u * np.abs(R), np.abs(Rp)
        acc = lhs < rhs
        masks.append(acc)
        margins.append(np.abs(lhs - rhs) / np.maximum(rhs, 1e-300))
        t[acc] = tp[acc]
        R = np.where(acc, Rp, R)
        accepted += int(acc.sum())
        n_pos += int((R > 0).sum())
        n_neg += int((R < 0).sum())
    return {"t": t, "R": R, "n_pos": n_pos, "n_neg": n_neg, "accepted": accepted,
            "masks": np.array(masks), "margins": np.array(margins)}

"""Seeded synthetic leveled digraphs and samples (numpy PCG64).

The paper's workloads are real CoS graphs for Hubbard-type expansions
(Sec. III); their construction rules are not in the paper, so random leveled
DAGs with the paper's level structure stand in for them.  A graph is a list of
levels l = 0..L-1 with widths W_l; level l owns the contiguous global node ids
[off_l, off_l + W_l); the root is node 0 (W_0 = 1) and the sink is node N-1
(W_{L-1} = 1).  Every edge joins level l-1 to level l (Fig. 2, Fig. 3) and
carries a propagator kind k and two time-variable indices (i, j).  Edges are
emitted per level in src order, the flattened layout of Fig. 3.

Random draws happen in a fixed order per workload: the graph (level by level:
fan-ins, parents, then kinds and time indices), then eps_k, then the times t.
"""
from __future__ import annotations

import dataclasses
import math
from typing import Callable, Dict, List, Optional, Sequence, Tuple

import numpy as np

BETA = 10.0


@dataclasses.dataclass
class FaninSpec:
    """Fan-in distribution of each non-root node.

    kind == "uniform":   f ~ U{1..fmax}
    kind == "geometric": f on 1..fmax with P(f) proportional to (1-p)^(f-1)
    The drawn f is capped at the width of the previous level; parents are then
    drawn uniformly without replacement from the previous level.
    """
    kind: str = "uniform"
    fmax: int = 3
    p: float = 0.31

    def draw(self, rng: np.random.Generator, n: int) -> np.ndarray:
        if self.kind == "uniform":
            return rng.integers(1, self.fmax + 1, size=n, dtype=np.int64)
        if self.kind == "geometric":
            f = np.arange(1, self.fmax + 1)
            w = (1.0 - self.p) ** (f - 1)
            return rng.choice(f, size=n, p=w / w.sum()).astype(np.int64)
        raise ValueError(f"unknown fan-in kind {self.kind!r}")


@dataclasses.dataclass
class Graph:
    """Per-level flattened edge lists, the input format of graph creation.

    widths:      int64 [L]
    edge_counts: int64 [L]; edge_counts[0] == 0, edge_counts[l] = edges into level l
    edges:       int32 [E, 5]; rows (src, dst, kind, i, j) with global node ids,
                 level-major (all edges into level 1, then level 2, ...)
    """
    widths: np.ndarray
    edge_counts: np.ndarray
    edges: np.ndarray
    num_kinds: int
    num_times: int

    @property
    def num_levels(self) -> int:
        return int(len(self.widths))

    @property
    def num_nodes(self) -> int:
        return int(self.widths.sum())

    @property
    def num_edges(self) -> int:
        return int(self.edges.shape[0])

    def offsets(self) -> np.ndarray:
        off = np.zeros(len(self.widths) + 1, dtype=np.int64)
        np.cumsum(self.widths, out=off[1:])
        return off


@dataclasses.dataclass
class Samples:
    """Sample inputs: eps[K] (float64), beta, and times t[S, D] (float64)."""
    eps: np.ndarray
    beta: float
    t: np.ndarray

    @property
    def num_samples(self) -> int:
        return int(self.t.shape[0])


@dataclasses.dataclass
class Workload:
    name: str
    graph: Graph
    samples: Samples


def _distinct_parents(rng: np.random.Generator, fanin: np.ndarray, width: int) -> np.ndarray:
    """Draw, per row, fanin[r] distinct parents in [0, width); returns [n, fmax] (-1 = unused)."""
    n = fanin.shape[0]
    fmax = int(fanin.max()) if n else 0
    out = rng.integers(0, width, size=(n, fmax), dtype=np.int64) if fmax else np.zeros((n, 0), np.int64)
    col = np.arange(fmax)[None, :]
    used = col < fanin[:, None]
    # Redraw any entry equal to an earlier used entry in its row until all are distinct.
    for _ in range(10_000):
        dup = np.zeros_like(used)
        for a in range(1, fmax):
            same = np.zeros(n, dtype=bool)
            for b in range(a):
                same |= out[:, a] == out[:, b]
            dup[:, a] = same & used[:, a]
        if not dup.any():
            break
        rows, cols = np.nonzero(dup)
        out[rows, cols] = rng.integers(0, width, size=rows.shape[0], dtype=np.int64)
    else:  # pragma: no cover - only reachable with fanin > width
        raise RuntimeError("could not draw distinct parents")
    out[~used] = -1
    return out


def make_graph(widths: Sequence[int], fanin: FaninSpec, num_kinds: int, num_times: int,
               rng: np.random.Generator) -> Graph:
    """Random leveled DAG: each node of level l >= 1 draws its parents from level l-1."""
    w = np.asarray(widths, dtype=np.int64)
    if len(w) < 2 or w[0] != 1 or w[-1] != 1 or (w < 1).any():
        raise ValueError("widths must start and end with 1 and be positive")
    off = np.zeros(len(w) + 1, dtype=np.int64)
    np.cumsum(w, out=off[1:])
    counts = np.zeros(len(w), dtype=np.int64)
    chunks: List[np.ndarray] = []
    for l in range(1, len(w)):
        n = int(w[l])
        f = np.minimum(fanin.draw(rng, n), w[l - 1])
        par = _distinct_parents(rng, f, int(w[l - 1]))
        rows, cols = np.nonzero(par >= 0)
        src = off[l - 1] + par[rows, cols]
        dst = off[l] + rows
        # Flattened per-level list in src order (Fig. 3), stable so equal srcs keep dst order.
        order = np.argsort(src, kind="stable")
        src, dst = src[order], dst[order]
        e = src.shape[0]
        kind = rng.integers(0, num_kinds, size=e, dtype=np.int64)
        ii = rng.integers(0, num_times, size=e, dtype=np.int64)
        jj = rng.integers(0, num_times, size=e, dtype=np.int64)
        chunks.append(np.stack([src, dst, kind, ii, jj], axis=1).astype(np.int32))
        counts[l] = e
    edges = np.concatenate(chunks, axis=0) if chunks else np.zeros((0, 5), np.int32)
    return Graph(widths=w, edge_counts=counts, edges=np.ascontiguousarray(edges),
                 num_kinds=int(num_kinds), num_times=int(num_times))


def make_eps(num_kinds: int, rng: np.random.Generator) -> np.ndarray:
    """eps_k ~ U[-2, 2]."""
    return rng.uniform(-2.0, 2.0, size=num_kinds)


def make_times(num_samples: int, num_times: int, beta: float, rng: np.random.Generator) -> np.ndarray:
    """t ~ U[0, beta)^D per sample, shape [S, D]."""
    return rng.uniform(0.0, beta, size=(num_samples, num_times))


def geometric_widths(num_levels: int, ratio: int, cap: int) -> List[int]:
    """W_l = min(cap, ratio^l, ratio^(L-1-l)): grows from 1 to cap and shrinks back to 1."""
    out = []
    for l in range(num_levels):
        e = min(l, num_levels - 1 - l)
        out.append(int(min(cap, ratio ** e)))
    return out


def widths_for_target(num_levels: int, target_nodes: int, ratio: int = 32) -> List[int]:
    """Geometric profile whose node count is close to target_nodes (ratio raised if needed)."""
    r = ratio
    while sum(geometric_widths(num_levels, r, 1 << 62)) < target_nodes and r < (1 << 30):
        r *= 2
    lo, hi = 1, max(1, target_nodes)
    while lo < hi:  # smallest cap with sum >= target
        mid = (lo + hi) // 2
        if sum(geometric_widths(num_levels, r, mid)) >= target_nodes:
            hi = mid
        else:
            lo = mid + 1
    return geometric_widths(num_levels, r, lo)


def _workload(name: str, seed: int, widths, fanin: FaninSpec, K: int, D: int, S: int,
              beta: float = BETA, num_samples_override: Optional[int] = None) -> Workload:
    rng = np.random.default_rng(seed)
    g = make_graph(widths, fanin, K, D, rng)
    eps = make_eps(K, rng)
    s = S if num_samples_override is None else num_samples_override
    t = make_times(s, D, beta, rng)
    return Workload(name, g, Samples(eps=eps, beta=beta, t=t))


TINY_WIDTHS = [1, 4, 8, 8, 4, 1]


def tiny(seed: int = 0, num_samples: int = 1024) -> Workload:
    """Tiny: L=6, widths [1,4,8,8,4,1], fan-in U{1..3}, K=4, D=6, 1024 samples."""
    return _workload("tiny", seed, TINY_WIDTHS, FaninSpec("uniform", 3), 4, 6, num_samples)


def medium(seed: int = 1, num_samples: int = 65536) -> Workload:
    """Medium: L=10, widths min(4096, 32^l, 32^(9-l)), fan-in U{1..4}, K=16, D=10, 65,536 samples."""
    return _workload("medium", seed, geometric_widths(10, 32, 4096), FaninSpec("uniform", 4),
                     16, 10, num_samples)


def large(seed: int = 2, num_samples: int = 1 << 20) -> Workload:
    """Large: L=14, widths min(2^18, 64^l, 64^(13-l)), truncated geometric fan-in on 1..6
    (p = 0.31, mean about 2.5), K=32, D=14, 2^20 samples."""
    return _workload("large", seed, geometric_widths(14, 64, 1 << 18),
                     FaninSpec("geometric", 6, 0.31), 32, 14, num_samples)


def _log_uniform_int(rng: np.random.Generator, lo: float, hi: float) -> int:
    return int(round(math.exp(rng.uniform(math.log(lo), math.log(hi)))))


def batched(seed: int = 3, num_graphs: int = 64, max_nodes: float = 1e6,
            max_samples: float = float(1 << 20), min_samples: float = 4096.0) -> List[Workload]:
    """Batched uneven: per graph order n ~ U{2..8}, L = 2n+2, N ~ logU[1e3, max_nodes],
    fan-in U{1..4}, K=16, D=L, S ~ logU[min_samples, max_samples]."""
    rng = np.random.default_rng(seed)
    out = []
    for gi in range(num_graphs):
        n = int(rng.integers(2, 9))
        L = 2 * n + 2
        N = _log_uniform_int(rng, 1e3, max_nodes)
        S = _log_uniform_int(rng, min_samples, max_samples)
        widths = widths_for_target(L, N)
        g = make_graph(widths, FaninSpec("uniform", 4), 16, L, rng)
        eps = make_eps(16, rng)
        t = make_times(S, L, BETA, rng)
        out.append(Workload(f"batched[{gi}]", g, Samples(eps=eps, beta=BETA, t=t)))
    return out


def serving_pool(seed: int = 4, pool_size: int = 128, max_nodes: float = 2e6) -> List[Tuple[Graph, np.ndarray]]:
    """Serving pool: graphs with order n ~ U{2..8}, L = 2n+2, N ~ logU[1e3, max_nodes],
    truncated geometric fan-in on 1..6, K=32, D=L; returns (graph, eps) pairs."""
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(pool_size):
        n = int(rng.integers(2, 9))
        L = 2 * n + 2
        N = _log_uniform_int(rng, 1e3, max_nodes)
        widths = widths_for_target(L, N)
        g = make_graph(widths, FaninSpec("geometric", 6, 0.31), 32, L, rng)
        out.append((g, make_eps(32, rng)))
    return out


def complete_layered_graph(widths: Sequence[int], num_kinds: int = 1, num_times: int = 1,
                           rng: Optional[np.random.Generator] = None) -> Graph:
    """Every node of level l-1 feeds every node of level l (edges in src order)."""
    w = np.asarray(widths, dtype=np.int64)
    off = np.zeros(len(w) + 1, dtype=np.int64)
    np.cumsum(w, out=off[1:])
    rng = rng or np.random.default_rng(0)
    rows, counts = [], np.zeros(len(w), dtype=np.int64)
    for l in range(1, len(w)):
        s, d = np.meshgrid(np.arange(w[l - 1]) + off[l - 1], np.arange(w[l]) + off[l], indexing="ij")
        e = s.size
        k = rng.integers(0, num_kinds, size=e)
        i = rng.integers(0, num_times, size=e)
        j = rng.integers(0, num_times, size=e)
        rows.append(np.stack([s.ravel(), d.ravel(), k, i, j], axis=1))
        counts[l] = e
    return Graph(w, counts, np.ascontiguousarray(np.concatenate(rows).astype(np.int32)), num_kinds, num_times)


def chain_graph(kinds: Sequence[int], ii: Sequence[int], jj: Sequence[int], num_kinds: int,
                num_times: int) -> Graph:
    """A single path of len(kinds) edges through levels of width 1."""
    L = len(kinds) + 1
    edges = np.array([[l - 1, l, kinds[l - 1], ii[l - 1], jj[l - 1]] for l in range(1, L)], dtype=np.int32)
    counts = np.array([0] + [1] * (L - 1), dtype=np.int64)
    return Graph(np.ones(L, dtype=np.int64), counts, edges.reshape(-1, 5), num_kinds, num_times)


def figure_graph() -> Graph:
    """The example graph of Fig. 2 / Fig. 3 with its elided middle closed.

    The figure draws levels 0..2 (edges 0->1, 0->2, 0->3 | 1->4, 1->5, 2->4,
    2->6, 3->7) and the last three levels (N-7->N-3, N-6->N-3, N-6->N-2,
    N-5->N-1, N-4->N-1 | N-3->N, N-2->N, N-1->N).  Identifying level 2 with
    level L-2 (nodes 4..7 = N-7..N-4) gives a 5-level graph with 12 nodes,
    numbered 0..11 here (the figure's N is node 11).  All edges use kind 0 and
    time indices (0, 0); callers replace those columns as needed.
    """
    pairs = [(0, 1), (0, 2), (0, 3),
             (1, 4), (1, 5), (2, 4), (2, 6), (3, 7),
             (4, 8), (5, 8), (5, 9), (6, 10), (7, 10),
             (8, 11), (9, 11), (10, 11)]
    edges = np.array([[s, d, 0, 0, 0] for s, d in pairs], dtype=np.int32)
    return Graph(np.array([1, 3, 4, 3, 1], dtype=np.int64), np.array([0, 3, 5, 5, 3], dtype=np.int64),
                 edges, 1, 1)


WORKLOADS: Dict[str, Callable[..., Workload]] = {"tiny": tiny, "medium": medium, "large": large}


# ---------------------------------------------------------------------------- counter-based times

_PHILOX_M0, _PHILOX_M1 = 0xD2511F53, 0xCD9E8D57
_PHILOX_W0, _PHILOX_W1 = 0x9E3779B9, 0xBB67AE85


def philox4x32_10(c0, c1, c2, c3, k0, k1):
    """Philox-4x32 with 10 rounds (Salmon, Moraes, Dror, Shaw, SC'11), vectorised over
    numpy uint32 arrays: each round multiplies two words by the round constants,
    mixes the high halves with the other words and the key, and bumps the key by the
    Weyl constants between rounds."""
    c0, c1, c2, c3 = (np.asarray(x, dtype=np.uint64) & 0xFFFFFFFF for x in (c0, c1, c2, c3))
    k0 = np.uint64(k0 & 0xFFFFFFFF)
    k1 = np.uint64(k1 & 0xFFFFFFFF)
    mask = np.uint64(0xFFFFFFFF)
    for r in range(10):
        if r:
            k0 = (k0 + np.uint64(_PHILOX_W0)) & mask
            k1 = (k1 + np.uint64(_PHILOX_W1)) & mask
        p0 = np.uint64(_PHILOX_M0) * c0
        p1 = np.uint64(_PHILOX_M1) * c2
        hi0, lo0 = p0 >> np.uint64(32), p0 & mask
        hi1, lo1 = p1 >> np.uint64(32), p1 & mask
        c0, c1, c2, c3 = (hi1 ^ c1 ^ k0) & mask, lo1, (hi0 ^ c3 ^ k1) & mask, lo0
    return c0, c1, c2, c3


def counter_times(seed: int, first_sample: int, num_samples: int, num_times: int, beta: float) -> np.ndarray:
    """Times t[s][i] ~ U[0, beta) from a counter-based generator: for sample index
    n = first_sample + s and pair m = i // 2, Philox-4x32-10 with counter
    (n mod 2^32, n >> 32, m, 0) and key (seed mod 2^32, seed >> 32) gives words w0..w3;
    t[s][2m] = beta * ((w1 << 32 | w0) >> 11) * 2^-53 and t[s][2m+1] likewise from
    (w3, w2).  Returns [S, D] float64."""
    S, D = int(num_samples), int(num_times)
    out = np.empty((S, D), dtype=np.float64)
    if S == 0:
        return out
    n = np.arange(first_sample, first_sample + S, dtype=np.uint64)
    lo, hi = n & np.uint64(0xFFFFFFFF), n >> np.uint64(32)
    for m in range((D + 1) // 2):
        w0, w1, w2, w3 = philox4x32_10(lo, hi, np.full(S, m, np.uint64), np.zeros(S, np.uint64),
                                       seed & 0xFFFFFFFF, (seed >> 32) & 0xFFFFFFFF)
        a = ((w1 << np.uint64(32)) | w0) >> np.uint64(11)
        b = ((w3 << np.uint64(32)) | w2) >> np.uint64(11)
        out[:, 2 * m] = beta * (a.astype(np.float64) * 2.0 ** -53)
        if 2 * m + 1 < D:
            out[:, 2 * m + 1] = beta * (b.astype(np.float64) * 2.0 ** -53)
    return out

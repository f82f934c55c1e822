"""Seeded synthetic inputs for the combinatorial-summation (CoS) graph evaluator.

This package draws random leveled digraphs and Monte Carlo samples. It holds
none of the method's arithmetic (no propagator, no path sums): it only produces
the integer edge lists and the real-valued inputs that both the CPU oracle and
the GPU path consume.
"""
from .generate import (  # noqa: F401
    Graph, Samples, Workload, FaninSpec, make_graph, make_eps, make_times,
    tiny, medium, large, batched, serving_pool, complete_layered_graph,
    chain_graph, figure_graph, geometric_widths, widths_for_target,
    WORKLOADS, philox4x32_10, counter_times,
)

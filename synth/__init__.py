"""Seeded synthetic RDF graphs and BGP workloads.

This package is shared input infrastructure: it generates int32 (s, p, o)
triple sets and basic graph patterns (BGPs) for the tests, the benchmark and
the oracle's own pins.  It performs none of the join method's arithmetic: it
draws random numbers, samples concrete subgraph instances with numpy lookups
and bounds result sizes with walk counts so that workloads stay within the
sizes a configuration promises.

Graph shape facts follow the paper's description of its datasets only
(degree sparsity of real RDF graphs in Sec. 1, dataset scales in the
dataset-statistics table of Sec. 8); no item of any public benchmark is
reproduced.
"""

from .graphs import CONFIGS, GraphConfig, make_graph, graph_stats, small_random_graph
from .queries import (BGP, bgp_row_bound, make_batched_queries, make_large_queries, make_large_served_queries,
                      make_queries)

__all__ = [
    "CONFIGS",
    "GraphConfig",
    "make_graph",
    "graph_stats",
    "small_random_graph",
    "BGP",
    "make_queries",
    "make_batched_queries",
    "make_large_queries",
    "make_large_served_queries",
    "bgp_row_bound",
]

"""Seeded synthetic graph workloads shared by the tests, the oracle checks and the bench.

This package only builds inputs: CSR arrays of undirected weighted graphs and
their planted labels.  It holds none of the clustering method's arithmetic (no
degrees, no operator, no power iteration, no k-means), so both the CPU oracle
and the CUDA path can consume its output without sharing method code.
"""
from .graphs import (
    Graph,
    sbm,
    sbm_by_degree,
    disjoint_cliques,
    cycle,
    complete,
    knn_mixture,
    mixture_points,
    image_grid,
    from_edges,
    with_isolated,
    permuted,
    equal_sizes,
    GraphBatch,
    union,
    sbm_batch,
    sbm_batch_gpu,
)

__all__ = [
    "Graph",
    "sbm",
    "sbm_by_degree",
    "disjoint_cliques",
    "cycle",
    "complete",
    "knn_mixture",
    "mixture_points",
    "image_grid",
    "from_edges",
    "with_isolated",
    "permuted",
    "equal_sizes",
    "GraphBatch",
    "union",
    "sbm_batch",
    "sbm_batch_gpu",
]

"""Seeded synthetic inputs shared by the CUDA path's tests/bench and the CPU oracle.

This package only *creates inputs*: simple undirected graphs in CSR form with the
shapes of the paper's workloads (heavy-tailed "complex networks" and sparse,
near-planar "road networks", Sec. 6, Table 1).  It holds none of the forest
closeness arithmetic (no Laplacian, no augmented graph, no sampling, no solve),
so that the oracle and the GPU path can both read the same graphs without
sharing any of the method's code.
"""
from .graphs import (  # noqa: F401
    Graph,
    from_edges,
    erdos_renyi,
    barabasi_albert,
    perturbed_grid,
    torus,
    rmat,
    complete,
    path,
    cycle,
    star,
    empty,
    random_small,
    uneven_batch,
    union,
)

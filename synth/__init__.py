"""Seeded synthetic graph generators shared by the tests, the oracle checks and
the benchmark.

This module holds no arithmetic of the method itself: it only builds
connected undirected graphs in CSR form (and uniform input vectors), with the
shapes of the workloads the paper evaluates on (Section 6, Table 1: sparse
social and web graphs with power-law degrees, diameters 8-24) plus the
high-diameter and geometric cases used to stress the sampler.

Every graph is returned as a :class:`Graph` with int64 ``row_ptr`` (n+1),
int32 ``col`` (nnz), optional float32 ``w`` (nnz, ``None`` = unit weights),
rows sorted by neighbour id, both arc directions present with equal weight,
no self-loops and no duplicate arcs.
"""
from .graphs import (Graph, from_edges, ba, grid2d, rmat, rgg, er, add_path,
                     star, path, cycle, complete, lognormal_weights,
                     batch_specs, batch_graph, uniform_vector)

__all__ = ["Graph", "from_edges", "ba", "grid2d", "rmat", "rgg", "er",
           "add_path", "star", "path", "cycle", "complete",
           "lognormal_weights", "batch_specs", "batch_graph", "uniform_vector"]

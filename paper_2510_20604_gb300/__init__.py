"""GB300 FastWalk: random walk centrality by sampling rooted spanning trees.

Thin Python binding of the C ABI declared in ``include/rwc.h`` (same function
names, argument marshalling only); every step of the computation runs in the
CUDA library ``librwc.so``.  Importing this package does not load the
library; the first call does, and raises :class:`RWCError` if it has not been
built (``python -c "import __graft_entry__ as g; g.build()"``).

Device buffers are passed as torch CUDA tensors (or raw integer pointers);
host buffers (graph CSR) as numpy arrays.
"""
from ._binding import (RWCError, Options, Stats, GraphInfo, lib, lib_path,
                       rwc_version, rwc_launch_count, rwc_last_error, rwc_graph_create, rwc_graph_info,
                       rwc_graph_destroy, rwc_sample_trees, rwc_sample_trees_noalloc, rwc_sync_status, rwc_pivot_solve,
                       rwc_estimate, rwc_recover,
                       rwc_solve, rwc_grad, rwc_batch_create, rwc_batch_sample,
                       rwc_batch_roots, rwc_autotune, rwc_batch_get_schedule, rwc_batch_set_schedule, rwc_batch_destroy, rwc_mre, rwc_kendall, rwc_auto_params, Params, rwc_trap_walks, rwc_predict_mre,
                       MODE_AUTO, MODE_GLOBAL, MODE_SHARED, MODE_WALKER, GRAPH_INT64_OFFSETS,
                       GRAPH_SKIP_CONNECTIVITY)
from .api import Graph, Batch, RWCFunction, fastwalk, fastwalk_auto, fastwalk_to_target

__all__ = [
    "RWCError", "Options", "Stats", "GraphInfo", "lib", "lib_path", "rwc_version",
    "rwc_launch_count",
    "rwc_last_error", "rwc_graph_create", "rwc_graph_info", "rwc_graph_destroy",
    "rwc_sample_trees", "rwc_sample_trees_noalloc", "rwc_sync_status", "rwc_pivot_solve", "rwc_estimate", "rwc_recover", "rwc_solve", "rwc_grad",
    "rwc_batch_create", "rwc_batch_sample", "rwc_batch_roots", "rwc_autotune",
    "rwc_batch_get_schedule", "rwc_batch_set_schedule",
    "rwc_batch_destroy", "rwc_mre", "rwc_kendall", "rwc_auto_params", "Params", "rwc_trap_walks", "rwc_predict_mre", "MODE_AUTO", "MODE_GLOBAL", "MODE_SHARED", "MODE_WALKER",
    "GRAPH_INT64_OFFSETS", "GRAPH_SKIP_CONNECTIVITY", "Graph", "Batch", "RWCFunction",
    "fastwalk", "fastwalk_auto", "fastwalk_to_target",
]

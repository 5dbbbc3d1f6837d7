"""Host-side logic of the Python layer (no GPU): the arc -> undirected edge
map that RWCFunction uses to spread per-edge weights onto both arcs."""
import numpy as np
import pytest

import synth
from _graphs import multigraph
from paper_2510_20604_gb300.api import _edge_index


def _check_pairing(g):
    eid = _edge_index(g.row_ptr, g.col)
    src = g.src()
    up = src < g.col
    m = int(up.sum())
    assert sorted(eid[up].tolist()) == list(range(m))
    assert (eid >= 0).all() and (eid < m).all()
    # every edge id is used by exactly one arc in each direction
    assert np.array_equal(np.bincount(eid[up], minlength=m), np.ones(m, int))
    assert np.array_equal(np.bincount(eid[~up], minlength=m), np.ones(m, int))
    # both arcs of an edge join the same two vertices
    a = np.empty(m, np.int64); b = np.empty(m, np.int64)
    a[eid[up]], b[eid[up]] = src[up], g.col[up]
    assert np.array_equal(a[eid[~up]], g.col[~up]) and np.array_equal(b[eid[~up]], src[~up])
    return eid


@pytest.mark.parametrize("weighted", [False, True])
def test_edge_index_pairs_parallel_arcs_in_order(weighted):
    g = multigraph(weighted)
    eid = _check_pairing(g)
    # distinct weights per edge land on both arcs of that edge: arc weights
    # built from per-edge weights are symmetric copy by copy
    m = int((g.src() < g.col).sum())
    w_edge = np.arange(1, m + 1, dtype=np.float64)
    warc = w_edge[eid]
    src = g.src()
    for u in range(g.n):
        for v in set(g.col[g.row_ptr[u]:g.row_ptr[u + 1]].tolist()):
            fwd = warc[g.row_ptr[u]:g.row_ptr[u + 1]][g.col[g.row_ptr[u]:g.row_ptr[u + 1]] == v]
            bwd = warc[g.row_ptr[v]:g.row_ptr[v + 1]][g.col[g.row_ptr[v]:g.row_ptr[v + 1]] == u]
            assert sorted(fwd.tolist()) == sorted(bwd.tolist())
    assert len(src) == len(eid)


def test_edge_index_simple_graphs():
    for g in (synth.grid2d(5, 7), synth.ba(300, 3, seed=1), synth.path(2)):
        _check_pairing(g)


def test_edge_index_rejects_unpaired_arcs():
    rp = np.array([0, 1, 1], np.int64)
    col = np.array([1], np.int32)
    with pytest.raises(ValueError):
        _edge_index(rp, col)

"""The allocation-free sampling entry point (rwc_sample_trees_noalloc).

Callers that cannot allocate device memory while sampling (hosts that forbid
allocation after start-up, exhausted device memory pools, or pools owned by an
allocator the library cannot draw from) use this entry point; it keeps its
scratch in a static device array of the library.  These tests call it through the C ABI twice in a row
and compare with rwc_sample_trees.  The file is named so that pytest collects
it last; it also passes when run alone in a fresh process.
"""
import numpy as np
import pytest
import torch

import paper_2510_20604_gb300 as rwc
import synth

pytestmark = pytest.mark.gpu


def _outputs(G, T):
    dev = torch.device("cuda")
    return (torch.zeros(G.n, dtype=torch.float64, device=dev),
            torch.empty((T, G.n), dtype=torch.int32, device=dev),
            torch.empty((T, G.n), dtype=torch.int32, device=dev))


@pytest.mark.parametrize("gname", ["grid", "ba", "weighted_rmat"])
def test_noalloc_matches_regular_entry_point_twice(gname):
    g = {"grid": lambda: synth.grid2d(120, 130),
         "ba": lambda: synth.ba(3000, 3, seed=4),
         "weighted_rmat": lambda: synth.rmat(16, 16, seed=2, sigma=1.0)}[gname]()
    G = rwc.Graph.from_synth(g)
    T = 40
    s_ref, p_ref, v_ref = _outputs(G, T)
    rwc.rwc_sample_trees(G.handle, 7, 11, T, s_ref, p_ref, v_ref)
    for _ in range(2):  # the static array keeps the previous call's contents
        s, p, v = _outputs(G, T)
        rwc.rwc_sample_trees_noalloc(G.handle, 7, 11, T, s, p, v)
        torch.cuda.synchronize()
        assert torch.equal(s, s_ref)
        assert torch.equal(p, p_ref)
        assert torch.equal(v, v_ref)


def test_noalloc_many_chunks_and_sums_only():
    # 262k-vertex grid: one tree takes about 3 MiB of the 32 MiB array, so 30
    # trees run in several chunks
    g = synth.grid2d(512, 512)
    G = rwc.Graph.from_synth(g)
    T = 30
    ref = torch.zeros(G.n, dtype=torch.float64, device="cuda")
    rwc.rwc_sample_trees(G.handle, 3, 0, T, ref)
    got = torch.zeros_like(ref)
    rwc.rwc_sample_trees_noalloc(G.handle, 3, 0, T, got)
    assert torch.equal(got, ref)


def test_noalloc_rejects_graph_beyond_the_static_array():
    g = synth.grid2d(1500, 1500)
    G = rwc.Graph.from_synth(g)
    s = torch.zeros(G.n, dtype=torch.float64, device="cuda")
    with pytest.raises(rwc.RWCError) as e:
        rwc.rwc_sample_trees_noalloc(G.handle, 1, 0, 1, s)
    assert e.value.status == 1
    assert "too large" in str(e.value)

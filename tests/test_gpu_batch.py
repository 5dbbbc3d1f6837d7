"""GPU parity of the batched sampler: every graph's sums equal the oracle's
(graph g uses Philox counter word 3 = g); the persistent launch, its CUDA
graph replay and the one-launch-per-graph baseline agree exactly."""
import numpy as np
import pytest
import torch

import paper_2510_20604_gb300 as rwc
import synth
from oracle import wilson as ow

pytestmark = pytest.mark.gpu


def _graphs(G=24, seed=5, nmax=3000):
    specs = synth.batch_specs(G, seed=seed, nmin=50, nmax=nmax)
    return [synth.batch_graph(i, n, kind, seed=seed) for i, (n, kind) in enumerate(specs)]


def test_batch_matches_oracle_and_modes_agree():
    gs = _graphs()
    B = rwc.Batch(gs)
    T = 12
    s_graph, st = B.sample(T, seed=3, use_graph=1)
    s_plain, _ = B.sample(T, seed=3, use_graph=0)
    s_base, _ = B.sample(T, seed=3, per_graph_launch=1)
    s_again, _ = B.sample(T, seed=3, use_graph=1)   # graph replay
    assert torch.equal(s_graph, s_plain) and torch.equal(s_graph, s_base) and torch.equal(s_graph, s_again)
    roots = B.roots()
    sums = s_graph.cpu().numpy()
    for i, g in enumerate(gs):
        ref = ow.Sampler(g, root=int(roots[i]), seed=3, graph_id=i).sample(0, T)
        assert int(roots[i]) == ow.max_degree_root(g)
        o = B.offsets
        assert np.array_equal(sums[o[i]:o[i + 1]], ref["sums"]), i
    assert st.trees == T * len(gs)


@pytest.mark.parametrize("sched", [(512, 0, 4, 1, 1), (512, 1024, 4, 1, 1), (256, 1024, 2, 0, 1),
                                   (256, 2500, 1, 1, 0), (128, 600, 16, 1, 0)])
def test_batch_schedules_match_oracle(sched):
    """One class block-per-tree; small graphs warp-per-tree; small graphs
    block-per-tree in small blocks; almost every graph warp-per-tree; a
    narrow large-class block with 16 trees per item: each schedule (two
    persistent kernels on forked streams when both classes are present)
    gives every member exactly the oracle's sums."""
    gs = _graphs(G=20, seed=13, nmax=3000)
    B = rwc.Batch(gs)
    B.set_schedule(*sched)
    assert B.schedule() == sched
    T = 9
    s, st = B.sample(T, seed=2, use_graph=1)
    assert st.block_threads == sched[0]
    sums = s.cpu().numpy()
    roots = B.roots()
    o = B.offsets
    for i, g in enumerate(gs):
        ref = ow.Sampler(g, root=int(roots[i]), seed=2, graph_id=i).sample(0, T)
        assert np.array_equal(sums[o[i]:o[i + 1]], ref["sums"]), (sched, i)


def test_batch_schedule_rejects_oversized_slices():
    gs = _graphs(G=6, seed=3, nmax=20000)
    B = rwc.Batch(gs)
    with pytest.raises(rwc.RWCError) as e:
        B.set_schedule(512, 20000, 1, 1, 1)    # 8 warps x 11 n bytes of shared memory
    assert e.value.status in (1, 6)
    with pytest.raises(rwc.RWCError):
        B.set_schedule(100, 0, 1, 0, 1)        # not a multiple of 32


def test_batch_autotune_and_large_graphs():
    gs = _graphs(G=10, seed=9, nmax=20000)
    B = rwc.Batch(gs)
    B.autotune(None)
    th, split, tile, warp, conc = B.schedule()
    assert th % 32 == 0 and tile >= 1 and split in (0, 512, 1024, 2048, 4096) and warp in (0, 1)
    assert conc in (0, 1)
    T = 5
    s, _ = B.sample(T, seed=1)
    sums = s.cpu().numpy()
    roots = B.roots()
    for i in (0, len(gs) - 1):
        ref = ow.Sampler(gs[i], root=int(roots[i]), seed=1, graph_id=i).sample(0, T)
        o = B.offsets
        assert np.array_equal(sums[o[i]:o[i + 1]], ref["sums"]), i


def test_batch_rejects_disconnected_member():
    gs = _graphs(G=3)
    bad = synth.from_edges(6, [0, 1, 3, 4], [1, 2, 4, 5])
    with pytest.raises(rwc.RWCError) as e:
        rwc.Batch(gs + [bad])
    assert e.value.status == 2


def test_weighted_batch_matches_oracle():
    """Members with lognormal edge weights (alias tables per graph): every
    graph's sums equal the oracle's."""
    gs = []
    for i, g in enumerate(_graphs(G=9, seed=11, nmax=2500)):
        a, b, _ = g.undirected()
        w = np.random.default_rng(100 + i).lognormal(0.0, 0.8, len(a)).astype(np.float32)
        gs.append(synth.from_edges(g.n, a, b, w))
    B = rwc.Batch(gs)
    T = 10
    s, _ = B.sample(T, seed=4)
    sums = s.cpu().numpy()
    roots = B.roots()
    for i, g in enumerate(gs):
        ref = ow.Sampler(g, root=int(roots[i]), seed=4, graph_id=i).sample(0, T)
        o = B.offsets
        assert np.array_equal(sums[o[i]:o[i + 1]], ref["sums"]), i

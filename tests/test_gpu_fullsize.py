"""Parity at the full sizes of the remaining workloads, on sampled outputs the
oracle can compute: R-MAT scale 24 with lognormal weights and int64 arc
offsets (sampled trees, bit-exact), the 1e5-node random geometric graph's
sketched gradient (sampled edges against the oracle's sparse route with the
same Philox sketch), and the 4096-graph batch (sampled graphs' sums)."""
import numpy as np
import pytest
import torch

import paper_2510_20604_gb300 as rwc
import synth
from oracle import grad as og
from oracle import wilson as ow

pytestmark = pytest.mark.gpu


def test_rmat24_weighted_sampled_trees_bit_exact():
    g = synth.rmat(24, 16, seed=0, sigma=1.0)
    G = rwc.Graph.from_synth(g, flags=rwc.GRAPH_INT64_OFFSETS)
    assert G.info.offsets64 == 1 and G.info.weighted == 1
    T, tree0 = 2, 250
    _, st, par, vis = G.sample(T, seed=1, tree0=tree0, want_trees=True)
    ref = ow.Sampler(g, root=G.root, seed=1).sample(tree0, T, want_trees=True, nthreads=T)
    assert np.array_equal(par.cpu().numpy(), ref["parents"])
    assert np.array_equal(vis.cpu().numpy(), ref["visits"])


def test_rgg100k_sketched_gradient_sampled_edges():
    g = synth.rgg(100_000, 12.0, seed=0, sigma=0.5)
    G = rwc.Graph.from_synth(g)
    c = synth.uniform_vector(g.n, 1)
    k, seed = 64, 77
    gg = G.grad(torch.tensor(c, dtype=torch.float64, device="cuda"), k=k, sketch_seed=seed,
                tol=1e-8).double().cpu().numpy()
    a, b, w = g.undirected()
    w = w.astype(np.float64)
    Q = ow.rademacher(k, g.n, seed)
    sel = np.sort(np.random.default_rng(0).choice(len(a), 300, replace=False))
    ref = og.grad_sketch_sparse(g.n, a.astype(np.int64), b.astype(np.int64), w, c, Q, sel)
    scale = np.abs(ref).max()
    assert np.max(np.abs(gg[sel] - ref)) <= 1e-4 * scale


def test_batch4096_sampled_graphs():
    specs = synth.batch_specs(4096, seed=0)
    gs = [synth.batch_graph(i, n, kind, seed=0) for i, (n, kind) in enumerate(specs)]
    B = rwc.Batch(gs)
    T = 256
    s, st = B.sample(T, seed=1)
    sums = s.cpu().numpy()
    roots = B.roots()
    o = B.offsets
    pick = [0, 1, 2, 4095] + list(np.random.default_rng(0).choice(4096, 4, replace=False))
    for i in pick:
        ref = ow.Sampler(gs[i], root=int(roots[i]), seed=1, graph_id=int(i)).sample(0, T, nthreads=8)
        assert np.array_equal(sums[o[i]:o[i + 1]], ref["sums"]), i
    assert st.trees == T * 4096

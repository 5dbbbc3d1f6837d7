"""Pins for the oracle's sequential Wilson sampler (Algorithm 3's loop).

Nothing here compares the oracle with itself: every check is against a fact
fixed by the mathematics -- spanning-tree structure, the spanning-tree law by
full enumeration (matrix-tree theorem), Kirchhoff's edge marginals w_e R_e,
Lemma 5.2 (E[visits_u] = (NL_v^-1)_uu) with the geometric variance
t_u (t_u - 1), closed-form special cases, independence of the start order
(Wilson's cycle-popping theorem), and exactness of sharded sums.
"""
import itertools
import math

import numpy as np
import pytest
from scipy import stats

import synth
from oracle import exact
from oracle import wilson as ow


def check_tree(g, root, parent):
    n = g.n
    assert parent[root] == -1
    rp, col = g.row_ptr, g.col
    for u in range(n):
        if u == root:
            continue
        p = parent[u]
        assert 0 <= p < n
        assert p in col[rp[u]:rp[u + 1]], (u, p)
    # acyclic and reaches root: depth by memoised walk
    depth = np.full(n, -1)
    depth[root] = 0
    for u in range(n):
        chain = []
        x = u
        while depth[x] < 0:
            chain.append(x)
            x = parent[x]
            assert len(chain) <= n
        for y in reversed(chain):
            depth[y] = depth[parent[y]] + 1


def small_weighted(seed=0, n=7, extra=4):
    rng = np.random.default_rng(seed)
    u = list(range(n - 1)); v = list(range(1, n))
    while len(u) < n - 1 + extra:
        a, b = rng.integers(0, n, 2)
        if a != b:
            u.append(int(a)); v.append(int(b))
    w = rng.lognormal(0, 0.7, size=len(u)).astype(np.float32)
    return synth.from_edges(n, u, v, w)


@pytest.mark.parametrize("gname", ["ba", "grid", "weighted"])
def test_trees_are_spanning_trees_and_counts_are_departures(gname):
    g = {"ba": lambda: synth.ba(300, 3, seed=2),
         "grid": lambda: synth.grid2d(9, 11),
         "weighted": lambda: synth.rgg(200, 8.0, seed=3, sigma=0.5)}[gname]()
    s = ow.Sampler(g, seed=11)
    out = s.sample(0, 20, want_trees=True)
    for t in range(20):
        check_tree(g, s.root, out["parents"][t])
    # Algorithm 3's count (+1 start, +1 per arrival, -1 at the endpoint)
    # equals the number of RandomNeighbor calls at each node
    order = np.array([u for u in range(g.n) if u != s.root], np.int32)
    par, vis, calls, d = s.tree_with_order(5, order)
    assert (vis.astype(np.int64) == calls.astype(np.int64)).all()
    assert d == int(calls.sum())
    assert (par == out["parents"][5]).all()
    assert (vis == out["visits"][5]).all()
    assert vis[s.root] == 0
    assert (vis[np.arange(g.n) != s.root] >= 1).all()
    assert np.array_equal(out["sums"], out["visits"].sum(0).astype(np.float64))


@pytest.mark.parametrize("gname", ["ba", "weighted", "grid"])
def test_result_independent_of_start_order(gname):
    """Wilson (1996): with per-vertex successor stacks, the tree and the
    number of stack entries used at each vertex do not depend on the order in
    which start nodes are processed."""
    g = {"ba": lambda: synth.ba(200, 3, seed=5),
         "weighted": lambda: small_weighted(4, n=40, extra=60),
         "grid": lambda: synth.grid2d(8, 8)}[gname]()
    s = ow.Sampler(g, seed=99)
    base = np.array([u for u in range(g.n) if u != s.root], np.int32)
    rng = np.random.default_rng(1)
    for tree in range(5):
        p0, v0, c0, _ = s.tree_with_order(tree, base)
        for _ in range(3):
            p1, v1, c1, _ = s.tree_with_order(tree, rng.permutation(base))
            assert (p0 == p1).all() and (v0 == v1).all() and (c0 == c1).all()


def test_star_rooted_at_centre_is_deterministic():
    g = synth.star(50, center=0)
    s = ow.Sampler(g, seed=5)
    assert s.root == 0
    out = s.sample(0, 10, want_trees=True)
    assert (out["parents"][:, 1:] == 0).all()
    assert (out["visits"][:, 1:] == 1).all()


def _enumerate_trees(g):
    a, b, w = g.undirected()
    m = len(a)
    w = np.ones(m) if w is None else w.astype(np.float64)
    trees = {}
    for comb in itertools.combinations(range(m), g.n - 1):
        par = list(range(g.n))

        def find(x):
            while par[x] != x:
                par[x] = par[par[x]]
                x = par[x]
            return x
        ok = True
        for e in comb:
            ra, rb = find(int(a[e])), find(int(b[e]))
            if ra == rb:
                ok = False
                break
            par[ra] = rb
        if ok:
            key = frozenset((min(int(a[e]), int(b[e])), max(int(a[e]), int(b[e]))) for e in comb)
            trees[key] = float(np.prod(w[list(comb)]))
    return trees


@pytest.mark.parametrize("gname", ["C4", "K4", "grid2x3", "weighted6"])
def test_spanning_tree_law_by_enumeration(gname):
    g = {"C4": lambda: synth.cycle(4), "K4": lambda: synth.complete(4),
         "grid2x3": lambda: synth.grid2d(2, 3),
         "weighted6": lambda: small_weighted(2, n=6, extra=3)}[gname]()
    trees = _enumerate_trees(g)
    keys = list(trees)
    # matrix-tree theorem: total weight = any cofactor of L
    L, _ = exact.laplacian(g)
    assert math.isclose(sum(trees.values()), np.linalg.det(L[1:, 1:]), rel_tol=1e-9)
    s = ow.Sampler(g, seed=2024)
    T = 20000
    out = s.sample(0, T, want_trees=True)
    idx = {k: i for i, k in enumerate(keys)}
    cnt = np.zeros(len(keys))
    for t in range(T):
        par = out["parents"][t]
        key = frozenset((min(u, int(par[u])), max(u, int(par[u])))
                        for u in range(g.n) if u != s.root)
        cnt[idx[key]] += 1
    p = np.array([trees[k] for k in keys])
    p /= p.sum()
    chi2 = ((cnt - T * p) ** 2 / (T * p)).sum()
    assert stats.chi2.sf(chi2, len(keys) - 1) > 1e-4, (chi2, len(keys))


def test_edge_marginals_are_weight_times_resistance():
    """Kirchhoff: P(e in T) = w_e R_e for the weighted uniform spanning tree."""
    g = small_weighted(8, n=12, extra=14)
    s = ow.Sampler(g, seed=31)
    T = 20000
    out = s.sample(0, T, want_trees=True)
    a, b, w = g.undirected()
    L, _ = exact.laplacian(g)
    P = exact.pinv_closed_form(L)
    for e in range(len(a)):
        u, v = int(a[e]), int(b[e])
        R = P[u, u] + P[v, v] - 2 * P[u, v]
        pe = float(w[e]) * R
        par = out["parents"]
        hits = ((par[:, u] == v) | (par[:, v] == u)).sum()
        se = math.sqrt(pe * (1 - pe) / T) + 1e-12
        assert abs(hits / T - pe) < 5 * se, (e, hits / T, pe)


@pytest.mark.parametrize("gname", ["ba", "weighted", "path"])
def test_expected_visits_equal_pivot_deleted_diagonal(gname):
    """Lemma 5.2: E[visits_u] = (NL_v^-1)_uu; visits_u is geometric, so
    Var = t_u (t_u - 1)."""
    g = {"ba": lambda: synth.ba(60, 3, seed=9),
         "weighted": lambda: small_weighted(3, n=30, extra=40),
         "path": lambda: synth.path(12)}[gname]()
    root = 0 if gname == "path" else None
    s = ow.Sampler(g, root=root, seed=77)
    T = 20000
    out = s.sample(0, T, want_trees=True)
    t = exact.tdiag(g, s.root)
    mean = out["sums"] / T
    vis = out["visits"].astype(np.float64)
    for u in range(g.n):
        if u == s.root:
            continue
        sd = math.sqrt(max(t[u] * (t[u] - 1), 1e-12) / T)
        assert abs(mean[u] - t[u]) < 5 * sd + 1e-9, (u, mean[u], t[u])
        var = vis[:, u].var()
        assert abs(var - t[u] * (t[u] - 1)) < 0.1 * t[u] * t[u] + 0.02, (u, var, t[u])
    if gname == "path":
        # path 0..L rooted at 0: t_u = 2u inside, L at the far end
        Lh = g.n - 1
        ref = np.array([0] + [2 * u for u in range(1, Lh)] + [Lh], np.float64)
        assert np.allclose(t, ref, atol=1e-9)


def test_threads_and_shards_give_identical_sums():
    g = synth.ba(500, 3, seed=1)
    s = ow.Sampler(g, seed=4)
    a = s.sample(0, 64, nthreads=1)
    b = s.sample(0, 64, nthreads=4)
    c1 = s.sample(0, 20, nthreads=2)
    c2 = s.sample(20, 44, nthreads=3)
    assert np.array_equal(a["sums"], b["sums"])
    assert np.array_equal(a["sums"], c1["sums"] + c2["sums"])
    assert a["draws"] == b["draws"] == c1["draws"] + c2["draws"]
    assert a["draws"] == int(a["sums"].sum())

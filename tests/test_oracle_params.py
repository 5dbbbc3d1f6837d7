"""Pins of the automatic parameters (Section 5): the spectral radius of P_v
against closed forms, the double-sweep diameter against all-pairs BFS, and
the sample-size and solver-accuracy formulas on hand-evaluated instances."""
import math

import numpy as np
import pytest

import synth
from oracle import params as op


@pytest.mark.parametrize("n", [3, 4, 7, 12])
def test_lambda_complete_graph(n):
    # P_v on K_n minus v: (J - I) / (n - 1) on n - 1 vertices; Perron root (n-2)/(n-1)
    assert op.spectral_radius_pv(synth.complete(n), 0) == pytest.approx((n - 2) / (n - 1), abs=1e-13)


@pytest.mark.parametrize("n", [3, 5, 10, 33])
def test_lambda_cycle(n):
    # C_n minus v is a path of n-1 vertices whose ends both step into v with
    # probability 1/2: P_v = tridiag(1/2, 0, 1/2), spectral radius cos(pi/n)
    assert op.spectral_radius_pv(synth.cycle(n), 3 % n) == pytest.approx(math.cos(math.pi / n), abs=1e-13)


def test_lambda_star_centre_and_leaf():
    g = synth.star(20, center=0)
    assert op.spectral_radius_pv(g, 0) == pytest.approx(0.0, abs=1e-15)
    # rooted at a leaf: the rest is a star of 18 leaves around the centre,
    # whose centre steps back to a leaf with probability 18/19 (radius sqrt(18/19))
    assert op.spectral_radius_pv(g, 5) == pytest.approx(math.sqrt(18 / 19), abs=1e-13)


def _diameter(g):
    return max(int(op.bfs_dist(g, s).max()) for s in range(g.n))


@pytest.mark.parametrize("gname", ["path", "grid", "tree", "ba", "cycle"])
def test_double_sweep(gname):
    g = {"path": lambda: synth.path(40),
         "grid": lambda: synth.grid2d(7, 11),
         "tree": lambda: synth.star(15, center=4),
         "ba": lambda: synth.ba(300, 2, seed=1),
         "cycle": lambda: synth.cycle(21)}[gname]()
    a, delta = op.double_sweep(g, 0)
    assert op.bfs_dist(g, 0)[a] == op.bfs_dist(g, 0).max()
    if gname in ("path", "grid", "tree", "cycle"):
        assert delta == _diameter(g)
    else:
        assert delta <= _diameter(g)
    if gname == "grid":
        assert delta == 7 + 11 - 2


def test_formulas_hand_evaluated():
    # K_4 rooted at 0: n = 4, m = 6, d = 3, ||d_-v|| = sqrt(27), lambda = 2/3
    t = op.walk_bound(4, 6.0, math.sqrt(27.0), 2.0 / 3.0)
    assert t == pytest.approx(math.log(1.0 / 6.0) / math.log(2.0 / 3.0), rel=1e-15)
    assert op.tree_count(0.1, 4, t) == math.ceil(200.0 * t * t * math.log(8.0))
    # theta for n = 4, m = 6, dmax = 3, Delta = 1: eps / (2 * 3 * (1 + 15/12)^2 * sqrt(24))
    assert op.solver_theta(0.1, 4, 6.0, 3.0, 1) == pytest.approx(0.1 / (6.0 * 2.25 ** 2 * math.sqrt(24.0)), rel=1e-15)
    assert op.walk_bound(5, 4.0, 2.0, 0.0) == 1.0
    p = op.auto_params(synth.complete(4), 0, 0.1)
    assert p["diameter"] == 1 and p["lambda"] == pytest.approx(2 / 3, abs=1e-13)
    assert p["trees"] == op.tree_count(0.1, 4, p["t"])


def test_lambda_of_parallel_arcs_is_that_of_summed_weights():
    """Parallel arcs act as one edge of summed weight: the multigraph's
    spectral radius equals that of the simple graph with merged weights."""
    from _graphs import multigraph
    for weighted in (False, True):
        g = multigraph(weighted)
        a, b, w = g.undirected()
        w = np.ones(len(a)) if w is None else w.astype(np.float64)
        key = a * g.n + b
        uk, inv = np.unique(key, return_inverse=True)
        ws = np.zeros(len(uk))
        np.add.at(ws, inv, w)
        simple = synth.from_edges(g.n, uk // g.n, uk % g.n, ws.astype(np.float32))
        lam_m = op.spectral_radius_pv(g, 0)
        lam_s = op.spectral_radius_pv(simple, 0)
        assert lam_m == pytest.approx(lam_s, rel=1e-6)


def _trapped_star(w_light=1e-4):
    """Star with centre 0 and ten unit-weight leaves, plus one light edge
    between leaves 1 and 2: a walk from any leaf reaches the centre (the
    pivot) at its first step with probability at least 1 / (1 + w_light)."""
    import synth
    u = [0] * 10 + [1]
    v = list(range(1, 11)) + [2]
    w = np.array([1.0] * 10 + [w_light], np.float32)
    return synth.from_edges(11, u, v, w)


def test_walk_bound_is_one_step_when_walks_are_trapped_at_once():
    """The walk-length bound counts steps: when every walk is trapped at its
    first step but for a fraction below 1/n, one step suffices, although the
    printed formula's value is below one (here about 0.26).  lambda is pinned
    by its closed form: P_v keeps only the two light arcs, each of
    probability w / (1 + w)."""
    g = _trapped_star()
    v = 0
    d = op.degrees(g)
    m = d.sum() / 2.0
    lam = op.spectral_radius_pv(g, v)
    wl = float(np.float32(1e-4))
    assert lam == pytest.approx(wl / (1.0 + wl), rel=1e-9)
    assert lam < 1.0 / g.n                      # untrapped after one step: < 1/n
    dn = float(np.sqrt(np.sum(np.delete(d, v) ** 2)))
    raw = math.log(m / (g.n * math.sqrt(g.n - 1) * dn)) / math.log(lam)
    assert raw < 1.0
    assert op.walk_bound(g.n, m, dn, lam) == 1.0
    p = op.auto_params(g, v, 0.3)
    assert p["t"] == 1.0
    assert p["trees"] == math.ceil(2.0 * math.log(2.0 * g.n) / 0.09)

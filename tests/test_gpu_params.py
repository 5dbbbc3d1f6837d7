"""GPU parity of the automatic parameters (Section 5) with the oracle: the
double-sweep diameter and its start vertex exactly; mu = 1 - lambda against
the dense spectral radius of P_v; t, the tree count and theta against the
oracle's formulas; full-size graphs against SciPy breadth-first distances."""
import math

import numpy as np
import pytest

import paper_2510_20604_gb300 as rwc
import synth
from oracle import params as op
from oracle import wilson as ow

pytestmark = pytest.mark.gpu

GRAPHS = {
    "path": lambda: synth.path(60),
    "cycle": lambda: synth.cycle(33),
    "K7": lambda: synth.complete(7),
    "star": lambda: synth.star(40, center=3),
    "grid": lambda: synth.grid2d(20, 23),
    "ba": lambda: synth.ba(500, 3, seed=1),
    "rmat12": lambda: synth.rmat(12, 8, seed=2),
    "weighted": lambda: synth.rgg(600, 10.0, seed=2, sigma=0.5),
    "parallel_arcs": lambda: __import__("_graphs").multigraph(True),
}


@pytest.mark.parametrize("gname", list(GRAPHS))
def test_auto_params_match_oracle(gname):
    g = GRAPHS[gname]()
    G = rwc.Graph.from_synth(g)
    eps = 0.05
    p = rwc.rwc_auto_params(G.handle, eps)
    ref = op.auto_params(g, G.root, eps)
    assert p.diameter == ref["diameter"]
    assert p.sweep_end == ref["sweep_end"]
    mu_ref = 1.0 - ref["lambda"]
    assert p.mu == pytest.approx(mu_ref, rel=1e-6, abs=1e-12)
    assert p.t == pytest.approx(ref["t"], rel=1e-6)
    # the tree count and theta follow from t and Delta by the same formulas
    d = ow.wdeg(g)
    assert p.trees == op.tree_count(eps, g.n, p.t)
    assert p.theta == pytest.approx(op.solver_theta(eps, g.n, d.sum() / 2, float(d.max()), p.diameter),
                                    rel=1e-12)


def test_closed_forms():
    G = rwc.Graph.from_synth(synth.complete(9))
    p = rwc.rwc_auto_params(G.handle, 0.1)
    assert p.lambda_ == pytest.approx(7 / 8, abs=1e-9) and p.diameter == 1
    G = rwc.Graph.from_synth(synth.cycle(101))
    p = rwc.rwc_auto_params(G.handle, 0.1)
    assert p.lambda_ == pytest.approx(math.cos(math.pi / 101), abs=1e-9) and p.diameter == 50
    G = rwc.Graph.from_synth(synth.star(50, center=0))
    p = rwc.rwc_auto_params(G.handle, 0.1)
    assert p.lambda_ == pytest.approx(0.0, abs=1e-12) and p.t == 1.0


def _scipy_double_sweep(g, v):
    sp = pytest.importorskip("scipy.sparse")
    cs = pytest.importorskip("scipy.sparse.csgraph")
    A = sp.csr_matrix((np.ones(len(g.col)), g.col, g.row_ptr), shape=(g.n, g.n))
    d1 = cs.shortest_path(A, method="D", unweighted=True, indices=[v])[0]
    a = int(np.flatnonzero(d1 == d1.max())[0])
    d2 = cs.shortest_path(A, method="D", unweighted=True, indices=[a])[0]
    return a, int(d2.max())


@pytest.mark.parametrize("which", ["grid1024", "rmat20"])
def test_full_size_diameter(which):
    """The benchmark graphs: the 1024^2 grid's diameter is 2046 (exact for
    grids), R-MAT 20 against SciPy's distances; lambda lies in (0, 1) with
    the inverse iteration converged."""
    g = synth.grid2d(1024, 1024) if which == "grid1024" else synth.rmat(20, 16, seed=0)
    G = rwc.Graph.from_synth(g)
    p = rwc.rwc_auto_params(G.handle, 0.1)
    a, delta = _scipy_double_sweep(g, G.root)
    assert (p.sweep_end, p.diameter) == (a, delta)
    if which == "grid1024":
        assert p.diameter == 2046
    assert 0.0 < p.mu < 1.0 and p.iterations < 30


def _trapped_star():
    u = [0] * 10 + [1]
    v = list(range(1, 11)) + [2]
    return synth.from_edges(11, u, v, np.array([1.0] * 10 + [1e-4], np.float32))


def test_walk_bound_clamp_on_device():
    """The graph where the printed walk-length formula gives about 0.26: the
    device's t is one step, as the oracle's."""
    g = _trapped_star()
    G = rwc.Graph.from_synth(g)
    p = rwc.rwc_auto_params(G.handle, 0.3)
    ref = op.auto_params(g, G.root, 0.3)
    assert G.root == 0 and p.t == 1.0 == ref["t"]
    assert p.trees == ref["trees"]
    # the grounded spectrum here is {1 - lambda, 1 (eight times), 1 + lambda}:
    # inverse iteration separates 1 - lambda from 1 only at rate
    # (1 - lambda), so within its iteration budget mu is resolved to ~1e-4
    # absolute, which keeps lambda below 1/n as the clamp needs
    assert abs(p.mu - (1.0 - ref["lambda"])) <= 1e-4
    assert 0.0 <= p.lambda_ < 1.0 / g.n


def test_fastwalk_auto_uses_the_algorithms_parameters():
    """fastwalk_auto samples l = rwc_auto_params(eps).trees trees and solves
    to theta (floored at 1e-12): its l and theta are the oracle's, its H is
    that of fastwalk with the same l and tolerance, and every vertex meets
    the performance theorem's guarantee pi_u |H~_u - H_u| <= eps against the
    dense exact centrality."""
    from oracle import exact as ex
    g = _trapped_star()
    G = rwc.Graph.from_synth(g)
    eps = 0.3
    H, p, tol = rwc.fastwalk_auto(G, eps, seed=5)
    ref = op.auto_params(g, G.root, eps)
    assert p.trees == ref["trees"] and tol == pytest.approx(max(ref["theta"], 1e-12), rel=1e-9)
    H2, _ = rwc.fastwalk(G, int(p.trees), seed=5, tol=tol)
    assert np.allclose(H.cpu().numpy(), H2.cpu().numpy(), rtol=1e-11, atol=0)
    Hx = ex.rwc_pinv(g)
    d = ow.wdeg(g)
    pi = d / d.sum()
    assert np.all(pi * np.abs(H.cpu().numpy() - Hx) <= eps)
    with pytest.raises(ValueError):
        rwc.fastwalk_auto(rwc.Graph.from_synth(synth.ba(2000, 3, seed=0)), 0.3)   # l ~ 3e8


def test_auto_params_are_bit_reproducible():
    # the inverse iteration's sums and its Laplacian solves run in a fixed
    # order, so lambda (and with it t, l and theta) has the same bits every call
    g = synth.rmat(13, 16, seed=2, sigma=1.0)
    G = rwc.Graph.from_synth(g)
    ps = [rwc.rwc_auto_params(G.handle, 0.1) for _ in range(3)]
    for p in ps[1:]:
        for f, _ in p._fields_:
            assert getattr(p, f) == getattr(ps[0], f), f

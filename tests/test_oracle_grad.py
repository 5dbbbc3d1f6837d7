"""Pins for the dense gradient of J(w) = sum_v c_v H_v(w) (oracle.grad)."""
import numpy as np
import pytest

import synth
from oracle import grad


def _edges(g):
    a, b, w = g.undirected()
    w = np.ones(len(a)) if w is None else w.astype(np.float64)
    return a, b, w


@pytest.mark.parametrize("seed", [0, 1])
def test_closed_form_matches_finite_difference(seed):
    g = synth.rgg(40, 8.0, seed=seed, sigma=0.5)
    a, b, w = _edges(g)
    c = synth.uniform_vector(g.n, seed + 100)
    gc = grad.grad_closed(g.n, a, b, w, c)
    gf = grad.grad_fd(g.n, a, b, w, c, h=1e-5)
    assert np.allclose(gc, gf, rtol=1e-6, atol=1e-6 * np.abs(gc).max())


def test_closed_form_matches_fd_on_200_node_graph_subset():
    g = synth.rgg(200, 12.0, seed=0, sigma=0.5)
    a, b, w = _edges(g)
    c = synth.uniform_vector(g.n, 5)
    gc = grad.grad_closed(g.n, a, b, w, c)
    sel = np.random.default_rng(0).choice(len(a), 40, replace=False)
    for e in sel:
        wp = w.copy(); wp[e] += 1e-5
        wm = w.copy(); wm[e] -= 1e-5
        fd = (grad.J(g.n, a, b, wp, c) - grad.J(g.n, a, b, wm, c)) / 2e-5
        assert abs(fd - gc[e]) <= 1e-6 * max(1.0, abs(gc[e])) + 1e-6 * np.abs(gc).max()


def test_sketch_with_identity_is_exact():
    g = synth.rgg(30, 8.0, seed=3, sigma=0.5)
    a, b, w = _edges(g)
    c = synth.uniform_vector(g.n, 3)
    gc = grad.grad_closed(g.n, a, b, w, c)
    gs = grad.grad_sketch(g.n, a, b, w, c, np.eye(g.n))
    assert np.allclose(gs, gc, rtol=1e-10, atol=1e-10 * np.abs(gc).max())


def test_sketch_is_unbiased():
    g = synth.rgg(30, 8.0, seed=4, sigma=0.5)
    a, b, w = _edges(g)
    c = synth.uniform_vector(g.n, 4)
    gc = grad.grad_closed(g.n, a, b, w, c)
    rng = np.random.default_rng(0)
    k = 16
    R = 400
    acc = np.zeros_like(gc)
    for _ in range(R):
        Q = rng.choice([-1.0, 1.0], size=(k, g.n)) / np.sqrt(k)
        acc += grad.grad_sketch(g.n, a, b, w, c, Q)
    mean = acc / R
    assert np.abs(mean - gc).max() < 0.05 * np.abs(gc).max()


def test_sparse_sketch_route_matches_dense_sketch():
    g = synth.rgg(120, 9.0, seed=8, sigma=0.5)
    a, b, w = _edges(g)
    c = synth.uniform_vector(g.n, 8)
    Q = np.random.default_rng(3).choice([-1.0, 1.0], size=(8, g.n)) / np.sqrt(8)
    dense = grad.grad_sketch(g.n, a, b, w, c, Q)
    sel = np.arange(0, len(a), 7)
    sparse = grad.grad_sketch_sparse(g.n, a, b, w, c, Q, sel)
    assert np.allclose(sparse, dense[sel], rtol=1e-8, atol=1e-8 * np.abs(dense).max())

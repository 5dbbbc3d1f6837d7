"""GPU gradient of J(w) = sum_v c_v H_v(w): exact mode (Q = I) against the
dense closed form and central finite differences (<= 1e-3 relative); sketch
mode against the oracle's sketched formula with the same Philox sketch, and
its error against the exact gradient reported as a number."""
import numpy as np
import pytest
import torch

import paper_2510_20604_gb300 as rwc
import synth
from oracle import grad as og
from oracle import wilson as ow

pytestmark = pytest.mark.gpu


def _edges(g):
    a, b, w = g.undirected()
    return a, b, (np.ones(len(a)) if w is None else w.astype(np.float64))


def test_exact_gradient_matches_dense_and_fd():
    g = synth.rgg(200, 12.0, seed=0, sigma=0.5)
    G = rwc.Graph.from_synth(g)
    c = synth.uniform_vector(g.n, 11)
    ct = torch.tensor(c, dtype=torch.float64, device="cuda")
    gg = G.grad(ct, k=0, tol=1e-10).double().cpu().numpy()
    a, b, w = _edges(g)
    ref = og.grad_closed(g.n, a, b, w, c)
    scale = np.abs(ref).max()
    assert np.max(np.abs(gg - ref)) <= 1e-3 * scale
    rel = np.abs(gg - ref) / np.maximum(np.abs(ref), 1e-3 * scale)
    assert np.median(rel) < 1e-4
    sel = np.random.default_rng(1).choice(len(a), 25, replace=False)
    for e in sel:
        wp = w.copy(); wp[e] += 1e-5
        wm = w.copy(); wm[e] -= 1e-5
        fd = (og.J(g.n, a, b, wp, c) - og.J(g.n, a, b, wm, c)) / 2e-5
        assert abs(gg[e] - fd) <= 1e-3 * max(abs(fd), 1e-2 * scale)


def test_sketch_gradient_matches_oracle_sketch():
    g = synth.rgg(300, 10.0, seed=3, sigma=0.5)
    G = rwc.Graph.from_synth(g)
    c = synth.uniform_vector(g.n, 4)
    ct = torch.tensor(c, dtype=torch.float64, device="cuda")
    k, seed = 64, 1234
    gg = G.grad(ct, k=k, sketch_seed=seed, tol=1e-10).double().cpu().numpy()
    a, b, w = _edges(g)
    Q = ow.rademacher(k, g.n, seed)
    ref = og.grad_sketch(g.n, a, b, w, c, Q)
    assert np.max(np.abs(gg - ref)) <= 1e-4 * np.abs(ref).max()
    exact = og.grad_closed(g.n, a, b, w, c)
    err = np.linalg.norm(gg - exact) / np.linalg.norm(exact)
    assert err < 0.5  # JL error at k = 64, reported by the benchmark as a number


def test_autograd_function_backward():
    g = synth.rgg(60, 8.0, seed=7, sigma=0.3)
    a, b, w = _edges(g)
    wt = torch.tensor(w, dtype=torch.float64, requires_grad=True)
    H = rwc.RWCFunction.apply(wt, g.row_ptr, g.col, 64, 1, 0, 0)
    c = torch.tensor(synth.uniform_vector(g.n, 2), dtype=torch.float64, device=H.device)
    (H * c).sum().backward()
    ref = og.grad_closed(g.n, a, b, w, c.cpu().numpy())
    assert np.max(np.abs(wt.grad.cpu().numpy() - ref)) <= 1e-3 * np.abs(ref).max()


def test_exact_gradient_on_parallel_arcs():
    """A weighted graph with doubled and tripled edges: one gradient entry per
    (a < b) arc, parallel copies equal, against the dense closed form."""
    from _graphs import multigraph
    g = multigraph(True)
    G = rwc.Graph.from_synth(g)
    c = synth.uniform_vector(g.n, 5)
    ct = torch.tensor(c, dtype=torch.float64, device="cuda")
    gg = G.grad(ct, k=0, tol=1e-10).double().cpu().numpy()
    a, b, w = _edges(g)
    ref = og.grad_closed(g.n, a, b, w, c)
    assert np.max(np.abs(gg - ref)) <= 1e-3 * np.abs(ref).max()
    same = (np.diff(a) == 0) & (np.diff(b) == 0)
    assert same.any() and np.allclose(gg[1:][same], gg[:-1][same], rtol=1e-6, atol=0)

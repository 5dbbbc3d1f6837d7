"""Dense gradient of J(w) = sum_v c_v H_v(w) with respect to the undirected
edge weights.  Test infrastructure only.

H_v(w) is the exact random walk centrality (Section 2.3) of the weighted graph,
written as H_v = vol L^+_vv - 2 (L^+ d)_v + d^T L^+ d / vol (see
``exact.rwc_pinv``).  For an edge e = (a, b) with weight w_e, dL/dw_e =
b_e b_e^T (b_e = e_a - e_b), dd/dw_e = e_a + e_b, dvol/dw_e = 2 and, since
b_e is orthogonal to 1, dL^+/dw_e = -L^+ b_e b_e^T L^+.  With x = L^+ c,
y = L^+ d and phi_e = L^+ b_e this gives

  dJ/dw_e = 2 sum_v c_v L^+_vv - vol sum_v c_v (phi_e)_v^2
            + 2 (x_a - x_b)(y_a - y_b) - 2 (x_a + x_b)
            + (sum c) [ (2 (y_a + y_b) - (y_a - y_b)^2) / vol - 2 d^T y / vol^2 ].

``grad_closed`` evaluates this with the dense L^+; ``grad_sketch`` evaluates
the same expression with sum_v c_v (phi_e)_v^2 replaced by
||Q C^1/2 L^+ b_e||^2 and sum_v c_v L^+_vv by the Hutchinson estimate
tr(Q C^1/2 L^+ C^1/2 Q^T), for a given k x n matrix Q (Johnson-Lindenstrauss
sketch; Q = I gives the exact value).  ``grad_fd`` is the central finite
difference of the dense J.  ``grad_sketch_sparse`` is ``grad_sketch`` for
large graphs at selected edges, with SciPy's sparse CG as the solve.

Pins (tests/test_oracle_grad.py): closed form against the finite difference;
the sketch with Q = I against the closed form; the sketch's mean over many
independent Q against the closed form.
"""
from __future__ import annotations

import numpy as np

from .exact import pinv_closed_form


def laplacian_from_edges(n, a, b, w):
    L = np.zeros((n, n))
    np.add.at(L, (a, b), -w)
    np.add.at(L, (b, a), -w)
    d = np.zeros(n)
    np.add.at(d, a, w)
    np.add.at(d, b, w)
    L[np.diag_indices(n)] += d
    return L, d


def J(n, a, b, w, c) -> float:
    L, d = laplacian_from_edges(n, a, b, np.asarray(w, np.float64))
    P = pinv_closed_form(L)
    vol = d.sum()
    Pd = P @ d
    H = vol * np.diag(P) - 2.0 * Pd + (d @ Pd) / vol
    return float(c @ H)


def _terms(n, a, b, w, c):
    L, d = laplacian_from_edges(n, a, b, np.asarray(w, np.float64))
    P = pinv_closed_form(L)
    vol = d.sum()
    x = P @ c
    y = P @ d
    return P, d, vol, x, y


def _assemble(a, b, trCP, sq, x, y, d, vol, csum):
    return (2.0 * trCP - vol * sq
            + 2.0 * (x[a] - x[b]) * (y[a] - y[b]) - 2.0 * (x[a] + x[b])
            + csum * ((2.0 * (y[a] + y[b]) - (y[a] - y[b]) ** 2) / vol
                      - 2.0 * (d @ y) / vol ** 2))


def grad_closed(n, a, b, w, c) -> np.ndarray:
    c = np.asarray(c, np.float64)
    P, d, vol, x, y = _terms(n, a, b, w, c)
    trCP = float(c @ np.diag(P))
    phi = P[:, a] - P[:, b]                     # n x m
    sq = (c[:, None] * phi * phi).sum(axis=0)   # sum_v c_v phi_v^2
    return _assemble(a, b, trCP, sq, x, y, d, vol, c.sum())


def grad_sketch(n, a, b, w, c, Q) -> np.ndarray:
    """Q: k x n sketch (rows of +-1/sqrt(k) for the JL estimate)."""
    c = np.asarray(c, np.float64)
    P, d, vol, x, y = _terms(n, a, b, w, c)
    Z = (Q * np.sqrt(c)[None, :]) @ P          # Q C^1/2 L^+   (k x n)
    trCP = float(np.sum(Z * (Q * np.sqrt(c)[None, :])))   # tr(Z C^1/2 Q^T)
    diff = Z[:, a] - Z[:, b]
    sq = (diff * diff).sum(axis=0)
    return _assemble(a, b, trCP, sq, x, y, d, vol, c.sum())


def grad_fd(n, a, b, w, c, h=1e-5) -> np.ndarray:
    w = np.asarray(w, np.float64)
    g = np.zeros(len(w))
    for e in range(len(w)):
        wp = w.copy(); wp[e] += h
        wm = w.copy(); wm[e] -= h
        g[e] = (J(n, a, b, wp, c) - J(n, a, b, wm, c)) / (2.0 * h)
    return g


def grad_sketch_sparse(n, a, b, w, c, Q, edges, tol=1e-12):
    """``grad_sketch`` for large graphs at selected edges only: the same
    expression with L^+ applied by a sparse conjugate-gradient solve (SciPy,
    one solve per column of [C^1/2 Q^T, c, d], each right-hand side projected
    onto 1-perp first)."""
    import scipy.sparse as sp
    from scipy.sparse.linalg import cg
    w = np.asarray(w, np.float64)
    c = np.asarray(c, np.float64)
    A = sp.coo_matrix((np.concatenate([w, w]), (np.concatenate([a, b]), np.concatenate([b, a]))),
                      shape=(n, n)).tocsr()
    d = np.asarray(A.sum(axis=1)).ravel()
    L = (sp.diags(d) - A).tocsr()
    Minv = sp.diags(1.0 / d)

    def pinv_apply(v):
        v = v - v.mean()
        try:
            x, info = cg(L, v, rtol=tol, atol=0.0, maxiter=20 * n, M=Minv)
        except TypeError:  # SciPy < 1.12 names the relative tolerance `tol`
            x, info = cg(L, v, tol=tol, atol=0.0, maxiter=20 * n, M=Minv)
        if info != 0:
            raise RuntimeError("oracle CG did not converge")
        return x - x.mean()

    k = Q.shape[0]
    sc = np.sqrt(c)
    Z = np.stack([pinv_apply(sc * Q[i]) for i in range(k)])   # Q C^1/2 L^+
    x = pinv_apply(c)
    y = pinv_apply(d)
    vol = d.sum()
    trCP = float(np.sum(Z * (Q * sc[None, :])))
    ea, eb = a[edges], b[edges]
    diff = Z[:, ea] - Z[:, eb]
    sq = (diff * diff).sum(axis=0)
    return _assemble(ea, eb, trCP, sq, x, y, d, vol, c.sum())

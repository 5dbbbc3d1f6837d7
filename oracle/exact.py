"""Dense FP64 ground truth for random walk centrality.  Test infrastructure only.

Weighted reading of the paper's unweighted definitions (Section 2.2): W is the
symmetric weight matrix (parallel arcs add), d = W 1 the weighted degrees,
vol = 1^T d (the paper's 2m), L = D - W, P = D^-1 W, pi = d / vol (Eq. 1),
normalized Laplacian NL = D^-1/2 L D^-1/2.

Random walk centrality H_v = sum_u pi_u H(u, v) (Section 2.3), computed by
three routes that share nothing but the dense matrices:

* ``rwc_pinv``: Section 2.2's closed form L^+ = (L + J/n)^-1 - J/n, then
  H_v = vol L^+_vv - 2 (L^+ d)_v + d^T L^+ d / vol (the hitting-time formula
  H(u,v) = sum_w d_w (L^+_uw - L^+_uv - L^+_vw + L^+_vv) averaged over pi).
* ``rwc_normalized``: Eq. 2, H_v = (NL^+)_vv / pi_v, with NL^+ from a
  symmetric eigendecomposition (the zero eigenvalue dropped).
* ``rwc_hitting``: the definition itself: for each target v solve
  (I - P_{-v}) h = 1 for the hitting times h_u = H(u, v), then H_v = pi . h.

Also: ``tdiag`` = diag of (NL_v)^-1 with row/column v deleted (Lemma 5.1's
t_u, Theorem 3.1's first term), and ``pivot_column`` = NL^+[:, v].

Pins (tests/test_oracle_exact.py): the three routes agree; closed forms on
complete graphs, cycles, stars and paths; t_u = d_u R_uv (proof of Theorem
3.1); Bozzo's identity (Section 3) against the eigen route.
"""
from __future__ import annotations

import numpy as np


def dense_weights(g) -> np.ndarray:
    W = np.zeros((g.n, g.n), dtype=np.float64)
    src = g.src()
    w = np.ones(g.nnz) if g.w is None else g.w.astype(np.float64)
    np.add.at(W, (src, g.col.astype(np.int64)), w)
    return W


def laplacian(g):
    """(L, d): dense Laplacian and weighted degrees (row sums of W)."""
    W = dense_weights(g)
    d = W.sum(axis=1)
    return np.diag(d) - W, d


def pinv_closed_form(L: np.ndarray) -> np.ndarray:
    """L^+ = (L + J/n)^-1 - J/n (Section 2.2), via a Cholesky solve of the
    SPD matrix L + J/n (connected graph)."""
    n = L.shape[0]
    J = np.full((n, n), 1.0 / n)
    A = L + J
    C = np.linalg.cholesky(A)
    Ainv = np.linalg.solve(C.T, np.linalg.solve(C, np.eye(n)))
    return Ainv - J


def rwc_pinv(g) -> np.ndarray:
    L, d = laplacian(g)
    P = pinv_closed_form(L)
    vol = d.sum()
    Pd = P @ d
    return vol * np.diag(P) - 2.0 * Pd + (d @ Pd) / vol


def normalized_pinv(g):
    """(NL^+, d) from a symmetric eigendecomposition of NL."""
    L, d = laplacian(g)
    s = 1.0 / np.sqrt(d)
    NL = s[:, None] * L * s[None, :]
    lam, V = np.linalg.eigh(NL)
    # connected graph: exactly one zero eigenvalue, eigenvector ~ D^1/2 1
    inv = np.zeros_like(lam)
    inv[1:] = 1.0 / lam[1:]
    return (V * inv[None, :]) @ V.T, d


def rwc_normalized(g) -> np.ndarray:
    NLp, d = normalized_pinv(g)
    pi = d / d.sum()
    return np.diag(NLp) / pi


def rwc_hitting(g) -> np.ndarray:
    W = dense_weights(g)
    d = W.sum(axis=1)
    P = W / d[:, None]
    pi = d / d.sum()
    n = g.n
    H = np.zeros(n)
    for v in range(n):
        keep = np.arange(n) != v
        A = np.eye(n - 1) - P[np.ix_(keep, keep)]
        h = np.linalg.solve(A, np.ones(n - 1))
        H[v] = pi[keep] @ h
    return H


def tdiag(g, v: int) -> np.ndarray:
    """t_u = ((NL_v)^-1)_uu for u != v (Lemma 5.1); 0 at v."""
    L, d = laplacian(g)
    s = 1.0 / np.sqrt(d)
    NL = s[:, None] * L * s[None, :]
    keep = np.arange(g.n) != v
    inv = np.linalg.inv(NL[np.ix_(keep, keep)])
    t = np.zeros(g.n)
    t[keep] = np.diag(inv)
    return t


def pivot_column(g, v: int) -> np.ndarray:
    """NL^+[:, v] (the pivot solve of the new computation paradigm)."""
    NLp, _ = normalized_pinv(g)
    return NLp[:, v].copy()


def effective_resistance(g, u: int, v: int) -> float:
    L, _ = laplacian(g)
    P = pinv_closed_form(L)
    return P[u, u] + P[v, v] - 2.0 * P[u, v]


def path_rwc_closed_form(n: int) -> np.ndarray:
    """H_v for the path 0..L (L = n-1) from the classical hitting times of a
    path: H(u,v) = (v-u)(v+u) for u < v and (u-v)(2L-u-v) for u > v,
    averaged over pi (degree 1 at the ends, 2 inside, vol = 2L)."""
    Lh = n - 1
    d = np.full(n, 2.0)
    d[0] = d[-1] = 1.0
    pi = d / (2.0 * Lh)
    H = np.zeros(n)
    for v in range(n):
        s = 0.0
        for u in range(n):
            if u < v:
                h = (v - u) * (v + u)
            elif u > v:
                h = (u - v) * (2 * Lh - u - v)
            else:
                h = 0
            s += pi[u] * h
        H[v] = s
    return H

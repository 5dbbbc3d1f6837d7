"""Automatic parameters of FastWalk (Section 5, "The Sampling Algorithm"):
the sample size l of the tree-count lemma and the solver accuracy theta of
the performance theorem, with the spectral radius lambda of P_v and the graph
diameter Delta they need.  Test infrastructure only; FP64.

* lambda: the largest absolute eigenvalue of P_v, the transition matrix
  D^-1 W with the pivot's row and column removed.  Here from the symmetric
  matrix D^-1/2 W D^-1/2 restricted to V \\ {v}, which has the same spectrum,
  by a dense symmetric eigensolver (the paper uses ARPACK).
* Delta: the diameter, estimated as the paper's experiments need it by a BFS
  double sweep: BFS from the pivot v, then BFS from the farthest vertex
  found (ties to the smallest id); Delta = the largest distance of the second
  sweep (a lower bound, exact on trees and grids).
* t = log( m / (n sqrt(n-1) ||d_-v||_2) ) / log(lambda): the walk length
  after which, by Lemma 5.4 of the cited work with beta = 1/n and s = 1, the
  expected fraction of walks not yet trapped at v is below beta.  Reading
  (the printed argument is ambiguous about where ||d_-v||_2 stands): it
  divides, so that lambda^t <= beta m / (sqrt(n-s) ||d_-v||_2); weighted
  graphs use m = vol / 2 and d = weighted degrees.  t is at least 1 (a walk
  takes a step), which also covers lambda = 0 (every walk trapped at once).
* l = ceil( 2 t^2 log(2n) / eps^2 )  (the tree-count lemma).
* theta = eps / ( 2 Delta d_max (1 + d_max (1 + n) / (2m))^2 sqrt(m n Delta) ).

Pins (tests/test_oracle_params.py): lambda for K_n is (n-2)/(n-1), for the
cycle C_n cos(pi/n) (a path with both ends trapped), for a star rooted at
its centre 0; the double sweep gives the exact diameter of paths, grids and
trees (against all-pairs BFS); formulas against hand-evaluated instances.
"""
from __future__ import annotations

from collections import deque
import math

import numpy as np


def degrees(g) -> np.ndarray:
    if g.w is None:
        return np.diff(g.row_ptr).astype(np.float64)
    d = np.zeros(g.n)
    for u in range(g.n):
        d[u] = float(np.sum(g.w[g.row_ptr[u]:g.row_ptr[u + 1]].astype(np.float64)))
    return d


def bfs_dist(g, s: int) -> np.ndarray:
    """Hop distances from s (plain queue BFS)."""
    dist = np.full(g.n, -1, dtype=np.int64)
    dist[s] = 0
    q = deque([s])
    rp, col = g.row_ptr, g.col
    while q:
        u = q.popleft()
        for c in col[rp[u]:rp[u + 1]]:
            if dist[c] < 0:
                dist[c] = dist[u] + 1
                q.append(int(c))
    return dist


def double_sweep(g, v: int) -> tuple[int, int]:
    """(a, Delta): a = the vertex farthest from v (smallest id on ties),
    Delta = the eccentricity of a."""
    d1 = bfs_dist(g, v)
    a = int(np.flatnonzero(d1 == d1.max())[0])
    d2 = bfs_dist(g, a)
    return a, int(d2.max())


def spectral_radius_pv(g, v: int) -> float:
    """Largest absolute eigenvalue of P_v (dense; small graphs)."""
    n = g.n
    d = degrees(g)
    W = np.zeros((n, n))
    src = g.src()
    np.add.at(W, (src, g.col.astype(np.int64)),
              g.w.astype(np.float64) if g.w is not None else 1.0)   # parallel arcs add up
    s = 1.0 / np.sqrt(d)
    M = s[:, None] * W * s[None, :]
    keep = np.arange(n) != v
    ev = np.linalg.eigvalsh(M[np.ix_(keep, keep)])
    return float(np.max(np.abs(ev)))


def walk_bound(n: int, m: float, d_minus_v_norm: float, lam: float) -> float:
    """t, at least one step."""
    if lam <= 0.0:
        return 1.0
    return max(1.0, math.log(m / (n * math.sqrt(n - 1) * d_minus_v_norm)) / math.log(lam))


def tree_count(eps: float, n: int, t: float) -> int:
    return int(math.ceil(2.0 * t * t * math.log(2.0 * n) / (eps * eps)))


def solver_theta(eps: float, n: int, m: float, dmax: float, delta: int) -> float:
    return eps / (2.0 * delta * dmax * (1.0 + dmax * (1.0 + n) / (2.0 * m)) ** 2
                  * math.sqrt(m * n * delta))


def auto_params(g, v: int, eps: float) -> dict:
    """All of the above for graph g and pivot v."""
    d = degrees(g)
    m = d.sum() / 2.0
    lam = spectral_radius_pv(g, v)
    a, delta = double_sweep(g, v)
    dn = float(np.sqrt(np.sum(np.delete(d, v) ** 2)))
    t = walk_bound(g.n, m, dn, lam)
    return {"lambda": lam, "sweep_end": a, "diameter": delta, "t": t,
            "trees": tree_count(eps, g.n, t), "theta": solver_theta(eps, g.n, m, float(d.max()), delta)}

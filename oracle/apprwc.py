"""Algorithm 1 (AppRWC) and the estimator of Section 5, in FP64.  Test
infrastructure only.

Steps, in the paper's order and notation (weighted reading: d = weighted
degrees, 2m -> vol = sum d):

1. b = D^1/2 (I - D^1/2 1 1^T D^1/2 / vol) e_v, i.e.
   b = sqrt(d_v) e_v - (sqrt(d_v) / vol) d.
2. z = LapSolve(L, b, theta): here any solution of L z = b (``solve_dense``
   uses the closed-form L^+ of Section 2.2; a caller may pass its own z).
3. y = (I - D^1/2 1 1^T D^1/2 / vol) D^1/2 z, i.e.
   y_u = sqrt(d_u) z_u - sqrt(d_u) (sum_w d_w z_w) / vol.
4. For u != v: H_u = ( t_u - (d_u/d_v) y_v + 2 sqrt(d_u/d_v) y_u ) / pi_u.
5. H_v = y_v / pi_v.

The Section 5 estimator feeds step 4 with t_u = S_u / l, S_u the sum over l
trees of the visit counts of Algorithm 3.

Pins (tests/test_oracle_exact.py): with the exact t (``exact.tdiag``) and the
exact z, the result equals the dense ground truth for every pivot v
(Theorem 3.1); y equals NL^+[:, v] (Bozzo's identity).
"""
from __future__ import annotations

import numpy as np


def rhs(d: np.ndarray, v: int) -> np.ndarray:
    vol = d.sum()
    sv = np.sqrt(d[v])
    b = -(sv / vol) * d
    b[v] += sv
    return b


def y_from_z(d: np.ndarray, z: np.ndarray) -> np.ndarray:
    vol = d.sum()
    sd = np.sqrt(d)
    return sd * z - sd * ((d * z).sum() / vol)


def recover(d: np.ndarray, v: int, t: np.ndarray, y: np.ndarray) -> np.ndarray:
    """Steps 4-5: H from t (t_v ignored) and y."""
    vol = d.sum()
    pi = d / vol
    H = np.empty_like(d)
    for u in range(len(d)):
        if u == v:
            H[u] = y[v] / pi[v]
        else:
            H[u] = (t[u] - (d[u] / d[v]) * y[v] + 2.0 * np.sqrt(d[u] / d[v]) * y[u]) / pi[u]
    return H


def recover_vec(d: np.ndarray, v: int, t: np.ndarray, y: np.ndarray) -> np.ndarray:
    """Same arithmetic as ``recover`` written with whole-array operations
    (for large n); each element is computed by the identical expression."""
    vol = d.sum()
    pi = d / vol
    H = (t - (d / d[v]) * y[v] + 2.0 * np.sqrt(d / d[v]) * y) / pi
    H[v] = y[v] / pi[v]
    return H


def solve_dense(L: np.ndarray, b: np.ndarray) -> np.ndarray:
    n = L.shape[0]
    J = np.full((n, n), 1.0 / n)
    return np.linalg.solve(L + J, b) - (b.sum() / n)  # L^+ b; b.sum() = 0 here


def estimate(d, v, sums, ntrees, z):
    """Section 5 estimator followed by Algorithm 1 steps 3-5."""
    t = np.asarray(sums, np.float64) / float(ntrees)
    y = y_from_z(d, z)
    return recover_vec(d, v, t, y), y


def predicted_mre(d: np.ndarray, v: int, sums: np.ndarray, T: int, H: np.ndarray) -> float:
    """Mean relative error to expect from T trees (the variance law of the
    visit counts): visits_u per tree are geometric with mean t_u, so t~_u =
    sums_u / T has variance t_u (t_u - 1) / T; H~_u = (t~_u - ...) / pi_u
    carries that error divided by pi_u (H~_v carries none), and a normal error
    of standard deviation s has mean absolute value sqrt(2/pi) s.  t_u is
    replaced by its estimate.  MRE = mean over all n vertices of
    sqrt(2/pi) se_u / |H_u|."""
    d = np.asarray(d, np.float64)
    pi = d / d.sum()
    t = np.asarray(sums, np.float64) / T
    se = np.sqrt(np.maximum(t * (t - 1.0), 0.0) / T) / pi
    se[v] = 0.0
    return float(np.sqrt(2.0 / np.pi) * np.mean(se / np.abs(H)))


def trees_for(mre: float, T: int, target: float) -> int:
    """Trees needed for the target MRE (the error falls as 1/sqrt(T))."""
    return int(np.ceil(T * (mre / target) ** 2))

"""Evaluation measures of Section 6 ("Evaluation Measures" and "Approximation
Quality"), in FP64 and exact integers.  Test infrastructure only.

* Mean relative error of an estimate H~ against a reference H:
      MRE = (1/n) sum_u |H_u - H~_u| / H_u.
* Kendall distance of two rankings (the paper's K(L1, L2), Kendall's tau-a):
      K = 2 (alpha - beta) / (n (n - 1)),
  alpha = concordant pairs, beta = discordant pairs; a pair tied in either
  ranking is neither.  ``kendall_counts`` returns alpha - beta exactly by
  brute force over all pairs (plain definition; blocks of rows only to
  bound memory), so it is meant for n up to a few tens of thousands.

Pins (tests/test_oracle_evaluate.py): identical and reversed rankings give
+1 and -1; hand-counted small cases with ties; with no ties tau-a equals
SciPy's tau-b (a library routine that coincides with tau-a then); tied
pairs counted by hand; an MRE of a uniformly scaled estimate equals the
scale error exactly.
"""
from __future__ import annotations

import numpy as np


def mre(H: np.ndarray, H_est: np.ndarray) -> float:
    """(1/n) sum_u |H_u - H~_u| / H_u."""
    H = np.asarray(H, dtype=np.float64)
    H_est = np.asarray(H_est, dtype=np.float64)
    return float(np.mean(np.abs(H - H_est) / H))


def kendall_counts(a: np.ndarray, b: np.ndarray, block: int = 2048) -> int:
    """alpha - beta over the unordered pairs {i, j}, i != j: the sum of
    sign(a_i - a_j) * sign(b_i - b_j) over i < j."""
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    n = a.shape[0]
    total = 0
    for i0 in range(0, n, block):
        ai = a[i0:i0 + block, None]
        bi = b[i0:i0 + block, None]
        s = np.sign(ai - a[None, :]) * np.sign(bi - b[None, :])
        # keep j > i only
        rows = np.arange(i0, min(n, i0 + block))[:, None]
        s = np.where(np.arange(n)[None, :] > rows, s, 0.0)
        total += int(s.sum())
    return total


def kendall_tau_a(a: np.ndarray, b: np.ndarray) -> float:
    """K(L1, L2) = 2 (alpha - beta) / (n (n - 1))."""
    n = len(a)
    if n < 2:
        return 0.0
    return 2.0 * kendall_counts(a, b) / (n * (n - 1.0))

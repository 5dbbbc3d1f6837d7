"""Pins of the evaluation measures (Section 6): Kendall distance K(L1, L2)
= 2 (alpha - beta) / (n (n - 1)) and the mean relative error."""
import numpy as np
import pytest

from oracle import evaluate as ev


def test_kendall_identical_and_reversed():
    x = np.random.default_rng(0).permutation(50).astype(float)
    assert ev.kendall_tau_a(x, x) == 1.0
    assert ev.kendall_tau_a(x, -x) == -1.0
    assert ev.kendall_counts(x, x) == 50 * 49 // 2


def test_kendall_hand_counted():
    # pairs (0,1) +, (0,2) +, (1,2) -  ->  (2 - 1) / 3
    assert ev.kendall_counts([1, 2, 3], [1, 3, 2]) == 1
    assert ev.kendall_tau_a([1, 2, 3], [1, 3, 2]) == pytest.approx(1 / 3, abs=0)
    # a pair tied in the first ranking counts neither way: (0,1) 0, (0,2) +, (1,2) +
    assert ev.kendall_counts([1, 1, 2], [1, 2, 3]) == 2
    # tied in both: all pairs 0
    assert ev.kendall_counts([5, 5, 5], [1, 1, 1]) == 0
    # n = 4 worked by hand: a = (4, 1, 3, 2), b = (3, 1, 4, 2)
    # pairs: (0,1) ++ ; (0,2) + - ; (0,3) ++ ; (1,2) ++ ; (1,3) ++ ; (2,3) ++  -> 5 - 1
    assert ev.kendall_counts([4, 1, 3, 2], [3, 1, 4, 2]) == 4


def test_kendall_matches_scipy_without_ties():
    stats = pytest.importorskip("scipy.stats")
    rng = np.random.default_rng(3)
    for n in (2, 17, 400, 3001):
        a = rng.standard_normal(n)
        b = a + rng.standard_normal(n) * 0.7
        tau_b = stats.kendalltau(a, b).statistic
        assert ev.kendall_tau_a(a, b) == pytest.approx(tau_b, abs=1e-12)


def test_kendall_ties_against_pair_loop():
    rng = np.random.default_rng(5)
    a = rng.integers(0, 6, 120).astype(float)
    b = rng.integers(0, 4, 120).astype(float)
    want = 0
    for i in range(120):
        for j in range(i + 1, 120):
            sa = int(a[i] > a[j]) - int(a[i] < a[j])
            sb = int(b[i] > b[j]) - int(b[i] < b[j])
            want += sa * sb
    assert ev.kendall_counts(a, b, block=7) == want


def test_mre_scaled_estimate():
    # small integers: H (1 +- 2^-k) and the quotients are exact in binary
    H = np.random.default_rng(1).integers(1, 1000, 1000).astype(np.float64)
    assert ev.mre(H, H) == 0.0
    assert ev.mre(H, H * (1 + 2.0 ** -7)) == 2.0 ** -7
    assert ev.mre(H, H * (1 - 2.0 ** -3)) == 2.0 ** -3

"""Pins for the oracle's Johnson-Lindenstrauss sketch (``oracle_rademacher``)
against facts that do not restate its code: the entries' exact magnitude,
the law of a Rademacher matrix (sign balance, E[Q^T Q] = I, uncorrelated
rows), and its counter layout checked entry by entry against an independent
Philox (Triton's, run by its CPU interpreter)."""
import json
import subprocess
import sys
import textwrap

import numpy as np
import pytest

from oracle import wilson as ow


@pytest.mark.parametrize("k", [1, 7, 64])
def test_entries_are_plus_minus_one_over_sqrt_k(k):
    Q = ow.rademacher(k, 1000, seed=3)
    assert Q.shape == (k, 1000)
    s = 1.0 / np.sqrt(k)
    assert np.all((Q == s) | (Q == -s))
    # both signs occur in every row long enough to show them
    assert np.all((Q > 0).any(1)) and np.all((Q < 0).any(1))


def test_sign_balance_over_a_million_entries():
    k, n = 64, 1 << 14
    Q = ow.rademacher(k, n, seed=11)
    neg = int((Q < 0).sum())
    N = k * n
    # Binomial(N, 1/2): 5 standard deviations
    assert abs(neg - N / 2) <= 5 * np.sqrt(N / 4)
    # per row and per column block the balance holds too (no constant sign
    # from a fixed counter word)
    rows = (Q < 0).sum(1)
    assert np.all(np.abs(rows - n / 2) <= 5 * np.sqrt(n / 4))


def test_gram_matrix_is_identity_in_expectation():
    """E[Q^T Q] = I: the diagonal is exactly 1 (k entries of 1/k), an
    off-diagonal entry is (1/k) * sum of k independent signs, mean 0 and
    variance 1/k.  Over many seeds and pairs the sample mean and variance
    must match within their sampling error."""
    k, n = 64, 256
    off = []
    rowc = []
    for seed in range(40):
        Q = ow.rademacher(k, n, seed=seed)
        G = Q.T @ Q
        assert np.allclose(np.diag(G), 1.0, atol=1e-12)
        iu = np.triu_indices(n, 1)
        off.append(G[iu])
        R = Q @ Q.T                    # row correlations: (1/k) sum_u s_iu s_ju
        ir = np.triu_indices(k, 1)
        rowc.append(R[ir] * k / np.sqrt(n))   # standardised: mean 0, variance 1
    off = np.concatenate(off)
    m = off.size
    assert abs(off.mean()) <= 5 * np.sqrt(1.0 / k / m)
    # variance of the sample variance for a scaled binomial is close to 2/k^2/m
    assert abs(off.var() - 1.0 / k) <= 5 * np.sqrt(2.0 / m) / k
    rowc = np.concatenate(rowc)
    assert abs(rowc.mean()) <= 5 / np.sqrt(rowc.size)
    assert abs(rowc.var() - 1.0) <= 5 * np.sqrt(2.0 / rowc.size)


def test_seeds_give_independent_sketches():
    k, n = 64, 4096
    A = ow.rademacher(k, n, seed=1)
    B = ow.rademacher(k, n, seed=2)
    agree = float((np.sign(A) == np.sign(B)).mean())
    assert abs(agree - 0.5) <= 5 * np.sqrt(0.25 / (k * n))
    # the high word of the seed is part of the key
    C = ow.rademacher(k, n, seed=1 | (5 << 32))
    assert not np.array_equal(A, C)


def test_counter_layout_against_triton_philox():
    """Entry (i, u) is negative exactly when the top bit of the first Philox
    output word for counter (i, u, 0xFFFFFFFF, 0) and key (seed lo, seed hi)
    is set.  Triton's Philox is an implementation independent of the oracle's;
    a transposed counter, another output word or a flipped sign all fail."""
    pytest.importorskip("triton")
    k, n, seed = 5, 37, (3 << 32) | 123456789
    code = textwrap.dedent(f"""
        import os, json
        os.environ["TRITON_INTERPRET"] = "1"
        import torch, triton, triton.language as tl
        @triton.jit
        def kern(out, c0p, c1p, seed, M, N: tl.constexpr):
            o = tl.arange(0, N)
            m = o < M
            c0 = tl.load(c0p + o, mask=m, other=0)
            c1 = tl.load(c1p + o, mask=m, other=0)
            c2 = tl.full([N], 0xFFFFFFFF, tl.uint32)
            c3 = tl.zeros([N], tl.uint32)
            a, b, c, d = tl.philox(seed, c0, c1, c2, c3, 10)
            tl.store(out + o, a, mask=m)
        M = {k * n}
        ii = torch.arange(M, dtype=torch.int64) // {n}
        uu = torch.arange(M, dtype=torch.int64) % {n}
        out = torch.zeros(M, dtype=torch.int32)
        kern[(1,)](out, ii.to(torch.uint32), uu.to(torch.uint32), {seed}, M, 256)
        print(json.dumps([x & 0xffffffff for x in out.tolist()]))
    """)
    r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, timeout=600)
    if r.returncode != 0:
        pytest.skip("triton interpreter unavailable: " + r.stderr[-300:])
    o0 = np.array(json.loads(r.stdout.strip().splitlines()[-1]), np.uint64).reshape(k, n)
    expect_neg = (o0 >> np.uint64(31)) == 1
    Q = ow.rademacher(k, n, seed)
    assert np.array_equal(Q < 0, expect_neg)

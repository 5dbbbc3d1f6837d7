"""Generator sanity: CSR conventions, sizes, symmetry and connectivity."""
import numpy as np
import pytest
from scipy.sparse import csr_matrix
from scipy.sparse.csgraph import connected_components

import synth


def check_csr(g):
    rp, col = g.row_ptr, g.col
    assert rp[0] == 0 and rp[-1] == len(col) and (np.diff(rp) >= 1).all()
    src = g.src()
    assert (src != col).all()
    for u in (0, g.n // 2, g.n - 1):
        row = col[rp[u]:rp[u + 1]]
        assert (np.diff(row) > 0).all()
    A = csr_matrix((np.ones(g.nnz) if g.w is None else g.w, col, rp), shape=(g.n, g.n))
    assert (abs(A - A.T)).nnz == 0
    assert connected_components(A, directed=False)[0] == 1


@pytest.mark.parametrize("make", [
    lambda: synth.ba(2000, 3, seed=0),
    lambda: synth.grid2d(32, 17),
    lambda: synth.rmat(12, 16, seed=0),
    lambda: synth.rmat(10, 16, seed=1, sigma=1.0),
    lambda: synth.rgg(3000, 12.0, seed=0, sigma=0.5),
    lambda: synth.er(1000, 8.0, seed=0),
])
def test_generated_graphs_are_valid(make):
    check_csr(make())


def test_sizes():
    g = synth.ba(2000, 3, seed=0)
    m = g.nnz // 2
    assert 3 * 1996 + 6 <= m <= 3 * 1996 + 6 + 1999
    gr = synth.grid2d(64, 64)
    assert gr.nnz == 2 * 2 * 64 * 63
    r = synth.rmat(12, 16, seed=0)
    assert r.nnz <= 16 * 4096 + 2 * 4095


def test_batch_specs_deterministic():
    a = synth.batch_specs(50, seed=0)
    b = synth.batch_specs(50, seed=0)
    assert a == b
    assert all(50 <= n <= 20000 for n, _ in a)
    g1 = synth.batch_graph(3, a[3][0], a[3][1])
    g2 = synth.batch_graph(3, a[3][0], a[3][1])
    assert np.array_equal(g1.col, g2.col)

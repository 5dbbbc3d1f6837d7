"""GPU parity of the pivot solve and recovery (Algorithm 1) against the
oracle: y against the dense NL^+[:, v]; H against the oracle's recovery on
the same sums and the same y to 1e-12 relative; the solver against dense
L^+; Monte Carlo error of the whole pipeline against exact FP64 H."""
import numpy as np
import pytest
import torch

import paper_2510_20604_gb300 as rwc
import synth
from oracle import apprwc, exact
from oracle import wilson as ow

pytestmark = pytest.mark.gpu


def _hub_graph():
    """A BA graph whose vertex 0 is also joined to 2500 others (a row of more
    than 2 * 1024 arcs: the solver's chunked heavy-row path)."""
    base = synth.ba(3000, 2, seed=4)
    src, dst = base.src(), base.col
    keep = src < dst
    a = list(src[keep]); b = list(dst[keep])
    have = set(b[i] for i in range(len(a)) if a[i] == 0)
    for v in range(1, 2501):
        if v not in have:
            a.append(0); b.append(v)
    return synth.from_edges(3000, np.array(a), np.array(b))


@pytest.mark.parametrize("gname", ["ba", "weighted", "grid", "hub", "rmat13w", "multi", "multiw"])
def test_pivot_column_and_recovery(gname):
    from _graphs import multigraph
    g = {"multi": lambda: multigraph(False),
         "multiw": lambda: multigraph(True),
         "ba": lambda: synth.ba(500, 3, seed=1),
         "weighted": lambda: synth.rgg(600, 10.0, seed=2, sigma=0.5),
         "grid": lambda: synth.grid2d(20, 23),
         "hub": _hub_graph,
         "rmat13w": lambda: synth.rmat(13, 16, seed=3, sigma=1.0)}[gname]()
    G = rwc.Graph.from_synth(g)
    T = 200
    sums, _, _, _ = G.sample(T, seed=3)
    H, y = G.estimate(sums, T, tol=1e-12, want_y=True)
    yh = y.cpu().numpy()
    yref = exact.pivot_column(g, G.root)
    assert np.max(np.abs(yh - yref)) <= 1e-9 * np.max(np.abs(yref))
    d = ow.wdeg(g)
    Href = apprwc.recover_vec(d, G.root, sums.cpu().numpy() / T, yh)
    rel = np.abs(H.cpu().numpy() - Href) / np.abs(Href)
    assert rel.max() < 1e-12, rel.max()
    # the recovery-only entry point gives the same numbers
    H2 = torch.empty_like(H)
    rwc.rwc_recover(G.handle, sums, T, y, H2)
    assert torch.allclose(H, H2, rtol=1e-15, atol=0)


def test_single_rhs_solve_with_heavy_rows():
    """k = 1 takes the one-launch cooperative solver, whose sparse product
    splits rows of more than 1024 arcs into warp-sized chunks."""
    g = _hub_graph()
    assert np.diff(g.row_ptr).max() > 2048
    G = rwc.Graph.from_synth(g)
    L, _ = exact.laplacian(g)
    P = exact.pinv_closed_form(L)
    b = np.random.default_rng(2).standard_normal(g.n)
    b -= b.mean()
    Bt = torch.tensor(b[None, :], dtype=torch.float64, device="cuda")
    X = torch.empty_like(Bt)
    rwc.rwc_solve(G.handle, 1, Bt, X, 1e-11)
    ref = P @ b
    err = np.abs(X.cpu().numpy()[0] - ref).max() / np.abs(ref).max()
    assert err < 1e-9, err


def test_solver_against_dense_pseudoinverse():
    g = synth.rgg(400, 9.0, seed=5, sigma=0.7)
    G = rwc.Graph.from_synth(g)
    L, _ = exact.laplacian(g)
    P = exact.pinv_closed_form(L)
    rng = np.random.default_rng(0)
    k = 5
    Bm = rng.standard_normal((k, g.n))
    Bt = torch.tensor(Bm, dtype=torch.float64, device="cuda")
    X = torch.empty_like(Bt)
    it = rwc.rwc_solve(G.handle, k, Bt, X, 1e-11)
    ref = (P @ Bm.T).T
    err = np.abs(X.cpu().numpy() - ref).max() / np.abs(ref).max()
    assert err < 1e-9, (err, it)


def test_small_config_mre_against_exact():
    """BA n=2000 + path, 1000 trees: MRE of the FastWalk estimate against the
    dense FP64 ground truth, inside the band predicted by the geometric
    variance of the visit counts (Lemma 5.2)."""
    g = synth.ba(2000, 3, seed=0)
    G = rwc.Graph.from_synth(g)
    T = 1000
    sums, _, _, _ = G.sample(T, seed=1)
    H = G.estimate(sums, T).cpu().numpy()
    Hx = exact.rwc_pinv(g)
    mre = float(np.mean(np.abs(H - Hx) / Hx))
    t = exact.tdiag(g, G.root)
    d = ow.wdeg(g)
    pi = d / d.sum()
    pred = float(np.sqrt(2 / np.pi) * np.mean(np.sqrt(np.maximum(t * (t - 1), 0) / T) / pi / Hx))
    assert 0.7 * pred < mre < 1.3 * pred, (mre, pred)
    assert mre < 0.02


def test_estimate_rejects_bad_arguments():
    g = synth.path(10)
    G = rwc.Graph.from_synth(g)
    s = torch.zeros(10, dtype=torch.float64, device="cuda")
    H = torch.empty_like(s)
    with pytest.raises(rwc.RWCError):
        rwc.rwc_estimate(G.handle, s, 0, 1e-10, H)
    with pytest.raises(TypeError):
        rwc.rwc_estimate(G.handle, s.float(), 1, 1e-10, H)


def test_fastwalk_to_target_stops_at_the_predicted_count():
    """The stopping rule in the pipeline: starting from 200 trees on the
    small configuration, trees are added until the predicted MRE is at most
    1%; the result equals one run of the final tree count (the added trees
    continue the global ids), and the measured MRE against the exact RWC is
    near the target."""
    g = synth.ba(2000, 3, seed=0)
    G = rwc.Graph.from_synth(g)
    H, T, mre = rwc.fastwalk_to_target(G, 0.01, first_trees=200, seed=1)
    assert T > 200 and mre <= 0.01
    H1, _ = rwc.fastwalk(G, T, seed=1)
    assert torch.allclose(H, H1, rtol=1e-9, atol=0)
    Hx = exact.rwc_pinv(g)
    measured = float(np.mean(np.abs(H.cpu().numpy() - Hx) / Hx))
    assert measured < 0.0125, measured


@pytest.mark.parametrize("gname", ["ba", "rmat", "weighted_heavy_rows"])
def test_pivot_solve_is_bit_reproducible(gname):
    """The pivot solve's sums run in a fixed order (block parts added in block
    order, no floating-point atomics), so the same input gives the same y and
    H bits on every call."""
    g = {"ba": lambda: synth.ba(3000, 3, seed=1),
         "rmat": lambda: synth.rmat(14, 16, seed=1),
         "weighted_heavy_rows": lambda: synth.rmat(13, 64, seed=4, sigma=1.0)}[gname]()
    G = rwc.Graph.from_synth(g)
    sums, _, _, _ = G.sample(16, seed=2)
    outs = [G.estimate(sums, 16, want_y=True) for _ in range(4)]
    for H, y in outs[1:]:
        assert torch.equal(H, outs[0][0]) and torch.equal(y, outs[0][1])


@pytest.mark.parametrize("gname", ["grid", "weighted_rmat"])
def test_pivot_solve_then_recover_equals_estimate(gname):
    """rwc_pivot_solve computes the pivot column alone (it needs no trees, so it
    can run beside the sampling, on another stream); with rwc_recover it gives
    rwc_estimate's y and H bit for bit."""
    g = {"grid": lambda: synth.grid2d(90, 70),
         "weighted_rmat": lambda: synth.rmat(13, 16, seed=6, sigma=1.0)}[gname]()
    G = rwc.Graph.from_synth(g)
    sums, _, _, _ = G.sample(12, seed=5)
    H_ref, y_ref = G.estimate(sums, 12, want_y=True)
    y = torch.empty(g.n, dtype=torch.float64, device="cuda")
    side = torch.cuda.Stream()
    rwc.rwc_pivot_solve(G.handle, 1e-10, y, stream=side.cuda_stream)
    H = torch.empty_like(y)
    rwc.rwc_recover(G.handle, sums, 12, y, H)
    assert torch.equal(y, y_ref) and torch.equal(H, H_ref)

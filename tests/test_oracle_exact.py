"""Pins for the dense ground truth (oracle.exact) and Algorithm 1 (oracle.apprwc)."""
import numpy as np
import pytest

import synth
from oracle import apprwc, exact
from oracle import wilson as ow


def rand_weighted(seed, n=9, extra=8):
    rng = np.random.default_rng(seed)
    u = list(range(n - 1)); v = list(range(1, n))
    while len(u) < n - 1 + extra:
        a, b = rng.integers(0, n, 2)
        if a != b:
            u.append(int(a)); v.append(int(b))
    w = rng.lognormal(0, 1.0, size=len(u)).astype(np.float32)
    return synth.from_edges(n, u, v, w)


@pytest.mark.parametrize("seed", range(4))
def test_three_routes_agree(seed):
    g = rand_weighted(seed)
    h1 = exact.rwc_pinv(g)
    h2 = exact.rwc_normalized(g)
    h3 = exact.rwc_hitting(g)
    assert np.allclose(h1, h3, rtol=1e-11, atol=0)
    assert np.allclose(h2, h3, rtol=1e-11, atol=0)


def test_routes_agree_on_generated_graphs():
    for g in (synth.ba(120, 3, seed=1), synth.rgg(150, 10.0, seed=2, sigma=0.5)):
        h1 = exact.rwc_pinv(g)
        h3 = exact.rwc_hitting(g)
        assert np.allclose(h1, h3, rtol=1e-10)


@pytest.mark.parametrize("n", [3, 5, 10, 17])
def test_closed_forms(n):
    assert np.allclose(exact.rwc_pinv(synth.complete(n)), (n - 1) ** 2 / n, rtol=1e-12)
    assert np.allclose(exact.rwc_pinv(synth.cycle(n)), (n * n - 1) / 6.0, rtol=1e-12)
    hs = exact.rwc_pinv(synth.star(n, center=0))
    assert np.isclose(hs[0], 0.5, rtol=1e-12)
    assert np.allclose(hs[1:], (4 * n - 7) / 2.0, rtol=1e-12)
    assert np.allclose(exact.rwc_pinv(synth.path(n)), exact.path_rwc_closed_form(n), rtol=1e-11)


@pytest.mark.parametrize("seed", range(3))
def test_tdiag_is_degree_times_resistance(seed):
    """Proof of Theorem 3.1: (NL_v^-1)_uu = d_u R_uv."""
    g = rand_weighted(seed + 10)
    _, d = exact.laplacian(g)
    v = 3
    t = exact.tdiag(g, v)
    for u in range(g.n):
        if u != v:
            assert np.isclose(t[u], d[u] * exact.effective_resistance(g, u, v), rtol=1e-10)


@pytest.mark.parametrize("seed", range(3))
def test_bozzo_identity_gives_pivot_column(seed):
    """Section 3: y = M D^1/2 L^+ D^1/2 M e_v equals NL^+[:, v]."""
    g = rand_weighted(seed + 20)
    L, d = exact.laplacian(g)
    for v in range(g.n):
        b = apprwc.rhs(d, v)
        assert abs(b.sum()) < 1e-12
        z = apprwc.solve_dense(L, b)
        y = apprwc.y_from_z(d, z)
        assert np.allclose(y, exact.pivot_column(g, v), atol=1e-12 * max(1, np.abs(y).max()))


@pytest.mark.parametrize("seed", range(3))
def test_theorem_3_1_every_pivot(seed):
    """Algorithm 1 with the exact diagonal reproduces H for every pivot v
    (Theorem 3.1, and the remark that H does not depend on v)."""
    g = rand_weighted(seed + 30, n=11, extra=12)
    L, d = exact.laplacian(g)
    H = exact.rwc_hitting(g)
    for v in range(g.n):
        t = exact.tdiag(g, v)
        z = apprwc.solve_dense(L, apprwc.rhs(d, v))
        Hv = apprwc.recover(d, v, t, apprwc.y_from_z(d, z))
        assert np.allclose(Hv, H, rtol=1e-10)
        Hv2 = apprwc.recover_vec(d, v, t, apprwc.y_from_z(d, z))
        assert np.array_equal(Hv, Hv2)


def test_estimator_converges_on_small_ba():
    """End to end on the oracle side: Algorithm 3's sums over many trees give
    H within the Monte Carlo band predicted from the geometric variance."""
    g = synth.ba(100, 3, seed=0)
    s = ow.Sampler(g, seed=1)
    T = 4000
    out = s.sample(0, T, nthreads=4)
    L, d = exact.laplacian(g)
    z = apprwc.solve_dense(L, apprwc.rhs(d, s.root))
    Hest, _ = apprwc.estimate(d, s.root, out["sums"], T, z)
    H = exact.rwc_pinv(g)
    t = exact.tdiag(g, s.root)
    pi = d / d.sum()
    sd = np.sqrt(np.maximum(t * (t - 1), 0) / T) / pi
    assert (np.abs(Hest - H) <= 5 * sd + 1e-9).all()
    mre = np.mean(np.abs(Hest - H) / H)
    pred = np.sqrt(2 / np.pi) * np.mean(sd / H)
    assert 0.5 * pred < mre < 1.5 * pred


def test_predicted_mre_matches_measured_error():
    """The variance-law prediction against the error the oracle's own trees
    actually make against the exact H (BA n = 2000 + path, the small
    configuration), at two tree counts; and the 1/sqrt(T) rule for the trees
    needed."""
    from oracle import apprwc
    from oracle import wilson as ow
    g = synth.ba(2000, 3, seed=0)
    s = ow.Sampler(g, seed=1)
    v = s.root
    d = ow.wdeg(g)
    Hx = exact.rwc_pinv(g)
    y = exact.pivot_column(g, v)
    for T in (400, 1600):
        sums = s.sample(0, T, nthreads=ow.cores())["sums"]
        H = apprwc.recover_vec(d, v, sums / T, y)
        measured = float(np.mean(np.abs(H - Hx) / Hx))
        pred = apprwc.predicted_mre(d, v, sums, T, H)
        assert 0.75 * pred < measured < 1.25 * pred, (T, measured, pred)
    assert apprwc.trees_for(0.02, 1000, 0.01) == 4000
    assert apprwc.trees_for(0.01, 1000, 0.01) == 1000

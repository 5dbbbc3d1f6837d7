"""GPU parity of the evaluation measures (Section 6) with the oracle: the
Kendall distance's alpha - beta is an exact integer and must match bit for
bit (sizes spanning several row and column tiles, ragged tails, ties,
-0.0 against +0.0); the mean relative error within 1e-12 relative (a sum in
a different order)."""
import numpy as np
import pytest
import torch

import paper_2510_20604_gb300 as rwc
from oracle import evaluate as ev

pytestmark = pytest.mark.gpu


def _cuda(x):
    return torch.as_tensor(np.asarray(x, dtype=np.float64), device="cuda")


@pytest.mark.parametrize("n", [0, 1, 2, 3, 1023, 1024, 1025, 2049, 5000])
def test_kendall_matches_oracle_with_ties(n):
    rng = np.random.default_rng(n)
    a = rng.integers(0, max(2, n // 3), n).astype(np.float64)
    b = a + rng.integers(-2, 3, n)
    tau, diff = rwc.rwc_kendall(_cuda(a), _cuda(b))
    want = ev.kendall_counts(a, b) if n >= 2 else 0
    assert diff == want
    if n >= 2:
        assert tau == pytest.approx(ev.kendall_tau_a(a, b), rel=1e-15, abs=0)


def test_kendall_continuous_and_signed_zero():
    rng = np.random.default_rng(7)
    a = rng.standard_normal(7001)
    b = a + rng.standard_normal(7001)
    a[:5] = [0.0, -0.0, 0.0, -0.0, 1e-300]
    b[:5] = [-0.0, 0.0, 1.0, 1.0, -1e-300]
    _, diff = rwc.rwc_kendall(_cuda(a), _cuda(b))
    assert diff == ev.kendall_counts(a, b)


def test_kendall_full_size_properties():
    """n = 2^20 (the RWC vectors of the grid and R-MAT 20): identical rankings
    give every pair concordant, reversed ones every pair discordant."""
    n = 1 << 20
    x = torch.randperm(n, device="cuda", generator=torch.Generator(device="cuda").manual_seed(0)).double()
    tau, diff = rwc.rwc_kendall(x, x)
    assert diff == n * (n - 1) // 2 and tau == 1.0
    tau, diff = rwc.rwc_kendall(x, -x)
    assert diff == -(n * (n - 1) // 2) and tau == -1.0


@pytest.mark.parametrize("n", [1, 255, 256, 257, 100_000, 1 << 20])
def test_mre_matches_oracle(n):
    rng = np.random.default_rng(n)
    H = rng.uniform(0.5, 50.0, n)
    He = H * (1 + rng.normal(0, 0.01, n))
    got = float(rwc.rwc_mre(_cuda(H), _cuda(He)).item())
    assert got == pytest.approx(ev.mre(H, He), rel=1e-12, abs=0)
    # deterministic reduction order
    assert float(rwc.rwc_mre(_cuda(H), _cuda(He)).item()) == got


def test_tree_count_sweep_small_config():
    """The accuracy sweep of Section 6 on the small configuration (BA n = 2000
    + path, exact H from the dense oracle), as curve shapes: with 4x the
    trees the device MRE halves (1/sqrt(l), within 25%) and the device
    Kendall distance to the exact ranking rises towards 1; both device
    measures equal the oracle's on the same vectors."""
    import synth
    from oracle import exact
    g = synth.ba(2000, 3, seed=0)
    G = rwc.Graph.from_synth(g)
    Hx = exact.rwc_pinv(g)
    Hx_d = _cuda(Hx)
    mres, taus = [], []
    for T in (250, 1000, 4000):
        sums, _, _, _ = G.sample(T, seed=1)
        H = G.estimate(sums, T)
        m = float(rwc.rwc_mre(Hx_d, H).item())
        tau, diff = rwc.rwc_kendall(H, Hx_d)
        Hn = H.cpu().numpy()
        assert m == pytest.approx(ev.mre(Hx, Hn), rel=1e-12, abs=0)
        assert diff == ev.kendall_counts(Hn, Hx)
        mres.append(m)
        taus.append(tau)
    for a, b in zip(mres, mres[1:]):
        assert 0.5 * 0.75 < b / a < 0.5 * 1.25, mres
    assert taus[0] < taus[1] < taus[2] < 1.0, taus


@pytest.mark.parametrize("gname", ["ba", "weighted", "rmat12"])
def test_predicted_mre_matches_oracle(gname):
    """The stopping rule on the device against the oracle's formula on the
    same sums and H (a sum in another order: 1e-12 relative); the trees for
    a target follow from it."""
    import synth
    from oracle import apprwc
    from oracle import wilson as ow
    g = {"ba": lambda: synth.ba(2000, 3, seed=0),
         "weighted": lambda: synth.rgg(600, 10.0, seed=2, sigma=0.5),
         "rmat12": lambda: synth.rmat(12, 16, seed=3)}[gname]()
    G = rwc.Graph.from_synth(g)
    T = 300
    sums, _, _, _ = G.sample(T, seed=1)
    H = G.estimate(sums, T)
    m, trees = rwc.rwc_predict_mre(G.handle, sums, T, H, target=0.01)
    want = apprwc.predicted_mre(ow.wdeg(g), G.root, sums.cpu().numpy(), T, H.cpu().numpy())
    assert m == pytest.approx(want, rel=1e-12, abs=0)
    assert abs(trees - apprwc.trees_for(m, T, 0.01)) <= 1

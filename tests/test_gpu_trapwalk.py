"""GPU parity of the straightforward trap-walk estimator (Section 5) with the
oracle: the per-vertex visit totals are integers and must match exactly,
for unit and weighted rows and int64 arc offsets; a walk cut by max_steps is
reported, not hidden."""
import numpy as np
import pytest
import torch

import paper_2510_20604_gb300 as rwc
import synth
from oracle import exact
from oracle import wilson as ow

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("gname,flags", [("ba", 0), ("weighted", 0), ("grid", 0),
                                         ("weighted", rwc.GRAPH_INT64_OFFSETS), ("parallel_arcs", 0)])
def test_trap_walk_counts_bit_exact(gname, flags):
    from _graphs import multigraph
    g = {"parallel_arcs": lambda: multigraph(True),
         "ba": lambda: synth.ba(400, 3, seed=2),
         "weighted": lambda: synth.rgg(300, 9.0, seed=3, sigma=0.8),
         "grid": lambda: synth.grid2d(13, 17)}[gname]()
    G = rwc.Graph.from_synth(g, flags=flags)
    R = 37
    sums = torch.zeros(g.n, dtype=torch.float64, device="cuda")
    steps = rwc.rwc_trap_walks(G.handle, 11, R, sums)
    want, wsteps = ow.Sampler(g, root=G.root, seed=11).trap_walks(R)
    assert np.array_equal(sums.cpu().numpy(), want.astype(np.float64))
    assert steps == wsteps


def test_estimate_from_trap_walks_matches_exact_in_expectation():
    g = synth.ba(300, 2, seed=6)
    G = rwc.Graph.from_synth(g)
    R = 3000
    sums = torch.zeros(g.n, dtype=torch.float64, device="cuda")
    rwc.rwc_trap_walks(G.handle, 5, R, sums)
    t = exact.tdiag(g, G.root)
    keep = np.arange(g.n) != G.root
    mean = sums.cpu().numpy()[keep] / R
    sd = np.sqrt(t[keep] * (t[keep] - 1.0) / R)
    assert (np.abs(mean - t[keep]) / np.maximum(sd, 1e-12)).max() < 5.5


def test_max_steps_is_reported():
    g = synth.path(200)
    G = rwc.Graph.from_synth(g)
    sums = torch.zeros(g.n, dtype=torch.float64, device="cuda")
    with pytest.raises(rwc.RWCError) as e:
        rwc.rwc_trap_walks(G.handle, 1, 4, sums, max_steps=3)
    assert e.value.status == 4

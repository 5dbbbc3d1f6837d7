"""Pins of the straightforward trap-walk estimator (Section 5, before
Wilson's algorithm): a walk from u stopped at the trap v visits u a
geometric number of times whose mean is t_u = (NL_v^-1)_uu (the lemma
connecting t with L_v^-1)."""
import numpy as np
import pytest

import synth
from oracle import exact
from oracle import wilson as ow


def test_star_rooted_at_centre_visits_once():
    g = synth.star(30, center=0)
    s = ow.Sampler(g, seed=2)
    counts, steps = s.trap_walks(50)
    assert counts[0] == 0 and (counts[1:] == 50).all()
    assert steps == 29 * 50


@pytest.mark.parametrize("gname", ["ba", "weighted", "path"])
def test_mean_visits_match_exact_diagonal(gname):
    g = {"ba": lambda: synth.ba(150, 2, seed=3),
         "weighted": lambda: synth.rgg(120, 8.0, seed=4, sigma=0.8),
         "path": lambda: synth.path(12)}[gname]()
    s = ow.Sampler(g, seed=7)
    R = 4000
    counts, _ = s.trap_walks(R)
    t = exact.tdiag(g, s.root)
    keep = np.arange(g.n) != s.root
    mean = counts[keep] / R
    # per-walk visits are geometric on {1, 2, ...} with mean t: variance t (t - 1)
    sd = np.sqrt(t[keep] * (t[keep] - 1.0) / R)
    z = np.abs(mean - t[keep]) / np.maximum(sd, 1e-12)
    assert z.max() < 5.5, z.max()
    # and the pooled error is consistent with those standard deviations
    assert np.mean(z ** 2) < 2.0


def test_threads_do_not_change_counts():
    g = synth.ba(120, 3, seed=1)
    s = ow.Sampler(g, seed=9)
    a, sa = s.trap_walks(300, nthreads=1)
    b, sb = s.trap_walks(300, nthreads=5)
    assert np.array_equal(a, b) and sa == sb

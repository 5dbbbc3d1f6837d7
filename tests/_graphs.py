"""Test graphs built from the synthetic generators (no method arithmetic)."""
import numpy as np

import synth


def multigraph(weighted):
    """A BA graph with some edges doubled or tripled (parallel arcs in both
    rows, each drawn as its own arc, i.e. weights summed)."""
    base = synth.ba(300, 2, seed=7)
    a, b, _ = base.undirected()
    rng = np.random.default_rng(7)
    rep = rng.integers(1, 4, len(a))
    ea = np.repeat(a, rep)
    eb = np.repeat(b, rep)
    src = np.concatenate([ea, eb])
    dst = np.concatenate([eb, ea])
    ww = rng.lognormal(0.0, 0.7, len(ea)).astype(np.float32)
    wts = np.concatenate([ww, ww])
    order = np.lexsort((wts, dst, src))
    src, dst, wts = src[order], dst[order], wts[order]
    rp = np.zeros(base.n + 1, np.int64)
    np.add.at(rp, src + 1, 1)
    rp = np.cumsum(rp)
    return synth.graphs.Graph(base.n, rp, dst.astype(np.int32), wts if weighted else None)

"""Asynchronous sampling (rwc_options_t.async_status = 1) and rwc_sync_status.

An asynchronous call only enqueues its kernels; device-side errors land in
the graph's status word and come back from rwc_sync_status.  The trees are
the same as those of the synchronous call.
"""
import ctypes

import pytest
import torch

import paper_2510_20604_gb300 as rwc
import synth

pytestmark = pytest.mark.gpu


def _sums(G, n, T, opt, seed=3, tree0=0, out=None):
    s = out if out is not None else torch.zeros(n, dtype=torch.float64, device="cuda")
    rwc.rwc_sample_trees(G.handle, seed, tree0, T, s, None, None, opt)
    return s


@pytest.mark.parametrize("gname,mode", [("ba", rwc.MODE_SHARED), ("ba", rwc.MODE_WALKER),
                                        ("grid", rwc.MODE_AUTO), ("weighted_rmat", rwc.MODE_WALKER)])
def test_async_sums_equal_sync_sums(gname, mode):
    g = {"ba": lambda: synth.ba(2000, 3, seed=1),
         "grid": lambda: synth.grid2d(160, 150),          # n > 20000: walker mode
         "weighted_rmat": lambda: synth.rmat(13, 16, seed=2, sigma=1.0)}[gname]()
    G = rwc.Graph.from_synth(g)
    ref = _sums(G, g.n, 40, rwc.Options(mode=mode))
    asy = rwc.Options(mode=mode, async_status=1)
    s = torch.zeros(g.n, dtype=torch.float64, device="cuda")
    assert rwc.rwc_sample_trees(G.handle, 3, 0, 25, s, None, None, asy) is None   # no stats
    _sums(G, g.n, 15, asy, tree0=25, out=s)           # two calls in a row, adding up
    rwc.rwc_sync_status(G.handle)
    assert torch.equal(s, ref)


def test_async_error_is_reported_by_sync_status_once():
    g = synth.grid2d(30, 30)
    G = rwc.Graph.from_synth(g)
    s = _sums(G, g.n, 4, rwc.Options(mode=rwc.MODE_SHARED, max_rounds=2, async_status=1))
    assert s is not None                               # the call itself succeeded
    with pytest.raises(rwc.RWCError) as e:
        rwc.rwc_sync_status(G.handle)
    assert e.value.status == 4 and "max_rounds" in str(e.value)
    rwc.rwc_sync_status(G.handle)                      # cleared
    # the handle stays usable, synchronously and asynchronously
    ref = _sums(G, g.n, 6, rwc.Options(mode=rwc.MODE_SHARED))
    got = _sums(G, g.n, 6, rwc.Options(mode=rwc.MODE_SHARED, async_status=1))
    rwc.rwc_sync_status(G.handle)
    assert torch.equal(got, ref)


def test_async_rejects_statistics_profiling_and_unsupported_modes():
    g = synth.ba(500, 3, seed=3)
    G = rwc.Graph.from_synth(g)
    s = torch.zeros(g.n, dtype=torch.float64, device="cuda")
    L = rwc.lib()
    opt = rwc.Options(async_status=1)
    st = rwc.Stats()
    assert L.rwc_sample_trees(G.handle, 1, 0, 2, s.data_ptr(), None, None, ctypes.byref(opt),
                              ctypes.byref(st), None) == 1
    assert "statistics" in rwc.rwc_last_error()
    for bad, status in ((rwc.Options(async_status=1, profile=1), 1),
                        (rwc.Options(mode=rwc.MODE_GLOBAL, async_status=1), 6),
                        (rwc.Options(mode=rwc.MODE_WALKER, walker_policy=4, async_status=1), 6)):
        with pytest.raises(rwc.RWCError) as e:
            rwc.rwc_sample_trees(G.handle, 1, 0, 2, s, None, None, bad)
        assert e.value.status == status
    rwc.rwc_sync_status(G.handle)
    assert float(s.abs().sum()) == 0.0

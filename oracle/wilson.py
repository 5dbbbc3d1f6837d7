"""ctypes binding of the oracle's sequential Wilson sampler (``wilson.c``).

Test infrastructure only.  Functions follow Algorithm 3 (FastWalk, Section 5)
with RandomNeighbor read from per-vertex successor stacks; see the header of
``wilson.c`` for the exact definition of every step.

Pins (tests/test_oracle_wilson.py): Philox against published known-answer
values and against Triton's Philox; alias tables against the exact encoded
probabilities; trees against structure, against the spanning-tree law by full
enumeration (matrix-tree theorem), against edge marginals w_e R_e (Kirchhoff)
and against independence of the start-node order; visit counts against
Lemma 5.2 (E[visits_u] = (L_v^-1)_uu) and the closed-form star/path cases.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import build as _build

_lib = None

_i64 = ctypes.c_int64
_i32 = ctypes.c_int32
_u32 = ctypes.c_uint32
_u64 = ctypes.c_uint64
_vp = ctypes.c_void_p


def lib():
    global _lib
    if _lib is None:
        path = _build.build()
        L = ctypes.CDLL(path)
        L.oracle_philox4x32_10.argtypes = [_vp, _vp, _vp]
        L.oracle_philox4x32_10.restype = None
        L.oracle_alias_build.argtypes = [_i64, _vp, _vp, _vp, _vp]
        L.oracle_alias_build.restype = ctypes.c_int
        L.oracle_succ.argtypes = [_i64, _vp, _vp, _vp, _vp, _u64, _u32, _i32, _u32, _u32]
        L.oracle_succ.restype = _i32
        L.oracle_wilson.argtypes = [_i64, _vp, _vp, _vp, _vp, _i32, _u64, _u32,
                                    _i64, _i64, ctypes.c_int, _vp, _vp, _vp, _vp]
        L.oracle_wilson.restype = ctypes.c_int
        L.oracle_wilson_order.argtypes = [_i64, _vp, _vp, _vp, _vp, _i32, _u64, _u32,
                                          _u32, _vp, _vp, _vp, _vp]
        L.oracle_wilson_order.restype = _i64
        L.oracle_wdeg.argtypes = [_i64, _vp, _vp, _vp]
        L.oracle_wdeg.restype = None
        L.oracle_rademacher.argtypes = [_i32, _i64, _u64, _vp]
        L.oracle_rademacher.restype = None
        L.oracle_trap_walks.argtypes = [_i64, _vp, _vp, _vp, _vp, _i32, _u64, _i64, _i64,
                                        ctypes.c_int, _vp, _vp]
        L.oracle_trap_walks.restype = ctypes.c_int
        _lib = L
    return _lib


def _p(a):
    return None if a is None else ctypes.c_void_p(a.ctypes.data)


def philox4x32_10(ctr, key):
    c = np.ascontiguousarray(ctr, dtype=np.uint32)
    k = np.ascontiguousarray(key, dtype=np.uint32)
    out = np.zeros(4, np.uint32)
    lib().oracle_philox4x32_10(_p(c), _p(k), _p(out))
    return out


def alias_tables(g):
    """(thr uint32[nnz], alias int32[nnz]) for a weighted graph, None for unit."""
    if g.w is None:
        return None, None
    rp = np.ascontiguousarray(g.row_ptr, np.int64)
    w = np.ascontiguousarray(g.w, np.float32)
    thr = np.zeros(g.nnz, np.uint32)
    al = np.zeros(g.nnz, np.int32)
    if lib().oracle_alias_build(g.n, _p(rp), _p(w), _p(thr), _p(al)) != 0:
        raise MemoryError("oracle alias build")
    return thr, al


def rademacher(k: int, n: int, seed: int) -> np.ndarray:
    """k x n sketch of +-1/sqrt(k) signs drawn from Philox (see wilson.c)."""
    Q = np.zeros((k, n), np.float64)
    lib().oracle_rademacher(int(k), int(n), int(seed), _p(Q))
    return Q


def wdeg(g) -> np.ndarray:
    """Weighted degrees d_u (FP64, each row summed in arc order)."""
    rp = np.ascontiguousarray(g.row_ptr, np.int64)
    w = None if g.w is None else np.ascontiguousarray(g.w, np.float32)
    d = np.zeros(g.n, np.float64)
    lib().oracle_wdeg(g.n, _p(rp), _p(w), _p(d))
    return d


def max_degree_root(g) -> int:
    """Pivot rule of Section 6 ("the node with the highest degree"), read for
    weighted graphs as the largest weighted degree; ties go to the smallest id
    (np.argmax returns the first maximum)."""
    return int(np.argmax(wdeg(g)))


class Sampler:
    """Holds a graph's CSR and alias tables for repeated oracle calls."""

    def __init__(self, g, root=None, seed=1, graph_id=0):
        self.g = g
        self.n = g.n
        self.rp = np.ascontiguousarray(g.row_ptr, np.int64)
        self.col = np.ascontiguousarray(g.col, np.int32)
        self.thr, self.alias = alias_tables(g)
        self.root = max_degree_root(g) if root is None else int(root)
        self.seed = int(seed)
        self.graph_id = int(graph_id)

    def succ(self, u, c, tree):
        return lib().oracle_succ(self.n, _p(self.rp), _p(self.col), _p(self.thr),
                                 _p(self.alias), self.seed, self.graph_id, u, c, tree)

    def sample(self, tree0, ntrees, nthreads=1, want_trees=False):
        """Run trees tree0..tree0+ntrees-1.  Returns dict with 'sums' (FP64
        [n], the integer visit totals), 'draws', and when want_trees the
        'parents' and 'visits' arrays [ntrees][n]."""
        sums = np.zeros(self.n, np.float64)
        par = np.zeros((ntrees, self.n), np.int32) if want_trees else None
        vis = np.zeros((ntrees, self.n), np.int32) if want_trees else None
        draws = np.zeros(1, np.int64)
        st = lib().oracle_wilson(self.n, _p(self.rp), _p(self.col), _p(self.thr),
                                 _p(self.alias), self.root, self.seed, self.graph_id,
                                 int(tree0), int(ntrees), int(nthreads), _p(sums),
                                 _p(par), _p(vis), _p(draws))
        if st != 0:
            raise RuntimeError(f"oracle_wilson status {st}")
        out = {"sums": sums, "draws": int(draws[0])}
        if want_trees:
            out["parents"] = par
            out["visits"] = vis
        return out

    def trap_walks(self, R, max_steps=1 << 40, nthreads=None):
        """Visit counts of the straightforward estimator: for every u != root,
        R walks from u stopped at the root; counts[u] = visits to u over them
        (time 0 included).  Returns (counts int64 [n], total steps)."""
        counts = np.zeros(self.n, np.int64)
        steps = np.zeros(1, np.int64)
        st = lib().oracle_trap_walks(self.n, _p(self.rp), _p(self.col), _p(self.thr), _p(self.alias),
                                     self.root, self.seed, int(R), int(max_steps),
                                     int(nthreads or cores()), _p(counts), _p(steps))
        if st != 0:
            raise RuntimeError(f"oracle_trap_walks status {st}")
        return counts, int(steps[0])

    def tree_with_order(self, tree, order):
        order = np.ascontiguousarray(order, np.int32)
        par = np.zeros(self.n, np.int32)
        vis = np.zeros(self.n, np.int32)
        calls = np.zeros(self.n, np.uint32)
        d = lib().oracle_wilson_order(self.n, _p(self.rp), _p(self.col), _p(self.thr),
                                      _p(self.alias), self.root, self.seed, self.graph_id,
                                      int(tree), _p(order), _p(par), _p(vis), _p(calls))
        if d < 0:
            raise RuntimeError(f"oracle_wilson_order status {d}")
        return par, vis, calls, int(d)


def cores() -> int:
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:  # pragma: no cover
        return os.cpu_count() or 1

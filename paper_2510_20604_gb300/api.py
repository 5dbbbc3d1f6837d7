"""Convenience objects over the C ABI: graph/batch handles that free
themselves, the FastWalk pipeline, and a torch.autograd.Function whose
backward is the library's hand-written gradient.  All computation happens in
librwc.so; this module only allocates torch buffers and forwards pointers."""
from __future__ import annotations

import ctypes

import numpy as np

from . import _binding as B


class _Handle(ctypes.c_void_p):
    """A C handle that keeps the Python object owning it alive: passing
    ``Graph(...).handle`` straight to a call cannot free the graph first."""


class Graph:
    """Device copy of a connected undirected graph (CSR, both arc directions)."""

    def __init__(self, row_ptr, col_idx, w=None, root=-1, flags=0):
        row_ptr = np.ascontiguousarray(row_ptr, np.int64)
        col_idx = np.ascontiguousarray(col_idx, np.int32)
        self.row_ptr, self.col_idx = row_ptr, col_idx
        self.w = None if w is None else np.ascontiguousarray(w, np.float32)
        self._ptr = B.rwc_graph_create(len(row_ptr) - 1, int(row_ptr[-1]), row_ptr, col_idx,
                                       self.w, root, flags)
        self.info = B.rwc_graph_info(self._ptr)

    @property
    def handle(self):
        if not self._ptr:
            raise B.RWCError(1, "graph handle used after close()")
        h = _Handle(self._ptr)
        h.owner = self
        return h

    @classmethod
    def from_synth(cls, g, root=-1, flags=0):
        return cls(g.row_ptr, g.col, g.w, root, flags)

    n = property(lambda self: self.info.n)
    nnz = property(lambda self: self.info.nnz)
    root = property(lambda self: self.info.root)
    vol = property(lambda self: self.info.vol)

    def close(self):
        if getattr(self, "_ptr", None):
            B.rwc_graph_destroy(self._ptr)
            self._ptr = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def sample(self, num_trees, seed=1, tree0=0, sums=None, want_trees=False, opt=None,
               stream=None):
        import torch
        dev = torch.device("cuda")
        if sums is None:
            sums = torch.zeros(self.n, dtype=torch.float64, device=dev)
        par = vis = None
        if want_trees:
            par = torch.empty((num_trees, self.n), dtype=torch.int32, device=dev)
            vis = torch.empty((num_trees, self.n), dtype=torch.int32, device=dev)
        st = B.rwc_sample_trees(self.handle, seed, tree0, num_trees, sums, par, vis, opt, stream)
        return sums, st, par, vis

    def estimate(self, sums, num_trees, tol=1e-10, want_y=False, stream=None):
        import torch
        H = torch.empty(self.n, dtype=torch.float64, device=sums.device)
        y = torch.empty_like(H) if want_y else None
        B.rwc_estimate(self.handle, sums, num_trees, tol, H, y, stream)
        return (H, y) if want_y else H

    def grad(self, c, k=64, sketch_seed=0, tol=1e-8, stream=None):
        import torch
        g = torch.empty(self.nnz // 2, dtype=torch.float32, device=c.device)
        B.rwc_grad(self.handle, c, k, sketch_seed, tol, g, stream)
        return g


def fastwalk(graph: Graph, num_trees: int, seed: int = 1, tol: float = 1e-10, stream=None):
    """Algorithm 3 (FastWalk) with a given tree count: sample, then AppRWC."""
    sums, st, _, _ = graph.sample(num_trees, seed=seed, stream=stream)
    return graph.estimate(sums, num_trees, tol=tol, stream=stream), st


def fastwalk_to_target(graph: Graph, target_mre: float, first_trees: int = 256,
                       max_trees: int = 1 << 22, seed: int = 1, tol: float = 1e-10, stream=None):
    """FastWalk with the variance-law stopping rule: sample ``first_trees``,
    estimate, and while the predicted MRE (rwc_predict_mre) exceeds the target
    add the trees it says are missing (trees continue the same global ids, so
    the result equals one run of the final count).  Returns (H, trees used,
    predicted MRE)."""
    if not target_mre > 0:
        raise ValueError("target_mre must be positive")
    T = max(1, int(first_trees))
    sums, _, _, _ = graph.sample(T, seed=seed, stream=stream)
    while True:
        H = graph.estimate(sums, T, tol=tol, stream=stream)
        mre, need = B.rwc_predict_mre(graph.handle, sums, T, H, target_mre, stream)
        if mre <= target_mre or T >= max_trees:
            return H, T, mre
        extra = min(max(need, T + 1) - T, max_trees - T)
        graph.sample(extra, seed=seed, tree0=T, sums=sums, stream=stream)
        T += extra


def fastwalk_auto(graph: Graph, eps: float, seed: int = 1, max_trees: int = 1 << 26,
                  theta_floor: float = 1e-12, stream=None):
    """Algorithm 3 (FastWalk) with its own parameters: the tree count l of the
    tree-count lemma and the LapSolve accuracy theta of the performance
    theorem, both from rwc_auto_params for the given eps.  theta is used as the
    pivot solve's relative residual, floored at ``theta_floor`` (the FP64
    residual refinement does not reach further).  The lemma's l is a
    worst-case bound that grows as t^2 with t = log(...) / log(lambda): on
    slowly mixing graphs it runs to 1e8 and more trees, so l above
    ``max_trees`` raises ValueError instead of sampling.  Returns (H, params,
    solver tolerance used)."""
    if not 0 < eps:
        raise ValueError("eps must be positive")
    p = B.rwc_auto_params(graph.handle, eps, stream=stream)
    if p.trees > max_trees:
        raise ValueError(f"the tree-count lemma asks for {p.trees} trees at eps={eps} "
                         f"(lambda={p.lambda_:.6f}, t={p.t:.1f}); above max_trees={max_trees}")
    tol = max(float(p.theta), float(theta_floor))
    sums, _, _, _ = graph.sample(int(p.trees), seed=seed, stream=stream)
    H = graph.estimate(sums, int(p.trees), tol=tol, stream=stream)
    return H, p, tol


class Batch:
    def __init__(self, graphs):
        """graphs: sequence of objects with row_ptr, col, w (synth.Graph)."""
        offs = [0]
        rps, cols, ws = [], [], []
        arc = 0
        for g in graphs:
            rps.append(np.asarray(g.row_ptr[:-1], np.int64) + arc)
            cols.append(np.asarray(g.col, np.int32))
            ws.append(g.w)
            arc += int(g.row_ptr[-1])
            offs.append(offs[-1] + g.n)
        rps.append(np.array([arc], np.int64))
        self.G = len(graphs)
        self.offsets = np.array(offs, np.int64)
        self.row_ptr = np.concatenate(rps)
        self.col = np.concatenate(cols)
        w = None if any(x is None for x in ws) else np.concatenate(ws).astype(np.float32)
        self._ptr = B.rwc_batch_create(self.G, self.offsets, self.row_ptr, self.col, w)
        self.N = int(self.offsets[-1])

    @property
    def handle(self):
        if not self._ptr:
            raise B.RWCError(1, "batch handle used after close()")
        h = _Handle(self._ptr)
        h.owner = self
        return h

    def roots(self):
        return B.rwc_batch_roots(self.handle, self.G)

    def sample(self, trees_per_graph, seed=1, sums=None, use_graph=1, per_graph_launch=0,
               stream=None):
        import torch
        if sums is None:
            sums = torch.zeros(self.N, dtype=torch.float64, device="cuda")
        st = B.rwc_batch_sample(self.handle, seed, trees_per_graph, sums, use_graph,
                                per_graph_launch, stream)
        return sums, st

    def autotune(self, cache_path=None, stream=None):
        B.rwc_autotune(self.handle, cache_path, stream)

    def schedule(self):
        """(large-class threads per block, split, trees per item, small class
        warp-per-tree, classes concurrent)."""
        return B.rwc_batch_get_schedule(self.handle)

    def set_schedule(self, threads, split, tile, warp=1, concurrent=1):
        B.rwc_batch_set_schedule(self.handle, threads, split, tile, warp, concurrent)

    def close(self):
        if getattr(self, "_ptr", None):
            B.rwc_batch_destroy(self._ptr)
            self._ptr = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _edge_index(row_ptr, col):
    """For every arc, the index of its undirected edge in (a < b) CSR order.
    Parallel arcs are paired in order: the k-th arc b -> a of a key {a, b}
    gets the edge of the k-th arc a -> b."""
    n = len(row_ptr) - 1
    src = np.repeat(np.arange(n, dtype=np.int64), np.diff(row_ptr))
    dst = col.astype(np.int64)
    up = src < dst
    eid = np.full(len(col), -1, np.int64)
    n_up = int(up.sum())
    eid[up] = np.arange(n_up)

    def keyed(key):
        # arcs sorted by (key, position), and each arc's rank among equal keys
        order = np.argsort(key, kind="stable")
        k = key[order]
        first = np.r_[True, k[1:] != k[:-1]]
        start = np.maximum.accumulate(np.where(first, np.arange(len(k)), 0))
        return order, k, np.arange(len(k)) - start

    o_up, k_up, r_up = keyed(src[up] * n + dst[up])
    o_dn, k_dn, r_dn = keyed(dst[~up] * n + src[~up])
    if not (np.array_equal(k_up, k_dn) and np.array_equal(r_up, r_dn)):
        raise ValueError("arcs are not paired with their reverses")
    dn_idx = np.nonzero(~up)[0]
    eid[dn_idx[o_dn]] = np.arange(n_up)[o_up]
    return eid


def _make_function():
    import torch

    class RWCFunction(torch.autograd.Function):
        """H = FastWalk estimate of the random walk centrality for edge weights
        w (one per undirected edge, (a < b) CSR order).  backward returns the
        gradient of the exact centrality, sum_v g_v dH_v/dw, computed by the
        library (rwc_grad) with a JL sketch of size k (k = 0: exact)."""

        @staticmethod
        def forward(ctx, w, row_ptr, col_idx, num_trees, seed, k, sketch_seed):
            eid = _edge_index(row_ptr, col_idx)
            warc = w.detach().double().cpu().numpy()[eid].astype(np.float32)
            g = Graph(row_ptr, col_idx, warc)
            H, _ = fastwalk(g, num_trees, seed)
            ctx.g, ctx.k, ctx.sketch_seed = g, k, sketch_seed
            ctx.w_device = w.device
            return H.to(w.dtype)

        @staticmethod
        def backward(ctx, gout):
            c = gout.detach().double().contiguous()
            grad = ctx.g.grad(c, ctx.k, ctx.sketch_seed)
            return grad.to(device=ctx.w_device, dtype=gout.dtype), None, None, None, None, None, None

    return RWCFunction


class _Lazy:
    _cls = None

    def __getattr__(self, name):
        if _Lazy._cls is None:
            _Lazy._cls = _make_function()
        return getattr(_Lazy._cls, name)


RWCFunction = _Lazy()

"""Graph generators (see the package docstring for the CSR conventions).

Recipes (all seeds go through numpy's PCG64 ``default_rng`` so the same seed
gives the same graph on every host):

* ``ba(n, m)``: Barabasi-Albert.  Start from the complete graph on m+1 nodes;
  each new node attaches to m distinct earlier nodes, each picked with
  probability proportional to its current degree (a uniform pick from the
  list of all edge endpoints, repeated until m distinct targets are found).
* ``grid2d(r, c)``: 4-neighbour grid, id = i*c + j.
* ``rmat(scale, ef)``: ef * 2^scale / 2 undirected samples; each sample picks
  one quadrant per level with probabilities (a, b, c, d) = (0.57, 0.19, 0.19,
  0.05), the row bit from quadrants c/d and the column bit from b/d.
  Self-loops dropped, duplicates merged, then symmetrised.  Vertex ids are
  not permuted.
* ``rgg(n, kbar)``: n points uniform in the unit square, an edge between
  points closer than r = sqrt(kbar / (pi (n - 1))) (no boundary correction,
  so the realised average degree is slightly below kbar).
* ``er(n, kbar)``: G(n, M) with M ~ Binomial(n(n-1)/2, kbar/(n-1)) uniformly
  drawn pairs; the few colliding pairs are dropped.
* ``add_path``: a random Hamiltonian path (a permutation of the nodes drawn
  from the graph's seed) whose edges are added unless already present, so the
  result is connected.  Path edges draw their weights from the graph's weight
  law (all 1 for unit weights).
* ``lognormal_weights``: FP32 lognormal(0, sigma) weight per undirected edge.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field
from typing import Optional

import numpy as np


@dataclass
class Graph:
    n: int
    row_ptr: np.ndarray          # int64 [n+1]
    col: np.ndarray              # int32 [nnz]
    w: Optional[np.ndarray]      # float32 [nnz] or None (unit weights)
    name: str = ""
    meta: dict = field(default_factory=dict)

    @property
    def nnz(self) -> int:
        return int(self.row_ptr[-1])

    def degrees_unweighted(self) -> np.ndarray:
        return np.diff(self.row_ptr)

    def src(self) -> np.ndarray:
        """Source node of every arc, int64 [nnz]."""
        return np.repeat(np.arange(self.n, dtype=np.int64), np.diff(self.row_ptr))

    def undirected(self):
        """(a, b, w) for every arc with a < b, in CSR arc order."""
        s = self.src()
        m = s < self.col
        w = None if self.w is None else self.w[m]
        return s[m], self.col[m].astype(np.int64), w


def from_edges(n: int, u, v, w=None, name: str = "", meta=None) -> Graph:
    """CSR graph from undirected edges.  Self-loops are dropped; of several
    copies of an edge the first one (in input order) is kept."""
    u = np.asarray(u, dtype=np.int64)
    v = np.asarray(v, dtype=np.int64)
    keep = u != v
    u, v = u[keep], v[keep]
    if w is not None:
        w = np.asarray(w, dtype=np.float32)[keep]
    a = np.minimum(u, v)
    b = np.maximum(u, v)
    key = a * n + b
    # first copy of every key (a stable sort keeps input order among equals),
    # then back into input order
    order = np.argsort(key, kind="stable")
    ks = key[order]
    first = order[np.concatenate(([True], ks[1:] != ks[:-1]))] if len(ks) else order
    first.sort()
    a, b = a[first], b[first]
    if w is not None:
        w = w[first]
    src = np.concatenate([a, b])
    dst = np.concatenate([b, a])
    order = np.argsort(src * n + dst, kind="stable")
    src, dst = src[order], dst[order]
    row_ptr = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(np.bincount(src, minlength=n), out=row_ptr[1:])
    ww = None if w is None else np.concatenate([w, w])[order].astype(np.float32)
    return Graph(n, row_ptr, dst.astype(np.int32), ww, name, dict(meta or {}))


def lognormal_weights(rng, m: int, sigma: float) -> np.ndarray:
    return rng.lognormal(0.0, sigma, size=m).astype(np.float32)


def _weights(rng, m: int, sigma: Optional[float]):
    return None if sigma is None else lognormal_weights(rng, m, sigma)


def add_path(n: int, u, v, w, rng, sigma: Optional[float]):
    """Append the edges of a random Hamiltonian path (existing edges win)."""
    perm = rng.permutation(n).astype(np.int64)
    pu, pv = perm[:-1], perm[1:]
    pw = _weights(rng, n - 1, sigma)
    u2 = np.concatenate([np.asarray(u, np.int64), pu])
    v2 = np.concatenate([np.asarray(v, np.int64), pv])
    w2 = None if w is None else np.concatenate([np.asarray(w, np.float32), pw])
    return u2, v2, w2


# ----------------------------------------------------------------- families

def ba(n: int, m: int = 3, seed: int = 0, sigma: Optional[float] = None,
       with_path: bool = True, name: str = "") -> Graph:
    rng = np.random.default_rng(seed)
    k0 = m + 1
    eu, ev = [], []
    for i in range(k0):
        for j in range(i + 1, k0):
            eu.append(i); ev.append(j)
    rep = np.empty(2 * (len(eu) + m * (n - k0)) + 8, dtype=np.int64)
    nrep = 0
    for a, b in zip(eu, ev):
        rep[nrep] = a; rep[nrep + 1] = b; nrep += 2
    block = rng.random(1 << 16)
    bi = 0
    for i in range(k0, n):
        chosen = []
        while len(chosen) < m:
            if bi == len(block):
                block = rng.random(1 << 16); bi = 0
            t = int(rep[int(block[bi] * nrep)]); bi += 1
            if t not in chosen:
                chosen.append(t)
        for t in chosen:
            eu.append(i); ev.append(t)
            rep[nrep] = i; rep[nrep + 1] = t; nrep += 2
    w = _weights(rng, len(eu), sigma)
    u, v = np.array(eu, np.int64), np.array(ev, np.int64)
    if with_path:
        u, v, w = add_path(n, u, v, w, rng, sigma)
    return from_edges(n, u, v, w, name or f"ba{n}_{m}",
                      {"kind": "ba", "m": m, "seed": seed})


def grid2d(rows: int, cols: int, name: str = "") -> Graph:
    ids = np.arange(rows * cols, dtype=np.int64).reshape(rows, cols)
    u = np.concatenate([ids[:, :-1].ravel(), ids[:-1, :].ravel()])
    v = np.concatenate([ids[:, 1:].ravel(), ids[1:, :].ravel()])
    return from_edges(rows * cols, u, v, None, name or f"grid{rows}x{cols}",
                      {"kind": "grid", "rows": rows, "cols": cols})


def rmat(scale: int, ef: int = 16, seed: int = 0, a=0.57, b=0.19, c=0.19,
         sigma: Optional[float] = None, with_path: bool = True,
         name: str = "") -> Graph:
    n = 1 << scale
    rng = np.random.default_rng(seed)
    nsamp = ef * n // 2
    ta = np.uint64(int(a * 2 ** 32))
    tb = np.uint64(int((a + b) * 2 ** 32))
    tc = np.uint64(int((a + b + c) * 2 ** 32))
    us, vs = [], []
    chunk = 1 << 22
    for s0 in range(0, nsamp, chunk):
        k = min(chunk, nsamp - s0)
        uu = np.zeros(k, dtype=np.int64)
        vv = np.zeros(k, dtype=np.int64)
        # level lvl's draws for the chunk's k samples (one call draws the
        # same stream as `scale` calls of k)
        rr = rng.integers(0, 2 ** 32, size=(scale, k), dtype=np.uint64)
        for lvl in range(scale):
            r = rr[lvl]
            row_bit = r >= tb                      # quadrants c, d
            col_bit = ((r >= ta) & (r < tb)) | (r >= tc)   # quadrants b, d
            sh = np.int64(scale - 1 - lvl)
            uu |= row_bit.astype(np.int64) << sh
            vv |= col_bit.astype(np.int64) << sh
        del rr
        us.append(uu); vs.append(vv)
    u = np.concatenate(us); v = np.concatenate(vs)
    keep = u != v
    u, v = u[keep], v[keep]
    lo, hi = np.minimum(u, v), np.maximum(u, v)
    key = np.sort(lo * n + hi)
    key = key[np.concatenate(([True], key[1:] != key[:-1]))] if len(key) else key
    u, v = key // n, key % n
    w = _weights(rng, len(u), sigma)
    if with_path:
        u, v, w = add_path(n, u, v, w, rng, sigma)
    return from_edges(n, u, v, w, name or f"rmat{scale}",
                      {"kind": "rmat", "scale": scale, "ef": ef, "seed": seed})


def rgg(n: int, kbar: float, seed: int = 0, sigma: Optional[float] = None,
        with_path: bool = True, name: str = "") -> Graph:
    from scipy.spatial import cKDTree
    rng = np.random.default_rng(seed)
    pts = rng.random((n, 2))
    r = math.sqrt(kbar / (math.pi * (n - 1)))
    pairs = cKDTree(pts).query_pairs(r, output_type="ndarray")
    pairs = pairs[np.lexsort((pairs[:, 1], pairs[:, 0]))]
    u, v = pairs[:, 0].astype(np.int64), pairs[:, 1].astype(np.int64)
    w = _weights(rng, len(u), sigma)
    if with_path:
        u, v, w = add_path(n, u, v, w, rng, sigma)
    return from_edges(n, u, v, w, name or f"rgg{n}",
                      {"kind": "rgg", "kbar": kbar, "radius": r, "seed": seed})


def er(n: int, kbar: float, seed: int = 0, sigma: Optional[float] = None,
       with_path: bool = True, name: str = "") -> Graph:
    rng = np.random.default_rng(seed)
    npairs = n * (n - 1) // 2
    p = min(1.0, kbar / (n - 1))
    m = int(rng.binomial(npairs, p))
    u = rng.integers(0, n, size=m, dtype=np.int64)
    v = rng.integers(0, n, size=m, dtype=np.int64)
    w = _weights(rng, m, sigma)
    if with_path:
        u, v, w = add_path(n, u, v, w, rng, sigma)
    return from_edges(n, u, v, w, name or f"er{n}",
                      {"kind": "er", "kbar": kbar, "seed": seed})


# ------------------------------------------------------- small closed forms

def star(n: int, center: int = 0) -> Graph:
    leaves = np.array([i for i in range(n) if i != center], np.int64)
    return from_edges(n, np.full(n - 1, center, np.int64), leaves, None, f"star{n}")


def path(n: int) -> Graph:
    a = np.arange(n - 1, dtype=np.int64)
    return from_edges(n, a, a + 1, None, f"path{n}")


def cycle(n: int) -> Graph:
    a = np.arange(n, dtype=np.int64)
    return from_edges(n, a, (a + 1) % n, None, f"cycle{n}")


def complete(n: int) -> Graph:
    iu = np.triu_indices(n, 1)
    return from_edges(n, iu[0], iu[1], None, f"K{n}")


# ------------------------------------------------------------------ batches

def batch_specs(G: int, seed: int = 0, nmin: int = 50, nmax: int = 20000):
    """Sizes log-uniform in [nmin, nmax] and kinds drawn equally from
    ('er', 'ba', 'rgg') for G graphs."""
    rng = np.random.default_rng(seed)
    sizes = np.floor(np.exp(rng.uniform(math.log(nmin), math.log(nmax), size=G))).astype(np.int64)
    kinds = rng.integers(0, 3, size=G)
    names = ("er", "ba", "rgg")
    return [(int(s), names[int(k)]) for s, k in zip(sizes, kinds)]


def batch_graph(g: int, n: int, kind: str, seed: int = 0) -> Graph:
    s = np.random.SeedSequence([seed, g])
    gseed = int(s.generate_state(1, dtype=np.uint64)[0] >> np.uint64(1))
    if kind == "er":
        return er(n, 8.0, gseed)
    if kind == "ba":
        return ba(n, 2, gseed)
    if kind == "rgg":
        return rgg(n, 10.0, gseed)
    raise ValueError(kind)


def uniform_vector(n: int, seed: int) -> np.ndarray:
    return np.random.default_rng(seed).random(n)

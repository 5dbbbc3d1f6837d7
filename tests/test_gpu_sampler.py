"""GPU parity of the tree sampler against the oracle's sequential Wilson
(Algorithm 3): parents and visit counts must be bit-identical for every tree,
in both sampler modes, on special graphs, generated graphs spanning several
tiles and chunks with ragged tails, weighted graphs (alias tables) and int64
arc offsets; plus sampled trees at the benchmark's full sizes."""
import numpy as np
import pytest
import torch

import paper_2510_20604_gb300 as rwc
import synth
from _graphs import multigraph
from oracle import wilson as ow

pytestmark = pytest.mark.gpu


def run_both(g, T, seed=1, root=-1, tree0=0, opt=None, flags=0):
    G = rwc.Graph.from_synth(g, root=root, flags=flags)
    sums, st, par, vis = G.sample(T, seed=seed, tree0=tree0, want_trees=True, opt=opt)
    ref = ow.Sampler(g, root=G.root, seed=seed).sample(tree0, T, want_trees=True)
    return G, sums.cpu().numpy(), par.cpu().numpy(), vis.cpu().numpy(), ref, st


def assert_exact(g, T, opt, seed=1, root=-1, tree0=0, flags=0):
    G, sums, par, vis, ref, st = run_both(g, T, seed, root, tree0, opt, flags)
    bad = np.nonzero((par != ref["parents"]).any(1) | (vis != ref["visits"]).any(1))[0]
    assert len(bad) == 0, f"{len(bad)} trees differ, first {bad[:5]}"
    assert np.array_equal(sums, ref["sums"])
    return st


SPECIAL = {
    "edge": lambda: synth.path(2),
    "star": lambda: synth.star(40, center=3),
    "path": lambda: synth.path(60),
    "cycle": lambda: synth.cycle(33),
    "K7": lambda: synth.complete(7),
    "grid2x2": lambda: synth.grid2d(2, 2),
    "grid8x8": lambda: synth.grid2d(8, 8),
    "grid5x7": lambda: synth.grid2d(5, 7),
    "weighted": lambda: synth.rgg(80, 6.0, seed=4, sigma=1.0),
}
MODES = {"shared": rwc.Options(mode=rwc.MODE_SHARED),
         "global": rwc.Options(mode=rwc.MODE_GLOBAL),
         "global_nojump": rwc.Options(mode=rwc.MODE_GLOBAL, use_jumps=0),
         "global_chunk3": rwc.Options(mode=rwc.MODE_GLOBAL, trees_per_chunk=3),
         "walker": rwc.Options(mode=rwc.MODE_WALKER),
         "walker_w32_chunk5": rwc.Options(mode=rwc.MODE_WALKER, block_threads=32, trees_per_chunk=5),
         "walker_w1024": rwc.Options(mode=rwc.MODE_WALKER, block_threads=1024),
         "walker_yield": rwc.Options(mode=rwc.MODE_WALKER, walker_policy=1),
         "walker_yield_w32": rwc.Options(mode=rwc.MODE_WALKER, walker_policy=1, block_threads=32),
         "walker_fresh": rwc.Options(mode=rwc.MODE_WALKER, walker_policy=3),
         "walker_fresh_w32": rwc.Options(mode=rwc.MODE_WALKER, walker_policy=3, block_threads=32),
         "walker_park": rwc.Options(mode=rwc.MODE_WALKER, walker_policy=4, max_wait_ns=5_000_000_000),
         "walker_park_chunk4": rwc.Options(mode=rwc.MODE_WALKER, walker_policy=4, trees_per_chunk=4,
                                           max_wait_ns=5_000_000_000)}


@pytest.mark.parametrize("mode", list(MODES))
@pytest.mark.parametrize("gname", list(SPECIAL))
def test_special_graphs_bit_exact(gname, mode):
    assert_exact(SPECIAL[gname](), 37, MODES[mode])


@pytest.mark.parametrize("mode", ["shared", "global", "global_chunk3", "walker", "walker_w32_chunk5",
                                  "walker_fresh", "walker_park"])
def test_small_ba_config_bit_exact(mode):
    """BA n=2000, 3 edges per node + Hamiltonian path, unit weights, 1000
    trees, Philox seed 1: every tree identical to the oracle's."""
    g = synth.ba(2000, 3, seed=0)
    opt = MODES[mode] if mode != "global_chunk3" else rwc.Options(mode=rwc.MODE_GLOBAL, trees_per_chunk=333)
    if mode == "walker_w32_chunk5":
        opt = rwc.Options(mode=rwc.MODE_WALKER, block_threads=32, trees_per_chunk=337)
    assert_exact(g, 1000, opt)


@pytest.mark.parametrize("mode", ["global", "global_nojump", "walker", "walker_w64", "walker_yield",
                                  "walker_wait", "walker_fresh", "walker_park"])
def test_grid_several_chunks_bit_exact(mode):
    g = synth.grid2d(61, 67)
    if mode.startswith("walker"):
        pol = {"walker_yield": 1, "walker_wait": 2, "walker_fresh": 3, "walker_park": 4}.get(mode, 0)
        opt = rwc.Options(mode=rwc.MODE_WALKER, trees_per_chunk=9,
                          block_threads=64 if mode == "walker_w64" else 0, walker_policy=pol)
    else:
        opt = rwc.Options(mode=rwc.MODE_GLOBAL, trees_per_chunk=9,
                          use_jumps=0 if mode == "global_nojump" else -1)
    assert_exact(g, 23, opt, root=-1)


def _king_graph(rows, cols):
    # 8-neighbour grid: degrees 3 to 8, so the walker draws from inline rows of 8
    ids = np.arange(rows * cols).reshape(rows, cols)
    us, vs = [], []
    for dr, dc in ((0, 1), (1, 0), (1, 1), (1, -1)):
        r0, r1 = max(0, -dr), rows - max(0, dr)
        c0, c1 = max(0, -dc), cols - max(0, dc)
        us.append(ids[r0:r1, c0:c1].ravel())
        vs.append(ids[r0 + dr:r1 + dr, c0 + dc:c1 + dc].ravel())
    return synth.from_edges(rows * cols, np.concatenate(us), np.concatenate(vs), name="king")


@pytest.mark.parametrize("mode", ["walker", "walker_w64", "walker_yield", "walker_fresh"])
@pytest.mark.parametrize("gname", ["king", "grid", "cycle"])
def test_bounded_degree_inline_rows_bit_exact(mode, gname):
    # degree <= 4 (grid, cycle) and <= 8 (king graph): the walker's draws pick
    # from inline neighbour rows; several chunks, many trees per chunk
    g = {"king": lambda: _king_graph(45, 53), "grid": lambda: synth.grid2d(70, 41),
         "cycle": lambda: synth.cycle(900)}[gname]()
    pol = {"walker_yield": 1, "walker_fresh": 3}.get(mode, 0)
    opt = rwc.Options(mode=rwc.MODE_WALKER, trees_per_chunk=13,
                      block_threads=64 if mode == "walker_w64" else 0, walker_policy=pol)
    assert_exact(g, 31, opt, root=-1)


def test_weighted_rmat_int64_offsets_bit_exact():
    g = synth.rmat(12, 16, seed=3, sigma=1.0)
    assert_exact(g, 16, rwc.Options(mode=rwc.MODE_GLOBAL), flags=rwc.GRAPH_INT64_OFFSETS)
    assert_exact(g, 8, rwc.Options(mode=rwc.MODE_GLOBAL))
    assert_exact(g, 16, rwc.Options(mode=rwc.MODE_WALKER), flags=rwc.GRAPH_INT64_OFFSETS)
    assert_exact(g, 16, rwc.Options(mode=rwc.MODE_WALKER, block_threads=128))
    assert_exact(g, 16, rwc.Options(mode=rwc.MODE_WALKER, walker_policy=4), flags=rwc.GRAPH_INT64_OFFSETS)


def test_weighted_rgg_shared_bit_exact():
    g = synth.rgg(3000, 12.0, seed=1, sigma=0.5)
    assert_exact(g, 40, rwc.Options(mode=rwc.MODE_SHARED))


def test_tree_offset_and_shards_add_up():
    g = synth.ba(1500, 3, seed=2)
    G = rwc.Graph.from_synth(g)
    a, _, _, _ = G.sample(50, seed=9)
    b, _, _, _ = G.sample(20, seed=9)
    G.sample(30, seed=9, tree0=20, sums=b)
    assert torch.equal(a, b)
    assert_exact(g, 10, rwc.Options(mode=rwc.MODE_GLOBAL), seed=9, tree0=4000000000)
    assert_exact(g, 10, rwc.Options(mode=rwc.MODE_WALKER), seed=9, tree0=4000000000)
    assert_exact(g, 10, rwc.Options(mode=rwc.MODE_WALKER, walker_policy=4), seed=9, tree0=4000000000)


def test_seed_high_bits_matter():
    g = synth.ba(300, 3, seed=2)
    assert_exact(g, 5, rwc.Options(mode=rwc.MODE_SHARED), seed=(7 << 32) | 5)


def test_explicit_root_and_empty_call():
    g = synth.grid2d(10, 10)
    assert_exact(g, 12, rwc.Options(mode=rwc.MODE_SHARED), root=55)
    G = rwc.Graph.from_synth(g)
    s = torch.zeros(g.n, dtype=torch.float64, device="cuda")
    st = rwc.rwc_sample_trees(G.handle, 1, 0, 0, s)
    assert st.trees == 0 and float(s.abs().sum()) == 0.0


@pytest.mark.parametrize("mode", [rwc.MODE_SHARED, rwc.MODE_GLOBAL, rwc.MODE_WALKER])
def test_profiled_call_times_its_phases_and_keeps_the_trees(mode):
    # profile = 1 times the kernels with CUDA events (in GLOBAL mode, inside
    # the captured round graphs); the sums are those of the unprofiled call
    g = synth.grid2d(40, 45)
    G = rwc.Graph.from_synth(g)
    ref, _, _, _ = G.sample(6, opt=rwc.Options(mode=mode))
    s, st, _, _ = G.sample(6, opt=rwc.Options(mode=mode, profile=1))
    assert torch.equal(s, ref)
    assert st.phase_ms[1] > 0 and st.phase_launches[1] >= 1
    if mode == rwc.MODE_GLOBAL:
        assert st.phase_ms[3] > 0 and st.phase_launches[3] == st.phase_launches[1]


def test_max_rounds_reports_not_converged():
    g = synth.grid2d(30, 30)
    G = rwc.Graph.from_synth(g)
    for mode in (rwc.MODE_SHARED, rwc.MODE_GLOBAL):
        with pytest.raises(rwc.RWCError) as e:
            G.sample(4, opt=rwc.Options(mode=mode, max_rounds=2))
        assert e.value.status == 4
        # the handle stays usable afterwards
        assert_exact(g, 3, rwc.Options(mode=mode))
    assert_exact(g, 3, rwc.Options(mode=rwc.MODE_WALKER))


def _check_tree(g, root, par):
    rp, col = g.row_ptr, g.col
    n = g.n
    assert par[root] == -1
    src = np.arange(n)
    m = src != root
    # every parent arc exists
    for u in np.nonzero(m)[0][:: max(1, n // 20000)]:
        assert par[u] in col[rp[u]:rp[u + 1]]
    # acyclic, reaches root: pointer jumping
    p = par.copy()
    p[root] = root
    for _ in range(64):
        p = p[p]
    assert (p == root).all()


def _check_trees_on_device(g, root, par, vis, draws):
    """Properties every sampled tree must have, checked for all trees on the
    device: the root has parent -1 and 0 visits, every other vertex has at
    least one visit and a parent among its neighbours, the visits add up to
    the draws, and following parents from any vertex reaches the root
    (pointer doubling)."""
    dev = par.device
    n = g.n
    # arcs as sorted keys u * n + w (rows ascending, each row sorted)
    keys = torch.as_tensor(g.src().astype(np.int64) * n + g.col.astype(np.int64), device=dev)
    assert bool((keys[1:] >= keys[:-1]).all())
    assert bool((par[:, root] == -1).all()) and bool((vis[:, root] == 0).all())
    nonroot = torch.ones(n, dtype=torch.bool, device=dev)
    nonroot[root] = False
    u = torch.arange(n, device=dev)[nonroot]
    assert int(vis.sum(dtype=torch.int64)) == draws
    for t in range(par.shape[0]):
        assert bool((vis[t, nonroot] >= 1).all()), t
        p = par[t].long()
        want = u * n + p[nonroot]
        pos = torch.clamp(torch.searchsorted(keys, want), max=keys.numel() - 1)
        assert bool((keys[pos] == want).all()), t
        q = p.clone()
        q[root] = root
        for _ in range(24):          # reaches 2^24 > n ancestors
            q = q[q]
        assert bool((q == root).all()), t


@pytest.mark.parametrize("which", ["grid1024", "rmat20"])
def test_full_size_bench_launch_config(which):
    """The benchmark's own launch at full size: 2000 trees resident at once,
    default options (automatic walkers per tree and conflict policy, which
    give 64 walkers and the fresh-start policy for this many trees).  Every
    tree is checked on the device for the spanning-tree properties, four
    chosen trees bit for bit against the oracle's sequential Wilson, and on
    R-MAT 20 the sums of all 2000 trees against the oracle's."""
    g = synth.grid2d(1024, 1024) if which == "grid1024" else synth.rmat(20, 16, seed=0)
    G = rwc.Graph.from_synth(g)
    T = 2000
    sums, st, par, vis = G.sample(T, seed=1, tree0=0, want_trees=True, opt=rwc.Options(profile=1))
    assert st.mode == rwc.MODE_WALKER and st.block_threads == 64 and st.chunks == 1
    s = ow.Sampler(g, root=G.root, seed=1)
    for t in (0, 1, 997, 1999):
        ref = s.sample(t, 1, want_trees=True)
        assert np.array_equal(par[t].cpu().numpy(), ref["parents"][0]), t
        assert np.array_equal(vis[t].cpu().numpy(), ref["visits"][0]), t
    _check_trees_on_device(g, G.root, par, vis, int(st.draws))
    if which == "rmat20":
        ref = s.sample(0, T, nthreads=ow.cores())
        assert np.array_equal(sums.cpu().numpy(), ref["sums"])
    else:
        assert float(sums.sum().item()) == float(st.draws)


@pytest.mark.parametrize("weighted", [False, True])
def test_graph_create_pivot_is_oracle_max_degree_root(weighted):
    """rwc_graph_create's pivot (root = -1): the largest weighted degree, ties
    to the smallest id, as the oracle computes it; on graphs built with tied
    maximum degrees (grids: four-way ties; weighted: equal weight sums at
    several vertices)."""
    cases = [synth.grid2d(7, 9), synth.grid2d(40, 40), synth.ba(500, 3, seed=5)]
    if weighted:
        g0 = synth.grid2d(12, 12)
        # weights from a symmetric function of the endpoints that makes
        # several vertices share the largest weighted degree
        src = g0.src()
        w = (1.0 + ((src % 3) == 0) + ((g0.col % 3) == 0)).astype(np.float32)
        cases = [synth.Graph(g0.n, g0.row_ptr, g0.col, w), synth.rgg(400, 8.0, seed=2, sigma=1.0)]
    for g in cases:
        G = rwc.Graph.from_synth(g)
        d = ow.wdeg(g)
        top = np.nonzero(d == d.max())[0]
        assert G.root == ow.max_degree_root(g) == int(top[0])
        if not weighted:
            assert len(top) > 1 or g.n == 500


@pytest.mark.parametrize("weighted", [False, True])
@pytest.mark.parametrize("mode", ["shared", "global", "walker", "walker_park"])
def test_parallel_arcs_bit_exact(mode, weighted):
    g = multigraph(weighted)
    assert (np.diff(g.col)[np.diff(g.src()) == 0] == 0).any()   # some parallel arcs
    assert_exact(g, 29, MODES[mode])


def test_walker_wait_bound_is_on_progress_not_elapsed_time():
    """The walker's waits fail only after the tree's block stops storing
    vertex words for max_wait_ns.  A 1 ms bound on a long-tailed tree (512 x
    512 grid, 32 walkers, each tree running for far longer than 1 ms, with
    walkers idling at the end while the last walks settle) must still finish,
    and bit-exactly."""
    g = synth.grid2d(512, 512)
    opt = rwc.Options(mode=rwc.MODE_WALKER, block_threads=32, max_wait_ns=1_000_000, profile=1)
    G = rwc.Graph.from_synth(g)
    sums, st, par, vis = G.sample(4, seed=1, tree0=5, want_trees=True, opt=opt)
    assert st.phase_ms[1] > 20.0     # the walker kernel ran far longer than 1 ms
    ref = ow.Sampler(g, root=G.root, seed=1).sample(5, 4, want_trees=True, nthreads=4)
    assert np.array_equal(par.cpu().numpy(), ref["parents"])
    assert np.array_equal(vis.cpu().numpy(), ref["visits"])

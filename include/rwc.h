/*
 * rwc.h -- C ABI of the GB300 FastWalk library (random walk centrality by
 * sampling rooted spanning trees).
 *
 * Paper: "Efficient Algorithms for Computing Random Walk Centrality"
 * (arXiv 2510.20604).  The library implements the data-parallel path of
 * FastWalk (Section 5, Algorithm 3) together with the pivot solve and
 * recovery of Algorithm 1 (AppRWC, Section 3), a gradient of the exact
 * centrality with respect to the edge weights, and a batched sampler for
 * many small graphs.
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 *  - Every function returns an rwc_status; RWC_OK (0) on success.  On any
 *    other value rwc_last_error() returns a message for the calling thread.
 *  - Buffers named host_* are host memory; every other pointer argument is
 *    device memory (for instance a torch tensor's data_ptr()).  The caller
 *    owns all of them.  The library copies graphs into device memory that it
 *    owns and frees in the matching *_destroy call.
 *  - stream is a cudaStream_t (NULL = the legacy default stream).  Work is
 *    enqueued on it; entry points that must inspect device results
 *    (rwc_sample_trees, rwc_sample_trees_noalloc, rwc_estimate,
 *    rwc_pivot_solve, rwc_recover, rwc_solve, rwc_grad, rwc_batch_sample,
 *    rwc_trap_walks, rwc_auto_params, rwc_predict_mre) synchronise
 *    that stream before returning, so their outputs are ready on return and
 *    device-side errors come back as their status.  rwc_sample_trees with
 *    rwc_options_t.async_status = 1 is the exception: it only enqueues, its
 *    status covers argument and launch errors, and device-side errors are
 *    recorded in the graph's status word and returned by rwc_sync_status.
 *  - Graphs are undirected, given as CSR with both arc directions: row u
 *    lists the neighbours of u.  Vertex ids are int32; n >= 2.
 *  - All functions are safe to call from several host threads on distinct
 *    handles; a single handle must not be used concurrently, except that
 *    rwc_pivot_solve (which only reads the graph's arrays) may run on one
 *    thread while the same handle samples on another.
 */
#ifndef RWC_H
#define RWC_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef int32_t rwc_status;
enum {
    RWC_OK = 0,
    RWC_ERR_INVALID = 1,        /* malformed argument or graph */
    RWC_ERR_NOT_CONNECTED = 2,  /* graph has more than one component */
    RWC_ERR_OOM = 3,            /* device or host allocation failed */
    RWC_ERR_NOT_CONVERGED = 4,  /* an iteration cap was reached */
    RWC_ERR_CUDA = 5,           /* a CUDA call failed */
    RWC_ERR_UNSUPPORTED = 6     /* valid request the library cannot serve */
};

typedef struct CUstream_st *rwc_stream_t;   /* same type as cudaStream_t */
typedef struct rwc_graph rwc_graph_t;
typedef struct rwc_batch rwc_batch_t;

/* Flags for rwc_graph_create. */
#define RWC_GRAPH_INT64_OFFSETS 0x1u  /* keep arc offsets as int64 on the device
                                         (always used when nnz >= 2^31) */
#define RWC_GRAPH_SKIP_CONNECTIVITY 0x2u  /* caller guarantees connectivity */

typedef struct {
    int64_t n;          /* vertices */
    int64_t nnz;        /* arcs (2 x undirected edges) */
    int32_t root;       /* pivot v used as the root of every tree */
    int32_t weighted;   /* 1 if weights were given (alias tables built) */
    int32_t offsets64;  /* 1 if arc offsets are int64 on the device */
    int32_t reserved;
    double vol;         /* sum of weighted degrees (the paper's 2m) */
    double dmax;        /* largest weighted degree */
    int64_t device_bytes;  /* device memory held by the graph */
} rwc_graph_info_t;

/* Sampler modes for rwc_options_t.mode. */
#define RWC_MODE_AUTO 0
#define RWC_MODE_GLOBAL 1   /* rounds over tree chunks, state in HBM */
#define RWC_MODE_SHARED 2   /* one thread block per tree, state in shared memory */
#define RWC_MODE_WALKER 3   /* concurrent Wilson walkers, one block per tree, state in HBM */

typedef struct {
    int32_t mode;             /* RWC_MODE_*; AUTO picks SHARED when the tree fits in
                                 shared memory, WALKER otherwise */
    int32_t max_rounds;       /* cap on popping rounds per chunk (0 = 1<<22) */
    int64_t trees_per_chunk;  /* GLOBAL/WALKER: trees resident at once (0 = auto) */
    int32_t use_jumps;        /* GLOBAL mode: 1 = jump pointers (default), 0 = off,
                                 -1 = default */
    int32_t block_threads;    /* SHARED: block size; WALKER: walkers per tree, at most
                                 512 (0 = auto) */
    int64_t memory_budget;    /* GLOBAL/WALKER: bytes of scratch to use (0 = auto) */
    int32_t profile;          /* 1 = time every kernel launch with CUDA events on
                                 the call's stream (fills rwc_stats_t.phase_*);
                                 2 = also count walker loop iterations per state
                                 (rwc_stats_t.diag; slower kernel variant) */
    int32_t walker_policy;    /* WALKER mode, when a walk runs into an earlier
                                 walk's path: 0 = default (3 when a tree has at
                                 most 64 walkers, else 1), 1 = yield (free the
                                 path, requeue, wait for the earlier walk to move
                                 on), 2 = wait (keep the path until the vertex
                                 changes owner), 3 = yield and take a fresh start
                                 at once while fresh starts remain (the wait of 1
                                 once only requeued starts are left), 4 = park:
                                 the later walk keeps its path, hung at the
                                 contested vertex, and its thread takes other
                                 work; the earlier walk takes the later path's
                                 suffix over (no path is released; 64 walkers
                                 per tree, 48 B of state per tree-vertex) */
    int64_t max_wait_ns;      /* WALKER mode: a wait inside the sampler fails with
                                 RWC_ERR_NOT_CONVERGED once its thread block (one
                                 tree) has stored no vertex word for this many
                                 nanoseconds (0 = 30 s); the bound is on a lack of
                                 progress, not on the length of any one wait */
    int32_t async_status;     /* 1 = return without synchronising the stream:
                                 device-side errors go to the graph's status
                                 word, read by rwc_sync_status.  WALKER (policies
                                 0-3) and SHARED modes only, with stats = NULL
                                 and profile = 0 (RWC_ERR_INVALID otherwise) */
    int32_t reserved;
} rwc_options_t;

/* Sampler phases reported in rwc_stats_t.  GLOBAL mode: INIT, WALK, POP
 * (classification is part of POP), ACCUM.  WALKER mode: INIT, WALK (the walker
 * kernel), ACCUM.  SHARED mode reports its single kernel as WALK. */
#define RWC_PHASE_INIT 0      /* first successor of every vertex */
#define RWC_PHASE_WALK 1      /* marked vertex -> next marked or settled vertex */
#define RWC_PHASE_CLASSIFY 2  /* cycle leaders on the compressed graph */
#define RWC_PHASE_POP 3       /* pop cycles: new successor draws */
#define RWC_PHASE_FINISH 4    /* return unpopped marks to the free pool */
#define RWC_PHASE_ACCUM 5     /* visits into FP64 sums, optional tree output */
#define RWC_NPHASE 6

typedef struct {
    int64_t trees;        /* trees sampled by the last call */
    int64_t draws;        /* successor draws (= sum of visits over all trees) */
    int64_t rounds;       /* GLOBAL/SHARED: popping rounds; WALKER: yielded walks
                             (counted with rwc_options_t.profile = 2 only) */
    int64_t walk_steps;   /* GLOBAL: pointer-chasing steps; WALKER: walker steps
                             (profile = 2 only) */
    int64_t chunks;       /* tree chunks processed */
    int32_t mode;         /* mode actually used */
    int32_t block_threads; /* WALKER: walkers (threads) per tree of the last chunk */
    int64_t marked;       /* compressed-graph nodes over all rounds (= draws) */
    /* with rwc_options_t.profile: device time (ms), launches and work units
     * per phase; units are vertices (INIT, ACCUM), pointer-chasing steps (WALK
     * in GLOBAL mode), successor draws (POP in GLOBAL mode; WALK in WALKER and
     * SHARED modes) and marked entries (CLASSIFY). */
    double phase_ms[RWC_NPHASE];
    int64_t phase_launches[RWC_NPHASE];
    int64_t phase_units[RWC_NPHASE];
    /* diagnostics; WALKER mode with profile = 2: [0..6] loop iterations
     * summed over all walkers in the states idle, walk, pop, release, settle,
     * wait-for-yield, wait-after-yield (or wait for an earlier walk's vertex);
     * [7] loop iterations summed over warps */
    int64_t diag[8];
} rwc_stats_t;

/* Message describing the last error on the calling thread ("" if none). */
const char *rwc_last_error(void);

/* Library version string. */
const char *rwc_version(void);

/* Number of CUDA kernel launches this library has issued in this process
 * (diagnostics; monotone, all threads). */
int64_t rwc_launch_count(void);

/*
 * Graph store (Section 2.2: G = (V, E), degrees, L = D - A; weighted reading:
 * d_u = sum of the weights of u's arcs, vol = sum_u d_u plays the role of 2m,
 * the walk moves from u to w with probability w_uw / d_u).
 *
 * host_row_ptr: int64 [n+1], row_ptr[0] = 0, non-decreasing, row_ptr[n] = nnz.
 * host_col_idx: int32 [nnz], neighbours of each row sorted ascending.
 * host_w:       float [nnz] positive finite weights, or NULL for unit weights.
 *               Arc (u,w) and arc (w,u) must carry equal weights.
 * root:         pivot v; -1 selects the vertex of largest weighted degree
 *               with ties to the smallest id (Section 6: "the node with the
 *               highest degree is selected as the pivot").
 * Validation: n >= 2, sorted rows, every arc has its reverse with equal
 * weight (repeated arcs are allowed and act as one edge of summed weight),
 * no self-loops, finite positive weights, connected (one BFS) unless
 * RWC_GRAPH_SKIP_CONNECTIVITY.  Returns RWC_ERR_INVALID or
 * RWC_ERR_NOT_CONNECTED without allocating on failure.
 * Weighted graphs get one Vose alias table per row, built on the host in
 * FP64 and stored on the device next to the arcs (16 B per arc).
 */
rwc_status rwc_graph_create(int64_t n, int64_t nnz, const int64_t *host_row_ptr,
                            const int32_t *host_col_idx, const float *host_w,
                            int32_t root, uint32_t flags, rwc_graph_t **out);
rwc_status rwc_graph_info(const rwc_graph_t *g, rwc_graph_info_t *host_out);
rwc_status rwc_graph_destroy(rwc_graph_t *g);

/*
 * Sample rooted spanning trees (Section 5, Algorithm 3, the loop over
 * i = 1..l) and accumulate each vertex's visit count.
 *
 * Tree i (i = tree0 .. tree0 + num_trees - 1) is the tree that Wilson's
 * algorithm rooted at the pivot produces when the c-th call of
 * RandomNeighbor(u) in that tree returns succ(u, c, i): Philox-4x32-10 with
 * counter (c, u, i, 0) and key (seed & 0xffffffff, seed >> 32), arc index
 * j = floor(o0 * deg(u) / 2^32), and for weighted graphs arc j kept when
 * o1 < thr_j, else its alias.  The result does not depend on the order in
 * which start nodes are processed (Wilson's cycle-popping theorem), so the
 * parallel sampler reproduces the sequential algorithm exactly.
 *
 * sums:    FP64 [n]; sums[u] += sum over the trees of visits_u (exact
 *          integers), where visits_u is Algorithm 3's count for u (the number
 *          of RandomNeighbor(u) calls); sums[root] is unchanged.
 * parents: NULL or int32 [num_trees][n]; parent of u in tree tree0+t,
 *          -1 for the root.
 * visits:  NULL or int32 [num_trees][n]; per-tree visit counts (0 at root).
 * opt:     NULL for defaults.  stats: NULL or host struct filled on return.
 * Requires tree0 + num_trees <= 2^32.  Returns RWC_ERR_NOT_CONVERGED if
 * max_rounds is reached (outputs then undefined).  Synchronises stream.
 */
rwc_status rwc_sample_trees(rwc_graph_t *g, uint64_t seed, int64_t tree0,
                            int64_t num_trees, double *sums, int32_t *parents,
                            int32_t *visits, const rwc_options_t *opt,
                            rwc_stats_t *stats, rwc_stream_t stream);

/*
 * Device-side status of the asynchronous calls on g (rwc_options_t.
 * async_status = 1).  Synchronises stream, then reads and clears g's status
 * word, which every asynchronous sampling call ORs its device-side errors
 * into as its last step on its stream: RWC_ERR_UNSUPPORTED (a pop count
 * overflowed), RWC_ERR_CUDA (an internal check failed), RWC_ERR_NOT_CONVERGED
 * (a walker wait ran out, or max_rounds was reached in SHARED mode), in that
 * order of precedence; the outputs of the failed call are undefined.  Errors
 * of calls still running on other streams are reported by a later call once
 * those streams are synchronised.  Not a counterpart of any step of the
 * paper: it completes the asynchronous form of rwc_sample_trees.
 */
rwc_status rwc_sync_status(rwc_graph_t *g, rwc_stream_t stream);

/*
 * rwc_sample_trees without any allocation (the paper has no counterpart).
 *
 * For callers that cannot allocate device memory while they sample:
 * real-time or embedded hosts that allow no allocation after start-up (an
 * allocation can block or fail at an unpredictable moment), and processes
 * whose device memory pool is exhausted or owned by another allocator that
 * the library cannot draw from.  It samples the
 * same trees as rwc_sample_trees (identical sums, parents and visits; the
 * concurrent-walker sampler) but keeps all of its scratch in one static
 * device array of RWC_NOALLOC_SCRATCH_BYTES inside this library, which every
 * GPU that loads the library holds until the process exits.  It calls no
 * cudaMalloc, cudaFree or other allocating routine; the caller still passes
 * the graph (already on the device) and the output buffers.
 *
 * Limits and rules:
 *  - One tree needs 12 n bytes plus 4 n for the start order; a graph that
 *    does not fit (n above roughly 2 million) gets RWC_ERR_INVALID.  Trees
 *    are processed in as many chunks as the array requires.
 *  - The first call on a device looks up the array's device address
 *    (cudaGetSymbolAddress) once, with that device current.
 *  - Every call on a device shares the one array, which keeps the last call's
 *    contents (the call clears what must start at zero); calls that overlap
 *    on the GPU (other streams, other host threads) race and corrupt each
 *    other: serialise them.
 * Arguments as for rwc_sample_trees; synchronises stream.
 */
#define RWC_NOALLOC_SCRATCH_BYTES (32u << 20)
rwc_status rwc_sample_trees_noalloc(rwc_graph_t *g, uint64_t seed, int64_t tree0,
                                    int64_t num_trees, double *sums, int32_t *parents,
                                    int32_t *visits, rwc_stream_t stream);

/*
 * Algorithm 1 (AppRWC) fed by the estimator of Section 5.
 *   t_u = sums[u] / num_trees                        (estimate of (NL_v^-1)_uu)
 *   b   = sqrt(d_v) e_v - (sqrt(d_v) / vol) d        (right-hand side)
 *   z   = L^+ b by Jacobi-preconditioned CG to relative residual cg_tol
 *         (the paper's LapSolve; FP32 SpMV inner solves, FP64 residual
 *         refinement, z kept in FP64)
 *   y_u = sqrt(d_u) z_u - sqrt(d_u) (sum_w d_w z_w) / vol   (pivot column)
 *   H_u = (t_u - (d_u/d_v) y_v + 2 sqrt(d_u/d_v) y_u) / pi_u, u != v (Eq. 3)
 *   H_v = y_v / pi_v
 * sums: FP64 [n] device; H_out: FP64 [n] device; y_out: NULL or FP64 [n].
 * cg_tol <= 0 selects 1e-10.  Returns RWC_ERR_NOT_CONVERGED if the solver
 * stalls.  Synchronises stream.
 */
rwc_status rwc_estimate(rwc_graph_t *g, const double *sums, int64_t num_trees,
                        double cg_tol, double *H_out, double *y_out,
                        rwc_stream_t stream);

/*
 * The pivot column of Algorithm 1 alone: the steps of rwc_estimate before the
 * recovery (b, z = L^+ b, y), which depend on the graph only and not on the
 * sampled trees, so that they can run while the trees are sampled (on
 * another stream, or once for many estimates of the same graph).  y: FP64
 * [n] device, the same bits as rwc_estimate's y_out for the same cg_tol;
 * rwc_recover(g, sums, num_trees, y, H) then gives rwc_estimate's H.
 * cg_tol <= 0 selects 1e-10.  Returns RWC_ERR_NOT_CONVERGED if the solver
 * stalls.  Synchronises stream.
 */
rwc_status rwc_pivot_solve(rwc_graph_t *g, double cg_tol, double *y, rwc_stream_t stream);

/*
 * Recovery step only (Algorithm 1, the recovery of H from t and y) for a given pivot column y
 * (FP64 [n] device): H from sums/num_trees and y as in rwc_estimate.
 */
rwc_status rwc_recover(rwc_graph_t *g, const double *sums, int64_t num_trees,
                       const double *y, double *H_out, rwc_stream_t stream);

/*
 * Laplacian solve used by rwc_estimate and rwc_grad: X = L^+ B for k
 * right-hand sides (block CG, Jacobi preconditioner, FP32 SpMM, FP64 dots
 * and FP64 residual refinement; each column's mean is removed first).
 * B, X: FP64 [k][n] device (column-major by right-hand side), may not alias.
 * iters_out: NULL or host int, outer+inner iterations used.
 */
rwc_status rwc_solve(rwc_graph_t *g, int32_t k, const double *B, double *X,
                     double tol, int32_t *iters_out, rwc_stream_t stream);

/*
 * Gradient of J(w) = sum_v c_v H_v(w) with respect to each undirected edge
 * weight, H the exact random walk centrality (Section 2.3,
 * H_v = vol L^+_vv - 2 (L^+ d)_v + d^T L^+ d / vol).  For edge e = (a, b),
 * with x = L^+ c, y = L^+ d, Z = Q C^1/2 L^+:
 *   dJ/dw_e = 2 tr(C L^+) - vol sum_i (Z_ia - Z_ib)^2
 *             + 2 (x_a - x_b)(y_a - y_b) - 2 (x_a + x_b)
 *             + (sum c) [ (2 (y_a + y_b) - (y_a - y_b)^2) / vol - 2 d^T y / vol^2 ]
 * and tr(C L^+) estimated by tr(Z C^1/2 Q^T).  Q (k x n) is the
 * Johnson-Lindenstrauss sketch: Q_iu = +-1/sqrt(k), the sign the top bit of
 * Philox output o0 for counter (i, u, 0xFFFFFFFF, 0) and key sketch_seed;
 * k = 0 means Q = I (exact, k = n right-hand sides; n <= 16384, else
 * RWC_ERR_UNSUPPORTED).  Every sum of the solve and of the assembly is taken
 * in a fixed order, so the same input gives the same bits on every call.
 * c: FP64 [n] device, any signs: the term sum_u c_u (L^+ b_e)_u^2 and
 * tr(C L^+) are linear in c, so negative entries get their own k sketch
 * columns with C^1/2 replaced by (max(-c, 0))^1/2 and enter with sign -
 * (the solve then has 2k + 2 right-hand sides).  grad_w: FP32 [nnz/2] device, one entry per
 * undirected edge in the order of arcs (a, b) with a < b in CSR order (the
 * repeated arcs of a multi-edge each get the same value).
 * Synchronises stream.
 */
rwc_status rwc_grad(rwc_graph_t *g, const double *c, int32_t k,
                    uint64_t sketch_seed, double cg_tol, float *grad_w,
                    rwc_stream_t stream);

/*
 * Batched sampler: many independent small graphs, all trees of all graphs in
 * one persistent launch (captured in a CUDA graph when use_graph != 0).
 * Graphs with more vertices than the schedule's split run one tree per thread
 * block, the others one tree per warp (several trees per block) or per small
 * block; see rwc_batch_set_schedule and rwc_autotune.
 * host_graph_offsets: int64 [G+1] vertex offsets of each graph inside the
 * concatenated CSR; host_row_ptr: int64 [N+1] with global arc offsets;
 * host_col_idx: int32 [nnz] LOCAL vertex ids (0..n_g-1); host_w NULL (unit
 * weights) or float [nnz].  Every graph is validated as in rwc_graph_create
 * and rooted at its own max-degree vertex.  Graph g's trees use Philox
 * counter word 3 = g, so graph g of a batch reproduces rwc_sample_trees on
 * that graph alone only for g = 0; the oracle reproduces every graph.
 */
rwc_status rwc_batch_create(int32_t G, const int64_t *host_graph_offsets,
                            const int64_t *host_row_ptr,
                            const int32_t *host_col_idx, const float *host_w,
                            rwc_batch_t **out);
/* sums: FP64 [N] device (per-vertex, graph g's block at its vertex offset),
 * accumulated.  per_graph_launch != 0 issues one launch per graph instead of
 * the persistent kernel (the baseline it is compared with).  roots_out: NULL
 * or host int32 [G]. */
rwc_status rwc_batch_sample(rwc_batch_t *b, uint64_t seed, int64_t trees_per_graph,
                            double *sums, int32_t use_graph, int32_t per_graph_launch,
                            rwc_stats_t *stats, rwc_stream_t stream);
rwc_status rwc_batch_roots(const rwc_batch_t *b, int32_t *host_roots);
/* Choose the schedule (block size, split between block-per-tree and
 * warp-per-tree, trees per work item) for this batch by timing candidates on
 * the device; the choice is cached in cache_path (JSON, may be NULL) under a
 * signature of the batch's sizes.  Synchronises stream. */
rwc_status rwc_autotune(rwc_batch_t *b, const char *cache_path, rwc_stream_t stream);
/* The batch's schedule.  threads: block size of the large class (graphs with
 * more than split vertices, one tree per block; a multiple of 32, <= 1024);
 * split: the largest n of the small class (0: one class); warp: 1 = the small
 * class runs one tree per warp (8 trees per 256-thread block), 0 = one tree
 * per 256-thread block; tile: trees per work item; concurrent: 1 = the two
 * classes' persistent kernels run on forked streams at the same time, 0 = one
 * after the other (both inside the call's one CUDA graph).  set returns
 * RWC_ERR_UNSUPPORTED when a class needs more than 227 KB of shared memory
 * per block (a tree of n vertices takes 11 n + 64 bytes).  host_sched: int32
 * [5] = {threads, split, tile, warp, concurrent}.  Schedules do not change the
 * trees. */
rwc_status rwc_batch_get_schedule(const rwc_batch_t *b, int32_t *host_sched);
rwc_status rwc_batch_set_schedule(rwc_batch_t *b, int32_t threads, int32_t split, int32_t tile,
                                  int32_t warp, int32_t concurrent);
rwc_status rwc_batch_destroy(rwc_batch_t *b);

/*
 * The straightforward estimator of Section 5 (the one Wilson's algorithm
 * improves on), for comparison: t_u = (NL_v^-1)_uu is the expected number of
 * visits to u of a random walk from u stopped when it meets the pivot v
 * (time 0 included).  For every u != v and r < walks_per_node, one such walk;
 * sums[u] += its visits to u, so that sums / walks_per_node estimates the same
 * t as the tree sampler's sums / num_trees (and can be passed to rwc_estimate
 * with num_trees = walks_per_node).  Step s of walk (u, r) moves by the tree
 * sampler's RandomNeighbor rule with Philox counter (s, u, r, 0xFFFFFFFE) and
 * key = seed.  walks_per_node in [0, 2^32], max_steps in [1, 2^32]: a walk
 * longer than max_steps ends the call with RWC_ERR_NOT_CONVERGED.
 * sums: FP64 [n] device, accumulated.  host_steps: NULL or total steps taken.
 * Synchronises stream.
 */
rwc_status rwc_trap_walks(rwc_graph_t *g, uint64_t seed, int64_t walks_per_node,
                          int64_t max_steps, double *sums, int64_t *host_steps,
                          rwc_stream_t stream);

/*
 * Automatic parameters (Section 5, "The Sampling Algorithm": the sample size
 * of the tree-count lemma and the solver accuracy of the performance theorem).
 *
 *   lambda = spectral radius of P_v (D^-1 W without the pivot's row and
 *            column), by inverse iteration on the normalised grounded
 *            Laplacian I - D^-1/2 W D^-1/2 restricted to V \ {v}; mu = 1 - lambda
 *   diameter = BFS double sweep from the pivot (a lower bound on Delta,
 *            exact on trees and grids); sweep_end = the vertex it starts the
 *            second sweep from (farthest from the pivot, smallest id on ties)
 *   t      = log(m / (n sqrt(n-1) |d_-v|_2)) / log(lambda), at least 1
 *            (m = vol / 2; walks longer than t are rarer than 1/n)
 *   trees  = ceil(2 t^2 log(2n) / eps^2)
 *   theta  = eps / (2 Delta d_max (1 + d_max (1 + n) / (2m))^2 sqrt(m n Delta))
 *
 * max_iters (<= 0: 30) and tol (<= 0: 1e-9) bound the inverse iteration,
 * which stops when mu changes by at most tol relative.  Each iteration is one
 * Laplacian solve.  Synchronises stream.
 */
typedef struct {
    double lambda;
    double mu;
    double t;
    double theta;
    int64_t trees;
    int64_t diameter;
    int32_t sweep_end;
    int32_t iterations;
} rwc_params_t;

rwc_status rwc_auto_params(rwc_graph_t *g, double eps, int32_t max_iters, double tol,
                           rwc_params_t *out, rwc_stream_t stream);

/*
 * Evaluation measures (Section 6, "Evaluation Measures" and "Approximation
 * Quality").
 *
 * rwc_mre: mean relative error (1/n) sum_u |H_u - H_est_u| / H_u of an
 * estimate against a reference.  H, H_est: device FP64 [n], H_u != 0.
 * out: device FP64 scalar, written (not accumulated).  The reduction order is
 * fixed, so repeated calls give identical results.  n >= 1.  Asynchronous on
 * stream.
 */
rwc_status rwc_mre(int64_t n, const double *H, const double *H_est, double *out,
                   rwc_stream_t stream);

/*
 * rwc_predict_mre: the stopping rule of the variance law of the visit counts.
 * Per tree, visits_u is geometric with mean t_u, so t~_u = sums_u / T has
 * variance t_u (t_u - 1) / T, and H~_u = (t~_u - ...) / pi_u carries that
 * error over pi_u (H~_v carries none); a normal error of standard deviation s
 * has mean absolute value sqrt(2/pi) s.  With t_u replaced by its estimate:
 *   mre   = (1/n) sum_{u != v} sqrt(2/pi) sqrt(t~_u (t~_u - 1) / T) / (pi_u |H_u|)
 *   trees = ceil(T (mre / target)^2), the trees for a target error
 * sums: FP64 [n] device (the visit totals of num_trees trees); H: FP64 [n]
 * device (rwc_estimate's output).  host_mre: host double; host_trees: NULL or
 * host int64, written when target > 0.  Synchronises stream.
 */
rwc_status rwc_predict_mre(rwc_graph_t *g, const double *sums, int64_t num_trees, const double *H,
                           double target, double *host_mre, int64_t *host_trees,
                           rwc_stream_t stream);

/*
 * rwc_kendall: Kendall distance of the rankings given by a and b,
 * K = 2 (alpha - beta) / (n (n - 1)), alpha / beta the concordant /
 * discordant pairs; a pair tied in a or in b counts neither way (Kendall's
 * tau-a).  a, b: device FP64 [n], no NaN (-0.0 equals +0.0).  out_diff:
 * device int64 scalar, written with alpha - beta (exact).  host_tau: NULL, or
 * a host double receiving K (then the call synchronises stream).  Every pair
 * is compared, O(n^2) work: 0 <= n <= 2^26.
 */
rwc_status rwc_kendall(int64_t n, const double *a, const double *b, int64_t *out_diff,
                       double *host_tau, rwc_stream_t stream);

#ifdef __cplusplus
}
#endif

#endif /* RWC_H */

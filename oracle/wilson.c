/*
 * ORACLE -- test infrastructure only.
 *
 * Plain, sequential CPU implementation of the FastWalk tree-sampling loop.
 * Only tests/, __graft_entry__.smoke() and bench.py's CPU-baseline legs may
 * load this library.  It shares no code, header or table with the CUDA path.
 *
 * What it computes, and where each piece is defined:
 *
 *  - philox4x32_10: the counter-based generator Philox-4x32 with 10 rounds,
 *    written from its published definition (Salmon, Moraes, Dror, Shaw,
 *    "Parallel random numbers: as easy as 1, 2, 3", SC'11, Section 3.1: the
 *    Philox S-box built from two 32x32->64 multiplies, the bijection on
 *    (X0,X1,X2,X3), and the Weyl key schedule).
 *
 *  - alias_build: Vose's alias method per CSR row (weighted graphs).  The
 *    paper is unweighted (Section 2.2); a weighted neighbour pick is our
 *    reading of RandomNeighbor for weighted graphs.  The exact procedure
 *    (FP64, FIFO work lists, uint32 thresholds) is fixed so that every
 *    implementation produces identical tables.
 *
 *  - succ(u, c, tree): the c-th entry of u's successor stack, i.e. the
 *    neighbour returned by the c-th call of RandomNeighbor(u) in this tree
 *    (Algorithm 3, the line "Next[u] <- RandomNeighbor(u)").  Philox counter
 *    = (c, u, tree, graph), key = (seed lo, seed hi); arc index j =
 *    floor(o0 * deg / 2^32); weighted rows keep j when o1 < thr[j], else take
 *    alias[j].
 *
 *  - wilson_tree: one iteration of Algorithm 3's outer loop: Wilson's
 *    algorithm rooted at the pivot v, start nodes in ascending id order
 *    (the "arbitrary ordering" of Algorithm 3), with the visit counting of
 *    Algorithm 3 kept as integers (+1 at the start node, +1 on each arrival,
 *    -1 at the in-tree endpoint); the 1/l scaling is applied once by the
 *    caller (Section 5, the estimator t~_u = sum_i t~_ui / l).
 *
 *  - trap_walks: the straightforward estimator Section 5 starts from (walks
 *    from every u stopped at the pivot, counting their visits to u), with
 *    Philox counter (step, u, walk, 0xFFFFFFFE) and the RandomNeighbor rule
 *    of succ().
 *
 * Build: gcc -O2 -ffp-contract=off -fPIC -shared -pthread (see build.py).
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <math.h>
#include <pthread.h>

/* ---------------------------------------------------------------- Philox */

static void mulhilo32(uint32_t a, uint32_t b, uint32_t *hi, uint32_t *lo)
{
    uint64_t p = (uint64_t)a * (uint64_t)b;
    *hi = (uint32_t)(p >> 32);
    *lo = (uint32_t)p;
}

/* Philox-4x32-10: ten rounds; the key is bumped by the Weyl constants
 * before every round but the first. */
void oracle_philox4x32_10(const uint32_t ctr_in[4], const uint32_t key_in[2],
                          uint32_t out[4])
{
    const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u;
    const uint32_t W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
    uint32_t x0 = ctr_in[0], x1 = ctr_in[1], x2 = ctr_in[2], x3 = ctr_in[3];
    uint32_t k0 = key_in[0], k1 = key_in[1];
    for (int r = 0; r < 10; ++r) {
        if (r > 0) { k0 += W0; k1 += W1; }
        uint32_t hi0, lo0, hi1, lo1;
        mulhilo32(M0, x0, &hi0, &lo0);
        mulhilo32(M1, x2, &hi1, &lo1);
        uint32_t y0 = hi1 ^ x1 ^ k0;
        uint32_t y1 = lo1;
        uint32_t y2 = hi0 ^ x3 ^ k1;
        uint32_t y3 = lo0;
        x0 = y0; x1 = y1; x2 = y2; x3 = y3;
    }
    out[0] = x0; out[1] = x1; out[2] = x2; out[3] = x3;
}

/* ----------------------------------------------------------- alias tables */

/* Vose's alias method for the arcs of one row, exactly as fixed for this
 * project:
 *   S   = sum of w_j in arc order (FP64)
 *   p_j = (w_j * deg) / S (FP64)
 *   small = {j : p_j < 1}, large = {j : p_j >= 1}, both FIFO in ascending j
 *   while both non-empty: s = pop(small); l = front(large);
 *       thr_s = p_s, alias_s = l; p_l = (p_l + p_s) - 1;
 *       if p_l < 1: move l from the front of large to the back of small
 *   every entry left in either list: probability 1, alias = itself
 *   thr (uint32) = min(floor(p * 2^32), 2^32 - 1); 2^32 - 1 for the leftovers
 * Returns 0, or -1 on allocation failure. */
static int alias_row(int64_t deg, const float *w, uint32_t *thr, int32_t *alias,
                     double *p, int64_t *small, int64_t *large)
{
    double S = 0.0;
    for (int64_t j = 0; j < deg; ++j) S = S + (double)w[j];
    int64_t ns_head = 0, ns_tail = 0, nl_head = 0, nl_tail = 0;
    for (int64_t j = 0; j < deg; ++j) {
        double pj = ((double)w[j] * (double)deg) / S;
        p[j] = pj;
        if (pj < 1.0) small[ns_tail++] = j; else large[nl_tail++] = j;
    }
    /* small can receive at most deg entries in total: every index enters it
     * at most once, so a linear buffer of length deg suffices. */
    while (ns_head < ns_tail && nl_head < nl_tail) {
        int64_t s = small[ns_head++];
        int64_t l = large[nl_head];
        double ps = p[s];
        double t = ps * 4294967296.0;
        thr[s] = (t >= 4294967295.0) ? 0xFFFFFFFFu : (uint32_t)t;
        alias[s] = (int32_t)l;
        p[l] = (p[l] + ps) - 1.0;
        if (p[l] < 1.0) { nl_head++; small[ns_tail++] = l; }
    }
    while (ns_head < ns_tail) { int64_t j = small[ns_head++]; thr[j] = 0xFFFFFFFFu; alias[j] = (int32_t)j; }
    while (nl_head < nl_tail) { int64_t j = large[nl_head++]; thr[j] = 0xFFFFFFFFu; alias[j] = (int32_t)j; }
    return 0;
}

int oracle_alias_build(int64_t n, const int64_t *rp, const float *w,
                       uint32_t *thr, int32_t *alias)
{
    int64_t maxdeg = 0;
    for (int64_t u = 0; u < n; ++u) {
        int64_t d = rp[u + 1] - rp[u];
        if (d > maxdeg) maxdeg = d;
    }
    if (maxdeg == 0) return 0;
    double *p = (double *)malloc(sizeof(double) * (size_t)maxdeg);
    int64_t *sm = (int64_t *)malloc(sizeof(int64_t) * (size_t)maxdeg);
    int64_t *lg = (int64_t *)malloc(sizeof(int64_t) * (size_t)maxdeg);
    if (!p || !sm || !lg) { free(p); free(sm); free(lg); return -1; }
    for (int64_t u = 0; u < n; ++u) {
        int64_t b = rp[u], d = rp[u + 1] - rp[u];
        if (d > 0) alias_row(d, w + b, thr + b, alias + b, p, sm, lg);
    }
    free(p); free(sm); free(lg);
    return 0;
}

/* ------------------------------------------------------------- successor */

typedef struct {
    int64_t n;
    const int64_t *rp;
    const int32_t *col;
    const uint32_t *thr;   /* NULL for unit weights */
    const int32_t *alias;  /* NULL for unit weights */
    int32_t root;
    uint32_t key[2];
    uint32_t graph_id;
} graph_t;

static int32_t succ(const graph_t *g, int32_t u, uint32_t c, uint32_t tree)
{
    uint32_t ctr[4] = { c, (uint32_t)u, tree, g->graph_id };
    uint32_t o[4];
    oracle_philox4x32_10(ctr, g->key, o);
    int64_t b = g->rp[u];
    uint32_t deg = (uint32_t)(g->rp[u + 1] - b);
    uint32_t j = (uint32_t)(((uint64_t)o[0] * (uint64_t)deg) >> 32);
    if (g->thr != NULL && o[1] >= g->thr[b + j]) j = (uint32_t)g->alias[b + j];
    return g->col[b + j];
}

int32_t oracle_succ(int64_t n, const int64_t *rp, const int32_t *col,
                    const uint32_t *thr, const int32_t *alias, uint64_t seed,
                    uint32_t graph_id, int32_t u, uint32_t c, uint32_t tree)
{
    graph_t g = { n, rp, col, thr, alias, -1,
                  { (uint32_t)seed, (uint32_t)(seed >> 32) }, graph_id };
    return succ(&g, u, c, tree);
}

/* ------------------------------------------------------------ Wilson loop */

typedef struct {
    uint8_t *in_tree;
    int32_t *next;
    uint32_t *calls;   /* calls of RandomNeighbor(u) so far in this tree */
    int64_t *vis;      /* Algorithm 3's per-tree count, kept as an integer */
} work_t;

static int work_alloc(work_t *w, int64_t n)
{
    w->in_tree = (uint8_t *)malloc((size_t)n);
    w->next = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
    w->calls = (uint32_t *)malloc(sizeof(uint32_t) * (size_t)n);
    w->vis = (int64_t *)malloc(sizeof(int64_t) * (size_t)n);
    return (w->in_tree && w->next && w->calls && w->vis) ? 0 : -1;
}

static void work_free(work_t *w)
{
    free(w->in_tree); free(w->next); free(w->calls); free(w->vis);
}

/* One tree.  order: the n-1 start nodes (NULL = ascending ids, skipping the
 * root).  Returns the number of RandomNeighbor calls (draws), or -1 when a
 * per-vertex call count would overflow 32 bits. */
static int64_t wilson_tree(const graph_t *g, uint32_t tree, const int32_t *order,
                           work_t *w)
{
    const int64_t n = g->n;
    const int32_t v = g->root;
    int64_t draws = 0;
    for (int64_t u = 0; u < n; ++u) {
        w->in_tree[u] = 0; w->next[u] = -1; w->calls[u] = 0; w->vis[u] = 0;
    }
    w->in_tree[v] = 1;
    for (int64_t i = 0, s = 0; s < n - 1; ++i) {
        int32_t j;
        if (order) { j = order[s]; }
        else { if (i == v) continue; j = (int32_t)i; }
        ++s;
        int32_t u = j;
        w->vis[u] += 1;
        while (!w->in_tree[u]) {
            if (w->calls[u] == 0xFFFFFFFFu) return -1;
            w->next[u] = succ(g, u, w->calls[u], tree);
            w->calls[u] += 1;
            ++draws;
            u = w->next[u];
            w->vis[u] += 1;
        }
        w->vis[u] -= 1;
        u = j;
        while (!w->in_tree[u]) { w->in_tree[u] = 1; u = w->next[u]; }
    }
    return draws;
}

typedef struct {
    const graph_t *g;
    int64_t tree0, ntrees;
    int nthreads, tid;
    double *sums;        /* private [n] */
    int32_t *parents;    /* shared [ntrees][n] or NULL */
    int32_t *visits;     /* shared [ntrees][n] or NULL */
    int64_t draws;
    int status;
} task_t;

static void *run_task(void *arg)
{
    task_t *t = (task_t *)arg;
    const int64_t n = t->g->n;
    work_t w;
    if (work_alloc(&w, n)) { work_free(&w); t->status = -2; return NULL; }
    for (int64_t i = t->tid; i < t->ntrees; i += t->nthreads) {
        int64_t d = wilson_tree(t->g, (uint32_t)(t->tree0 + i), NULL, &w);
        if (d < 0) { t->status = -3; break; }
        t->draws += d;
        for (int64_t u = 0; u < n; ++u) t->sums[u] += (double)w.vis[u];
        if (t->parents) memcpy(t->parents + i * n, w.next, sizeof(int32_t) * (size_t)n);
        if (t->visits)
            for (int64_t u = 0; u < n; ++u) t->visits[i * n + u] = (int32_t)w.vis[u];
    }
    work_free(&w);
    return NULL;
}

/* Sample trees tree0 .. tree0+ntrees-1 and add each node's visit count to
 * sums[u] (sums += sum over trees of visits; exact integers in FP64).
 * parents/visits: NULL or [ntrees][n].  nthreads >= 1 worker threads, one
 * tree at a time each.  *draws_out: total RandomNeighbor calls.
 * Returns 0, -2 on allocation failure, -3 on call-count overflow. */
int oracle_wilson(int64_t n, const int64_t *rp, const int32_t *col,
                  const uint32_t *thr, const int32_t *alias, int32_t root,
                  uint64_t seed, uint32_t graph_id, int64_t tree0, int64_t ntrees,
                  int nthreads, double *sums, int32_t *parents, int32_t *visits,
                  int64_t *draws_out)
{
    graph_t g = { n, rp, col, thr, alias, root,
                  { (uint32_t)seed, (uint32_t)(seed >> 32) }, graph_id };
    if (nthreads < 1) nthreads = 1;
    if (nthreads > ntrees && ntrees > 0) nthreads = (int)ntrees;
    task_t *tasks = (task_t *)calloc((size_t)nthreads, sizeof(task_t));
    pthread_t *th = (pthread_t *)calloc((size_t)nthreads, sizeof(pthread_t));
    if (!tasks || !th) { free(tasks); free(th); return -2; }
    int status = 0;
    for (int i = 0; i < nthreads; ++i) {
        tasks[i].g = &g; tasks[i].tree0 = tree0; tasks[i].ntrees = ntrees;
        tasks[i].nthreads = nthreads; tasks[i].tid = i;
        tasks[i].parents = parents; tasks[i].visits = visits;
        tasks[i].sums = (double *)calloc((size_t)n, sizeof(double));
        if (!tasks[i].sums) status = -2;
    }
    if (status == 0) {
        if (nthreads == 1) run_task(&tasks[0]);
        else {
            for (int i = 0; i < nthreads; ++i) pthread_create(&th[i], NULL, run_task, &tasks[i]);
            for (int i = 0; i < nthreads; ++i) pthread_join(th[i], NULL);
        }
        int64_t d = 0;
        for (int i = 0; i < nthreads; ++i) {
            if (tasks[i].status) status = tasks[i].status;
            d += tasks[i].draws;
            for (int64_t u = 0; u < n; ++u) sums[u] += tasks[i].sums[u];
        }
        if (draws_out) *draws_out = d;
    }
    for (int i = 0; i < nthreads; ++i) free(tasks[i].sums);
    free(tasks); free(th);
    return status;
}

/* One tree with an explicit start-node order (the n-1 non-root nodes), for
 * checking that the result does not depend on the order.  parent, visits,
 * calls: [n].  Returns draws or a negative status. */
int64_t oracle_wilson_order(int64_t n, const int64_t *rp, const int32_t *col,
                            const uint32_t *thr, const int32_t *alias,
                            int32_t root, uint64_t seed, uint32_t graph_id,
                            uint32_t tree, const int32_t *order,
                            int32_t *parent, int32_t *visits, uint32_t *calls)
{
    graph_t g = { n, rp, col, thr, alias, root,
                  { (uint32_t)seed, (uint32_t)(seed >> 32) }, graph_id };
    work_t w;
    if (work_alloc(&w, n)) { work_free(&w); return -2; }
    int64_t d = wilson_tree(&g, tree, order, &w);
    if (d >= 0) {
        memcpy(parent, w.next, sizeof(int32_t) * (size_t)n);
        for (int64_t u = 0; u < n; ++u) visits[u] = (int32_t)w.vis[u];
        memcpy(calls, w.calls, sizeof(uint32_t) * (size_t)n);
    }
    work_free(&w);
    return d;
}

/* Weighted degree d_u = sum of the row's weights in arc order (FP64); the
 * row length when w is NULL. */
void oracle_wdeg(int64_t n, const int64_t *rp, const float *w, double *d)
{
    for (int64_t u = 0; u < n; ++u) {
        if (w == NULL) { d[u] = (double)(rp[u + 1] - rp[u]); continue; }
        double s = 0.0;
        for (int64_t j = rp[u]; j < rp[u + 1]; ++j) s = s + (double)w[j];
        d[u] = s;
    }
}

/* Johnson-Lindenstrauss sketch Q (k x n, row-major) with Q_iu = +-1/sqrt(k):
 * the sign is the top bit of Philox output o0 for counter (i, u, 0xFFFFFFFF, 0)
 * and key (seed lo, seed hi) (set bit = negative). */
void oracle_rademacher(int32_t k, int64_t n, uint64_t seed, double *Q)
{
    const uint32_t key[2] = { (uint32_t)seed, (uint32_t)(seed >> 32) };
    const double s = 1.0 / sqrt((double)k);
    for (int32_t i = 0; i < k; ++i)
        for (int64_t u = 0; u < n; ++u) {
            uint32_t ctr[4] = { (uint32_t)i, (uint32_t)u, 0xFFFFFFFFu, 0u }, o[4];
            oracle_philox4x32_10(ctr, key, o);
            Q[(int64_t)i * n + u] = (o[0] >> 31) ? -s : s;
        }
}

/* ------------------------------------------------------------ trap walks */

/* The straightforward estimator of Section 5 (before Wilson's algorithm is
 * brought in): t_u = (L_v^-1)_uu is the expected number of visits to u of a
 * random walk started at u and stopped when it meets the trap v (the lemma
 * connecting t_u with L_v^-1), time 0 included.  For every u != v and every
 * r < R, one such walk; counts[u] += its visits to u.  Step s of walk (u, r)
 * moves from x by the RandomNeighbor rule of succ() (multiply-high index,
 * alias coin for weighted rows) with Philox counter (s, u, r, 0xFFFFFFFE) and
 * key (seed lo, seed hi).  *steps_out: total steps.  Returns 0, or 1 if a walk
 * took more than max_steps steps (the walk is cut there and the run flagged). */
struct tw_task {
    const graph_t *g;
    int64_t R, max_steps, steps;
    int32_t u0, u1;
    int64_t *counts;
    int status;
};

static void *tw_run(void *arg)
{
    struct tw_task *t = (struct tw_task *)arg;
    const graph_t *g = t->g;
    for (int32_t u = t->u0; u < t->u1; ++u) {
        if (u == g->root) continue;
        for (int64_t r = 0; r < t->R; ++r) {
            int32_t x = u;
            int64_t c = 0, s = 0;
            while (x != g->root) {
                if (x == u) ++c;
                if (s >= t->max_steps) { t->status = 1; break; }
                uint32_t ctr[4] = { (uint32_t)s, (uint32_t)u, (uint32_t)r, 0xFFFFFFFEu };
                uint32_t o[4];
                oracle_philox4x32_10(ctr, g->key, o);
                const int64_t b = g->rp[x];
                const uint32_t deg = (uint32_t)(g->rp[x + 1] - b);
                uint32_t j = (uint32_t)(((uint64_t)o[0] * (uint64_t)deg) >> 32);
                if (g->thr != NULL && o[1] >= g->thr[b + j]) j = (uint32_t)g->alias[b + j];
                x = g->col[b + j];
                ++s;
            }
            t->counts[u] += c;
            t->steps += s;
        }
    }
    return NULL;
}

int oracle_trap_walks(int64_t n, const int64_t *rp, const int32_t *col,
                      const uint32_t *thr, const int32_t *alias, int32_t root,
                      uint64_t seed, int64_t R, int64_t max_steps, int nthreads,
                      int64_t *counts, int64_t *steps_out)
{
    graph_t g = { n, rp, col, thr, alias, root,
                  { (uint32_t)seed, (uint32_t)(seed >> 32) }, 0 };
    if (nthreads < 1) nthreads = 1;
    if (nthreads > n) nthreads = (int)n;
    struct tw_task *tasks = (struct tw_task *)calloc((size_t)nthreads, sizeof(struct tw_task));
    pthread_t *th = (pthread_t *)calloc((size_t)nthreads, sizeof(pthread_t));
    if (!tasks || !th) { free(tasks); free(th); return -2; }
    const int64_t step = (n + nthreads - 1) / nthreads;
    for (int i = 0; i < nthreads; ++i) {
        tasks[i].g = &g; tasks[i].R = R; tasks[i].max_steps = max_steps; tasks[i].counts = counts;
        tasks[i].u0 = (int32_t)(i * step < n ? i * step : n);
        tasks[i].u1 = (int32_t)((i + 1) * step < n ? (i + 1) * step : n);
    }
    /* disjoint u ranges: each task writes only its own counts[u] */
    for (int i = 0; i < nthreads; ++i) pthread_create(&th[i], NULL, tw_run, &tasks[i]);
    int status = 0;
    int64_t steps = 0;
    for (int i = 0; i < nthreads; ++i) {
        pthread_join(th[i], NULL);
        if (tasks[i].status) status = tasks[i].status;
        steps += tasks[i].steps;
    }
    if (steps_out) *steps_out = steps;
    free(tasks); free(th);
    return status;
}

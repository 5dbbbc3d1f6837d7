// Asynchronous Wilson walkers (HBM mode for large graphs).
//
// Each tree is handled by one thread block whose threads are concurrent
// Wilson walkers on the same successor stacks (Algorithm 3: a walk from a
// start node follows RandomNeighbor until it reaches the tree, erasing loops).
// Every vertex has one 64-bit word
//     [ successor p : 32 | pop count k : 20 | owner : 12 ]
// owner = FREE, SETTLED (in the tree) or the id of the walker whose current
// loop-erased path contains the vertex; p caches succ(u, k) (or INVALID).
// Operations, each a pop of a genuine cycle of the "top" graph or pure
// bookkeeping, so by Wilson's cycle-popping theorem the final tree and every
// k_u equal those of the sequential algorithm:
//   claim   a FREE vertex x the head points to (64-bit CAS), draw p_x if
//           needed, x becomes the head;
//   pop     if the head points into the walker's own path, the loop from that
//           vertex to the head is a cycle of the top graph: k++ on each of its
//           vertices, all but the re-entered vertex become FREE;
//   settle  if the head points to a SETTLED vertex the whole path joins the
//           tree;
//   yield   if the head points into another walker's path, the walker whose
//           start comes later in the processing order releases its path
//           (owners set to FREE, cached p kept) and requeues its start.
// A walker that yielded takes no requeued start until the walker it yielded
// to has changed state (every walker publishes a version counter), so the
// earlier walk gets the contested vertex first; with few walkers per tree it
// takes a fresh start at once while fresh starts remain (by default), since
// those lie elsewhere in the graph.  The earliest active walk never yields, so the block always makes
// progress.
// Waits are bounded; on exhaustion the block records an error and stops.
#include <algorithm>
#include <cstring>
#include <numeric>
#include <random>
#include <type_traits>
#include <vector>

#include "rwc_common.cuh"

namespace rwc {
namespace {

constexpr uint32_t OWN_BITS = 12;
constexpr uint64_t OWN_MASK = (1ull << OWN_BITS) - 1;
constexpr uint32_t OWN_FREE = 0xFFF, OWN_SET = 0xFFE;
constexpr uint32_t K_BITS = 20;
constexpr uint64_t K_MAX = (1ull << K_BITS) - 1;
constexpr uint32_t P_INVALID = 0xFFFFFFFFu;

constexpr int WERR_KOVF = 1;     // a pop count exceeded 2^20 - 1
constexpr int WERR_WAIT = 2;     // a bounded wait ran out
constexpr int WERR_LOOP = 4;     // internal: a path walk exceeded n steps

__device__ __forceinline__ uint32_t W_own(uint64_t w) { return (uint32_t)(w & OWN_MASK); }
__device__ __forceinline__ uint32_t W_k(uint64_t w) { return (uint32_t)((w >> OWN_BITS) & K_MAX); }
__device__ __forceinline__ uint32_t W_p(uint64_t w) { return (uint32_t)(w >> 32); }
__device__ __forceinline__ uint64_t W_pack(uint32_t p, uint32_t k, uint32_t own) {
    return ((uint64_t)p << 32) | ((uint64_t)k << OWN_BITS) | own;
}
// Every access to a tree's state comes from the one thread block that owns
// the tree, so block-scope relaxed loads, stores and CAS are enough (kernel
// boundaries order them with the init and accumulation kernels).
__device__ __forceinline__ uint64_t ldv(const uint64_t *a) {
    uint64_t v;
    asm volatile("ld.relaxed.cta.global.u64 %0, [%1];" : "=l"(v) : "l"(a) : "memory");
    return v;
}
__device__ __forceinline__ void stv(uint64_t *a, uint64_t v) {
    asm volatile("st.relaxed.cta.global.u64 [%0], %1;" ::"l"(a), "l"(v) : "memory");
}
__device__ __forceinline__ uint64_t cas_cta(uint64_t *a, uint64_t cmp, uint64_t val) {
    return atomicCAS_block(reinterpret_cast<unsigned long long *>(a), (unsigned long long)cmp,
                           (unsigned long long)val);
}
__device__ __forceinline__ int32_t ld32(const int32_t *a) {
    int32_t v;
    asm volatile("ld.relaxed.cta.global.s32 %0, [%1];" : "=r"(v) : "l"(a) : "memory");
    return v;
}
__device__ __forceinline__ void st32(int32_t *a, int32_t v) {
    asm volatile("st.relaxed.cta.global.s32 [%0], %1;" ::"l"(a), "r"(v) : "memory");
}

struct WState {
    uint64_t *word;        // [B][n]
    int32_t *retry;        // [B][n-1] requeued start indices (circular)
    const int32_t *order;  // [n-1] start order (a permutation of the non-root vertices)
    int *err;
    unsigned long long *ctr;   // [0] steps, [1] yields, [2] pops, [3] next tree
    unsigned long long *diag;  // [8] loop iterations per walker state
};

__global__ void w_init(int64_t n, int32_t root, uint64_t *word, int64_t B) {
    const int64_t tot = B * n;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < tot;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t u = i % n;
        word[i] = (u == root) ? W_pack(P_INVALID, 0, OWN_SET) : W_pack(P_INVALID, 0, OWN_FREE);
    }
}

// Retry queue: slots hold start index + 1 (0 = empty); a producer reserves a
// slot with the tail counter and then fills it, a consumer reserves with the
// head counter and waits (bounded) for the fill, then empties the slot.
__device__ __forceinline__ void rq_push(int32_t *rq, int *tail, int64_t cap, int v) {
    const int pos = atomicAdd(tail, 1);
    st32(rq + pos % cap, v + 1);
    __threadfence_block();
}

__device__ __forceinline__ uint64_t gtimer() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Walker states.  Each loop iteration ("tick") does one vertex of work per
// walker (up to 8 on graphs with inline rows, below), and the memory
// accesses of all states are issued by the
// same instructions: one load of a vertex word (with the row of the vertex
// that may be drawn), then the stores, the claim CAS and the successor draw,
// whose arc load overlaps the CAS (on graphs of degree at most 8 the draw
// picks from an inline row loaded beside the word, with no arc load).  The
// lanes of a warp thus pay about two dependent memory round trips per step,
// whatever mix of states they are in.  Waits poll shared memory or the one
// vertex word.  (Loading the next tick's word at the end of a tick, while a
// claim is in flight, was measured slower on every graph: 29% on a 256² grid,
// 43% on a 1024² grid, 24% on R-MAT 20.)
enum : int { S_IDLE = 0, S_WALK, S_POP, S_REL, S_SET, S_WAITK, S_WAITV, S_WAITH, S_DONE };

// Register cap of the walker kernel: 52 registers are used without spills
// (56 with inline rows of 4, 58 with rows of 8), which keeps 16 to 18 blocks
// of 64 walkers per SM resident, at least 2432 trees on 152 SMs.  (A cap of
// 40 lets 96-walker blocks keep 2000 trees resident, but its spills cost more
// than the extra walkers gain.)
#ifndef RWC_WALKER_MAXNREG
#define RWC_WALKER_MAXNREG 64
#endif

// The row of a vertex that may be drawn: its CSR bounds (EW = 0), or, for
// graphs whose degrees are at most EW (4 or 8), its inline neighbour list
// (heads in arc order, -1 after the last), read with one or two 16-byte loads.
template <bool OFF64, int EW>
struct DrawRow {
    int4 e[EW / 4];
    __device__ __forceinline__ void load(const DevGraph &g, int32_t u) {
#pragma unroll
        for (int i = 0; i < EW / 4; ++i) e[i] = __ldg(g.ell + (int64_t)u * (EW / 4) + i);
    }
    // head of the arc picked by the 32-bit uniform x: arc floor(x deg / 2^32)
    __device__ __forceinline__ int32_t pick(uint32_t x) const {
        uint32_t deg = 0;
#pragma unroll
        for (int i = 0; i < EW / 4; ++i)
            deg += (e[i].x >= 0) + (e[i].y >= 0) + (e[i].z >= 0) + (e[i].w >= 0);
        const uint32_t j = __umulhi(x, deg);
        const int4 q = (EW == 4 || j < 4) ? e[0] : e[EW / 4 - 1];
        const uint32_t jj = j & 3u;
        return jj < 2 ? (jj == 0 ? q.x : q.y) : (jj == 2 ? q.z : q.w);
    }
};
template <bool OFF64>
struct DrawRow<OFF64, 0> {
    int64_t rb;
    uint32_t deg;
    __device__ __forceinline__ void load(const DevGraph &g, int32_t u) { row_bounds<OFF64>(g, u, rb, deg); }
    template <bool WT>
    __device__ __forceinline__ int32_t pick_csr(const DevGraph &g, uint32_t x, uint32_t y) const {
        const uint32_t j = __umulhi(x, deg);
        if (WT) {
            const WArc arc = g.warc[rb + j];
            return (y < arc.thr) ? arc.col : arc.alias_col;
        }
        return __ldg(g.col + rb + j);
    }
};

template <bool OFF64, bool WT, int EW, bool DIAG>
__global__ void __maxnreg__(RWC_WALKER_MAXNREG) w_trees(DevGraph g, WState s, int64_t B, uint32_t tree0,
                                                uint32_t k0, uint32_t k1, int64_t max_wait_ns,
                                                int wait_policy) {
    const int n = (int)g.n;            // the host keeps n below 2^31 - 2
    const int nstart = n - 1;
    const uint32_t me = threadIdx.x;
    constexpr int INF = 0x7fffffff;
    __shared__ int sh_tree;
    __shared__ int sh_next;             // next fresh start index
    __shared__ int sh_rhead, sh_rtail;  // retry queue
    __shared__ int sh_active;           // walkers holding a start
    __shared__ int sh_err;
    __shared__ unsigned sh_prog;        // rewritten by every walker that stores a vertex word
    // claim locks of graphs with inline rows (below); all free between ticks
    constexpr int NLOCK = 256;
    constexpr int KSTEP = EW > 0 ? 8 : 1;   // vertex steps per tick and lane (below)
    __shared__ int sh_lock[EW > 0 ? NLOCK : 1];
    if constexpr (EW > 0)
        for (int i = threadIdx.x; i < NLOCK; i += blockDim.x) sh_lock[i] = 0;
    // prio[W], kill[W], killer[W], ver[W], killv[W], wprog[W] (24 W bytes), then wt0[W]
    extern __shared__ __align__(8) int sh[];
    int *prio = sh;
    int *kill = sh + blockDim.x;
    int *killer = sh + 2 * blockDim.x;
    int *ver = sh + 3 * blockDim.x;
    int *killv = sh + 4 * blockDim.x;   // the contested vertex of a yield request
    unsigned *wprog = (unsigned *)(sh + 5 * blockDim.x);   // block progress seen when a wait began
    uint64_t *wt0 = (uint64_t *)(sh + 6 * blockDim.x);   // time of that sighting
    unsigned long long steps = 0, yields = 0, pops = 0;
    unsigned long long it_state[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};

    for (;;) {
        if (threadIdx.x == 0) {
            sh_tree = (int)atomicAdd(&s.ctr[3], 1ull);
            sh_next = 0; sh_rhead = 0; sh_rtail = 0; sh_active = 0; sh_err = 0; sh_prog = 0;
        }
        prio[threadIdx.x] = INF;
        kill[threadIdx.x] = -1;
        killer[threadIdx.x] = -1;
        ver[threadIdx.x] = 0;
        killv[threadIdx.x] = -1;
        __syncthreads();
        const int t = sh_tree;
        if (t >= B) break;
        uint64_t *st = s.word + (int64_t)t * n;
        int32_t *rq = s.retry + (int64_t)t * nstart;
        const uint32_t tree = tree0 + (uint32_t)t;

        int state = S_IDLE;
        int32_t start = -1, head = -1, hp = -1, cur = -1, popx = -1;
        int32_t cut = -1;             // release: suffix from `cut` first, then the prefix
        uint32_t kx = 0;              // new pop count of the vertex a pop re-enters
        int myprio = INF, wait_on = -1, wait_ver = 0, wait_prio = 0;
        int pend_idx = -1;            // next fresh start, fetched one walk ahead
        int32_t pend_start = -1;
        int walked = 0;          // vertices visited in the current POP/REL/SET pass
        uint32_t polls = 0;
        auto vread = [](const int *a) { return *(const volatile int *)a; };
        auto bump = [&]() { *(volatile int *)&ver[me] = ver[me] + 1; };
        // true when the block has made no progress (no vertex word stored by
        // any of its walkers) for max_wait_ns while this walker waited: waits
        // are bounded by a lack of progress, not by their own length
        auto waited_out = [&]() {
            if (polls++ == 0) {
                wprog[me] = *(volatile unsigned *)&sh_prog;
                wt0[me] = gtimer();
                return false;
            }
            if ((polls & 255) == 0) {
                const unsigned pr = *(volatile unsigned *)&sh_prog;
                if (pr != wprog[me]) {
                    wprog[me] = pr;
                    wt0[me] = gtimer();
                } else if (gtimer() - wt0[me] > (uint64_t)max_wait_ns) {
                    atomicOr(&sh_err, WERR_WAIT);
                    return true;
                }
            }
            return false;
        };
        // after a yield: wait for the winner to move on before the next start
        // (policy bit 2 skips the wait while fresh starts remain, since a
        // fresh start is elsewhere in the graph)
        auto must_wait = [&]() {
            return !(wait_policy & 2) || (pend_idx < 0 && vread(&sh_next) >= nstart);
        };
        auto take_fresh = [&]() {
            if (vread(&sh_next) < nstart) {
                const int i = atomicAdd(&sh_next, 1);
                if (i < nstart) return i;
            }
            return -1;
        };
        auto drop_start = [&](bool requeue) {
            if (requeue) {
                rq_push(rq, &sh_rtail, nstart, myprio);
                if (DIAG) ++yields;
            }
            *(volatile int *)&prio[me] = INF;
            bump();
            start = -1; head = -1;
            atomicSub(&sh_active, 1);
            polls = 0;
        };
        // Lockstep: every tick starts with a warp vote, so a waiting walker
        // polls once per tick instead of spinning ahead of the others.
        // Finished walkers idle until the whole warp is done; errors end the
        // loop for everyone through the vote.
        for (;;) {
            const bool err = vread(&sh_err) != 0;
            if (__any_sync(0xffffffffu, err)) break;

            if (__all_sync(0xffffffffu, state == S_DONE)) break;
            // a warp whose walkers all wait gives its issue slots to the others
            if (__all_sync(0xffffffffu, state == S_DONE || state == S_WAITV || state == S_WAITK ||
                                            state == S_WAITH))
                __nanosleep(200);
            if (DIAG && (threadIdx.x & 31) == 0) ++it_state[S_DONE];   // warp iterations
            if (state == S_DONE) continue;
            if (DIAG) ++it_state[state];
            do {
            // ---- transitions that touch no vertex word
            bool hold = false;          // no vertex word this tick
            if (state == S_WAITV) {
                // after yielding: wait until the walker yielded to has moved on
                if (vread(&ver[wait_on]) == wait_ver && vread(&prio[wait_on]) != INF) {
                    if (waited_out()) break;
                    hold = true;
                } else {
                    state = S_IDLE;
                    polls = 0;
                }
            }
            if (state == S_IDLE) {
                // the prefetched fresh start, else a fresh one, else a requeued one
                int idx = -1;
                int32_t sv = -1;
                if (pend_idx >= 0) {
                    idx = pend_idx; sv = pend_start; pend_idx = -1;
                } else {
                    idx = take_fresh();
                    if (idx < 0) {
                        const int hd = vread(&sh_rhead);
                        if (hd < vread(&sh_rtail) && atomicCAS(&sh_rhead, hd, hd + 1) == hd) {
                            int32_t *slot = rq + hd % nstart;
                            uint64_t t0 = gtimer();
                            int32_t v = ld32(slot);
                            while (v == 0 && gtimer() - t0 < (uint64_t)max_wait_ns) v = ld32(slot);
                            if (v == 0) { atomicOr(&sh_err, WERR_WAIT); break; }
                            idx = v - 1;
                            st32(slot, 0);
                        }
                    }
                    if (idx >= 0) { sv = s.order[idx]; hold = true; }   // its word next tick
                }
                if (idx < 0) {
                    // a premature "done" is harmless: a walker that requeues a
                    // start takes it back itself when it becomes idle
                    const int act = vread(&sh_active);
                    if (act == 0 && vread(&sh_rhead) >= vread(&sh_rtail) && vread(&sh_next) >= nstart)
                        state = S_DONE;
                    else if (waited_out())
                        break;
                    continue;
                }
                polls = 0;
                start = sv; head = -1; myprio = idx;
                *(volatile int *)&kill[me] = -1;
                atomicAdd(&sh_active, 1);
                *(volatile int *)&prio[me] = idx;
                bump();
                state = S_WALK;
                // fetch the next fresh start now; it is used when this walk ends
                const int ni = take_fresh();
                if (ni >= 0) { pend_idx = ni; pend_start = s.order[ni]; }
            }
            if (state == S_WALK && !hold && vread(&kill[me]) == myprio) {
                // an earlier walk asked for a vertex of this path: release it
                const int kb = vread(&killer[me]);
                const int kv = vread(&killv[me]);
                *(volatile int *)&kill[me] = -1;
                wait_on = kb;
                if (kb >= 0) wait_ver = vread(&ver[kb]);
                cut = -1;
                if (head >= 0 && kv >= 0 && kv < n) {
                    // free the requested vertex first (checked on its load)
                    cut = kv; cur = kv; walked = 0; state = S_REL;
                } else if (head >= 0) {
                    cur = start; walked = 0; state = S_REL;
                } else {
                    drop_start(true);
                    state = (wait_on >= 0 && must_wait()) ? S_WAITV : S_IDLE;
                    continue;
                }
            }
            if (hold) continue;

            // a lane in WALK, POP, REL or SET goes on for up to KSTEP vertex
            // steps in one tick while each step makes progress (a store, a
            // held claim or a change of pass), so one tick's fixed cost (votes,
            // the other lanes' states) is shared by several steps: 7% on a
            // 1024² grid with 8; on R-MAT under load the longer divergent ticks
            // cost more than they save (R-MAT 20: 9% slower with 2), so there
            // a lane takes one step per tick
            for (int ms = 0;; ++ms) {
            const int st0 = state;
            // ---- the vertex word of this tick, and the row of a possible draw
            int32_t a = -1, dv = -1;
            if (state == S_WALK || state == S_WAITK || state == S_WAITH) a = head < 0 ? start : hp;
            else if (state == S_POP || state == S_REL || state == S_SET) a = cur;
            if (state == S_WALK) dv = a;
            else if (state == S_POP && cur == head) dv = popx;
            if (a < 0) break;
            const uint64_t w = ldv(st + a);
            DrawRow<OFF64, EW> row;
            if (dv >= 0) row.load(g, dv);

            // ---- decide: at most one store, one CAS and one draw
            int32_t s_v = -1;  uint64_t s_val = 0;               // store
            int32_t c_v = -1;  uint64_t c_cmp = 0, c_val = 0;    // claim CAS
            int32_t d_u = -1;  uint32_t d_k = 0;                 // draw succ(d_u, d_k)
            int after = 0;     // 1: claim, 2: end of a pop, 3/4: end of a release/settle
            if (state == S_WAITK || state == S_WAITH) {
                // WAITK: asked walker wait_on to yield the vertex a; WAITH (wait
                // policy): a lies on an earlier walk's path.  Wait until a has
                // left that path (a request to yield is served from WALK).
                bool still = W_own(w) == (uint32_t)wait_on && vread(&kill[me]) != myprio;
                if (state == S_WAITK) still = still && vread(&prio[wait_on]) == wait_prio;
                if (still) {
                    if (waited_out()) break;
                } else {
                    state = S_WALK;
                    polls = 0;
                }
                break;
            }
            if (state == S_POP) {
                // one vertex of the loop popx -> ... -> head (popx itself was
                // done by the walk step that found the loop)
                const uint32_t k = W_k(w) + 1u;
                if (k > K_MAX) { atomicOr(&sh_err, WERR_KOVF); break; }
                if (W_own(w) != me || ++walked > n) { atomicOr(&sh_err, WERR_LOOP); break; }
                if (DIAG) ++pops;
                s_v = cur; s_val = W_pack(P_INVALID, k, OWN_FREE);
                if (cur == head) { d_u = popx; d_k = kx; after = 2; }
                else cur = (int32_t)W_p(w);
            } else if (state == S_REL || state == S_SET) {
                // one vertex of the path.  SET: start -> head.  REL: when a
                // walker asked for vertex `cut`, first cut -> head, then
                // start -> the vertex before cut; otherwise start -> head.
                if (state == S_REL && cut >= 0 && cur == cut && head != -2 && W_own(w) != me) {
                    // the requested vertex has left the path meanwhile
                    cut = -1; cur = start; walked = 0;
                    break;
                }
                if (W_own(w) != me || ++walked > n) { atomicOr(&sh_err, WERR_LOOP); break; }
                s_v = cur; s_val = (w & ~OWN_MASK) | (state == S_REL ? OWN_FREE : OWN_SET);
                const int32_t nxt = (int32_t)W_p(w);
                bool last = false;
                if (state == S_REL && cut >= 0) {
                    if (cur == head) {           // end of the suffix pass
                        if (start == cut) last = true;
                        else { cur = start; head = -2; }   // head = -2 marks the prefix pass
                    } else if (head == -2 && nxt == cut) {
                        last = true;             // vertex before cut: prefix done
                    } else {
                        cur = nxt;
                    }
                } else if (cur == head) {
                    last = true;
                } else {
                    cur = nxt;
                }
                if (last) after = state == S_REL ? 3 : 4;   // the walk ends after the store
            } else {
                // S_WALK: one step of the loop-erased walk from the head
                const int32_t x = a;
                const uint32_t ox = W_own(w);
                if (DIAG) ++steps;
                if (ox == OWN_SET) {
                    if (head >= 0) { cur = start; walked = 0; state = S_SET; }
                    else { drop_start(false); state = S_IDLE; }
                } else if (ox == me) {
                    // x -> ... -> head -> x is a cycle: pop it, x first (x stays
                    // on the path and gets its new successor at the end)
                    const uint32_t k = W_k(w) + 1u;
                    if (k > K_MAX) { atomicOr(&sh_err, WERR_KOVF); break; }
                    if (DIAG) ++pops;
                    kx = k; popx = x; walked = 1;
                    cur = (int32_t)W_p(w);
                    state = S_POP;
                } else if (ox == OWN_FREE) {
                    c_v = x; c_cmp = w; c_val = (w & ~OWN_MASK) | me;
                    if (W_p(w) == P_INVALID) { d_u = x; d_k = W_k(w); }
                    after = 1;
                } else {
                    // x is on another walker's path: the later walk yields
                    const int op = vread(&prio[ox]);
                    if (op == INF) {
                        // the owner has just dropped its walk: look again
                    } else if (myprio < op) {
                        *(volatile int *)&killer[ox] = (int)me;
                        *(volatile int *)&killv[ox] = x;
                        __threadfence_block();
                        *(volatile int *)&kill[ox] = op;
                        wait_on = (int)ox; wait_prio = op; polls = 0;
                        state = S_WAITK;
                    } else if (wait_policy & 1) {
                        wait_on = (int)ox; polls = 0;
                        state = S_WAITH;
                    } else {
                        wait_on = (int)ox;
                        wait_ver = vread(&ver[ox]);
                        cut = -1;
                        if (head >= 0) { cur = start; walked = 0; state = S_REL; }
                        else { drop_start(true); state = must_wait() ? S_WAITV : S_IDLE; }
                    }
                }
            }

            // ---- memory: store, claim (in flight during the draw), draw
            // a stored word marks the block as progressing: any new value of
            // sh_prog restarts the waits' clocks (the SM clock keeps it changing)
            if (s_v >= 0 || c_v >= 0) *(volatile unsigned *)&sh_prog = (unsigned)clock();
            if (s_v >= 0) stv(st + s_v, s_val);
            uint64_t old = 0;
            if (c_v >= 0) {
                if constexpr (EW > 0) {
                    // bounded-degree graphs, whose step waits on the tick latency
                    // of single trees: the claim takes a shared-memory lock (a
                    // hash of the vertex), re-reads the word and stores the claim,
                    // instead of an L2 round trip for a CAS (8% shorter ticks on a
                    // 256² grid tree alone; on R-MAT under load the CAS is faster,
                    // 11% on R-MAT 20).  A busy lock fails the claim, which is
                    // retried next tick.  Every writer of a FREE word claims it
                    // under the lock, so the re-read sees the last claim.
                    int *lk = &sh_lock[((uint32_t)c_v * 0x9E3779B1u) >> 24];
                    if (atomicCAS(lk, 0, 1) == 0) {
                        __threadfence_block();
                        old = ldv(st + c_v);
                        if (old == c_cmp) stv(st + c_v, c_val);
                        __threadfence_block();
                        atomicExch(lk, 0);
                    } else {
                        old = ~c_cmp;
                    }
                } else {
                    old = cas_cta(st + c_v, c_cmp, c_val);
                }
            }
            int32_t px = -1;
            if (d_u >= 0) {
                const Ctr4 o = philox4x32_10(Ctr4{d_k, (uint32_t)d_u, tree, 0u}, k0, k1);
                if constexpr (EW > 0) px = row.pick(o.x);
                else px = row.template pick_csr<WT>(g, o.x, o.y);
            }
            if (after == 1) {
                if (old == c_cmp) {
                    // claimed: x becomes the head
                    hp = d_u >= 0 ? px : (int32_t)W_p(c_cmp);
                    if (d_u >= 0) stv(st + c_v, W_pack((uint32_t)px, W_k(c_cmp), me));
                    head = c_v;
                    bump();
                }
                // a failed claim looks again next tick
            } else if (after == 2) {
                stv(st + popx, W_pack((uint32_t)px, kx, me));
                head = popx; hp = px;
                bump();
                state = S_WALK;
            } else if (after >= 3) {
                cut = -1;
                drop_start(after == 3);
                state = (after == 3 && wait_on >= 0 && must_wait()) ? S_WAITV : S_IDLE;
            }
            const bool go = (state == S_WALK || state == S_POP || state == S_REL || state == S_SET) &&
                            !(c_v >= 0 && old != c_cmp) && (s_v >= 0 || c_v >= 0 || state != st0);
            if (!go || ms + 1 >= KSTEP) break;
            }
            } while (0);
        }
        __syncthreads();
        if (threadIdx.x == 0 && sh_err) atomicOr(s.err, sh_err);
        if (sh_err) break;
    }
    if (DIAG && steps) atomicAdd(&s.ctr[0], steps);
    if (DIAG && yields) atomicAdd(&s.ctr[1], yields);
    if (DIAG && pops) atomicAdd(&s.ctr[2], pops);
    if (DIAG && s.diag)
        for (int i = 0; i < 8; ++i) {
            // [0..6] lane iterations per state (wait-for-owner counted with
            // wait-after-yield), [7] warp iterations
            const unsigned long long v = i == 7 ? it_state[S_DONE]
                                       : it_state[i] + (i == S_WAITV ? it_state[S_WAITH] : 0ull);
            if (v) atomicAdd(&s.diag[i], v);
        }
}

// visits_u = k_u + 1 over the chunk's trees into sums; optional per-tree output.
__global__ void w_accum(int64_t n, int32_t root, const uint64_t *word, int64_t B, double *sums,
                        int32_t *parents, int32_t *visits, unsigned long long *draws) {
    unsigned long long local = 0;
    for (int64_t u = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; u < n;
         u += (int64_t)gridDim.x * blockDim.x) {
        int64_t acc = 0;
        for (int64_t t = 0; t < B; ++t) {
            const uint64_t w = word[t * n + u];
            const int32_t vis = (u == root) ? 0 : (int32_t)W_k(w) + 1;
            acc += vis;
            if (parents) parents[t * n + u] = (u == root) ? -1 : (int32_t)W_p(w);
            if (visits) visits[t * n + u] = vis;
        }
        local += (unsigned long long)acc;
        if (sums && u != root) sums[u] += (double)acc;
    }
    for (int o = 16; o > 0; o >>= 1) local += __shfl_xor_sync(0xffffffffu, local, o);
    if ((threadIdx.x & 31) == 0 && local) atomicAdd(draws, local);
}

// Dynamic shared memory of a walker block of W threads: six int arrays and
// one uint64 array (24 W bytes keep it 8-byte aligned).
inline size_t walker_smem(int W) { return (size_t)W * (6 * sizeof(int) + 8); }

template <int V> using int_c = std::integral_constant<int, V>;

// f(off64, weighted, inline row width) as compile-time constants
template <class F>
void dispatch(const DevGraph &g, F f) {
    if (g.off64) {
        if (g.weighted) f(std::true_type{}, std::true_type{}, int_c<0>{});
        else f(std::true_type{}, std::false_type{}, int_c<0>{});
    } else {
        if (g.weighted) f(std::false_type{}, std::true_type{}, int_c<0>{});
        else if (g.ell_w == 4) f(std::false_type{}, std::false_type{}, int_c<4>{});
        else if (g.ell_w == 8) f(std::false_type{}, std::false_type{}, int_c<8>{});
        else f(std::false_type{}, std::false_type{}, int_c<0>{});
    }
}

}  // namespace

// Start order shared by every tree of a graph: a fixed pseudo-random
// permutation of the non-root vertices (the result does not depend on it).
rwc_status walker_order(rwc_graph *G, const int32_t **out) {
    if (G->walk_order) { *out = G->walk_order; return RWC_OK; }
    const int64_t n = G->g.n;
    std::vector<int32_t> ord;
    ord.reserve(n - 1);
    for (int64_t u = 0; u < n; ++u)
        if (u != G->g.root) ord.push_back((int32_t)u);
    std::mt19937_64 rng(0x5eed5eedULL);
    for (int64_t i = (int64_t)ord.size() - 1; i > 0; --i) {
        const int64_t j = (int64_t)(rng() % (uint64_t)(i + 1));
        std::swap(ord[i], ord[j]);
    }
    int32_t *d = nullptr;
    RWC_CUDA_TRY(graph_alloc(G, (void **)&d, ord.size() * sizeof(int32_t)));
    RWC_CUDA_TRY(cudaMemcpy(d, ord.data(), ord.size() * sizeof(int32_t), cudaMemcpyHostToDevice));
    G->walk_order = d;
    *out = d;
    return RWC_OK;
}

rwc_status sample_walker(rwc_graph *G, uint64_t seed, int64_t tree0, int64_t T, double *sums,
                         int32_t *parents, int32_t *visits, const rwc_options_t &o,
                         rwc_stats_t *st, cudaStream_t stream) {
    if (o.walker_policy == 4) return sample_park(G, seed, tree0, T, sums, parents, visits, o, st, stream);
    const DevGraph &g = G->g;
    const int64_t n = g.n;
    if (n >= ((int64_t)1 << 31) - 2) return set_error(RWC_ERR_UNSUPPORTED, "n too large for walker mode");
    const int32_t *order = nullptr;
    RWC_TRY(walker_order(G, &order));
    const size_t per_tree = (size_t)n * (8 + 4) + 256;
    int64_t B = o.trees_per_chunk;
    if (B <= 0) {
        size_t fr = 0, tot = 0;
        RWC_CUDA_TRY(cudaMemGetInfo(&fr, &tot));
        const size_t budget = o.memory_budget > 0 ? (size_t)o.memory_budget : (size_t)(fr * 0.6);
        B = (int64_t)std::max<size_t>(1, budget / per_tree);
    }
    B = std::min(B, T);
    // walkers per tree: chosen per launch below (the largest block that keeps
    // every tree of the chunk resident at once, so no tree waits for a wave)
    int W = o.block_threads > 0 ? std::max(32, std::min(512, o.block_threads / 32 * 32)) : 0;
    const uint32_t k0 = (uint32_t)seed, k1 = (uint32_t)(seed >> 32);
    void *buf = nullptr;
    const size_t bytes = (size_t)B * n * 8 + (size_t)B * (n - 1) * 4 + 256;
    RWC_CUDA_TRY(cudaMallocAsync(&buf, bytes, stream));
    struct Free {
        void *p; cudaStream_t s;
        ~Free() { cudaFreeAsync(p, s); }
    } fr{buf, stream};
    WState ws;
    ws.word = (uint64_t *)buf;
    ws.retry = (int32_t *)((char *)buf + (size_t)B * n * 8);
    char *tail = (char *)buf + (size_t)B * n * 8 + (size_t)B * (n - 1) * 4;
    tail = (char *)(((uintptr_t)tail + 63) & ~(uintptr_t)63);
    ws.order = order;
    ws.err = (int *)tail;                                  // @0
    ws.ctr = (unsigned long long *)(tail + 8);             // @8..40
    unsigned long long *draws = (unsigned long long *)(tail + 40);
    ws.diag = (unsigned long long *)(tail + 64);
    const bool prof = o.profile != 0;
    cudaEvent_t ev[6] = {};
    if (prof) for (auto &e : ev) cudaEventCreate(&e);
    struct EvFree {
        cudaEvent_t *e; bool on;
        ~EvFree() { if (on) for (int i = 0; i < 6; ++i) cudaEventDestroy(e[i]); }
    } evf{ev, prof};
    // a wait fails when its block made no progress for this long (ns)
    const int64_t max_wait = o.max_wait_ns > 0 ? o.max_wait_ns : (int64_t)30 * 1000000000;
    const int sms = num_sms();
    int64_t *h = G->host_scalars;
    for (int64_t c0 = 0; c0 < T; c0 += B) {
        const int64_t Bc = std::min(B, T - c0);
        RWC_CUDA_TRY(cudaMemsetAsync(tail, 0, 128, stream));
        RWC_CUDA_TRY(cudaMemsetAsync(ws.retry, 0, (size_t)Bc * (n - 1) * 4, stream));
        if (prof) cudaEventRecord(ev[0], stream);
        ::rwc::count_launches(1);
        w_init<<<sms * 8, 256, 0, stream>>>(n, g.root, ws.word, Bc);
        if (prof) cudaEventRecord(ev[1], stream);
        rwc_status status = RWC_OK;
        dispatch(g, [&](auto off64, auto wt, auto ew) {
            constexpr bool O = decltype(off64)::value, WT = decltype(wt)::value;
            constexpr int EW = decltype(ew)::value;
            auto kern = (o.profile >= 2) ? w_trees<O, WT, EW, true> : w_trees<O, WT, EW, false>;
            int Wc = W, per_sm = 0;
            if (Wc == 0) {
                // largest multiple of 32 in [64, 512] whose resident blocks cover
                // the chunk; 64 when none does (the chunk then runs in waves)
                Wc = 64;
                for (int cand = 512; cand >= 64; cand -= 32) {
                    int ps = 0;
                    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&ps, kern, cand, walker_smem(cand));
                    if ((int64_t)sms * ps >= Bc) { Wc = cand; break; }
                }
            }
            const size_t smem = walker_smem(Wc);
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, Wc, smem);
            if (per_sm < 1) { status = set_error(RWC_ERR_UNSUPPORTED, "walker block does not fit"); return; }
            const int64_t blocks = std::min<int64_t>(Bc, (int64_t)sms * per_sm);
            if (st) st->block_threads = Wc;
            ::rwc::count_launches(1);
            // default conflict policy: with few walkers per tree (many trees)
            // a walker that yielded takes a fresh start at once (3), with many
            // it waits for the winner (1), which keeps collisions down
            const int pol = o.walker_policy != 0 ? o.walker_policy : (Wc <= 64 ? 3 : 1);
            kern<<<(unsigned)blocks, Wc, smem, stream>>>(g, ws, Bc, (uint32_t)(tree0 + c0), k0, k1, max_wait,
                                                         pol == 2 ? 1 : pol == 3 ? 2 : 0);
        });
        RWC_TRY(status);
        if (prof) cudaEventRecord(ev[2], stream);
        ::rwc::count_launches(1);
        w_accum<<<sms * 8, 256, 0, stream>>>(n, g.root, ws.word, Bc, sums,
                                             parents ? parents + c0 * n : nullptr,
                                             visits ? visits + c0 * n : nullptr, draws);
        if (prof) cudaEventRecord(ev[3], stream);
        RWC_CUDA_TRY(cudaGetLastError());
        if (o.async_status) {
            // no host synchronisation: the chunk's error bits go to the
            // graph's status word (rwc_sync_status)
            ::rwc::count_launches(1);
            fold_status<<<1, 1, 0, stream>>>((const int *)tail, 0, G->dev_status);
            RWC_CUDA_TRY(cudaGetLastError());
            continue;
        }
        RWC_CUDA_TRY(cudaMemcpyAsync(h, tail, 128, cudaMemcpyDeviceToHost, stream));
        RWC_CUDA_TRY(cudaStreamSynchronize(stream));
        const int e = (int)(h[0] & 0xffffffff);
        if (e & WERR_KOVF) return set_error(RWC_ERR_UNSUPPORTED, "a vertex was popped more than 2^20 - 1 times");
        if (e & WERR_LOOP) return set_error(RWC_ERR_CUDA, "walker internal check failed");
        if (e & WERR_WAIT) return set_error(RWC_ERR_NOT_CONVERGED, "a walker wait exceeded its bound");
        if (st)
            for (int i = 0; i < 8; ++i) st->diag[i] += h[8 + i];
        if (st) {
            st->chunks += 1;
            st->walk_steps += h[1];
            st->rounds += h[2];          // yields (re-queued walks)
            st->draws += h[5];
            st->marked += h[5];
            st->phase_units[RWC_PHASE_INIT] += Bc * n;
            st->phase_units[RWC_PHASE_WALK] += h[5];   // successor draws
            st->phase_units[RWC_PHASE_ACCUM] += Bc * n;
            if (prof) {
                float a = 0, b2 = 0, c = 0;
                cudaEventElapsedTime(&a, ev[0], ev[1]);
                cudaEventElapsedTime(&b2, ev[1], ev[2]);
                cudaEventElapsedTime(&c, ev[2], ev[3]);
                st->phase_ms[RWC_PHASE_INIT] += a;
                st->phase_ms[RWC_PHASE_WALK] += b2;
                st->phase_ms[RWC_PHASE_ACCUM] += c;
                st->phase_launches[RWC_PHASE_INIT] += 1;
                st->phase_launches[RWC_PHASE_WALK] += 1;
                st->phase_launches[RWC_PHASE_ACCUM] += 1;
            }
        }
    }
    if (st) st->mode = RWC_MODE_WALKER;
    return RWC_OK;
}

}  // namespace rwc

// ---------------------------------------------------------------------------
// Allocation-free sampling.  Some callers cannot allocate device memory while
// they sample: real-time or embedded hosts that forbid allocation after
// start-up, and processes whose memory pool is exhausted or owned by another
// allocator.
// rwc_sample_trees_noalloc samples with the walker kernels above, keeping all
// of its scratch (start order, per-tree vertex words, requeue buffers and
// counters) in one fixed array of this file; the caller still passes the
// graph and the output buffers.
#include <mutex>

namespace rwc {
namespace {

constexpr size_t NOALLOC_BYTES = (size_t)32 << 20;   // 32 MiB
static __device__ __align__(256) unsigned char g_noalloc_scratch[NOALLOC_BYTES];

// Device address of g_noalloc_scratch, resolved once per device (host code
// may not use the symbol itself as a pointer).
struct NoallocAddr {
    std::mutex mu;
    void *ptr[64] = {};
};
NoallocAddr g_noalloc_addr;

rwc_status noalloc_scratch(void **out) {
    int dev = 0;
    RWC_CUDA_TRY(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 64) return set_error(RWC_ERR_UNSUPPORTED, "device index %d out of range", dev);
    std::lock_guard<std::mutex> lock(g_noalloc_addr.mu);
    if (!g_noalloc_addr.ptr[dev]) {
        void *p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p)
            return set_error(RWC_ERR_CUDA, "cudaGetSymbolAddress of the static scratch failed: %s",
                             cudaGetErrorString(e));
        g_noalloc_addr.ptr[dev] = p;
    }
    *out = g_noalloc_addr.ptr[dev];
    return RWC_OK;
}

// Start order for the allocation-free path: i -> (a i + c) mod (n-1) with a
// coprime to n-1, mapped onto the non-root vertices (any order gives the
// same trees).
__global__ void w_affine_order(int64_t n, int32_t root, uint64_t a, uint64_t c, int32_t *order) {
    const int64_t m = n - 1;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < m;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t j = (int64_t)((a * (uint64_t)i + c) % (uint64_t)m);
        order[i] = (int32_t)(j < root ? j : j + 1);
    }
}

uint64_t gcd64(uint64_t x, uint64_t y) {
    while (y) { const uint64_t t = x % y; x = y; y = t; }
    return x;
}

}  // namespace
}  // namespace rwc

extern "C" rwc_status rwc_sample_trees_noalloc(rwc_graph_t *G, uint64_t seed, int64_t tree0,
                                               int64_t T, double *sums, int32_t *parents,
                                               int32_t *visits, rwc_stream_t stream_) {
    using namespace rwc;
    clear_error();
    if (!G) return set_error(RWC_ERR_INVALID, "graph is NULL");
    if (T < 0 || tree0 < 0 || tree0 + T > ((int64_t)1 << 32))
        return set_error(RWC_ERR_INVALID, "tree range must lie in [0, 2^32)");
    if (T == 0) return RWC_OK;
    const DevGraph &g = G->g;
    const int64_t n = g.n;
    cudaStream_t stream = (cudaStream_t)stream_;
    // layout: order [n-1] int32 | counters (64 B) | per tree: words [n] u64 + requeue [n-1] int32
    const size_t order_b = (((size_t)(n - 1) * 4) + 255) & ~(size_t)255;
    const size_t tail_b = 256;
    const size_t tree_b = (((size_t)n * 8 + (size_t)(n - 1) * 4) + 255) & ~(size_t)255;
    if (order_b + tail_b + tree_b > NOALLOC_BYTES)
        return set_error(RWC_ERR_INVALID,
                         "graph too large for rwc_sample_trees_noalloc: one tree needs %zu bytes of "
                         "scratch, the static array holds %zu",
                         order_b + tail_b + tree_b, NOALLOC_BYTES);
    void *base = nullptr;
    RWC_TRY(noalloc_scratch(&base));
    char *p = (char *)base;
    int32_t *order = (int32_t *)p;
    char *tail = p + order_b;
    char *trees = tail + tail_b;
    const int64_t B = std::min<int64_t>(T, (int64_t)((NOALLOC_BYTES - order_b - tail_b) / tree_b));
    WState ws;
    ws.word = (uint64_t *)trees;
    ws.retry = (int32_t *)(trees + (size_t)B * n * 8);
    ws.order = order;
    ws.err = (int *)tail;
    ws.ctr = (unsigned long long *)(tail + 8);
    unsigned long long *draws = (unsigned long long *)(tail + 40);
    ws.diag = (unsigned long long *)(tail + 64);
    const uint64_t m = (uint64_t)(n - 1);
    uint64_t a = (uint64_t)(0.6180339887 * (double)m) | 1ull;
    while (m > 1 && gcd64(a % m, m) != 1) ++a;
    const int sms = num_sms();
    ::rwc::count_launches(1);
    w_affine_order<<<sms * 4, 256, 0, stream>>>(n, g.root, m > 1 ? a % m : 1, seed % (m ? m : 1), order);
    const int W = (g.nnz / std::max<int64_t>(1, n) <= 6) ? 64 : 256;
    const uint32_t k0 = (uint32_t)seed, k1 = (uint32_t)(seed >> 32);
    int64_t *h = G->host_scalars;
    for (int64_t c0 = 0; c0 < T; c0 += B) {
        const int64_t Bc = std::min(B, T - c0);
        RWC_CUDA_TRY(cudaMemsetAsync(tail, 0, 128, stream));
        RWC_CUDA_TRY(cudaMemsetAsync(ws.retry, 0, (size_t)Bc * (n - 1) * 4, stream));
        ::rwc::count_launches(1);
        w_init<<<sms * 8, 256, 0, stream>>>(n, g.root, ws.word, Bc);
        rwc_status status = RWC_OK;
        dispatch(g, [&](auto off64, auto wt, auto ew) {
            auto kern = w_trees<decltype(off64)::value, decltype(wt)::value, decltype(ew)::value, false>;
            const size_t smem = walker_smem(W);
            int per_sm = 0;
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, W, smem);
            if (per_sm < 1) { status = set_error(RWC_ERR_UNSUPPORTED, "walker block does not fit"); return; }
            const int64_t blocks = std::min<int64_t>(Bc, (int64_t)sms * per_sm);
            ::rwc::count_launches(1);
            kern<<<(unsigned)blocks, W, smem, stream>>>(g, ws, Bc, (uint32_t)(tree0 + c0), k0, k1,
                                                        (int64_t)30 * 1000000000, 1);
        });
        RWC_TRY(status);
        ::rwc::count_launches(1);
        w_accum<<<sms * 8, 256, 0, stream>>>(n, g.root, ws.word, Bc, sums,
                                             parents ? parents + c0 * n : nullptr,
                                             visits ? visits + c0 * n : nullptr, draws);
        RWC_CUDA_TRY(cudaGetLastError());
        RWC_CUDA_TRY(cudaMemcpyAsync(h, tail, 48, cudaMemcpyDeviceToHost, stream));
        RWC_CUDA_TRY(cudaStreamSynchronize(stream));
        const int e = (int)(h[0] & 0xffffffff);
        if (e & WERR_KOVF) return set_error(RWC_ERR_UNSUPPORTED, "a vertex was popped more than 2^20 - 1 times");
        if (e & WERR_LOOP) return set_error(RWC_ERR_CUDA, "walker internal check failed");
        if (e & WERR_WAIT) return set_error(RWC_ERR_NOT_CONVERGED, "a walker wait exceeded its bound");
    }
    return RWC_OK;
}

// Concurrent Wilson walkers with parked paths (RWC_MODE_WALKER, policy 4).
//
// Same successor stacks, same trees as every other schedule (Wilson's
// cycle-popping theorem: popping genuine cycles of the "top" graph in any
// order ends in the sequential algorithm's tree and pop counts).  What
// differs from the walker kernel of walker.cu is what happens when a walk
// runs into another walk's loop-erased path:
//   - the later walk (larger start index) PARKS: its path stays claimed and
//     hangs at the vertex it points to; the thread takes other work.  A
//     parked path is woken when that vertex leaves the earlier path (settled
//     into the tree or freed by a pop) and is then resumed by any idle
//     walker, which continues it from where it hung;
//   - the earlier walk takes the later path's suffix over (relabels it as
//     its own) and continues from its end: a parked path is relabelled by
//     the earlier walk itself, an active one by its own walker at its next
//     step boundary, which parks the remaining prefix.
// No path is ever released, so no cached successor is walked twice.
// A path is named by the index of its start vertex in the start order; the
// earliest live path is never parked, so the tree always progresses.
//
// Per (tree, vertex): a 16-byte word {successor, pop count, owner path,
// flags}; flag 1 = some parked path hangs at this vertex.  Whoever settles or
// frees a flagged vertex queues it; an idle walker then scans the vertex's
// neighbours for parked heads pointing at it and makes those paths
// resumable.  Per (tree, path): status and the vertex it hangs at.
// Waits are bounded by a lack of progress; on exhaustion the block records
// an error and stops.
#include <algorithm>
#include <cstring>
#include <vector>

#include "rwc_common.cuh"

namespace rwc {
namespace {

typedef unsigned __int128 u128;

constexpr uint32_t O_FREE = 0xFFFFFFFFu, O_SET = 0xFFFFFFFEu;
constexpr uint32_t P_NONE = 0xFFFFFFFFu;
constexpr uint32_t F_ATT = 1u;

// path status (pstat); an active path stores PS_ACTIVE + its walker's index
constexpr int PS_DEAD = 0, PS_PARKING = 1, PS_PARKED = 2, PS_RESUMABLE = 3, PS_ADOPTING = 4,
              PS_ACTIVE = 16;

constexpr int HAND_BUSY = -2;    // wait_for: the awaited path is handing over
constexpr int PERR_WAIT = 2;     // a bounded wait ran out
constexpr int PERR_LOOP = 4;     // internal: a path walk exceeded n steps or a ring overflowed

__device__ __forceinline__ u128 pk(uint4 v) {
    return (u128)v.x | ((u128)v.y << 32) | ((u128)v.z << 64) | ((u128)v.w << 96);
}
__device__ __forceinline__ uint4 upk(u128 v) {
    return make_uint4((uint32_t)v, (uint32_t)(v >> 32), (uint32_t)(v >> 64), (uint32_t)(v >> 96));
}
__device__ __forceinline__ bool same(uint4 a, uint4 b) {
    return a.x == b.x && a.y == b.y && a.z == b.z && a.w == b.w;
}
// Every access to a tree's state comes from the one block that owns the
// tree: block-scope relaxed loads and atomics are enough.
__device__ __forceinline__ uint4 ld4(const uint4 *a) {
    uint4 r;
    asm volatile("ld.relaxed.cta.global.v4.u32 {%0,%1,%2,%3}, [%4];"
                 : "=r"(r.x), "=r"(r.y), "=r"(r.z), "=r"(r.w) : "l"(a) : "memory");
    return r;
}
__device__ __forceinline__ uint4 cas4(uint4 *a, uint4 cmp, uint4 val) {
    return upk(atomicCAS_block(reinterpret_cast<u128 *>(a), pk(cmp), pk(val)));
}
__device__ __forceinline__ int ldi(const int *a) {
    int v;
    asm volatile("ld.relaxed.cta.global.s32 %0, [%1];" : "=r"(v) : "l"(a) : "memory");
    return v;
}
__device__ __forceinline__ void sti(int *a, int v) {
    asm volatile("st.relaxed.cta.global.s32 [%0], %1;" ::"l"(a), "r"(v) : "memory");
}
__device__ __forceinline__ uint64_t gclock() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

struct PState {
    uint4 *word;           // [B][n]
    int *pstat;            // [B][n-1] per path (start index)
    int *patt;             // [B][n-1] vertex a parked path hangs at
    int *retry;            // [B][n-1] requeued start indices + 1 (ring)
    int *resume;           // [B][2(n-1)] resumable paths + 1 (ring; stale entries are skipped)
    int *wake;             // [B][2n] flagged vertices + 1 (ring)
    const int32_t *order;  // [n-1] start order
    int *err;
    unsigned long long *ctr;   // [3] next tree, [4] draws (unused here)
    unsigned long long *diag;  // [9] DIAG: lane ticks per state, [8] warp ticks
};

__global__ void p_init(int64_t n, int32_t root, uint4 *word, int *pstat, int64_t B) {
    const int64_t tot = B * n;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < tot;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t u = i % n;
        word[i] = make_uint4(P_NONE, 0u, u == root ? O_SET : O_FREE, 0u);
    }
    const int64_t tp = B * (n - 1);
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < tp;
         i += (int64_t)gridDim.x * blockDim.x)
        pstat[i] = PS_DEAD;
}

enum : int { S_IDLE = 0, S_WALK, S_POP, S_SET, S_ADOPT, S_HAND, S_WAITK, S_WAKE, S_DONE };

template <bool OFF64, bool WT, bool DIAG>
__global__ void __launch_bounds__(64, 14) w_park(DevGraph g, PState s, int64_t B, uint32_t tree0,
                                             uint32_t k0, uint32_t k1, int64_t max_wait_ns) {
    unsigned long long it_state[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};   // DIAG: lane ticks per state
    const int n = (int)g.n;
    const int nstart = n - 1;
    const int me = threadIdx.x;
    __shared__ int sh_tree, sh_err, sh_next, sh_live;
    __shared__ unsigned sh_prog;
    __shared__ int rq_h, rq_t, rs_h, rs_t, wk_h, wk_t;   // retry, resume, wake rings
    extern __shared__ __align__(8) int sh[];
    // per walker: a request posted to it (k_w: the asking walker, k_v: the
    // path asked); the asking walker's own request (req_p: its path, req_x:
    // the vertex it wants), mailbox (head, hp, ok), wait bookkeeping
    int *k_w = sh, *req_p = sh + blockDim.x, *k_v = sh + 2 * blockDim.x, *req_x = sh + 3 * blockDim.x;
    int *mb_h = sh + 4 * blockDim.x, *mb_p = sh + 5 * blockDim.x, *mb_ok = sh + 6 * blockDim.x;
    // the path a waiting walker waits for (or HAND_BUSY once that path has
    // committed to hand its suffix over); -1 when not waiting
    int *wait_for = sh + 7 * blockDim.x;
    unsigned *wprog = (unsigned *)(sh + 8 * blockDim.x);
    uint64_t *wt0 = (uint64_t *)(sh + 10 * blockDim.x);

    for (;;) {
        if (me == 0) {
            sh_tree = (int)atomicAdd(&s.ctr[3], 1ull);
            sh_err = 0; sh_next = 0; sh_live = 0; sh_prog = 0;
            rq_h = rq_t = rs_h = rs_t = wk_h = wk_t = 0;
        }
        k_w[me] = -1; req_p[me] = -1; k_v[me] = -1; req_x[me] = -1;
        mb_h[me] = -1; mb_p[me] = -1; mb_ok[me] = 0; wait_for[me] = -1;
        __syncthreads();
        const int t = sh_tree;
        if (t >= B) break;
        uint4 *W = s.word + (int64_t)t * n;
        int *pstat = s.pstat + (int64_t)t * nstart;
        int *patt = s.patt + (int64_t)t * nstart;
        int *retry = s.retry + (int64_t)t * nstart;
        int *resume = s.resume + (int64_t)t * 2 * nstart;
        int *wake = s.wake + (int64_t)t * 2 * n;
        const uint32_t tree = tree0 + (uint32_t)t;

        int state = S_IDLE;
        const uint64_t tree_t0 = gclock();
        int path = -1, start = -1, head = -1, hp = -1, cur = -1, popx = -1, aq = -1, qv = -1;
        int kw = -1, kp = -1, end = -1, walked = 0;
        uint32_t kx = 0;
        uint32_t polls = 0;

        auto vread = [](const int *a) { return *(const volatile int *)a; };
        auto progress = [&]() { *(volatile unsigned *)&sh_prog = (unsigned)clock(); };
        auto waited_out = [&]() {
            if (polls++ == 0) {
                wprog[me] = *(volatile unsigned *)&sh_prog;
                wt0[me] = gclock();
                return false;
            }
            if ((polls & 255) == 0) {
                const unsigned pr = *(volatile unsigned *)&sh_prog;
                if (pr != wprog[me]) { wprog[me] = pr; wt0[me] = gclock(); }
                else if (gclock() - wt0[me] > (uint64_t)max_wait_ns) { atomicOr(&sh_err, PERR_WAIT); return true; }
            }
            return false;
        };
        // an internal check failed: record which (the first one) and stop
        auto fail = [&](int where) {
            atomicOr(&sh_err, PERR_LOOP);
            atomicCAS(s.err + 1, 0, where);
        };
        // rings of value+1 entries: push reserves a slot with the tail and
        // fills it; pop reserves with the head and waits (bounded) for the fill
        auto push = [&](int *ring, int *tail, const int *hd, int cap, int v) {
            const int pos = atomicAdd(tail, 1);
            if (pos - vread(hd) >= cap) { fail(1); return; }
            sti(ring + pos % cap, v + 1);
            __threadfence_block();
        };
        auto pop = [&](int *ring, int *hd, const int *tail, int cap) -> int {
            const int h0 = vread(hd);
            if (h0 >= vread(tail) || atomicCAS(hd, h0, h0 + 1) != h0) return -1;
            int *slot = ring + h0 % cap;
            const uint64_t t0 = gclock();
            int v = ldi(slot);
            while (v == 0 && gclock() - t0 < (uint64_t)max_wait_ns) v = ldi(slot);
            if (v == 0) { atomicOr(&sh_err, PERR_WAIT); return -1; }
            sti(slot, 0);
            return v - 1;
        };
        auto is_path = [&](uint32_t o) { return o < (uint32_t)nstart; };
        auto die = [&]() {
            sti(pstat + path, PS_DEAD);
            atomicSub(&sh_live, 1);
            path = -1; head = -1; state = S_IDLE; polls = 0;
        };
        // hang path p's head at vertex a (owned by an earlier path, or by the
        // walk that took p's suffix over): status first, then the flag on a;
        // false when a changed under us (p is then made resumable)
        auto hang = [&](int p, int a) {
            if ((unsigned)a >= (unsigned)n) { fail(2); return false; }
            sti(patt + p, a);
            sti(pstat + p, PS_PARKING);
            __threadfence_block();
            for (int tries = 0; tries < 64; ++tries) {
                const uint4 w = ld4(W + a);
                if (!is_path(w.z) || (int)w.z >= p) break;   // a left an earlier path
                uint4 nw = w;
                nw.w |= F_ATT;
                // always an atomic on a (also when the flag is already set), so
                // that it is ordered with the owner's atomic that frees or
                // settles a and then queues a for waking
                if (same(cas4(W + a, w, nw), w)) {
                    atomicCAS(pstat + p, PS_PARKING, PS_PARKED);
                    return true;
                }
            }
            // a is free, settled or later-owned: p must look again itself
            if (atomicCAS(pstat + p, PS_PARKING, PS_RESUMABLE) == PS_PARKING)
                push(resume, &rs_t, &rs_h, 2 * nstart, p);
            return false;
        };

        // a vertex index about to be used: out of range ends the tree with
        // an internal error instead of an access outside the buffers
        auto bad = [&](int v) {
            if ((unsigned)v >= (unsigned)n) { fail(3); return true; }
            return false;
        };
        for (uint32_t tick = 0;; ++tick) {
            if (__any_sync(0xffffffffu, vread(&sh_err) != 0)) break;
            if (__all_sync(0xffffffffu, state == S_DONE)) break;
            // every tree ends within 4 x max_wait_ns, whatever happens
            if (me == 0 && (tick & 4095) == 0 && gclock() - tree_t0 > 4 * (uint64_t)max_wait_ns)
                atomicOr(&sh_err, PERR_WAIT);
            if (__all_sync(0xffffffffu, state == S_DONE || state == S_WAITK || state == S_IDLE))
                __nanosleep(100);
            if (DIAG && (threadIdx.x & 31) == 0) ++it_state[S_DONE];   // warp ticks
            if (state == S_DONE) continue;
            if (DIAG) ++it_state[state];
            do {
            if (state == S_IDLE) {
                // 1) a resumable path, 2) a flagged vertex to scan, 3) a fresh
                // start, 4) a requeued start
                const int q = pop(resume, &rs_h, &rs_t, 2 * nstart);
                if (q >= 0) {
                    if (atomicCAS(pstat + q, PS_RESUMABLE, PS_ACTIVE + me) != PS_RESUMABLE) break;  // stale
                    path = q; start = s.order[q]; head = -2; hp = ldi(patt + q);
                    k_v[me] = -1; mb_ok[me] = 0;
                    state = S_WALK; polls = 0; progress();
                    break;
                }
                const int v = pop(wake, &wk_h, &wk_t, 2 * n);
                if (v >= 0) { qv = v; cur = 0; state = S_WAKE; polls = 0; break; }
                int idx = -1;
                if (vread(&sh_next) < nstart) {
                    const int i = atomicAdd(&sh_next, 1);
                    if (i < nstart) idx = i;
                }
                if (idx < 0) idx = pop(retry, &rq_h, &rq_t, nstart);
                if (idx >= 0) {
                    path = idx; start = s.order[idx]; head = -1; hp = -1;
                    k_v[me] = -1; mb_ok[me] = 0;
                    state = S_WALK; polls = 0;
                    break;
                }
                if (vread(&sh_live) == 0 && vread(&sh_next) >= nstart && vread(&rq_h) >= vread(&rq_t) &&
                    vread(&rs_h) >= vread(&rs_t) && vread(&wk_h) >= vread(&wk_t))
                    state = S_DONE;
                else if (waited_out())
                    break;
                break;
            }
            if (state == S_WAKE) {
                // vertex qv was settled or freed while paths hung at it: one
                // neighbour per tick, a parked head there pointing at qv wakes
                if (bad(qv)) break;
                int64_t rb; uint32_t deg;
                row_bounds<OFF64>(g, qv, rb, deg);
                if (cur >= (int)deg) { state = S_IDLE; break; }
                const int h = WT ? g.warc[rb + cur].col : __ldg(g.col + rb + cur);
                ++cur;
                if (bad(h)) break;
                __threadfence_block();
                const uint4 w = ld4(W + h);
                if (is_path(w.z) && (int)w.x == qv) {
                    const int p = (int)w.z;
                    const int st = ldi(pstat + p);
                    if ((st == PS_PARKED || st == PS_PARKING) && ldi(patt + p) == qv &&
                        atomicCAS(pstat + p, st, PS_RESUMABLE) == st)
                        push(resume, &rs_t, &rs_h, 2 * nstart, p);
                }
                break;
            }
            if (state == S_WAITK) {
                // asked the active path aq for vertex cur: wait for the suffix
                if (vread(&mb_ok[me])) {
                    mb_ok[me] = 0;
                    *(volatile int *)&wait_for[me] = -1;
                    head = mb_h[me]; hp = mb_p[me];
                    state = S_WALK; polls = 0; progress();
                    break;
                }
                if (vread(&wait_for[me]) == HAND_BUSY) { if (waited_out()) break; break; }   // handover under way
                if (bad(cur)) break;
                const uint4 w = ld4(W + cur);
                const int st = ldi(pstat + aq);
                if ((int)w.z != aq || st == PS_PARKED || st == PS_RESUMABLE) {
                    // the situation changed: withdraw, unless aq has just
                    // committed to hand over (then wait for the mailbox)
                    if (atomicCAS(&wait_for[me], aq, -1) == aq) { state = S_WALK; polls = 0; }
                    break;
                }
                if (st >= PS_ACTIVE) {
                    const int vw = st - PS_ACTIVE;
                    const int other = vread(&k_w[vw]);
                    if (vread(&k_v[vw]) != aq || other < 0 || other >= (int)blockDim.x ||
                        vread(&req_p[other]) > path) {
                        // (re)post: the victim reads this walker's own
                        // request fields, which stay fixed while it waits
                        *(volatile int *)&k_w[vw] = me;
                        __threadfence_block();
                        *(volatile int *)&k_v[vw] = aq;
                    }
                }
                if (waited_out()) break;
                break;
            }
            if (state == S_HAND) {
                // hand the suffix cur .. head over to path kp (walker kw)
                if (bad(cur)) break;
                const uint4 w = ld4(W + cur);
                if ((int)w.z != path || ++walked > n) { fail(4); break; }
                uint4 nw = w;
                nw.z = (uint32_t)kp;
                if (!same(cas4(W + cur, w, nw), w)) break;   // a flag arrived: again
                progress();
                if ((int)w.x == hp) {
                    // cur was the head: post the mailbox, park the prefix
                    mb_h[kw] = cur; mb_p[kw] = hp;
                    __threadfence_block();
                    *(volatile int *)&mb_ok[kw] = 1;
                    if (end == start) {
                        // the whole path moved, start included: its start is
                        // looked at again later (a later pop could free it)
                        push(retry, &rq_t, &rq_h, nstart, path);
                        die();
                        break;
                    }
                    hang(path, end);
                    path = -1; head = -1; state = S_IDLE; polls = 0;
                    break;
                }
                cur = (int)w.x;
                break;
            }
            if (state == S_ADOPT) {
                // take the parked path aq's suffix cur .. (the vertex before its
                // hang point `end`) over as this path's
                if (bad(cur)) break;
                const uint4 w = ld4(W + cur);
                if ((int)w.z != aq || ++walked > n) { fail(5); break; }
                uint4 nw = w;
                nw.z = (uint32_t)path;
                if (!same(cas4(W + cur, w, nw), w)) break;
                progress();
                if ((int)w.x == end) {
                    head = cur; hp = end;
                    // aq keeps its prefix, now hanging at the first adopted vertex
                    if (s.order[aq] == qv) {
                        sti(pstat + aq, PS_DEAD);
                        atomicSub(&sh_live, 1);
                        push(retry, &rq_t, &rq_h, nstart, aq);
                    } else {
                        hang(aq, qv);
                    }
                    state = S_WALK; polls = 0;
                    break;
                }
                cur = (int)w.x;
                break;
            }
            if (state == S_POP) {
                // one vertex of the loop popx -> ... -> head: pop count + 1, free
                if (bad(cur) || bad(popx)) break;
                const uint4 w = ld4(W + cur);
                if ((int)w.z != path || ++walked > n) { fail(6); break; }
                const uint4 nw = make_uint4(P_NONE, w.y + 1u, O_FREE, 0u);
                const uint4 old = cas4(W + cur, w, nw);
                if (!same(old, w)) break;   // a flag arrived: again
                progress();
                if (w.w & F_ATT) push(wake, &wk_t, &wk_h, 2 * n, cur);
                if (cur == head) {
                    // popx gets its next successor and becomes the head
                    int64_t rb; uint32_t deg;
                    row_bounds<OFF64>(g, popx, rb, deg);
                    const Ctr4 o = philox4x32_10(Ctr4{kx, (uint32_t)popx, tree, 0u}, k0, k1);
                    const uint32_t j = __umulhi(o.x, deg);
                    int px;
                    if (WT) { const WArc arc = g.warc[rb + j]; px = (o.y < arc.thr) ? arc.col : arc.alias_col; }
                    else px = __ldg(g.col + rb + j);
                    for (int tries = 0;; ++tries) {
                        const uint4 wp = ld4(W + popx);
                        const uint4 np = make_uint4((uint32_t)px, kx, (uint32_t)path, wp.w);
                        if (same(cas4(W + popx, wp, np), wp)) break;
                        if (tries > 1000) { fail(7); break; }
                    }
                    head = popx; hp = px;
                    state = S_WALK;
                } else {
                    cur = (int)w.x;
                }
                break;
            }
            if (state == S_SET) {
                // one vertex of the path start -> head joins the tree
                if (bad(cur)) break;
                const uint4 w = ld4(W + cur);
                if ((int)w.z != path || ++walked > n) { fail(8); break; }
                const uint4 nw = make_uint4(w.x, w.y, O_SET, 0u);
                if (!same(cas4(W + cur, w, nw), w)) break;
                progress();
                if (w.w & F_ATT) push(wake, &wk_t, &wk_h, 2 * n, cur);
                if ((int)w.x == hp) { die(); break; }
                cur = (int)w.x;
                break;
            }
            // ---- S_WALK: one step of the loop-erased walk
            const int a = head == -1 ? start : hp;
            if (bad(a)) break;
            const uint4 w = ld4(W + a);
            const uint32_t o = w.z;
            if (head != -1 && o != O_SET && (int)o != path && vread(&k_v[me]) == path) {
                // an earlier walk asked for vertex k_x: hand the suffix from
                // there over (the head's successor lies outside the path)
                kw = vread(&k_w[me]);
                k_v[me] = -1;
                // commit only while the asker still waits for this path; its
                // request fields are then fixed
                if (kw >= 0 && kw < (int)blockDim.x && atomicCAS(&wait_for[kw], path, HAND_BUSY) == path) {
                    const int x = vread(&req_x[kw]);
                    kp = vread(&req_p[kw]);
                    if (bad(x)) break;
                    const uint4 wx = ld4(W + x);
                    if ((int)wx.z == path && kp >= 0 && kp < path) {
                        cur = x; end = x; walked = 0; hp = a;
                        state = S_HAND;
                        break;
                    }
                    *(volatile int *)&wait_for[kw] = path;   // not ours any more: the asker looks again
                }
            }
            if (o == O_SET) {
                if (head == -1) { path = -1; state = S_IDLE; break; }   // start already in the tree
                cur = start; walked = 0; state = S_SET;
                break;
            }
            if ((int)o == path) {
                // a -> ... -> head -> a is a cycle: pop it (a first, at the end)
                kx = w.y + 1u; popx = a; cur = (int)w.x; walked = 1;
                state = S_POP;
                break;
            }
            if (o == O_FREE) {
                uint4 nw = w;
                nw.z = (uint32_t)path;
                if (w.x == P_NONE) {
                    int64_t rb; uint32_t deg;
                    row_bounds<OFF64>(g, a, rb, deg);
                    const Ctr4 r = philox4x32_10(Ctr4{w.y, (uint32_t)a, tree, 0u}, k0, k1);
                    const uint32_t j = __umulhi(r.x, deg);
                    if (WT) { const WArc arc = g.warc[rb + j]; nw.x = (uint32_t)((r.y < arc.thr) ? arc.col : arc.alias_col); }
                    else nw.x = (uint32_t)__ldg(g.col + rb + j);
                }
                if (!same(cas4(W + a, w, nw), w)) break;   // lost a race: look again
                progress();
                if (head == -1) {
                    sti(pstat + path, PS_ACTIVE + me);
                    atomicAdd(&sh_live, 1);
                }
                head = a; hp = (int)nw.x;
                break;
            }
            // a lies on another path q
            const int q = (int)o;
            if (head == -1) {
                // the start lies on another path: look again later
                push(retry, &rq_t, &rq_h, nstart, path);
                path = -1; state = S_IDLE;
                break;
            }
            if (q < path) {
                // q is earlier: park this path at a
                if (hang(path, a)) { path = -1; head = -1; state = S_IDLE; polls = 0; }
                else { path = -1; head = -1; state = S_IDLE; polls = 0; }
                break;
            }
            // q is later: take its suffix from a over
            const int st = ldi(pstat + q);
            if ((st == PS_PARKED || st == PS_RESUMABLE) && atomicCAS(pstat + q, st, PS_ADOPTING) == st) {
                // q may have run and parked again since a was read (the same
                // status twice): a must still be q's, else give q back
                __threadfence_block();
                if ((int)ld4(W + a).z != q) { hang(q, ldi(patt + q)); break; }
                aq = q; qv = a; cur = a; end = ldi(patt + q); walked = 0;
                state = S_ADOPT;
                break;
            }
            aq = q; cur = a; state = S_WAITK; polls = 0;
            *(volatile int *)&req_x[me] = a;
            *(volatile int *)&req_p[me] = path;
            __threadfence_block();
            *(volatile int *)&wait_for[me] = q;
            } while (0);
        }
        __syncthreads();
        if (me == 0 && sh_err) atomicOr(s.err, sh_err);
        if (sh_err) break;
    }
    if (DIAG && s.diag)
        for (int i = 0; i < 9; ++i)
            if (it_state[i]) atomicAdd(&s.diag[i], it_state[i]);
}

// visits_u = k_u + 1 over the chunk's trees into sums; optional per-tree output.
__global__ void p_accum(int64_t n, int32_t root, const uint4 *word, int64_t B, double *sums,
                        int32_t *parents, int32_t *visits, unsigned long long *draws) {
    unsigned long long local = 0;
    for (int64_t u = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; u < n;
         u += (int64_t)gridDim.x * blockDim.x) {
        int64_t acc = 0;
        for (int64_t t = 0; t < B; ++t) {
            const uint4 w = word[t * n + u];
            const int32_t vis = (u == root) ? 0 : (int32_t)w.y + 1;
            acc += vis;
            if (parents) parents[t * n + u] = (u == root) ? -1 : (int32_t)w.x;
            if (visits) visits[t * n + u] = vis;
        }
        local += (unsigned long long)acc;
        if (sums && u != root) sums[u] += (double)acc;
    }
    for (int o = 16; o > 0; o >>= 1) local += __shfl_xor_sync(0xffffffffu, local, o);
    if ((threadIdx.x & 31) == 0 && local) atomicAdd(draws, local);
}

template <class F>
void dispatch(const DevGraph &g, F f) {
    if (g.off64) {
        if (g.weighted) f(std::true_type{}, std::true_type{});
        else f(std::true_type{}, std::false_type{});
    } else {
        if (g.weighted) f(std::false_type{}, std::true_type{});
        else f(std::false_type{}, std::false_type{});
    }
}

inline size_t park_smem(int W) { return (size_t)W * (10 * sizeof(int) + 8); }

}  // namespace

rwc_status sample_park(rwc_graph *G, uint64_t seed, int64_t tree0, int64_t T, double *sums,
                       int32_t *parents, int32_t *visits, const rwc_options_t &o, rwc_stats_t *st,
                       cudaStream_t stream) {
    const DevGraph &g = G->g;
    const int64_t n = g.n;
    if (n >= ((int64_t)1 << 31) - 2) return set_error(RWC_ERR_UNSUPPORTED, "n too large for walker mode");
    const int32_t *order = nullptr;
    RWC_TRY(walker_order(G, &order));
    // per tree: 16 n (words) + 4 (n-1) x 5 (status, hang point, retry, resume x 2) + 8 n (wake)
    const size_t per_tree = (size_t)n * 16 + (size_t)(n - 1) * 20 + (size_t)n * 8 + 1024;
    int64_t B = o.trees_per_chunk;
    if (B <= 0) {
        size_t fr = 0, tot = 0;
        RWC_CUDA_TRY(cudaMemGetInfo(&fr, &tot));
        const size_t budget = o.memory_budget > 0 ? (size_t)o.memory_budget : (size_t)(fr * 0.6);
        B = (int64_t)std::max<size_t>(1, budget / per_tree);
    }
    B = std::min(B, T);
    const int Wc = 64;
    const uint32_t k0 = (uint32_t)seed, k1 = (uint32_t)(seed >> 32);
    void *buf = nullptr;
    const size_t a_word = ((size_t)B * n * 16 + 255) & ~(size_t)255;
    const size_t a_int = ((size_t)B * (n - 1) * 4 + 255) & ~(size_t)255;
    const size_t a_wake = ((size_t)B * n * 8 + 255) & ~(size_t)255;
    const size_t bytes = a_word + 5 * a_int + a_wake + 256;
    RWC_CUDA_TRY(cudaMallocAsync(&buf, bytes, stream));
    struct Free {
        void *p; cudaStream_t s;
        ~Free() { cudaFreeAsync(p, s); }
    } fr{buf, stream};
    char *q = (char *)buf;
    PState ps;
    ps.word = (uint4 *)q; q += a_word;
    ps.pstat = (int *)q; q += a_int;
    ps.patt = (int *)q; q += a_int;
    ps.retry = (int *)q; q += a_int;
    ps.resume = (int *)q; q += 2 * a_int;
    ps.wake = (int *)q; q += a_wake;
    char *tail = q;
    ps.order = order;
    ps.err = (int *)tail;
    ps.ctr = (unsigned long long *)(tail + 8);
    ps.diag = (unsigned long long *)(tail + 64);
    unsigned long long *draws = (unsigned long long *)(tail + 40);
    const bool prof = o.profile != 0;
    cudaEvent_t ev[4] = {};
    if (prof) for (auto &e : ev) cudaEventCreate(&e);
    struct EvFree {
        cudaEvent_t *e; bool on;
        ~EvFree() { if (on) for (int i = 0; i < 4; ++i) cudaEventDestroy(e[i]); }
    } evf{ev, prof};
    const int64_t max_wait = o.max_wait_ns > 0 ? o.max_wait_ns : (int64_t)30 * 1000000000;
    const int sms = num_sms();
    int64_t *h = G->host_scalars;
    for (int64_t c0 = 0; c0 < T; c0 += B) {
        const int64_t Bc = std::min(B, T - c0);
        RWC_CUDA_TRY(cudaMemsetAsync(tail, 0, 160, stream));
        RWC_CUDA_TRY(cudaMemsetAsync(ps.retry, 0, (size_t)Bc * (n - 1) * 4, stream));
        RWC_CUDA_TRY(cudaMemsetAsync(ps.resume, 0, (size_t)Bc * (n - 1) * 8, stream));
        RWC_CUDA_TRY(cudaMemsetAsync(ps.wake, 0, (size_t)Bc * n * 8, stream));
        if (prof) cudaEventRecord(ev[0], stream);
        ::rwc::count_launches(1);
        p_init<<<sms * 8, 256, 0, stream>>>(n, g.root, ps.word, ps.pstat, Bc);
        if (prof) cudaEventRecord(ev[1], stream);
        rwc_status status = RWC_OK;
        dispatch(g, [&](auto off64, auto wt) {
            auto kern = (o.profile >= 2) ? w_park<decltype(off64)::value, decltype(wt)::value, true>
                                         : w_park<decltype(off64)::value, decltype(wt)::value, false>;
            const size_t smem = park_smem(Wc);
            int per_sm = 0;
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, Wc, smem);
            if (per_sm < 1) { status = set_error(RWC_ERR_UNSUPPORTED, "walker block does not fit"); return; }
            const int64_t blocks = std::min<int64_t>(Bc, (int64_t)sms * per_sm);
            if (st) st->block_threads = Wc;
            ::rwc::count_launches(1);
            kern<<<(unsigned)blocks, Wc, smem, stream>>>(g, ps, Bc, (uint32_t)(tree0 + c0), k0, k1, max_wait);
        });
        RWC_TRY(status);
        if (prof) cudaEventRecord(ev[2], stream);
        ::rwc::count_launches(1);
        p_accum<<<sms * 8, 256, 0, stream>>>(n, g.root, ps.word, Bc, sums,
                                             parents ? parents + c0 * n : nullptr,
                                             visits ? visits + c0 * n : nullptr, draws);
        if (prof) cudaEventRecord(ev[3], stream);
        RWC_CUDA_TRY(cudaGetLastError());
        RWC_CUDA_TRY(cudaMemcpyAsync(h, tail, 160, cudaMemcpyDeviceToHost, stream));
        RWC_CUDA_TRY(cudaStreamSynchronize(stream));
        const int e = (int)(h[0] & 0xffffffff);
        if (e & PERR_LOOP)
            return set_error(RWC_ERR_CUDA, "walker internal check %d failed", (int)(h[0] >> 32));
        if (e & PERR_WAIT) return set_error(RWC_ERR_NOT_CONVERGED, "a walker wait exceeded its bound");
        if (st) {
            // diag: [0..6] lane ticks in idle, walk, pop, settle, take-over,
            // hand-over, wait; [7] warp ticks
            for (int i = 0; i < 7; ++i) st->diag[i] += h[8 + i];
            st->diag[7] += h[8 + 8];
            st->chunks += 1;
            st->draws += h[5];
            st->marked += h[5];
            st->phase_units[RWC_PHASE_INIT] += Bc * n;
            st->phase_units[RWC_PHASE_WALK] += h[5];
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

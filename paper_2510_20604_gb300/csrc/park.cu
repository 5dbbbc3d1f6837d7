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
// Per (tree, vertex): a 16-byte word {successor, pop count, owner path, 0},
// written by its owner with plain stores (claims are a CAS), and a flag: 1 =
// some parked path hangs at this vertex.  A walk that hangs sets the flag and
// then checks the vertex's owner again; an owner that settles or frees a
// vertex stores the word and then takes the flag (fences between, so one of
// the two sees the other) and queues a flagged vertex; an idle walker scans
// that vertex's neighbours for parked heads pointing at it and makes those
// paths resumable.  Per (tree, path): status and the vertex it hangs at.
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
__device__ __forceinline__ void st4(uint4 *a, uint4 v) {
    asm volatile("st.relaxed.cta.global.v4.u32 [%0], {%1,%2,%3,%4};"
                 ::"l"(a), "r"(v.x), "r"(v.y), "r"(v.z), "r"(v.w) : "memory");
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
    int *flag;             // [B][n] 1: some parked path hangs at this vertex
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

// Walker states.  Every tick a walker does at most: one 16-byte vertex-word
// load, one int load (a path status, a hang point or a neighbour id) and the
// row bounds of a vertex it may draw for, all issued together; then at most
// one 16-byte CAS and one int CAS, issued together.  So the lanes of a warp
// pay about two dependent memory round trips per tick whatever mix of states
// they are in (a state machine that ran each state's accesses in its own
// branch paid them once per state present in the warp).
enum : int { S_IDLE = 0, S_WALK, S_POP, S_SET, S_ADOPT, S_HAND, S_WAITK, S_WAKE, S_DONE,
             S_POPX, S_HANG, S_QCHK, S_ADPREP };

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
        int *flag = s.flag + (int64_t)t * n;
        const uint32_t tree = tree0 + (uint32_t)t;

        int state = S_IDLE;
        const uint64_t tree_t0 = gclock();
        int path = -1, start = -1, head = -1, hp = -1, cur = -1, popx = -1, aq = -1, qv = -1;
        int kp = -1, end = -1, walked = 0;
        int hg_p = -1, hg_a = -1, hg_next = S_IDLE;   // S_HANG: path, vertex, state after
        int wv = -1, wj = 0;                            // S_WAKE: neighbour in hand, next arc
        int64_t rbx = 0;                                // row of popx (S_POPX), of qv (S_WAKE)
        uint32_t degx = 0;
        uint32_t kx = 0;
        uint32_t polls = 0;
        int pend_v = -1, pend_f = 0;   // the flag taken from vertex pend_v last tick

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
        auto bad = [&](int v) {
            if ((unsigned)v >= (unsigned)n) { fail(3); return true; }
            return false;
        };
        auto die = [&]() {
            sti(pstat + path, PS_DEAD);
            atomicSub(&sh_live, 1);
            path = -1; head = -1; state = S_IDLE; polls = 0;
        };
        // start hanging path p's head at vertex a: status, then the flag on
        // a, then (S_HANG, next tick) a's owner is looked at again: if a is
        // still an earlier path's, p is parked, else p is made resumable;
        // then the state becomes `next`
        auto begin_hang = [&](int p, int a, int next) {
            sti(patt + p, a);
            sti(pstat + p, PS_PARKING);
            __threadfence_block();
            atomicOr(flag + a, 1);
            __threadfence_block();
            hg_p = p; hg_a = a; hg_next = next;
            state = S_HANG;
        };
        // an owner's settle or free of vertex v: word first, then the flag
        // (its value is looked at next tick)
        auto release_flag = [&](int v) {
            __threadfence_block();
            pend_f = atomicExch(flag + v, 0);
            pend_v = v;
        };
        auto draw = [&](int v, uint32_t c, int64_t rb, uint32_t deg) -> int {
            const Ctr4 o = philox4x32_10(Ctr4{c, (uint32_t)v, tree, 0u}, k0, k1);
            const uint32_t j = __umulhi(o.x, deg);
            if (WT) { const WArc arc = g.warc[rb + j]; return (o.y < arc.thr) ? arc.col : arc.alias_col; }
            return __ldg(g.col + rb + j);
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
            if (pend_v >= 0) {
                if (pend_f) push(wake, &wk_t, &wk_h, 2 * n, pend_v);
                pend_v = -1;
            }
            if (state == S_DONE) continue;
            if (DIAG) ++it_state[state <= S_WAKE ? state : state == S_POPX ? S_POP : S_WALK];

            // ---------------- phase A: work that needs no vertex word
            if (state == S_IDLE) {
                // 1) a resumable path, 2) a flagged vertex to scan, 3) a fresh
                // start, 4) a requeued start
                const int q = pop(resume, &rs_h, &rs_t, 2 * nstart);
                if (q >= 0) {
                    if (atomicCAS(pstat + q, PS_RESUMABLE, PS_ACTIVE + me) == PS_RESUMABLE) {
                        path = q; start = s.order[q]; head = -2; hp = ldi(patt + q);
                        k_v[me] = -1; mb_ok[me] = 0;
                        state = S_WALK; polls = 0; progress();
                    }
                } else {
                    const int v = pop(wake, &wk_h, &wk_t, 2 * n);
                    if (v >= 0) {
                        qv = v;
                        if (!bad(v)) {
                            row_bounds<OFF64>(g, v, rbx, degx);
                            wj = 0; wv = -1; state = S_WAKE; polls = 0;
                        }
                    } else {
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
                        } else if (vread(&sh_live) == 0 && vread(&sh_next) >= nstart &&
                                   vread(&rq_h) >= vread(&rq_t) && vread(&rs_h) >= vread(&rs_t) &&
                                   vread(&wk_h) >= vread(&wk_t)) {
                            state = S_DONE;
                        } else {
                            waited_out();
                        }
                    }
                }
                continue;   // the new state's first access comes next tick
            }
            if (state == S_WAITK) {
                if (vread(&mb_ok[me])) {
                    mb_ok[me] = 0;
                    *(volatile int *)&wait_for[me] = -1;
                    head = mb_h[me]; hp = mb_p[me];
                    state = S_WALK; polls = 0; progress();
                    continue;
                }
                if (vread(&wait_for[me]) == HAND_BUSY) { waited_out(); continue; }   // handover under way
            }

            // ---------------- phase B: the tick's loads, issued together
            int la = -1;                 // vertex word
            const int *aux = nullptr;    // int (status, hang point, neighbour id)
            int rowv = -1;               // row bounds of a vertex that may be drawn for
            switch (state) {
                case S_WALK: la = head == -1 ? start : hp; rowv = la; break;
                case S_POP: la = cur; if (cur == head) rowv = popx; break;
                case S_POPX: la = popx; break;
                case S_SET: case S_ADOPT: case S_HAND: la = cur; break;
                case S_WAITK: la = cur; aux = pstat + aq; break;
                case S_WAKE:
                    la = wv;
                    if (wj < (int)degx) aux = WT ? &g.warc[rbx + wj].col : g.col + rbx + wj;
                    break;
                case S_HANG: la = hg_a; break;
                case S_QCHK: la = hp; aux = pstat + aq; break;
                case S_ADPREP: la = hp; aux = patt + aq; break;
                default: break;
            }
            if (la >= 0 && bad(la)) continue;
            uint4 w = make_uint4(0, 0, 0, 0);
            int ai = 0;
            int64_t rb = 0;
            uint32_t deg = 0;
            if (la >= 0) w = ld4(W + la);
            if (aux) ai = ldi(aux);
            if (rowv >= 0) row_bounds<OFF64>(g, rowv, rb, deg);

            // ---------------- phase C: decide; at most one 16-byte CAS and
            // one int CAS, issued together in phase D
            uint4 *c_a = nullptr; uint4 c_cmp = w, c_val = w;   // 16-byte CAS (claims)
            uint4 *s_a = nullptr; uint4 s_val = w;              // 16-byte store (owner's writes)
            int *i_a = nullptr; int i_cmp = 0, i_val = 0;       // int CAS
            int dv = -1;                  // vertex to draw a successor for (claim)
            int after = 0;                // what phase E does with the outcome
            const uint32_t o = w.z;
            switch (state) {
                case S_WALK: {
                    const int a = la;
                    if (head != -1 && o != O_SET && (int)o != path && vread(&k_v[me]) == path) {
                        // an earlier walk asked for a vertex of this path: at
                        // this clean point (the successor lies outside the
                        // path) commit, if the asker still waits
                        const int kw2 = vread(&k_w[me]);
                        k_v[me] = -1;
                        if (kw2 >= 0 && kw2 < (int)blockDim.x &&
                            atomicCAS(&wait_for[kw2], path, HAND_BUSY) == path) {
                            const int x = vread(&req_x[kw2]);
                            kp = vread(&req_p[kw2]);
                            if (!bad(x) && kp >= 0 && kp < path) {
                                cur = x; end = x; walked = 0; qv = kw2;   // qv: the asker's walker
                                state = S_HAND;     // x's ownership is checked on its load
                                break;
                            }
                            *(volatile int *)&wait_for[kw2] = path;   // give it back
                        }
                    }
                    if (o == O_SET) {
                        if (head == -1) { path = -1; state = S_IDLE; }   // the start is in the tree
                        else { cur = start; walked = 0; state = S_SET; }
                    } else if ((int)o == path) {
                        // a -> ... -> head -> a is a cycle: pop it, a last
                        kx = w.y + 1u; popx = a; cur = (int)w.x; walked = 1;
                        state = S_POP;
                    } else if (o == O_FREE) {
                        c_a = W + a; c_cmp = w; c_val = make_uint4(w.x, w.y, (uint32_t)path, 0u);
                        if (w.x == P_NONE) dv = a;
                        after = 1;
                    } else if (head == -1) {
                        // the start lies on another path: look again later
                        push(retry, &rq_t, &rq_h, nstart, path);
                        path = -1; state = S_IDLE;
                    } else if ((int)o < path) {
                        begin_hang(path, a, S_IDLE);   // an earlier path: hang here
                    } else {
                        aq = (int)o; state = S_QCHK;   // a later path: look at its status
                    }
                    break;
                }
                case S_QCHK: {
                    // the later path aq owns hp: take its suffix over if it is
                    // parked, else ask its walker to hand it over
                    if ((int)o != aq) { state = S_WALK; break; }
                    if (ai == PS_PARKED || ai == PS_RESUMABLE) {
                        i_a = pstat + aq; i_cmp = ai; i_val = PS_ADOPTING; after = 6;
                    } else {
                        cur = hp; state = S_WAITK; polls = 0;
                        *(volatile int *)&req_x[me] = hp;
                        *(volatile int *)&req_p[me] = path;
                        __threadfence_block();
                        *(volatile int *)&wait_for[me] = aq;
                    }
                    break;
                }
                case S_ADPREP: {
                    // holding aq ADOPTING: hp must still be aq's (it may have
                    // run and parked again since), else give aq back
                    if ((int)o != aq) { begin_hang(aq, ai, S_WALK); break; }
                    qv = hp; cur = hp; end = ai; walked = 0; state = S_ADOPT;
                    break;
                }
                case S_WAITK: {
                    if ((int)o != aq || ai == PS_PARKED || ai == PS_RESUMABLE) {
                        // the situation changed: withdraw, unless aq has just
                        // committed to hand over (then wait for the mailbox)
                        if (atomicCAS(&wait_for[me], aq, -1) == aq) { state = S_WALK; polls = 0; }
                        break;
                    }
                    if (ai >= PS_ACTIVE) {
                        const int vw = ai - PS_ACTIVE;
                        const int other = vread(&k_w[vw]);
                        if (vread(&k_v[vw]) != aq || other < 0 || other >= (int)blockDim.x ||
                            vread(&req_p[other]) > path) {
                            *(volatile int *)&k_w[vw] = me;
                            __threadfence_block();
                            *(volatile int *)&k_v[vw] = aq;
                        }
                    }
                    waited_out();
                    break;
                }
                case S_HAND: {
                    // hand cur .. head over to path kp
                    if ((int)o != path || ++walked > n) {
                        if (cur == end && walked <= 1) {
                            // the asked vertex left this path: the asker looks again
                            *(volatile int *)&wait_for[qv] = path;
                            walked = 0; state = S_WALK;
                        } else fail(4);
                        break;
                    }
                    s_a = W + cur; s_val = make_uint4(w.x, w.y, (uint32_t)kp, 0u);
                    after = 4;
                    break;
                }
                case S_ADOPT: {
                    if ((int)o != aq || ++walked > n) { fail(5); break; }
                    s_a = W + cur; s_val = make_uint4(w.x, w.y, (uint32_t)path, 0u);
                    after = 5;
                    break;
                }
                case S_POP: {
                    if ((int)o != path || ++walked > n) { fail(6); break; }
                    s_a = W + cur; s_val = make_uint4(P_NONE, w.y + 1u, O_FREE, 0u);
                    after = 2;
                    break;
                }
                case S_POPX: {
                    if ((int)o != path) { fail(7); break; }
                    // popx gets its next successor (drawn into hp last tick) and
                    // becomes the head
                    s_a = W + popx; s_val = make_uint4((uint32_t)hp, kx, (uint32_t)path, 0u);
                    after = 7;
                    break;
                }
                case S_SET: {
                    if ((int)o != path || ++walked > n) { fail(8); break; }
                    s_a = W + cur; s_val = make_uint4(w.x, w.y, O_SET, 0u);
                    after = 3;
                    break;
                }
                case S_HANG: {
                    // the flag is on hg_a (set before this load): if hg_a is
                    // still an earlier path's, its owner will see the flag when
                    // it settles or frees hg_a; else hg_p looks again itself
                    if (!is_path(o) || (int)o >= hg_p) {
                        i_a = pstat + hg_p; i_cmp = PS_PARKING; i_val = PS_RESUMABLE; after = 9;
                    } else {
                        i_a = pstat + hg_p; i_cmp = PS_PARKING; i_val = PS_PARKED; after = 8;
                    }
                    break;
                }
                case S_WAKE: {
                    // neighbour wv of the woken vertex qv: a parked head there
                    // pointing at qv is made resumable
                    if (wv >= 0 && is_path(o) && (int)w.x == qv) {
                        const int p = (int)o;
                        i_a = pstat + p; i_cmp = PS_PARKED; i_val = PS_RESUMABLE; after = 10;
                    }
                    if (wj < (int)degx) { wv = ai; ++wj; }
                    else if (!i_a) state = S_IDLE;
                    else wj = (int)degx + 1;   // finish after this CAS
                    break;
                }
                default: break;
            }

            // ---------------- phase D: the tick's atomics, issued together
            uint4 c_old = c_cmp;
            int i_old = i_cmp;
            int px = -1;
            if (c_a) c_old = cas4(c_a, c_cmp, c_val);
            if (s_a) st4(s_a, s_val);
            if (i_a) i_old = atomicCAS(i_a, i_cmp, i_val);
            if (dv >= 0) px = draw(dv, w.y, rb, deg);   // the arc load overlaps the CAS
            const bool c_ok = c_a && same(c_old, c_cmp);
            const bool i_ok = i_a && i_old == i_cmp;

            // ---------------- phase E: outcomes
            switch (after) {
                case 1:   // claim
                    if (!c_ok) break;   // lost a race: look again
                    progress();
                    if (head == -1) { sti(pstat + path, PS_ACTIVE + me); atomicAdd(&sh_live, 1); }
                    head = la;
                    if (dv >= 0) {
                        st4(W + la, make_uint4((uint32_t)px, w.y, (uint32_t)path, 0u));
                        hp = px;
                    } else {
                        hp = (int)w.x;
                    }
                    break;
                case 2:   // pop
                    progress();
                    release_flag(cur);
                    if (cur == head) {
                        rbx = rb; degx = deg;
                        hp = draw(popx, kx, rbx, degx);
                        state = S_POPX;
                    } else {
                        cur = (int)w.x;
                    }
                    break;
                case 7:   // popx's new successor
                    head = popx;   // hp holds the successor
                    state = S_WALK;
                    break;
                case 3:   // settle
                    progress();
                    release_flag(cur);
                    if ((int)w.x == hp) die();
                    else cur = (int)w.x;
                    break;
                case 4:   // hand over one vertex
                    progress();
                    if ((int)w.x == hp) {
                        // cur was the head: post the mailbox, hang the prefix
                        mb_h[qv] = cur; mb_p[qv] = hp;
                        __threadfence_block();
                        *(volatile int *)&mb_ok[qv] = 1;
                        if (end == start) {
                            // the whole path moved, start included: look at
                            // the start again later (a later pop could free it)
                            push(retry, &rq_t, &rq_h, nstart, path);
                            die();
                        } else {
                            begin_hang(path, end, S_IDLE);
                        }
                    } else {
                        cur = (int)w.x;
                    }
                    break;
                case 5:   // take one vertex over
                    progress();
                    if ((int)w.x == end) {
                        head = cur; hp = end;
                        // aq keeps its prefix, now hanging at the first vertex taken
                        if (s.order[aq] == qv) {
                            sti(pstat + aq, PS_DEAD);
                            atomicSub(&sh_live, 1);
                            push(retry, &rq_t, &rq_h, nstart, aq);
                            state = S_WALK;
                        } else {
                            begin_hang(aq, qv, S_WALK);
                        }
                    } else {
                        cur = (int)w.x;
                    }
                    break;
                case 6:   // won aq's status: check hp is still aq's
                    if (i_ok) state = S_ADPREP;
                    else state = S_WALK;
                    break;
                case 8:   // parked (or a waker came first and queued hg_p)
                    if (hg_p == path && hg_next == S_IDLE) path = -1;
                    state = hg_next; polls = 0;
                    if (state == S_IDLE) head = -1;
                    break;
                case 9:   // hg_p could not hang: make it resumable
                    if (i_ok) push(resume, &rs_t, &rs_h, 2 * nstart, hg_p);
                    if (hg_p == path && hg_next == S_IDLE) path = -1;
                    state = hg_next; polls = 0;
                    if (state == S_IDLE) head = -1;
                    break;
                case 10:  // a parked head at the woken vertex
                    if (i_ok) push(resume, &rs_t, &rs_h, 2 * nstart, (int)o);
                    else if (i_old == PS_PARKING && atomicCAS(pstat + (int)o, PS_PARKING, PS_RESUMABLE) == PS_PARKING)
                        push(resume, &rs_t, &rs_h, 2 * nstart, (int)o);
                    if (wj > (int)degx) state = S_IDLE;
                    break;
                default: break;
            }
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
    // + 4 n (flags)
    const size_t per_tree = (size_t)n * 16 + (size_t)(n - 1) * 20 + (size_t)n * 12 + 1024;
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
    const size_t a_flag = ((size_t)B * n * 4 + 255) & ~(size_t)255;
    const size_t bytes = a_word + 5 * a_int + a_wake + a_flag + 256;
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
    ps.flag = (int *)q; q += a_flag;
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
        RWC_CUDA_TRY(cudaMemsetAsync(ps.flag, 0, (size_t)Bc * n * 4, stream));
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

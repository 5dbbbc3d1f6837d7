// Parallel cycle-popping tree sampler (Section 5, Algorithm 3's loop over
// trees, Wilson's algorithm rooted at the pivot v).
//
// Every non-root vertex u has a successor stack succ(u, 0), succ(u, 1), ...
// (Philox-keyed by (c, u, tree, graph)); the current top is succ(u, k_u),
// k_u = pops so far.  Wilson (1996) shows that popping the cycles of the
// "top" graph in any order ends in the same tree with the same k_u, and that
// the sequential walk of Algorithm 3 is one such order.  Algorithm 3's count
// for u is its number of RandomNeighbor(u) calls = k_u + 1.
//
// The parallel order used here pops, in each round, every cycle of the top
// graph at once.  A cycle of round r+1 must contain a vertex popped in round
// r (all other tops are unchanged, and every cycle of round r was popped), so
// each round only searches from the vertices popped in the previous round
// (the "marked" list):
//   walk:     each marked vertex follows tops to the next marked vertex or to
//             a settled vertex (one whose chain reaches the root); segments
//             that reach the root are settled on the spot.
//   classify: on the compressed graph of marked vertices, a node is on a
//             cycle iff its chain returns to it; the smallest node of each
//             cycle is its leader (Brent's cycle detection bounds the walk).
//   pop:      each leader walks its cycle, advancing every vertex's stack and
//             appending it to the next marked list.
// GLOBAL mode keeps per-(tree, vertex) records in HBM for a chunk of trees at
// a time and adds jump pointers over unchanged chain segments.  A jump from y
// to z is recorded with z's pop count; if any vertex strictly between them is
// later popped, its cycle runs through z, so z's pop count changes and the
// jump is rejected.  SHARED mode runs one tree per thread block with all
// state in shared memory.
#include <algorithm>
#include <cstdio>
#include <cstring>
#include <vector>

#include "rwc_common.cuh"
#include "smem_tree.cuh"

namespace rwc {
namespace {

constexpr int32_t TAG_FREE = -1;
constexpr int32_t TAG_SETTLED = -2;
constexpr int8_t CLS_OTHER = 0, CLS_LEADER = 1, CLS_TREE = 2;  // compressed-node classes

constexpr int ERR_BRENT = 1;     // compressed walk exceeded its bound
constexpr int ERR_LOOP = 4;      // a pointer chase exceeded n steps (internal error)

// ------------------------------------------------------------- GLOBAL mode
// Per (tree, vertex) record, 32 bytes:
//   w0 = p | tag << 32   (successor; tag = SETTLED, or the index in the marked
//                         list of round `stamp`)
//   w1 = k | stamp << 32 (pop count; round in which the vertex was last marked)
//   w2 = J | kj << 32    (jump target and the target's pop count when recorded)
// A vertex is marked in round r iff tag >= 0 and stamp == r, so marks of
// earlier rounds need no reset.
struct __align__(32) VRec {
    unsigned long long w0, w1, w2, w3;
};

__device__ __forceinline__ int32_t lo32(unsigned long long v) { return (int32_t)(uint32_t)v; }
__device__ __forceinline__ int32_t hi32(unsigned long long v) { return (int32_t)(uint32_t)(v >> 32); }
__device__ __forceinline__ unsigned long long pack(int32_t lo, int32_t hi) {
    return (unsigned long long)(uint32_t)lo | ((unsigned long long)(uint32_t)hi << 32);
}
__device__ __forceinline__ int32_t *tag_ptr(VRec *r) { return reinterpret_cast<int32_t *>(&r->w0) + 1; }

// first two words of a record in one 16-byte load
__device__ __forceinline__ ulonglong2 head(const VRec *r) {
    return *reinterpret_cast<const ulonglong2 *>(r);
}
// settled, or marked in round rr
__device__ __forceinline__ bool stops(ulonglong2 h, int32_t rr) {
    const int32_t tag = hi32(h.x);
    return tag == TAG_SETTLED || (tag >= 0 && hi32(h.y) == rr);
}

struct GState {
    VRec *rec;                 // [B][n]
    unsigned long long *M[2];  // marked lists: (tree << 32) | u; round r uses M[r & 1]
    int32_t *nm;               // [cap] compressed successor (-1 = reaches root)
    int64_t *cnt;              // [2] list lengths
    int *err;                  // device error word
    unsigned *done;            // blocks finished in the current pop launch
    unsigned long long *steps; // walk-step counter
    unsigned long long *marked;// marked entries over all rounds (= draws)
    int *round;                // current round (starts at 1)
    int64_t cap;
};

template <bool OFF64, bool W>
__global__ void __launch_bounds__(256) g_init(DevGraph g, GState s, int64_t B, uint32_t tree0,
                                              uint32_t k0, uint32_t k1) {
    const int64_t n = g.n, total = B * n;
    const int32_t root = g.root;
    for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < total;
         idx += (int64_t)gridDim.x * blockDim.x) {
        const int64_t t = idx / n;
        const int32_t u = (int32_t)(idx - t * n);
        VRec r;
        if (u == root) {
            r.w0 = pack(-1, TAG_SETTLED);
            r.w1 = 0ull;
        } else {
            const int64_t ord = t * (n - 1) + (u < root ? u : u - 1);
            const int32_t p = succ<OFF64, W>(g, u, 0u, tree0 + (uint32_t)t, 0u, k0, k1);
            r.w0 = pack(p, (int32_t)ord);
            r.w1 = pack(0, 1);
            s.M[1][ord] = ((unsigned long long)t << 32) | (uint32_t)u;
        }
        r.w2 = pack(-1, 0);
        r.w3 = 0ull;
        s.rec[idx] = r;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        s.cnt[0] = 0;
        s.cnt[1] = B * (n - 1);
        *s.round = 1;
        *s.done = 0;
    }
}

// Phase 1: walk from every marked vertex to the next marked or settled vertex.
__global__ void __launch_bounds__(256) g_walk(const int64_t n, GState s, int use_jumps) {
    const int32_t rr = *s.round;
    const int cur = rr & 1;
    const int64_t m = s.cnt[cur];
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        s.cnt[cur ^ 1] = 0;
        if (m) atomicAdd(s.marked, (unsigned long long)m);
    }
    unsigned long long local_steps = 0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < m;
         i += (int64_t)gridDim.x * blockDim.x) {
        const unsigned long long e = s.M[cur][i];
        VRec *base = s.rec + (int64_t)(e >> 32) * n;
        const int32_t u = (int32_t)(uint32_t)e;
        const int32_t first = lo32(base[u].w0);
        int32_t x = first, last = -1;
        uint32_t klast = 0;
        int64_t plain = 0, steps = 0;
        ulonglong2 hx;
        for (;;) {
            hx = head(base + x);
            if (stops(hx, rr)) break;
            if (++steps > n) { atomicOr(s.err, ERR_LOOP); hx.x = pack(0, TAG_SETTLED); break; }
            if (use_jumps) {
                const unsigned long long w2 = base[x].w2;
                const int32_t J = lo32(w2);
                if (J >= 0) {
                    const ulonglong2 hj = head(base + J);
                    if ((uint32_t)hj.y == (uint32_t)(w2 >> 32)) {
                        last = J; klast = (uint32_t)hj.y;
                        x = lo32(hj.x);
                        continue;
                    }
                }
            }
            last = x;
            klast = (uint32_t)hx.y;
            x = lo32(hx.x);
            ++plain;
        }
        local_steps += steps + 1;
        if (hi32(hx.x) == TAG_SETTLED) {
            // the whole segment reaches the root: settle what we can see
            s.nm[i] = -1;
            *tag_ptr(base + u) = TAG_SETTLED;
            int32_t y = first;
            for (int64_t q = 0;; ++q) {
                const ulonglong2 hy = head(base + y);
                if (stops(hy, rr)) break;
                if (q > n) { atomicOr(s.err, ERR_LOOP); break; }
                *tag_ptr(base + y) = TAG_SETTLED;
                y = lo32(hy.x);
            }
        } else {
            s.nm[i] = hi32(hx.x);
            if (use_jumps && plain > 2 && last >= 0) {
                // path compression: every vertex of the segment jumps to `last`
                int32_t y = first;
                const unsigned long long jw = pack(last, (int32_t)klast);
                for (int64_t q = 0; y != last; ++q) {
                    if (q > n) { atomicOr(s.err, ERR_LOOP); break; }
                    const unsigned long long w0 = base[y].w0, w2 = base[y].w2;
                    int32_t nx = lo32(w0);
                    const int32_t J = lo32(w2);
                    if (J >= 0 && J != last && (uint32_t)base[J].w1 == (uint32_t)(w2 >> 32)) nx = J;
                    base[y].w2 = jw;
                    y = nx;
                }
            }
        }
    }
    if (local_steps) atomicAdd(s.steps, local_steps);
}

__device__ __forceinline__ int64_t block_excl_scan(int64_t v, int64_t &total) {
    __shared__ int64_t warp_sums[32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    int64_t x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int64_t y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) warp_sums[wid] = x;
    __syncthreads();
    if (wid == 0) {
        int64_t t = lane < nw ? warp_sums[lane] : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int64_t y = __shfl_up_sync(0xffffffffu, t, o);
            if (lane >= o) t += y;
        }
        if (lane < nw) warp_sums[lane] = t;
    }
    __syncthreads();
    const int64_t before = (wid > 0 ? warp_sums[wid - 1] : 0) + x - v;
    total = warp_sums[nw - 1];
    __syncthreads();
    return before;
}

// Phase 2: classify each compressed node (leader of a cycle / reaches the
// root / other) and let the leaders pop their cycles; the last block to
// finish advances the round.
template <bool OFF64, bool W>
__global__ void __launch_bounds__(256) g_pop(DevGraph g, GState s, uint32_t tree0, uint32_t k0,
                                             uint32_t k1) {
    const int64_t n = g.n;
    const int32_t rr = *s.round;
    const int cur = rr & 1;
    const int64_t m = s.cnt[cur];
    __shared__ int64_t blockbase;
    for (int64_t chunk = blockIdx.x * (int64_t)blockDim.x; chunk < m;
         chunk += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = chunk + threadIdx.x;
        int64_t len = 0;
        VRec *base = nullptr;
        int32_t u0 = -1;
        int64_t t = 0;
        int8_t c = CLS_OTHER;
        if (i < m) {
            // Brent's cycle detection on the compressed graph; the smallest
            // index of a cycle is its leader
            int64_t x = s.nm[i];
            int64_t saved = -3, power = 1, lam = 0;
            for (int64_t it = 0;; ++it) {
                if (x < 0) { c = CLS_TREE; break; }
                if (x == i) { c = CLS_LEADER; break; }
                if (x < i || x == saved) break;
                if (it > 2 * m + 4) { atomicOr(s.err, ERR_BRENT); break; }
                if (++lam == power) { saved = x; power <<= 1; lam = 0; }
                x = s.nm[x];
            }
            const unsigned long long e = s.M[cur][i];
            t = (int64_t)(e >> 32);
            base = s.rec + t * n;
            u0 = (int32_t)(uint32_t)e;
            if (c == CLS_LEADER) {
                int32_t w = u0;
                do {
                    if (++len > n) { atomicOr(s.err, ERR_LOOP); len = 0; break; }
                    w = lo32(base[w].w0);
                } while (w != u0);
            }
        }
        int64_t total;
        const int64_t off = block_excl_scan(len, total);
        if (threadIdx.x == 0)
            blockbase = total ? (int64_t)atomicAdd((unsigned long long *)&s.cnt[cur ^ 1], (unsigned long long)total) : 0;
        __syncthreads();
        if (len) {
            int64_t pos = blockbase + off;
            int32_t w = u0;
            const uint32_t tree = tree0 + (uint32_t)t;
            do {
                const ulonglong2 hw = head(base + w);
                const int32_t nx = lo32(hw.x);
                const uint32_t k = (uint32_t)hw.y + 1u;
                const int32_t p = succ<OFF64, W>(g, w, k, tree, 0u, k0, k1);
                base[w].w0 = pack(p, (int32_t)pos);
                base[w].w1 = pack((int32_t)k, rr + 1);
                base[w].w2 = pack(-1, 0);
                s.M[cur ^ 1][pos] = ((unsigned long long)t << 32) | (uint32_t)w;
                ++pos;
                w = nx;
            } while (w != u0);
        }
        if (c == CLS_TREE) {
            int32_t y = u0;
            int64_t q = 0;
            for (;;) {
                if (++q > n) { atomicOr(s.err, ERR_LOOP); break; }
                *tag_ptr(base + y) = TAG_SETTLED;
                y = lo32(base[y].w0);
                if (stops(head(base + y), rr)) break;
            }
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        __threadfence();
        if (atomicAdd(s.done, 1u) == gridDim.x - 1) {
            *s.done = 0;
            *s.round = rr + 1;
        }
    }
}

// Final: visits_u = k_u + 1 summed over the chunk's trees into sums (FP64).
__global__ void __launch_bounds__(256) g_accum(const int64_t n, const int32_t root, const VRec *rec,
                                               int64_t B, double *sums, int32_t *parents,
                                               int32_t *visits) {
    for (int64_t u = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; u < n;
         u += (int64_t)gridDim.x * blockDim.x) {
        int64_t acc = 0;
        for (int64_t t = 0; t < B; ++t) {
            const VRec &r = rec[t * n + u];
            const int32_t k = (int32_t)(uint32_t)r.w1;
            const int32_t vis = (u == root) ? 0 : k + 1;
            acc += vis;
            if (parents) parents[t * n + u] = (u == root) ? -1 : lo32(r.w0);
            if (visits) visits[t * n + u] = vis;
        }
        if (sums && u != root) sums[u] += (double)acc;
    }
}

size_t shared_bytes(int64_t n) { return smem_tree_bytes(n); }

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

struct Scratch {
    void *p = nullptr;
    cudaStream_t st = nullptr;
    explicit Scratch(cudaStream_t s) : st(s) {}
    ~Scratch() { if (p) cudaFreeAsync(p, st); }
};

}  // namespace

static rwc_status sample_shared(rwc_graph *G, uint64_t seed, int64_t tree0, int64_t T, double *sums,
                                int32_t *parents, int32_t *visits, const rwc_options_t &o,
                                rwc_stats_t *st, cudaStream_t stream) {
    const DevGraph &g = G->g;
    const size_t smem = shared_bytes(g.n);
    int threads = o.block_threads > 0 ? o.block_threads : (g.n <= 4096 ? 256 : 512);
    threads = std::max(32, std::min(1024, threads / 32 * 32));
    Scratch scr(stream);
    RWC_CUDA_TRY(cudaMallocAsync(&scr.p, 64, stream));
    int *err = (int *)scr.p;
    unsigned long long *rounds = (unsigned long long *)((char *)scr.p + 16);
    RWC_CUDA_TRY(cudaMemsetAsync(scr.p, 0, 64, stream));
    // rounds and draws counters are adjacent: rounds[0], rounds[1]
    const uint32_t k0 = (uint32_t)seed, k1 = (uint32_t)(seed >> 32);
    const int64_t max_rounds = o.max_rounds > 0 ? o.max_rounds : (1 << 22);
    const bool prof = o.profile != 0;
    cudaEvent_t ev[2] = {nullptr, nullptr};
    if (prof) { cudaEventCreate(&ev[0]); cudaEventCreate(&ev[1]); }
    rwc_status status = RWC_OK;
    dispatch(g, [&](auto off64, auto wt) {
        constexpr bool O = decltype(off64)::value, Wt = decltype(wt)::value;
        auto kern = s_trees<O, Wt>;
        cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        int per_sm = 0;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, threads, smem);
        if (per_sm < 1) { status = set_error(RWC_ERR_UNSUPPORTED, "graph too large for shared mode"); return; }
        const int64_t blocks = std::min<int64_t>(T, (int64_t)num_sms() * per_sm);
        if (prof) cudaEventRecord(ev[0], stream);
        ::rwc::count_launches(1); kern<<<(unsigned)blocks, threads, smem, stream>>>(g, (uint32_t)tree0, T, k0, k1, 0u, max_rounds,
                                                          sums, parents, visits, err, rounds);
        if (prof) cudaEventRecord(ev[1], stream);
    });
    RWC_TRY(status);
    RWC_CUDA_TRY(cudaGetLastError());
    if (o.async_status) {
        // no host synchronisation: the error bits go to the graph's status word
        ::rwc::count_launches(1);
        fold_status<<<1, 1, 0, stream>>>(err, 1, G->dev_status);
        RWC_CUDA_TRY(cudaGetLastError());
        return RWC_OK;
    }
    int64_t *h = G->host_scalars;
    RWC_CUDA_TRY(cudaMemcpyAsync(h, scr.p, 32, cudaMemcpyDeviceToHost, stream));
    RWC_CUDA_TRY(cudaStreamSynchronize(stream));
    if (prof) {
        float ms = 0.f;
        cudaEventElapsedTime(&ms, ev[0], ev[1]);
        if (st) { st->phase_ms[RWC_PHASE_WALK] += ms; st->phase_launches[RWC_PHASE_WALK] += 1; }
        cudaEventDestroy(ev[0]);
        cudaEventDestroy(ev[1]);
    }
    const int e = (int)(h[0] & 0xffffffff);
    if (e & SM_ERR_KOVF) return set_error(RWC_ERR_UNSUPPORTED, "a vertex was popped more than 65535 times; use RWC_MODE_GLOBAL");
    if (e & SM_ERR_LOOP) return set_error(RWC_ERR_CUDA, "sampler internal check failed");
    if (e) return set_error(RWC_ERR_NOT_CONVERGED, "cycle popping exceeded max_rounds");
    if (st) {
        st->rounds += h[2];
        st->draws += h[3];
        st->marked += h[3];
        st->chunks += 1;
        st->mode = RWC_MODE_SHARED;
        st->phase_units[RWC_PHASE_WALK] += h[3];
    }
    return RWC_OK;
}

static rwc_status sample_global(rwc_graph *G, uint64_t seed, int64_t tree0, int64_t T, double *sums,
                                int32_t *parents, int32_t *visits, const rwc_options_t &o,
                                rwc_stats_t *st, cudaStream_t stream) {
    const DevGraph &g = G->g;
    const int64_t n = g.n;
    const size_t per_tree = (size_t)n * (sizeof(VRec) + 2 * 8 + 4) + 256;
    int64_t B = o.trees_per_chunk;
    if (B <= 0) {
        size_t fr = 0, tot = 0;
        RWC_CUDA_TRY(cudaMemGetInfo(&fr, &tot));
        size_t budget = o.memory_budget > 0 ? (size_t)o.memory_budget : (size_t)(fr * 0.6);
        B = (int64_t)std::max<size_t>(1, budget / per_tree);
    }
    B = std::min(B, T);
    // list indices are int32 tags
    B = std::min<int64_t>(B, std::max<int64_t>(1, ((int64_t)1 << 31) / std::max<int64_t>(1, n - 1) - 1));
    const int use_jumps = o.use_jumps < 0 ? 1 : o.use_jumps;
    const int64_t max_rounds = o.max_rounds > 0 ? o.max_rounds : (1 << 22);
    const uint32_t k0 = (uint32_t)seed, k1 = (uint32_t)(seed >> 32);
    const int64_t cap = B * (n - 1);

    Scratch scr(stream);
    const size_t bytes = (size_t)B * n * sizeof(VRec) + 2 * (size_t)cap * 8 + (size_t)cap * 4 + 256;
    RWC_CUDA_TRY(cudaMallocAsync(&scr.p, bytes, stream));
    char *p = (char *)scr.p;
    GState s;
    s.rec = (VRec *)p; p += (size_t)B * n * sizeof(VRec);
    s.M[0] = (unsigned long long *)p; p += (size_t)cap * 8;
    s.M[1] = (unsigned long long *)p; p += (size_t)cap * 8;
    s.nm = (int32_t *)p; p += (size_t)cap * 4;
    p = (char *)(((uintptr_t)p + 63) & ~(uintptr_t)63);
    // scratch tail: cnt[2] @0, err @16, done @20, steps @24, marked @32, round @40
    char *tail = p;
    s.cnt = (int64_t *)tail;
    s.err = (int *)(tail + 16);
    s.done = (unsigned *)(tail + 20);
    s.steps = (unsigned long long *)(tail + 24);
    s.marked = (unsigned long long *)(tail + 32);
    s.round = (int *)(tail + 40);
    s.cap = cap;

    const bool prof = o.profile != 0;
    constexpr int Q = 32;          // rounds per captured graph
    // events: [2q], [2q+1] around walk of round q; [2Q + 2q], +1 around pop;
    // [4Q..4Q+3] around init and accum
    std::vector<cudaEvent_t> ev;
    if (prof) {
        ev.resize(4 * Q + 4);
        for (auto &e : ev) cudaEventCreate(&e);
    }
    struct Guard {
        std::vector<cudaEvent_t> &v;
        cudaGraphExec_t exec = nullptr;
        cudaStream_t cs = nullptr;
        ~Guard() {
            for (auto e : v) cudaEventDestroy(e);
            if (exec) cudaGraphExecDestroy(exec);
            if (cs) cudaStreamDestroy(cs);
        }
    } guard{ev};
    auto ms_between = [&](int a, int b) {
        float ms = 0.f;
        cudaEventElapsedTime(&ms, ev[a], ev[b]);
        return (double)ms;
    };
    RWC_CUDA_TRY(cudaStreamCreateWithFlags(&guard.cs, cudaStreamNonBlocking));
    const int sms = num_sms();
    const unsigned grid = (unsigned)(sms * 8);
    int64_t *h = G->host_scalars;
    int64_t tot_steps = 0, tot_marked = 0;
    for (int64_t c0 = 0; c0 < T; c0 += B) {
        const int64_t Bc = std::min(B, T - c0);
        const uint32_t t0 = (uint32_t)(tree0 + c0);
        RWC_CUDA_TRY(cudaMemsetAsync(tail, 0, 48, stream));
        if (prof) cudaEventRecord(ev[4 * Q], stream);
        dispatch(g, [&](auto off64, auto wt) {
            constexpr bool O = decltype(off64)::value, Wt = decltype(wt)::value;
            ::rwc::count_launches(1);
            g_init<O, Wt><<<grid, 256, 0, stream>>>(g, s, Bc, t0, k0, k1);
        });
        if (prof) cudaEventRecord(ev[4 * Q + 1], stream);
        RWC_CUDA_TRY(cudaGetLastError());
        // capture Q rounds once per chunk; replays advance the device round
        if (guard.exec) { cudaGraphExecDestroy(guard.exec); guard.exec = nullptr; }
        {
            cudaGraph_t gr = nullptr;
            RWC_CUDA_TRY(cudaStreamBeginCapture(guard.cs, cudaStreamCaptureModeThreadLocal));
            for (int q = 0; q < Q; ++q) {
                // events recorded inside the captured rounds must be external
                // records (graph nodes that record them on replay) to be timed
                if (prof) cudaEventRecordWithFlags(ev[2 * q], guard.cs, cudaEventRecordExternal);
                g_walk<<<grid, 256, 0, guard.cs>>>(n, s, use_jumps);
                if (prof) {
                    cudaEventRecordWithFlags(ev[2 * q + 1], guard.cs, cudaEventRecordExternal);
                    cudaEventRecordWithFlags(ev[2 * Q + 2 * q], guard.cs, cudaEventRecordExternal);
                }
                dispatch(g, [&](auto off64, auto wt) {
                    constexpr bool O = decltype(off64)::value, Wt = decltype(wt)::value;
                    g_pop<O, Wt><<<grid, 256, 0, guard.cs>>>(g, s, t0, k0, k1);
                });
                if (prof) cudaEventRecordWithFlags(ev[2 * Q + 2 * q + 1], guard.cs, cudaEventRecordExternal);
            }
            const cudaError_t ce = cudaStreamEndCapture(guard.cs, &gr);
            if (ce != cudaSuccess) {
                if (gr) cudaGraphDestroy(gr);
                return set_error(RWC_ERR_CUDA, "capturing the round graph failed: %s", cudaGetErrorString(ce));
            }
            const cudaError_t ie = cudaGraphInstantiate(&guard.exec, gr, 0);
            cudaGraphDestroy(gr);
            RWC_CUDA_TRY(ie);
        }
        int64_t rounds = 0;
        for (;;) {
            ::rwc::count_launches(2 * Q);
            RWC_CUDA_TRY(cudaGraphLaunch(guard.exec, stream));
            rounds += Q;
            RWC_CUDA_TRY(cudaMemcpyAsync(h, tail, 48, cudaMemcpyDeviceToHost, stream));
            RWC_CUDA_TRY(cudaStreamSynchronize(stream));
            if (prof && st) {
                for (int q = 0; q < Q; ++q) {
                    st->phase_ms[RWC_PHASE_WALK] += ms_between(2 * q, 2 * q + 1);
                    st->phase_ms[RWC_PHASE_POP] += ms_between(2 * Q + 2 * q, 2 * Q + 2 * q + 1);
                }
                st->phase_launches[RWC_PHASE_WALK] += Q;
                st->phase_launches[RWC_PHASE_POP] += Q;
            }
            const int err = (int)(h[2] & 0xffffffff);
            if (err)
                return set_error(RWC_ERR_CUDA, "sampler internal check failed (code %d)", err);
            const int32_t rr = (int32_t)(h[5] & 0xffffffff);
            if (h[rr & 1] == 0) break;
            if (rounds >= max_rounds)
                return set_error(RWC_ERR_NOT_CONVERGED, "cycle popping exceeded max_rounds (%lld)", (long long)max_rounds);
        }
        if (prof) cudaEventRecord(ev[4 * Q + 2], stream);
        ::rwc::count_launches(1);
        g_accum<<<grid, 256, 0, stream>>>(n, g.root, s.rec, Bc, sums,
                                          parents ? parents + c0 * n : nullptr,
                                          visits ? visits + c0 * n : nullptr);
        if (prof) cudaEventRecord(ev[4 * Q + 3], stream);
        RWC_CUDA_TRY(cudaGetLastError());
        RWC_CUDA_TRY(cudaStreamSynchronize(stream));
        tot_steps += (int64_t)h[3];
        tot_marked += (int64_t)h[4];
        if (st) {
            st->rounds += (int64_t)(h[5] & 0xffffffff) - 1;
            st->chunks += 1;
            st->phase_units[RWC_PHASE_INIT] += Bc * n;
            st->phase_units[RWC_PHASE_ACCUM] += Bc * n;
            st->phase_units[RWC_PHASE_POP] += (int64_t)h[4] - Bc * (n - 1);
            if (prof) {
                st->phase_ms[RWC_PHASE_INIT] += ms_between(4 * Q, 4 * Q + 1);
                st->phase_ms[RWC_PHASE_ACCUM] += ms_between(4 * Q + 2, 4 * Q + 3);
                st->phase_launches[RWC_PHASE_INIT] += 1;
                st->phase_launches[RWC_PHASE_ACCUM] += 1;
            }
        }
    }
    if (st) {
        st->mode = RWC_MODE_GLOBAL;
        st->walk_steps = tot_steps;
        st->marked = tot_marked;
        st->draws = tot_marked;
        st->phase_units[RWC_PHASE_WALK] = tot_steps;
        st->phase_units[RWC_PHASE_CLASSIFY] = tot_marked;
        st->phase_units[RWC_PHASE_FINISH] = 0;
    }
    return RWC_OK;
}

}  // namespace rwc

extern "C" rwc_status rwc_sample_trees(rwc_graph_t *G, uint64_t seed, int64_t tree0, int64_t T,
                                       double *sums, int32_t *parents, int32_t *visits,
                                       const rwc_options_t *opt, rwc_stats_t *stats,
                                       rwc_stream_t stream) {
    using namespace rwc;
    clear_error();
    if (!G) return set_error(RWC_ERR_INVALID, "graph is NULL");
    if (T < 0 || tree0 < 0 || tree0 + T > ((int64_t)1 << 32))
        return set_error(RWC_ERR_INVALID, "tree range must lie in [0, 2^32)");
    rwc_options_t o;
    memset(&o, 0, sizeof(o));
    o.use_jumps = -1;
    if (opt) o = *opt;
    if (stats) memset(stats, 0, sizeof(*stats));
    if (o.walker_policy < 0 || o.walker_policy > 4)
        return set_error(RWC_ERR_INVALID, "unknown walker policy %d", o.walker_policy);
    if (T == 0) return RWC_OK;
    const DevGraph &g = G->g;
    int mode = o.mode;
    if (mode == RWC_MODE_AUTO)
        mode = (g.n <= 20000 && shared_bytes(g.n) <= 200 * 1024) ? RWC_MODE_SHARED : RWC_MODE_WALKER;
    if (mode == RWC_MODE_SHARED && (g.n > 32767 || shared_bytes(g.n) > 227 * 1024))
        return set_error(RWC_ERR_UNSUPPORTED, "shared mode needs n <= 20000");
    if (o.async_status) {
        if (stats || o.profile)
            return set_error(RWC_ERR_INVALID, "asynchronous sampling (async_status = 1) fills no "
                                              "statistics: pass stats = NULL and profile = 0");
        if (mode == RWC_MODE_GLOBAL || (mode == RWC_MODE_WALKER && o.walker_policy == 4))
            return set_error(RWC_ERR_UNSUPPORTED, "asynchronous sampling needs WALKER mode (policies "
                                                  "0-3) or SHARED mode");
    }
    rwc_status s;
    try {
        if (mode == RWC_MODE_SHARED)
            s = sample_shared(G, seed, tree0, T, sums, parents, visits, o, stats, (cudaStream_t)stream);
        else if (mode == RWC_MODE_WALKER)
            s = sample_walker(G, seed, tree0, T, sums, parents, visits, o, stats, (cudaStream_t)stream);
        else if (mode == RWC_MODE_GLOBAL)
            s = sample_global(G, seed, tree0, T, sums, parents, visits, o, stats, (cudaStream_t)stream);
        else
            return set_error(RWC_ERR_INVALID, "unknown sampler mode %d", mode);
    } catch (const std::bad_alloc &) {
        return set_error(RWC_ERR_OOM, "host allocation failed");
    }
    if (s == RWC_OK && stats) stats->trees = T;
    return s;
}

extern "C" rwc_status rwc_sync_status(rwc_graph_t *G, rwc_stream_t stream) {
    using namespace rwc;
    clear_error();
    if (!G) return set_error(RWC_ERR_INVALID, "graph is NULL");
    RWC_CUDA_TRY(cudaStreamSynchronize((cudaStream_t)stream));
    int e = 0;
    RWC_CUDA_TRY(cudaMemcpy(&e, G->dev_status, sizeof(int), cudaMemcpyDeviceToHost));
    if (!e) return RWC_OK;
    RWC_CUDA_TRY(cudaMemset(G->dev_status, 0, sizeof(int)));
    if (e & STATUS_KOVF) return set_error(RWC_ERR_UNSUPPORTED, "a vertex was popped too many times "
                                          "(2^20 - 1 in WALKER mode, 65535 in SHARED mode)");
    if (e & STATUS_INTERNAL) return set_error(RWC_ERR_CUDA, "sampler internal check failed");
    if (e & STATUS_WAIT) return set_error(RWC_ERR_NOT_CONVERGED, "a walker wait exceeded its bound");
    return set_error(RWC_ERR_NOT_CONVERGED, "cycle popping exceeded max_rounds");
}

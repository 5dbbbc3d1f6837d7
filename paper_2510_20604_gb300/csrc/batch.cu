// Batched sampler: all trees of thousands of small graphs in one CUDA-graph
// launch.  Work items (graph, tile of trees) are pulled from device counters
// by persistent kernels (no grid-wide barrier).  The graphs are split by size:
// those with more than `split` vertices run block-per-tree; the others run
// warp-per-tree (every warp of a block pulls its own items and keeps its tree
// in its own slice of the block's shared memory) or block-per-tree with small
// blocks, as the schedule says.  The two classes run as two persistent
// kernels on forked streams, so each gets the shared-memory size (and thus
// the occupancy) its own graphs need; the fork and join are captured into the
// call's CUDA graph, which is replayed.  The autotuner times candidate
// schedules on the device.  Tree state lives in shared memory (smem_tree.cuh).
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "rwc_common.cuh"
#include "smem_tree.cuh"

namespace rwc {
namespace {

struct BGraph {
    int64_t voff;   // first vertex in the concatenated arrays
    int32_t n;
    int32_t root;
};

struct BItem {
    int32_t g;
    int32_t tile;   // index of the tile of trees within the graph
};

// One work item: the tiles' trees of graph it.g, run by the group Grp whose
// tree state is carved from `region`.  Adds the visit totals to sums.
// Returns the group-uniform error mask.
template <bool OFF64, bool W, class Grp>
__device__ int run_item(const DevGraph &base, const BGraph *__restrict__ graphs, BItem it,
                        unsigned char *region, int tile, int64_t T, uint32_t k0, uint32_t k1,
                        int64_t max_rounds, double *sums, unsigned long long *round_ctr) {
    const BGraph bg = graphs[it.g];
    DevGraph g = base;
    g.n = bg.n;
    g.root = bg.root;
    if (OFF64) g.rp64 = base.rp64 + bg.voff;
    else g.rp32 = base.rp32 + bg.voff;
    SmemTree S;
    S.carve(region, bg.n);
    for (int u = Grp::rank(); u < bg.n; u += Grp::size()) S.acc[u] = 0;
    const int64_t t0 = (int64_t)it.tile * tile, t1 = std::min<int64_t>(T, t0 + tile);
    int mask = 0;
    unsigned long long rounds = 0;
    for (int64_t t = t0; t < t1 && !mask; ++t) {
        int64_t r = 0;
        mask = smem_tree<OFF64, W, Grp>(g, S, (uint32_t)t, (uint32_t)it.g, k0, k1, max_rounds,
                                        nullptr, nullptr, &r);
        rounds += (unsigned long long)r;
    }
    Grp::sync();
    if (mask) return mask;
    unsigned long long draws = 0;
    for (int u = Grp::rank(); u < bg.n; u += Grp::size()) {
        draws += S.acc[u];
        if (S.acc[u]) atomicAdd(sums + bg.voff + u, (double)S.acc[u]);
    }
    if (draws) atomicAdd(round_ctr + 1, draws);
    if (Grp::rank() == 0 && rounds) atomicAdd(round_ctr, rounds);
    return 0;
}

// Persistent kernel over both item lists: first every block pulls
// block-per-tree items, then every warp pulls warp-per-tree items into its
// own shared-memory slice of warp_slice bytes.
template <bool OFF64, bool W>
__global__ void b_persistent(DevGraph base, const BGraph *__restrict__ graphs,
                             const BItem *__restrict__ bitems, int64_t nb,
                             const BItem *__restrict__ witems, int64_t nw, int *next_item,
                             int warp_slice, int tile, int64_t T, uint32_t k0, uint32_t k1,
                             int64_t max_rounds, double *sums, int *err,
                             unsigned long long *round_ctr) {
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ int item;
    for (;;) {
        __syncthreads();
        if (threadIdx.x == 0) item = atomicAdd(next_item, 1);
        __syncthreads();
        const int i = item;
        if (i >= nb) break;
        const int mask = run_item<OFF64, W, BlockGroup>(base, graphs, bitems[i], smem, tile, T, k0, k1,
                                                        max_rounds, sums, round_ctr);
        if (mask) { if (threadIdx.x == 0) atomicOr(err, mask); return; }
    }
    if (nw == 0) return;
    unsigned char *region = smem + (size_t)(threadIdx.x >> 5) * warp_slice;
    for (;;) {
        int i = 0;
        if ((threadIdx.x & 31) == 0) i = atomicAdd(next_item + 1, 1);
        i = __shfl_sync(0xffffffffu, i, 0);
        if (i >= nw) break;
        const int mask = run_item<OFF64, W, WarpGroup>(base, graphs, witems[i], region, tile, T, k0, k1,
                                                       max_rounds, sums, round_ctr);
        if (mask) { if ((threadIdx.x & 31) == 0) atomicOr(err, mask); return; }
    }
}

template <class F>
void dispatch(bool off64, bool weighted, F f) {
    if (off64) {
        if (weighted) f(std::true_type{}, std::true_type{});
        else f(std::true_type{}, std::false_type{});
    } else {
        if (weighted) f(std::false_type{}, std::true_type{});
        else f(std::false_type{}, std::false_type{});
    }
}

}  // namespace
}  // namespace rwc

using namespace rwc;

struct rwc_batch {
    int32_t G = 0;
    int64_t N = 0, nnz = 0;
    bool off64 = false, weighted = false;
    std::vector<BGraph> hgraphs;
    std::vector<int32_t> roots;
    DevGraph base;                     // concatenated CSR (local column ids)
    BGraph *graphs = nullptr;
    // schedule: block size of the large graphs, the largest n of the small
    // class (0: one class), small class warp-per-tree (1) or block-per-tree
    // with SMALL_THREADS threads (0), trees per work item
    int threads = 512;
    int split = 1024;
    int warp = 1;
    int tile = 4;
    int conc = 1;                      // 1: the classes run concurrently (forked streams)
    cudaStream_t side = nullptr;       // the small class's stream (forked from the call's)
    cudaEvent_t fork = nullptr, join = nullptr;
    int max_n[2] = {0, 0};             // largest n of the block / warp item lists
    BItem *items[2] = {nullptr, nullptr};
    int64_t nitems[2] = {0, 0};
    int64_t items_T = -1;              // T the item lists were built for
    int64_t items_tile = -1, items_split = -1;
    void *scratch = nullptr;           // [0] err, [8] rounds, [16] draws, [32..48) item counters
    std::vector<void *> allocs;
    // captured launches
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    uint64_t cap_seed = 0;
    int64_t cap_T = -1;
    double *cap_sums = nullptr;
    cudaStream_t cap_stream = nullptr;
    int64_t *host = nullptr;
};

namespace {

cudaError_t balloc(rwc_batch *b, void **p, size_t bytes) {
    cudaError_t e = cudaMalloc(p, bytes ? bytes : 16);
    if (e == cudaSuccess) b->allocs.push_back(*p);
    return e;
}

void drop_graph(rwc_batch *b) {
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    b->exec = nullptr;
    b->graph = nullptr;
    b->cap_T = -1;
}

// Bytes of one warp's shared-memory slice for trees of up to n vertices.
size_t warp_slice_bytes(int n) { return (smem_tree_bytes(n) + 15) & ~(size_t)15; }

constexpr int SMALL_THREADS = 256;   // block size of the small class (8 warps)

// Dynamic shared memory of each class's kernel for the current schedule.
size_t class_smem(const rwc_batch *b, int c) {
    if (!b->nitems[c]) return 64;
    if (c == 1 && b->warp) return (size_t)(SMALL_THREADS / 32) * warp_slice_bytes(b->max_n[1]);
    return std::max<size_t>(smem_tree_bytes(b->max_n[c]), 64);
}
size_t batch_smem(const rwc_batch *b) { return std::max(class_smem(b, 0), class_smem(b, 1)); }

// Work items for T trees per graph: list 0 (block-per-tree) holds graphs with
// more than `split` vertices, list 1 (warp-per-tree) the others; each list
// runs its largest graphs first.
rwc_status build_items(rwc_batch *b, int64_t T) {
    if (b->items_T == T && b->items_tile == b->tile && b->items_split == b->split) return RWC_OK;
    for (int c = 0; c < 2; ++c) {
        std::vector<BItem> v;
        std::vector<int32_t> order;
        for (int32_t g = 0; g < b->G; ++g) {
            const int cls = b->hgraphs[g].n <= b->split ? 1 : 0;
            if (cls == c) order.push_back(g);
        }
        std::stable_sort(order.begin(), order.end(),
                         [&](int32_t x, int32_t y) { return b->hgraphs[x].n > b->hgraphs[y].n; });
        const int64_t ntile = (T + b->tile - 1) / b->tile;
        for (int32_t g : order)
            for (int64_t t = 0; t < ntile; ++t) v.push_back(BItem{g, (int32_t)t});
        if (b->items[c]) { cudaFree(b->items[c]); b->allocs.erase(std::find(b->allocs.begin(), b->allocs.end(), (void *)b->items[c])); }
        b->items[c] = nullptr;
        b->nitems[c] = (int64_t)v.size();
        if (!v.empty()) {
            RWC_CUDA_TRY(balloc(b, (void **)&b->items[c], v.size() * sizeof(BItem)));
            RWC_CUDA_TRY(cudaMemcpy(b->items[c], v.data(), v.size() * sizeof(BItem), cudaMemcpyHostToDevice));
        }
        b->max_n[c] = 0;
        for (int32_t g : order) b->max_n[c] = std::max(b->max_n[c], b->hgraphs[g].n);
    }
    b->items_T = T;
    b->items_tile = b->tile;
    b->items_split = b->split;
    drop_graph(b);
    return RWC_OK;
}

// Enqueue one call: the large class on st, the small class on the batch's
// side stream forked from st and joined back.
rwc_status enqueue(rwc_batch *b, uint64_t seed, int64_t T, double *sums, cudaStream_t st) {
    int *err = (int *)b->scratch;
    unsigned long long *rounds = (unsigned long long *)((char *)b->scratch + 8);
    int *counters = (int *)((char *)b->scratch + 32);   // [0..1] large class, [2..3] small class
    RWC_CUDA_TRY(cudaMemsetAsync((char *)b->scratch + 32, 0, 16, st));
    const uint32_t k0 = (uint32_t)seed, k1 = (uint32_t)(seed >> 32);
    if (batch_smem(b) > 227 * 1024) return set_error(RWC_ERR_UNSUPPORTED, "batch schedule needs %zu bytes of shared memory", batch_smem(b));
    const bool fork = b->conc && b->nitems[0] && b->nitems[1];
    if (fork) {
        RWC_CUDA_TRY(cudaEventRecord(b->fork, st));
        RWC_CUDA_TRY(cudaStreamWaitEvent(b->side, b->fork, 0));
    }
    rwc_status status = RWC_OK;
    for (int c = 0; c < 2 && status == RWC_OK; ++c) {
        if (!b->nitems[c]) continue;
        const bool warp = c == 1 && b->warp;
        const int threads = c == 0 ? b->threads : SMALL_THREADS;
        const size_t smem = class_smem(b, c);
        cudaStream_t s = (c == 1 && fork) ? b->side : st;
        dispatch(b->off64, b->weighted, [&](auto o64, auto wt) {
            auto kern = b_persistent<decltype(o64)::value, decltype(wt)::value>;
            cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            int per_sm = 0;
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, threads, smem);
            if (per_sm < 1) { status = set_error(RWC_ERR_UNSUPPORTED, "batch block does not fit on an SM"); return; }
            const int64_t per_block = warp ? threads / 32 : 1;
            const int64_t want = (b->nitems[c] + per_block - 1) / per_block;
            const int64_t blocks = std::max<int64_t>(1, std::min<int64_t>(want, (int64_t)num_sms() * per_sm));
            ::rwc::count_launches(1);
            kern<<<(unsigned)blocks, threads, smem, s>>>(
                b->base, b->graphs, warp ? nullptr : b->items[c], warp ? 0 : b->nitems[c],
                warp ? b->items[c] : nullptr, warp ? b->nitems[c] : 0, counters + 2 * c,
                warp ? (int)warp_slice_bytes(b->max_n[c]) : 0, b->tile, T, k0, k1, (int64_t)1 << 22,
                sums, err, rounds);
        });
    }
    if (fork) {
        RWC_CUDA_TRY(cudaEventRecord(b->join, b->side));
        RWC_CUDA_TRY(cudaStreamWaitEvent(st, b->join, 0));
    }
    RWC_TRY(status);
    RWC_CUDA_TRY(cudaGetLastError());
    return RWC_OK;
}

rwc_status finish(rwc_batch *b, rwc_stats_t *stats, int mode, int64_t T, cudaStream_t st) {
    RWC_CUDA_TRY(cudaMemcpyAsync(b->host, b->scratch, 24, cudaMemcpyDeviceToHost, st));
    RWC_CUDA_TRY(cudaStreamSynchronize(st));
    const int e = (int)(b->host[0] & 0xffffffff);
    if (e & SM_ERR_KOVF) return set_error(RWC_ERR_UNSUPPORTED, "a vertex was popped more than 65535 times");
    if (e & SM_ERR_LOOP) return set_error(RWC_ERR_CUDA, "sampler internal check failed");
    if (e) return set_error(RWC_ERR_NOT_CONVERGED, "cycle popping exceeded max_rounds");
    if (stats) {
        stats->trees = T * b->G;
        stats->rounds = b->host[1];
        stats->draws = b->host[2];
        stats->marked = b->host[2];
        stats->chunks = 1;
        stats->mode = mode;
        stats->block_threads = mode == 3 ? 0 : b->threads;   // the large class's block size
    }
    return RWC_OK;
}

}  // namespace

extern "C" rwc_status rwc_batch_create(int32_t G, const int64_t *voff, const int64_t *rp,
                                       const int32_t *col, const float *w, rwc_batch_t **out) {
    clear_error();
    if (!out || G <= 0 || !voff || !rp || !col) return set_error(RWC_ERR_INVALID, "bad argument");
    *out = nullptr;
    if (voff[0] != 0) return set_error(RWC_ERR_INVALID, "graph offsets must start at 0");
    const int64_t N = voff[G];
    const int64_t nnz = rp[N];
    if (rp[0] != 0) return set_error(RWC_ERR_INVALID, "row_ptr[0] must be 0");
    std::vector<BGraph> hg(G);
    std::vector<int32_t> roots(G);
    std::vector<int64_t> lrp;
    for (int32_t g = 0; g < G; ++g) {
        const int64_t v0 = voff[g], n = voff[g + 1] - v0;
        if (n < 2 || n > 20000) return set_error(RWC_ERR_INVALID, "graph %d: batch graphs need 2 <= n <= 20000", g);
        lrp.resize(n + 1);
        for (int64_t u = 0; u <= n; ++u) lrp[u] = rp[v0 + u] - rp[v0];
        const int32_t *gc = col + rp[v0];
        const float *gw = w ? w + rp[v0] : nullptr;
        rwc_status s = validate_csr(n, lrp[n], lrp.data(), gc, gw);
        if (s != RWC_OK) return set_error(s, "graph %d: %s", g, rwc_last_error());
        if (!csr_connected(n, lrp.data(), gc)) return set_error(RWC_ERR_NOT_CONNECTED, "graph %d is not connected", g);
        double best = -1.0;
        int32_t arg = 0;
        for (int64_t u = 0; u < n; ++u) {
            double d = 0.0;
            if (gw) for (int64_t j = lrp[u]; j < lrp[u + 1]; ++j) d = d + (double)gw[j - 0];
            else d = (double)(lrp[u + 1] - lrp[u]);
            if (d > best) { best = d; arg = (int32_t)u; }
        }
        hg[g] = BGraph{v0, (int32_t)n, arg};
        roots[g] = arg;
    }
    rwc_batch *b = new (std::nothrow) rwc_batch();
    if (!b) return set_error(RWC_ERR_OOM, "host allocation failed");
    auto fail = [&](cudaError_t e) {
        for (void *p : b->allocs) cudaFree(p);
        if (b->host) cudaFreeHost(b->host);
        delete b;
        return set_error(e == cudaErrorMemoryAllocation ? RWC_ERR_OOM : RWC_ERR_CUDA, "batch upload: %s",
                         cudaGetErrorString(e));
    };
    b->G = G; b->N = N; b->nnz = nnz; b->hgraphs = hg; b->roots = roots;
    b->weighted = (w != nullptr);
    b->off64 = nnz >= ((int64_t)1 << 31) - 1;
    cudaError_t e;
    DevGraph &d = b->base;
    d.n = N; d.nnz = nnz; d.weighted = b->weighted; d.off64 = b->off64;
    if (b->off64) {
        int64_t *p;
        if ((e = balloc(b, (void **)&p, (N + 1) * 8)) != cudaSuccess) return fail(e);
        if ((e = cudaMemcpy(p, rp, (N + 1) * 8, cudaMemcpyHostToDevice)) != cudaSuccess) return fail(e);
        d.rp64 = p;
    } else {
        std::vector<int32_t> r32(N + 1);
        for (int64_t i = 0; i <= N; ++i) r32[i] = (int32_t)rp[i];
        int32_t *p;
        if ((e = balloc(b, (void **)&p, (N + 1) * 4)) != cudaSuccess) return fail(e);
        if ((e = cudaMemcpy(p, r32.data(), (N + 1) * 4, cudaMemcpyHostToDevice)) != cudaSuccess) return fail(e);
        d.rp32 = p;
    }
    {
        int32_t *p;
        if ((e = balloc(b, (void **)&p, nnz * 4)) != cudaSuccess) return fail(e);
        if ((e = cudaMemcpy(p, col, nnz * 4, cudaMemcpyHostToDevice)) != cudaSuccess) return fail(e);
        d.col = p;
    }
    if (w) {
        std::vector<WArc> arcs(nnz);
        std::vector<double> prob;
        std::vector<int64_t> ql, qh;
        std::vector<uint32_t> thr;
        std::vector<int32_t> al;
        for (int64_t u = 0; u < N; ++u) {
            const int64_t b0 = rp[u], deg = rp[u + 1] - rp[u];
            thr.resize(deg); al.resize(deg);
            vose_row(w + b0, deg, thr.data(), al.data(), prob, ql, qh);
            for (int64_t j = 0; j < deg; ++j) arcs[b0 + j] = WArc{col[b0 + j], thr[j], col[b0 + al[j]], al[j]};
        }
        WArc *p;
        if ((e = balloc(b, (void **)&p, nnz * sizeof(WArc))) != cudaSuccess) return fail(e);
        if ((e = cudaMemcpy(p, arcs.data(), nnz * sizeof(WArc), cudaMemcpyHostToDevice)) != cudaSuccess) return fail(e);
        d.warc = p;
    }
    if ((e = balloc(b, (void **)&b->graphs, G * sizeof(BGraph))) != cudaSuccess) return fail(e);
    if ((e = cudaMemcpy(b->graphs, hg.data(), G * sizeof(BGraph), cudaMemcpyHostToDevice)) != cudaSuccess) return fail(e);
    if ((e = balloc(b, &b->scratch, 128)) != cudaSuccess) return fail(e);
    if ((e = cudaMallocHost((void **)&b->host, 64)) != cudaSuccess) return fail(e);
    if ((e = cudaStreamCreateWithFlags(&b->side, cudaStreamNonBlocking)) != cudaSuccess ||
        (e = cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming)) != cudaSuccess ||
        (e = cudaEventCreateWithFlags(&b->join, cudaEventDisableTiming)) != cudaSuccess) {
        if (b->fork) cudaEventDestroy(b->fork);
        if (b->side) cudaStreamDestroy(b->side);
        return fail(e);
    }
    *out = b;
    return RWC_OK;
}

extern "C" rwc_status rwc_batch_roots(const rwc_batch_t *b, int32_t *host_roots) {
    if (!b || !host_roots) return set_error(RWC_ERR_INVALID, "bad argument");
    memcpy(host_roots, b->roots.data(), b->roots.size() * sizeof(int32_t));
    return RWC_OK;
}

extern "C" rwc_status rwc_batch_sample(rwc_batch_t *b, uint64_t seed, int64_t T, double *sums,
                                       int32_t use_graph, int32_t per_graph_launch,
                                       rwc_stats_t *stats, rwc_stream_t stream) {
    clear_error();
    if (!b || !sums || T <= 0 || T > ((int64_t)1 << 31)) return set_error(RWC_ERR_INVALID, "bad argument");
    if (stats) memset(stats, 0, sizeof(*stats));
    cudaStream_t st = (cudaStream_t)stream;
    RWC_CUDA_TRY(cudaMemsetAsync(b->scratch, 0, 32, st));
    if (per_graph_launch) {
        // baseline: one launch per graph, same per-tree kernel
        int *err = (int *)b->scratch;
        unsigned long long *rounds = (unsigned long long *)((char *)b->scratch + 8);
        const uint32_t k0 = (uint32_t)seed, k1 = (uint32_t)(seed >> 32);
        for (int32_t g = 0; g < b->G; ++g) {
            const BGraph &bg = b->hgraphs[g];
            DevGraph dg = b->base;
            dg.n = bg.n; dg.root = bg.root;
            if (b->off64) dg.rp64 = b->base.rp64 + bg.voff; else dg.rp32 = b->base.rp32 + bg.voff;
            const int thr = bg.n <= 2048 ? 256 : 512;   // the block sizes of a plain per-graph launch
            const size_t smem = smem_tree_bytes(bg.n);
            rwc_status status = RWC_OK;
            dispatch(b->off64, b->weighted, [&](auto o64, auto wt) {
                auto kern = s_trees<decltype(o64)::value, decltype(wt)::value>;
                cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
                int per_sm = 0;
                cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, thr, smem);
                if (per_sm < 1) { status = set_error(RWC_ERR_UNSUPPORTED, "graph %d does not fit", g); return; }
                const int64_t blocks = std::min<int64_t>(T, (int64_t)num_sms() * per_sm);
                ::rwc::count_launches(1); kern<<<(unsigned)blocks, thr, smem, st>>>(dg, 0u, T, k0, k1, (uint32_t)g, (int64_t)1 << 22,
                                                           sums + bg.voff, nullptr, nullptr, err, rounds);
            });
            RWC_TRY(status);
        }
        RWC_CUDA_TRY(cudaGetLastError());
        return finish(b, stats, 3, T, st);
    }
    RWC_TRY(build_items(b, T));
    if (!use_graph) {
        RWC_TRY(enqueue(b, seed, T, sums, st));
        return finish(b, stats, 4, T, st);
    }
    if (!b->exec || b->cap_seed != seed || b->cap_T != T || b->cap_sums != sums || b->cap_stream != st) {
        drop_graph(b);
        cudaStream_t cs;
        RWC_CUDA_TRY(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
        rwc_status s = RWC_OK;
        cudaError_t e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
        if (e == cudaSuccess) {
            s = enqueue(b, seed, T, sums, cs);
            cudaGraph_t gr = nullptr;
            e = cudaStreamEndCapture(cs, &gr);
            if (s == RWC_OK && e == cudaSuccess) {
                b->graph = gr;
                e = cudaGraphInstantiate(&b->exec, gr, 0);
            } else if (gr) {
                cudaGraphDestroy(gr);
            }
        }
        cudaStreamDestroy(cs);
        RWC_TRY(s);
        if (e != cudaSuccess) { drop_graph(b); return set_error(RWC_ERR_CUDA, "CUDA graph capture: %s", cudaGetErrorString(e)); }
        b->cap_seed = seed; b->cap_T = T; b->cap_sums = sums; b->cap_stream = st;
    }
    RWC_CUDA_TRY(cudaGraphLaunch(b->exec, st));
    return finish(b, stats, 5, T, st);
}

namespace {
// Checks a schedule against the batch's graphs; the item lists must be built.
bool schedule_fits(const rwc_batch *b) { return batch_smem(b) <= 227 * 1024; }
}  // namespace

extern "C" rwc_status rwc_batch_get_schedule(const rwc_batch_t *b, int32_t *host_sched) {
    clear_error();
    if (!b || !host_sched) return set_error(RWC_ERR_INVALID, "bad argument");
    host_sched[0] = b->threads;
    host_sched[1] = b->split;
    host_sched[2] = b->tile;
    host_sched[3] = b->warp;
    host_sched[4] = b->conc;
    return RWC_OK;
}

extern "C" rwc_status rwc_batch_set_schedule(rwc_batch_t *b, int32_t threads, int32_t split, int32_t tile,
                                             int32_t warp, int32_t concurrent) {
    clear_error();
    if (!b || threads < 32 || threads > 1024 || threads % 32 || split < 0 || split > 20000 || tile < 1 ||
        (warp != 0 && warp != 1) || (concurrent != 0 && concurrent != 1))
        return set_error(RWC_ERR_INVALID, "schedule needs threads in [32, 1024] (a multiple of 32), "
                                          "0 <= split <= 20000, tile >= 1, warp and concurrent 0 or 1");
    int wmax = 0, bmax = 0;
    for (const BGraph &g : b->hgraphs) {
        if (g.n <= split) wmax = std::max(wmax, g.n);
        else bmax = std::max(bmax, g.n);
    }
    const size_t small = wmax ? (warp ? (size_t)(SMALL_THREADS / 32) * warp_slice_bytes(wmax) : smem_tree_bytes(wmax)) : 0;
    const size_t need = std::max(bmax ? smem_tree_bytes(bmax) : 0, small);
    if (need > 227 * 1024)
        return set_error(RWC_ERR_UNSUPPORTED, "schedule needs %zu bytes of shared memory per block", need);
    b->threads = threads;
    b->split = split;
    b->tile = tile;
    b->warp = warp;
    b->conc = concurrent;
    b->items_T = -1;
    drop_graph(b);
    return RWC_OK;
}

extern "C" rwc_status rwc_autotune(rwc_batch_t *b, const char *cache_path, rwc_stream_t stream) {
    clear_error();
    if (!b) return set_error(RWC_ERR_INVALID, "bad argument");
    cudaStream_t st = (cudaStream_t)stream;
    char sig[128];
    snprintf(sig, sizeof(sig), "G%d_N%lld_E%lld", b->G, (long long)b->N, (long long)b->nnz);
    if (cache_path) {
        FILE *f = fopen(cache_path, "r");
        if (f) {
            char buf[4096];
            size_t len = fread(buf, 1, sizeof(buf) - 1, f);
            fclose(f);
            buf[len] = 0;
            const char *p = strstr(buf, sig);
            const char *colon = p ? strchr(p, ':') : nullptr;
            int th, sp, tl, wp, cc;
            if (colon && sscanf(colon + 1, " [%d, %d, %d, %d, %d]", &th, &sp, &tl, &wp, &cc) == 5 &&
                rwc_batch_set_schedule(b, th, sp, tl, wp, cc) == RWC_OK)
                return RWC_OK;
            clear_error();
        }
    }
    double *sums = nullptr;
    RWC_CUDA_TRY(cudaMallocAsync((void **)&sums, b->N * sizeof(double), st));
    // coordinate search from the current schedule, each candidate timed on
    // 16 trees per graph: the split with the small class warp- or
    // block-per-tree, then the large class's block size, then trees per item,
    // then concurrent or sequential classes
    const int64_t Tp = 16;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    struct Sched { int th, sp, tl, wp, cc; };
    Sched best_s{b->threads, b->split, b->tile, b->warp, b->conc};
    float best = 1e30f;
    rwc_status status = RWC_OK;
    auto time_one = [&](const Sched &c) -> float {
        b->threads = c.th; b->split = c.sp; b->tile = c.tl; b->warp = c.wp; b->conc = c.cc;
        b->items_T = -1;
        if ((status = build_items(b, Tp)) != RWC_OK) return -1.f;
        if (!schedule_fits(b)) return 1e30f;
        cudaMemsetAsync(b->scratch, 0, 32, st);
        if (enqueue(b, 12345, Tp, sums, st) != RWC_OK) { clear_error(); return 1e30f; }
        cudaEventRecord(e0, st);
        cudaMemsetAsync(b->scratch, 0, 32, st);
        if (enqueue(b, 12346, Tp, sums, st) != RWC_OK) { clear_error(); return 1e30f; }
        cudaEventRecord(e1, st);
        cudaEventSynchronize(e1);
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        return ms;
    };
    auto consider = [&](Sched c) -> bool {
        const float ms = time_one(c);
        if (ms < 0.f) return false;
        if (ms < best) { best = ms; best_s = c; }
        return true;
    };
    {
        const int splits[][2] = {{0, 0}, {512, 1}, {1024, 1}, {2048, 1}, {1024, 0}, {2048, 0}, {4096, 0}};
        for (auto &sw : splits) { Sched c = best_s; c.sp = sw[0]; c.wp = sw[1]; if (!consider(c)) goto done; }
        const Sched base1 = best_s;
        for (int th : {256, 512, 1024}) { Sched c = base1; c.th = th; if (!consider(c)) goto done; }
        const Sched base2 = best_s;
        for (int tl : {1, 4, 16}) { Sched c = base2; c.tl = tl; if (!consider(c)) goto done; }
        const Sched base3 = best_s;
        for (int cc : {0, 1}) { Sched c = base3; c.cc = cc; if (!consider(c)) goto done; }
    }
done:
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFreeAsync(sums, st);
    RWC_CUDA_TRY(cudaStreamSynchronize(st));
    RWC_TRY(status);
    b->threads = best_s.th; b->split = best_s.sp; b->tile = best_s.tl; b->warp = best_s.wp; b->conc = best_s.cc;
    b->items_T = -1;
    drop_graph(b);
    if (cache_path) {
        FILE *f = fopen(cache_path, "w");
        if (f) {
            fprintf(f, "{\"%s\": [%d, %d, %d, %d, %d]}\n", sig, best_s.th, best_s.sp, best_s.tl, best_s.wp, best_s.cc);
            fclose(f);
        }
    }
    return RWC_OK;
}

extern "C" rwc_status rwc_batch_destroy(rwc_batch_t *b) {
    if (!b) return RWC_OK;
    drop_graph(b);
    if (b->side) cudaStreamSynchronize(b->side);
    for (void *p : b->allocs) cudaFree(p);
    if (b->host) cudaFreeHost(b->host);
    if (b->join) cudaEventDestroy(b->join);
    if (b->fork) cudaEventDestroy(b->fork);
    if (b->side) cudaStreamDestroy(b->side);
    delete b;
    return RWC_OK;
}

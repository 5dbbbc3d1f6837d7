// Internal declarations shared by the library's translation units.
#pragma once

#include <atomic>
#include <cuda_runtime.h>
#include <stdint.h>
#include <string>
#include <vector>

#include "rwc.h"

namespace rwc {

// ------------------------------------------------------------ error model
rwc_status set_error(rwc_status st, const char *fmt, ...);
void clear_error();

#define RWC_CUDA_TRY(expr)                                                    \
    do {                                                                      \
        cudaError_t e_ = (expr);                                              \
        if (e_ != cudaSuccess) {                                              \
            return ::rwc::set_error(e_ == cudaErrorMemoryAllocation ? RWC_ERR_OOM \
                                                                    : RWC_ERR_CUDA, \
                                    "%s failed: %s (%s:%d)", #expr,           \
                                    cudaGetErrorString(e_), __FILE__, __LINE__); \
        }                                                                     \
    } while (0)

#define RWC_TRY(expr)                                                         \
    do {                                                                      \
        rwc_status s_ = (expr);                                               \
        if (s_ != RWC_OK) return s_;                                          \
    } while (0)

// ----------------------------------------------------------- device graph
// Arc record of a weighted graph: the arc's head, its alias threshold and
// the head of its alias arc, so that one 16-byte load resolves a weighted
// neighbour pick.
struct __align__(16) WArc {
    int32_t col;
    uint32_t thr;
    int32_t alias_col;
    int32_t alias_idx;
};

struct DevGraph {
    int64_t n = 0, nnz = 0;
    int32_t root = 0;
    bool weighted = false;
    bool off64 = false;
    const int32_t *rp32 = nullptr;   // [n+1] when !off64
    const int64_t *rp64 = nullptr;   // [n+1] when off64
    const int32_t *col = nullptr;    // [nnz] arc heads
    const WArc *warc = nullptr;      // [nnz] when weighted
    const float *w = nullptr;        // [nnz] when weighted (solver)
    const double *d = nullptr;       // [n] weighted degrees
    const float *dinv32 = nullptr;   // [n] 1/d (Jacobi preconditioner)
    double vol = 0.0, dmax = 0.0;
    // rows with more than HEAVY_DEG arcs, cut into chunks of HEAVY_CHUNK arcs
    // so that a sparse product can give every chunk its own warp
    int64_t hc_n = 0;                // chunks
    const int32_t *hc_row = nullptr; // [hc_n] row of each chunk (a row's chunks are consecutive)
    const int64_t *hc_beg = nullptr; // [hc_n] first arc of each chunk
    const int32_t *hfirst = nullptr; // [n] first chunk of a heavy row, -1 for other rows
    // the other rows grouped by degree for the sparse products: bin b (b = 0..4)
    // holds the rows of at most 2^(b+1) arcs (more than 16 for b = 4), each
    // read by 2^(b+1) lanes; rows bin_rows[bin_off[b] .. bin_off[b+1])
    const int32_t *bin_rows = nullptr;
    int64_t bin_off[6] = {0, 0, 0, 0, 0, 0};
    // unweighted graphs with int32 offsets whose degrees are all at most 8:
    // every row's heads inline, ell_w (4 or 8) slots per vertex in arc order,
    // -1 after the last (0 = none)
    const int4 *ell = nullptr;
    int ell_w = 0;
};

constexpr int64_t HEAVY_DEG = 1024;
constexpr int64_t HEAVY_CHUNK = 1024;

}  // namespace rwc

struct rwc_graph {
    rwc::DevGraph g;
    int64_t device_bytes = 0;
    void *allocs[16] = {};
    int nallocs = 0;
    // pinned host scalars used by synchronising entry points
    int64_t *host_scalars = nullptr;
    // start order of the walker sampler (device, n-1 entries), made on first use
    int32_t *walk_order = nullptr;
    // device status word of asynchronous sampling calls (STATUS_* bits)
    int *dev_status = nullptr;
};

namespace rwc {

cudaError_t graph_alloc(rwc_graph *G, void **p, size_t bytes);

// Walker sampler (walker.cu) and its parked-path variant (park.cu, policy 4).
rwc_status sample_walker(rwc_graph *G, uint64_t seed, int64_t tree0, int64_t T, double *sums,
                         int32_t *parents, int32_t *visits, const rwc_options_t &o,
                         rwc_stats_t *st, cudaStream_t stream);
rwc_status sample_park(rwc_graph *G, uint64_t seed, int64_t tree0, int64_t T, double *sums,
                       int32_t *parents, int32_t *visits, const rwc_options_t &o,
                       rwc_stats_t *st, cudaStream_t stream);
// The walkers' start order (a fixed permutation of the non-root vertices, on
// the device, made on first use and kept with the graph).
rwc_status walker_order(rwc_graph *G, const int32_t **out);

// Host-side CSR checks (graph.cu): see rwc_graph_create for the rules.
rwc_status validate_csr(int64_t n, int64_t nnz, const int64_t *rp, const int32_t *col,
                        const float *w);
bool csr_connected(int64_t n, const int64_t *rp, const int32_t *col);
// Vose alias table of one row (graph.cu), scratch vectors supplied by caller.
void vose_row(const float *w, int64_t deg, uint32_t *thr, int32_t *alias,
              std::vector<double> &prob, std::vector<int64_t> &lo_q, std::vector<int64_t> &hi_q);

// X = L^+ B for node-major [n][k] FP64 arrays (solver.cu).
rwc_status solve_nodemajor(rwc_graph *G, int k, const double *B, double *X, double tol,
                           int *iters_out, cudaStream_t st);

// --------------------------------------------------------------- Philox
// Philox-4x32 with 10 rounds (Salmon, Moraes, Dror, Shaw, SC'11): each round
// multiplies words 0 and 2 by the two Philox constants, and mixes the high
// halves into words 1 and 3 with the round key; the key advances by the two
// Weyl constants between rounds.
struct Ctr4 { uint32_t x, y, z, w; };

__host__ __device__ __forceinline__ uint32_t mulhi32(uint32_t a, uint32_t b) {
#ifdef __CUDA_ARCH__
    return __umulhi(a, b);
#else
    return (uint32_t)(((uint64_t)a * (uint64_t)b) >> 32);
#endif
}

__host__ __device__ __forceinline__ Ctr4 philox4x32_10(Ctr4 c, uint32_t k0, uint32_t k1) {
    const uint32_t A = 0xD2511F53u, B = 0xCD9E8D57u;
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const uint32_t hA = mulhi32(A, c.x), lA = A * c.x;
        const uint32_t hB = mulhi32(B, c.z), lB = B * c.z;
        c = Ctr4{hB ^ c.y ^ k0, lB, hA ^ c.w ^ k1, lA};
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    return c;
}

// Row bounds of vertex u.
template <bool OFF64>
__device__ __forceinline__ void row_bounds(const DevGraph &g, int32_t u, int64_t &b, uint32_t &deg) {
    if (OFF64) {
        const int64_t b0 = __ldg(g.rp64 + u), b1 = __ldg(g.rp64 + u + 1);
        b = b0; deg = (uint32_t)(b1 - b0);
    } else {
        const int32_t b0 = __ldg(g.rp32 + u), b1 = __ldg(g.rp32 + u + 1);
        b = b0; deg = (uint32_t)(b1 - b0);
    }
}

// The c-th successor-stack entry of vertex u in tree `tree` of graph `gid`:
// the neighbour returned by the c-th call of RandomNeighbor(u) (Algorithm 3).
template <bool OFF64, bool WEIGHTED>
__device__ __forceinline__ int32_t succ(const DevGraph &g, int32_t u, uint32_t c, uint32_t tree,
                                        uint32_t gid, uint32_t k0, uint32_t k1) {
    int64_t b; uint32_t deg;
    row_bounds<OFF64>(g, u, b, deg);
    const Ctr4 o = philox4x32_10(Ctr4{c, (uint32_t)u, tree, gid}, k0, k1);
    const uint32_t j = __umulhi(o.x, deg);
    if (WEIGHTED) {
        const WArc a = g.warc[b + j];
        return (o.y < a.thr) ? a.col : a.alias_col;
    } else {
        return __ldg(g.col + b + j);
    }
}

// ------------------------------------------ asynchronous status word
// Bits of rwc_graph::dev_status, set by asynchronous sampling calls and read
// and cleared by rwc_sync_status.
constexpr int STATUS_KOVF = 1;       // a pop count overflowed
constexpr int STATUS_WAIT = 2;       // a walker wait ran out
constexpr int STATUS_INTERNAL = 4;   // an internal consistency check failed
constexpr int STATUS_ROUNDS = 8;     // max_rounds reached (shared mode)

// dst |= the status bits of a sampler's error word: walker words use the
// STATUS_* values already; shared-mode words (rounds 1, overflow 2, check 4)
// are mapped.  One thread.  (static: every translation unit has its own copy.)
static __global__ void fold_status(const int *err, int shared_codes, int *dst) {
    const int e = *err;
    if (!e) return;
    int b = e;
    if (shared_codes)
        b = ((e & 1) ? STATUS_ROUNDS : 0) | ((e & 2) ? STATUS_KOVF : 0) | ((e & 4) ? STATUS_INTERNAL : 0);
    atomicOr(dst, b);
}

// ------------------------------------------------------------- helpers
// Library-wide kernel launch counter (graph.cu).
void count_launches(int64_t k);

// ------------------------------------------------ fixed-order reductions
// A sum whose order does not depend on scheduling: each thread adds its
// grid-stride elements in index order, a warp combines its lanes with a fixed
// shuffle tree, and thread 0 adds the block's warps in warp order.  Blocks
// store their sums in parts[blockIdx.x] and sum_parts (one block) adds the
// parts in block order, so a launch of the same size on the same input gives
// the same bits every time.
__device__ __forceinline__ double block_sum_fixed(double v) {
    __shared__ double ws[32];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    __syncthreads();   // an earlier call's reader is done with ws
    if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = v;
    __syncthreads();
    double s = 0.0;
    if (threadIdx.x == 0)
        for (int w = 0; w < (int)((blockDim.x + 31) >> 5); ++w) s += ws[w];
    return s;   // meaningful in thread 0
}

// out[j] = sum over b < nparts of parts[j * stride + b], in order of b, for
// j < nvals.  One block: thread t adds parts t, t + blockDim, ... in order,
// then block_sum_fixed.  (static: every translation unit has its own copy.)
static __global__ void sum_parts(const double *parts, int nparts, int stride, int nvals, double *out) {
    for (int j = 0; j < nvals; ++j) {
        double s = 0.0;
        for (int b = threadIdx.x; b < nparts; b += blockDim.x) s += parts[(int64_t)j * stride + b];
        s = block_sum_fixed(s);
        if (threadIdx.x == 0) out[j] = s;
    }
}

// SM count of the current device, cached per device index.
inline int num_sms() {
    static std::atomic<int> cache[64];
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0) dev = 0;
    int sms = dev < 64 ? cache[dev].load(std::memory_order_relaxed) : 0;
    if (sms <= 0) {
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (sms <= 0) sms = 1;
        if (dev < 64) cache[dev].store(sms, std::memory_order_relaxed);
    }
    return sms;
}

}  // namespace rwc

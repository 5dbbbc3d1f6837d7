// The straightforward estimator of Section 5, the one Wilson's algorithm
// improves on: t_u = (NL_v^-1)_uu is the expected number of visits to u of a
// random walk from u stopped when it meets the trap v (time 0 included).  For
// every u != v and r < R one such walk, one thread per walk (grid-stride over
// the (n - 1) R walks, the R walks of one start adjacent so that a warp starts
// together); sums[u] += visits to u (FP64 atomics of integers: exact).  Step s
// of walk (u, r) moves by the tree sampler's RandomNeighbor rule with Philox
// counter (s, u, r, 0xFFFFFFFE).  Every step is one dependent row-bounds and
// arc gather, so the kernel is latency bound like the tree sampler.
#include <algorithm>

#include "rwc_common.cuh"

namespace rwc {
namespace {

template <bool OFF64, bool WT>
__global__ void tw_walks(DevGraph g, uint32_t k0, uint32_t k1, int64_t R, int64_t max_steps,
                         double *sums, unsigned long long *steps_total, int *err) {
    const int64_t nw = (g.n - 1) * R;
    const int32_t root = g.root;
    unsigned long long local = 0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < nw;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t up = i / R;
        const uint32_t r = (uint32_t)(i - up * R);
        const int32_t u = (int32_t)(up < root ? up : up + 1);
        int32_t x = u;
        uint32_t c = 0;
        int64_t s = 0;
        while (x != root) {
            if (x == u) ++c;
            if (s >= max_steps) { atomicOr(err, 1); break; }
            int64_t b; uint32_t deg;
            row_bounds<OFF64>(g, x, b, deg);
            const Ctr4 o = philox4x32_10(Ctr4{(uint32_t)s, (uint32_t)u, r, 0xFFFFFFFEu}, k0, k1);
            const uint32_t j = __umulhi(o.x, deg);
            if (WT) {
                const WArc a = g.warc[b + j];
                x = (o.y < a.thr) ? a.col : a.alias_col;
            } else {
                x = __ldg(g.col + b + j);
            }
            ++s;
        }
        if (c) atomicAdd(sums + u, (double)c);
        local += (unsigned long long)s;
    }
    for (int o = 16; o > 0; o >>= 1) local += __shfl_xor_sync(0xffffffffu, local, o);
    if ((threadIdx.x & 31) == 0 && local) atomicAdd(steps_total, local);
}

}  // namespace
}  // namespace rwc

extern "C" rwc_status rwc_trap_walks(rwc_graph_t *G, uint64_t seed, int64_t walks_per_node,
                                     int64_t max_steps, double *sums, int64_t *host_steps,
                                     rwc_stream_t stream_) {
    using namespace rwc;
    clear_error();
    if (!G || !sums) return set_error(RWC_ERR_INVALID, "rwc_trap_walks: graph and sums required");
    if (walks_per_node < 0 || walks_per_node > ((int64_t)1 << 32))
        return set_error(RWC_ERR_INVALID, "walks_per_node must lie in [0, 2^32]");
    if (max_steps <= 0 || max_steps > ((int64_t)1 << 32))
        return set_error(RWC_ERR_INVALID, "max_steps must lie in [1, 2^32]");
    if (host_steps) *host_steps = 0;
    if (walks_per_node == 0) return RWC_OK;
    const DevGraph &g = G->g;
    cudaStream_t st = (cudaStream_t)stream_;
    void *scratch = nullptr;
    RWC_CUDA_TRY(cudaMallocAsync(&scratch, 64, st));
    struct Free {
        void *p; cudaStream_t s;
        ~Free() { cudaFreeAsync(p, s); }
    } fr{scratch, st};
    RWC_CUDA_TRY(cudaMemsetAsync(scratch, 0, 64, st));
    unsigned long long *steps = (unsigned long long *)scratch;
    int *err = (int *)((char *)scratch + 8);
    const int64_t nw = (g.n - 1) * walks_per_node;
    const unsigned blocks = (unsigned)std::max<int64_t>(1, std::min<int64_t>((int64_t)num_sms() * 16, (nw + 255) / 256));
    const uint32_t k0 = (uint32_t)seed, k1 = (uint32_t)(seed >> 32);
    count_launches(1);
    if (g.off64) {
        if (g.weighted) tw_walks<true, true><<<blocks, 256, 0, st>>>(g, k0, k1, walks_per_node, max_steps, sums, steps, err);
        else tw_walks<true, false><<<blocks, 256, 0, st>>>(g, k0, k1, walks_per_node, max_steps, sums, steps, err);
    } else {
        if (g.weighted) tw_walks<false, true><<<blocks, 256, 0, st>>>(g, k0, k1, walks_per_node, max_steps, sums, steps, err);
        else tw_walks<false, false><<<blocks, 256, 0, st>>>(g, k0, k1, walks_per_node, max_steps, sums, steps, err);
    }
    RWC_CUDA_TRY(cudaGetLastError());
    int64_t *h = G->host_scalars;
    RWC_CUDA_TRY(cudaMemcpyAsync(h, scratch, 16, cudaMemcpyDeviceToHost, st));
    RWC_CUDA_TRY(cudaStreamSynchronize(st));
    if (host_steps) *host_steps = h[0];
    if ((int)(h[1] & 0xffffffff)) return set_error(RWC_ERR_NOT_CONVERGED, "a trap walk exceeded max_steps = %lld", (long long)max_steps);
    return RWC_OK;
}

// Evaluation measures of Section 6: the mean relative error of an estimate
// and the Kendall distance of two rankings, on the device.
//
// MRE = (1/n) sum_u |H_u - H~_u| / H_u: block partial sums in a fixed order,
// then one block adds the partials in a fixed order (deterministic).
//
// K(L1, L2) = 2 (alpha - beta) / (n (n - 1)) with alpha / beta the concordant
// / discordant pairs (tied pairs count neither way): every pair i < j is
// compared once.  Each double becomes an order-preserving 64-bit key (-0.0
// merged into +0.0 so that the two compare equal, as they do as doubles), a
// block keeps 4 rows per thread in registers and streams a tile of 2048 keys
// through shared memory; per-thread counts are exact int32, block totals are
// added with 64-bit integer atomics (exact, order independent).  O(n^2)
// comparisons, ALU bound.
#include <algorithm>
#include <cmath>
#include <cstring>

#include "rwc_common.cuh"

namespace rwc {
namespace {

constexpr int MRE_THREADS = 256;
constexpr int MRE_BLOCKS = 1024;

__global__ void mre_partial(int64_t n, const double *H, const double *He, double *part) {
    __shared__ double sh[MRE_THREADS];
    double acc = 0.0;
    for (int64_t u = blockIdx.x * (int64_t)MRE_THREADS + threadIdx.x; u < n;
         u += (int64_t)gridDim.x * MRE_THREADS)
        acc += fabs(H[u] - He[u]) / H[u];
    sh[threadIdx.x] = acc;
    __syncthreads();
    for (int s = MRE_THREADS / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) sh[threadIdx.x] += sh[threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x == 0) part[blockIdx.x] = sh[0];
}

__global__ void mre_final(int nb, int64_t n, const double *part, double *out) {
    __shared__ double sh[MRE_THREADS];
    double acc = 0.0;
    for (int i = threadIdx.x; i < nb; i += MRE_THREADS) acc += part[i];
    sh[threadIdx.x] = acc;
    __syncthreads();
    for (int s = MRE_THREADS / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) sh[threadIdx.x] += sh[threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x == 0) *out = sh[0] / (double)n;
}

// Predicted MRE (variance law of the visit counts): block partial sums of
// sqrt(t (t - 1) / T) / (pi_u |H_u|) over u != v, t = sums_u / T.
__global__ void pmre_partial(int64_t n, const double *d, double vol, int32_t v, const double *sums,
                             double invT, const double *H, double *part) {
    __shared__ double sh[MRE_THREADS];
    double acc = 0.0;
    for (int64_t u = blockIdx.x * (int64_t)MRE_THREADS + threadIdx.x; u < n;
         u += (int64_t)gridDim.x * MRE_THREADS) {
        if (u == v) continue;
        const double t = sums[u] * invT;
        const double se = sqrt(fmax(t * (t - 1.0), 0.0) * invT) / (d[u] / vol);
        acc += se / fabs(H[u]);
    }
    sh[threadIdx.x] = acc;
    __syncthreads();
    for (int s = MRE_THREADS / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) sh[threadIdx.x] += sh[threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x == 0) part[blockIdx.x] = sh[0];
}

constexpr int KT_THREADS = 256;
constexpr int KT_ROWS = 4;                          // rows per thread
constexpr int KT_BI = KT_THREADS * KT_ROWS;         // rows per block
constexpr int KT_BJ = 2048;                         // columns per shared tile

// Order-preserving key of a double: a > b  <=>  key(a) > key(b) (no NaN).
__device__ __forceinline__ uint64_t okey(double x) {
    uint64_t b = (uint64_t)__double_as_longlong(x);
    if (b == 0x8000000000000000ull) b = 0;          // -0.0 == +0.0
    return (b >> 63) ? ~b : (b | 0x8000000000000000ull);
}

__device__ __forceinline__ int sgn_cmp(uint64_t p, uint64_t q) { return (int)(p > q) - (int)(p < q); }

__global__ void __launch_bounds__(KT_THREADS) kendall_tiles(int64_t n, const double *a, const double *b,
                                                           unsigned long long *out) {
    __shared__ uint64_t ka[KT_BJ], kb[KT_BJ];
    __shared__ long long red[KT_THREADS / 32];
    const int64_t i0 = (int64_t)blockIdx.x * KT_BI;
    const int64_t j0 = (int64_t)blockIdx.y * KT_BJ;
    // pairs i < j only: a tile wholly at or below the diagonal has none
    if (j0 + KT_BJ - 1 <= i0) return;
    const int64_t jn = min((int64_t)KT_BJ, n - j0);
    for (int t = threadIdx.x; t < jn; t += KT_THREADS) {
        ka[t] = okey(a[j0 + t]);
        kb[t] = okey(b[j0 + t]);
    }
    uint64_t ra[KT_ROWS], rb[KT_ROWS];
    int64_t ri[KT_ROWS];
#pragma unroll
    for (int r = 0; r < KT_ROWS; ++r) {
        ri[r] = i0 + threadIdx.x + (int64_t)r * KT_THREADS;
        ra[r] = ri[r] < n ? okey(a[ri[r]]) : 0;
        rb[r] = ri[r] < n ? okey(b[ri[r]]) : 0;
    }
    __syncthreads();
    int cnt = 0;
    const bool above = j0 > i0 + KT_BI - 1;     // every j of the tile exceeds every i
    if (above) {
        // rows past n contribute nothing only if masked: keep them out
        bool live[KT_ROWS];
#pragma unroll
        for (int r = 0; r < KT_ROWS; ++r) live[r] = ri[r] < n;
        for (int t = 0; t < jn; ++t) {
            const uint64_t xa = ka[t], xb = kb[t];
#pragma unroll
            for (int r = 0; r < KT_ROWS; ++r)
                if (live[r]) cnt += sgn_cmp(ra[r], xa) * sgn_cmp(rb[r], xb);
        }
    } else {
        for (int t = 0; t < jn; ++t) {
            const uint64_t xa = ka[t], xb = kb[t];
            const int64_t j = j0 + t;
#pragma unroll
            for (int r = 0; r < KT_ROWS; ++r)
                if (ri[r] < j) cnt += sgn_cmp(ra[r], xa) * sgn_cmp(rb[r], xb);
        }
    }
    long long v = cnt;
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
        long long s = 0;
        for (int w = 0; w < KT_THREADS / 32; ++w) s += red[w];
        if (s) atomicAdd(out, (unsigned long long)s);
    }
}

}  // namespace
}  // namespace rwc

extern "C" rwc_status rwc_mre(int64_t n, const double *H, const double *H_est, double *out,
                              rwc_stream_t stream_) {
    using namespace rwc;
    clear_error();
    if (n < 1 || !H || !H_est || !out) return set_error(RWC_ERR_INVALID, "rwc_mre: n >= 1 and non-NULL pointers required");
    cudaStream_t stream = (cudaStream_t)stream_;
    const int nb = (int)std::min<int64_t>(MRE_BLOCKS, (n + MRE_THREADS - 1) / MRE_THREADS);
    double *part = nullptr;
    RWC_CUDA_TRY(cudaMallocAsync(&part, sizeof(double) * nb, stream));
    count_launches(2);
    mre_partial<<<nb, MRE_THREADS, 0, stream>>>(n, H, H_est, part);
    mre_final<<<1, MRE_THREADS, 0, stream>>>(nb, n, part, out);
    const cudaError_t e = cudaGetLastError();
    cudaFreeAsync(part, stream);
    RWC_CUDA_TRY(e);
    return RWC_OK;
}

extern "C" rwc_status rwc_kendall(int64_t n, const double *a, const double *b, int64_t *out_diff,
                                  double *host_tau, rwc_stream_t stream_) {
    using namespace rwc;
    clear_error();
    if (n < 0 || !out_diff || (n > 0 && (!a || !b)))
        return set_error(RWC_ERR_INVALID, "rwc_kendall: n >= 0 and non-NULL pointers required");
    if (n > ((int64_t)1 << 26))
        return set_error(RWC_ERR_INVALID, "rwc_kendall: n must be at most 2^26");
    cudaStream_t stream = (cudaStream_t)stream_;
    RWC_CUDA_TRY(cudaMemsetAsync(out_diff, 0, sizeof(int64_t), stream));
    if (n >= 2) {
        const dim3 grid((unsigned)((n + KT_BI - 1) / KT_BI), (unsigned)((n + KT_BJ - 1) / KT_BJ));
        count_launches(1);
        kendall_tiles<<<grid, KT_THREADS, 0, stream>>>(n, a, b, (unsigned long long *)out_diff);
        RWC_CUDA_TRY(cudaGetLastError());
    }
    if (host_tau) {
        int64_t s = 0;
        RWC_CUDA_TRY(cudaMemcpyAsync(&s, out_diff, sizeof(s), cudaMemcpyDeviceToHost, stream));
        RWC_CUDA_TRY(cudaStreamSynchronize(stream));
        *host_tau = n >= 2 ? 2.0 * (double)s / ((double)n * (double)(n - 1)) : 0.0;
    }
    return RWC_OK;
}

extern "C" rwc_status rwc_predict_mre(rwc_graph_t *G, const double *sums, int64_t num_trees,
                                      const double *H, double target, double *host_mre,
                                      int64_t *host_trees, rwc_stream_t stream_) {
    using namespace rwc;
    clear_error();
    if (!G || !sums || !H || !host_mre || num_trees <= 0)
        return set_error(RWC_ERR_INVALID, "rwc_predict_mre: graph, sums, H, host_mre and num_trees > 0 required");
    const DevGraph &g = G->g;
    const int64_t n = g.n;
    cudaStream_t stream = (cudaStream_t)stream_;
    const int nb = (int)std::min<int64_t>(MRE_BLOCKS, (n + MRE_THREADS - 1) / MRE_THREADS);
    double *part = nullptr;
    RWC_CUDA_TRY(cudaMallocAsync(&part, sizeof(double) * (nb + 1), stream));
    count_launches(2);
    pmre_partial<<<nb, MRE_THREADS, 0, stream>>>(n, g.d, g.vol, g.root, sums, 1.0 / (double)num_trees, H, part);
    mre_final<<<1, MRE_THREADS, 0, stream>>>(nb, n, part, part + nb);
    cudaError_t e = cudaGetLastError();
    double m = 0.0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&m, part + nb, sizeof(double), cudaMemcpyDeviceToHost, stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(stream);
    cudaFreeAsync(part, stream);
    RWC_CUDA_TRY(e);
    *host_mre = std::sqrt(2.0 / M_PI) * m;
    if (host_trees && target > 0.0)
        *host_trees = (int64_t)std::ceil((double)num_trees * (*host_mre / target) * (*host_mre / target));
    return RWC_OK;
}

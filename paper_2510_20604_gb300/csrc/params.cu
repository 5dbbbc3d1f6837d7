// Automatic parameters of FastWalk (Section 5, "The Sampling Algorithm"):
// the sample size l of the tree-count lemma and the solver accuracy theta of
// the performance theorem, from the spectral radius lambda of P_v and the
// graph diameter Delta.
//
// Delta: BFS double sweep (BFS from the pivot, then from the farthest vertex
// found, ties to the smallest id; Delta = the second eccentricity), one
// cooperative launch per sweep with a grid-wide barrier per level.
//
// lambda: P_v = D^-1 W without the pivot's row and column is similar to
// M = D^-1/2 W D^-1/2 on V \ {v}, whose Perron root lambda is the spectral
// radius.  mu = 1 - lambda is the smallest eigenvalue of the normalised
// grounded Laplacian N = I - M = D^-1/2 L_-v D^-1/2, found by inverse
// iteration x <- N^-1 x / |N^-1 x| (the Perron vector is positive, so the
// start x = D^1/2 1 on V \ {v} has a component along it).  Each step needs
// L_-v w = c: with c~ = c padded by 0 at v, z = L^+ (c~ - (sum c) e_v) gives
// w = z - z_v (then L (z - z_v 1) = c~ - (sum c) e_v, whose rows u != v are
// the grounded system).  mu is estimated by the Rayleigh quotient of N^-1,
// <x, x> / <x, N^-1 x>.
#include <algorithm>
#include <cmath>
#include <cstring>

#include <cooperative_groups.h>

#include "rwc_common.cuh"

namespace cg = cooperative_groups;

namespace rwc {
namespace {

constexpr int PT = 256;

struct Buf {
    void *p = nullptr;
    cudaStream_t st;
    explicit Buf(cudaStream_t s) : st(s) {}
    ~Buf() { if (p) cudaFreeAsync(p, st); }
};

__device__ __forceinline__ int ld_gpu(const int *a) {
    int v;
    asm volatile("ld.relaxed.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(a) : "memory");
    return v;
}

template <bool OFF64>
__device__ __forceinline__ void row_range(const DevGraph &g, int64_t u, int64_t &b, int64_t &e) {
    if (OFF64) { b = g.rp64[u]; e = g.rp64[u + 1]; }
    else { b = g.rp32[u]; e = g.rp32[u + 1]; }
}

// Level-synchronous BFS from src: dist[u] = hops, out[0] = eccentricity of
// src.  flag[L % 3] records whether level L reached a new vertex and is read
// by every thread after the barrier that ends level L.  The flag of level
// L + 1 is cleared at the start of level L: its slot was last read after the
// barrier of level L - 2, and every thread has passed the barrier of level
// L - 1 since (two slots would let a fast thread clear a flag that a slow one
// has yet to read).
template <bool OFF64>
__global__ void __launch_bounds__(PT) bfs_coop(DevGraph g, int32_t src, int32_t *dist, int *flag,
                                                int *out) {
    cg::grid_group grid = cg::this_grid();
    const int64_t tid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int64_t nthr = (int64_t)gridDim.x * blockDim.x;
    for (int64_t u = tid; u < g.n; u += nthr) dist[u] = (u == src) ? 0 : -1;
    if (tid == 0) { flag[0] = 0; flag[1] = 0; flag[2] = 0; }
    grid.sync();
    int L = 0;
    for (; L < g.n; ++L) {
        if (tid == 0) flag[(L + 1) % 3] = 0;
        bool any = false;
        for (int64_t u = tid; u < g.n; u += nthr) {
            if (ld_gpu(dist + u) != L) continue;
            int64_t b, e;
            row_range<OFF64>(g, u, b, e);
            for (int64_t j = b; j < e; ++j) {
                const int32_t c = g.col[j];
                if (ld_gpu(dist + c) < 0 && atomicCAS(dist + c, -1, L + 1) == -1) any = true;
            }
        }
        if (any) atomicOr(flag + (L % 3), 1);
        grid.sync();
        if (ld_gpu(flag + (L % 3)) == 0) break;
    }
    if (tid == 0) out[0] = L;
}

// out[1] = smallest vertex at distance out[0].
__global__ void farthest_min_id(int64_t n, const int32_t *dist, int *out) {
    const int ecc = out[0];
    for (int64_t u = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; u < n;
         u += (int64_t)gridDim.x * blockDim.x)
        if (dist[u] == ecc) atomicMin(out + 1, (int)u);
}

// Sums of the inverse iteration in a fixed order: each kernel stores its
// block sums (block_sum_fixed) as parts[b] and, for a second sum,
// parts[stride + b]; sum_parts adds them in block order.
__device__ __forceinline__ void store_parts(double s0, double s1, int nv, double *parts, int stride) {
    s0 = block_sum_fixed(s0);
    if (threadIdx.x == 0) parts[blockIdx.x] = s0;
    if (nv > 1) {
        s1 = block_sum_fixed(s1);
        if (threadIdx.x == 0) parts[stride + blockIdx.x] = s1;
    }
}

// x_u = sqrt(d_u) for u != v, 0 at v; sums |x|^2 and |d_-v|^2.
__global__ void ii_start(int64_t n, const double *d, int32_t v, double *x, double *parts, int stride) {
    double s0 = 0.0, s1 = 0.0;
    for (int64_t u = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; u < n;
         u += (int64_t)gridDim.x * blockDim.x) {
        const double xv = u == v ? 0.0 : sqrt(d[u]);
        x[u] = xv;
        s0 += xv * xv;
        if (u != v) s1 += d[u] * d[u];
    }
    store_parts(s0, s1, 2, parts, stride);
}

// c~ = D^1/2 x / |x| (0 at v); sum c.
__global__ void ii_rhs(int64_t n, const double *d, int32_t v, const double *x, const double *xn2,
                       double *c, double *parts, int stride) {
    const double inv = 1.0 / sqrt(*xn2);
    double s = 0.0;
    for (int64_t u = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; u < n;
         u += (int64_t)gridDim.x * blockDim.x) {
        const double cv = u == v ? 0.0 : sqrt(d[u]) * x[u] * inv;
        c[u] = cv;
        s += cv;
    }
    store_parts(s, 0.0, 1, parts, stride);
}

__global__ void ii_ground(int32_t v, double *c, const double *sum) { c[v] -= *sum; }

// y = D^1/2 (z - z_v) (0 at v) written over x after the sums <x, y> / |x|
// and |y|^2.
__global__ void ii_step(int64_t n, const double *d, int32_t v, const double *z, const double *xn2,
                        double *x, double *parts, int stride) {
    const double zv = z[v], inv = 1.0 / sqrt(*xn2);
    double s0 = 0.0, s1 = 0.0;
    for (int64_t u = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; u < n;
         u += (int64_t)gridDim.x * blockDim.x) {
        const double yv = u == v ? 0.0 : sqrt(d[u]) * (z[u] - zv);
        s0 += x[u] * inv * yv;
        s1 += yv * yv;
        x[u] = yv;
    }
    store_parts(s0, s1, 2, parts, stride);
}

unsigned grid_n(int64_t n) {
    return (unsigned)std::max<int64_t>(1, std::min<int64_t>((int64_t)num_sms() * 8, (n + PT - 1) / PT));
}

rwc_status bfs_sweep(const DevGraph &g, int32_t src, int32_t *dist, int *flag, int *out, cudaStream_t st) {
    rwc_status status = RWC_OK;
    auto run = [&](auto kern) {
        int per_sm = 0;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, PT, 0);
        if (per_sm < 1) { status = set_error(RWC_ERR_UNSUPPORTED, "BFS block does not fit"); return; }
        const unsigned blocks = (unsigned)std::min<int64_t>((int64_t)num_sms() * per_sm, (g.n + PT - 1) / PT);
        DevGraph gg = g;
        int32_t s = src;
        void *args[] = {&gg, &s, &dist, &flag, &out};
        count_launches(1);
        const cudaError_t e = cudaLaunchCooperativeKernel((const void *)kern, blocks, PT, args, 0, st);
        if (e != cudaSuccess) status = set_error(RWC_ERR_CUDA, "BFS launch failed: %s", cudaGetErrorString(e));
    };
    if (g.off64) run(bfs_coop<true>);
    else run(bfs_coop<false>);
    return status;
}

}  // namespace
}  // namespace rwc

extern "C" rwc_status rwc_auto_params(rwc_graph_t *G, double eps, int32_t max_iters, double tol,
                                      rwc_params_t *out, rwc_stream_t stream_) {
    using namespace rwc;
    clear_error();
    if (!G || !out || !(eps > 0.0)) return set_error(RWC_ERR_INVALID, "rwc_auto_params: graph, out and eps > 0 required");
    if (max_iters <= 0) max_iters = 30;
    if (!(tol > 0.0)) tol = 1e-9;
    memset(out, 0, sizeof(*out));
    const DevGraph &g = G->g;
    const int64_t n = g.n;
    cudaStream_t st = (cudaStream_t)stream_;
    Buf buf(st);
    // dist [n] int32 | x, c, z [n] FP64 | scratch (flags, ints, sums)
    const size_t dist_b = (((size_t)n * 4) + 255) & ~(size_t)255;
    const int pstride = num_sms() * 8;    // grid_n's largest grid
    RWC_CUDA_TRY(cudaMallocAsync(&buf.p, dist_b + 3 * (size_t)n * 8 + 256 + 2 * (size_t)pstride * 8, st));
    int32_t *dist = (int32_t *)buf.p;
    double *x = (double *)((char *)buf.p + dist_b), *c = x + n, *z = c + n;
    char *sc = (char *)(z + n);
    int *flag = (int *)sc;            // [3]
    int *iout = (int *)(sc + 16);     // [0] eccentricity, [1] farthest vertex
    double *acc = (double *)(sc + 64);
    double *parts = (double *)(sc + 256);   // [2][pstride] block parts
    int64_t *h = G->host_scalars;
    const unsigned gs = grid_n(n);

    // ---- Delta by a BFS double sweep from the pivot
    int ends[2] = {g.root, 0}, ecc[2] = {0, 0};
    for (int sweep = 0; sweep < 2; ++sweep) {
        RWC_TRY(bfs_sweep(g, ends[sweep], dist, flag, iout, st));
        const int big = 0x7fffffff;
        RWC_CUDA_TRY(cudaMemcpyAsync(iout + 1, &big, sizeof(int), cudaMemcpyHostToDevice, st));
        count_launches(1);
        farthest_min_id<<<gs, PT, 0, st>>>(n, dist, iout);
        RWC_CUDA_TRY(cudaGetLastError());
        RWC_CUDA_TRY(cudaMemcpyAsync(h, iout, 2 * sizeof(int), cudaMemcpyDeviceToHost, st));
        RWC_CUDA_TRY(cudaStreamSynchronize(st));
        const int *hi = (const int *)h;
        ecc[sweep] = hi[0];
        if (sweep == 0) ends[1] = hi[1];
    }
    out->sweep_end = ends[1];
    out->diameter = ecc[1];

    // ---- lambda by inverse iteration on the normalised grounded Laplacian
    const int32_t v = g.root;
    RWC_CUDA_TRY(cudaMemsetAsync(acc, 0, 4 * sizeof(double), st));
    count_launches(2);
    ii_start<<<gs, PT, 0, st>>>(n, g.d, v, x, parts, pstride);
    sum_parts<<<1, PT, 0, st>>>(parts, (int)gs, pstride, 2, acc);   // acc[0] = |x|^2, acc[1] = |d_-v|^2
    RWC_CUDA_TRY(cudaGetLastError());
    double hv[2];
    RWC_CUDA_TRY(cudaMemcpyAsync(hv, acc, 2 * sizeof(double), cudaMemcpyDeviceToHost, st));
    RWC_CUDA_TRY(cudaStreamSynchronize(st));
    const double dnorm = std::sqrt(hv[1]);
    double *xn2 = acc + 2;           // |x|^2 of the current iterate
    RWC_CUDA_TRY(cudaMemcpyAsync(xn2, acc, sizeof(double), cudaMemcpyDeviceToDevice, st));
    double mu = 0.0, prev = 0.0;
    int it = 0;
    for (; it < max_iters; ++it) {
        RWC_CUDA_TRY(cudaMemsetAsync(acc, 0, 2 * sizeof(double), st));
        count_launches(3);
        ii_rhs<<<gs, PT, 0, st>>>(n, g.d, v, x, xn2, c, parts, pstride);
        sum_parts<<<1, PT, 0, st>>>(parts, (int)gs, pstride, 1, acc);
        ii_ground<<<1, 1, 0, st>>>(v, c, acc);
        RWC_CUDA_TRY(cudaGetLastError());
        RWC_TRY(solve_nodemajor(G, 1, c, z, 1e-11, nullptr, st));
        RWC_CUDA_TRY(cudaMemsetAsync(acc, 0, 2 * sizeof(double), st));
        count_launches(2);
        ii_step<<<gs, PT, 0, st>>>(n, g.d, v, z, xn2, x, parts, pstride);
        sum_parts<<<1, PT, 0, st>>>(parts, (int)gs, pstride, 2, acc);
        RWC_CUDA_TRY(cudaGetLastError());
        RWC_CUDA_TRY(cudaMemcpyAsync(xn2, acc + 1, sizeof(double), cudaMemcpyDeviceToDevice, st));
        RWC_CUDA_TRY(cudaMemcpyAsync(hv, acc, 2 * sizeof(double), cudaMemcpyDeviceToHost, st));
        RWC_CUDA_TRY(cudaStreamSynchronize(st));
        if (!(hv[0] > 0.0)) return set_error(RWC_ERR_NOT_CONVERGED, "inverse iteration lost its direction");
        mu = 1.0 / hv[0];             // <x, x> / <x, N^-1 x> with |x| = 1
        if (it > 0 && std::fabs(mu - prev) <= tol * mu) { ++it; break; }
        prev = mu;
    }
    out->iterations = it;
    out->mu = mu;
    out->lambda = 1.0 - mu;

    // ---- the formulas (host scalars)
    const double m = g.vol / 2.0, nd = (double)n;
    const double log_lambda = std::log1p(-mu);
    out->t = (mu >= 1.0 || !(log_lambda < 0.0)) ? 1.0
             : std::log(m / (nd * std::sqrt(nd - 1.0) * dnorm)) / log_lambda;
    if (out->t < 1.0) out->t = 1.0;
    out->trees = (int64_t)std::ceil(2.0 * out->t * out->t * std::log(2.0 * nd) / (eps * eps));
    const double Dl = (double)std::max(1, ecc[1]);
    const double f = 1.0 + g.dmax * (1.0 + nd) / (2.0 * m);
    out->theta = eps / (2.0 * Dl * g.dmax * f * f * std::sqrt(m * nd * Dl));
    return RWC_OK;
}

// Algorithm 1 (AppRWC) fed by Section 5's estimator, the public Laplacian
// solve, and the gradient of the exact centrality.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "rwc_common.cuh"

namespace rwc {
namespace {

constexpr int TPB = 256;

struct Buf {
    void *p = nullptr;
    cudaStream_t st;
    explicit Buf(cudaStream_t s) : st(s) {}
    ~Buf() { if (p) cudaFreeAsync(p, st); }
};

unsigned grid_for(int64_t work) {
    const int64_t cap = (int64_t)num_sms() * 8;
    return (unsigned)std::max<int64_t>(1, std::min<int64_t>(cap, (work + TPB - 1) / TPB));
}

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// parts[block] = this block's share of sum_i a[i] * b[i] (b may be NULL:
// sum a), in a fixed order; sum_parts adds the blocks in order.
__global__ void dot64(int64_t n, const double *a, const double *b, double *parts) {
    double s = 0.0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        s += b ? a[i] * b[i] : a[i];
    s = block_sum_fixed(s);
    if (threadIdx.x == 0) parts[blockIdx.x] = s;
}

// Algorithm 1, right-hand side: b = sqrt(d_v) e_v - (sqrt(d_v) / vol) d.
__global__ void rhs_pivot(int64_t n, const double *d, int32_t v, double vol, double *b) {
    const double sv = sqrt(d[v]);
    for (int64_t u = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; u < n;
         u += (int64_t)gridDim.x * blockDim.x)
        b[u] = -(sv / vol) * d[u] + (u == v ? sv : 0.0);
}

// Algorithm 1, pivot column: y_u = sqrt(d_u) z_u - sqrt(d_u) (sum_w d_w z_w) / vol.
__global__ void y_from_z(int64_t n, const double *d, const double *z, const double *dz, double vol,
                         double *y) {
    const double m = *dz / vol;
    for (int64_t u = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; u < n;
         u += (int64_t)gridDim.x * blockDim.x) {
        const double sd = sqrt(d[u]);
        y[u] = sd * z[u] - sd * m;
    }
}

// Algorithm 1, recovery, with t_u = sums_u / l (Section 5's estimator).
__global__ void recover(int64_t n, const double *d, int32_t v, double vol, const double *sums,
                        double inv_l, const double *y, double *H) {
    const double dv = d[v], yv = y[v];
    for (int64_t u = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; u < n;
         u += (int64_t)gridDim.x * blockDim.x) {
        const double du = d[u];
        const double pi = du / vol;
        if (u == v) {
            H[u] = yv / pi;
        } else {
            const double t = sums[u] * inv_l;
            const double r = du / dv;
            H[u] = (t - r * yv + 2.0 * sqrt(r) * y[u]) / pi;
        }
    }
}

// [k][n] <-> [n][k]
__global__ void transpose64(int64_t rows, int64_t cols, const double *in, double *out) {
    const int64_t tot = rows * cols;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < tot;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t r = i / cols, c = i - r * cols;
        out[c * rows + r] = in[i];
    }
}

// Gradient right-hand sides, node-major [n][NP K + 2], NP = 1 or 2 parts:
//   columns i < K: sqrt(c+_u) Q_iu, and with NP = 2 columns K + i:
//   sqrt(c-_u) Q_iu (c+ = max(c, 0), c- = max(-c, 0); the same Q for both
//   parts; Q Rademacher +-1/sqrt(K) from Philox, or Q = I when exact),
//   column NP K: c_u, column NP K + 1: d_u.  sum_u c_u phi_u^2 is linear in c,
//   so the two parts' sketches enter the gradient with signs + and -.
__global__ void grad_rhs(int64_t n, int K, int NP, int exact, const double *c, const double *d,
                         uint32_t k0, uint32_t k1, double *R) {
    const int64_t KS = (int64_t)NP * K, cols = KS + 2, tot = n * cols;
    const double scale = exact ? 1.0 : 1.0 / sqrt((double)K);
    for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < tot;
         idx += (int64_t)gridDim.x * blockDim.x) {
        const int64_t u = idx / cols;
        const int64_t j = idx - u * cols;
        double val;
        if (j == KS) val = c[u];
        else if (j == KS + 1) val = d[u];
        else {
            const int part = (int)(j / K), i = (int)(j - (int64_t)part * K);
            double q;
            if (exact) q = (i == u) ? 1.0 : 0.0;
            else {
                const Ctr4 o = philox4x32_10(Ctr4{(uint32_t)i, (uint32_t)u, 0xFFFFFFFFu, 0u}, k0, k1);
                q = (o.x >> 31) ? -scale : scale;
            }
            const double cu = part == 0 ? fmax(c[u], 0.0) : fmax(-c[u], 0.0);
            val = sqrt(cu) * q;
        }
        R[idx] = val;
    }
}

// 1 in *flag if some c_u < 0 (the signed split needs the second part).
__global__ void any_negative(int64_t n, const double *c, int *flag) {
    for (int64_t u = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; u < n;
         u += (int64_t)gridDim.x * blockDim.x)
        if (c[u] < 0.0) *flag = 1;
}

// tr(C L^+) estimate tr(Z C^1/2 Q^T) = sum_u sum_i X[u][i] R[u][i] over the
// sketch columns, the second part (c-) with sign -.  Block parts in parts
// (added in block order by sum_parts).
__global__ void grad_trace(int64_t n, int K, int NP, const double *X, const double *R, double *parts) {
    const int64_t KS = (int64_t)NP * K, cols = KS + 2, tot = n * cols;
    double s = 0.0;
    for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < tot;
         idx += (int64_t)gridDim.x * blockDim.x) {
        const int64_t j = idx % cols;
        if (j < K) s += X[idx] * R[idx];
        else if (j < KS) s -= X[idx] * R[idx];
    }
    s = block_sum_fixed(s);
    if (threadIdx.x == 0) parts[blockIdx.x] = s;
}

// sum_u X[u][col] * w[u]: block parts in parts (added by sum_parts).
__global__ void col_dot(int64_t n, int64_t cols, int64_t col, const double *X, const double *w,
                        double *parts) {
    double s = 0.0;
    for (int64_t u = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; u < n;
         u += (int64_t)gridDim.x * blockDim.x)
        s += X[u * cols + col] * w[u];
    s = block_sum_fixed(s);
    if (threadIdx.x == 0) parts[blockIdx.x] = s;
}

// Number of arcs (a, b) with b > a in each row (rows sorted ascending).
template <bool OFF64>
__global__ void upper_counts(DevGraph g, int32_t *cnt, int32_t *first) {
    for (int64_t a = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; a < g.n;
         a += (int64_t)gridDim.x * blockDim.x) {
        int64_t lo = OFF64 ? g.rp64[a] : g.rp32[a];
        const int64_t e = OFF64 ? g.rp64[a + 1] : g.rp32[a + 1];
        int64_t hi = e;
        while (lo < hi) {
            const int64_t mid = (lo + hi) >> 1;
            if (g.col[mid] > a) hi = mid; else lo = mid + 1;
        }
        first[a] = (int32_t)(lo - (OFF64 ? g.rp64[a] : g.rp32[a]));
        cnt[a] = (int32_t)(e - lo);
    }
}

// dJ/dw_e for every arc (a, b) with a < b; one warp per row.  Columns of X:
// NP K sketch columns (the c- part with sign -), then x = L^+ c, y = L^+ d.
template <bool OFF64>
__global__ void grad_edges(DevGraph g, int K, int NP, const double *X, const int64_t *off,
                           const int32_t *first, const double *scal, float *out) {
    const int KS = NP * K;
    const int64_t cols = (int64_t)KS + 2;
    const double trCP = scal[0], dTy = scal[1], csum = scal[2];
    const double vol = g.vol;
    const int lane = threadIdx.x & 31;
    const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t a = warp; a < g.n; a += nwarps) {
        const int64_t rb = OFF64 ? g.rp64[a] : g.rp32[a];
        const int64_t re = OFF64 ? g.rp64[a + 1] : g.rp32[a + 1];
        const double xa = X[a * cols + KS], ya = X[a * cols + KS + 1];
        for (int64_t j = rb + first[a]; j < re; ++j) {
            const int64_t b = g.col[j];
            double sq = 0.0;
            for (int i = lane; i < KS; i += 32) {
                const double df = X[a * cols + i] - X[b * cols + i];
                sq += (i < K) ? df * df : -(df * df);
            }
            sq = warp_sum(sq);
            if (lane == 0) {
                const double xb = X[b * cols + KS], yb = X[b * cols + KS + 1];
                const double gval = 2.0 * trCP - vol * sq + 2.0 * (xa - xb) * (ya - yb) - 2.0 * (xa + xb) +
                                    csum * ((2.0 * (ya + yb) - (ya - yb) * (ya - yb)) / vol -
                                            2.0 * dTy / (vol * vol));
                out[off[a] + (j - rb - first[a])] = (float)gval;
            }
        }
    }
}

template <class F>
void dispatch_off(const DevGraph &g, F f) {
    if (g.off64) f(std::true_type{});
    else f(std::false_type{});
}

}  // namespace
}  // namespace rwc

using namespace rwc;

extern "C" rwc_status rwc_recover(rwc_graph_t *G, const double *sums, int64_t T, const double *y,
                                  double *H, rwc_stream_t stream) {
    clear_error();
    if (!G || !sums || !y || !H || T <= 0) return set_error(RWC_ERR_INVALID, "bad argument");
    const DevGraph &g = G->g;
    cudaStream_t st = (cudaStream_t)stream;
    ::rwc::count_launches(1); recover<<<grid_for(g.n), TPB, 0, st>>>(g.n, g.d, g.root, g.vol, sums, 1.0 / (double)T, y, H);
    RWC_CUDA_TRY(cudaGetLastError());
    RWC_CUDA_TRY(cudaStreamSynchronize(st));
    return RWC_OK;
}

namespace rwc {
namespace {
// Algorithm 1's pivot column: b = sqrt(d_v) e_v - (sqrt(d_v) / vol) d,
// z = L^+ b, y_u = sqrt(d_u) z_u - sqrt(d_u) (sum_w d_w z_w) / vol.  It
// depends on the graph only, not on the sampled trees.  Enqueued on st; the
// solver itself synchronises st between refinements.
rwc_status pivot_column(rwc_graph *G, double tol, double *y, cudaStream_t st) {
    const DevGraph &g = G->g;
    const int64_t n = g.n;
    Buf buf(st);
    const unsigned gs = grid_for(n);
    RWC_CUDA_TRY(cudaMallocAsync(&buf.p, (size_t)n * 2 * sizeof(double) + (size_t)(gs + 8) * sizeof(double), st));
    double *b = (double *)buf.p, *z = b + n;
    double *dz = (double *)((char *)buf.p + (size_t)n * 2 * sizeof(double));
    double *parts = dz + 8;
    ::rwc::count_launches(1); rhs_pivot<<<gs, TPB, 0, st>>>(n, g.d, g.root, g.vol, b);
    RWC_CUDA_TRY(cudaGetLastError());
    RWC_TRY(solve_nodemajor(G, 1, b, z, tol > 0 ? tol : 1e-10, nullptr, st));
    ::rwc::count_launches(1); dot64<<<gs, TPB, 0, st>>>(n, g.d, z, parts);
    ::rwc::count_launches(1); sum_parts<<<1, TPB, 0, st>>>(parts, (int)gs, 0, 1, dz);
    ::rwc::count_launches(1); y_from_z<<<gs, TPB, 0, st>>>(n, g.d, z, dz, g.vol, y);
    RWC_CUDA_TRY(cudaGetLastError());
    return RWC_OK;
}
}  // namespace
}  // namespace rwc

extern "C" rwc_status rwc_pivot_solve(rwc_graph_t *G, double tol, double *y, rwc_stream_t stream) {
    clear_error();
    if (!G || !y) return set_error(RWC_ERR_INVALID, "bad argument");
    cudaStream_t st = (cudaStream_t)stream;
    RWC_TRY(pivot_column(G, tol, y, st));
    RWC_CUDA_TRY(cudaStreamSynchronize(st));
    return RWC_OK;
}

extern "C" rwc_status rwc_estimate(rwc_graph_t *G, const double *sums, int64_t T, double tol,
                                   double *H, double *y_out, rwc_stream_t stream) {
    clear_error();
    if (!G || !sums || !H || T <= 0) return set_error(RWC_ERR_INVALID, "bad argument");
    const DevGraph &g = G->g;
    cudaStream_t st = (cudaStream_t)stream;
    const int64_t n = g.n;
    Buf buf(st);
    double *y = y_out;
    if (!y) {
        RWC_CUDA_TRY(cudaMallocAsync(&buf.p, (size_t)n * sizeof(double), st));
        y = (double *)buf.p;
    }
    RWC_TRY(pivot_column(G, tol, y, st));
    ::rwc::count_launches(1); recover<<<grid_for(n), TPB, 0, st>>>(n, g.d, g.root, g.vol, sums, 1.0 / (double)T, y, H);
    RWC_CUDA_TRY(cudaGetLastError());
    RWC_CUDA_TRY(cudaStreamSynchronize(st));
    return RWC_OK;
}

extern "C" rwc_status rwc_solve(rwc_graph_t *G, int32_t k, const double *B, double *X, double tol,
                                int32_t *iters_out, rwc_stream_t stream) {
    clear_error();
    if (!G || !B || !X || k <= 0) return set_error(RWC_ERR_INVALID, "bad argument");
    const int64_t n = G->g.n;
    cudaStream_t st = (cudaStream_t)stream;
    Buf buf(st);
    RWC_CUDA_TRY(cudaMallocAsync(&buf.p, (size_t)n * k * 2 * sizeof(double), st));
    double *Bn = (double *)buf.p, *Xn = Bn + (size_t)n * k;
    const unsigned gs = grid_for(n * k);
    ::rwc::count_launches(1); transpose64<<<gs, TPB, 0, st>>>(k, n, B, Bn);
    RWC_CUDA_TRY(cudaGetLastError());
    int it = 0;
    RWC_TRY(solve_nodemajor(G, k, Bn, Xn, tol, &it, st));
    ::rwc::count_launches(1); transpose64<<<gs, TPB, 0, st>>>(n, k, Xn, X);
    RWC_CUDA_TRY(cudaGetLastError());
    RWC_CUDA_TRY(cudaStreamSynchronize(st));
    if (iters_out) *iters_out = it;
    return RWC_OK;
}

extern "C" rwc_status rwc_grad(rwc_graph_t *G, const double *c, int32_t k, uint64_t seed, double tol,
                               float *grad_w, rwc_stream_t stream) {
    clear_error();
    if (!G || !c || !grad_w || k < 0) return set_error(RWC_ERR_INVALID, "bad argument");
    const DevGraph &g = G->g;
    const int64_t n = g.n;
    const int exact = (k == 0);
    const int K = exact ? (int)n : k;
    if (exact && n > 16384) return set_error(RWC_ERR_UNSUPPORTED, "exact gradient (k = 0) needs n <= 16384");
    cudaStream_t st = (cudaStream_t)stream;
    // signed c: a second set of K sketch columns for the negative part
    int NP = 1;
    {
        int *flag = nullptr;
        RWC_CUDA_TRY(cudaMallocAsync((void **)&flag, sizeof(int), st));
        RWC_CUDA_TRY(cudaMemsetAsync(flag, 0, sizeof(int), st));
        ::rwc::count_launches(1); any_negative<<<grid_for(n), TPB, 0, st>>>(n, c, flag);
        int h = 0;
        const cudaError_t e1 = cudaMemcpyAsync(&h, flag, sizeof(int), cudaMemcpyDeviceToHost, st);
        const cudaError_t e2 = cudaStreamSynchronize(st);
        cudaFreeAsync(flag, st);
        RWC_CUDA_TRY(e1);
        RWC_CUDA_TRY(e2);
        NP = h ? 2 : 1;
    }
    const int64_t cols = (int64_t)NP * K + 2;
    Buf buf(st);
    const size_t pcap = (size_t)num_sms() * 8;   // grid_for's largest grid: block parts below
    const size_t bytes = (size_t)n * cols * 2 * sizeof(double) + (size_t)n * (8 + 4 + 4) + 256 +
                         pcap * sizeof(double);
    RWC_CUDA_TRY(cudaMallocAsync(&buf.p, bytes, st));
    double *R = (double *)buf.p, *X = R + (size_t)n * cols;
    int64_t *off = (int64_t *)(X + (size_t)n * cols);
    int32_t *cnt = (int32_t *)(off + n), *first = cnt + n;
    double *scal = (double *)(((uintptr_t)(first + n) + 63) & ~(uintptr_t)63);   // [8]
    double *tparts = scal + 8;                                                      // [pcap]
    ::rwc::count_launches(1); grad_rhs<<<grid_for(n * cols), TPB, 0, st>>>(n, K, NP, exact, c, g.d, (uint32_t)seed,
                                                 (uint32_t)(seed >> 32), R);
    RWC_CUDA_TRY(cudaGetLastError());
    RWC_TRY(solve_nodemajor(G, (int)cols, R, X, tol > 0 ? tol : 1e-8, nullptr, st));
    RWC_CUDA_TRY(cudaMemsetAsync(scal, 0, 4 * sizeof(double), st));
    {   // tr(C L^+), d^T y and sum c, each in a fixed order (block parts added in
        // block order)
        const unsigned gt = grid_for(n * cols), gn = grid_for(n);
        ::rwc::count_launches(2);
        grad_trace<<<gt, TPB, 0, st>>>(n, K, NP, X, R, tparts);
        sum_parts<<<1, TPB, 0, st>>>(tparts, (int)gt, 0, 1, scal);
        ::rwc::count_launches(2);
        col_dot<<<gn, TPB, 0, st>>>(n, cols, cols - 1, X, g.d, tparts);   // d^T y
        sum_parts<<<1, TPB, 0, st>>>(tparts, (int)gn, 0, 1, scal + 1);
        ::rwc::count_launches(2);
        dot64<<<gn, TPB, 0, st>>>(n, c, nullptr, tparts);
        sum_parts<<<1, TPB, 0, st>>>(tparts, (int)gn, 0, 1, scal + 2);
    }
    dispatch_off(g, [&](auto o64) {
        ::rwc::count_launches(1); upper_counts<decltype(o64)::value><<<grid_for(n), TPB, 0, st>>>(g, cnt, first);
    });
    RWC_CUDA_TRY(cudaGetLastError());
    std::vector<int32_t> hc(n);
    std::vector<int64_t> ho(n);
    RWC_CUDA_TRY(cudaMemcpyAsync(hc.data(), cnt, (size_t)n * 4, cudaMemcpyDeviceToHost, st));
    RWC_CUDA_TRY(cudaStreamSynchronize(st));
    int64_t acc = 0;
    for (int64_t a = 0; a < n; ++a) { ho[a] = acc; acc += hc[a]; }
    RWC_CUDA_TRY(cudaMemcpyAsync(off, ho.data(), (size_t)n * 8, cudaMemcpyHostToDevice, st));
    dispatch_off(g, [&](auto o64) {
        ::rwc::count_launches(1); grad_edges<decltype(o64)::value><<<grid_for(n * 32), TPB, 0, st>>>(g, K, NP, X, off, first, scal, grad_w);
    });
    RWC_CUDA_TRY(cudaGetLastError());
    RWC_CUDA_TRY(cudaStreamSynchronize(st));
    return RWC_OK;
}

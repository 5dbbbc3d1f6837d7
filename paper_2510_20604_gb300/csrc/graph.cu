// Graph store: host-side validation, weighted degrees, pivot choice, alias
// tables, and the device copy (Section 2.2's graph and matrices, read for
// weighted graphs: d = weighted degree, vol = sum d in place of 2m).
#include <algorithm>
#include <new>
#include <atomic>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <thread>
#include <vector>

#include "rwc_common.cuh"

namespace rwc {

static thread_local std::string g_last_error;

rwc_status set_error(rwc_status st, const char *fmt, ...) {
    char buf[1024];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    g_last_error = buf;
    return st;
}

void clear_error() { g_last_error.clear(); }

static std::atomic<int64_t> g_launches{0};
void count_launches(int64_t k) { g_launches.fetch_add(k, std::memory_order_relaxed); }

cudaError_t graph_alloc(rwc_graph *G, void **p, size_t bytes) {
    if (G->nallocs >= (int)(sizeof(G->allocs) / sizeof(G->allocs[0]))) return cudaErrorMemoryAllocation;
    cudaError_t e = cudaMalloc(p, bytes ? bytes : 16);
    if (e == cudaSuccess) {
        G->allocs[G->nallocs++] = *p;
        G->device_bytes += (int64_t)bytes;
    }
    return e;
}

static void graph_free(rwc_graph *G) {
    for (int i = 0; i < G->nallocs; ++i) cudaFree(G->allocs[i]);
    G->nallocs = 0;
    if (G->host_scalars) cudaFreeHost(G->host_scalars);
    G->host_scalars = nullptr;
}

// Run f(lo, hi) over [0, n) on a few host threads.
template <class F>
static void parallel_rows(int64_t n, F f) {
    unsigned hw = std::thread::hardware_concurrency();
    int nt = (int)std::min<int64_t>(std::max(1u, std::min(hw, 32u)), std::max<int64_t>(1, n / 4096));
    if (nt <= 1) { f((int64_t)0, n); return; }
    std::vector<std::thread> th;
    int64_t step = (n + nt - 1) / nt;
    for (int t = 0; t < nt; ++t) {
        int64_t lo = t * step, hi = std::min(n, lo + step);
        if (lo >= hi) break;
        th.emplace_back([=, &f] { f(lo, hi); });
    }
    for (auto &x : th) x.join();
}

// Vose's alias method for one row, in the fixed form every implementation of
// this project follows: FP64 probabilities p_j = w_j * deg / S (S summed in
// arc order); two FIFO work lists in ascending index; a small entry s is
// paired with the entry l at the front of the large list (thr_s = p_s,
// alias_s = l, p_l <- (p_l + p_s) - 1, and l moves to the back of the small
// list once p_l < 1); entries left over keep probability 1.  Thresholds are
// floor(p * 2^32) clamped to 2^32 - 1.
void vose_row(const float *w, int64_t deg, uint32_t *thr, int32_t *alias,
                     std::vector<double> &prob, std::vector<int64_t> &lo_q,
                     std::vector<int64_t> &hi_q) {
    double total = 0.0;
    for (int64_t j = 0; j < deg; ++j) total = total + (double)w[j];
    prob.resize(deg);
    lo_q.clear();
    hi_q.clear();
    for (int64_t j = 0; j < deg; ++j) {
        prob[j] = ((double)w[j] * (double)deg) / total;
        (prob[j] < 1.0 ? lo_q : hi_q).push_back(j);
    }
    auto to_u32 = [](double p) -> uint32_t {
        const double scaled = p * 4294967296.0;
        return scaled >= 4294967295.0 ? 0xFFFFFFFFu : (uint32_t)scaled;
    };
    size_t lo_head = 0, hi_head = 0;
    while (lo_head < lo_q.size() && hi_head < hi_q.size()) {
        const int64_t s = lo_q[lo_head++];
        const int64_t l = hi_q[hi_head];
        thr[s] = to_u32(prob[s]);
        alias[s] = (int32_t)l;
        prob[l] = (prob[l] + prob[s]) - 1.0;
        if (prob[l] < 1.0) {
            ++hi_head;
            lo_q.push_back(l);
        }
    }
    for (size_t i = lo_head; i < lo_q.size(); ++i) { thr[lo_q[i]] = 0xFFFFFFFFu; alias[lo_q[i]] = (int32_t)lo_q[i]; }
    for (size_t i = hi_head; i < hi_q.size(); ++i) { thr[hi_q[i]] = 0xFFFFFFFFu; alias[hi_q[i]] = (int32_t)hi_q[i]; }
}

struct HostCheck {
    std::atomic<int> bad{0};
    std::atomic<int64_t> bad_row{-1};
    const char *why = nullptr;
    void fail(int64_t u, const char *w) {
        int z = 0;
        if (bad.compare_exchange_strong(z, 1)) { bad_row = u; why = w; }
    }
};

rwc_status validate_csr(int64_t n, int64_t nnz, const int64_t *rp, const int32_t *col,
                        const float *w) {
    if (n < 2) return set_error(RWC_ERR_INVALID, "n must be >= 2 (got %lld)", (long long)n);
    if (n >= ((int64_t)1 << 31) - 1) return set_error(RWC_ERR_INVALID, "n must fit int32 ids");
    if (nnz < 0 || nnz >= ((int64_t)1 << 40)) return set_error(RWC_ERR_INVALID, "bad nnz");
    if (!rp || (nnz > 0 && !col)) return set_error(RWC_ERR_INVALID, "null CSR pointer");
    if (rp[0] != 0 || rp[n] != nnz)
        return set_error(RWC_ERR_INVALID, "row_ptr[0] must be 0 and row_ptr[n] == nnz");
    for (int64_t u = 0; u < n; ++u)
        if (rp[u + 1] < rp[u]) return set_error(RWC_ERR_INVALID, "row_ptr decreases at row %lld", (long long)u);
    HostCheck chk;
    parallel_rows(n, [&](int64_t lo, int64_t hi) {
        std::vector<float> a, b;
        for (int64_t u = lo; u < hi && !chk.bad; ++u) {
            const int64_t b0 = rp[u], b1 = rp[u + 1];
            if (b1 == b0) { chk.fail(u, "isolated vertex"); return; }
            if (b1 - b0 >= ((int64_t)1 << 32)) { chk.fail(u, "row longer than 2^32 arcs"); return; }
            for (int64_t j = b0; j < b1; ++j) {
                const int32_t c = col[j];
                if (c < 0 || c >= n) { chk.fail(u, "column index out of range"); return; }
                if (c == u) { chk.fail(u, "self-loop"); return; }
                if (j > b0 && col[j - 1] > c) { chk.fail(u, "row not sorted"); return; }
                if (w && !(std::isfinite(w[j]) && w[j] > 0.0f)) { chk.fail(u, "weight not finite and positive"); return; }
            }
            // every run of equal heads must match the reverse run in the head's row
            for (int64_t j = b0; j < b1;) {
                const int32_t c = col[j];
                int64_t e = j;
                while (e < b1 && col[e] == c) ++e;
                const int32_t *rb = col + rp[c], *re = col + rp[c + 1];
                const int32_t *lo_it = std::lower_bound(rb, re, (int32_t)u);
                const int32_t *hi_it = std::upper_bound(lo_it, re, (int32_t)u);
                if (hi_it - lo_it != e - j) { chk.fail(u, "arc without matching reverse arc"); return; }
                if (w) {
                    a.assign(w + j, w + e);
                    b.assign(w + (lo_it - col), w + (hi_it - col));
                    std::sort(a.begin(), a.end());
                    std::sort(b.begin(), b.end());
                    if (a != b) { chk.fail(u, "reverse arcs carry different weights"); return; }
                }
                j = e;
            }
        }
    });
    if (chk.bad)
        return set_error(RWC_ERR_INVALID, "invalid graph at row %lld: %s", (long long)chk.bad_row.load(), chk.why);
    return RWC_OK;
}

bool csr_connected(int64_t n, const int64_t *rp, const int32_t *col) {
    std::vector<uint8_t> seen(n, 0);
    std::vector<int32_t> q;
    q.reserve(n);
    q.push_back(0);
    seen[0] = 1;
    for (size_t h = 0; h < q.size(); ++h) {
        const int32_t u = q[h];
        for (int64_t j = rp[u]; j < rp[u + 1]; ++j) {
            const int32_t c = col[j];
            if (!seen[c]) { seen[c] = 1; q.push_back(c); }
        }
    }
    return (int64_t)q.size() == n;
}

template <class T>
static cudaError_t upload(rwc_graph *G, T **dst, const T *src, size_t count) {
    cudaError_t e = graph_alloc(G, (void **)dst, count * sizeof(T));
    if (e != cudaSuccess) return e;
    return cudaMemcpy(*dst, src, count * sizeof(T), cudaMemcpyHostToDevice);
}

static rwc_status create_impl(int64_t n, int64_t nnz, const int64_t *rp, const int32_t *col,
                              const float *w, int32_t root, uint32_t flags, rwc_graph_t **out) {
    if (!out) return set_error(RWC_ERR_INVALID, "out is NULL");
    *out = nullptr;
    RWC_TRY(validate_csr(n, nnz, rp, col, w));
    if (!(flags & RWC_GRAPH_SKIP_CONNECTIVITY) && !csr_connected(n, rp, col))
        return set_error(RWC_ERR_NOT_CONNECTED, "graph is not connected");

    // weighted degrees in arc order (FP64), vol, pivot
    std::vector<double> d(n);
    parallel_rows(n, [&](int64_t lo, int64_t hi) {
        for (int64_t u = lo; u < hi; ++u) {
            if (!w) { d[u] = (double)(rp[u + 1] - rp[u]); continue; }
            double s = 0.0;
            for (int64_t j = rp[u]; j < rp[u + 1]; ++j) s = s + (double)w[j];
            d[u] = s;
        }
    });
    double vol = 0.0, dmax = -1.0;
    int32_t arg = 0;
    for (int64_t u = 0; u < n; ++u) {
        vol += d[u];
        if (d[u] > dmax) { dmax = d[u]; arg = (int32_t)u; }
    }
    if (root < -1 || root >= n) return set_error(RWC_ERR_INVALID, "root out of range");
    if (root == -1) root = arg;

    rwc_graph *G = new (std::nothrow) rwc_graph();
    if (!G) return set_error(RWC_ERR_OOM, "host allocation failed");
    DevGraph &g = G->g;
    g.n = n; g.nnz = nnz; g.root = root; g.weighted = (w != nullptr);
    g.off64 = (flags & RWC_GRAPH_INT64_OFFSETS) || nnz >= ((int64_t)1 << 31) - 1;
    g.vol = vol; g.dmax = dmax;

    auto fail = [&](cudaError_t e, const char *what) {
        graph_free(G);
        delete G;
        return set_error(e == cudaErrorMemoryAllocation ? RWC_ERR_OOM : RWC_ERR_CUDA,
                         "%s: %s", what, cudaGetErrorString(e));
    };
    cudaError_t e;
    if (g.off64) {
        int64_t *p;
        if ((e = upload(G, &p, rp, (size_t)n + 1)) != cudaSuccess) return fail(e, "row_ptr");
        g.rp64 = p;
    } else {
        std::vector<int32_t> rp32(n + 1);
        for (int64_t u = 0; u <= n; ++u) rp32[u] = (int32_t)rp[u];
        int32_t *p;
        if ((e = upload(G, &p, rp32.data(), (size_t)n + 1)) != cudaSuccess) return fail(e, "row_ptr");
        g.rp32 = p;
    }
    {
        int32_t *p;
        if ((e = upload(G, &p, col, (size_t)nnz)) != cudaSuccess) return fail(e, "col_idx");
        g.col = p;
    }
    if (w) {
        std::vector<WArc> arcs(nnz);
        parallel_rows(n, [&](int64_t lo, int64_t hi) {
            std::vector<double> prob;
            std::vector<int64_t> ql, qh;
            std::vector<uint32_t> thr;
            std::vector<int32_t> al;
            for (int64_t u = lo; u < hi; ++u) {
                const int64_t b = rp[u], deg = rp[u + 1] - rp[u];
                thr.resize(deg); al.resize(deg);
                vose_row(w + b, deg, thr.data(), al.data(), prob, ql, qh);
                for (int64_t j = 0; j < deg; ++j)
                    arcs[b + j] = WArc{col[b + j], thr[j], col[b + al[j]], al[j]};
            }
        });
        WArc *pa;
        if ((e = upload(G, &pa, arcs.data(), (size_t)nnz)) != cudaSuccess) return fail(e, "alias tables");
        g.warc = pa;
        float *pw;
        if ((e = upload(G, &pw, w, (size_t)nnz)) != cudaSuccess) return fail(e, "weights");
        g.w = pw;
    }
    {
        double *pd;
        if ((e = upload(G, &pd, d.data(), (size_t)n)) != cudaSuccess) return fail(e, "degrees");
        g.d = pd;
        std::vector<float> di(n);
        for (int64_t u = 0; u < n; ++u) di[u] = (float)(1.0 / d[u]);
        float *pdi;
        if ((e = upload(G, &pdi, di.data(), (size_t)n)) != cudaSuccess) return fail(e, "inverse degrees");
        g.dinv32 = pdi;
    }
    {
        // chunks of the heavy rows (a row's chunks consecutive, rows in order)
        std::vector<int32_t> crow, hf;
        std::vector<int64_t> cbeg;
        for (int64_t u = 0; u < n; ++u) {
            const int64_t deg = rp[u + 1] - rp[u];
            if (deg <= HEAVY_DEG) continue;
            if (hf.empty()) hf.assign(n, -1);
            hf[u] = (int32_t)crow.size();
            for (int64_t j = rp[u]; j < rp[u + 1]; j += HEAVY_CHUNK) {
                crow.push_back((int32_t)u);
                cbeg.push_back(j);
            }
        }
        if (!crow.empty()) {
            int32_t *pr, *ph;
            int64_t *pb;
            if ((e = upload(G, &pr, crow.data(), crow.size())) != cudaSuccess) return fail(e, "heavy rows");
            if ((e = upload(G, &pb, cbeg.data(), cbeg.size())) != cudaSuccess) return fail(e, "heavy rows");
            if ((e = upload(G, &ph, hf.data(), hf.size())) != cudaSuccess) return fail(e, "heavy rows");
            g.hc_n = (int64_t)crow.size(); g.hc_row = pr; g.hc_beg = pb; g.hfirst = ph;
        }
    }
    {
        // rows of at most HEAVY_DEG arcs by degree bin (2, 4, 8, 16, more arcs)
        std::vector<int32_t> bins[5];
        for (int64_t u = 0; u < n; ++u) {
            const int64_t deg = rp[u + 1] - rp[u];
            if (deg > HEAVY_DEG) continue;
            const int b = deg <= 2 ? 0 : deg <= 4 ? 1 : deg <= 8 ? 2 : deg <= 16 ? 3 : 4;
            bins[b].push_back((int32_t)u);
        }
        std::vector<int32_t> all;
        all.reserve((size_t)n);
        for (int b = 0; b < 5; ++b) {
            g.bin_off[b] = (int64_t)all.size();
            all.insert(all.end(), bins[b].begin(), bins[b].end());
        }
        g.bin_off[5] = (int64_t)all.size();
        if (!all.empty()) {
            int32_t *pbr;
            if ((e = upload(G, &pbr, all.data(), all.size())) != cudaSuccess) return fail(e, "degree bins");
            g.bin_rows = pbr;
        }
    }
    if (!w && !g.off64) {
        // inline neighbour lists for bounded-degree graphs (grids, meshes)
        int64_t maxdeg = 0;
        for (int64_t u = 0; u < n; ++u) maxdeg = std::max<int64_t>(maxdeg, rp[u + 1] - rp[u]);
        const int ew = maxdeg <= 4 ? 4 : maxdeg <= 8 ? 8 : 0;
        if (ew) {
            std::vector<int32_t> rows((size_t)n * ew, -1);
            for (int64_t u = 0; u < n; ++u)
                for (int64_t j = rp[u]; j < rp[u + 1]; ++j) rows[(size_t)u * ew + (j - rp[u])] = col[j];
            int32_t *pe;
            if ((e = upload(G, &pe, rows.data(), rows.size())) != cudaSuccess) return fail(e, "inline rows");
            g.ell = reinterpret_cast<const int4 *>(pe);
            g.ell_w = ew;
        }
    }
    {
        int *ps;
        if ((e = graph_alloc(G, (void **)&ps, 256)) != cudaSuccess) return fail(e, "status word");
        if ((e = cudaMemset(ps, 0, 256)) != cudaSuccess) return fail(e, "status word");
        G->dev_status = ps;
    }
    if ((e = cudaMallocHost((void **)&G->host_scalars, 64 * sizeof(int64_t))) != cudaSuccess)
        return fail(e, "pinned scalars");
    *out = G;
    return RWC_OK;
}

}  // namespace rwc

extern "C" {

const char *rwc_last_error(void) { return rwc::g_last_error.c_str(); }

const char *rwc_version(void) { return "rwc-gb300 0.1 (sm_103a)"; }

int64_t rwc_launch_count(void) { return rwc::g_launches.load(); }

rwc_status rwc_graph_create(int64_t n, int64_t nnz, const int64_t *host_row_ptr,
                            const int32_t *host_col_idx, const float *host_w, int32_t root,
                            uint32_t flags, rwc_graph_t **out) {
    rwc::clear_error();
    try {
        return rwc::create_impl(n, nnz, host_row_ptr, host_col_idx, host_w, root, flags, out);
    } catch (const std::bad_alloc &) {
        return rwc::set_error(RWC_ERR_OOM, "host allocation failed");
    }
}

rwc_status rwc_graph_info(const rwc_graph_t *G, rwc_graph_info_t *o) {
    if (!G || !o) return rwc::set_error(RWC_ERR_INVALID, "null argument");
    const rwc::DevGraph &g = G->g;
    o->n = g.n; o->nnz = g.nnz; o->root = g.root; o->weighted = g.weighted;
    o->offsets64 = g.off64; o->reserved = 0; o->vol = g.vol; o->dmax = g.dmax;
    o->device_bytes = G->device_bytes;
    return RWC_OK;
}

rwc_status rwc_graph_destroy(rwc_graph_t *G) {
    if (!G) return RWC_OK;
    rwc::graph_free(G);
    delete G;
    return RWC_OK;
}

}  // extern "C"

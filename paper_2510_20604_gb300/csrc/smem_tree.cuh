// One rooted spanning tree per thread block, all state in shared memory.
// Same round structure as the HBM sampler (walk / classify / pop / finish),
// specialised for n <= 20000: vertex-indexed flags instead of marked lists,
// int16 vertex ids, uint16 pop counts, no jump pointers.
#pragma once

#include "rwc_common.cuh"

namespace rwc {

constexpr int SM_ERR_ROUNDS = 1;   // max_rounds reached
constexpr int SM_ERR_KOVF = 2;     // a pop count exceeded 65535
constexpr int SM_ERR_LOOP = 4;     // internal: a pointer chase exceeded n steps

constexpr uint8_t SF_MARK = 1, SF_SET = 2, SF_NEXT = 4, SF_LEAD = 8, SF_TREE = 16;

// Shared-memory bytes for a tree of n vertices (acc, P, K, NM, F).
__host__ __device__ inline size_t smem_tree_bytes(int64_t n) { return (size_t)n * 11 + 64; }

struct SmemTree {
    uint32_t *acc;   // visit accumulator over the trees a block runs
    int16_t *P;      // current top
    uint16_t *K;     // pops
    int16_t *NM;     // compressed successor
    uint8_t *F;      // flags
    __device__ void carve(unsigned char *smem, int n) {
        acc = reinterpret_cast<uint32_t *>(smem);
        P = reinterpret_cast<int16_t *>(acc + n);
        K = reinterpret_cast<uint16_t *>(P + n);
        NM = reinterpret_cast<int16_t *>(K + n);
        F = reinterpret_cast<uint8_t *>(NM + n);
    }
};

// The thread group that runs one tree: a whole thread block, or one warp
// (warp-per-tree, for small graphs: several trees per block, synchronised
// with __syncwarp instead of block barriers).
struct BlockGroup {
    static __device__ __forceinline__ int rank() { return threadIdx.x; }
    static __device__ __forceinline__ int size() { return blockDim.x; }
    static __device__ __forceinline__ void sync() { __syncthreads(); }
    static __device__ __forceinline__ int any(int p) { return __syncthreads_or(p); }
};
struct WarpGroup {
    static __device__ __forceinline__ int rank() { return threadIdx.x & 31; }
    static __device__ __forceinline__ int size() { return 32; }
    static __device__ __forceinline__ void sync() { __syncwarp(); }
    static __device__ __forceinline__ int any(int p) { return __any_sync(0xffffffffu, p); }
};

// Runs one tree; adds visits to S.acc; optionally writes the tree's parents
// and visits rows.  Must be called by every thread of the group.  Returns a
// group-uniform error mask (0 on success); *rounds gets the round count.
template <bool OFF64, bool W, class Grp = BlockGroup>
__device__ int smem_tree(const DevGraph &g, const SmemTree &S, uint32_t tree, uint32_t gid,
                         uint32_t k0, uint32_t k1, int64_t max_rounds, int32_t *par_row,
                         int32_t *vis_row, int64_t *rounds) {
    const int n = (int)g.n;
    const int root = g.root;
    int16_t *P = S.P;
    uint16_t *K = S.K;
    int16_t *NM = S.NM;
    uint8_t *F = S.F;
    Grp::sync();
    for (int u = Grp::rank(); u < n; u += Grp::size()) {
        K[u] = 0;
        if (u == root) { F[u] = SF_SET; P[u] = -1; }
        else { F[u] = SF_MARK; P[u] = (int16_t)succ<OFF64, W>(g, u, 0u, tree, gid, k0, k1); }
    }
    Grp::sync();
    int any = 1, bad = 0, lerr = 0;
    int64_t r = 0;
    while (any) {
        if (++r > max_rounds) { lerr |= SM_ERR_ROUNDS; bad = 1; break; }
        // walk to the next marked or settled vertex
        for (int u = Grp::rank(); u < n; u += Grp::size()) {
            if (!(F[u] & SF_MARK)) continue;
            int x = P[u];
            for (int q = 0; !(F[x] & (SF_MARK | SF_SET)); ++q) {
                if (q > n) { lerr |= SM_ERR_LOOP; x = root; break; }
                x = P[x];
            }
            NM[u] = (F[x] & SF_SET) ? (int16_t)-1 : (int16_t)x;
        }
        Grp::sync();
        // classify: leader (smallest vertex of its cycle), reaches root, other
        for (int u = Grp::rank(); u < n; u += Grp::size()) {
            if (!(F[u] & SF_MARK)) continue;
            int x = NM[u], saved = -3, power = 1, lam = 0;
            uint8_t c = 0;
            for (int it = 0;; ++it) {
                if (x < 0) { c = SF_TREE; break; }
                if (x == u) { c = SF_LEAD; break; }
                if (x < u || x == saved) break;
                if (it > 2 * n + 4) { lerr |= SM_ERR_LOOP; break; }
                if (++lam == power) { saved = x; power <<= 1; lam = 0; }
                x = NM[x];
            }
            F[u] |= c;
        }
        Grp::sync();
        // pop cycles / settle segments that reach the root
        for (int u = Grp::rank(); u < n; u += Grp::size()) {
            const uint8_t f = F[u];
            if (f & SF_LEAD) {
                int w = u, q = 0;
                do {
                    if (++q > n) { lerr |= SM_ERR_LOOP; break; }
                    const int nx = P[w];
                    const uint32_t k = (uint32_t)K[w] + 1u;
                    if (k > 0xFFFFu) { lerr |= SM_ERR_KOVF; break; }
                    K[w] = (uint16_t)k;
                    P[w] = (int16_t)succ<OFF64, W>(g, w, k, tree, gid, k0, k1);
                    F[w] |= SF_NEXT;
                    w = nx;
                } while (w != u);
            } else if (f & SF_TREE) {
                int y = u, q = 0;
                do {
                    if (++q > n) { lerr |= SM_ERR_LOOP; break; }
                    F[y] |= SF_SET;
                    y = P[y];
                } while (!(F[y] & (SF_MARK | SF_SET)));
            }
        }
        Grp::sync();
        // popped vertices form the next marked set
        int mine = 0;
        for (int u = Grp::rank(); u < n; u += Grp::size()) {
            const uint8_t f = F[u];
            const uint8_t nf = (uint8_t)((f & SF_SET) | ((f & SF_NEXT) ? SF_MARK : 0));
            F[u] = nf;
            mine |= (nf & SF_MARK);
        }
        any = Grp::any(mine);
        bad = Grp::any(lerr);
        if (bad) break;
    }
    const int berr = Grp::any(lerr) ? 1 : 0;
    *rounds = r;
    if (!berr) {
        for (int u = Grp::rank(); u < n; u += Grp::size()) {
            const uint32_t vis = (u == root) ? 0u : (uint32_t)K[u] + 1u;
            S.acc[u] += vis;
            if (par_row) par_row[u] = (u == root) ? -1 : (int32_t)P[u];
            if (vis_row) vis_row[u] = (int32_t)vis;
        }
    }
    // error mask, identical in every thread: OR of lerr over the block
    int mask = 0;
    for (int bit = 1; bit <= 4; bit <<= 1)
        if (Grp::any(lerr & bit)) mask |= bit;
    return mask;
}

// One block runs trees blockIdx.x, blockIdx.x + gridDim.x, ... of one graph.
template <bool OFF64, bool W>
__global__ void s_trees(DevGraph g, uint32_t tree0, int64_t ntrees, uint32_t k0, uint32_t k1,
                        uint32_t gid, int64_t max_rounds, double *sums, int32_t *parents,
                        int32_t *visits, int *err, unsigned long long *round_ctr) {
    extern __shared__ __align__(16) unsigned char smem[];
    const int n = (int)g.n;
    SmemTree S;
    S.carve(smem, n);
    for (int u = threadIdx.x; u < n; u += blockDim.x) S.acc[u] = 0;
    unsigned long long rounds_here = 0;
    int mask = 0;
    for (int64_t t = blockIdx.x; t < ntrees && !mask; t += gridDim.x) {
        int64_t r = 0;
        mask = smem_tree<OFF64, W>(g, S, tree0 + (uint32_t)t, gid, k0, k1, max_rounds,
                                   parents ? parents + t * n : nullptr,
                                   visits ? visits + t * n : nullptr, &r);
        rounds_here += (unsigned long long)r;
    }
    __syncthreads();
    if (mask) { if (threadIdx.x == 0) atomicOr(err, mask); return; }
    unsigned long long draws = 0;
    for (int u = threadIdx.x; u < n; u += blockDim.x) {
        draws += S.acc[u];
        if (sums && S.acc[u]) atomicAdd(sums + u, (double)S.acc[u]);
    }
    if (draws) atomicAdd(round_ctr + 1, draws);
    if (threadIdx.x == 0 && rounds_here) atomicAdd(round_ctr, rounds_here);
}

}  // namespace rwc

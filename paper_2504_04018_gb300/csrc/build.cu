// GPU construction of the segment tree's graphs (the index of Section 4.2,
// Algorithm 3's tree: root [0, N-1], split at mid, no graph when
// r - l < leaf_size).
//
// Each graph node gets a flat proximity graph over its points. Instead of
// inserting points one by one with a beam search per insertion, every point
// of a node is "inserted" at once with a candidate pool made of
//   - its knn_k exact nearest neighbours inside the node (tiled brute force),
//   - its sample_k nearest points among an evenly spaced sample of the node
//     (long-range candidates, the role early insertions play in incremental
//     construction),
// from which edge occlusion (HNSW's neighbour-selection heuristic: keep c
// unless an already kept s has d(c, s) < d(c, u)) keeps at most M forward
// edges; reverse edges are then added and rows longer than R = 2M are
// re-selected with the same rule over the R * 2 closest candidates.
#include "esg_internal.cuh"

#include <algorithm>
#include <vector>

#include <cub/cub.cuh>

esg_status esg_launch_bruteforce_mode(int mode, const float *base, int64_t n, int32_t d,
                                      const float *queries, int64_t nq, const int64_t *l,
                                      const int64_t *r, int32_t k, int64_t *out_ids,
                                      float *out_dist, int32_t *out_count, const int64_t *id_map,
                                      int32_t exclude_self, const float *xnorm,
                                      const float *qnorm, cudaStream_t stream);
__global__ void row_norms_kernel(const float *X, int64_t n, int d, float *out);

namespace {

constexpr int kMaxPool = 256;   // candidate pool per point (knn_k + sample_k)
constexpr int kMaxRow = 128;    // R

// Node of `depth` that contains point i: its range, or an empty range when
// the node is a leaf (no graph). Also the node's index within the depth.
__global__ void point_node_kernel(int64_t n, int32_t leaf, int depth, int64_t *lo, int64_t *hi,
                                  int32_t *node_idx) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    int64_t l = 0, r = n - 1;
    int32_t idx = 0;
    bool ok = true;
    for (int t = 0; t < depth; ++t) {
        if (r - l < leaf) { ok = false; break; }
        int64_t mid = l + (r - l) / 2;
        if (i <= mid) { r = mid; idx = 2 * idx; } else { l = mid + 1; idx = 2 * idx + 1; }
    }
    if (ok && r - l < leaf) ok = false;
    lo[i] = ok ? l : 1;
    hi[i] = ok ? r : 0;
    node_idx[i] = ok ? idx : -1;
}

__global__ void gather_rows_kernel(const float *X, int d, const int64_t *rows, int64_t m, float *out) {
    int64_t i = blockIdx.x;
    if (i >= m) return;
    const float *src = X + rows[i] * d;
    float *dst = out + i * d;
    for (int j = threadIdx.x; j < d; j += blockDim.x) dst[j] = src[j];
}

__global__ void sample_range_kernel(int64_t n, const int32_t *node_idx, const int64_t *s_off,
                                    const int64_t *s_cnt, int64_t *lo, int64_t *hi) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    int32_t j = node_idx[i];
    if (j < 0) { lo[i] = 1; hi[i] = 0; return; }
    lo[i] = s_off[j];
    hi[i] = s_off[j] + s_cnt[j] - 1;
}

// Warp-cooperative distance between rows a and b.
__device__ __forceinline__ float row_dist(const float *X, int d, int metric, uint32_t a, uint32_t b) {
    const int lane = threadIdx.x & 31;
    const float *xa = X + (size_t)a * d, *xb = X + (size_t)b * d;
    float acc = 0.f;
    for (int j = lane; j < d; j += 32) {
        float u = __ldg(xa + j), v = __ldg(xb + j);
        if (metric == ESG_L2SQ) { float t = u - v; acc = fmaf(t, t, acc); }
        else acc = fmaf(u, v, acc);
    }
    acc = warp_sum_group(acc, 32);
    return metric == ESG_L2SQ ? acc : -acc;
}

// Edge occlusion over pool[0..m) (sorted ascending by distance to u, no
// duplicates, u excluded): keep c unless some kept s has d(c, s) < d(c, u).
// Returns the number kept (<= max_keep) in keep[].
__device__ int occlusion_select(const float *X, int d, int metric, const Cand *pool, int m,
                                int max_keep, uint32_t *keep) {
    int kept = 0;
    for (int i = 0; i < m && kept < max_keep; ++i) {
        const uint32_t c = pool[i].id;
        const float dcu = pool[i].d;
        bool good = true;
        for (int s = 0; s < kept; ++s) {
            if (row_dist(X, d, metric, c, keep[s]) < dcu) { good = false; break; }
        }
        if (good) {
            if ((threadIdx.x & 31) == 0) keep[kept] = c;
            __syncwarp();
            ++kept;
        }
    }
    return kept;
}

// Forward edges: merge the two candidate lists of point i, drop self and
// repeats, recompute exact distances, select by occlusion.
__global__ void forward_kernel(const float *X, int64_t n, int d, int metric, const int32_t *node_idx,
                               const int64_t *knn_ids, int K, const int64_t *smp_ids, int Ks,
                               int M, uint32_t *fwd, int32_t *indeg) {
    __shared__ Cand pool_s[4][kMaxPool];  // m <= kMaxPool, a power of two
    __shared__ uint32_t keep_s[4][kMaxRow];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    int64_t i = blockIdx.x * (int64_t)(blockDim.x >> 5) + w;
    if (i >= n) return;
    uint32_t *out = fwd + i * (int64_t)M;
    if (node_idx[i] < 0) {
        for (int j = lane; j < M; j += 32) out[j] = ESG_NONE;
        return;
    }
    Cand *pool = pool_s[w];
    int m = 0;
    // gather candidate ids (knn first, then sample), skipping self / invalid / repeats
    for (int src = 0; src < 2; ++src) {
        const int64_t *ids = src == 0 ? knn_ids + i * (int64_t)K : smp_ids + i * (int64_t)Ks;
        const int cnt = src == 0 ? K : Ks;
        for (int b0 = 0; b0 < cnt; b0 += 32) {
            int j = b0 + lane;
            int64_t id = j < cnt ? ids[j] : -1;
            bool ok = id >= 0 && id != i;
            if (ok) {
                for (int t = 0; t < m; ++t) if (pool[t].id == (uint32_t)id) { ok = false; break; }
            }
            // repeats within this chunk
            unsigned bal = __ballot_sync(0xffffffffu, ok);
            for (int o = 0; o < 32; ++o) {
                int64_t other = __shfl_sync(0xffffffffu, id, o);
                if (o < lane && ((bal >> o) & 1) && other == id) ok = false;
            }
            bal = __ballot_sync(0xffffffffu, ok);
            if (ok && m + __popc(bal & ((1u << lane) - 1)) < kMaxPool)
                pool[m + __popc(bal & ((1u << lane) - 1))] = Cand{0.f, (uint32_t)id};
            m = min(m + __popc(bal), kMaxPool);
            __syncwarp();
        }
    }
    // exact distances to u = i
    for (int t = 0; t < m; ++t) {
        float dd = row_dist(X, d, metric, (uint32_t)i, pool[t].id);
        if (lane == 0) pool[t].d = dd;
    }
    __syncwarp();
    // sort pool ascending
    {
        const int P = next_pow2_int(max(m, 2));
        for (int j = m + lane; j < P; j += 32) pool[j] = Cand{INFINITY, ESG_NONE};
        __syncwarp();
        warp_sort_pow2(pool, P);
    }
    int kept = occlusion_select(X, d, metric, pool, m, M, keep_s[w]);
    for (int j = lane; j < M; j += 32) {
        uint32_t v = j < kept ? keep_s[w][j] : ESG_NONE;
        out[j] = v;
        if (v != ESG_NONE) atomicAdd(&indeg[v], 1);
    }
}

__global__ void scatter_reverse_kernel(int64_t n, int M, const uint32_t *fwd, const int64_t *off,
                                       int32_t *cursor, uint32_t *rev) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    for (int j = 0; j < M; ++j) {
        uint32_t v = fwd[i * (int64_t)M + j];
        if (v == ESG_NONE) break;
        int pos = atomicAdd(&cursor[v], 1);
        rev[off[v] + pos] = (uint32_t)i;
    }
}

// Final row of point u: forward edges plus reverse edges; when more than R,
// re-select by occlusion among the 2R closest.
__global__ void final_row_kernel(const float *X, int64_t n, int d, int metric, const int32_t *node_idx,
                                 int M, int R, const uint32_t *fwd, const int64_t *off,
                                 const int32_t *indeg, const uint32_t *rev, uint32_t *adj_depth) {
    __shared__ Cand pool_s[4][2 * kMaxPool];  // cap + 32 rounded up to a power of two
    __shared__ uint32_t keep_s[4][kMaxRow];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    int64_t u = blockIdx.x * (int64_t)(blockDim.x >> 5) + w;
    if (u >= n) return;
    uint32_t *row = adj_depth + u * (int64_t)R;
    if (node_idx[u] < 0) {
        for (int j = lane; j < R; j += 32) row[j] = ESG_NONE;
        return;
    }
    Cand *pool = pool_s[w];
    const int cap = 2 * R <= kMaxPool ? 2 * R : kMaxPool;
    int m = 0;  // sorted, unique, at most cap
    const int nf = M;
    const int64_t nr = indeg[u];
    const int64_t total = nf + nr;
    for (int64_t b0 = 0; b0 < total; b0 += 32) {
        int64_t j = b0 + lane;
        uint32_t id = ESG_NONE;
        if (j < nf) id = fwd[u * (int64_t)M + j];
        else if (j < total) id = rev[off[u] + (j - nf)];
        float dd = INFINITY;
        // distances: one warp-wide reduction per candidate of the chunk
        for (int o = 0; o < 32; ++o) {
            uint32_t c = __shfl_sync(0xffffffffu, id, o);
            if (c == ESG_NONE) continue;
            float t = row_dist(X, d, metric, (uint32_t)u, c);
            if (lane == o) dd = t;
        }
        // drop ids already pooled
        bool ok = id != ESG_NONE;
        if (ok) for (int t = 0; t < m; ++t) if (pool[t].id == id) { ok = false; break; }
        unsigned bal = __ballot_sync(0xffffffffu, ok);
        for (int o = 0; o < 32; ++o) {
            uint32_t other = __shfl_sync(0xffffffffu, id, o);
            if (o < lane && ((bal >> o) & 1) && other == id) ok = false;
        }
        bal = __ballot_sync(0xffffffffu, ok);
        int c = __popc(bal);
        if (c == 0) continue;
        // append, sort, then keep the `cap` closest
        if (ok) pool[m + __popc(bal & ((1u << lane) - 1))] = Cand{dd, id};
        __syncwarp();
        {
            const int mm = m + c;
            const int P = next_pow2_int(max(mm, 2));
            for (int j = mm + lane; j < P; j += 32) pool[j] = Cand{INFINITY, ESG_NONE};
            __syncwarp();
            warp_sort_pow2(pool, P);
        }
        m = min(m + c, cap);
    }
    int kept;
    if (m <= R) {
        kept = m;
        for (int j = lane; j < m; j += 32) keep_s[w][j] = pool[j].id;
        __syncwarp();
    } else {
        kept = occlusion_select(X, d, metric, pool, m, R, keep_s[w]);
    }
    for (int j = lane; j < R; j += 32) row[j] = j < kept ? keep_s[w][j] : ESG_NONE;
}

}  // namespace

int esg_graph_depths(int64_t n, int32_t leaf_size) {
    // every node of a depth has size floor or ceil of n / 2^t; the depth
    // holds a graph node iff its largest node is wider than the leaf size
    int L = 0;
    int64_t big = n;  // size of the largest node at depth L
    while (big - 1 >= leaf_size) {
        ++L;
        big = (big + 1) / 2;
    }
    return L;
}

namespace {
struct HostNode { int64_t l, r; int32_t heap; };

void nodes_at_depth(int64_t n, int32_t leaf, int depth, std::vector<HostNode> &out) {
    out.clear();
    std::vector<HostNode> cur{{0, n - 1, 0}};
    for (int t = 0; t < depth; ++t) {
        std::vector<HostNode> nxt;
        for (auto &nd : cur) {
            if (nd.r - nd.l < leaf) continue;
            int64_t mid = nd.l + (nd.r - nd.l) / 2;
            nxt.push_back({nd.l, mid, 2 * nd.heap + 1});
            nxt.push_back({mid + 1, nd.r, 2 * nd.heap + 2});
        }
        cur.swap(nxt);
    }
    for (auto &nd : cur) out.push_back(nd);
}
}  // namespace

esg_status esg_build_graphs(esg_index *ix, const esg_build_params &p, cudaStream_t stream) {
    const int64_t n = ix->n;
    const int d = ix->d;
    const int L = ix->L, R = ix->R, M = p.M, E = ix->E;
    const int K = std::min(p.knn_k, kMaxPool);
    const int Ks = std::min(p.sample_k, kMaxPool - K);
    const int S = std::max(1, p.sample_size);
    if (L == 0) return ESG_OK;

    std::vector<int32_t> entries_h((size_t)ix->n_heap * E, -1);
    int64_t *lo = nullptr, *hi = nullptr, *knn = nullptr, *smp = nullptr, *s_rows = nullptr;
    int64_t *s_off_d = nullptr, *s_cnt_d = nullptr, *off = nullptr;
    int32_t *node_idx = nullptr, *cnt = nullptr, *indeg = nullptr, *cursor = nullptr;
    float *dist = nullptr, *xnorm = nullptr, *S_mat = nullptr, *snorm = nullptr;
    uint32_t *fwd = nullptr, *rev = nullptr;
    void *cub_tmp = nullptr;
    size_t cub_bytes = 0;
    esg_status st = ESG_OK;
#define B_TRY(expr) do { cudaError_t _e = (expr); if (_e != cudaSuccess) { esg_set_error(std::string(#expr) + ": " + cudaGetErrorString(_e)); st = _e == cudaErrorMemoryAllocation ? ESG_ERR_OOM : ESG_ERR_CUDA; goto done; } } while (0)
    {
    B_TRY(cudaMalloc(&lo, sizeof(int64_t) * n));
    B_TRY(cudaMalloc(&hi, sizeof(int64_t) * n));
    B_TRY(cudaMalloc(&node_idx, sizeof(int32_t) * n));
    B_TRY(cudaMalloc(&knn, sizeof(int64_t) * n * std::max(K, 1)));
    B_TRY(cudaMalloc(&smp, sizeof(int64_t) * n * std::max(Ks, 1)));
    B_TRY(cudaMalloc(&dist, sizeof(float) * n * std::max(std::max(K, Ks), 1)));
    B_TRY(cudaMalloc(&cnt, sizeof(int32_t) * n));
    B_TRY(cudaMalloc(&xnorm, sizeof(float) * n));
    B_TRY(cudaMalloc(&fwd, sizeof(uint32_t) * n * M));
    B_TRY(cudaMalloc(&indeg, sizeof(int32_t) * (n + 1)));
    B_TRY(cudaMalloc(&cursor, sizeof(int32_t) * n));
    B_TRY(cudaMalloc(&off, sizeof(int64_t) * (n + 1)));
    B_TRY(cudaMalloc(&rev, sizeof(uint32_t) * n * M));
    row_norms_kernel<<<ceil_div_i(n, 256), 256, 0, stream>>>(ix->X, n, d, xnorm);
    B_TRY(cudaGetLastError());
    B_TRY(cub::DeviceScan::ExclusiveSum(nullptr, cub_bytes, (int32_t *)nullptr, (int64_t *)nullptr, (int)(n + 1)));
    B_TRY(cudaMalloc(&cub_tmp, cub_bytes));
    const int mode = ix->metric == ESG_IP ? 1 : 2;
    std::vector<HostNode> nodes;
    for (int t = 0; t < L; ++t) {
        point_node_kernel<<<ceil_div_i(n, 256), 256, 0, stream>>>(n, ix->leaf_size, t, lo, hi, node_idx);
        B_TRY(cudaGetLastError());
        // exact knn_k nearest inside the node
        if (K > 0) {
            st = esg_launch_bruteforce_mode(mode, ix->X, n, d, ix->X, n, lo, hi, K, knn, dist, cnt,
                                            nullptr, 1, xnorm, xnorm, stream);
            if (st != ESG_OK) goto done;
        }
        // sample of each graph node at this depth
        nodes_at_depth(n, ix->leaf_size, t, nodes);
        std::vector<int64_t> s_off(nodes.size(), 0), s_cnt(nodes.size(), 0), rows;
        for (size_t j = 0; j < nodes.size(); ++j) {
            const HostNode &nd = nodes[j];
            const int64_t size = nd.r - nd.l + 1;
            // entry points of this node: E ranks evenly spaced
            if (nd.r - nd.l >= ix->leaf_size) {
                int ce = (int)std::min<int64_t>(E, size);
                for (int e = 0; e < ce; ++e)
                    entries_h[(size_t)nd.heap * E + e] = (int32_t)(nd.l + (int64_t)e * size / ce);
                int64_t cs = std::min<int64_t>(S, size);
                s_off[j] = (int64_t)rows.size();
                s_cnt[j] = cs;
                for (int64_t e = 0; e < cs; ++e) rows.push_back(nd.l + e * size / cs);
            }
        }
        if (Ks > 0 && !rows.empty()) {
            int64_t ns = (int64_t)rows.size();
            B_TRY(cudaMalloc(&s_rows, sizeof(int64_t) * ns));
            B_TRY(cudaMalloc(&S_mat, sizeof(float) * ns * d));
            B_TRY(cudaMalloc(&snorm, sizeof(float) * ns));
            B_TRY(cudaMalloc(&s_off_d, sizeof(int64_t) * nodes.size()));
            B_TRY(cudaMalloc(&s_cnt_d, sizeof(int64_t) * nodes.size()));
            B_TRY(cudaMemcpyAsync(s_rows, rows.data(), sizeof(int64_t) * ns, cudaMemcpyHostToDevice, stream));
            B_TRY(cudaMemcpyAsync(s_off_d, s_off.data(), sizeof(int64_t) * nodes.size(), cudaMemcpyHostToDevice, stream));
            B_TRY(cudaMemcpyAsync(s_cnt_d, s_cnt.data(), sizeof(int64_t) * nodes.size(), cudaMemcpyHostToDevice, stream));
            gather_rows_kernel<<<(unsigned)ns, 128, 0, stream>>>(ix->X, d, s_rows, ns, S_mat);
            B_TRY(cudaGetLastError());
            row_norms_kernel<<<ceil_div_i(ns, 256), 256, 0, stream>>>(S_mat, ns, d, snorm);
            B_TRY(cudaGetLastError());
            // per-point range = its node's sample block (node index at this depth)
            sample_range_kernel<<<ceil_div_i(n, 256), 256, 0, stream>>>(n, node_idx, s_off_d, s_cnt_d, lo, hi);
            B_TRY(cudaGetLastError());
            st = esg_launch_bruteforce_mode(mode, S_mat, ns, d, ix->X, n, lo, hi, Ks, smp, dist, cnt,
                                            s_rows, 0, snorm, xnorm, stream);
            if (st != ESG_OK) goto done;
            B_TRY(cudaStreamSynchronize(stream));
            cudaFree(s_rows); cudaFree(S_mat); cudaFree(snorm); cudaFree(s_off_d); cudaFree(s_cnt_d);
            s_rows = nullptr; S_mat = nullptr; snorm = nullptr; s_off_d = nullptr; s_cnt_d = nullptr;
        } else {
            B_TRY(cudaMemsetAsync(smp, 0xFF, sizeof(int64_t) * n * std::max(Ks, 1), stream));
        }
        // forward edges by occlusion, then reverse edges
        B_TRY(cudaMemsetAsync(indeg, 0, sizeof(int32_t) * (n + 1), stream));
        B_TRY(cudaMemsetAsync(cursor, 0, sizeof(int32_t) * n, stream));
        forward_kernel<<<ceil_div_i(n, 4), 128, 0, stream>>>(ix->X, n, d, ix->metric, node_idx, knn, K,
                                                               smp, Ks, M, fwd, indeg);
        B_TRY(cudaGetLastError());
        B_TRY(cub::DeviceScan::ExclusiveSum(cub_tmp, cub_bytes, indeg, off, (int)(n + 1), stream));
        scatter_reverse_kernel<<<ceil_div_i(n, 256), 256, 0, stream>>>(n, M, fwd, off, cursor, rev);
        B_TRY(cudaGetLastError());
        final_row_kernel<<<ceil_div_i(n, 4), 128, 0, stream>>>(
            ix->X, n, d, ix->metric, node_idx, M, R, fwd, off, indeg, rev,
            ix->adj + (size_t)t * (size_t)n * (size_t)R);
        B_TRY(cudaGetLastError());
        B_TRY(cudaStreamSynchronize(stream));
    }
    B_TRY(cudaMemcpyAsync(ix->entries, entries_h.data(), sizeof(int32_t) * entries_h.size(),
                          cudaMemcpyHostToDevice, stream));
    B_TRY(cudaStreamSynchronize(stream));
    }
done:
#undef B_TRY
    cudaFree(lo); cudaFree(hi); cudaFree(node_idx); cudaFree(knn); cudaFree(smp); cudaFree(dist);
    cudaFree(cnt); cudaFree(xnorm); cudaFree(fwd); cudaFree(indeg); cudaFree(cursor); cudaFree(off);
    cudaFree(rev); cudaFree(cub_tmp); cudaFree(s_rows); cudaFree(S_mat); cudaFree(snorm);
    cudaFree(s_off_d); cudaFree(s_cnt_d);
    return st;
}

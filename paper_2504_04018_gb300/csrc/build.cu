// GPU construction of the ESG index: Build-2D-Index (Algorithm 3).
//
// The tree: root [0, N-1], children [l, mid] and [mid+1, r] with
// mid = floor((l + r) / 2), no graph when r - l < leaf_size. A graph node's
// graph is the left child's graph (copied: the child keeps its own) with the
// points mid+1..r inserted in increasing rank order; when the left child is a
// leaf the graph is first built from scratch over [l, mid] by insertion.
// Insertion follows HNSW's flat layer: a beam search (ef = ef_construction)
// from the node's first point finds candidates, edge occlusion keeps at most
// M of them (keep c unless an already kept s has d(c, s) < d(c, u)), and each
// chosen neighbour gets the reverse edge, re-selecting its row by occlusion
// when it would exceed R = 2M.
//
// GPU schedule: depths are processed bottom-up; within a depth all nodes
// advance together. Points are inserted in rounds: a round inserts, for every
// node, the next max(1, inserted / batch_div) points of its rank order as one
// batch of independent searches (the warp beam-search kernel) over the graph
// as it stood before the round, then applies their forward edges and the
// reverse-edge updates. A batch never exceeds 1/batch_div of the graph it is
// inserted into, so points of a round miss only each other as candidates.
#include "esg_internal.cuh"

#include <algorithm>
#include <vector>

#include <cub/cub.cuh>

esg_status esg_run_search_items(const float *X, int64_t n, int d, int metric, const uint32_t *adj,
                                int R, const int32_t *entries, int E, const int64_t *qidx,
                                const esg_piece *pieces, int64_t n_items, int ef, int k,
                                int max_exp, Cand *res, int32_t *res_cnt, int32_t *res_status,
                                int64_t *res_stats, cudaStream_t stream);

namespace {

constexpr int kMaxPool = 256;   // candidates considered when re-selecting a row
constexpr int kMaxRow = 128;    // R

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

// Edge occlusion over pool[0..m) (ascending by distance to the base point,
// no duplicates, base excluded): keep c unless some kept s has
// d(c, s) < d(c, base). Returns the number kept (<= max_keep) in keep[].
__device__ int occlusion_select(const float *X, int d, int metric, const Cand *pool, int m,
                                int max_keep, uint32_t *keep) {
    int kept = 0;
    for (int i = 0; i < m && kept < max_keep; ++i) {
        const uint32_t c = pool[i].id & ESG_ID_MASK;
        const float dcb = pool[i].d;
        bool good = true;
        for (int s = 0; s < kept; ++s) {
            if (row_dist(X, d, metric, c, keep[s]) < dcb) { good = false; break; }
        }
        if (good) {
            if ((threadIdx.x & 31) == 0) keep[kept] = c;
            __syncwarp();
            ++kept;
        }
    }
    return kept;
}

// Forward edges of the inserted points: occlusion over each point's search
// result (already ascending), at most M; the point's row becomes those
// edges, padded with NONE. Counts the reverse edges each target receives.
__global__ void forward_kernel(const float *X, int d, int metric, int64_t n_items, const int64_t *pts,
                               const Cand *res, const int32_t *res_cnt, int efc, int M, int R,
                               uint32_t *adj_depth, int32_t *indeg) {
    __shared__ uint32_t keep_s[4][kMaxRow];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int64_t it = blockIdx.x * (int64_t)(blockDim.x >> 5) + w;
    if (it >= n_items) return;
    const int64_t p = pts[it];
    const Cand *pool = res + it * (int64_t)efc;
    const int m = res_cnt[it];
    int kept = occlusion_select(X, d, metric, pool, m, M, keep_s[w]);
    uint32_t *row = adj_depth + p * (int64_t)R;
    for (int j = lane; j < R; j += 32) {
        uint32_t v = j < kept ? keep_s[w][j] : ESG_NONE;
        row[j] = v;
        if (v != ESG_NONE) atomicAdd(&indeg[v], 1);
    }
}

__global__ void scatter_reverse_kernel(int64_t n_items, const int64_t *pts, int M, int R,
                                       const uint32_t *adj_depth, const int64_t *off,
                                       int32_t *cursor, uint32_t *rev) {
    int64_t it = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (it >= n_items) return;
    const int64_t p = pts[it];
    const uint32_t *row = adj_depth + p * (int64_t)R;
    for (int j = 0; j < M; ++j) {
        uint32_t v = row[j];
        if (v == ESG_NONE) break;
        int pos = atomicAdd(&cursor[v], 1);
        rev[off[v] + pos] = (uint32_t)p;
    }
}

// Reverse edges into point v: append the new sources to v's row; when the
// row would exceed R, re-select it by occlusion among the (at most
// kMaxPool) closest of old row + new sources.
__global__ void reverse_update_kernel(const float *X, int64_t n, int d, int metric, int R,
                                      const int64_t *off, const int32_t *indeg, const uint32_t *rev,
                                      uint32_t *adj_depth) {
    __shared__ Cand pool_s[4][2 * kMaxPool];
    __shared__ uint32_t keep_s[4][kMaxRow];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int64_t v = blockIdx.x * (int64_t)(blockDim.x >> 5) + w;
    if (v >= n) return;
    const int nr = indeg[v];
    if (nr == 0) return;
    uint32_t *row = adj_depth + v * (int64_t)R;
    int deg = 0;
    for (int b0 = 0; b0 < R; b0 += 32) {
        bool has = b0 + lane < R && row[b0 + lane] != ESG_NONE;
        deg += __popc(__ballot_sync(0xffffffffu, has));
    }
    const uint32_t *src = rev + off[v];
    if (deg + nr <= R) {
        for (int j = lane; j < nr; j += 32) row[deg + j] = src[j];
        return;
    }
    Cand *pool = pool_s[w];
    const int cap = kMaxPool;
    int m = 0;
    const int total = deg + nr;
    for (int b0 = 0; b0 < total; b0 += 32) {
        const int j = b0 + lane;
        uint32_t id = ESG_NONE;
        if (j < deg) id = row[j];
        else if (j < total) id = src[j - deg];
        float dd = INFINITY;
        for (int o = 0; o < 32; ++o) {
            uint32_t c = __shfl_sync(0xffffffffu, id, o);
            if (c == ESG_NONE) continue;
            float t = row_dist(X, d, metric, (uint32_t)v, c);
            if (lane == o) dd = t;
        }
        const bool ok = id != ESG_NONE;
        const unsigned bal = __ballot_sync(0xffffffffu, ok);
        const int c = __popc(bal);
        if (ok) pool[m + __popc(bal & ((1u << lane) - 1))] = Cand{dd, id};
        __syncwarp();
        const int mm = m + c;
        const int P = next_pow2_int(max(mm, 2));
        for (int t = mm + lane; t < P; t += 32) pool[t] = Cand{INFINITY, ESG_NONE};
        __syncwarp();
        warp_sort_pow2(pool, P);
        m = min(mm, cap);
    }
    const int kept = occlusion_select(X, d, metric, pool, m, R, keep_s[w]);
    for (int j = lane; j < R; j += 32) row[j] = j < kept ? keep_s[w][j] : ESG_NONE;
}

struct HostNode { int64_t l, r; int32_t heap; };

void nodes_at_depth(int64_t n, int32_t leaf, int depth, std::vector<HostNode> &out) {
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
    out.clear();
    for (auto &nd : cur) if (nd.r - nd.l >= leaf) out.push_back(nd);
}

}  // namespace

int esg_graph_depths(int64_t n, int32_t leaf_size) {
    // every node of a depth has size floor or ceil of n / 2^t; the depth
    // holds a graph node iff its largest node is wider than the leaf size
    int L = 0;
    int64_t big = n;
    while (big - 1 >= leaf_size) {
        ++L;
        big = (big + 1) / 2;
    }
    return L;
}

esg_status esg_build_graphs(esg_index *ix, const esg_build_params &p, cudaStream_t stream) {
    const int64_t n = ix->n;
    const int d = ix->d;
    const int L = ix->L, R = ix->R, M = p.M, E = ix->E;
    const int efc = std::max(p.ef_construction, M);
    const int div = std::max(1, p.batch_div);
    if (L == 0) return ESG_OK;

    std::vector<int32_t> entries_h((size_t)ix->n_heap * E, -1);
    std::vector<int32_t> build_entry((size_t)ix->n_heap, -1);
    int64_t *pts = nullptr, *off = nullptr, *stats = nullptr;
    esg_piece *pieces = nullptr;
    Cand *res = nullptr;
    int32_t *res_cnt = nullptr, *indeg = nullptr, *cursor = nullptr, *bentry = nullptr;
    uint32_t *rev = nullptr;
    void *cub_tmp = nullptr;
    size_t cub_bytes = 0;
    int64_t cap_items = 0;
    esg_status st = ESG_OK;
    std::vector<HostNode> nodes;
    std::vector<int64_t> h_pts;
    std::vector<esg_piece> h_pieces;
#define B_TRY(expr) do { cudaError_t _e = (expr); if (_e != cudaSuccess) { esg_set_error(std::string(#expr) + ": " + cudaGetErrorString(_e)); st = _e == cudaErrorMemoryAllocation ? ESG_ERR_OOM : ESG_ERR_CUDA; goto done; } } while (0)
    // largest round: one batch per node, at most size / div + 1 points each
    cap_items = n / div + ((int64_t)1 << (L - 1)) + 64;
    cap_items = std::min<int64_t>(cap_items, n);
    B_TRY(cudaMalloc(&pts, sizeof(int64_t) * cap_items));
    B_TRY(cudaMalloc(&pieces, sizeof(esg_piece) * cap_items));
    B_TRY(cudaMalloc(&res, sizeof(Cand) * cap_items * efc));
    B_TRY(cudaMalloc(&res_cnt, sizeof(int32_t) * cap_items * 2));
    B_TRY(cudaMalloc(&stats, sizeof(int64_t) * cap_items * ESG_ITEM_STATS));
    B_TRY(cudaMalloc(&indeg, sizeof(int32_t) * (n + 1)));
    B_TRY(cudaMalloc(&cursor, sizeof(int32_t) * n));
    B_TRY(cudaMalloc(&off, sizeof(int64_t) * (n + 1)));
    B_TRY(cudaMalloc(&rev, sizeof(uint32_t) * cap_items * M));
    B_TRY(cudaMalloc(&bentry, sizeof(int32_t) * ix->n_heap));
    B_TRY(cub::DeviceScan::ExclusiveSum(nullptr, cub_bytes, (int32_t *)nullptr, (int64_t *)nullptr, (int)(n + 1)));
    B_TRY(cudaMalloc(&cub_tmp, cub_bytes));
    B_TRY(cudaMemsetAsync(indeg, 0, sizeof(int32_t) * (n + 1), stream));
    for (int t = L - 1; t >= 0; --t) {
        nodes_at_depth(n, ix->leaf_size, t, nodes);
        uint32_t *adj_t = ix->adj + (size_t)t * (size_t)n * (size_t)R;
        std::vector<int64_t> inserted(nodes.size(), 0);
        for (size_t j = 0; j < nodes.size(); ++j) {
            const HostNode &nd = nodes[j];
            const int64_t mid = nd.l + (nd.r - nd.l) / 2;
            const int64_t size = nd.r - nd.l + 1;
            build_entry[nd.heap] = (int32_t)nd.l;  // insertion searches start at the first point
            int ce = (int)std::min<int64_t>(E, size);
            for (int e = 0; e < ce; ++e)
                entries_h[(size_t)nd.heap * E + e] = (int32_t)(nd.l + (int64_t)e * size / ce);
            if (mid - nd.l >= ix->leaf_size) {
                // the left child holds a graph: copy its rows (Algorithm 3, line 7 reading)
                B_TRY(cudaMemcpyAsync(adj_t + nd.l * (size_t)R, ix->adj + ((size_t)(t + 1) * n + nd.l) * R,
                                      sizeof(uint32_t) * (size_t)(mid - nd.l + 1) * R,
                                      cudaMemcpyDeviceToDevice, stream));
                inserted[j] = mid - nd.l + 1;
            } else {
                inserted[j] = 1;  // first point of a fresh graph: no edges
            }
        }
        B_TRY(cudaMemcpyAsync(bentry, build_entry.data(), sizeof(int32_t) * ix->n_heap,
                              cudaMemcpyHostToDevice, stream));
        for (;;) {
            h_pts.clear();
            h_pieces.clear();
            for (size_t j = 0; j < nodes.size(); ++j) {
                const HostNode &nd = nodes[j];
                const int64_t size = nd.r - nd.l + 1;
                if (inserted[j] >= size) continue;
                int64_t b = std::max<int64_t>(1, inserted[j] / div);
                b = std::min(b, size - inserted[j]);
                for (int64_t q = 0; q < b; ++q) {
                    h_pts.push_back(nd.l + inserted[j] + q);
                    esg_piece pc;
                    pc.node_l = nd.l; pc.node_r = nd.r; pc.pl = nd.l; pc.pr = nd.r;
                    pc.heap = nd.heap; pc.depth = t; pc.kind = ESG_PIECE_GRAPH; pc.reserved = 0;
                    h_pieces.push_back(pc);
                }
                inserted[j] += b;
            }
            const int64_t ni = (int64_t)h_pts.size();
            if (ni == 0) break;
            if (ni > cap_items) { esg_set_error("build: round larger than its buffers"); st = ESG_ERR_CUDA; goto done; }
            B_TRY(cudaMemcpyAsync(pts, h_pts.data(), sizeof(int64_t) * ni, cudaMemcpyHostToDevice, stream));
            B_TRY(cudaMemcpyAsync(pieces, h_pieces.data(), sizeof(esg_piece) * ni, cudaMemcpyHostToDevice, stream));
            st = esg_run_search_items(ix->X, n, d, ix->metric, ix->adj, R, bentry, 1, pts, pieces, ni,
                                      efc, efc, 0, res, res_cnt, res_cnt + cap_items, stats, stream);
            if (st != ESG_OK) goto done;
            B_TRY(cudaMemsetAsync(cursor, 0, sizeof(int32_t) * n, stream));
            forward_kernel<<<ceil_div_i(ni, 4), 128, 0, stream>>>(ix->X, d, ix->metric, ni, pts, res, res_cnt,
                                                                 efc, M, R, adj_t, indeg);
            B_TRY(cudaGetLastError());
            B_TRY(cub::DeviceScan::ExclusiveSum(cub_tmp, cub_bytes, indeg, off, (int)(n + 1), stream));
            scatter_reverse_kernel<<<ceil_div_i(ni, 256), 256, 0, stream>>>(ni, pts, M, R, adj_t, off, cursor, rev);
            B_TRY(cudaGetLastError());
            reverse_update_kernel<<<ceil_div_i(n, 4), 128, 0, stream>>>(ix->X, n, d, ix->metric, R, off,
                                                                        indeg, rev, adj_t);
            B_TRY(cudaGetLastError());
            B_TRY(cudaMemsetAsync(indeg, 0, sizeof(int32_t) * (n + 1), stream));
            B_TRY(cudaStreamSynchronize(stream));
        }
    }
    B_TRY(cudaMemcpyAsync(ix->entries, entries_h.data(), sizeof(int32_t) * entries_h.size(),
                          cudaMemcpyHostToDevice, stream));
    B_TRY(cudaStreamSynchronize(stream));
done:
#undef B_TRY
    cudaFree(pts); cudaFree(pieces); cudaFree(res); cudaFree(res_cnt); cudaFree(stats);
    cudaFree(indeg); cudaFree(cursor); cudaFree(off); cudaFree(rev); cudaFree(bentry);
    cudaFree(cub_tmp);
    return st;
}

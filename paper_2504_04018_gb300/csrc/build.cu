// GPU construction of the ESG index: Build-2D-Index (Algorithm 3) for the
// segment tree of fanout f, and Build-1D-Index (Algorithm 2) for the prefix
// graphs of the half-bounded layout.
//
// Tree: root [0, N-1]; the children of [l, r] are [b_j, b_{j+1} - 1] with
// b_j = l + ceil(j len / f) (f = 2: [l, mid], [mid+1, r]); no graph when
// r - l < leaf_size. A graph node's graph is its first child's graph (copied:
// the child keeps its own) with the node's other points inserted in
// increasing rank order; when the first child is a leaf the graph is first
// built from scratch over it by insertion.
// Prefix layout: one graph grown by inserting ranks 0, 1, ..., N-1, copied
// out whenever it holds n_i = floor(N / B^i) points (Algorithm 2's snapshots).
// Insertion follows HNSW's flat layer: a beam search (ef = ef_construction)
// from the graph's first point finds candidates, edge occlusion keeps at most
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
// Prefix rounds also stop at every snapshot size.
#include "esg_internal.cuh"
#include "decompose.cuh"

#include <algorithm>
#include <vector>

#include <cub/cub.cuh>

esg_status esg_run_search_items(const float *X, int64_t n, int d, int metric, const uint32_t *adj,
                                const int64_t *row_off, int R, const int32_t *entries, int E,
                                const int64_t *qidx, const esg_piece *pieces, int64_t n_items, int ef,
                                int k, int max_exp, Cand *res, int32_t *res_cnt, int32_t *res_status,
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

// Graph nodes (r - l >= leaf) at `depth` of the fanout-f tree over [0, n-1].
void nodes_at_depth(int64_t n, int32_t leaf, int32_t f, int depth, std::vector<HostNode> &out) {
    std::vector<HostNode> cur{{0, n - 1, 0}};
    for (int t = 0; t < depth; ++t) {
        std::vector<HostNode> nxt;
        for (auto &nd : cur) {
            if (nd.r - nd.l < leaf) continue;
            const int64_t len = nd.r - nd.l + 1;
            for (int j = 0; j < f; ++j) {
                const int64_t a = esg_child_lo(nd.l, len, f, j), b = esg_child_lo(nd.l, len, f, j + 1) - 1;
                if (a <= b) nxt.push_back({a, b, f * nd.heap + 1 + j});
            }
        }
        cur.swap(nxt);
    }
    out.clear();
    for (auto &nd : cur) if (nd.r - nd.l >= leaf) out.push_back(nd);
}

// Buffers of the insertion rounds (one batch of concurrent insertions).
struct Rounds {
    int64_t *pts = nullptr, *off = nullptr, *stats = nullptr;
    esg_piece *pieces = nullptr;
    Cand *res = nullptr;
    int32_t *res_cnt = nullptr, *indeg = nullptr, *cursor = nullptr, *bentry = nullptr;
    uint32_t *rev = nullptr;
    void *cub_tmp = nullptr;
    size_t cub_bytes = 0;
    int64_t cap = 0;
    ~Rounds() {
        cudaFree(pts); cudaFree(pieces); cudaFree(res); cudaFree(res_cnt); cudaFree(stats);
        cudaFree(indeg); cudaFree(cursor); cudaFree(off); cudaFree(rev); cudaFree(bentry);
        cudaFree(cub_tmp);
    }
};

#define B_TRY(expr) do { cudaError_t _e = (expr); if (_e != cudaSuccess) { esg_set_error(std::string(#expr) + ": " + cudaGetErrorString(_e)); return _e == cudaErrorMemoryAllocation ? ESG_ERR_OOM : ESG_ERR_CUDA; } } while (0)

esg_status rounds_alloc(Rounds &B, const esg_index *ix, int64_t cap, int efc, int M) {
    const int64_t n = ix->n;
    B.cap = cap;
    B_TRY(esg_malloc((void **)&B.pts, sizeof(int64_t) * cap));
    B_TRY(esg_malloc((void **)&B.pieces, sizeof(esg_piece) * cap));
    B_TRY(esg_malloc((void **)&B.res, sizeof(Cand) * cap * efc));
    B_TRY(esg_malloc((void **)&B.res_cnt, sizeof(int32_t) * cap * 2));
    B_TRY(esg_malloc((void **)&B.stats, sizeof(int64_t) * cap * ESG_ITEM_STATS));
    B_TRY(esg_malloc((void **)&B.indeg, sizeof(int32_t) * (n + 1)));
    B_TRY(esg_malloc((void **)&B.cursor, sizeof(int32_t) * n));
    B_TRY(esg_malloc((void **)&B.off, sizeof(int64_t) * (n + 1)));
    B_TRY(esg_malloc((void **)&B.rev, sizeof(uint32_t) * cap * M));
    B_TRY(esg_malloc((void **)&B.bentry, sizeof(int32_t) * std::max<int64_t>(ix->n_heap, 1)));
    B_TRY(cub::DeviceScan::ExclusiveSum(nullptr, B.cub_bytes, (int32_t *)nullptr, (int64_t *)nullptr, (int)(n + 1)));
    B_TRY(esg_malloc((void **)&B.cub_tmp, B.cub_bytes));
    B_TRY(cudaMemset(B.indeg, 0, sizeof(int32_t) * (n + 1)));
    return ESG_OK;
}

// One insertion round: the points h_pts (each into the graph of its piece,
// all at graph level `level`) searched concurrently on the graph as it stood
// before the round, then their forward edges and the reverse-edge updates.
esg_status insert_round(esg_index *ix, const esg_build_params &p, Rounds &B, int level,
                        const std::vector<int64_t> &h_pts, const std::vector<esg_piece> &h_pieces,
                        cudaStream_t stream) {
    const int64_t n = ix->n, ni = (int64_t)h_pts.size();
    const int R = ix->R, M = p.M, d = ix->d;
    const int efc = std::max(p.ef_construction, M);
    if (ni > B.cap) { esg_set_error("build: round larger than its buffers"); return ESG_ERR_CUDA; }
    uint32_t *adj_t = ix->adj + (size_t)ix->level_off[level] * R;
    B_TRY(cudaMemcpyAsync(B.pts, h_pts.data(), sizeof(int64_t) * ni, cudaMemcpyHostToDevice, stream));
    B_TRY(cudaMemcpyAsync(B.pieces, h_pieces.data(), sizeof(esg_piece) * ni, cudaMemcpyHostToDevice, stream));
    esg_status st = esg_run_search_items(ix->X, n, d, ix->metric, ix->adj, ix->row_off, R, B.bentry, 1, B.pts,
                                         B.pieces, ni, efc, efc, 0, B.res, B.res_cnt, B.res_cnt + B.cap,
                                         B.stats, stream);
    if (st != ESG_OK) return st;
    B_TRY(cudaMemsetAsync(B.cursor, 0, sizeof(int32_t) * n, stream));
    forward_kernel<<<ceil_div_i(ni, 4), 128, 0, stream>>>(ix->X, d, ix->metric, ni, B.pts, B.res, B.res_cnt,
                                                         efc, M, R, adj_t, B.indeg);
    B_TRY(cudaGetLastError());
    B_TRY(cub::DeviceScan::ExclusiveSum(B.cub_tmp, B.cub_bytes, B.indeg, B.off, (int)(n + 1), stream));
    scatter_reverse_kernel<<<ceil_div_i(ni, 256), 256, 0, stream>>>(ni, B.pts, M, R, adj_t, B.off, B.cursor, B.rev);
    B_TRY(cudaGetLastError());
    reverse_update_kernel<<<ceil_div_i(n, 4), 128, 0, stream>>>(ix->X, n, d, ix->metric, R, B.off,
                                                                B.indeg, B.rev, adj_t);
    B_TRY(cudaGetLastError());
    B_TRY(cudaMemsetAsync(B.indeg, 0, sizeof(int32_t) * (n + 1), stream));
    B_TRY(cudaStreamSynchronize(stream));
    return ESG_OK;
}

esg_piece whole_piece(int64_t l, int64_t r, int32_t heap, int32_t level) {
    esg_piece pc;
    pc.node_l = l; pc.node_r = r; pc.pl = l; pc.pr = r;
    pc.heap = heap; pc.depth = level; pc.kind = ESG_PIECE_GRAPH; pc.reserved = 0;
    return pc;
}

// Entry points of a graph node: E ranks evenly spaced over [l, r].
void set_entries(std::vector<int32_t> &ent, int E, int64_t h, int64_t l, int64_t r) {
    const int64_t size = r - l + 1;
    const int ce = (int)std::min<int64_t>(E, size);
    for (int e = 0; e < ce; ++e) ent[(size_t)h * E + e] = (int32_t)(l + (int64_t)e * size / ce);
}

// Build-2D-Index (Algorithm 3), fanout f: depths bottom-up, all nodes of a
// depth together; a node copies its first child's rows when that child holds
// a graph (else starts from its first point) and inserts the rest in rounds.
esg_status build_tree(esg_index *ix, const esg_build_params &p, Rounds &B, std::vector<int32_t> &entries_h,
                      cudaStream_t stream) {
    const int64_t n = ix->n;
    const int L = ix->L, R = ix->R, f = ix->fanout;
    const int div = std::max(1, p.batch_div);
    std::vector<int32_t> build_entry((size_t)ix->n_heap, -1);
    std::vector<HostNode> nodes;
    std::vector<int64_t> h_pts;
    std::vector<esg_piece> h_pieces;
    for (int t = L - 1; t >= 0; --t) {
        nodes_at_depth(n, ix->leaf_size, f, t, nodes);
        uint32_t *adj_t = ix->adj + (size_t)ix->level_off[t] * R;
        std::vector<int64_t> inserted(nodes.size(), 0);
        for (size_t j = 0; j < nodes.size(); ++j) {
            const HostNode &nd = nodes[j];
            const int64_t b1 = esg_child_lo(nd.l, nd.r - nd.l + 1, f, 1);   // first child [l, b1 - 1]
            build_entry[nd.heap] = (int32_t)nd.l;  // insertion searches start at the first point
            set_entries(entries_h, ix->E, nd.heap, nd.l, nd.r);
            if (b1 - 1 - nd.l >= ix->leaf_size) {
                // the first child holds a graph: copy its rows (Algorithm 3, copy-then-insert)
                B_TRY(cudaMemcpyAsync(adj_t + nd.l * (size_t)R, ix->adj + ((size_t)ix->level_off[t + 1] + nd.l) * R,
                                      sizeof(uint32_t) * (size_t)(b1 - nd.l) * R, cudaMemcpyDeviceToDevice, stream));
                inserted[j] = b1 - nd.l;
            } else {
                inserted[j] = 1;  // first point of a fresh graph: no edges
            }
        }
        B_TRY(cudaMemcpyAsync(B.bentry, build_entry.data(), sizeof(int32_t) * ix->n_heap,
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
                    h_pieces.push_back(whole_piece(nd.l, nd.r, nd.heap, t));
                }
                inserted[j] += b;
            }
            if (h_pts.empty()) break;
            esg_status st = insert_round(ix, p, B, t, h_pts, h_pieces, stream);
            if (st != ESG_OK) return st;
        }
    }
    return ESG_OK;
}

// Build-1D-Index (Algorithm 2), base B: one graph grown at level 0 (the whole
// set) by inserting ranks 0, 1, ... in rounds that stop at each prefix size
// n_i = floor(n / B^i); when it holds exactly n_i points its rows 0..n_i-1
// are copied to level i (snapshot).
esg_status build_prefix(esg_index *ix, const esg_build_params &p, Rounds &B, std::vector<int32_t> &entries_h,
                        cudaStream_t stream) {
    const int L = ix->L, R = ix->R;
    const int div = std::max(1, p.batch_div);
    std::vector<int32_t> build_entry((size_t)ix->n_heap, 0);
    for (int i = 0; i < L; ++i) set_entries(entries_h, ix->E, i, 0, ix->level_rows[i] - 1);
    B_TRY(cudaMemcpyAsync(B.bentry, build_entry.data(), sizeof(int32_t) * ix->n_heap, cudaMemcpyHostToDevice, stream));
    std::vector<int64_t> h_pts;
    std::vector<esg_piece> h_pieces;
    int64_t inserted = 1;                  // rank 0: no edges
    int lev = L - 1;                       // next snapshot: the smallest prefix
    for (;;) {
        while (lev >= 1 && inserted == ix->level_rows[lev]) {
            B_TRY(cudaMemcpyAsync(ix->adj + (size_t)ix->level_off[lev] * R, ix->adj,
                                  sizeof(uint32_t) * (size_t)ix->level_rows[lev] * R, cudaMemcpyDeviceToDevice,
                                  stream));
            --lev;
        }
        if (inserted >= ix->n) break;
        const int64_t stop = lev >= 1 ? ix->level_rows[lev] : ix->n;
        int64_t b = std::max<int64_t>(1, inserted / div);
        b = std::min(b, stop - inserted);
        h_pts.clear();
        h_pieces.clear();
        for (int64_t q = 0; q < b; ++q) {
            h_pts.push_back(inserted + q);
            h_pieces.push_back(whole_piece(0, ix->n - 1, 0, 0));
        }
        esg_status st = insert_round(ix, p, B, 0, h_pts, h_pieces, stream);
        if (st != ESG_OK) return st;
        inserted += b;
    }
    B_TRY(cudaStreamSynchronize(stream));
    return ESG_OK;
}

}  // namespace

int esg_graph_depths(int64_t n, int32_t leaf_size, int32_t layout, int32_t fanout) {
    int L = 0;
    if (layout == ESG_LAYOUT_PREFIX) {
        for (int64_t m = n; m >= 1; m /= fanout) ++L;
        return L;
    }
    // every node of depth t has at most ceil(n / f^t) points and the first
    // node that size; the depth holds a graph node iff that size exceeds the
    // leaf size
    int64_t big = n;
    while (big - 1 >= leaf_size) {
        ++L;
        big = (big + fanout - 1) / fanout;
    }
    return L;
}

esg_status esg_set_layout(esg_index *ix) {
    const int f = ix->fanout;
    if (f < 2 || f > 16 || (ix->layout != ESG_LAYOUT_TREE && ix->layout != ESG_LAYOUT_PREFIX)) {
        esg_set_error("layout must be tree or prefix, fanout 2..16");
        return ESG_ERR_INVALID_ARG;
    }
    ix->L = esg_graph_depths(ix->n, ix->leaf_size, ix->layout, f);
    ix->level_off.assign(ix->L, 0);
    ix->level_rows.assign(ix->L, 0);
    int64_t rows = 0;
    if (ix->layout == ESG_LAYOUT_PREFIX) {
        int64_t m = ix->n;
        for (int i = 0; i < ix->L; ++i) { ix->level_off[i] = rows; ix->level_rows[i] = m; rows += m; m /= f; }
        ix->n_heap = ix->L;
    } else {
        int64_t nodes = 0, w = 1;
        for (int t = 0; t < ix->L; ++t) {
            ix->level_off[t] = rows; ix->level_rows[t] = ix->n; rows += ix->n;
            nodes += w;
            if (nodes > ((int64_t)1 << 31) / (2 * f)) {
                esg_set_error("tree too deep for int32 node numbers (raise leaf_size)");
                return ESG_ERR_UNSUPPORTED;
            }
            w *= f;
        }
        ix->n_heap = nodes;
    }
    ix->adj_rows = rows;
    return ESG_OK;
}

esg_status esg_build_graphs(esg_index *ix, const esg_build_params &p, cudaStream_t stream) {
    if (ix->L == 0) return ESG_OK;
    const int efc = std::max(p.ef_construction, p.M);
    const int div = std::max(1, p.batch_div);
    // largest round: one batch per node, at most size / div + 1 points each
    int64_t nodes_deepest = 1;
    for (int t = 1; t < ix->L && ix->layout == ESG_LAYOUT_TREE; ++t) nodes_deepest *= ix->fanout;
    const int64_t cap = std::min<int64_t>(ix->n, ix->n / div + std::min<int64_t>(nodes_deepest, ix->n) + 64);
    Rounds B;
    esg_status st = rounds_alloc(B, ix, cap, efc, p.M);
    if (st != ESG_OK) return st;
    std::vector<int32_t> entries_h((size_t)ix->n_heap * ix->E, -1);
    st = ix->layout == ESG_LAYOUT_PREFIX ? build_prefix(ix, p, B, entries_h, stream)
                                         : build_tree(ix, p, B, entries_h, stream);
    if (st != ESG_OK) return st;
    B_TRY(cudaMemcpyAsync(ix->entries, entries_h.data(), sizeof(int32_t) * entries_h.size(),
                          cudaMemcpyHostToDevice, stream));
    B_TRY(cudaStreamSynchronize(stream));
    return ESG_OK;
}
#undef B_TRY

// Internal declarations shared by the translation units of libesg.
#pragma once

#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <cuda_fp8.h>
#include <stdint.h>
#include <string>
#include <vector>

#include "../../include/esg.h"

#define ESG_NONE 0xFFFFFFFFu
#define ESG_MLP_FEATURES 9
// classes of k (floor(log2 k), capped) with their own beam-width margin
#define ESG_MLP_KBUCKETS 12
// per-item search statistics: expansions, evaluations, out-of-range
// evaluations, re-ranked rows, start and end time (ns, %globaltimer)
#define ESG_ITEM_STATS 6
// per-query statistics returned by esg_search_batch (see esg.h)
#define ESG_QUERY_STATS 6

// Largest search batch: the (query, piece) items of a batch (two per query)
// are numbered with int32 in the processing order.
constexpr int64_t kMaxBatch = (int64_t)1 << 30;
#define ESG_EXPANDED 0x80000000u
#define ESG_ID_MASK 0x7FFFFFFFu

// ----------------------------------------------------------------- errors

void esg_set_error(const std::string &msg);

// Every device allocation of the library goes through these. They carry the
// host-side fault injection of the failure-detection tests: with the
// environment variable ESG_FAULT_ALLOC=K (K >= 1), the K-th allocation the
// library attempts after that value was set fails as if the device were out
// of memory (no GPU fault is involved).
bool esg_fault_alloc();
inline cudaError_t esg_malloc(void **p, size_t bytes) {
    if (esg_fault_alloc()) { *p = nullptr; return cudaErrorMemoryAllocation; }
    return cudaMalloc(p, bytes);
}
// Stream-ordered scratch comes from the library's own memory pool on the
// current device, which keeps up to ESG_POOL_KEEP_MB (default 8192) MiB of
// freed memory mapped between calls (the default pool returns it at every
// synchronisation, and mapping hundreds of MB again costs a call a fraction
// of a millisecond); null if the pool could not be made (then the default pool).
cudaMemPool_t esg_scratch_pool();
inline cudaError_t esg_malloc_async(void **p, size_t bytes, cudaStream_t stream) {
    if (esg_fault_alloc()) { *p = nullptr; return cudaErrorMemoryAllocation; }
    cudaMemPool_t pool = esg_scratch_pool();
    return pool ? cudaMallocFromPoolAsync(p, bytes, pool, stream) : cudaMallocAsync(p, bytes, stream);
}

#define ESG_CUDA_TRY(expr)                                                                 \
    do {                                                                                   \
        cudaError_t _e = (expr);                                                           \
        if (_e != cudaSuccess) {                                                           \
            esg_set_error(std::string(#expr) + ": " + cudaGetErrorString(_e));            \
            return _e == cudaErrorMemoryAllocation ? ESG_ERR_OOM : ESG_ERR_CUDA;           \
        }                                                                                  \
    } while (0)

// ------------------------------------------------------------------ index

struct esg_index {
    int64_t n = 0;
    int32_t d = 0;
    int32_t metric = 0;
    int32_t storage = 0;
    int32_t leaf_size = 0;
    int32_t layout = ESG_LAYOUT_TREE;
    int32_t fanout = 2;      // tree fanout f, or the prefix layout's base B
    int32_t L = 0;           // graph levels: depths holding graph nodes, or prefix graphs
    int32_t R = 0;           // row width of the adjacency
    int32_t E = 0;           // entry points per node
    int32_t M = 0;
    int64_t n_heap = 0;      // graph nodes with entries: (f^L - 1) / (f - 1), or L
    int64_t adj_rows = 0;    // rows of adj over all levels
    std::vector<int64_t> level_off;   // first adj row of each level (rank i of level t: row level_off[t] + i)
    std::vector<int64_t> level_rows;  // ranks 0..level_rows[t] - 1 have rows at level t
    int64_t *row_off = nullptr;       // level_off on the device
    int device = 0;
    float *X = nullptr;              // [n, d] fp32, rank order
    __nv_bfloat16 *Xb = nullptr;     // [n, d] bf16 (storage BF16)
    __nv_fp8_e4m3 *X8 = nullptr;     // [n, d] fp8 (storage FP8)
    float *scale8 = nullptr;         // [n] per-row fp8 scale
    uint32_t *adj = nullptr;         // [adj_rows, R]
    int32_t *entries = nullptr;      // [n_heap, E]
    int64_t *perm = nullptr;         // [n] rank -> original id (device)
    std::vector<int64_t> perm_host;  // same on the host
    std::vector<double> attr_sorted; // sorted attribute values (host), may be empty
    // learned beam-width predictor: [params, mu, sigma, margins] on the
    // device and the host; null / 0 when untrained
    float *mlp = nullptr;
    std::vector<float> mlp_host;
    int32_t mlp_ready = 0;
    int32_t mlp_ef_lo = 8, mlp_ef_hi = 128;
};

// Number of graph levels: depths of the fanout-f tree that hold at least
// one graph node, or prefix graphs floor(n / B^i) >= 1 of the prefix layout.
int esg_graph_depths(int64_t n, int32_t leaf_size, int32_t layout, int32_t fanout);
// Fill the layout fields of `ix` (L, n_heap, adj_rows, level_off,
// level_rows) from n, leaf_size, layout and fanout; ESG_ERR_UNSUPPORTED when
// the node table would not fit int32 node numbers.
esg_status esg_set_layout(esg_index *ix);

// What a search decomposes its query ranges by (see decompose.cuh).
struct DecomposeSpec {
    int64_t n;
    int32_t leaf;       // leaf size of the tree layout
    int32_t fanout;     // tree fanout f, or prefix base B
    int32_t layout;     // esg_layout
    int32_t post_root;  // 1: one piece on the root graph
};
inline DecomposeSpec esg_spec_of(const esg_index *ix, int post_root) {
    return DecomposeSpec{ix->n, ix->leaf_size, ix->fanout, ix->layout, post_root};
}

// --------------------------------------------------------- launch helpers

struct SearchLaunch {
    const esg_index *ix;
    const float *queries;
    int64_t nq;
    const int64_t *l, *r;
    const int32_t *k;
    int32_t k_max;
    esg_search_params p;
    int64_t *out_ids;
    float *out_dist;
    int32_t *out_count;
    int32_t *out_status;
    int64_t *out_stats;
};

// Range checks of esg_search_params shared by every batched search entry
// point (sets the error message, prefixed with `who`).
esg_status esg_check_search_params(const esg_search_params &p, const char *who);

esg_status esg_launch_decompose(const DecomposeSpec &spec, const int64_t *l, const int64_t *r,
                                int64_t nq, esg_piece *pieces, int32_t *npieces,
                                cudaStream_t stream);
esg_status esg_launch_search(const SearchLaunch &s, cudaStream_t stream);

// One launch of the beam-search kernel: kernel, shape, shared memory.
struct KernelPlan {
    void *fn;
    int vpl, lpr, C, H, G, wpb, nvec, width, BB, efk, lpe;
    size_t smem;
    int64_t grid;
};
// Largest per-query beam width (max(ef, k)) of the small budget class; 0 =
// one class (the default: with lists of 2 ef items the widest plans still
// reach the register-bound occupancy, and a second launch adds a tail; the
// environment variable ESG_SMALL_CLASS_EF sets it).
constexpr int kSmallClassEf = 0;
// Launch plan of one search call. The queries may be split into two budget
// classes by max(ef_q, k): class 0 (at most kSmallClassEf) and class 1, each
// searched by its own launch whose lists and visited tables are sized for
// that class, so that the narrow beams of most queries are not run at the
// occupancy of the widest one.
struct SearchPlan {
    const void *Xt;       // traversal rows
    int ef, efk;
    bool learned;         // per-query ef and expansion budget from the predictor
    int nclass;           // 1: every query in cls[0]; 2: cls[0] small, cls[1] large
    int small_ef;         // class bound when nclass == 2, else 0
    KernelPlan cls[2];
    int64_t n_items;
    size_t scratch_bytes;
};
// Validate and plan a search; scratch_bytes tells how much device scratch
// esg_search_enqueue needs.
esg_status esg_search_prepare(const SearchLaunch &s, SearchPlan &plan);
// As esg_search_prepare, but shrink the persistent grid (fewer concurrent
// warps; results do not depend on it) until the scratch fits in max_scratch
// bytes. ESG_ERR_INVALID_ARG if it cannot fit even with one block.
esg_status esg_search_prepare_capped(const SearchLaunch &s, size_t max_scratch, SearchPlan &plan);
// Enqueue the search on `stream` using caller-provided scratch (no allocation).
esg_status esg_search_enqueue(const SearchLaunch &s, const SearchPlan &plan, void *scratch,
                              cudaStream_t stream);
esg_status esg_launch_bruteforce(const float *base, int64_t n, int32_t d, int metric,
                                 const float *queries, int64_t nq, const int64_t *l,
                                 const int64_t *r, int32_t k, int64_t *out_ids, float *out_dist,
                                 int32_t *out_count, const int64_t *id_map, int32_t exclude_self,
                                 cudaStream_t stream);
esg_status esg_build_graphs(esg_index *ix, const esg_build_params &p, cudaStream_t stream);
esg_status esg_make_storage(esg_index *ix, cudaStream_t stream);

// learned predictor (mlp.cu): features + per-query ef and expansion budget
int esg_mlp_param_count();
// floats of the predictor blob: params, mu, sigma, the ef and expansion
// margins, one ef margin offset per class of k
inline int esg_mlp_blob_floats() { return esg_mlp_param_count() + 2 * ESG_MLP_FEATURES + 2 + ESG_MLP_KBUCKETS; }
__host__ __device__ inline int esg_k_bucket(int k) {
    int b = 0;
    while (b + 1 < ESG_MLP_KBUCKETS && (k >> (b + 1)) > 0) ++b;   // floor(log2 k), capped
    return b;
}
esg_status esg_predict_budget(const esg_index *ix, int post_root, const float *queries, int64_t nq, const int64_t *l,
                              const int64_t *r, const int32_t *k, int32_t k_max, int ef_fixed,
                              float *feat, int32_t *ef_q, int32_t *maxexp_q, cudaStream_t stream);
// per-query hits of returned ids against exact ids (batch.cu)
esg_status esg_recall_hits(int64_t nq, int32_t k_max, const int32_t *k, const int64_t *ids, const int32_t *cnt,
                           const int64_t *gt, const int32_t *gcnt, int32_t *hits, cudaStream_t stream);

// benchmark timing hooks (profile.cu)
bool esg_prof_on();
void esg_prof_count(int64_t launches);
void esg_prof_tensor_flops(double flops);
int esg_prof_begin(cudaStream_t stream);
void esg_prof_end(int idx, cudaStream_t stream);

// --------------------------------------------------------- device helpers

struct Cand {
    float d;
    uint32_t id;  // bit 31: expanded flag (search lists only)
};

__device__ __forceinline__ bool cand_less(float da, uint32_t ia, float db, uint32_t ib) {
    return da < db || (da == db && (ia & ESG_ID_MASK) < (ib & ESG_ID_MASK));
}
__device__ __forceinline__ bool cand_less(const Cand &a, const Cand &b) {
    return cand_less(a.d, a.id, b.d, b.id);
}
__device__ __forceinline__ bool cand_eq(const Cand &a, const Cand &b) {
    return a.d == b.d && (a.id & ESG_ID_MASK) == (b.id & ESG_ID_MASK);
}

// Bitonic sort of 64 candidates in shared memory by one warp (ascending).
__device__ __forceinline__ void warp_sort64(Cand *v) {
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int size = 2; size <= 64; size <<= 1) {
#pragma unroll
        for (int stride = size >> 1; stride > 0; stride >>= 1) {
            // each lane owns one compare-exchange pair of the 32 pairs
            int i = 2 * stride * (lane / stride) + (lane % stride);
            int j = i + stride;
            bool up = ((i & size) == 0);
            Cand a = v[i], b = v[j];
            bool swap = up ? cand_less(b, a) : cand_less(a, b);
            __syncwarp();
            if (swap) { v[i] = b; v[j] = a; }
            __syncwarp();
        }
    }
}

// Bitonic sort of one candidate per lane across the warp (ascending by lane),
// in registers with shuffles.
__device__ __forceinline__ void warp_sort32_reg(float &d, uint32_t &id) {
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int size = 2; size <= 32; size <<= 1) {
#pragma unroll
        for (int stride = size >> 1; stride > 0; stride >>= 1) {
            const float od = __shfl_xor_sync(0xffffffffu, d, stride);
            const uint32_t oid = __shfl_xor_sync(0xffffffffu, id, stride);
            const bool lower = (lane & stride) == 0;        // I keep the smaller if ascending
            const bool up = (lane & size) == 0;
            const bool other_less = cand_less(od, oid, d, id);
            const bool take = (lower == up) ? other_less : !other_less && !(od == d && oid == id);
            if (take) { d = od; id = oid; }
        }
    }
}

// Bitonic sort of P (a power of two, <= 1024) candidates in shared memory by
// one warp (ascending); pad unused slots with {+inf, ESG_NONE} first.
__device__ __forceinline__ void warp_sort_pow2(Cand *v, int P) {
    const int lane = threadIdx.x & 31;
    for (int size = 2; size <= P; size <<= 1) {
        for (int stride = size >> 1; stride > 0; stride >>= 1) {
            for (int p = lane; p < P / 2; p += 32) {
                int i = 2 * stride * (p / stride) + (p % stride);
                int j = i + stride;
                bool up = ((i & size) == 0);
                Cand a = v[i], b = v[j];
                bool swap = up ? cand_less(b, a) : cand_less(a, b);
                if (swap) { v[i] = b; v[j] = a; }
            }
            __syncwarp();
        }
    }
}

__device__ __forceinline__ int next_pow2_int(int x) {
    int p = 1;
    while (p < x) p <<= 1;
    return p;
}

// Number of items of sorted list `v[0..n)` strictly less than `x`.
__device__ __forceinline__ int lower_rank(const Cand *v, int n, const Cand &x) {
    int lo = 0, hi = n;
    while (lo < hi) {
        int mid = (lo + hi) >> 1;
        if (cand_less(v[mid], x)) lo = mid + 1; else hi = mid;
    }
    return lo;
}

__device__ __forceinline__ float warp_sum_group(float v, int group) {
    for (int off = group >> 1; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
    return v;
}

static inline int ceil_div_i(int64_t a, int64_t b) { return (int)((a + b - 1) / b); }

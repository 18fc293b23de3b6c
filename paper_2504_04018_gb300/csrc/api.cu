// C ABI entry points of libesg (declared in include/esg.h): argument checks,
// index lifetime, re-ranking, save/load, and dispatch to the kernels.
#include "esg_internal.cuh"

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <numeric>
#include <string>
#include <vector>

namespace {
thread_local std::string g_last_error;

template <typename T>
esg_status dev_alloc(T **p, size_t count) {
    *p = nullptr;
    if (count == 0) return ESG_OK;
    cudaError_t e = esg_malloc((void **)p, sizeof(T) * count);
    if (e != cudaSuccess) {
        esg_set_error(std::string("cudaMalloc: ") + cudaGetErrorString(e));
        *p = nullptr;
        return ESG_ERR_OOM;
    }
    return ESG_OK;
}

void free_index_memory(esg_index *ix) {
    if (!ix) return;
    cudaFree(ix->X); cudaFree(ix->Xb); cudaFree(ix->X8); cudaFree(ix->scale8);
    cudaFree(ix->adj); cudaFree(ix->entries); cudaFree(ix->perm); cudaFree(ix->mlp);
    cudaFree(ix->row_off);
    ix->X = nullptr; ix->Xb = nullptr; ix->X8 = nullptr; ix->scale8 = nullptr;
    ix->adj = nullptr; ix->entries = nullptr; ix->perm = nullptr; ix->mlp = nullptr;
    ix->row_off = nullptr;
}

bool dim_ok(int32_t d) { return d >= 4 && d <= 1024 && d % 4 == 0; }

// Common tail of build/import/load: allocate device arrays for the shape
// (esg_set_layout first) and copy the level offsets.
esg_status alloc_index(esg_index *ix) {
    esg_status s;
    if ((s = dev_alloc(&ix->X, (size_t)ix->n * ix->d)) != ESG_OK) return s;
    if ((s = dev_alloc(&ix->adj, (size_t)ix->adj_rows * ix->R)) != ESG_OK) return s;
    if ((s = dev_alloc(&ix->entries, (size_t)ix->n_heap * ix->E)) != ESG_OK) return s;
    if ((s = dev_alloc(&ix->perm, (size_t)ix->n)) != ESG_OK) return s;
    if ((s = dev_alloc(&ix->row_off, (size_t)std::max(ix->L, 1))) != ESG_OK) return s;
    if (ix->L > 0)
        ESG_CUDA_TRY(cudaMemcpy(ix->row_off, ix->level_off.data(), sizeof(int64_t) * ix->L, cudaMemcpyHostToDevice));
    return ESG_OK;
}

uint32_t crc32_update(uint32_t crc, const void *data, size_t len) {
    static uint32_t table[256];
    static bool init = false;
    if (!init) {
        for (uint32_t i = 0; i < 256; ++i) {
            uint32_t c = i;
            for (int k = 0; k < 8; ++k) c = (c & 1) ? 0xEDB88320u ^ (c >> 1) : c >> 1;
            table[i] = c;
        }
        init = true;
    }
    const unsigned char *p = (const unsigned char *)data;
    crc = ~crc;
    for (size_t i = 0; i < len; ++i) crc = table[(crc ^ p[i]) & 0xFF] ^ (crc >> 8);
    return ~crc;
}
}  // namespace

void esg_set_error(const std::string &msg) { g_last_error = msg; }

cudaMemPool_t esg_scratch_pool() {
    static std::mutex mu;
    static cudaMemPool_t pools[64] = {};
    static bool tried[64] = {};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return nullptr;
    std::lock_guard<std::mutex> lock(mu);
    if (!tried[dev]) {
        tried[dev] = true;
        cudaMemPoolProps props = {};
        props.allocType = cudaMemAllocationTypePinned;
        props.handleTypes = cudaMemHandleTypeNone;
        props.location.type = cudaMemLocationTypeDevice;
        props.location.id = dev;
        cudaMemPool_t pool = nullptr;
        if (cudaMemPoolCreate(&pool, &props) == cudaSuccess) {
            const char *keep = getenv("ESG_POOL_KEEP_MB");
            const long long mb = keep && *keep ? atoll(keep) : 8192;
            uint64_t bytes = (uint64_t)(mb > 0 ? mb : 0) << 20;
            cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &bytes);
            pools[dev] = pool;
        } else {
            cudaGetLastError();   // clear it: the default pool serves instead
        }
    }
    return pools[dev];
}

bool esg_fault_alloc() {
    static std::mutex mu;
    static std::string seen;
    static long long count = 0;
    const char *v = getenv("ESG_FAULT_ALLOC");
    const std::string cur = v ? v : "";
    std::lock_guard<std::mutex> lk(mu);
    if (cur != seen) { seen = cur; count = 0; }   // a new value starts a new count
    if (cur.empty()) return false;
    const long long k = atoll(cur.c_str());
    return k >= 1 && ++count == k;
}

esg_status esg_check_search_params(const esg_search_params &p, const char *who) {
    if (p.ef < 1 || p.ef > 1024 || p.max_expansions < 0 || p.width < 0 || p.width > 4 ||
        !(p.warps_per_block == 0 || p.warps_per_block == 1 || p.warps_per_block == 2 ||
          p.warps_per_block == 4) ||
        (p.hash_slots != 0 && (p.hash_slots < 1024 || p.hash_slots > 16384 ||
                               (p.hash_slots & (p.hash_slots - 1)))) ||
        p.lanes_per_row < 0 || p.lanes_per_row > 32 || (p.lanes_per_row & (p.lanes_per_row - 1)) ||
        !(p.max_registers == 0 || p.max_registers == 96 || p.max_registers == 128) ||
        !(p.post_root == 0 || p.post_root == 1)) {
        esg_set_error(std::string(who) + ": search parameter out of range");
        return ESG_ERR_INVALID_ARG;
    }
    return ESG_OK;
}

extern "C" {

const char *esg_last_error(void) { return g_last_error.c_str(); }

const char *esg_status_str(esg_status s) {
    switch (s) {
        case ESG_OK: return "ok";
        case ESG_ERR_INVALID_ARG: return "invalid argument";
        case ESG_ERR_OOM: return "out of memory";
        case ESG_ERR_CUDA: return "CUDA error";
        case ESG_ERR_IO: return "I/O error";
        case ESG_ERR_CORRUPT: return "corrupt index file";
        case ESG_ERR_TIMEOUT: return "timeout";
        case ESG_ERR_UNSUPPORTED: return "unsupported";
    }
    return "unknown status";
}

esg_build_params esg_build_params_default(void) {
    esg_build_params p;
    p.M = 16;
    p.leaf_size = 256;
    p.n_entries = 16;
    p.ef_construction = 200;
    p.batch_div = 8;
    p.fanout = 2;
    p.metric = ESG_L2SQ;
    p.storage = ESG_F32;
    p.layout = ESG_LAYOUT_TREE;
    p.reserved = 0;
    return p;
}

esg_search_params esg_search_params_default(void) {
    esg_search_params p;
    p.ef = 64;
    p.max_expansions = 0;
    p.rerank = 1;
    p.use_learned = 0;
    p.traversal = ESG_F32;
    p.width = 1;
    p.warps_per_block = 0;
    p.hash_slots = 0;
    p.lanes_per_row = 0;
    p.post_root = 0;
    p.max_registers = 0;
    return p;
}

esg_train_params esg_train_params_default(void) {
    esg_train_params p;
    p.target_recall = 0.95f;
    p.per_query_recall = 1.0f;
    p.quantile = 0.9f;
    p.lr = 1e-3f;
    p.val_fraction = 0.2f;
    p.epochs = 60;
    p.batch = 1024;
    p.ef_lo = 8;
    p.ef_hi = 128;
    p.traversal = ESG_F32;
    p.per_k_class = 0;
    p.seed = 4005;
    return p;
}

esg_status esg_build(const float *vectors, int64_t n, int32_t d, const double *attr,
                     const esg_build_params *params, esg_index **out) {
    if (!out) { esg_set_error("out is NULL"); return ESG_ERR_INVALID_ARG; }
    *out = nullptr;
    if (!vectors || n < 1 || n >= ((int64_t)1 << 31) - 1 || !dim_ok(d) || d % 8 != 0) {
        esg_set_error("esg_build: need vectors != NULL, 1 <= n < 2^31-1, 8 <= d <= 1024, d % 8 == 0");
        return ESG_ERR_INVALID_ARG;
    }
    esg_build_params p = params ? *params : esg_build_params_default();
    if (p.fanout == 0) p.fanout = 2;
    if (p.M < 1 || 2 * p.M > 128 || p.leaf_size < 1 || p.n_entries < 1 || p.n_entries > 32 ||
        p.ef_construction < 1 || p.ef_construction > 1024 || p.batch_div < 1 ||
        p.fanout < 2 || p.fanout > 16 || (p.layout != ESG_LAYOUT_TREE && p.layout != ESG_LAYOUT_PREFIX) ||
        (p.metric != ESG_L2SQ && p.metric != ESG_IP) ||
        (p.storage != ESG_F32 && p.storage != ESG_BF16 && p.storage != ESG_FP8E4M3)) {
        esg_set_error("esg_build: parameter out of range");
        return ESG_ERR_INVALID_ARG;
    }
    if (attr) for (int64_t i = 0; i < n; ++i) if (std::isnan(attr[i])) {
        esg_set_error("esg_build: NaN attribute");
        return ESG_ERR_INVALID_ARG;
    }
    esg_index *ix = new (std::nothrow) esg_index();
    if (!ix) return ESG_ERR_OOM;
    ix->n = n; ix->d = d; ix->metric = p.metric; ix->storage = p.storage;
    ix->leaf_size = p.leaf_size; ix->M = p.M; ix->R = 2 * p.M; ix->E = p.n_entries;
    ix->layout = p.layout; ix->fanout = p.fanout;
    {
        esg_status ls = esg_set_layout(ix);
        if (ls != ESG_OK) { delete ix; return ls; }
    }
    cudaGetDevice(&ix->device);
    // re-ranking: rank i = i-th smallest attribute, ties by row
    ix->perm_host.resize(n);
    std::iota(ix->perm_host.begin(), ix->perm_host.end(), (int64_t)0);
    if (attr) {
        std::stable_sort(ix->perm_host.begin(), ix->perm_host.end(),
                         [attr](int64_t a, int64_t b) { return attr[a] < attr[b]; });
        ix->attr_sorted.resize(n);
        for (int64_t i = 0; i < n; ++i) ix->attr_sorted[i] = attr[ix->perm_host[i]];
    }
    esg_status s = alloc_index(ix);
    cudaStream_t stream = nullptr;
    std::vector<float> ranked;
    if (s == ESG_OK && cudaStreamCreateWithFlags(&stream, cudaStreamNonBlocking) != cudaSuccess) {
        esg_set_error("cudaStreamCreate failed"); s = ESG_ERR_CUDA;
    }
    if (s == ESG_OK) {
        try {
            ranked.resize((size_t)n * d);
        } catch (...) { s = ESG_ERR_OOM; }
    }
    if (s == ESG_OK) {
        for (int64_t i = 0; i < n; ++i)
            std::memcpy(&ranked[(size_t)i * d], vectors + (size_t)ix->perm_host[i] * d, sizeof(float) * d);
        cudaError_t e = cudaMemcpyAsync(ix->X, ranked.data(), sizeof(float) * n * d, cudaMemcpyHostToDevice, stream);
        if (e == cudaSuccess) e = cudaMemcpyAsync(ix->perm, ix->perm_host.data(), sizeof(int64_t) * n, cudaMemcpyHostToDevice, stream);
        if (e == cudaSuccess && ix->L > 0) e = cudaMemsetAsync(ix->adj, 0xFF, sizeof(uint32_t) * ix->adj_rows * ix->R, stream);
        if (e == cudaSuccess && ix->n_heap > 0) e = cudaMemsetAsync(ix->entries, 0xFF, sizeof(int32_t) * ix->n_heap * ix->E, stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(stream);
        if (e != cudaSuccess) { esg_set_error(cudaGetErrorString(e)); s = ESG_ERR_CUDA; }
    }
    if (s == ESG_OK) s = esg_build_graphs(ix, p, stream);
    if (s == ESG_OK) s = esg_make_storage(ix, stream);
    if (stream) cudaStreamDestroy(stream);
    if (s != ESG_OK) { free_index_memory(ix); delete ix; return s; }
    *out = ix;
    return ESG_OK;
}

esg_status esg_index_import(const float *vectors, const int64_t *perm, int64_t n, int32_t d,
                            esg_metric metric, int32_t leaf_size, esg_layout layout, int32_t fanout,
                            const uint32_t *adj, int32_t L, int32_t R, const int32_t *entries,
                            int32_t n_entries, esg_dtype storage, esg_index **out) {
    if (!out) { esg_set_error("out is NULL"); return ESG_ERR_INVALID_ARG; }
    *out = nullptr;
    if (!vectors || n < 1 || n >= ((int64_t)1 << 31) - 1 || !dim_ok(d) ||
        (layout == ESG_LAYOUT_TREE && leaf_size < 1) ||
        R < 1 || R > 128 || n_entries < 1 || n_entries > 32 || (L > 0 && (!adj || !entries)) ||
        (metric != ESG_L2SQ && metric != ESG_IP)) {
        esg_set_error("esg_index_import: argument out of range");
        return ESG_ERR_INVALID_ARG;
    }
    esg_index *ix = new (std::nothrow) esg_index();
    if (!ix) return ESG_ERR_OOM;
    // the prefix layout has no leaves; its leaf size is kept at 1
    ix->n = n; ix->d = d; ix->metric = metric; ix->storage = storage;
    ix->leaf_size = std::max<int32_t>(leaf_size, 1);
    ix->layout = layout; ix->fanout = fanout; ix->R = R; ix->M = R / 2; ix->E = n_entries;
    {
        esg_status ls = esg_set_layout(ix);
        if (ls == ESG_OK && L != ix->L) {
            esg_set_error("esg_index_import: L does not match (n, leaf_size, layout, fanout)");
            ls = ESG_ERR_INVALID_ARG;
        }
        // every id must name a row of its level, every entry a rank of its node's level
        for (int t = 0; ls == ESG_OK && t < ix->L; ++t) {
            const uint32_t *a = adj + (size_t)ix->level_off[t] * R;
            for (size_t i = 0; i < (size_t)ix->level_rows[t] * R; ++i)
                if (a[i] != ESG_NONE && (int64_t)a[i] >= ix->level_rows[t]) { ls = ESG_ERR_INVALID_ARG; break; }
        }
        for (int64_t h = 0; ls == ESG_OK && h < ix->n_heap; ++h) {
            const int64_t lim = layout == ESG_LAYOUT_PREFIX ? ix->level_rows[h] : n;
            for (int e = 0; e < n_entries; ++e)
                if (entries[h * n_entries + e] >= lim) { ls = ESG_ERR_INVALID_ARG; break; }
        }
        if (ls != ESG_OK) {
            if (ls == ESG_ERR_INVALID_ARG && L == ix->L)
                esg_set_error("esg_index_import: an adjacency id or entry lies outside its level");
            delete ix;
            return ls;
        }
    }
    cudaGetDevice(&ix->device);
    ix->perm_host.resize(n);
    if (perm) std::memcpy(ix->perm_host.data(), perm, sizeof(int64_t) * n);
    else std::iota(ix->perm_host.begin(), ix->perm_host.end(), (int64_t)0);
    esg_status s = alloc_index(ix);
    if (s == ESG_OK) {
        cudaError_t e = cudaMemcpy(ix->X, vectors, sizeof(float) * n * d, cudaMemcpyHostToDevice);
        if (e == cudaSuccess) e = cudaMemcpy(ix->perm, ix->perm_host.data(), sizeof(int64_t) * n, cudaMemcpyHostToDevice);
        if (e == cudaSuccess && L > 0) e = cudaMemcpy(ix->adj, adj, sizeof(uint32_t) * ix->adj_rows * R, cudaMemcpyHostToDevice);
        if (e == cudaSuccess && L > 0) e = cudaMemcpy(ix->entries, entries, sizeof(int32_t) * ix->n_heap * n_entries, cudaMemcpyHostToDevice);
        if (e != cudaSuccess) { esg_set_error(cudaGetErrorString(e)); s = ESG_ERR_CUDA; }
    }
    if (s == ESG_OK) s = esg_make_storage(ix, nullptr);
    if (s == ESG_OK && cudaDeviceSynchronize() != cudaSuccess) s = ESG_ERR_CUDA;
    if (s != ESG_OK) { free_index_memory(ix); delete ix; return s; }
    *out = ix;
    return ESG_OK;
}

esg_status esg_index_info(const esg_index *ix, int64_t *n, int32_t *d, int32_t *L, int32_t *R,
                          int32_t *n_entries, int32_t *leaf_size, int32_t *metric, int32_t *storage) {
    if (!ix) { esg_set_error("index is NULL"); return ESG_ERR_INVALID_ARG; }
    if (n) *n = ix->n;
    if (d) *d = ix->d;
    if (L) *L = ix->L;
    if (R) *R = ix->R;
    if (n_entries) *n_entries = ix->E;
    if (leaf_size) *leaf_size = ix->leaf_size;
    if (metric) *metric = ix->metric;
    if (storage) *storage = ix->storage;
    return ESG_OK;
}

esg_status esg_index_layout(const esg_index *ix, int32_t *layout, int32_t *fanout, int64_t *nodes,
                            int64_t *adj_rows) {
    if (!ix) { esg_set_error("index is NULL"); return ESG_ERR_INVALID_ARG; }
    if (layout) *layout = ix->layout;
    if (fanout) *fanout = ix->fanout;
    if (nodes) *nodes = ix->n_heap;
    if (adj_rows) *adj_rows = ix->adj_rows;
    return ESG_OK;
}

esg_status esg_index_export(const esg_index *ix, uint32_t *adj, int32_t *entries, int64_t *perm) {
    if (!ix) { esg_set_error("index is NULL"); return ESG_ERR_INVALID_ARG; }
    if (adj && ix->L > 0) ESG_CUDA_TRY(cudaMemcpy(adj, ix->adj, sizeof(uint32_t) * ix->adj_rows * ix->R, cudaMemcpyDeviceToHost));
    if (entries && ix->n_heap > 0) ESG_CUDA_TRY(cudaMemcpy(entries, ix->entries, sizeof(int32_t) * ix->n_heap * ix->E, cudaMemcpyDeviceToHost));
    if (perm) std::memcpy(perm, ix->perm_host.data(), sizeof(int64_t) * ix->n);
    return ESG_OK;
}

esg_status esg_index_export_rows(const esg_index *ix, int32_t level, int64_t row0, int64_t nrows,
                                 uint32_t *adj) {
    if (!ix || (!adj && nrows > 0) || level < 0 || level >= ix->L || row0 < 0 || nrows < 0 ||
        row0 + nrows > ix->level_rows[level]) {
        esg_set_error("esg_index_export_rows: bad argument");
        return ESG_ERR_INVALID_ARG;
    }
    if (nrows > 0)
        ESG_CUDA_TRY(cudaMemcpy(adj, ix->adj + ((size_t)ix->level_off[level] + row0) * ix->R,
                                sizeof(uint32_t) * nrows * ix->R, cudaMemcpyDeviceToHost));
    return ESG_OK;
}

esg_status esg_index_export_storage(const esg_index *ix, esg_dtype dtype, void *rows, float *scale) {
    if (!ix || !rows) { esg_set_error("esg_index_export_storage: bad argument"); return ESG_ERR_INVALID_ARG; }
    const size_t count = (size_t)ix->n * ix->d;
    if (dtype == ESG_BF16 && ix->Xb) {
        ESG_CUDA_TRY(cudaMemcpy(rows, ix->Xb, 2 * count, cudaMemcpyDeviceToHost));
    } else if (dtype == ESG_FP8E4M3 && ix->X8) {
        ESG_CUDA_TRY(cudaMemcpy(rows, ix->X8, count, cudaMemcpyDeviceToHost));
        if (scale) ESG_CUDA_TRY(cudaMemcpy(scale, ix->scale8, sizeof(float) * ix->n, cudaMemcpyDeviceToHost));
    } else {
        esg_set_error("esg_index_export_storage: index holds no rows of that type");
        return ESG_ERR_INVALID_ARG;
    }
    return ESG_OK;
}

esg_status esg_index_add_storage(esg_index *ix, esg_dtype dtype) {
    if (!ix || (dtype != ESG_BF16 && dtype != ESG_FP8E4M3)) {
        esg_set_error("esg_index_add_storage: bad argument");
        return ESG_ERR_INVALID_ARG;
    }
    if ((dtype == ESG_BF16 && ix->Xb) || (dtype == ESG_FP8E4M3 && ix->X8)) return ESG_OK;
    const int32_t keep = ix->storage;
    ix->storage = dtype;
    esg_status s = esg_make_storage(ix, nullptr);
    ix->storage = keep == ESG_F32 ? dtype : keep;
    return s;
}

void esg_free(esg_index *ix) {
    if (!ix) return;
    free_index_memory(ix);
    delete ix;
}

esg_status esg_decompose_batch(int64_t n, int32_t leaf_size, esg_layout layout, int32_t fanout,
                               int32_t post_root, const int64_t *l, const int64_t *r, int64_t nq,
                               esg_piece *out_pieces, int32_t *out_npieces, esg_stream_t stream) {
    if (n < 1 || leaf_size < 1 || nq < 0 || fanout < 2 || fanout > 16 ||
        (layout != ESG_LAYOUT_TREE && layout != ESG_LAYOUT_PREFIX) ||
        (nq > 0 && (!l || !r || !out_pieces || !out_npieces))) {
        esg_set_error("esg_decompose_batch: bad argument");
        return ESG_ERR_INVALID_ARG;
    }
    const DecomposeSpec spec{n, leaf_size, fanout, (int32_t)layout, post_root ? 1 : 0};
    return esg_launch_decompose(spec, l, r, nq, out_pieces, out_npieces, (cudaStream_t)stream);
}

esg_status esg_search_batch(const esg_index *ix, const float *queries, int64_t nq, const int64_t *l,
                            const int64_t *r, const int32_t *k, int32_t k_max,
                            const esg_search_params *params, int64_t *out_ids, float *out_dist,
                            int32_t *out_count, int32_t *out_status, int64_t *out_stats,
                            esg_stream_t stream) {
    if (!ix || nq < 0 || nq >= kMaxBatch || k_max < 1 || k_max > 1024 ||
        (nq > 0 && (!queries || !l || !r || !out_ids || !out_dist || !out_count))) {
        esg_set_error("esg_search_batch: bad argument");
        return ESG_ERR_INVALID_ARG;
    }
    if (((uintptr_t)queries) % 16 != 0) {
        esg_set_error("esg_search_batch: queries must be 16-byte aligned");
        return ESG_ERR_INVALID_ARG;
    }
    SearchLaunch s;
    s.ix = ix; s.queries = queries; s.nq = nq; s.l = l; s.r = r; s.k = k; s.k_max = k_max;
    s.p = params ? *params : esg_search_params_default();
    if (esg_check_search_params(s.p, "esg_search_batch") != ESG_OK) return ESG_ERR_INVALID_ARG;
    s.out_ids = out_ids; s.out_dist = out_dist; s.out_count = out_count;
    s.out_status = out_status; s.out_stats = out_stats;
    return esg_launch_search(s, (cudaStream_t)stream);
}

esg_status esg_bruteforce_filtered_knn(const float *base, int64_t n, int32_t d, esg_metric metric,
                                       const float *queries, int64_t nq, const int64_t *l,
                                       const int64_t *r, int32_t k, int64_t *out_ids,
                                       float *out_dist, int32_t *out_count, esg_stream_t stream) {
    if (n < 1 || n >= ((int64_t)1 << 31) - 1 || !dim_ok(d) || nq < 0 || k < 1 || k > 1024 ||
        (metric != ESG_L2SQ && metric != ESG_IP) ||
        (nq > 0 && (!base || !queries || !l || !r || !out_ids || !out_dist || !out_count))) {
        esg_set_error("esg_bruteforce_filtered_knn: bad argument");
        return ESG_ERR_INVALID_ARG;
    }
    if (((uintptr_t)base) % 16 != 0 || ((uintptr_t)queries) % 16 != 0) {
        esg_set_error("esg_bruteforce_filtered_knn: base and queries must be 16-byte aligned");
        return ESG_ERR_INVALID_ARG;
    }
    return esg_launch_bruteforce(base, n, d, metric, queries, nq, l, r, k, out_ids, out_dist,
                                 out_count, nullptr, 0, (cudaStream_t)stream);
}

esg_status esg_attr_to_rank_range(const esg_index *ix, const double *lo, const double *hi, int64_t nq,
                                  int64_t *l, int64_t *r) {
    if (!ix || nq < 0 || (nq > 0 && (!lo || !hi || !l || !r))) {
        esg_set_error("esg_attr_to_rank_range: bad argument");
        return ESG_ERR_INVALID_ARG;
    }
    for (int64_t i = 0; i < nq; ++i) {
        if (ix->attr_sorted.empty()) {
            // attribute = original row: ranks are rows
            double a = std::ceil(lo[i]), b = std::floor(hi[i]);
            int64_t la = (int64_t)std::max(0.0, a), rb = (int64_t)std::min((double)(ix->n - 1), b);
            l[i] = la; r[i] = rb;
            if (la > rb) { l[i] = rb + 1; }
        } else {
            const auto &A = ix->attr_sorted;
            int64_t la = std::lower_bound(A.begin(), A.end(), lo[i]) - A.begin();
            int64_t rb = (std::upper_bound(A.begin(), A.end(), hi[i]) - A.begin()) - 1;
            l[i] = la; r[i] = rb;
            if (la > rb) l[i] = rb + 1;
        }
    }
    return ESG_OK;
}

// ------------------------------------------------------------ save / load

namespace {
const char kMagic[8] = {'E', 'S', 'G', 'G', 'B', '3', '0', '0'};
const uint32_t kVersion = 5;

struct FileHeader {
    char magic[8];
    uint32_t version;
    int32_t d, metric, storage, leaf_size, L, R, E, M;
    int64_t n;
    int64_t n_heap;
    uint64_t attr_count;
    uint64_t mlp_count;       // floats of the learned predictor's blob (0: none)
    int32_t mlp_ef_lo, mlp_ef_hi;
    int32_t storage_mask;     // bit t: rows of esg_dtype t are held (low-precision copies are rebuilt on load)
    int32_t layout;           // esg_layout
    int32_t fanout;           // tree fanout or prefix base
    int32_t reserved;
    int64_t adj_rows;         // rows of the adjacency section
};

bool write_section(FILE *f, const void *data, size_t bytes) {
    uint64_t len = bytes;
    uint32_t crc = crc32_update(0, data, bytes);
    return fwrite(&len, 8, 1, f) == 1 && (bytes == 0 || fwrite(data, 1, bytes, f) == bytes) &&
           fwrite(&crc, 4, 1, f) == 1;
}

esg_status read_section(FILE *f, void *data, size_t bytes) {
    uint64_t len = 0;
    uint32_t crc = 0;
    if (fread(&len, 8, 1, f) != 1) return ESG_ERR_CORRUPT;
    if (len != bytes) return ESG_ERR_CORRUPT;
    if (bytes && fread(data, 1, bytes, f) != bytes) return ESG_ERR_CORRUPT;
    if (fread(&crc, 4, 1, f) != 1) return ESG_ERR_CORRUPT;
    if (crc != crc32_update(0, data, bytes)) return ESG_ERR_CORRUPT;
    return ESG_OK;
}
}  // namespace

esg_status esg_save(const esg_index *ix, const char *path) {
    if (!ix || !path) { esg_set_error("esg_save: bad argument"); return ESG_ERR_INVALID_ARG; }
    std::vector<float> X((size_t)ix->n * ix->d);
    std::vector<uint32_t> adj((size_t)ix->adj_rows * ix->R);
    std::vector<int32_t> ent((size_t)ix->n_heap * ix->E);
    ESG_CUDA_TRY(cudaMemcpy(X.data(), ix->X, sizeof(float) * X.size(), cudaMemcpyDeviceToHost));
    if (!adj.empty()) ESG_CUDA_TRY(cudaMemcpy(adj.data(), ix->adj, sizeof(uint32_t) * adj.size(), cudaMemcpyDeviceToHost));
    if (!ent.empty()) ESG_CUDA_TRY(cudaMemcpy(ent.data(), ix->entries, sizeof(int32_t) * ent.size(), cudaMemcpyDeviceToHost));
    FILE *f = fopen(path, "wb");
    if (!f) { esg_set_error(std::string("esg_save: cannot open ") + path); return ESG_ERR_IO; }
    FileHeader h;
    std::memset(&h, 0, sizeof(h));
    std::memcpy(h.magic, kMagic, 8);
    h.version = kVersion; h.d = ix->d; h.metric = ix->metric; h.storage = ix->storage;
    h.leaf_size = ix->leaf_size; h.L = ix->L; h.R = ix->R; h.E = ix->E; h.M = ix->M; h.n = ix->n;
    h.n_heap = ix->n_heap; h.attr_count = ix->attr_sorted.size();
    h.layout = ix->layout; h.fanout = ix->fanout; h.adj_rows = ix->adj_rows;
    h.mlp_count = ix->mlp_ready ? ix->mlp_host.size() : 0;
    h.mlp_ef_lo = ix->mlp_ef_lo; h.mlp_ef_hi = ix->mlp_ef_hi;
    h.storage_mask = (1 << ESG_F32) | (ix->Xb ? 1 << ESG_BF16 : 0) | (ix->X8 ? 1 << ESG_FP8E4M3 : 0);
    bool ok = write_section(f, &h, sizeof(h)) && write_section(f, X.data(), sizeof(float) * X.size()) &&
              write_section(f, ix->perm_host.data(), sizeof(int64_t) * ix->n) &&
              write_section(f, adj.data(), sizeof(uint32_t) * adj.size()) &&
              write_section(f, ent.data(), sizeof(int32_t) * ent.size()) &&
              write_section(f, ix->attr_sorted.data(), sizeof(double) * ix->attr_sorted.size()) &&
              write_section(f, ix->mlp_host.data(), sizeof(float) * h.mlp_count);
    ok = (fclose(f) == 0) && ok;
    if (!ok) { esg_set_error("esg_save: write failed"); return ESG_ERR_IO; }
    return ESG_OK;
}

esg_status esg_load(const char *path, esg_index **out) {
    if (!path || !out) { esg_set_error("esg_load: bad argument"); return ESG_ERR_INVALID_ARG; }
    *out = nullptr;
    FILE *f = fopen(path, "rb");
    if (!f) { esg_set_error(std::string("esg_load: cannot open ") + path); return ESG_ERR_IO; }
    FileHeader h;
    esg_status s = read_section(f, &h, sizeof(h));
    esg_index shape;   // the layout the header's parameters imply
    shape.n = h.n; shape.leaf_size = h.leaf_size; shape.layout = h.layout; shape.fanout = h.fanout;
    if (s == ESG_OK && (std::memcmp(h.magic, kMagic, 8) != 0 || h.version != kVersion || h.n < 1 ||
                        h.leaf_size < 1 || esg_set_layout(&shape) != ESG_OK))
        s = ESG_ERR_CORRUPT;
    if (s == ESG_OK && (!dim_ok(h.d) || h.R < 1 || h.R > 128 || h.E < 1 ||
                        h.E > 32 || h.n_heap != shape.n_heap || h.L != shape.L || h.adj_rows != shape.adj_rows ||
                        (h.attr_count != 0 && h.attr_count != (uint64_t)h.n) ||
                        (h.mlp_count != 0 && h.mlp_count != (uint64_t)esg_mlp_blob_floats())))
        s = ESG_ERR_CORRUPT;
    std::vector<float> X;
    std::vector<int64_t> perm;
    std::vector<uint32_t> adj;
    std::vector<int32_t> ent;
    std::vector<double> attr;
    std::vector<float> mlp;
    if (s == ESG_OK) {
        try {
            X.resize((size_t)h.n * h.d); perm.resize(h.n); adj.resize((size_t)h.adj_rows * h.R);
            ent.resize((size_t)h.n_heap * h.E); attr.resize(h.attr_count); mlp.resize(h.mlp_count);
        } catch (...) { s = ESG_ERR_OOM; }
    }
    if (s == ESG_OK) s = read_section(f, X.data(), sizeof(float) * X.size());
    if (s == ESG_OK) s = read_section(f, perm.data(), sizeof(int64_t) * perm.size());
    if (s == ESG_OK) s = read_section(f, adj.data(), sizeof(uint32_t) * adj.size());
    if (s == ESG_OK) s = read_section(f, ent.data(), sizeof(int32_t) * ent.size());
    if (s == ESG_OK) s = read_section(f, attr.data(), sizeof(double) * attr.size());
    if (s == ESG_OK) s = read_section(f, mlp.data(), sizeof(float) * mlp.size());
    fclose(f);
    if (s != ESG_OK) {
        if (s == ESG_ERR_CORRUPT) esg_set_error("esg_load: file is not a valid index (header, size or CRC)");
        return s;
    }
    esg_index *ix = nullptr;
    s = esg_index_import(X.data(), perm.data(), h.n, h.d, (esg_metric)h.metric, h.leaf_size,
                         (esg_layout)h.layout, h.fanout, adj.data(), h.L, h.R, ent.data(), h.E,
                         (esg_dtype)h.storage, &ix);
    if (s != ESG_OK) return s;
    ix->M = h.M;
    ix->attr_sorted.swap(attr);
    for (int t : {ESG_BF16, ESG_FP8E4M3}) {
        if (!(h.storage_mask & (1 << t))) continue;
        s = esg_index_add_storage(ix, (esg_dtype)t);
        if (s != ESG_OK) { esg_free(ix); return s; }
    }
    if (!mlp.empty()) {
        s = esg_predictor_set(ix, mlp.data(), h.mlp_ef_lo, h.mlp_ef_hi);
        if (s != ESG_OK) { esg_free(ix); return s; }
    }
    *out = ix;
    return ESG_OK;
}

}  // extern "C"

// Batched search replayed as one CUDA graph (esg_batch_*), and the
// autotuner (esg_autotune). Host runtime around the search kernels.
#include "esg_internal.cuh"

#include <algorithm>
#include <map>
#include <vector>

struct esg_batch {
    const esg_index *ix = nullptr;
    int64_t max_nq = 0;
    int32_t k_max = 0;
    int32_t use_k = 0;
    esg_search_params p;
    float *queries = nullptr;
    int64_t *l = nullptr, *r = nullptr;
    int32_t *k = nullptr;
    int64_t *ids = nullptr;
    float *dist = nullptr;
    int32_t *count = nullptr, *status = nullptr;
    int64_t *stats = nullptr;
    void *scratch = nullptr;
    size_t scratch_bytes = 0;
    cudaStream_t cap_stream = nullptr;
    std::map<int64_t, cudaGraphExec_t> graphs;
};

namespace {
SearchLaunch launch_for(const esg_batch *b, int64_t nq) {
    SearchLaunch s;
    s.ix = b->ix; s.queries = b->queries; s.nq = nq; s.l = b->l; s.r = b->r;
    s.k = b->use_k ? b->k : nullptr; s.k_max = b->k_max; s.p = b->p;
    s.out_ids = b->ids; s.out_dist = b->dist; s.out_count = b->count;
    s.out_status = b->status; s.out_stats = b->stats;
    return s;
}

void release(esg_batch *b) {
    for (auto &kv : b->graphs) cudaGraphExecDestroy(kv.second);
    b->graphs.clear();
    cudaFree(b->queries); cudaFree(b->l); cudaFree(b->r); cudaFree(b->k); cudaFree(b->ids);
    cudaFree(b->dist); cudaFree(b->count); cudaFree(b->status); cudaFree(b->stats);
    cudaFree(b->scratch);
    if (b->cap_stream) cudaStreamDestroy(b->cap_stream);
}
}  // namespace

extern "C" {

esg_status esg_batch_create(const esg_index *ix, int64_t max_nq, int32_t k_max, int32_t use_k,
                            const esg_search_params *params, esg_batch **out) {
    if (!out) { esg_set_error("out is NULL"); return ESG_ERR_INVALID_ARG; }
    *out = nullptr;
    if (!ix || max_nq < 1 || max_nq >= kMaxBatch || k_max < 1 || k_max > 1024) {
        esg_set_error("esg_batch_create: bad argument");
        return ESG_ERR_INVALID_ARG;
    }
    if (params && esg_check_search_params(*params, "esg_batch_create") != ESG_OK) return ESG_ERR_INVALID_ARG;
    esg_batch *b = new (std::nothrow) esg_batch();
    if (!b) return ESG_ERR_OOM;
    b->ix = ix; b->max_nq = max_nq; b->k_max = k_max; b->use_k = use_k;
    b->p = params ? *params : esg_search_params_default();
    esg_status st = ESG_OK;
    auto A = [&](void **p, size_t bytes) {
        if (st != ESG_OK) return;
        cudaError_t e = esg_malloc((void **)p, bytes);
        if (e != cudaSuccess) { esg_set_error(cudaGetErrorString(e)); st = ESG_ERR_OOM; }
    };
    A((void **)&b->queries, sizeof(float) * max_nq * ix->d);
    A((void **)&b->l, sizeof(int64_t) * max_nq);
    A((void **)&b->r, sizeof(int64_t) * max_nq);
    A((void **)&b->k, sizeof(int32_t) * max_nq);
    A((void **)&b->ids, sizeof(int64_t) * max_nq * k_max);
    A((void **)&b->dist, sizeof(float) * max_nq * k_max);
    A((void **)&b->count, sizeof(int32_t) * max_nq);
    A((void **)&b->status, sizeof(int32_t) * max_nq);
    A((void **)&b->stats, sizeof(int64_t) * max_nq * ESG_QUERY_STATS);
    if (st == ESG_OK) {
        // scratch sized for the largest batch (per-item buffers grow with nq)
        SearchPlan plan;
        SearchLaunch s = launch_for(b, max_nq);
        st = esg_search_prepare(s, plan);
        if (st == ESG_OK) {
            b->scratch_bytes = plan.scratch_bytes;
            A(&b->scratch, b->scratch_bytes);
        }
    }
    if (st == ESG_OK && cudaStreamCreateWithFlags(&b->cap_stream, cudaStreamNonBlocking) != cudaSuccess) {
        esg_set_error("cudaStreamCreate failed");
        st = ESG_ERR_CUDA;
    }
    if (st != ESG_OK) { release(b); delete b; return st; }
    *out = b;
    return ESG_OK;
}

esg_status esg_batch_buffers(esg_batch *b, float **queries, int64_t **l, int64_t **r, int32_t **k,
                             int64_t **ids, float **dist, int32_t **count, int32_t **status,
                             int64_t **stats) {
    if (!b) { esg_set_error("batch is NULL"); return ESG_ERR_INVALID_ARG; }
    if (queries) *queries = b->queries;
    if (l) *l = b->l;
    if (r) *r = b->r;
    if (k) *k = b->k;
    if (ids) *ids = b->ids;
    if (dist) *dist = b->dist;
    if (count) *count = b->count;
    if (status) *status = b->status;
    if (stats) *stats = b->stats;
    return ESG_OK;
}

esg_status esg_batch_run(esg_batch *b, int64_t nq, esg_stream_t stream) {
    if (!b || nq < 0 || nq > b->max_nq) { esg_set_error("esg_batch_run: bad argument"); return ESG_ERR_INVALID_ARG; }
    if (nq == 0) return ESG_OK;
    auto it = b->graphs.find(nq);
    const bool fresh = it == b->graphs.end();
    if (fresh) {
        SearchLaunch s = launch_for(b, nq);
        SearchPlan plan;
        esg_status st = esg_search_prepare(s, plan);
        if (st != ESG_OK) return st;
        if (plan.scratch_bytes > b->scratch_bytes) { esg_set_error("esg_batch_run: scratch too small"); return ESG_ERR_CUDA; }
        ESG_CUDA_TRY(cudaStreamBeginCapture(b->cap_stream, cudaStreamCaptureModeThreadLocal));
        st = esg_search_enqueue(s, plan, b->scratch, b->cap_stream);
        cudaGraph_t g = nullptr;
        cudaError_t e = cudaStreamEndCapture(b->cap_stream, &g);
        if (st != ESG_OK) { if (g) cudaGraphDestroy(g); return st; }
        if (e != cudaSuccess) { esg_set_error(cudaGetErrorString(e)); return ESG_ERR_CUDA; }
        cudaGraphExec_t exec = nullptr;
        e = cudaGraphInstantiate(&exec, g, 0);
        cudaGraphDestroy(g);
        if (e != cudaSuccess) { esg_set_error(cudaGetErrorString(e)); return ESG_ERR_CUDA; }
        it = b->graphs.emplace(nq, exec).first;
    }
    // a capture already counted its kernels: prep, order, search, merge, and
    // the budget network with the learned budget
    if (!fresh) esg_prof_count(4 + (b->p.use_learned && b->ix->mlp_ready ? 1 : 0));
    ESG_CUDA_TRY(cudaGraphLaunch(it->second, (cudaStream_t)stream));
    return ESG_OK;
}

void esg_batch_free(esg_batch *b) {
    if (!b) return;
    release(b);
    delete b;
}

}  // extern "C"

// ------------------------------------------------------------------ autotune

namespace {
// hits[i] = |returned ids of query i  ∩  its first min(k_i, gcnt_i) gt ids|
// (k null: k_i = k_max); the recall denominator of query i is min(k_i, gcnt_i)
__global__ void recall_hits_kernel(int64_t nq, int32_t k_max, const int32_t *k, const int64_t *ids,
                                   const int32_t *cnt, const int64_t *gt, const int32_t *gcnt, int32_t *hits) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= nq) return;
    int kk = k ? k[i] : k_max;
    kk = kk < 0 ? 0 : (kk > k_max ? k_max : kk);
    const int g = min(gcnt[i], kk);
    int h = 0;
    for (int a = 0; a < min(cnt[i], kk); ++a) {
        const int64_t x = ids[i * k_max + a];
        for (int b = 0; b < g; ++b)
            if (gt[i * k_max + b] == x) { ++h; break; }
    }
    hits[i] = h;
}
}  // namespace

esg_status esg_recall_hits(int64_t nq, int32_t k_max, const int32_t *k, const int64_t *ids, const int32_t *cnt,
                           const int64_t *gt, const int32_t *gcnt, int32_t *hits, cudaStream_t stream) {
    recall_hits_kernel<<<ceil_div_i(nq, 128), 128, 0, stream>>>(nq, k_max, k, ids, cnt, gt, gcnt, hits);
    ESG_CUDA_TRY(cudaGetLastError());
    return ESG_OK;
}

extern "C" esg_status esg_autotune(const esg_index *ix, const float *queries, int64_t nq,
                                   const int64_t *l, const int64_t *r, const int32_t *k,
                                   int32_t k_max, const int64_t *gt_ids, const int32_t *gt_count,
                                   float target_recall, const esg_search_params *base,
                                   esg_search_params *out, float *report, esg_stream_t stream_v) {
    if (!ix || !queries || nq < 1 || nq >= kMaxBatch || !l || !r || k_max < 1 || k_max > 1024 || !gt_ids || !gt_count ||
        !out || !(target_recall > 0.f && target_recall <= 1.f)) {
        esg_set_error("esg_autotune: bad argument");
        return ESG_ERR_INVALID_ARG;
    }
    cudaStream_t stream = (cudaStream_t)stream_v;
    esg_search_params p = base ? *base : esg_search_params_default();
    p.warps_per_block = 0; p.hash_slots = 0; p.lanes_per_row = 0; p.max_registers = 0;
    int64_t *ids = nullptr;
    float *dist = nullptr;
    int32_t *cnt = nullptr, *hits = nullptr;
    void *scratch = nullptr;
    size_t scratch_bytes = 0;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    std::vector<int32_t> h_hits(nq), h_gc(nq);
    esg_status st = ESG_OK;
    double gt_total = 0;
    auto search = [&](const esg_search_params &pp) -> esg_status {
        SearchLaunch s;
        s.ix = ix; s.queries = queries; s.nq = nq; s.l = l; s.r = r; s.k = k; s.k_max = k_max;
        s.p = pp; s.out_ids = ids; s.out_dist = dist; s.out_count = cnt; s.out_status = nullptr;
        s.out_stats = nullptr;
        SearchPlan plan;
        esg_status s2 = esg_search_prepare(s, plan);
        if (s2 != ESG_OK) return s2;
        if (plan.scratch_bytes > scratch_bytes) {
            cudaFree(scratch);
            scratch = nullptr;
            if (esg_malloc((void **)&scratch, plan.scratch_bytes) != cudaSuccess) { esg_set_error("autotune: scratch"); return ESG_ERR_OOM; }
            scratch_bytes = plan.scratch_bytes;
        }
        return esg_search_enqueue(s, plan, scratch, stream);
    };
    auto recall_of = [&](const esg_search_params &pp, double &rec) -> esg_status {
        esg_status s2 = search(pp);
        if (s2 != ESG_OK) return s2;
        recall_hits_kernel<<<ceil_div_i(nq, 128), 128, 0, stream>>>(nq, k_max, k, ids, cnt, gt_ids, gt_count, hits);
        if (cudaMemcpyAsync(h_hits.data(), hits, sizeof(int32_t) * nq, cudaMemcpyDeviceToHost, stream) != cudaSuccess ||
            cudaStreamSynchronize(stream) != cudaSuccess) { esg_set_error("autotune: recall copy"); return ESG_ERR_CUDA; }
        double h = 0;
        for (int64_t i = 0; i < nq; ++i) h += h_hits[i];
        rec = gt_total > 0 ? h / gt_total : 1.0;
        return ESG_OK;
    };
    auto time_of = [&](const esg_search_params &pp, float &ms, int reps) -> esg_status {
        float best = 1e30f;
        for (int rep = 0; rep < reps; ++rep) {
            cudaEventRecord(e0, stream);
            esg_status s2 = search(pp);
            if (s2 != ESG_OK) return s2;
            cudaEventRecord(e1, stream);
            if (cudaEventSynchronize(e1) != cudaSuccess) { esg_set_error("autotune: timing"); return ESG_ERR_CUDA; }
            float t = 0.f;
            cudaEventElapsedTime(&t, e0, e1);
            if (rep > 0) best = std::min(best, t);   // first run warms up
        }
        ms = best;
        return ESG_OK;
    };
    const int efs[] = {8, 12, 16, 20, 24, 32, 40, 48, 64, 96, 128, 192, 256, 384, 512, 768, 1024};
    struct Cand_ { esg_search_params p; double recall; float ms; };
    std::vector<Cand_> found;
    if (esg_malloc((void **)&ids, sizeof(int64_t) * nq * k_max) != cudaSuccess ||
        esg_malloc((void **)&dist, sizeof(float) * nq * k_max) != cudaSuccess ||
        esg_malloc((void **)&cnt, sizeof(int32_t) * nq) != cudaSuccess ||
        esg_malloc((void **)&hits, sizeof(int32_t) * nq) != cudaSuccess ||
        cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
        esg_set_error("autotune: allocation");
        st = ESG_ERR_OOM;
    }
    if (st == ESG_OK) {
        std::vector<int32_t> h_k(nq, k_max);
        if (cudaMemcpy(h_gc.data(), gt_count, sizeof(int32_t) * nq, cudaMemcpyDeviceToHost) != cudaSuccess ||
            (k && cudaMemcpy(h_k.data(), k, sizeof(int32_t) * nq, cudaMemcpyDeviceToHost) != cudaSuccess)) {
            esg_set_error("autotune: gt copy"); st = ESG_ERR_CUDA;
        }
        for (int64_t i = 0; i < nq; ++i) gt_total += std::min(h_gc[i], std::max(0, std::min(h_k[i], k_max)));
    }
    // 1. smallest ef reaching the target, per search width (with the learned
    //    budget, ef is only the fallback: keep it and check the recall)
    if (st == ESG_OK && p.use_learned && ix->mlp_ready) {
        for (int width = 1; width <= 2 && st == ESG_OK; ++width) {
            esg_search_params pp = p;
            pp.width = width;
            double rec = 0;
            st = recall_of(pp, rec);
            if (st == ESG_OK && rec >= target_recall) found.push_back({pp, rec, 0.f});
        }
    }
    for (int width = 1; width <= 2 && st == ESG_OK && !(p.use_learned && ix->mlp_ready); ++width) {
        for (int ef : efs) {
            if (ef < 1) continue;
            esg_search_params pp = p;
            pp.ef = ef;
            pp.width = width;
            double rec = 0;
            st = recall_of(pp, rec);
            if (st != ESG_OK) break;
            if (rec >= target_recall) { found.push_back({pp, rec, 0.f}); break; }
        }
    }
    // 2. fastest launch shape for each candidate: every shape timed once
    //    (best of 3 after a warm-up run), then the few fastest re-timed with
    //    more repetitions, since neighbouring shapes often differ by less
    //    than the run-to-run spread of a single timing
    struct Timed { esg_search_params p; double recall; float ms; };
    std::vector<Timed> timed;
    for (auto &c : found) {
        if (st != ESG_OK) break;
        const int lprs[] = {0, 4, 8, 16, 32};
        for (int wpb : {1, 2, 4}) {
            for (int hs : {0, 1024, 4096, 8192}) {   // 0: the default, 2,048 slots
                for (int lpr : lprs) {
                    for (int mr : {128, 96}) {
                        esg_search_params pp = c.p;
                        pp.warps_per_block = wpb; pp.hash_slots = hs; pp.lanes_per_row = lpr;
                        pp.max_registers = mr;
                        float ms = 0.f;
                        esg_status s2 = time_of(pp, ms, 4);
                        if (s2 == ESG_ERR_UNSUPPORTED) continue;   // shape not valid for this row
                        if (s2 != ESG_OK) { st = s2; break; }
                        timed.push_back({pp, c.recall, ms});
                    }
                    if (st != ESG_OK) break;
                }
                if (st != ESG_OK) break;
            }
            if (st != ESG_OK) break;
        }
    }
    std::sort(timed.begin(), timed.end(), [](const Timed &x, const Timed &y) { return x.ms < y.ms; });
    esg_search_params best{};
    double best_rec = 0;
    float best_ms = 1e30f;
    for (size_t i = 0; st == ESG_OK && i < std::min<size_t>(timed.size(), 6); ++i) {
        float ms = 0.f;
        st = time_of(timed[i].p, ms, 12);
        if (st == ESG_OK && ms < best_ms) { best_ms = ms; best = timed[i].p; best_rec = timed[i].recall; }
    }
    if (st == ESG_OK && found.empty()) { esg_set_error("autotune: no setting reaches the target recall"); st = ESG_ERR_UNSUPPORTED; }
    if (st == ESG_OK) {
        *out = best;
        if (report) { report[0] = (float)best_rec; report[1] = best_ms; }
    }
    cudaFree(ids); cudaFree(dist); cudaFree(cnt); cudaFree(hits); cudaFree(scratch);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    return st;
}

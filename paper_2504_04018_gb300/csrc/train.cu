// Training of the learned search budget (esg_train_predictor): traces of the
// plain fixed-ef search give, per training query, the smallest beam width
// in a grid whose recall reaches the per-query target and the expansions it
// used; the MLP of mlp.cu regresses log2 of both with a pinball loss
// (over-predicting is cheaper than missing neighbours), trained with its own
// GPU kernels and Adam; a margin on the predicted log2 ef is then calibrated
// on held-out queries so their mean recall reaches the target.
#include "esg_internal.cuh"

#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

extern "C" {
esg_status esg_mlp_loss_grad(const float *params, const float *X, const float *T, const float *mu,
                             const float *sigma, int64_t B, float quantile, float *grad, float *loss,
                             esg_stream_t stream);
esg_status esg_mlp_adam_step(float *params, const float *grad, float *m, float *v, int32_t step,
                             float lr, esg_stream_t stream);
esg_status esg_query_features(const esg_index *ix, const float *queries, int64_t nq, const int64_t *l,
                              const int64_t *r, const int32_t *k, int32_t k_max, float *feat,
                              esg_stream_t stream);
esg_status esg_predictor_set(esg_index *ix, const float *blob_host, int32_t ef_lo, int32_t ef_hi);
}

namespace {

// SplitMix64 (Steele, Lea, Flood 2014): the seeded generator of the initial
// weights and of the minibatch order.
struct SplitMix64 {
    uint64_t s;
    uint64_t next() {
        uint64_t z = (s += 0x9E3779B97F4A7C15ull);
        z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
        z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
        return z ^ (z >> 31);
    }
    double uniform() { return (next() >> 11) * (1.0 / 9007199254740992.0); }
};

struct DevBuf {
    void *p = nullptr;
    ~DevBuf() { cudaFree(p); }
};

}  // namespace

extern "C" esg_status esg_train_predictor(esg_index *ix, const float *queries, int64_t nq,
                                          const int64_t *l, const int64_t *r, const int32_t *k,
                                          int32_t k_max, const int64_t *gt_ids, const int32_t *gt_count,
                                          const esg_train_params *tp_in, float *report,
                                          esg_stream_t stream_v) {
    if (!ix || !queries || nq < 16 || nq >= kMaxBatch || !l || !r || k_max < 1 || k_max > 1024 || !gt_ids || !gt_count) {
        esg_set_error("esg_train_predictor: bad argument");
        return ESG_ERR_INVALID_ARG;
    }
    esg_train_params tp = tp_in ? *tp_in : esg_train_params_default();
    if (!(tp.target_recall > 0.f && tp.target_recall <= 1.f) || !(tp.quantile > 0.f && tp.quantile < 1.f) ||
        tp.epochs < 1 || tp.batch < 8 || !(tp.lr > 0.f) || !(tp.val_fraction > 0.f && tp.val_fraction < 1.f) ||
        tp.ef_lo < 1 || tp.ef_hi < tp.ef_lo || tp.ef_hi > 1024) {
        esg_set_error("esg_train_predictor: parameter out of range");
        return ESG_ERR_INVALID_ARG;
    }
    cudaStream_t stream = (cudaStream_t)stream_v;
    const int F = ESG_MLP_FEATURES, P = esg_mlp_param_count();
    const int64_t n_val = std::max<int64_t>(8, (int64_t)(nq * tp.val_fraction));
    const int64_t n_tr = nq - n_val;
    if (n_tr < 8) { esg_set_error("esg_train_predictor: too few training queries"); return ESG_ERR_INVALID_ARG; }

    DevBuf ids_b, dist_b, cnt_b, stats_b, hits_b, feat_b;
    auto alloc = [&](DevBuf &b, size_t bytes) -> bool { return esg_malloc((void **)&b.p, bytes) == cudaSuccess; };
    if (!alloc(ids_b, sizeof(int64_t) * nq * k_max) || !alloc(dist_b, sizeof(float) * nq * k_max) ||
        !alloc(cnt_b, sizeof(int32_t) * nq) || !alloc(stats_b, sizeof(int64_t) * nq * ESG_QUERY_STATS) ||
        !alloc(hits_b, sizeof(int32_t) * nq) || !alloc(feat_b, sizeof(float) * nq * F)) {
        esg_set_error("esg_train_predictor: allocation");
        return ESG_ERR_OOM;
    }
    int64_t *ids = (int64_t *)ids_b.p;
    float *dist = (float *)dist_b.p;
    int32_t *cnt = (int32_t *)cnt_b.p, *hits = (int32_t *)hits_b.p;
    int64_t *stats = (int64_t *)stats_b.p;
    float *feat = (float *)feat_b.p;

    std::vector<int32_t> gc(nq), h_hits(nq);
    std::vector<int64_t> h_stats(nq * ESG_QUERY_STATS);
    ESG_CUDA_TRY(cudaMemcpy(gc.data(), gt_count, sizeof(int32_t) * nq, cudaMemcpyDeviceToHost));
    {
        // recall denominators: min(k_i, ground-truth count)
        std::vector<int32_t> hk(nq, k_max);
        if (k) ESG_CUDA_TRY(cudaMemcpy(hk.data(), k, sizeof(int32_t) * nq, cudaMemcpyDeviceToHost));
        for (int64_t i = 0; i < nq; ++i) gc[i] = std::min(gc[i], std::max(0, std::min(hk[i], k_max)));
    }
    esg_search_params sp = esg_search_params_default();
    sp.traversal = (esg_dtype)tp.traversal;
    sp.width = 1;
    sp.use_learned = 0;

    // 1. traces of the plain search over a grid of beam widths
    std::vector<int> grid;
    for (int e : {8, 12, 16, 24, 32, 48, 64, 96, 128, 192, 256, 384, 512, 768, 1024})
        if (e >= tp.ef_lo && e <= tp.ef_hi) grid.push_back(e);
    if (grid.empty() || grid.back() != tp.ef_hi) grid.push_back(tp.ef_hi);
    std::vector<float> label_ef(nq, std::log2((float)tp.ef_hi)), label_exp(nq, 0.f);
    std::vector<char> done(nq, 0);
    for (int ef : grid) {
        sp.ef = ef;
        SearchLaunch s;
        s.ix = ix; s.queries = queries; s.nq = nq; s.l = l; s.r = r; s.k = k; s.k_max = k_max; s.p = sp;
        s.out_ids = ids; s.out_dist = dist; s.out_count = cnt; s.out_status = nullptr; s.out_stats = stats;
        esg_status st = esg_launch_search(s, stream);
        if (st == ESG_OK) st = esg_recall_hits(nq, k_max, k, ids, cnt, gt_ids, gt_count, hits, stream);
        if (st != ESG_OK) return st;
        ESG_CUDA_TRY(cudaMemcpyAsync(h_hits.data(), hits, sizeof(int32_t) * nq, cudaMemcpyDeviceToHost, stream));
        ESG_CUDA_TRY(cudaMemcpyAsync(h_stats.data(), stats, sizeof(int64_t) * nq * ESG_QUERY_STATS, cudaMemcpyDeviceToHost, stream));
        ESG_CUDA_TRY(cudaStreamSynchronize(stream));
        for (int64_t i = 0; i < nq; ++i) {
            const double rec = gc[i] > 0 ? (double)h_hits[i] / gc[i] : 1.0;
            if (ef == grid.back() && !done[i]) label_exp[i] = std::log2((float)std::max<int64_t>(1, h_stats[i * ESG_QUERY_STATS]));
            if (!done[i] && rec >= tp.per_query_recall) {
                done[i] = 1;
                label_ef[i] = std::log2((float)ef);
                label_exp[i] = std::log2((float)std::max<int64_t>(1, h_stats[i * ESG_QUERY_STATS]));
            }
        }
    }
    // 2. features and their standardisation (training split)
    {
        esg_status st = esg_query_features(ix, queries, nq, l, r, k, k_max, feat, stream);
        if (st != ESG_OK) return st;
    }
    std::vector<float> hf(nq * F);
    ESG_CUDA_TRY(cudaMemcpyAsync(hf.data(), feat, sizeof(float) * nq * F, cudaMemcpyDeviceToHost, stream));
    ESG_CUDA_TRY(cudaStreamSynchronize(stream));
    std::vector<float> mu(F, 0.f), sigma(F, 1.f);
    for (int f = 0; f < F; ++f) {
        double s = 0, s2 = 0;
        for (int64_t i = 0; i < n_tr; ++i) { s += hf[i * F + f]; s2 += (double)hf[i * F + f] * hf[i * F + f]; }
        const double m = s / n_tr, var = std::max(0.0, s2 / n_tr - m * m);
        mu[f] = (float)m;
        sigma[f] = (float)std::max(std::sqrt(var), 1e-3);
    }
    // 3. initial weights: uniform(+-sqrt(6 / fan_in)) for the weights, zero biases
    SplitMix64 rng{tp.seed};
    std::vector<float> params(P, 0.f);
    {
        const int H = 64, O = 2;
        int o = 0;
        auto fill = [&](int count, int fan_in) {
            const double a = std::sqrt(6.0 / fan_in);
            for (int i = 0; i < count; ++i) params[o++] = (float)((2.0 * rng.uniform() - 1.0) * a);
        };
        fill(F * H, F); o += H;
        fill(H * H, H); o += H;
        fill(H * O, H); o += O;
    }
    DevBuf p_b, g_b, m_b, v_b, mu_b, sg_b, xb_b, tb_b;
    if (!alloc(p_b, sizeof(float) * P) || !alloc(g_b, sizeof(float) * P) || !alloc(m_b, sizeof(float) * P) ||
        !alloc(v_b, sizeof(float) * P) || !alloc(mu_b, sizeof(float) * F) || !alloc(sg_b, sizeof(float) * F) ||
        !alloc(xb_b, sizeof(float) * tp.batch * F) || !alloc(tb_b, sizeof(float) * tp.batch * 2)) {
        esg_set_error("esg_train_predictor: allocation");
        return ESG_ERR_OOM;
    }
    ESG_CUDA_TRY(cudaMemcpy(p_b.p, params.data(), sizeof(float) * P, cudaMemcpyHostToDevice));
    ESG_CUDA_TRY(cudaMemset(m_b.p, 0, sizeof(float) * P));
    ESG_CUDA_TRY(cudaMemset(v_b.p, 0, sizeof(float) * P));
    ESG_CUDA_TRY(cudaMemcpy(mu_b.p, mu.data(), sizeof(float) * F, cudaMemcpyHostToDevice));
    ESG_CUDA_TRY(cudaMemcpy(sg_b.p, sigma.data(), sizeof(float) * F, cudaMemcpyHostToDevice));
    // 4. minibatch Adam over shuffled training rows
    std::vector<int64_t> order(n_tr);
    for (int64_t i = 0; i < n_tr; ++i) order[i] = i;
    std::vector<float> xb(tp.batch * F), tb(tp.batch * 2);
    int32_t step = 0;
    float last_loss = 0.f;
    for (int ep = 0; ep < tp.epochs; ++ep) {
        for (int64_t i = n_tr - 1; i > 0; --i) std::swap(order[i], order[(int64_t)(rng.next() % (uint64_t)(i + 1))]);
        for (int64_t b0 = 0; b0 + tp.batch <= n_tr || (b0 == 0 && n_tr < tp.batch); b0 += tp.batch) {
            const int64_t B = std::min<int64_t>(tp.batch, n_tr - b0);
            for (int64_t j = 0; j < B; ++j) {
                const int64_t row = order[b0 + j];
                for (int f = 0; f < F; ++f) xb[j * F + f] = hf[row * F + f];
                tb[j * 2 + 0] = label_ef[row];
                tb[j * 2 + 1] = label_exp[row];
            }
            ESG_CUDA_TRY(cudaMemcpyAsync(xb_b.p, xb.data(), sizeof(float) * B * F, cudaMemcpyHostToDevice, stream));
            ESG_CUDA_TRY(cudaMemcpyAsync(tb_b.p, tb.data(), sizeof(float) * B * 2, cudaMemcpyHostToDevice, stream));
            const bool last = ep == tp.epochs - 1 && b0 + 2 * tp.batch > n_tr;
            esg_status st = esg_mlp_loss_grad((float *)p_b.p, (float *)xb_b.p, (float *)tb_b.p, (float *)mu_b.p,
                                              (float *)sg_b.p, B, tp.quantile, (float *)g_b.p,
                                              last ? &last_loss : nullptr, stream);
            if (st == ESG_OK) st = esg_mlp_adam_step((float *)p_b.p, (float *)g_b.p, (float *)m_b.p,
                                                     (float *)v_b.p, ++step, tp.lr, stream);
            if (st != ESG_OK) return st;
            if (n_tr < tp.batch) break;
        }
    }
    ESG_CUDA_TRY(cudaMemcpyAsync(params.data(), p_b.p, sizeof(float) * P, cudaMemcpyDeviceToHost, stream));
    ESG_CUDA_TRY(cudaStreamSynchronize(stream));
    // 5. calibrate the ef margin on the held-out split (bisection in log2
    // units): one margin for all queries against their pooled recall, then,
    // if asked, an offset per class of k (floor(log2 k)) so that each class
    // reaches the target on its own (the pooled recall weighs a query by its
    // k, so one margin leaves the small-k classes below the target)
    const int KB = ESG_MLP_KBUCKETS;
    std::vector<float> blob(esg_mlp_blob_floats(), 0.f);
    std::memcpy(blob.data(), params.data(), sizeof(float) * P);
    std::memcpy(blob.data() + P, mu.data(), sizeof(float) * F);
    std::memcpy(blob.data() + P + F, sigma.data(), sizeof(float) * F);
    float *margins = blob.data() + P + 2 * F;   // [ef, expansions, ef offset per class of k]
    const float exp_margin = 1.0f;   // expansion budget: twice the predicted expansions
    std::vector<int> vb(n_val);
    std::vector<double> gv_b(KB, 0.0);
    std::vector<int64_t> nv_b(KB, 0);
    double gv = 0;
    {
        std::vector<int32_t> hk(nq, k_max);
        if (k) ESG_CUDA_TRY(cudaMemcpy(hk.data(), k, sizeof(int32_t) * nq, cudaMemcpyDeviceToHost));
        for (int64_t i = n_tr; i < nq; ++i) {
            const int b = esg_k_bucket(std::max(1, std::min(hk[i], k_max)));
            vb[i - n_tr] = b;
            gv_b[b] += gc[i];
            ++nv_b[b];
            gv += gc[i];
        }
    }
    std::vector<double> rec_b(KB, 1.0);
    auto val_recall = [&](double &rec, double &mean_ef) -> esg_status {
        margins[1] = exp_margin;
        esg_status st = esg_predictor_set(ix, blob.data(), tp.ef_lo, tp.ef_hi);
        if (st != ESG_OK) return st;
        esg_search_params q = sp;
        q.use_learned = 1;
        q.ef = tp.ef_hi;
        SearchLaunch s;
        s.ix = ix; s.queries = queries + n_tr * (int64_t)ix->d; s.nq = n_val; s.l = l + n_tr; s.r = r + n_tr;
        s.k = k ? k + n_tr : nullptr; s.k_max = k_max; s.p = q;
        s.out_ids = ids; s.out_dist = dist; s.out_count = cnt; s.out_status = nullptr; s.out_stats = stats;
        st = esg_launch_search(s, stream);
        if (st == ESG_OK) st = esg_recall_hits(n_val, k_max, k ? k + n_tr : nullptr, ids, cnt, gt_ids + n_tr * k_max, gt_count + n_tr, hits, stream);
        if (st != ESG_OK) return st;
        ESG_CUDA_TRY(cudaMemcpyAsync(h_hits.data(), hits, sizeof(int32_t) * n_val, cudaMemcpyDeviceToHost, stream));
        ESG_CUDA_TRY(cudaMemcpyAsync(h_stats.data(), stats, sizeof(int64_t) * n_val * ESG_QUERY_STATS, cudaMemcpyDeviceToHost, stream));
        ESG_CUDA_TRY(cudaStreamSynchronize(stream));
        double h = 0, ev = 0;
        std::vector<double> h_b(KB, 0.0);
        for (int64_t i = 0; i < n_val; ++i) {
            h += h_hits[i];
            h_b[vb[i]] += h_hits[i];
            ev += h_stats[i * ESG_QUERY_STATS + 1];
        }
        rec = gv > 0 ? h / gv : 1.0;
        for (int b = 0; b < KB; ++b) rec_b[b] = gv_b[b] > 0 ? h_b[b] / gv_b[b] : 1.0;
        mean_ef = ev / n_val;   // distance evaluations per query
        return ESG_OK;
    };
    float lo = -4.f, hi = 4.f;
    double rec_hi = 0, cost_hi = 0;
    margins[0] = hi;
    esg_status st = val_recall(rec_hi, cost_hi);
    if (st != ESG_OK) return st;
    if (rec_hi < tp.target_recall) {
        ix->mlp_ready = 0;
        esg_set_error("esg_train_predictor: even the largest margin misses the target recall");
        return ESG_ERR_UNSUPPORTED;
    }
    for (int it = 0; it < 10; ++it) {
        const float mid = 0.5f * (lo + hi);
        double rec = 0, cost = 0;
        margins[0] = mid;
        st = val_recall(rec, cost);
        if (st != ESG_OK) return st;
        if (rec >= tp.target_recall) hi = mid; else lo = mid;
    }
    margins[0] = hi;
    // per-class offsets, all classes bisected together (a search serves all
    // of them); a class with too few held-out queries keeps offset 0, and a
    // class whose widest offset misses the target keeps that widest offset
    const int64_t kMinClass = 64;
    std::vector<float> olo(KB, -4.f), ohi(KB, 4.f);
    bool any = false;
    for (int b = 0; b < KB; ++b) if (nv_b[b] >= kMinClass) any = true;
    if (any && tp.per_k_class) {
        for (int it = 0; it < 10; ++it) {
            for (int b = 0; b < KB; ++b) margins[2 + b] = nv_b[b] >= kMinClass ? 0.5f * (olo[b] + ohi[b]) : 0.f;
            double rec = 0, cost = 0;
            st = val_recall(rec, cost);
            if (st != ESG_OK) return st;
            for (int b = 0; b < KB; ++b) {
                if (nv_b[b] < kMinClass) continue;
                const float mid = margins[2 + b];
                if (rec_b[b] >= tp.target_recall) ohi[b] = mid; else olo[b] = mid;
            }
        }
        for (int b = 0; b < KB; ++b) margins[2 + b] = nv_b[b] >= kMinClass ? ohi[b] : 0.f;
    }
    double rec_f = 0, cost_f = 0;
    st = val_recall(rec_f, cost_f);
    if (st != ESG_OK) return st;
    if (report) {
        report[0] = last_loss;
        report[1] = (float)rec_f;
        report[2] = hi;
        report[3] = (float)cost_f;
    }
    return ESG_OK;
}

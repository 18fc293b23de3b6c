// Range-filtered graph search on the GPU: elastic decomposition (Algorithm 4),
// warp beam search with the POST filter (Algorithm 1), exact leaf scan, and
// the final merge of the two piece lists.
//
// Work decomposition: one warp per (query, piece) work item, taken from an
// atomic queue by a persistent grid. Each warp keeps, in its own shared
// memory slice:
//   - a sorted candidate list of (distance, rank) pairs holding the result
//     queue Q (the in-range items, at most ef) interleaved with the
//     not-yet-expanded out-of-range candidates of P that are closer than the
//     worst of Q; items farther than the ef-th in-range item are dropped,
//     since Algorithm 1 would never expand or return them;
//   - a visited set (open addressing over ranks) in shared memory, or in a
//     global-memory slot for large beam widths;
//   - the batch of newly reached neighbours of the current expansion.
// One expansion = pop the best unexpanded candidate, read its R neighbour
// ranks (one coalesced row), test-and-set them in the visited set, gather the
// new rows with 16-byte loads (LPR lanes per row), reduce the distances with
// shuffles, admit those that pass Algorithm 1's test (|Q| < ef or closer than
// the worst of Q), sort them (in registers when at most 32) and merge them
// into the list by rank.
#include "esg_internal.cuh"
#include "decompose.cuh"
#include "search_kernel.cuh"

#include <algorithm>
#include <cstdlib>

using esg_sk::SearchArgs;
using esg_sk::SearchFn;

namespace {

// Validate queries and decompose their ranges (one thread per query).
__global__ void prep_kernel(DecomposeSpec spec, const int64_t *l, const int64_t *r,
                            const int32_t *k, int32_t k_max, int64_t nq, esg_piece *pieces,
                            int32_t *kq, int32_t *qstatus) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= nq) return;
    int64_t lq = l[i], rq = r[i];
    int kk = k ? k[i] : k_max;
    esg_piece pcs[2];
    int cnt = 0;
    bool ok = kk >= 1 && kk <= k_max && lq >= 0 && lq <= rq && rq < spec.n;
    if (ok) cnt = esg_decompose_one(spec, lq, rq, pcs);
    if (!ok || cnt <= 0) {
        pcs[0].kind = ESG_PIECE_NONE; pcs[1].kind = ESG_PIECE_NONE;
        kk = 0;
    }
    pieces[2 * i] = pcs[0];
    pieces[2 * i + 1] = pcs[1];
    kq[i] = kk;
    qstatus[i] = (ok && cnt > 0) ? 0 : ESG_Q_INVALID;
}

// Processing order of the search items, longest first by query (one block,
// counting sort over log-spaced cost buckets; the order within a bucket is
// arbitrary and does not change any result). A query's two pieces are placed
// next to each other, its longer piece first, and the query is keyed by that
// longer piece: the launch keeps its short tail (long searches start early)
// and a query's latency inside the batch stays that of its own pieces.
// Estimated cost of an item: a graph piece ~ ef (1 + log2 of its node size),
// a scan piece ~ its width / 64 rows, an empty piece 0.
constexpr int kOrderThreads = 1024;
constexpr int kOrderBuckets = 64;

__device__ __forceinline__ int order_bucket(const esg_piece &pc, int ef) {
    float c = 0.f;
    if (pc.kind == ESG_PIECE_GRAPH)
        c = (float)ef * (1.f + log2f((float)(pc.node_r - pc.node_l + 1)));
    else if (pc.kind == ESG_PIECE_SCAN)
        c = (float)(pc.pr - pc.pl + 1) * (1.f / 64.f);
    const int b = (int)(4.f * log2f(1.f + c));   // 4 buckets per doubling
    return kOrderBuckets - 1 - min(b, kOrderBuckets - 1);
}

// With split_ef > 0 the queries are also split into the budget classes of
// SearchPlan (class 1 when max(ef_q, k) > split_ef): class 0's items come
// first, and range[2c], range[2c + 1] receive the first and one-past-last
// position of class c.
__global__ void __launch_bounds__(kOrderThreads) order_items_kernel(const esg_piece *pieces, const int32_t *ef_q,
                                                                    const int32_t *kq, int ef, int split_ef,
                                                                    int64_t nq, int32_t *order, int32_t *range) {
    __shared__ int32_t cnt[2 * kOrderBuckets];
    if (threadIdx.x < 2 * kOrderBuckets) cnt[threadIdx.x] = 0;
    __syncthreads();
    // buckets count down from the longest estimated cost, class 0 first
    for (int64_t q = threadIdx.x; q < nq; q += kOrderThreads) {
        const int e = ef_q ? ef_q[q] : ef;
        const int cls = split_ef > 0 && max(e, kq[q]) > split_ef ? 1 : 0;
        const int b = min(order_bucket(pieces[2 * q], e), order_bucket(pieces[2 * q + 1], e));
        atomicAdd(&cnt[cls * kOrderBuckets + b], 2);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        int32_t run = 0;
        for (int b = 0; b < 2 * kOrderBuckets; ++b) {
            if (b == kOrderBuckets) { range[1] = run; range[2] = run; }
            const int32_t c = cnt[b]; cnt[b] = run; run += c;
        }
        range[0] = 0;
        range[3] = run;
    }
    __syncthreads();
    for (int64_t q = threadIdx.x; q < nq; q += kOrderThreads) {
        const int e = ef_q ? ef_q[q] : ef;
        const int cls = split_ef > 0 && max(e, kq[q]) > split_ef ? 1 : 0;
        const int b0 = order_bucket(pieces[2 * q], e), b1 = order_bucket(pieces[2 * q + 1], e);
        const int32_t pos = atomicAdd(&cnt[cls * kOrderBuckets + min(b0, b1)], 2);
        const bool second_first = b1 < b0;
        order[pos] = (int32_t)(2 * q + (second_first ? 1 : 0));
        order[pos + 1] = (int32_t)(2 * q + (second_first ? 0 : 1));
    }
}

// Merge the (at most two) sorted piece lists of each query into its top k
// (Algorithm 4, last step), map ranks to original ids, pad the rest.
__global__ void merge_kernel(int64_t nq, int32_t k_max, const int32_t *kq, const Cand *res,
                             const int32_t *res_cnt, const int32_t *res_status,
                             const int64_t *res_stats, const int32_t *qstatus,
                             const int64_t *perm, const esg_piece *pieces, int64_t *out_ids,
                             float *out_dist, int32_t *out_count, int32_t *out_status,
                             int64_t *out_stats) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= nq) return;
    int k = kq[i];
    const Cand *A = res + (2 * i) * (int64_t)k_max;
    const Cand *B = res + (2 * i + 1) * (int64_t)k_max;
    int na = k > 0 ? res_cnt[2 * i] : 0, nb = k > 0 ? res_cnt[2 * i + 1] : 0;
    int ia = 0, ib = 0, o = 0;
    int64_t *oid = out_ids + i * (int64_t)k_max;
    float *od = out_dist + i * (int64_t)k_max;
    while (o < k && (ia < na || ib < nb)) {
        bool takeA = ib >= nb || (ia < na && cand_less(A[ia], B[ib]));
        Cand c = takeA ? A[ia++] : B[ib++];
        oid[o] = perm[c.id];
        od[o] = c.d;
        ++o;
    }
    for (int j = o; j < k_max; ++j) { oid[j] = -1; od[j] = INFINITY; }
    out_count[i] = o;
    if (out_status) {
        int s = qstatus[i];
        if (k > 0) s |= res_status[2 * i] | res_status[2 * i + 1];
        out_status[i] = s;
    }
    if (out_stats) {
        const bool va = pieces[2 * i].kind != ESG_PIECE_NONE, vb = pieces[2 * i + 1].kind != ESG_PIECE_NONE;
        const int64_t *sa = res_stats + 2 * i * ESG_ITEM_STATS, *sb = sa + ESG_ITEM_STATS;
        int64_t *os = out_stats + i * ESG_QUERY_STATS;
        for (int c = 0; c < 4; ++c) os[c] = k > 0 ? sa[c] + sb[c] : 0;
        os[4] = (int64_t)va + (int64_t)vb;
        // device latency: first item taken by a warp to last item finished
        int64_t lat = 0;
        if (k > 0 && (va || vb)) {
            const int64_t t0 = va && vb ? min(sa[4], sb[4]) : (va ? sa[4] : sb[4]);
            const int64_t t1 = va && vb ? max(sa[5], sb[5]) : (va ? sa[5] : sb[5]);
            lat = t1 - t0;
        }
        os[5] = lat;
    }
}

__global__ void decompose_kernel(DecomposeSpec spec, const int64_t *l, const int64_t *r,
                                 int64_t nq, esg_piece *out, int32_t *npieces) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= nq) return;
    esg_piece p[2];
    int c = esg_decompose_one(spec, l[i], r[i], p);
    out[2 * i] = p[0];
    out[2 * i + 1] = p[1];
    npieces[i] = c < 0 ? 0 : c;
}

typedef void (*SearchFn)(SearchArgs);

SearchFn pick_search(int st, int vpl, bool occ5 = false) {
    if (st == ESG_BF16) return esg_sk::pick_bf16(vpl, occ5);
    if (st == ESG_FP8E4M3) return esg_sk::pick_fp8(vpl, occ5);
    return esg_sk::pick_f32(vpl, occ5);
}

int env_int(const char *name, int dflt) {
    const char *v = getenv(name);
    return v && *v ? atoi(v) : dflt;
}

}  // namespace
int esg_pick_vpl(int d, int *lpr);
int esg_vpl_for_lpr(int nvec, int lpr);
namespace {

// Kernel, launch shape and shared memory for a search (or construction)
// call; knobs left at 0 are chosen automatically.
esg_status make_plan(int d, int R, int efk, int64_t n_items, int st, int width, int wpb_req,
                     int hash_req, int lpr_req, int mr_req, KernelPlan &pl, int list_per_ef = 2) {
    pl.width = std::max(1, std::min(width, 4));
    pl.BB = 64;
    while (pl.BB < pl.width * R) pl.BB <<= 1;
    const int esize = st == ESG_BF16 ? 2 : (st == ESG_FP8E4M3 ? 1 : 4);
    if ((d * esize) % 16 != 0 || d % 4 != 0) { esg_set_error("row size not a multiple of 16 bytes"); return ESG_ERR_UNSUPPORTED; }
    pl.nvec = d * esize / 16;
    if (lpr_req > 0) {
        pl.lpr = lpr_req;
        pl.vpl = esg_vpl_for_lpr(pl.nvec, lpr_req);
    } else {
        pl.vpl = esg_pick_vpl(pl.nvec * 4, &pl.lpr);
    }
    if (pl.vpl == 0) { esg_set_error("unsupported dimension / lanes per row"); return ESG_ERR_UNSUPPORTED; }
    if (R > 128) { esg_set_error("R > 128"); return ESG_ERR_UNSUPPORTED; }
    // candidate list: Q (at most ef in-range items) interleaved with the
    // unexpanded out-of-range candidates closer than its worst, list_per_ef
    // times ef items (at least 2: the in-place FP32 re-rank sorts a power of
    // two >= ef in it); on the elastic pieces (at least half of a node in
    // range) twice ef measured no loss of recall at 10^7 points
    const int lpe = std::max(2, std::min(8, list_per_ef));
    pl.lpe = lpe;
    pl.C = ((std::max(lpe * efk, 256) + 31) / 32) * 32;
    if (pl.C > 4096) pl.C = 4096;
    // shared visited table: 2,048 slots unless asked otherwise for an item
    // whose list is the smallest (256 items); the kernel gives an item with
    // a wider beam two fewer slots per list item above that (its own list
    // and table share one arena of C items + H slots), down to 1,024 slots.
    // The global overflow table takes what does not fit. A table sized for
    // the widest beam (up to 8K slots) cost more warps per SM than its
    // overflow probes save: at 10^7 points, ef 128, k up to 100, 185 vs
    // 125 ms per 100k-query call (FP32 rows)
    const int hs = hash_req > 0 ? hash_req : env_int("ESG_HASH_DEFAULT", 2048);
    pl.H = std::max(hs - 2 * (pl.C - 256), std::min(hs, 1024));
    pl.H = std::max(pl.H, 4 * R);
    pl.H = (pl.H + 3) & ~3;
    pl.G = 16384;
    while (pl.G < 256 * efk && pl.G < (1 << 20)) pl.G <<= 1;
    pl.wpb = wpb_req > 0 ? wpb_req : 2;
    pl.smem = ((size_t)pl.H * 4 + (size_t)pl.C * 8 + (size_t)pl.BB * 12 + 32 * 8 + 16 + 128 +
               (((size_t)d * 4 + 15) & ~(size_t)15)) * pl.wpb;
    int dev = 0, sms = 0, per_sm = 0;
    ESG_CUDA_TRY(cudaGetDevice(&dev));
    ESG_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    if (pl.smem > 227 * 1024) { esg_set_error("search plan needs too much shared memory"); return ESG_ERR_UNSUPPORTED; }
    // the 128- and the 96-register builds: resident blocks per SM of each
    SearchFn f128 = pick_search(st, pl.vpl), f96 = pick_search(st, pl.vpl, true);
    if (f128 == nullptr) { esg_set_error("no search kernel for this dimension and row type"); return ESG_ERR_UNSUPPORTED; }
    if (mr_req == 96 && f96 == nullptr) {
        esg_set_error("no 96-register search kernel for this row type and lanes per row");
        return ESG_ERR_UNSUPPORTED;
    }
    int per_sm128 = 0, per_sm96 = 0;
    ESG_CUDA_TRY(cudaFuncSetAttribute(f128, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)pl.smem));
    ESG_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm128, f128, pl.wpb * 32, pl.smem));
    if (f96 != nullptr && mr_req != 128) {
        ESG_CUDA_TRY(cudaFuncSetAttribute(f96, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)pl.smem));
        ESG_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm96, f96, pl.wpb * 32, pl.smem));
    }
    // automatic: the 96-register build only where more searches reside with
    // it (at 10^7 points, d = 96, 100k queries: BF16 rows at ef 128 118.9
    // vs 129.5 ms per call, FP8 116.5 vs 128.4)
    const bool use96 = mr_req == 96 || (mr_req == 0 && f96 != nullptr && per_sm96 > per_sm128);
    SearchFn fn = use96 ? f96 : f128;
    per_sm = use96 ? per_sm96 : per_sm128;
    pl.fn = (void *)fn;
    if (per_sm < 1) { esg_set_error("search kernel does not fit on an SM"); return ESG_ERR_UNSUPPORTED; }
    pl.grid = std::min<int64_t>((int64_t)sms * per_sm, (n_items + pl.wpb - 1) / pl.wpb);
    if (pl.grid < 1) pl.grid = 1;
    pl.efk = efk;
    return ESG_OK;
}

}  // namespace

// Lanes per row (LPR) and float4 per lane (VPL) for rows of d floats: prefer
// 4 lanes per row (8 rows per warp instruction, two shuffle steps per
// reduction; 5-7 % faster than 8 lanes on FP32 rows of 96 dimensions), then
// 8; wider rows use 16 or 32 lanes.
int esg_pick_vpl(int d, int *lpr) {
    if (d % 4) return 0;
    const int nvec = d / 4;
    const int lprs[] = {4, 8, 2, 1, 16, 32};
    for (int L : lprs) {
        if (nvec % L) continue;
        const int v = nvec / L;
        if (v == 1 || v == 2 || v == 3 || v == 4 || v == 6 || v == 8) { *lpr = L; return v; }
    }
    return 0;
}

// Vectors per lane when `lpr` lanes share a row of `nvec` 16-byte vectors
// (0 if that split is not supported).
int esg_vpl_for_lpr(int nvec, int lpr) {
    if (lpr < 1 || lpr > 32 || (lpr & (lpr - 1)) || nvec % lpr) return 0;
    const int v = nvec / lpr;
    return (v == 1 || v == 2 || v == 3 || v == 4 || v == 6 || v == 8) ? v : 0;
}

esg_status esg_launch_decompose(const DecomposeSpec &spec, const int64_t *l, const int64_t *r,
                                int64_t nq, esg_piece *pieces, int32_t *npieces, cudaStream_t stream) {
    if (nq == 0) return ESG_OK;
    decompose_kernel<<<ceil_div_i(nq, 256), 256, 0, stream>>>(spec, l, r, nq, pieces, npieces);
    ESG_CUDA_TRY(cudaGetLastError());
    return ESG_OK;
}

namespace {
struct ScratchLayout {
    size_t pieces, kq, qs, res, cnt, stats, hash, feat, efq, mxq, order, queue, total;
};

size_t al256(size_t x) { return (x + 255) & ~(size_t)255; }

size_t hash_bytes(const SearchPlan &plan) {
    size_t b = 0;
    for (int c = 0; c < plan.nclass; ++c)
        b = std::max(b, (size_t)plan.cls[c].grid * plan.cls[c].wpb * plan.cls[c].G * 8);
    return b;
}

ScratchLayout scratch_layout(int64_t nq, int32_t k_max, const SearchPlan &plan) {
    const int64_t n_items = 2 * nq;
    ScratchLayout L;
    size_t off = 0;
    L.pieces = off; off += al256(sizeof(esg_piece) * n_items);
    L.kq = off; off += al256(sizeof(int32_t) * nq);
    L.qs = off; off += al256(sizeof(int32_t) * nq);
    L.res = off; off += al256(sizeof(Cand) * n_items * k_max);
    L.cnt = off; off += al256(sizeof(int32_t) * n_items * 2);
    L.stats = off; off += al256(sizeof(int64_t) * n_items * ESG_ITEM_STATS);
    // the class launches run one after the other and share the overflow tables
    L.hash = off; off += al256(hash_bytes(plan));
    L.feat = off; off += plan.learned ? al256(sizeof(float) * nq * ESG_MLP_FEATURES) : 0;
    L.efq = off; off += plan.learned ? al256(sizeof(int32_t) * nq) : 0;
    L.mxq = off; off += plan.learned ? al256(sizeof(int32_t) * nq) : 0;
    L.order = off; off += al256(sizeof(int32_t) * n_items);
    L.queue = off; off += 256;   // a work counter and an item range per class
    L.total = off;
    return L;
}
}  // namespace

esg_status esg_search_prepare(const SearchLaunch &s, SearchPlan &plan) {
    const esg_index *ix = s.ix;
    const int ef = std::max(s.p.ef, 1);
    if (ef > 1024) { esg_set_error("ef > 1024"); return ESG_ERR_INVALID_ARG; }
    const bool learned = s.p.use_learned && ix->mlp_ready;
    // with the learned budget the list and visited table are sized for its ef range
    const int efk = std::max(learned ? std::max(ix->mlp_ef_hi, ef) : ef, s.k_max);
    const int st_trav = s.p.traversal;
    const void *Xt = ix->X;
    if (st_trav == ESG_BF16) Xt = ix->Xb;
    else if (st_trav == ESG_FP8E4M3) Xt = ix->X8;
    else if (st_trav != ESG_F32) { esg_set_error("unknown traversal type"); return ESG_ERR_INVALID_ARG; }
    if (Xt == nullptr) { esg_set_error("index has no rows of the requested traversal type (build with that storage)"); return ESG_ERR_INVALID_ARG; }
    // two budget classes when some queries may need a beam wider than the
    // small class's and others may not: the learned budget, or a fixed ef
    // below the class bound with a larger k_max
    const int64_t n_items = 2 * std::max<int64_t>(s.nq, 1);
    const int small_ef = env_int("ESG_SMALL_CLASS_EF", kSmallClassEf);
    plan.nclass = (small_ef > 0 && efk > small_ef && (learned || ef <= small_ef)) ? 2 : 1;
    plan.small_ef = plan.nclass == 2 ? small_ef : 0;
    const int ef_cls[2] = {plan.nclass == 2 ? small_ef : efk, efk};
    // POST on the root keeps every reached point while fewer than ef
    // in-range points are known: a long list (the baseline's own cost)
    const int lpe = s.p.post_root ? 8 : env_int("ESG_LIST_PER_EF", 2);
    for (int c = 0; c < plan.nclass; ++c) {
        esg_status pst = make_plan(ix->d, ix->R, ef_cls[c], n_items, st_trav, s.p.width, s.p.warps_per_block,
                                   s.p.hash_slots, s.p.lanes_per_row, s.p.max_registers, plan.cls[c], lpe);
        if (pst != ESG_OK) return pst;
    }
    plan.n_items = n_items;
    plan.Xt = Xt;
    plan.learned = learned;
    plan.ef = ef;
    plan.efk = efk;
    plan.scratch_bytes = scratch_layout(std::max<int64_t>(s.nq, 1), s.k_max, plan).total;
    return ESG_OK;
}

esg_status esg_search_prepare_capped(const SearchLaunch &s, size_t max_scratch, SearchPlan &plan) {
    esg_status st = esg_search_prepare(s, plan);
    if (st != ESG_OK) return st;
    const int64_t nq = std::max<int64_t>(s.nq, 1);
    auto grid_above_one = [&]() {
        for (int c = 0; c < plan.nclass; ++c) if (plan.cls[c].grid > 1) return true;
        return false;
    };
    while (plan.scratch_bytes > max_scratch && grid_above_one()) {
        for (int c = 0; c < plan.nclass; ++c) plan.cls[c].grid = std::max<int64_t>(1, plan.cls[c].grid / 2);
        plan.scratch_bytes = scratch_layout(nq, s.k_max, plan).total;
    }
    if (plan.scratch_bytes > max_scratch) {
        esg_set_error("batch too large for the fixed scratch array (reduce nq or k_max)");
        return ESG_ERR_INVALID_ARG;
    }
    return ESG_OK;
}

esg_status esg_search_enqueue(const SearchLaunch &s, const SearchPlan &plan, void *scratch_v,
                              cudaStream_t stream) {
    const esg_index *ix = s.ix;
    if (s.nq == 0) return ESG_OK;
    const int64_t n_items = 2 * s.nq;
    const ScratchLayout L = scratch_layout(s.nq, s.k_max, plan);
    unsigned char *scratch = (unsigned char *)scratch_v;
    esg_piece *pieces = (esg_piece *)(scratch + L.pieces);
    int32_t *kq = (int32_t *)(scratch + L.kq);
    int32_t *qs = (int32_t *)(scratch + L.qs);
    Cand *res = (Cand *)(scratch + L.res);
    int32_t *res_cnt = (int32_t *)(scratch + L.cnt);
    int32_t *res_status = res_cnt + n_items;
    int64_t *res_stats = (int64_t *)(scratch + L.stats);
    unsigned long long *ghash = (unsigned long long *)(scratch + L.hash);
    unsigned long long *queue = (unsigned long long *)(scratch + L.queue);   // [2] work counters
    int32_t *range = (int32_t *)(scratch + L.queue + 64);                     // [2][2] item ranges
    const size_t bytes_hash = hash_bytes(plan);

    ESG_CUDA_TRY(cudaMemsetAsync(queue, 0, 2 * sizeof(unsigned long long), stream));
    ESG_CUDA_TRY(cudaMemsetAsync(ghash, 0, bytes_hash, stream));   // tag 0: free for every item
    prep_kernel<<<ceil_div_i(s.nq, 256), 256, 0, stream>>>(esg_spec_of(ix, s.p.post_root), s.l, s.r, s.k,
                                                           s.k_max, s.nq, pieces, kq, qs);
    ESG_CUDA_TRY(cudaGetLastError());
    int32_t *ef_q = nullptr, *maxexp_q = nullptr;
    if (plan.learned) {
        ef_q = (int32_t *)(scratch + L.efq);
        maxexp_q = (int32_t *)(scratch + L.mxq);
        esg_status pst = esg_predict_budget(ix, s.p.post_root, s.queries, s.nq, s.l, s.r, s.k, s.k_max,
                                            plan.ef, (float *)(scratch + L.feat), ef_q, maxexp_q, stream);
        if (pst != ESG_OK) return pst;
        esg_prof_count(1);   // features + network, one kernel
    }
    // items longest first: a warp that takes a long search late would
    // leave the others idle at the end of the launch
    int32_t *order = (int32_t *)(scratch + L.order);
    order_items_kernel<<<1, kOrderThreads, 0, stream>>>(pieces, ef_q, kq, plan.ef, plan.small_ef, s.nq, order,
                                                        range);
    ESG_CUDA_TRY(cudaGetLastError());
    SearchArgs a;
    a.order = order;
    a.ef_q = ef_q; a.maxexp_q = maxexp_q;
    a.X = ix->X; a.adj = ix->adj; a.row_off = ix->row_off; a.entries = ix->entries; a.queries = s.queries;
    a.qidx = nullptr; a.kconst = 0; a.qshift = 1;
    a.pieces = pieces; a.kq = kq; a.n = ix->n; a.n_items = n_items;
    a.d = ix->d; a.R = ix->R; a.E = ix->E;
    a.Xv = reinterpret_cast<const uint4 *>(plan.Xt); a.scale8 = ix->scale8; a.rerank = s.p.rerank;
    a.metric = ix->metric; a.ef = plan.ef;
    a.max_exp = s.p.max_expansions > 0 ? s.p.max_expansions : 16 * plan.ef + 256;
    a.k_max = s.k_max; a.ghash = ghash;
    a.res = res; a.res_cnt = res_cnt; a.res_status = res_status; a.res_stats = res_stats;
    // the large class first: its items are the longest
    for (int c = plan.nclass - 1; c >= 0; --c) {
        const KernelPlan &kp = plan.cls[c];
        a.nvec = kp.nvec; a.width = kp.width; a.BB = kp.BB; a.LPR = kp.lpr;
        a.H = kp.H; a.C = kp.C; a.G = kp.G; a.lpe = kp.lpe;
        a.queue = queue + c;
        a.range = range + 2 * c;
        const int pidx = esg_prof_begin(stream);
        ((SearchFn)kp.fn)<<<(unsigned)kp.grid, kp.wpb * 32, kp.smem, stream>>>(a);
        const cudaError_t ce = cudaGetLastError();
        esg_prof_end(pidx, stream);
        if (ce != cudaSuccess) { esg_set_error(cudaGetErrorString(ce)); return ESG_ERR_CUDA; }
    }
    esg_prof_count(3 + plan.nclass);  // prep, order, search per class, merge
    merge_kernel<<<ceil_div_i(s.nq, 128), 128, 0, stream>>>(
        s.nq, s.k_max, kq, res, res_cnt, res_status, res_stats, qs, ix->perm, pieces,
        s.out_ids, s.out_dist, s.out_count, s.out_status, s.out_stats);
    ESG_CUDA_TRY(cudaGetLastError());
    return ESG_OK;
}

esg_status esg_launch_search(const SearchLaunch &s, cudaStream_t stream) {
    if (s.nq == 0) return ESG_OK;
    SearchPlan plan;
    esg_status st = esg_search_prepare(s, plan);
    if (st != ESG_OK) return st;
    void *scratch = nullptr;
    ESG_CUDA_TRY(esg_malloc_async((void **)&scratch, plan.scratch_bytes, stream));
    st = esg_search_enqueue(s, plan, scratch, stream);
    const cudaError_t fe = cudaFreeAsync(scratch, stream);
    if (st == ESG_OK && fe != cudaSuccess) { esg_set_error(cudaGetErrorString(fe)); st = ESG_ERR_CUDA; }
    return st;
}

// Beam search over prepared work items (graph construction): item i searches
// the piece pieces[i] for the row qidx[i] of X, keeping the best k results in
// res[i * k ..]. Entry points come from `entries` (E per node); the rows of
// rank p at level t are adj[(row_off[t] + p) * R ..].
esg_status esg_run_search_items(const float *X, int64_t n, int d, int metric, const uint32_t *adj,
                                const int64_t *row_off, int R, const int32_t *entries, int E,
                                const int64_t *qidx, const esg_piece *pieces, int64_t n_items, int ef,
                                int k, int max_exp, Cand *res, int32_t *res_cnt, int32_t *res_status,
                                int64_t *res_stats, cudaStream_t stream) {
    if (n_items == 0) return ESG_OK;
    KernelPlan plan;
    esg_status pst = make_plan(d, R, std::max(ef, k), n_items, ESG_F32, 1, 0, 0, 0, 0, plan);
    if (pst != ESG_OK) return pst;
    const size_t bytes_hash = (size_t)plan.grid * plan.wpb * plan.G * 8;
    unsigned char *scratch = nullptr;
    ESG_CUDA_TRY(esg_malloc_async((void **)&scratch, bytes_hash + 256, stream));
    unsigned long long *queue = (unsigned long long *)scratch;
    unsigned long long *ghash = (unsigned long long *)(scratch + 256);
    esg_status st = ESG_OK;
    cudaError_t ce = cudaMemsetAsync(queue, 0, sizeof(unsigned long long), stream);
    if (ce == cudaSuccess) ce = cudaMemsetAsync(ghash, 0, bytes_hash, stream);
    if (ce == cudaSuccess) {
        SearchArgs a;
        a.X = X; a.adj = adj; a.row_off = row_off; a.entries = entries; a.queries = X; a.qidx = qidx;
        a.pieces = pieces; a.kq = nullptr; a.kconst = k; a.qshift = 0;
        a.ef_q = nullptr; a.maxexp_q = nullptr;
        a.n = n; a.n_items = n_items; a.d = d; a.nvec = plan.nvec; a.LPR = plan.lpr; a.R = R; a.E = E;
        a.Xv = reinterpret_cast<const uint4 *>(X); a.scale8 = nullptr; a.rerank = 0;
        a.width = plan.width; a.BB = plan.BB;
        a.metric = metric; a.ef = ef; a.max_exp = max_exp > 0 ? max_exp : 16 * ef + 256;
        a.k_max = k; a.H = plan.H; a.C = plan.C; a.lpe = plan.lpe; a.ghash = ghash; a.G = plan.G; a.queue = queue;
        a.res = res; a.res_cnt = res_cnt; a.res_status = res_status; a.res_stats = res_stats;
        ((SearchFn)plan.fn)<<<(unsigned)plan.grid, plan.wpb * 32, plan.smem, stream>>>(a);
        ce = cudaGetLastError();
    }
    if (ce != cudaSuccess) { esg_set_error(cudaGetErrorString(ce)); st = ESG_ERR_CUDA; }
    cudaError_t fe = cudaFreeAsync(scratch, stream);
    if (st == ESG_OK && fe != cudaSuccess) { esg_set_error(cudaGetErrorString(fe)); st = ESG_ERR_CUDA; }
    return st;
}

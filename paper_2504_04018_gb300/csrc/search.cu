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
// the worst of Q), sort them (bitonic, 64 wide) and merge them into the list.
#include "esg_internal.cuh"
#include "decompose.cuh"

#include <algorithm>
#include <cstdlib>

namespace {

constexpr int kBatch = 64;  // neighbours handled per expansion (R <= 64 per pass)

struct WarpSmem {
    uint32_t *hash;
    Cand *list;
    Cand *list2;
    Cand *batch;
    uint32_t *nbuf;
    int *hcount;
};

__device__ __forceinline__ uint32_t hash_mix(uint32_t x) {
    x ^= x >> 16; x *= 0x7feb352dU; x ^= x >> 15; x *= 0x846ca68bU; x ^= x >> 16;
    return x;
}

// Visited set of one beam search: an open-addressing table in shared memory
// backed, once it reaches its load limit, by a larger table in a per-warp
// global-memory slot. visit() returns false iff `id` was already visited.
// Only when both tables are at their limits is an id reported as new without
// being stored (`saturated`; the list de-duplication then catches repeats).
struct Visited {
    uint32_t *hs;   // shared table, hmask + 1 slots
    uint32_t hmask;
    int *hcount;
    int hlimit;
    uint32_t *hg;   // global overflow table, gmask + 1 slots (all ESG_NONE when unused)
    uint32_t gmask;
    int *gcount;
    int glimit;
};

__device__ __forceinline__ bool visit(const Visited &v, uint32_t id, bool *saturated, bool *used_g) {
    uint32_t h = hash_mix(id) & v.hmask;
    for (uint32_t probe = 0; probe <= v.hmask; ++probe) {
        const uint32_t slot = (h + probe) & v.hmask;
        const uint32_t cur = v.hs[slot];
        if (cur == id) return false;
        if (cur == ESG_NONE) {
            if (*(volatile int *)v.hcount >= v.hlimit) break;   // continue in the global table
            const uint32_t prev = atomicCAS(&v.hs[slot], ESG_NONE, id);
            if (prev == ESG_NONE) { atomicAdd(v.hcount, 1); return true; }
            if (prev == id) return false;
        }
    }
    if (v.hg == nullptr) { *saturated = true; return true; }
    *used_g = true;
    h = hash_mix(id ^ 0x9e3779b9u) & v.gmask;
    for (uint32_t probe = 0; probe <= v.gmask; ++probe) {
        const uint32_t slot = (h + probe) & v.gmask;
        const uint32_t cur = *(volatile uint32_t *)&v.hg[slot];
        if (cur == id) return false;
        if (cur == ESG_NONE) {
            if (*(volatile int *)v.gcount >= v.glimit) { *saturated = true; return true; }
            const uint32_t prev = atomicCAS(&v.hg[slot], ESG_NONE, id);
            if (prev == ESG_NONE) { atomicAdd(v.gcount, 1); return true; }
            if (prev == id) return false;
        }
    }
    *saturated = true;
    return true;
}

// Storage types of the traversal rows (esg_dtype): elements per 16-byte vector.
template <int ST> struct Store;
template <> struct Store<ESG_F32> { static constexpr int EPV = 4; };
template <> struct Store<ESG_BF16> { static constexpr int EPV = 8; };
template <> struct Store<ESG_FP8E4M3> { static constexpr int EPV = 16; };

// Accumulate the distance terms of one 16-byte vector of a row against the
// query slice qs[0..EPV) (FP32 accumulation; FP8 codes times the row scale).
template <int ST>
__device__ __forceinline__ float accum_vec(const uint4 &raw, const float *qs, float scale, int metric,
                                           float acc) {
    float x[Store<ST>::EPV];
    if (ST == ESG_F32) {
        x[0] = __uint_as_float(raw.x); x[1] = __uint_as_float(raw.y);
        x[2] = __uint_as_float(raw.z); x[3] = __uint_as_float(raw.w);
    } else if (ST == ESG_BF16) {
        const uint32_t w4[4] = {raw.x, raw.y, raw.z, raw.w};
#pragma unroll
        for (int t = 0; t < 4; ++t) {
            x[2 * t] = __uint_as_float(w4[t] << 16);
            x[2 * t + 1] = __uint_as_float(w4[t] & 0xFFFF0000u);
        }
    } else {
        const uint32_t w4[4] = {raw.x, raw.y, raw.z, raw.w};
#pragma unroll
        for (int t = 0; t < 4; ++t) {
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                __nv_fp8x2_storage_t pair = (__nv_fp8x2_storage_t)((w4[t] >> (16 * h)) & 0xFFFFu);
                __half2_raw hr = __nv_cvt_fp8x2_to_halfraw2(pair, __NV_E4M3);
                float2 f = __half22float2(*reinterpret_cast<__half2 *>(&hr));
                x[4 * t + 2 * h] = f.x * scale;
                x[4 * t + 2 * h + 1] = f.y * scale;
            }
        }
    }
    const float4 *q4 = reinterpret_cast<const float4 *>(qs);
#pragma unroll
    for (int e = 0; e < Store<ST>::EPV; e += 4) {
        const float4 q = q4[e / 4];
        if (metric == ESG_L2SQ) {
            float a = q.x - x[e], b = q.y - x[e + 1], c = q.z - x[e + 2], d = q.w - x[e + 3];
            acc = fmaf(a, a, acc); acc = fmaf(b, b, acc); acc = fmaf(c, c, acc); acc = fmaf(d, d, acc);
        } else {
            acc = fmaf(q.x, x[e], acc); acc = fmaf(q.y, x[e + 1], acc);
            acc = fmaf(q.z, x[e + 2], acc); acc = fmaf(q.w, x[e + 3], acc);
        }
    }
    return acc;
}

// Distances from the query (FP32, staged in shared memory `qs`) to the rows
// listed in nbuf[0..m), written to batch[0..m). Rows are nvec 16-byte
// vectors; LPR lanes share a row, each loading VPL vectors, and the loads of
// U passes are all issued before any reduction.
template <int ST, int VPL>
__device__ __forceinline__ void eval_rows(const uint4 *__restrict__ Xv, const float *__restrict__ scale8,
                                          int nvec, int LPR, const float *qs, const uint32_t *nbuf,
                                          int m, Cand *batch, int metric) {
    constexpr int EPV = Store<ST>::EPV;
    const int lane = threadIdx.x & 31;
    const int s = lane & (LPR - 1);
    const int g = lane / LPR;
    const int rows_per_pass = 32 / LPR;
    // vectors in flight per lane scaled so that at most ~16 FP32-equivalent
    // vectors are decoded per pass
    constexpr int W = ST == ESG_F32 ? 1 : (ST == ESG_BF16 ? 2 : 4);
    constexpr int U0 = 16 / (VPL * W);
    constexpr int U = U0 < 1 ? 1 : (U0 > 8 ? 8 : U0);
    for (int base = 0; base < m; base += rows_per_pass * U) {
        uint4 xv[U][VPL];
        uint32_t id[U];
        float sc[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int row = base + u * rows_per_pass + g;
            id[u] = row < m ? nbuf[row] : ESG_NONE;
            sc[u] = 1.f;
            if (id[u] != ESG_NONE) {
                const uint4 *p = Xv + (size_t)id[u] * nvec + s;
#pragma unroll
                for (int v = 0; v < VPL; ++v) xv[u][v] = __ldg(p + v * LPR);
                if (ST == ESG_FP8E4M3) sc[u] = __ldg(scale8 + id[u]);
            } else {
#pragma unroll
                for (int v = 0; v < VPL; ++v) xv[u][v] = make_uint4(0, 0, 0, 0);
            }
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
            float acc = 0.f;
#pragma unroll
            for (int v = 0; v < VPL; ++v)
                acc = accum_vec<ST>(xv[u][v], qs + (s + v * LPR) * EPV, sc[u], metric, acc);
            acc = warp_sum_group(acc, LPR);
            const int row = base + u * rows_per_pass + g;
            if (s == 0 && row < m) batch[row] = Cand{metric == ESG_L2SQ ? acc : -acc, id[u]};
        }
    }
    __syncwarp();
}

// Exact FP32 distances of the rows in nbuf[0..m) (re-rank of candidates
// found with low-precision rows): 8 lanes per row.
__device__ __forceinline__ void eval_rows_fp32(const float *__restrict__ X, int d, const float *qs,
                                               const uint32_t *nbuf, int m, Cand *out, int metric) {
    const int lane = threadIdx.x & 31;
    const int s = lane & 7, g = lane >> 3;
    const int nv = d / 4;
    const float4 *q4 = reinterpret_cast<const float4 *>(qs);
    for (int base = 0; base < m; base += 4) {
        const int row = base + g;
        const uint32_t id = row < m ? nbuf[row] : ESG_NONE;
        float acc = 0.f;
        if (id != ESG_NONE) {
            const float4 *x4 = reinterpret_cast<const float4 *>(X + (size_t)id * d);
#pragma unroll 4
            for (int v = s; v < nv; v += 8) {
                const float4 x = __ldg(x4 + v), q = q4[v];
                if (metric == ESG_L2SQ) {
                    float a = q.x - x.x, b = q.y - x.y, c = q.z - x.z, e = q.w - x.w;
                    acc = fmaf(a, a, acc); acc = fmaf(b, b, acc); acc = fmaf(c, c, acc); acc = fmaf(e, e, acc);
                } else {
                    acc = fmaf(q.x, x.x, acc); acc = fmaf(q.y, x.y, acc);
                    acc = fmaf(q.z, x.z, acc); acc = fmaf(q.w, x.w, acc);
                }
            }
        }
        acc = warp_sum_group(acc, 8);
        if (s == 0 && row < m) out[row] = Cand{metric == ESG_L2SQ ? acc : -acc, id};
    }
    __syncwarp();
}

// Merge the sorted, duplicate-free batch B[0..b) into the sorted list
// A[0..a), writing O (capacity C). Returns the new length min(a + b, C).
__device__ __forceinline__ int warp_merge(const Cand *A, int a, const Cand *B, int b, Cand *O, int C) {
    const int lane = threadIdx.x & 31;
    for (int i = lane; i < a; i += 32) {
        Cand x = A[i];
        int pos = i + lower_rank(B, b, x);
        if (pos < C) O[pos] = x;
    }
    for (int j = lane; j < b; j += 32) {
        Cand x = B[j];
        int pos = j + lower_rank(A, a, x);
        if (pos < C) O[pos] = x;
    }
    __syncwarp();
    return min(a + b, C);
}

// List state of one beam search.
struct ListState {
    int len;       // items in the list
    int qn;        // in-range items kept (<= ef)
    Cand qworst;   // the ef-th in-range item when qn == ef, else +inf
    int first;     // position of the best unexpanded item, -1 if none
};

// Cut the list after its ef-th in-range item (Q keeps the best ef; nothing
// behind it can be expanded or returned) and refresh |Q| and the worst of Q.
__device__ __forceinline__ void truncate_list(const Cand *list, ListState &st, int ef,
                                              uint32_t pl, uint32_t pr) {
    const int lane = threadIdx.x & 31;
    int seen = 0;
    st.qn = 0;
    st.qworst = Cand{INFINITY, ESG_NONE};
    st.first = -1;
    for (int base = 0; base < st.len; base += 32) {
        const int i = base + lane;
        const uint32_t raw = i < st.len ? list[i].id : ESG_NONE;
        const uint32_t id = raw & ESG_ID_MASK;
        const bool inr = i < st.len && id >= pl && id <= pr;
        const unsigned bal = __ballot_sync(0xffffffffu, inr);
        const unsigned unexp = __ballot_sync(0xffffffffu, i < st.len && !(raw & ESG_EXPANDED));
        const int c = __popc(bal);
        if (seen + c >= ef) {
            // position of the (ef - seen)-th set bit of bal
            const int need = ef - seen;
            unsigned b = bal;
            for (int t = 1; t < need; ++t) b &= b - 1;
            const int pos = base + __ffs(b) - 1;
            st.len = pos + 1;
            st.qn = ef;
            st.qworst = list[pos];
            const unsigned keep_unexp = unexp & (pos - base == 31 ? 0xffffffffu : ((1u << (pos - base + 1)) - 1));
            if (st.first < 0 && keep_unexp) st.first = base + __ffs(keep_unexp) - 1;
            return;
        }
        if (st.first < 0 && unexp) st.first = base + __ffs(unexp) - 1;
        seen += c;
    }
    st.qn = seen;
}

// Admitted candidates sit in batch[0..64) (rejected slots hold +inf). Sort
// them and merge them into `list`, returning the merged list (list or list2)
// after truncation. Batches of at most 32 are sorted in registers.
__device__ __forceinline__ Cand *admit_batch(Cand *batch, Cand *cbuf, Cand *list, Cand *list2,
                                             ListState &st, int ef, int C, uint32_t pl, uint32_t pr,
                                             int &status) {
    const int lane = threadIdx.x & 31;
    const Cand x0 = batch[lane], x1 = batch[lane + 32];
    const bool k0 = x0.id != ESG_NONE, k1 = x1.id != ESG_NONE;
    const unsigned b0 = __ballot_sync(0xffffffffu, k0), b1 = __ballot_sync(0xffffffffu, k1);
    const int b = __popc(b0) + __popc(b1);
    if (b == 0) return list;
    const Cand *B;
    if (b <= 32) {
        const unsigned below = (1u << lane) - 1;
        if (k0) cbuf[__popc(b0 & below)] = x0;
        if (k1) cbuf[__popc(b0) + __popc(b1 & below)] = x1;
        __syncwarp();
        float d = lane < b ? cbuf[lane].d : INFINITY;
        uint32_t id = lane < b ? cbuf[lane].id : ESG_NONE;
        __syncwarp();
        warp_sort32_reg(d, id);
        cbuf[lane] = Cand{d, id};
        __syncwarp();
        B = cbuf;
    } else {
        warp_sort64(batch);
        B = batch;
    }
    if (st.len + b > C) status |= ESG_Q_OVERFLOW;
    st.len = warp_merge(list, st.len, B, b, list2, C);
    truncate_list(list2, st, ef, pl, pr);
    return list2;
}

struct SearchArgs {
    const float *X;        // FP32 rows (re-rank, and traversal when st == F32)
    const uint4 *Xv;       // traversal rows (FP32, BF16 or FP8) as 16-byte vectors
    const float *scale8;   // FP8 per-row scales
    int rerank;
    const uint32_t *adj;
    const int32_t *entries;
    const float *queries;
    const int64_t *qidx;   // optional: query row of an item (build: the inserted point)
    const esg_piece *pieces;
    const int32_t *kq;     // per-query k (validated), 0 = invalid; null = kconst
    int kconst;
    int qshift;            // query of item i = i >> qshift (2 pieces per query: 1)
    int64_t n;
    int64_t n_items;
    int d, nvec, LPR, R, E, metric;
    int ef, max_exp, k_max;
    int H, C;
    uint32_t *ghash;       // global overflow visited tables, G slots per warp (all ESG_NONE), or null
    int G;
    unsigned long long *queue;  // atomic work counter
    Cand *res;             // [n_items, k_max]
    int32_t *res_cnt;      // [n_items]
    int32_t *res_status;   // [n_items]
    int64_t *res_stats;    // [n_items, 4]
};

template <int ST, int VPL>
__global__ void __launch_bounds__(64, 8)
search_kernel(SearchArgs a) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int lane = threadIdx.x & 31;
    const int wib = threadIdx.x >> 5;
    const int wpb = blockDim.x >> 5;
    const size_t qbytes = ((size_t)a.d * 4 + 15) & ~(size_t)15;
    const size_t per_warp = (size_t)a.H * 4 + (size_t)a.C * 8 * 2 + kBatch * 8 + 32 * 8 +
                            kBatch * 4 + 16 + qbytes;
    unsigned char *base = smem_raw + per_warp * wib;
    WarpSmem w;
    size_t off = 0;
    w.list = (Cand *)(base + off); off += (size_t)a.C * 8;
    w.list2 = (Cand *)(base + off); off += (size_t)a.C * 8;
    w.batch = (Cand *)(base + off); off += kBatch * 8;
    Cand *cbuf = (Cand *)(base + off); off += 32 * 8;
    w.nbuf = (uint32_t *)(base + off); off += kBatch * 4;
    w.hcount = (int *)(base + off); off += 16;
    float *qs = (float *)(base + off); off += qbytes;
    const int gwarp = blockIdx.x * wpb + wib;
    w.hash = (uint32_t *)(base + off);
    Visited vis;
    vis.hs = w.hash;
    vis.hmask = (uint32_t)a.H - 1;
    vis.hcount = w.hcount;
    vis.hlimit = (a.H * 3) / 4;
    vis.hg = a.ghash ? a.ghash + (size_t)gwarp * a.G : nullptr;
    vis.gmask = (uint32_t)a.G - 1;
    vis.gcount = w.hcount + 1;
    vis.glimit = (a.G * 3) / 4;

    for (;;) {
        int64_t item = 0;
        if (lane == 0) item = (int64_t)atomicAdd(a.queue, 1ULL);
        item = __shfl_sync(0xffffffffu, item, 0);
        if (item >= a.n_items) break;
        const int64_t qi = item >> a.qshift;
        const esg_piece pc = a.pieces[item];
        const int kq = a.kq ? a.kq[qi] : a.kconst;
        int64_t n_exp = 0, n_eval = 0, n_oor = 0, n_rr = 0;
        int status = 0;
        if (pc.kind == ESG_PIECE_NONE || kq <= 0) {
            if (lane == 0) { a.res_cnt[item] = 0; a.res_status[item] = 0; }
            if (lane < 4) a.res_stats[item * 4 + lane] = 0;
            continue;
        }
        const uint32_t pl = (uint32_t)pc.pl, pr = (uint32_t)pc.pr;
        const bool is_graph = pc.kind == ESG_PIECE_GRAPH;
        // low-precision scans keep ef candidates for the FP32 re-rank
        const bool do_rerank = ST != ESG_F32 && a.rerank;
        const int ef = (is_graph || do_rerank) ? max(a.ef, kq) : kq;

        // query in shared memory (FP32)
        {
            const int64_t qrow = a.qidx ? a.qidx[item] : qi;
            const float4 *q4 = reinterpret_cast<const float4 *>(a.queries + qrow * (int64_t)a.d);
            for (int v = lane; v < a.d / 4; v += 32) reinterpret_cast<float4 *>(qs)[v] = __ldg(q4 + v);
            __syncwarp();
        }
        ListState st{0, 0, Cand{INFINITY, ESG_NONE}, -1};
        Cand *list = w.list, *list2 = w.list2;
        bool saturated = false;

        if (!is_graph) {
            // Leaf piece: exact scan of [pl, pr] (Algorithm 4, first branch).
            for (int64_t c0 = pl; c0 <= (int64_t)pr; c0 += kBatch) {
                const int m = (int)(((int64_t)pr - c0 + 1) < kBatch ? ((int64_t)pr - c0 + 1) : kBatch);
                for (int j = lane; j < m; j += 32) w.nbuf[j] = (uint32_t)(c0 + j);
                __syncwarp();
                eval_rows<ST, VPL>(a.Xv, a.scale8, a.nvec, a.LPR, qs, w.nbuf, m, w.batch, a.metric);
                n_eval += m;
                for (int j = lane; j < kBatch; j += 32) {
                    const bool keep = j < m && (st.qn < ef || cand_less(w.batch[j], st.qworst));
                    if (!keep) w.batch[j] = Cand{INFINITY, ESG_NONE};
                }
                __syncwarp();
                Cand *nl = admit_batch(w.batch, cbuf, list, list2, st, ef, a.C, pl, pr, status);
                if (nl != list) { list2 = list; list = nl; }
            }
        } else {
            // Graph piece: Algorithm 1 with POST filtering to [pl, pr].
            for (int i = lane; i < a.H; i += 32) w.hash[i] = ESG_NONE;
            if (lane == 0) { w.hcount[0] = 0; w.hcount[1] = 0; }
            __syncwarp();
            bool used_g = false;
            const uint32_t *adj = a.adj + (size_t)pc.depth * (size_t)a.n * a.R;
            // entry points: into P, and into Q when in range
            {
                uint32_t e = ESG_NONE;
                if (lane < a.E) {
                    const int32_t v = a.entries[(size_t)pc.heap * a.E + lane];
                    if (v >= 0 && v < a.n) e = (uint32_t)v;
                }
                const bool nw = e != ESG_NONE && visit(vis, e, &saturated, &used_g);
                const unsigned bal = __ballot_sync(0xffffffffu, nw);
                if (nw) w.nbuf[__popc(bal & ((1u << lane) - 1))] = e;
                const int m = __popc(bal);
                __syncwarp();
                eval_rows<ST, VPL>(a.Xv, a.scale8, a.nvec, a.LPR, qs, w.nbuf, m, w.batch, a.metric);
                n_eval += m;
                for (int j = lane; j < kBatch; j += 32) {
                    if (j >= m) w.batch[j] = Cand{INFINITY, ESG_NONE};
                    else n_oor += (w.batch[j].id < pl || w.batch[j].id > pr);
                }
                __syncwarp();
                Cand *nl = admit_batch(w.batch, cbuf, list, list2, st, ef, a.C, pl, pr, status);
                if (nl != list) { list2 = list; list = nl; }
            }
            // all items before `hint` are expanded
            int hint = st.first < 0 ? st.len : st.first;
            for (;;) {
                // best unexpanded candidate
                int pos = -1;
                for (int b0 = hint & ~31; b0 < st.len; b0 += 32) {
                    const int i = b0 + lane;
                    const bool f = i >= hint && i < st.len && !(list[i].id & ESG_EXPANDED);
                    const unsigned bal = __ballot_sync(0xffffffffu, f);
                    if (bal) { pos = b0 + __ffs(bal) - 1; break; }
                }
                if (pos < 0) break;
                if (n_exp >= a.max_exp) { status |= ESG_Q_TRUNCATED; break; }
                const uint32_t u = list[pos].id & ESG_ID_MASK;
                const bool u_in = u >= pl && u <= pr;
                __syncwarp();
                if (u_in) {
                    if (lane == 0) list[pos].id = u | ESG_EXPANDED;
                    hint = pos + 1;
                } else {
                    // an expanded out-of-range point is neither in Q nor in P
                    const int cnt = st.len - 1 - pos;
                    for (int b0 = 0; b0 < cnt; b0 += 32) {
                        const bool act = b0 + lane < cnt;
                        Cand nx;
                        if (act) nx = list[pos + b0 + lane + 1];
                        __syncwarp();
                        if (act) list[pos + b0 + lane] = nx;
                        __syncwarp();
                    }
                    st.len -= 1;
                    hint = pos;
                }
                __syncwarp();
                ++n_exp;
                // neighbours of u, in chunks of 64
                const uint32_t *row = adj + (size_t)u * a.R;
                for (int c64 = 0; c64 < a.R; c64 += 64) {
                    uint32_t v0 = c64 + lane < a.R ? __ldg(row + c64 + lane) : ESG_NONE;
                    uint32_t v1 = c64 + lane + 32 < a.R ? __ldg(row + c64 + lane + 32) : ESG_NONE;
                    if (v0 >= (uint64_t)a.n) v0 = ESG_NONE;   // malformed imported graph: ignore
                    if (v1 >= (uint64_t)a.n) v1 = ESG_NONE;
                    const bool n0 = v0 != ESG_NONE && visit(vis, v0, &saturated, &used_g);
                    const bool n1 = v1 != ESG_NONE && visit(vis, v1, &saturated, &used_g);
                    const unsigned b0 = __ballot_sync(0xffffffffu, n0);
                    const unsigned b1 = __ballot_sync(0xffffffffu, n1);
                    const int c0 = __popc(b0);
                    if (n0) w.nbuf[__popc(b0 & ((1u << lane) - 1))] = v0;
                    if (n1) w.nbuf[c0 + __popc(b1 & ((1u << lane) - 1))] = v1;
                    const int m = c0 + __popc(b1);
                    __syncwarp();
                    if (m == 0) continue;
                    eval_rows<ST, VPL>(a.Xv, a.scale8, a.nvec, a.LPR, qs, w.nbuf, m, w.batch, a.metric);
                    n_eval += m;
                    // Algorithm 1's admission test, then de-duplication against
                    // the list (only needed once the visited set saturates)
                    const bool sat = __any_sync(0xffffffffu, saturated);
                    for (int j = lane; j < kBatch; j += 32) {
                        bool keep = false;
                        if (j < m) {
                            const Cand x = w.batch[j];
                            n_oor += (x.id < pl || x.id > pr);
                            keep = st.qn < ef || cand_less(x, st.qworst);
                            if (keep && sat) {
                                const int p = lower_rank(list, st.len, x);
                                if (p < st.len && cand_eq(list[p], x)) keep = false;
                            }
                        }
                        if (!keep) w.batch[j] = Cand{INFINITY, ESG_NONE};
                    }
                    __syncwarp();
                    Cand *nl = admit_batch(w.batch, cbuf, list, list2, st, ef, a.C, pl, pr, status);
                    if (nl != list) {
                        list2 = list; list = nl;
                        hint = st.first < 0 ? st.len : st.first;
                    }
                }  // neighbour chunk
            }
            if (__any_sync(0xffffffffu, saturated)) status |= ESG_Q_OVERFLOW;
            if (__any_sync(0xffffffffu, used_g)) {
                // leave the overflow table clean for the warp's next item
                for (int i = lane; i < a.G; i += 32) vis.hg[i] = ESG_NONE;
                __syncwarp();
            }
        }
        // FP32 re-rank of the final in-range candidates found on low-precision rows
        if (do_rerank && st.len > 0) {
            int cnt = 0;
            for (int b0 = 0; b0 < st.len; b0 += 32) {
                const int i = b0 + lane;
                const uint32_t id = i < st.len ? (list[i].id & ESG_ID_MASK) : ESG_NONE;
                const bool inr = i < st.len && id >= pl && id <= pr;
                const unsigned bal = __ballot_sync(0xffffffffu, inr);
                const int pos = cnt + __popc(bal & ((1u << lane) - 1));
                if (inr && pos < ef) list2[pos] = Cand{0.f, id};
                cnt += __popc(bal);
                if (cnt >= ef) break;
            }
            cnt = min(cnt, ef);
            __syncwarp();
            for (int c0 = 0; c0 < cnt; c0 += kBatch) {
                const int m = min(kBatch, cnt - c0);
                for (int j = lane; j < m; j += 32) w.nbuf[j] = list2[c0 + j].id;
                __syncwarp();
                eval_rows_fp32(a.X, a.d, qs, w.nbuf, m, list2 + c0, a.metric);
            }
            n_rr += cnt;
            const int P = next_pow2_int(max(cnt, 2));
            for (int j = cnt + lane; j < P; j += 32) list2[j] = Cand{INFINITY, ESG_NONE};
            __syncwarp();
            warp_sort_pow2(list2, P);
            Cand *t = list; list = list2; list2 = t;
            st.len = cnt;
        }
        // emit the first min(k, |Q|) in-range items
        {
            int written = 0;
            Cand *out = a.res + item * (int64_t)a.k_max;
            for (int b0 = 0; b0 < st.len && written < kq; b0 += 32) {
                const int i = b0 + lane;
                const uint32_t id = i < st.len ? (list[i].id & ESG_ID_MASK) : ESG_NONE;
                const bool inr = i < st.len && id >= pl && id <= pr;
                const unsigned bal = __ballot_sync(0xffffffffu, inr);
                const int pos = written + __popc(bal & ((1u << lane) - 1));
                if (inr && pos < kq) out[pos] = Cand{list[i].d, id};
                written += __popc(bal);
            }
            written = min(written, kq);
            n_exp = __shfl_sync(0xffffffffu, n_exp, 0);
            for (int o = 16; o > 0; o >>= 1) n_oor += __shfl_xor_sync(0xffffffffu, n_oor, o);
            if (lane == 0) {
                a.res_cnt[item] = written;
                a.res_status[item] = status;
                a.res_stats[item * 4 + 0] = n_exp;
                a.res_stats[item * 4 + 1] = n_eval;
                a.res_stats[item * 4 + 2] = n_oor;
                a.res_stats[item * 4 + 3] = n_rr;
            }
        }
        __syncwarp();
    }
}

// Validate queries and decompose their ranges (one thread per query).
__global__ void prep_kernel(int64_t n, int32_t leaf, const int64_t *l, const int64_t *r,
                            const int32_t *k, int32_t k_max, int64_t nq, esg_piece *pieces,
                            int32_t *kq, int32_t *qstatus) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= nq) return;
    int64_t lq = l[i], rq = r[i];
    int kk = k ? k[i] : k_max;
    esg_piece pcs[2];
    int cnt = 0;
    bool ok = kk >= 1 && kk <= k_max && lq >= 0 && lq <= rq && rq < n;
    if (ok) cnt = esg_decompose_one(n, leaf, lq, rq, pcs);
    if (!ok || cnt <= 0) {
        pcs[0].kind = ESG_PIECE_NONE; pcs[1].kind = ESG_PIECE_NONE;
        kk = 0;
    }
    pieces[2 * i] = pcs[0];
    pieces[2 * i + 1] = pcs[1];
    kq[i] = kk;
    qstatus[i] = (ok && cnt > 0) ? 0 : ESG_Q_INVALID;
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
        int64_t np = (pieces[2 * i].kind != ESG_PIECE_NONE) + (pieces[2 * i + 1].kind != ESG_PIECE_NONE);
        for (int c = 0; c < 4; ++c)
            out_stats[i * 5 + c] = k > 0 ? res_stats[2 * i * 4 + c] + res_stats[(2 * i + 1) * 4 + c] : 0;
        out_stats[i * 5 + 4] = np;
    }
}

__global__ void decompose_kernel(int64_t n, int32_t leaf, const int64_t *l, const int64_t *r,
                                 int64_t nq, esg_piece *out, int32_t *npieces) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= nq) return;
    esg_piece p[2];
    int c = esg_decompose_one(n, leaf, l[i], r[i], p);
    out[2 * i] = p[0];
    out[2 * i + 1] = p[1];
    npieces[i] = c < 0 ? 0 : c;
}

typedef void (*SearchFn)(SearchArgs);

SearchFn pick_search(int st, int vpl) {
    if (st == ESG_F32) {
        switch (vpl) {
            case 1: return search_kernel<ESG_F32, 1>;
            case 2: return search_kernel<ESG_F32, 2>;
            case 3: return search_kernel<ESG_F32, 3>;
            case 4: return search_kernel<ESG_F32, 4>;
            case 6: return search_kernel<ESG_F32, 6>;
            case 8: return search_kernel<ESG_F32, 8>;
        }
    } else if (st == ESG_BF16) {
        switch (vpl) {
            case 1: return search_kernel<ESG_BF16, 1>;
            case 2: return search_kernel<ESG_BF16, 2>;
            case 3: return search_kernel<ESG_BF16, 3>;
            case 4: return search_kernel<ESG_BF16, 4>;
            case 6: return search_kernel<ESG_BF16, 6>;
        }
    } else if (st == ESG_FP8E4M3) {
        switch (vpl) {
            case 1: return search_kernel<ESG_FP8E4M3, 1>;
            case 2: return search_kernel<ESG_FP8E4M3, 2>;
            case 3: return search_kernel<ESG_FP8E4M3, 3>;
        }
    }
    return nullptr;
}

int env_int(const char *name, int dflt) {
    const char *v = getenv(name);
    return v && *v ? atoi(v) : dflt;
}

// Launch shape and shared-memory plan of the beam-search kernel.
struct SearchPlan {
    SearchFn fn;
    int vpl, lpr, C, H, G, wpb, nvec;
    size_t smem;
    int64_t grid;
};

}  // namespace
int esg_pick_vpl(int d, int *lpr);
namespace {

esg_status make_plan(int d, int R, int efk, int64_t n_items, int st, SearchPlan &pl) {
    const int esize = st == ESG_BF16 ? 2 : (st == ESG_FP8E4M3 ? 1 : 4);
    if ((d * esize) % 16 != 0 || d % 4 != 0) { esg_set_error("row size not a multiple of 16 bytes"); return ESG_ERR_UNSUPPORTED; }
    pl.nvec = d * esize / 16;
    pl.vpl = esg_pick_vpl(pl.nvec * 4, &pl.lpr);
    if (pl.vpl == 0) { esg_set_error("unsupported dimension"); return ESG_ERR_UNSUPPORTED; }
    if (R > 128) { esg_set_error("R > 128"); return ESG_ERR_UNSUPPORTED; }
    pl.fn = pick_search(st, pl.vpl);
    if (pl.fn == nullptr) { esg_set_error("no search kernel for this dimension and row type"); return ESG_ERR_UNSUPPORTED; }
    pl.C = ((std::max(8 * efk, 256) + 31) / 32) * 32;
    if (pl.C > 4096) pl.C = 4096;
    // shared visited table: ~64 slots per unit of beam width, 2K..8K slots;
    // the global overflow table takes what does not fit
    const int per_ef = env_int("ESG_HASH_PER_EF", 64);
    const int hmax = env_int("ESG_HASH_MAX", 8192);
    pl.H = 2048;
    while (pl.H < per_ef * efk && pl.H < hmax) pl.H <<= 1;
    while (pl.H < 4 * R) pl.H <<= 1;
    pl.G = 16384;
    while (pl.G < 256 * efk && pl.G < (1 << 20)) pl.G <<= 1;
    pl.wpb = 2;
    pl.smem = ((size_t)pl.H * 4 + (size_t)pl.C * 16 + kBatch * 12 + 32 * 8 + 16 +
               (((size_t)d * 4 + 15) & ~(size_t)15)) * pl.wpb;
    int dev = 0, sms = 0, per_sm = 0;
    ESG_CUDA_TRY(cudaGetDevice(&dev));
    ESG_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    ESG_CUDA_TRY(cudaFuncSetAttribute(pl.fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)pl.smem));
    ESG_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, pl.fn, pl.wpb * 32, pl.smem));
    if (per_sm < 1) { esg_set_error("search kernel does not fit on an SM"); return ESG_ERR_UNSUPPORTED; }
    pl.grid = std::min<int64_t>((int64_t)sms * per_sm, (n_items + pl.wpb - 1) / pl.wpb);
    if (pl.grid < 1) pl.grid = 1;
    return ESG_OK;
}

}  // namespace

// Lanes per row (LPR) and float4 per lane (VPL) for rows of d floats: prefer
// 8 lanes per row (4 rows per warp instruction, short shuffle reductions);
// wider rows use 16 or 32 lanes.
int esg_pick_vpl(int d, int *lpr) {
    if (d % 4) return 0;
    const int nvec = d / 4;
    const int lprs[] = {8, 4, 2, 1, 16, 32};
    for (int L : lprs) {
        if (nvec % L) continue;
        const int v = nvec / L;
        if (v == 1 || v == 2 || v == 3 || v == 4 || v == 6 || v == 8) { *lpr = L; return v; }
    }
    return 0;
}

esg_status esg_launch_decompose(int64_t n, int32_t leaf_size, const int64_t *l, const int64_t *r,
                                int64_t nq, esg_piece *pieces, int32_t *npieces, cudaStream_t stream) {
    if (nq == 0) return ESG_OK;
    decompose_kernel<<<ceil_div_i(nq, 256), 256, 0, stream>>>(n, leaf_size, l, r, nq, pieces, npieces);
    ESG_CUDA_TRY(cudaGetLastError());
    return ESG_OK;
}

esg_status esg_launch_search(const SearchLaunch &s, cudaStream_t stream) {
    const esg_index *ix = s.ix;
    if (s.nq == 0) return ESG_OK;
    int ef = std::max(s.p.ef, 1);
    if (ef > 1024) { esg_set_error("ef > 1024"); return ESG_ERR_INVALID_ARG; }
    const int efk = std::max(ef, s.k_max);
    const int64_t n_items = 2 * s.nq;
    SearchPlan plan;
    const int st_trav = s.p.traversal;
    const void *Xt = ix->X;
    if (st_trav == ESG_BF16) Xt = ix->Xb;
    else if (st_trav == ESG_FP8E4M3) Xt = ix->X8;
    else if (st_trav != ESG_F32) { esg_set_error("unknown traversal type"); return ESG_ERR_INVALID_ARG; }
    if (Xt == nullptr) { esg_set_error("index has no rows of the requested traversal type (build with that storage)"); return ESG_ERR_INVALID_ARG; }
    esg_status pst = make_plan(ix->d, ix->R, efk, n_items, st_trav, plan);
    if (pst != ESG_OK) return pst;
    const int wpb = plan.wpb;
    const int64_t grid = plan.grid;

    // scratch: pieces, k, status, per-item results, global visited sets
    size_t bytes_pieces = sizeof(esg_piece) * n_items;
    size_t bytes_kq = sizeof(int32_t) * s.nq;
    size_t bytes_qs = sizeof(int32_t) * s.nq;
    size_t bytes_res = sizeof(Cand) * n_items * s.k_max;
    size_t bytes_cnt = sizeof(int32_t) * n_items * 2;
    size_t bytes_stats = sizeof(int64_t) * n_items * 4;
    size_t bytes_hash = (size_t)grid * wpb * plan.G * 4;
    auto al = [](size_t x) { return (x + 255) & ~(size_t)255; };
    size_t total = al(bytes_pieces) + al(bytes_kq) + al(bytes_qs) + al(bytes_res) + al(bytes_cnt) +
                   al(bytes_stats) + al(bytes_hash) + 256;
    unsigned char *scratch = nullptr;
    ESG_CUDA_TRY(cudaMallocAsync((void **)&scratch, total, stream));
    unsigned char *p = scratch;
    esg_piece *pieces = (esg_piece *)p; p += al(bytes_pieces);
    int32_t *kq = (int32_t *)p; p += al(bytes_kq);
    int32_t *qs = (int32_t *)p; p += al(bytes_qs);
    Cand *res = (Cand *)p; p += al(bytes_res);
    int32_t *res_cnt = (int32_t *)p;
    int32_t *res_status = res_cnt + n_items;
    p += al(bytes_cnt);
    int64_t *res_stats = (int64_t *)p; p += al(bytes_stats);
    uint32_t *ghash = (uint32_t *)p; p += al(bytes_hash);
    unsigned long long *queue = (unsigned long long *)p;

    esg_status st = ESG_OK;
    cudaError_t ce = cudaMemsetAsync(queue, 0, sizeof(unsigned long long), stream);
    if (ce == cudaSuccess) ce = cudaMemsetAsync(ghash, 0xFF, bytes_hash, stream);
    if (ce != cudaSuccess) { esg_set_error(cudaGetErrorString(ce)); st = ESG_ERR_CUDA; }
    if (st == ESG_OK) {
        prep_kernel<<<ceil_div_i(s.nq, 256), 256, 0, stream>>>(ix->n, ix->leaf_size, s.l, s.r, s.k,
                                                               s.k_max, s.nq, pieces, kq, qs);
        ce = cudaGetLastError();
        if (ce != cudaSuccess) { esg_set_error(cudaGetErrorString(ce)); st = ESG_ERR_CUDA; }
    }
    if (st == ESG_OK) {
        SearchArgs a;
        a.X = ix->X; a.adj = ix->adj; a.entries = ix->entries; a.queries = s.queries;
        a.qidx = nullptr; a.kconst = 0; a.qshift = 1;
        a.pieces = pieces; a.kq = kq; a.n = ix->n; a.n_items = n_items;
        a.d = ix->d; a.nvec = plan.nvec; a.R = ix->R; a.E = ix->E;
        a.Xv = reinterpret_cast<const uint4 *>(Xt); a.scale8 = ix->scale8; a.rerank = s.p.rerank;
        a.metric = ix->metric; a.ef = ef; a.LPR = plan.lpr;
        a.max_exp = s.p.max_expansions > 0 ? s.p.max_expansions : 16 * ef + 256;
        a.k_max = s.k_max; a.H = plan.H; a.C = plan.C; a.ghash = ghash; a.G = plan.G; a.queue = queue;
        a.res = res; a.res_cnt = res_cnt; a.res_status = res_status; a.res_stats = res_stats;
        const int pidx = esg_prof_begin(stream);
        plan.fn<<<(unsigned)grid, wpb * 32, plan.smem, stream>>>(a);
        ce = cudaGetLastError();
        esg_prof_end(pidx, stream);
        if (ce != cudaSuccess) { esg_set_error(cudaGetErrorString(ce)); st = ESG_ERR_CUDA; }
    }
    if (st == ESG_OK) {
        esg_prof_count(3);  // prep, search, merge
        merge_kernel<<<ceil_div_i(s.nq, 128), 128, 0, stream>>>(
            s.nq, s.k_max, kq, res, res_cnt, res_status, res_stats, qs, ix->perm, pieces,
            s.out_ids, s.out_dist, s.out_count, s.out_status, s.out_stats);
        ce = cudaGetLastError();
        if (ce != cudaSuccess) { esg_set_error(cudaGetErrorString(ce)); st = ESG_ERR_CUDA; }
    }
    cudaError_t fe = cudaFreeAsync(scratch, stream);
    if (st == ESG_OK && fe != cudaSuccess) { esg_set_error(cudaGetErrorString(fe)); st = ESG_ERR_CUDA; }
    return st;
}

// Beam search over prepared work items (graph construction): item i searches
// the piece pieces[i] for the row qidx[i] of X, keeping the best k results in
// res[i * k ..]. Entry points come from `entries` (E per heap node).
esg_status esg_run_search_items(const float *X, int64_t n, int d, int metric, const uint32_t *adj,
                                int R, const int32_t *entries, int E, const int64_t *qidx,
                                const esg_piece *pieces, int64_t n_items, int ef, int k,
                                int max_exp, Cand *res, int32_t *res_cnt, int32_t *res_status,
                                int64_t *res_stats, cudaStream_t stream) {
    if (n_items == 0) return ESG_OK;
    SearchPlan plan;
    esg_status pst = make_plan(d, R, std::max(ef, k), n_items, ESG_F32, plan);
    if (pst != ESG_OK) return pst;
    const size_t bytes_hash = (size_t)plan.grid * plan.wpb * plan.G * 4;
    unsigned char *scratch = nullptr;
    ESG_CUDA_TRY(cudaMallocAsync((void **)&scratch, bytes_hash + 256, stream));
    unsigned long long *queue = (unsigned long long *)scratch;
    uint32_t *ghash = (uint32_t *)(scratch + 256);
    esg_status st = ESG_OK;
    cudaError_t ce = cudaMemsetAsync(queue, 0, sizeof(unsigned long long), stream);
    if (ce == cudaSuccess) ce = cudaMemsetAsync(ghash, 0xFF, bytes_hash, stream);
    if (ce == cudaSuccess) {
        SearchArgs a;
        a.X = X; a.adj = adj; a.entries = entries; a.queries = X; a.qidx = qidx;
        a.pieces = pieces; a.kq = nullptr; a.kconst = k; a.qshift = 0;
        a.n = n; a.n_items = n_items; a.d = d; a.nvec = plan.nvec; a.LPR = plan.lpr; a.R = R; a.E = E;
        a.Xv = reinterpret_cast<const uint4 *>(X); a.scale8 = nullptr; a.rerank = 0;
        a.metric = metric; a.ef = ef; a.max_exp = max_exp > 0 ? max_exp : 16 * ef + 256;
        a.k_max = k; a.H = plan.H; a.C = plan.C; a.ghash = ghash; a.G = plan.G; a.queue = queue;
        a.res = res; a.res_cnt = res_cnt; a.res_status = res_status; a.res_stats = res_stats;
        plan.fn<<<(unsigned)plan.grid, plan.wpb * 32, plan.smem, stream>>>(a);
        ce = cudaGetLastError();
    }
    if (ce != cudaSuccess) { esg_set_error(cudaGetErrorString(ce)); st = ESG_ERR_CUDA; }
    cudaError_t fe = cudaFreeAsync(scratch, stream);
    if (st == ESG_OK && fe != cudaSuccess) { esg_set_error(cudaGetErrorString(fe)); st = ESG_ERR_CUDA; }
    return st;
}

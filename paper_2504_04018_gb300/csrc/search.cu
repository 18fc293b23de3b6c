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

// Returns false iff `id` is already in the visited set. When the set has
// reached its load limit the id is reported as new without being stored
// (the caller's list de-duplication then catches repeats still listed).
__device__ __forceinline__ bool visit(uint32_t *hash, uint32_t hmask, int *hcount, int hlimit,
                                      uint32_t id, bool *saturated) {
    uint32_t h = hash_mix(id) & hmask;
    for (uint32_t probe = 0; probe <= hmask; ++probe) {
        uint32_t slot = (h + probe) & hmask;
        uint32_t cur = hash[slot];
        if (cur == id) return false;
        if (cur == ESG_NONE) {
            if (*(volatile int *)hcount >= hlimit) { *saturated = true; return true; }
            uint32_t prev = atomicCAS(&hash[slot], ESG_NONE, id);
            if (prev == ESG_NONE) { atomicAdd(hcount, 1); return true; }
            if (prev == id) return false;
        }
    }
    *saturated = true;
    return true;
}

// Distances from the query (held in registers as VPL float4 per lane, LPR
// lanes per row) to the rows listed in nbuf[0..m); written to batch[0..m).
template <int VPL>
__device__ __forceinline__ void eval_rows(const float4 *__restrict__ X4, int nvec, int LPR,
                                          const float4 (&qv)[VPL], const uint32_t *nbuf, int m,
                                          Cand *batch, int metric) {
    const int lane = threadIdx.x & 31;
    const int s = lane & (LPR - 1);
    const int g = lane / LPR;
    const int rows_per_pass = 32 / LPR;
    constexpr int U = (VPL <= 2) ? 4 : 2;
    for (int base = 0; base < m; base += rows_per_pass * U) {
        float4 xv[U][VPL];
        uint32_t id[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            int row = base + u * rows_per_pass + g;
            id[u] = row < m ? nbuf[row] : ESG_NONE;
            if (id[u] != ESG_NONE) {
                const float4 *p = X4 + (size_t)id[u] * nvec + s;
#pragma unroll
                for (int v = 0; v < VPL; ++v) xv[u][v] = __ldg(p + v * LPR);
            } else {
#pragma unroll
                for (int v = 0; v < VPL; ++v) xv[u][v] = make_float4(0.f, 0.f, 0.f, 0.f);
            }
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
            float acc = 0.f;
            if (metric == ESG_L2SQ) {
#pragma unroll
                for (int v = 0; v < VPL; ++v) {
                    float a = qv[v].x - xv[u][v].x, b = qv[v].y - xv[u][v].y;
                    float c = qv[v].z - xv[u][v].z, e = qv[v].w - xv[u][v].w;
                    acc = fmaf(a, a, acc); acc = fmaf(b, b, acc);
                    acc = fmaf(c, c, acc); acc = fmaf(e, e, acc);
                }
            } else {
#pragma unroll
                for (int v = 0; v < VPL; ++v) {
                    acc = fmaf(qv[v].x, xv[u][v].x, acc); acc = fmaf(qv[v].y, xv[u][v].y, acc);
                    acc = fmaf(qv[v].z, xv[u][v].z, acc); acc = fmaf(qv[v].w, xv[u][v].w, acc);
                }
            }
            acc = warp_sum_group(acc, LPR);
            int row = base + u * rows_per_pass + g;
            if (s == 0 && row < m) batch[row] = Cand{metric == ESG_L2SQ ? acc : -acc, id[u]};
        }
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
};

// Cut the list after its ef-th in-range item (Q keeps the best ef; nothing
// behind it can be expanded or returned) and refresh |Q| and the worst of Q.
__device__ __forceinline__ void truncate_list(const Cand *list, ListState &st, int ef,
                                              uint32_t pl, uint32_t pr) {
    const int lane = threadIdx.x & 31;
    int seen = 0;
    st.qn = 0;
    st.qworst = Cand{INFINITY, ESG_NONE};
    for (int base = 0; base < st.len; base += 32) {
        int i = base + lane;
        uint32_t id = i < st.len ? (list[i].id & ESG_ID_MASK) : ESG_NONE;
        bool inr = i < st.len && id >= pl && id <= pr;
        unsigned bal = __ballot_sync(0xffffffffu, inr);
        int c = __popc(bal);
        if (seen + c >= ef) {
            // position of the (ef - seen)-th set bit of bal
            int need = ef - seen;
            unsigned b = bal;
            for (int t = 1; t < need; ++t) b &= b - 1;
            int pos = base + __ffs(b) - 1;
            st.len = pos + 1;
            st.qn = ef;
            st.qworst = list[pos];
            return;
        }
        seen += c;
    }
    st.qn = seen;
}

struct SearchArgs {
    const float *X;
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
    uint32_t *ghash;       // global visited sets, one H-slot per warp, or null
    unsigned long long *queue;  // atomic work counter
    Cand *res;             // [n_items, k_max]
    int32_t *res_cnt;      // [n_items]
    int32_t *res_status;   // [n_items]
    int64_t *res_stats;    // [n_items, 3]
};

template <int VPL>
__global__ void __launch_bounds__(64)
search_kernel(SearchArgs a) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int lane = threadIdx.x & 31;
    const int wib = threadIdx.x >> 5;
    const int wpb = blockDim.x >> 5;
    const bool smem_hash = a.ghash == nullptr;
    size_t per_warp = (smem_hash ? (size_t)a.H * 4 : 0) + (size_t)a.C * 8 * 2 + kBatch * 8 +
                      kBatch * 4 + 16;
    unsigned char *base = smem_raw + per_warp * wib;
    WarpSmem w;
    size_t off = 0;
    w.list = (Cand *)(base + off); off += (size_t)a.C * 8;
    w.list2 = (Cand *)(base + off); off += (size_t)a.C * 8;
    w.batch = (Cand *)(base + off); off += kBatch * 8;
    w.nbuf = (uint32_t *)(base + off); off += kBatch * 4;
    w.hcount = (int *)(base + off); off += 16;
    const int gwarp = blockIdx.x * wpb + wib;
    w.hash = smem_hash ? (uint32_t *)(base + off) : a.ghash + (size_t)gwarp * a.H;
    const uint32_t hmask = (uint32_t)a.H - 1;
    const int hlimit = (a.H * 3) / 4;
    const float4 *X4 = reinterpret_cast<const float4 *>(a.X);

    for (;;) {
        int64_t item = 0;
        if (lane == 0) item = (int64_t)atomicAdd(a.queue, 1ULL);
        item = __shfl_sync(0xffffffffu, item, 0);
        if (item >= a.n_items) break;
        const int64_t qi = item >> a.qshift;
        const esg_piece pc = a.pieces[item];
        const int kq = a.kq ? a.kq[qi] : a.kconst;
        int64_t n_exp = 0, n_eval = 0, n_oor = 0;
        int status = 0;
        if (pc.kind == ESG_PIECE_NONE || kq <= 0) {
            if (lane == 0) { a.res_cnt[item] = 0; a.res_status[item] = 0; }
            if (lane < 3) a.res_stats[item * 3 + lane] = 0;
            continue;
        }
        const uint32_t pl = (uint32_t)pc.pl, pr = (uint32_t)pc.pr;
        const bool is_graph = pc.kind == ESG_PIECE_GRAPH;
        const int ef = is_graph ? max(a.ef, kq) : kq;

        // query slice in registers
        float4 qv[VPL];
        {
            const int64_t qrow = a.qidx ? a.qidx[item] : qi;
            const float4 *q4 = reinterpret_cast<const float4 *>(a.queries + qrow * (int64_t)a.d);
            const int s = lane & (a.LPR - 1);
#pragma unroll
            for (int v = 0; v < VPL; ++v) qv[v] = __ldg(q4 + s + v * a.LPR);
        }
        ListState st{0, 0, Cand{INFINITY, ESG_NONE}};
        Cand *list = w.list, *list2 = w.list2;
        bool saturated = false;

        if (!is_graph) {
            // Leaf piece: exact scan of [pl, pr] (Algorithm 4, first branch).
            for (int64_t c0 = pl; c0 <= (int64_t)pr; c0 += kBatch) {
                int m = (int)(((int64_t)pr - c0 + 1) < kBatch ? ((int64_t)pr - c0 + 1) : kBatch);
                for (int j = lane; j < m; j += 32) w.nbuf[j] = (uint32_t)(c0 + j);
                __syncwarp();
                eval_rows<VPL>(X4, a.nvec, a.LPR, qv, w.nbuf, m, w.batch, a.metric);
                n_eval += m;
                for (int j = lane; j < kBatch; j += 32) {
                    bool keep = j < m && (st.qn < ef || cand_less(w.batch[j], st.qworst));
                    if (!keep) w.batch[j] = Cand{INFINITY, ESG_NONE};
                }
                __syncwarp();
                warp_sort64(w.batch);
                int b = 0;
                for (int j = lane; j < kBatch; j += 32) b += w.batch[j].id != ESG_NONE;
                for (int o = 16; o > 0; o >>= 1) b += __shfl_xor_sync(0xffffffffu, b, o);
                st.len = warp_merge(list, st.len, w.batch, b, list2, a.C);
                Cand *t = list; list = list2; list2 = t;
                truncate_list(list, st, ef, pl, pr);
            }
        } else {
            // Graph piece: Algorithm 1 with POST filtering to [pl, pr].
            for (int i = lane; i < a.H; i += 32) w.hash[i] = ESG_NONE;
            if (lane == 0) *w.hcount = 0;
            __syncwarp();
            const uint32_t *adj = a.adj + (size_t)pc.depth * (size_t)a.n * a.R;
            // entry points: into P, and into Q when in range
            {
                uint32_t e = ESG_NONE;
                if (lane < a.E) {
                    int32_t v = a.entries[(size_t)pc.heap * a.E + lane];
                    if (v >= 0 && v < a.n) e = (uint32_t)v;
                }
                bool nw = e != ESG_NONE && visit(w.hash, hmask, w.hcount, hlimit, e, &saturated);
                unsigned bal = __ballot_sync(0xffffffffu, nw);
                if (nw) w.nbuf[__popc(bal & ((1u << lane) - 1))] = e;
                int m = __popc(bal);
                __syncwarp();
                eval_rows<VPL>(X4, a.nvec, a.LPR, qv, w.nbuf, m, w.batch, a.metric);
                n_eval += m;
                for (int j = lane; j < kBatch; j += 32) {
                    if (j >= m) w.batch[j] = Cand{INFINITY, ESG_NONE};
                    else n_oor += (w.batch[j].id < pl || w.batch[j].id > pr);
                }
                __syncwarp();
                warp_sort64(w.batch);
                st.len = warp_merge(list, 0, w.batch, m, list2, a.C);
                Cand *t = list; list = list2; list2 = t;
                truncate_list(list, st, ef, pl, pr);
            }
            for (;;) {
                // best unexpanded candidate
                int pos = -1;
                for (int b0 = 0; b0 < st.len; b0 += 32) {
                    int i = b0 + lane;
                    bool f = i < st.len && !(list[i].id & ESG_EXPANDED);
                    unsigned bal = __ballot_sync(0xffffffffu, f);
                    if (bal) { pos = b0 + __ffs(bal) - 1; break; }
                }
                if (pos < 0) break;
                if (n_exp >= a.max_exp) { status |= ESG_Q_TRUNCATED; break; }
                const uint32_t u = list[pos].id & ESG_ID_MASK;
                const bool u_in = u >= pl && u <= pr;
                __syncwarp();
                if (u_in) {
                    if (lane == 0) list[pos].id = u | ESG_EXPANDED;
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
                bool n0 = v0 != ESG_NONE && visit(w.hash, hmask, w.hcount, hlimit, v0, &saturated);
                bool n1 = v1 != ESG_NONE && visit(w.hash, hmask, w.hcount, hlimit, v1, &saturated);
                unsigned b0 = __ballot_sync(0xffffffffu, n0);
                unsigned b1 = __ballot_sync(0xffffffffu, n1);
                int c0 = __popc(b0);
                if (n0) w.nbuf[__popc(b0 & ((1u << lane) - 1))] = v0;
                if (n1) w.nbuf[c0 + __popc(b1 & ((1u << lane) - 1))] = v1;
                int m = c0 + __popc(b1);
                __syncwarp();
                if (m == 0) continue;  // next chunk
                eval_rows<VPL>(X4, a.nvec, a.LPR, qv, w.nbuf, m, w.batch, a.metric);
                n_eval += m;
                // Algorithm 1's admission test, then de-duplication against
                // the list (only needed once the visited set saturates)
                for (int j = lane; j < kBatch; j += 32) {
                    bool keep = false;
                    if (j < m) {
                        Cand x = w.batch[j];
                        n_oor += (x.id < pl || x.id > pr);
                        keep = st.qn < ef || cand_less(x, st.qworst);
                        if (keep && saturated) {
                            int p = lower_rank(list, st.len, x);
                            if (p < st.len && cand_eq(list[p], x)) keep = false;
                        }
                    }
                    if (!keep) w.batch[j] = Cand{INFINITY, ESG_NONE};
                }
                __syncwarp();
                warp_sort64(w.batch);
                int b = 0;
                for (int j = lane; j < kBatch; j += 32) b += w.batch[j].id != ESG_NONE;
                for (int o = 16; o > 0; o >>= 1) b += __shfl_xor_sync(0xffffffffu, b, o);
                if (b == 0) continue;  // next chunk
                if (st.len + b > a.C) status |= ESG_Q_OVERFLOW;
                st.len = warp_merge(list, st.len, w.batch, b, list2, a.C);
                Cand *t = list; list = list2; list2 = t;
                truncate_list(list, st, ef, pl, pr);
                }  // neighbour chunk
            }
            if (saturated) status |= ESG_Q_OVERFLOW;
        }
        // emit the first min(k, |Q|) in-range items
        {
            int written = 0;
            Cand *out = a.res + item * (int64_t)a.k_max;
            for (int b0 = 0; b0 < st.len && written < kq; b0 += 32) {
                int i = b0 + lane;
                uint32_t id = i < st.len ? (list[i].id & ESG_ID_MASK) : ESG_NONE;
                bool inr = i < st.len && id >= pl && id <= pr;
                unsigned bal = __ballot_sync(0xffffffffu, inr);
                int pos = written + __popc(bal & ((1u << lane) - 1));
                if (inr && pos < kq) out[pos] = Cand{list[i].d, id};
                written += __popc(bal);
            }
            written = min(written, kq);
            if (lane == 0) {
                a.res_cnt[item] = written;
                a.res_status[item] = status;
                a.res_stats[item * 3 + 0] = n_exp;
                a.res_stats[item * 3 + 1] = n_eval;
                a.res_stats[item * 3 + 2] = n_oor;
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
        for (int c = 0; c < 3; ++c)
            out_stats[i * 4 + c] = k > 0 ? res_stats[2 * i * 3 + c] + res_stats[(2 * i + 1) * 3 + c] : 0;
        out_stats[i * 4 + 3] = np;
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

SearchFn pick_search(int vpl) {
    switch (vpl) {
        case 1: return search_kernel<1>;
        case 2: return search_kernel<2>;
        case 3: return search_kernel<3>;
        case 4: return search_kernel<4>;
        case 6: return search_kernel<6>;
        case 8: return search_kernel<8>;
        default: return nullptr;
    }
}

int env_int(const char *name, int dflt) {
    const char *v = getenv(name);
    return v && *v ? atoi(v) : dflt;
}

}  // namespace

int esg_pick_vpl(int d, int *lpr) {
    int nvec = d / 4;
    const int vpls[] = {1, 2, 3, 4, 6, 8};
    for (int v : vpls) {
        if (nvec % v) continue;
        int L = nvec / v;
        if (L == 1 || L == 2 || L == 4 || L == 8 || L == 16 || L == 32) { *lpr = L; return v; }
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
    int efk = std::max(ef, s.k_max);
    int lpr = 0;
    int vpl = esg_pick_vpl(ix->d, &lpr);
    if (vpl == 0) { esg_set_error("unsupported dimension"); return ESG_ERR_UNSUPPORTED; }
    if (ix->R > 128) { esg_set_error("R > 128"); return ESG_ERR_UNSUPPORTED; }
    int C = ((std::max(4 * efk, efk + 64) + 31) / 32) * 32;
    if (C > 4096) C = 4096;
    // visited set: open addressing, power of two, sized from the beam width
    int H = 4096;
    const int hash_per_ef = env_int("ESG_HASH_PER_EF", 64);
    while (H < hash_per_ef * efk && H < (1 << 22)) H <<= 1;
    while (H < 4 * ix->R) H <<= 1;
    const int wpb = 2;
    const bool smem_hash = (size_t)H * 4 <= (size_t)env_int("ESG_SMEM_HASH_BYTES", 32768);
    size_t per_warp = (smem_hash ? (size_t)H * 4 : 0) + (size_t)C * 16 + kBatch * 12 + 16;
    size_t smem = per_warp * wpb;
    int64_t n_items = 2 * s.nq;
    SearchFn fn = pick_search(vpl);
    int dev = 0, sms = 0, per_sm = 0;
    ESG_CUDA_TRY(cudaGetDevice(&dev));
    ESG_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    ESG_CUDA_TRY(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    ESG_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, wpb * 32, smem));
    if (per_sm < 1) { esg_set_error("search kernel does not fit on an SM"); return ESG_ERR_UNSUPPORTED; }
    int64_t grid = std::min<int64_t>((int64_t)sms * per_sm, (n_items + wpb - 1) / wpb);
    if (grid < 1) grid = 1;

    // scratch: pieces, k, status, per-item results, global visited sets
    size_t bytes_pieces = sizeof(esg_piece) * n_items;
    size_t bytes_kq = sizeof(int32_t) * s.nq;
    size_t bytes_qs = sizeof(int32_t) * s.nq;
    size_t bytes_res = sizeof(Cand) * n_items * s.k_max;
    size_t bytes_cnt = sizeof(int32_t) * n_items * 2;
    size_t bytes_stats = sizeof(int64_t) * n_items * 3;
    size_t bytes_hash = smem_hash ? 0 : (size_t)grid * wpb * H * 4;
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
    uint32_t *ghash = smem_hash ? nullptr : (uint32_t *)p; p += al(bytes_hash);
    unsigned long long *queue = (unsigned long long *)p;

    esg_status st = ESG_OK;
    cudaError_t ce = cudaMemsetAsync(queue, 0, sizeof(unsigned long long), stream);
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
        a.d = ix->d; a.nvec = ix->d / 4; a.LPR = lpr; a.R = ix->R; a.E = ix->E;
        a.metric = ix->metric; a.ef = ef;
        a.max_exp = s.p.max_expansions > 0 ? s.p.max_expansions : 16 * ef + 256;
        a.k_max = s.k_max; a.H = H; a.C = C; a.ghash = ghash; a.queue = queue;
        a.res = res; a.res_cnt = res_cnt; a.res_status = res_status; a.res_stats = res_stats;
        const int pidx = esg_prof_begin(stream);
        fn<<<(unsigned)grid, wpb * 32, smem, stream>>>(a);
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
    int lpr = 0;
    int vpl = esg_pick_vpl(d, &lpr);
    if (vpl == 0) { esg_set_error("unsupported dimension"); return ESG_ERR_UNSUPPORTED; }
    const int efk = std::max(ef, k);
    int C = ((std::max(2 * efk, efk + 64) + 31) / 32) * 32;
    int H = 1024;
    const int hash_per_ef = env_int("ESG_BUILD_HASH_PER_EF", 48);
    while (H < hash_per_ef * efk && H < (1 << 22)) H <<= 1;
    while (H < 4 * R) H <<= 1;
    const int wpb = 2;
    const bool smem_hash = (size_t)H * 4 <= (size_t)env_int("ESG_SMEM_HASH_BYTES", 65536);
    size_t per_warp = (smem_hash ? (size_t)H * 4 : 0) + (size_t)C * 16 + kBatch * 12 + 16;
    size_t smem = per_warp * wpb;
    SearchFn fn = pick_search(vpl);
    int dev = 0, sms = 0, per_sm = 0;
    ESG_CUDA_TRY(cudaGetDevice(&dev));
    ESG_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    ESG_CUDA_TRY(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    ESG_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, wpb * 32, smem));
    if (per_sm < 1) { esg_set_error("search kernel does not fit on an SM"); return ESG_ERR_UNSUPPORTED; }
    int64_t grid = std::min<int64_t>((int64_t)sms * per_sm, (n_items + wpb - 1) / wpb);
    if (grid < 1) grid = 1;
    size_t bytes_hash = smem_hash ? 0 : (size_t)grid * wpb * H * 4;
    unsigned char *scratch = nullptr;
    ESG_CUDA_TRY(cudaMallocAsync((void **)&scratch, bytes_hash + 256, stream));
    unsigned long long *queue = (unsigned long long *)scratch;
    uint32_t *ghash = smem_hash ? nullptr : (uint32_t *)(scratch + 256);
    esg_status st = ESG_OK;
    cudaError_t ce = cudaMemsetAsync(queue, 0, sizeof(unsigned long long), stream);
    if (ce == cudaSuccess) {
        SearchArgs a;
        a.X = X; a.adj = adj; a.entries = entries; a.queries = X; a.qidx = qidx;
        a.pieces = pieces; a.kq = nullptr; a.kconst = k; a.qshift = 0;
        a.n = n; a.n_items = n_items; a.d = d; a.nvec = d / 4; a.LPR = lpr; a.R = R; a.E = E;
        a.metric = metric; a.ef = ef; a.max_exp = max_exp > 0 ? max_exp : 16 * ef + 256;
        a.k_max = k; a.H = H; a.C = C; a.ghash = ghash; a.queue = queue;
        a.res = res; a.res_cnt = res_cnt; a.res_status = res_status; a.res_stats = res_stats;
        fn<<<(unsigned)grid, wpb * 32, smem, stream>>>(a);
        ce = cudaGetLastError();
    }
    if (ce != cudaSuccess) { esg_set_error(cudaGetErrorString(ce)); st = ESG_ERR_CUDA; }
    cudaError_t fe = cudaFreeAsync(scratch, stream);
    if (st == ESG_OK && fe != cudaSuccess) { esg_set_error(cudaGetErrorString(fe)); st = ESG_ERR_CUDA; }
    return st;
}

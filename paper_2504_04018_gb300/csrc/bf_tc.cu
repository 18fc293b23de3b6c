// Exact range-filtered k-NN on the 5th-generation tensor cores (tcgen05).
//
// Dot products q.x come from three BF16 MMAs per K step accumulated in FP32
// in tensor memory (split precision: q = q_hi + q_lo, x = x_hi + x_lo with
// BF16 parts, q.x ~ q_hi.x_hi + q_hi.x_lo + q_lo.x_hi; the dropped q_lo.x_lo
// and the split residuals are below 2^-17 relative). Queries are sorted and
// tiled by 128 (one TMEM lane each); a query tile visits the 128-point tiles
// its ranges cover (128 TMEM columns per tile). The pipelined kernel below
// is warp-specialised: bulk copies of pre-swizzled operand blocks, one MMA
// thread, and eight epilogue warps that keep the K1 best approximate
// distances per query.
//
// A second kernel recomputes exact FP32 distances (direct form) of those
// candidates, sorts them, and certifies the result: with delta_q a bound on
// |approximate - exact| for every point of the range, the top k is proven
// when the exact k-th distance is below (K1-th approximate distance -
// delta_q). Queries without a certificate run again with a longer list, then
// through the exact SIMT brute force.
#include "esg_internal.cuh"

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <vector>

esg_status esg_bruteforce_redo(const float *base, int64_t n, int32_t d, int metric, const float *queries,
                               int64_t nq, const int64_t *l, const int64_t *r, int32_t k,
                               const std::vector<int64_t> &idx, int64_t *out_ids, float *out_dist,
                               int32_t *out_count, cudaStream_t stream);

namespace {

constexpr int TM = 128;            // queries per CTA (TMEM lanes)
constexpr int TN = 128;            // points per tile (TMEM columns)
constexpr int TK = 64;             // K chunk: 64 BF16 = one 128-byte swizzled row
constexpr int CHUNK = TM * TK * 2; // bytes of one 128 x 64 BF16 operand chunk (16 KB)

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}

// Shared-memory matrix descriptor: K-major operand, 128-byte swizzle, rows of
// 128 bytes, 8-row groups 1024 bytes apart (stride byte offset), sm_100
// descriptor version 1.
__device__ __forceinline__ uint64_t sdesc(uint32_t saddr) {
    uint64_t d = 0;
    d |= (uint64_t)((saddr & 0x3FFFFu) >> 4);
    d |= (uint64_t)(16u >> 4) << 16;
    d |= (uint64_t)(1024u >> 4) << 32;
    d |= (uint64_t)1 << 46;
    d |= (uint64_t)2 << 61;
    return d;
}

// Instruction descriptor of kind::f16: FP32 accumulator, BF16 A and B, both
// K-major, N = TN, M = TM.
constexpr uint32_t kIdesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(TN >> 3) << 17) |
                            ((uint32_t)(TM >> 4) << 24);

__device__ __forceinline__ void mma_bf16(uint32_t tmem_d, uint64_t a, uint64_t b, uint32_t acc) {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n"
        :: "r"(tmem_d), "l"(a), "l"(b), "r"(kIdesc), "r"(acc));
}

__device__ __forceinline__ void mma_commit(uint32_t mbar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
                 :: "r"(mbar) : "memory");
}

// 64 consecutive accumulator columns of the warp's 32 TMEM lanes (one
// register each), waiting for the load inside the same asm statement so that
// no use of the registers can be scheduled before the wait.
__device__ __forceinline__ void tmem_ld64(uint32_t taddr, float *v) {
    uint32_t r[64];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x64.b32 "
        "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16,%17,%18,%19,%20,%21,%22,%23,%24,"
        "%25,%26,%27,%28,%29,%30,%31,%32,%33,%34,%35,%36,%37,%38,%39,%40,%41,%42,%43,%44,%45,%46,"
        "%47,%48,%49,%50,%51,%52,%53,%54,%55,%56,%57,%58,%59,%60,%61,%62,%63}, [%64];\n\t"
        "tcgen05.wait::ld.sync.aligned;"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]),
          "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]),
          "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]),
          "=r"(r[29]), "=r"(r[30]), "=r"(r[31]), "=r"(r[32]), "=r"(r[33]), "=r"(r[34]), "=r"(r[35]),
          "=r"(r[36]), "=r"(r[37]), "=r"(r[38]), "=r"(r[39]), "=r"(r[40]), "=r"(r[41]), "=r"(r[42]),
          "=r"(r[43]), "=r"(r[44]), "=r"(r[45]), "=r"(r[46]), "=r"(r[47]), "=r"(r[48]), "=r"(r[49]),
          "=r"(r[50]), "=r"(r[51]), "=r"(r[52]), "=r"(r[53]), "=r"(r[54]), "=r"(r[55]), "=r"(r[56]),
          "=r"(r[57]), "=r"(r[58]), "=r"(r[59]), "=r"(r[60]), "=r"(r[61]), "=r"(r[62]), "=r"(r[63])
        : "r"(taddr)
        : "memory");
#pragma unroll
    for (int i = 0; i < 64; ++i) v[i] = __uint_as_float(r[i]);
}

__global__ void max_kernel(const float *v, int64_t n, float *out) {
    float m = 0.f;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        m = fmaxf(m, v[i]);
    for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0) atomicMax((int *)out, __float_as_int(m));   // m >= 0
}

// Exact re-rank and certificate, one warp per query.
__global__ void rerank_certify_kernel(const float *X, const float *Q, int d, int metric, int64_t nq,
                                      int k, int K1, const float *cand_d, const int32_t *cand_i,
                                      const int32_t *cand_n, const float *qrownorm, const float *xmax,
                                      int64_t *out_ids, float *out_dist,
                                      int32_t *out_count, int32_t *redo) {
    __shared__ Cand buf[4][128];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int64_t q = blockIdx.x * (int64_t)(blockDim.x >> 5) + w;
    if (q >= nq) return;
    Cand *b = buf[w];
    const int m = cand_n[q];
    if (m < 0) {  // invalid range
        for (int j = lane; j < k; j += 32) { out_ids[q * k + j] = -1; out_dist[q * k + j] = INFINITY; }
        if (lane == 0) { out_count[q] = 0; redo[q] = 0; }
        return;
    }
    const float *qq = Q + q * (int64_t)d;
    for (int e = 0; e < m; ++e) {
        const int32_t row = cand_i[q * K1 + e];
        const float *x = X + (int64_t)row * d;
        float acc = 0.f;
        for (int j = lane; j < d; j += 32) {
            if (metric == ESG_L2SQ) { const float t = qq[j] - x[j]; acc = fmaf(t, t, acc); }
            else acc = fmaf(qq[j], x[j], acc);
        }
        acc = warp_sum_group(acc, 32);
        if (lane == 0) b[e] = Cand{metric == ESG_L2SQ ? acc : -acc, (uint32_t)row};
    }
    __syncwarp();
    const int P = 128;
    for (int j = m + lane; j < P; j += 32) b[j] = Cand{INFINITY, ESG_NONE};
    __syncwarp();
    warp_sort_pow2(b, P);
    const int c = min(k, m);
    bool certified = c > 0;
    if (m == K1) {   // the list is full: points may have been left out
        // |approximate - exact| for any point of the range (unit roundoff of
        // BF16 2^-8, of FP32 2^-24): the split residuals and the dropped
        // lo*lo product stay below 3.1 * 2^-16 |q_i||x_i| per term, the FP32
        // accumulation of 3d products below 6d * 2^-24 (twice the rounding
        // bound, for truncating adders); the squared distance doubles the dot
        // product error and adds the rounding of the norms and the final sum.
        const double qn = qrownorm[q], xm = xmax[0];
        const double dot_err = (3.1 * 0x1p-16 + 6.0 * d * 0x1p-24) * qn * xm;
        const double delta = metric == ESG_L2SQ ? 2.0 * dot_err + (d + 4.0) * 0x1p-24 * (qn * qn + xm * xm)
                                                : dot_err;
        const double bound = (double)cand_d[q * K1 + K1 - 1] - delta;
        // the re-ranked FP32 distance itself is within d * 2^-23 relative
        const double dk = (double)b[c - 1].d;
        certified = dk + fabs(dk) * d * 0x1p-23 < bound;
    }
    for (int j = lane; j < k; j += 32) {
        out_ids[q * k + j] = j < c ? (int64_t)b[j].id : -1;
        out_dist[q * k + j] = j < c ? b[j].d : INFINITY;
    }
    if (lane == 0) { out_count[q] = c; redo[q] = certified ? 0 : 1; }
}


// ------------------------------------------------------------------------
// Pipelined version. The operands are pre-tiled in global memory in exactly
// the shared-memory layout the MMA descriptors name (one 32 KB block per
// 128 rows x 64 dimensions: BF16 hi part, then lo part, 128-byte swizzle,
// zero padding past the last row and dimension), so every stage is one bulk
// copy on the TMA engine. Queries are sorted by (log2 of range width, l)
// and grouped into tiles of 128; a query tile only visits the point tiles
// that its queries' ranges cover; the CTAs (one per SM) run contiguous
// shares of that sequence of equal estimated cost, cut into work items at
// query-tile boundaries. Each CTA is warp-specialised:
//   warp 0      bulk copies: the item's query tile (resident), then a ring of
//               S point-tile stages;
//   warp 1      one thread issues the MMAs into one of two TMEM accumulators
//               (128 columns each) and commits them to mbarriers;
//   warps 2..9  epilogue: each reads half a row (64 columns) of the finished
//               accumulator into registers and releases it; the tile is then
//               passed through shared memory half by half so that one warp
//               handles one query row at a time: range mask, distance, a
//               ballot against the row's current K1-th distance, and, for the
//               rare candidates that pass, an insertion into the row's sorted
//               list held across the warp's lanes. A CTA runs a contiguous
//               share of the items, so a row's list carries over between its
//               items of the same query tile; the lists go to global memory
//               and a merge kernel combines them per query.
// Every wait is bounded (2 s of global time); a wait that runs out sets the
// error flag and all roles leave their loops.

constexpr int STAGE = 2 * CHUNK;          // hi + lo of a 128 x 64 block
constexpr int kEpiWarps = 8;
constexpr int kThreads2 = 64 + 32 * kEpiWarps;
constexpr int kMaxK1v2 = 64;
constexpr int kTS = 65;                   // row stride of the transposed half tile
constexpr int kMaxStages = 6;
// Limit of the waits that let work already issued finish before a CTA exits
// (bulk copies, MMAs); the pipeline's own waits take Tc2Args::wait_ns.
constexpr unsigned long long kWaitNs = 2000000000ull;

struct WorkItem {
    int32_t qtile, off, cnt, pad;
};

struct Tc2Args {
    const unsigned char *xs, *qs;   // tiled operand blocks
    const float *xnorm, *qnorm;     // squared norms (queries in caller order)
    const int64_t *l, *r;
    const int32_t *qorder;          // sorted position -> caller's query index
    const WorkItem *items;
    const int32_t *tiles;           // point-tile ids of all items
    const int32_t *cta_first;       // [grid + 1]: CTA c runs items [cta_first[c], cta_first[c + 1])
    int n_items;
    int64_t nv;                     // number of valid (sorted) queries
    int nk, metric, K1, S;
    int stream_a;                   // 1: each stage carries the query tile's K chunk too
    int64_t n;                      // points
    float *part_d;                  // [n_items][128][K1]
    int32_t *part_i;                // [n_items][128][K1]
    int32_t *part_n;                // [n_items][128]
    int32_t *err;
    unsigned long long wait_ns;     // limit of a pipeline wait (ESG_BF_WAIT_NS; default 2 s)
    int32_t stall;                  // failure-detection test: the producer first waits on a
                                    // barrier nothing arrives on, before it issues any copy
};

__device__ __forceinline__ unsigned long long gtime() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ bool mbar_try(uint32_t mbar, uint32_t parity) {
    uint32_t done = 0;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}\n"
        : "=r"(done) : "r"(mbar), "r"(parity) : "memory");
    return done != 0;
}

// Bounded wait for the phase of the given parity. Gives up when another role
// has aborted (unless `ignore_abort`) or after limit_ns; on a timeout it
// raises the abort flag and the error flag.
__device__ bool wait_phase(uint32_t mbar, uint32_t parity, volatile int *abort_f, int32_t *err,
                           unsigned long long limit_ns, bool ignore_abort = false) {
    unsigned long long t0 = 0;
    for (uint32_t it = 1;; ++it) {
        if (mbar_try(mbar, parity)) return true;
        if ((it & 127) == 0) {
            if (!ignore_abort && *abort_f) return false;
            const unsigned long long t = gtime();
            if (t0 == 0) t0 = t;
            else if (t - t0 > limit_ns) {
                *abort_f = 1;
                atomicExch(err, 1);
                return false;
            }
        }
    }
}

__device__ __forceinline__ void mbar_init(uint32_t mbar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" :: "r"(mbar), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint32_t mbar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" :: "r"(mbar), "r"(bytes) : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint32_t mbar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" :: "r"(mbar) : "memory");
}
// Bulk global -> shared copy on the TMA engine, completion counted in bytes
// on the mbarrier (addresses 16-byte aligned, size a multiple of 16).
__device__ __forceinline__ void bulk_g2s(uint32_t dst, const void *src, uint32_t bytes, uint32_t mbar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
                 :: "r"(dst), "l"(src), "r"(bytes), "r"(mbar) : "memory");
}

__device__ __forceinline__ void epi_bar() {   // the 256 epilogue threads
    asm volatile("bar.sync 1, %0;" :: "n"(32 * kEpiWarps) : "memory");
}

__device__ __forceinline__ void pair_bar(int quarter) {   // the two warps of a lane quarter
    asm volatile("bar.sync %0, 64;" :: "r"(2 + quarter) : "memory");
}

// Lexicographic (distance, row) order of the candidate lists.
__device__ __forceinline__ bool dl_less(float da, int32_t ia, float db, int32_t ib) {
    return da < db || (da == db && ia < ib);
}

// One compare-exchange stage of a bitonic network over 64 (distance, index)
// pairs, element e = lane + 32 h in (d[h], i[h]); pairs compare by dl_less.
// Element e meets e ^ j; in a block of size kk that sorts ascending (up) the
// lower position keeps the smaller pair. `desc` flips every direction.
__device__ __forceinline__ void bitonic_stage(float (&d)[2], int32_t (&i)[2], int lane, int kk, int j, bool desc) {
    if (j == 32) {   // partners in the same lane (only in the 64-wide block)
        const bool sw = desc ? dl_less(d[0], i[0], d[1], i[1]) : dl_less(d[1], i[1], d[0], i[0]);
        if (sw) {
            const float td = d[0]; d[0] = d[1]; d[1] = td;
            const int32_t ti = i[0]; i[0] = i[1]; i[1] = ti;
        }
        return;
    }
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        const float od = __shfl_xor_sync(0xffffffffu, d[h], j);
        const int32_t oi = __shfl_xor_sync(0xffffffffu, i[h], j);
        const bool up = (((lane + 32 * h) & kk) == 0) != desc;
        const bool low = (lane & j) == 0;
        const bool take = low == up ? dl_less(od, oi, d[h], i[h]) : dl_less(d[h], i[h], od, oi);
        if (take) { d[h] = od; i[h] = oi; }
    }
}

// Bitonic sort of the 64 pairs (ascending, or descending with `desc`).
__device__ __forceinline__ void bitonic_sort64(float (&d)[2], int32_t (&i)[2], int lane, bool desc) {
#pragma unroll
    for (int kk = 2; kk <= 64; kk <<= 1)
#pragma unroll
        for (int j = kk >> 1; j > 0; j >>= 1) bitonic_stage(d, i, lane, kk, j, desc);
}

// A sorted list (ascending) and 64 sorted candidates (descending), both padded
// with (+inf, INT32_MAX): the element-wise smaller pairs are the 64 smallest of
// the union as a bitonic sequence, which one merge pass sorts ascending.
__device__ __forceinline__ void bitonic_merge_into(float (&ld)[2], int32_t (&li)[2], const float (&cd)[2],
                                                   const int32_t (&ci)[2], int lane) {
#pragma unroll
    for (int h = 0; h < 2; ++h)
        if (dl_less(cd[h], ci[h], ld[h], li[h])) { ld[h] = cd[h]; li[h] = ci[h]; }
#pragma unroll
    for (int j = 32; j > 0; j >>= 1) bitonic_stage(ld, li, lane, 64, j, false);
}

// Candidates of one row and half tile from which the epilogue sorts and
// merges them in one network instead of inserting them one at a time (a list
// that is still filling: the first tile of a work item).
constexpr int kBulkMin = 32;

__global__ void __launch_bounds__(kThreads2, 1) tc_knn2_kernel(Tc2Args a) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    unsigned char *base = (unsigned char *)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    const int K1 = a.K1;
    // resident query tile: sA holds its nk K chunks for the whole item, a stage
    // one point chunk; streamed (large d): a stage holds the query chunk and
    // the point chunk of one K step
    const int stage_bytes = a.stream_a ? 2 * STAGE : STAGE;
    unsigned char *sA = base;
    unsigned char *sB = sA + (a.stream_a ? (size_t)0 : (size_t)a.nk * STAGE);
    float *T = (float *)(sB + (size_t)a.S * stage_bytes);    // [128][kTS] half tile, transposed
    float *s_xn = T + TM * kTS;                              // [4 pairs][2][128] tile norms
    float *L_d = s_xn + 8 * TN;                              // [128][K1] per-row lists
    int32_t *L_i = (int32_t *)(L_d + TM * K1);
    int32_t *r_lo = L_i + TM * K1, *r_hi = r_lo + TM, *r_cnt = r_hi + TM, *r_ti = r_cnt + TM;
    float *r_qn = (float *)(r_ti + TM), *r_td = r_qn + TM;
    uint32_t *s_flag = (uint32_t *)(r_td + TM);              // [2 halves][4 quarters] row masks
    uint64_t *bars = (uint64_t *)(s_flag + 8);
    uint64_t *full = bars, *empty = bars + a.S;
    uint64_t *a_full = bars + 2 * a.S, *a_empty = a_full + 1;
    uint64_t *acc_full = a_full + 2, *acc_empty = a_full + 4, *drain = a_full + 6;
    uint32_t *tmem_slot = (uint32_t *)(a_full + 7);
    volatile int *abort_f = (volatile int *)(tmem_slot + 1);
    uint64_t *never = a_full + 8;                             // nothing arrives on it
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    // this CTA's contiguous share of the work items
    const int it_begin = a.cta_first[blockIdx.x];
    const int it_end = a.cta_first[blockIdx.x + 1];

    if (threadIdx.x == 0) {
        for (int s = 0; s < a.S; ++s) {
            mbar_init(smem_u32(full + s), 1);
            mbar_init(smem_u32(empty + s), 1);
        }
        mbar_init(smem_u32(a_full), 1);
        mbar_init(smem_u32(a_empty), 1);
        for (int b = 0; b < 2; ++b) {
            mbar_init(smem_u32(acc_full + b), 1);
            mbar_init(smem_u32(acc_empty + b), kEpiWarps);
        }
        mbar_init(smem_u32(drain), 1);
        mbar_init(smem_u32(never), 1);
        *abort_f = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                     :: "r"(smem_u32(tmem_slot)), "r"(2 * TN) : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = *tmem_slot;

    if (warp == 0) {
        if (lane == 0) {
            // ---------------- producer
            uint32_t s = 0, ps = 0, pa = 0;
            uint32_t issued[kMaxStages] = {0};
            uint32_t ipar[kMaxStages] = {0};
            bool a_pending = false;
            uint32_t a_par = 0;
            bool ok = true;
            if (a.stall && !wait_phase(smem_u32(never), 0u, abort_f, a.err, a.wait_ns)) ok = false;
            for (int it = it_begin; ok && it < it_end; ++it) {
                const WorkItem I = a.items[it];
                if (!a.stream_a) {
                    if (!wait_phase(smem_u32(a_empty), pa ^ 1u, abort_f, a.err, a.wait_ns)) { ok = false; break; }
                    mbar_expect_tx(smem_u32(a_full), (uint32_t)(a.nk * STAGE));
                    for (int kc = 0; kc < a.nk; ++kc)
                        bulk_g2s(smem_u32(sA + (size_t)kc * STAGE),
                                 a.qs + ((int64_t)I.qtile * a.nk + kc) * STAGE, STAGE, smem_u32(a_full));
                    a_pending = true; a_par = pa;
                    pa ^= 1u;
                }
                for (int j = 0; ok && j < I.cnt; ++j) {
                    const int64_t t = a.tiles[I.off + j];
                    for (int kc = 0; kc < a.nk; ++kc) {
                        if (!wait_phase(smem_u32(empty + s), ps ^ 1u, abort_f, a.err, a.wait_ns)) { ok = false; break; }
                        unsigned char *sg = sB + (size_t)s * stage_bytes;
                        mbar_expect_tx(smem_u32(full + s), (uint32_t)stage_bytes);
                        if (a.stream_a) {
                            bulk_g2s(smem_u32(sg), a.qs + ((int64_t)I.qtile * a.nk + kc) * STAGE, STAGE,
                                     smem_u32(full + s));
                            sg += STAGE;
                        }
                        bulk_g2s(smem_u32(sg), a.xs + (t * a.nk + kc) * STAGE, STAGE, smem_u32(full + s));
                        issued[s] = 1; ipar[s] = ps;
                        if (++s == (uint32_t)a.S) { s = 0; ps ^= 1u; }
                    }
                }
            }
            if (!ok) {
                // let the copies already issued land before the CTA can exit
                for (int q = 0; q < a.S; ++q)
                    if (issued[q]) wait_phase(smem_u32(full + q), ipar[q], abort_f, a.err, kWaitNs, true);
                if (a_pending) wait_phase(smem_u32(a_full), a_par, abort_f, a.err, kWaitNs, true);
            }
        }
    } else if (warp == 1) {
        if (lane == 0) {
            // ---------------- MMA issuer
            uint32_t s = 0, ps = 0, pa = 0, acc_it = 0;
            uint32_t pacc[2] = {0u, 0u};
            bool ok = true;
            for (int it = it_begin; ok && it < it_end; ++it) {
                const int cnt = a.items[it].cnt;
                if (!a.stream_a) {
                    if (!wait_phase(smem_u32(a_full), pa, abort_f, a.err, a.wait_ns)) { ok = false; break; }
                    pa ^= 1u;
                }
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                for (int j = 0; ok && j < cnt; ++j) {
                    const uint32_t b = acc_it & 1u;
                    if (!wait_phase(smem_u32(acc_empty + b), pacc[b] ^ 1u, abort_f, a.err, a.wait_ns)) { ok = false; break; }
                    pacc[b] ^= 1u;
                    ++acc_it;
                    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                    const uint32_t dt = tmem + b * TN;
                    for (int kc = 0; kc < a.nk; ++kc) {
                        if (!wait_phase(smem_u32(full + s), ps, abort_f, a.err, a.wait_ns)) { ok = false; break; }
                        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                        const uint32_t sg = smem_u32(sB + (size_t)s * stage_bytes);
                        const uint32_t ah = a.stream_a ? sg : smem_u32(sA + (size_t)kc * STAGE), al = ah + CHUNK;
                        const uint32_t bh = a.stream_a ? sg + STAGE : sg, bl = bh + CHUNK;
#pragma unroll
                        for (int st = 0; st < TK / 16; ++st) {
                            const uint32_t off = st * 32;
                            mma_bf16(dt, sdesc(ah + off), sdesc(bh + off), (kc == 0 && st == 0) ? 0u : 1u);
                            mma_bf16(dt, sdesc(ah + off), sdesc(bl + off), 1u);
                            mma_bf16(dt, sdesc(al + off), sdesc(bh + off), 1u);
                        }
                        mma_commit(smem_u32(empty + s));
                        if (++s == (uint32_t)a.S) { s = 0; ps ^= 1u; }
                    }
                    if (ok) mma_commit(smem_u32(acc_full + b));
                }
                if (ok && !a.stream_a) mma_commit(smem_u32(a_empty));
            }
            // all MMAs issued by this thread complete before the CTA exits
            mma_commit(smem_u32(drain));
            wait_phase(smem_u32(drain), 0u, abort_f, a.err, kWaitNs, true);
        }
    } else {
        // ---------------- epilogue (256 threads, 4 pairs of warps)
        // The two warps of a pair read the same 32 TMEM lanes (rows), one
        // column half each, and are the only ones to touch those rows' state:
        // within a tile they synchronise with a 64-thread barrier of their
        // own. Block-wide barriers remain only where rows change hands (a new
        // query tile, the write-out). After an aborted wait the loops still
        // run to the end (every wait then returns at once), so that all
        // threads meet the same barriers; the host reports the error.
        const int ew = warp - 2;            // 0..7
        const int et = ew * 32 + lane;      // 0..255
        const int quarter = warp & 3;       // TMEM lanes this warp may read
        const int half = ew >> 2;           // column half it reads
        const int pt_i = half * 32 + lane;  // thread index within the pair
        const int my_row = quarter * 32 + lane;
        const bool l2 = a.metric == ESG_L2SQ;
        uint32_t acc_it = 0, tcount = 0;
        uint32_t pe[2] = {0u, 0u};
        int cur_qt = -1;
        // squared norms of a tile into the pair's buffer
        auto load_norms = [&](int32_t tile, float *dst) {
            if (!l2) return;
            const int32_t p0 = tile * TN + pt_i, p1 = p0 + 64;
            dst[pt_i] = p0 < a.n ? __ldg(a.xnorm + p0) : 0.f;
            dst[pt_i + 64] = p1 < a.n ? __ldg(a.xnorm + p1) : 0.f;
        };
        // the CTA's items are consecutive pieces of the covered-tile sequence,
        // so its tiles are one run a.tiles[g_beg, g_end): the index of the
        // tile after next and the next tile's norms are fetched into
        // registers a tile ahead of their use
        const int32_t g_beg = it_begin < it_end ? a.items[it_begin].off : 0;
        const int32_t g_end = it_begin < it_end ? a.items[it_end - 1].off + a.items[it_end - 1].cnt : 0;
        int32_t g_cur = g_beg;
        int32_t tile_cur = g_beg < g_end ? a.tiles[g_beg] : 0;
        int32_t tile_nx = g_beg + 1 < g_end ? a.tiles[g_beg + 1] : -1;
        if (g_beg < g_end) load_norms(tile_cur, s_xn + (quarter * 2) * TN);
        for (int it = it_begin; it < it_end; ++it) {
            const WorkItem I = a.items[it];
            if (I.qtile != cur_qt) {
                // new query tile: per-row state (the lists of the previous tile
                // were written out at the end of its last item)
                if (et < TM) {
                    const int64_t sp = (int64_t)I.qtile * TM + et;
                    int32_t lo = 1, hi = 0;
                    float qn = 0.f;
                    if (sp < a.nv) {
                        const int32_t o = a.qorder[sp];
                        lo = (int32_t)a.l[o]; hi = (int32_t)a.r[o];
                        if (l2) qn = a.qnorm[o];
                    }
                    r_lo[et] = lo; r_hi[et] = hi; r_qn[et] = qn;
                    r_cnt[et] = 0; r_td[et] = INFINITY; r_ti[et] = 0x7FFFFFFF;
                }
                cur_qt = I.qtile;
                epi_bar();
            }
            for (int j = 0; j < I.cnt; ++j, ++g_cur) {
                const int32_t pt = tile_cur * TN;   // first point of the tile
                float *xs_cur = s_xn + (quarter * 2 + (tcount & 1u)) * TN;
                // the next tile's norms (stored after the filter into the
                // pair's other buffer, whose last readers finished before the
                // previous tile's pair barriers) and the index after it
                float *xs_nx = s_xn + (quarter * 2 + ((tcount + 1u) & 1u)) * TN;
                float xn_a = 0.f, xn_b = 0.f;
                if (l2 && tile_nx >= 0) {
                    const int32_t p0 = tile_nx * TN + pt_i, p1 = p0 + 64;
                    xn_a = p0 < a.n ? __ldg(a.xnorm + p0) : 0.f;
                    xn_b = p1 < a.n ? __ldg(a.xnorm + p1) : 0.f;
                }
                const int32_t tile_nx2 = g_cur + 2 < g_end ? __ldg(a.tiles + g_cur + 2) : -1;
                ++tcount;
                const uint32_t b = acc_it & 1u;
                wait_phase(smem_u32(acc_full + b), pe[b], abort_f, a.err, a.wait_ns);
                pe[b] ^= 1u;
                ++acc_it;
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                // the row's range within this half tile; a warp none of whose
                // 32 rows covers it skips the accumulator load and the filter
                const int32_t pbm = pt + half * 64;
                const int32_t lo = r_lo[my_row], hi = r_hi[my_row];
                const int jl = lo - pbm > 0 ? lo - pbm : 0;
                const int jh = hi - pbm < 63 ? hi - pbm : 63;
                const uint64_t rng = jl <= jh ? ((~0ull >> (63 - (jh - jl))) << jl) : 0ull;
                const bool warp_in = __any_sync(0xffffffffu, rng != 0ull);
                float v[64];
                if (warp_in) tmem_ld64(tmem + ((uint32_t)(quarter * 32) << 16) + b * TN + half * 64, v);
                asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
                __syncwarp();
                if (lane == 0) mbar_arrive(smem_u32(acc_empty + b));
                // filter, one thread per row and half: distances of the 64
                // columns, range mask, and the columns at or below the row's
                // current K1-th distance (a superset of the insertions)
                uint64_t cand = 0ull;
                if (warp_in) {
                    const float qn = r_qn[my_row], tdm = r_td[my_row];
                    const float4 *xv = (const float4 *)(xs_cur + half * 64);
#pragma unroll
                    for (int c4 = 0; c4 < 16; ++c4) {
                        const float4 x4 = xv[c4];
                        const float xx[4] = {x4.x, x4.y, x4.z, x4.w};
#pragma unroll
                        for (int e = 0; e < 4; ++e) {
                            const int c = c4 * 4 + e;
                            const float dd = l2 ? qn + xx[e] - 2.f * v[c] : -v[c];
                            v[c] = dd;
                            cand |= (uint64_t)(dd <= tdm) << c;
                        }
                    }
                    cand &= rng;
                }
                if (l2 && tile_nx >= 0) { xs_nx[pt_i] = xn_a; xs_nx[pt_i + 64] = xn_b; }
                const bool fl = cand != 0ull;
                const uint32_t wm = __ballot_sync(0xffffffffu, fl);
                if (lane == 0) s_flag[half * 4 + quarter] = wm;
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    // flagged rows of this half pass their distances through
                    // shared memory (out-of-range columns as +inf)
                    if (half == h && fl) {
#pragma unroll
                        for (int c = 0; c < 64; ++c)
                            T[my_row * kTS + c] = ((rng >> c) & 1ull) ? v[c] : INFINITY;
                    }
                    pair_bar(quarter);
                    // warp-cooperative insertion: the k-th flagged row of the
                    // pair's 32 goes to the pair's warp k mod 2
                    const int32_t pb = pt + h * 64;
                    uint32_t w = s_flag[h * 4 + quarter];
                    int k = 0;
                    while (w != 0u) {
                        const int bit = __ffs(w) - 1;
                        w &= w - 1;
                        if ((k++ & 1) != half) continue;
                        const int r = quarter * 32 + bit;
                        const int32_t p0 = pb + lane, p1 = p0 + 32;
                        const float d0 = T[r * kTS + lane], d1 = T[r * kTS + lane + 32];
                        float td = r_td[r];
                        int32_t ti = r_ti[r];
                        uint32_t m0 = __ballot_sync(0xffffffffu, d0 < INFINITY && dl_less(d0, p0, td, ti));
                        uint32_t m1 = __ballot_sync(0xffffffffu, d1 < INFINITY && dl_less(d1, p1, td, ti));
                        if ((m0 | m1) == 0u) continue;                  // warp-uniform
                        // the row's list in registers: entries lane and lane + 32
                        int cnt = r_cnt[r];
                        float ld0 = lane < cnt ? L_d[r * K1 + lane] : INFINITY;
                        int32_t li0 = lane < cnt ? L_i[r * K1 + lane] : 0x7FFFFFFF;
                        float ld1 = lane + 32 < cnt ? L_d[r * K1 + lane + 32] : INFINITY;
                        int32_t li1 = lane + 32 < cnt ? L_i[r * K1 + lane + 32] : 0x7FFFFFFF;
                        const int nc = __popc(m0) + __popc(m1);
                        if (nc >= kBulkMin) {
                            // the K1 smallest of list and candidates in one
                            // network: the same list as inserting one by one
                            const bool in0 = (m0 >> lane) & 1u, in1 = (m1 >> lane) & 1u;
                            float cd[2] = {in0 ? d0 : INFINITY, in1 ? d1 : INFINITY};
                            int32_t ci[2] = {in0 ? p0 : 0x7FFFFFFF, in1 ? p1 : 0x7FFFFFFF};
                            bitonic_sort64(cd, ci, lane, true);
                            float ld[2] = {ld0, ld1};
                            int32_t li[2] = {li0, li1};
                            bitonic_merge_into(ld, li, cd, ci, lane);
                            ld0 = ld[0]; li0 = li[0]; ld1 = ld[1]; li1 = li[1];
                            cnt = min(K1, cnt + nc);
                            if (cnt == K1) {
                                const int e = K1 - 1;
                                td = __shfl_sync(0xffffffffu, e < 32 ? ld0 : ld1, e & 31);
                                ti = __shfl_sync(0xffffffffu, e < 32 ? li0 : li1, e & 31);
                            }
                            m0 = m1 = 0u;
                        }
                        while ((m0 | m1) != 0u) {
                            const bool second = m0 == 0u;
                            const int src = __ffs(second ? m1 : m0) - 1;
                            if (second) m1 &= m1 - 1; else m0 &= m0 - 1;
                            const float cd = __shfl_sync(0xffffffffu, second ? d1 : d0, src);
                            const int32_t ci = pb + (second ? 32 : 0) + src;
                            if (cnt == K1 && !dl_less(cd, ci, td, ti)) continue;
                            const int pos = __popc(__ballot_sync(0xffffffffu, lane < cnt && dl_less(ld0, li0, cd, ci))) +
                                            __popc(__ballot_sync(0xffffffffu, lane + 32 < cnt && dl_less(ld1, li1, cd, ci)));
                            const float u0d = __shfl_up_sync(0xffffffffu, ld0, 1);
                            const int32_t u0i = __shfl_up_sync(0xffffffffu, li0, 1);
                            float u1d = __shfl_up_sync(0xffffffffu, ld1, 1);
                            int32_t u1i = __shfl_up_sync(0xffffffffu, li1, 1);
                            const float t31d = __shfl_sync(0xffffffffu, ld0, 31);
                            const int32_t t31i = __shfl_sync(0xffffffffu, li0, 31);
                            if (lane == 0) { u1d = t31d; u1i = t31i; }
                            if (lane > pos) { ld0 = u0d; li0 = u0i; }
                            else if (lane == pos) { ld0 = cd; li0 = ci; }
                            if (lane + 32 > pos) { ld1 = u1d; li1 = u1i; }
                            else if (lane + 32 == pos) { ld1 = cd; li1 = ci; }
                            if (cnt < K1) ++cnt;
                            if (cnt == K1) {
                                const int e = K1 - 1;
                                td = __shfl_sync(0xffffffffu, e < 32 ? ld0 : ld1, e & 31);
                                ti = __shfl_sync(0xffffffffu, e < 32 ? li0 : li1, e & 31);
                            }
                        }
                        if (lane < cnt) { L_d[r * K1 + lane] = ld0; L_i[r * K1 + lane] = li0; }
                        if (lane + 32 < cnt) { L_d[r * K1 + lane + 32] = ld1; L_i[r * K1 + lane + 32] = li1; }
                        if (lane == 0) { r_cnt[r] = cnt; r_td[r] = td; r_ti[r] = ti; }
                        __syncwarp();
                    }
                    pair_bar(quarter);
                }
                tile_cur = tile_nx;
                tile_nx = tile_nx2;
            }
            // write the lists out when this is the CTA's last item of the
            // query tile (a row's list then covers all of the tile's items
            // this CTA ran); other items record empty lists
            const bool flush = it + 1 == it_end || a.items[it + 1].qtile != I.qtile;
            if (flush) epi_bar();   // every pair's insertions are done
            for (int r = et; r < TM; r += 32 * kEpiWarps) {
                const int c = flush ? r_cnt[r] : 0;
                a.part_n[(int64_t)it * TM + r] = c;
            }
            if (flush) {
                for (int idx = et; idx < TM * K1; idx += 32 * kEpiWarps) {
                    const int r = idx / K1, e = idx % K1;
                    if (e < r_cnt[r]) {
                        a.part_d[(int64_t)it * TM * K1 + idx] = L_d[idx];
                        a.part_i[(int64_t)it * TM * K1 + idx] = L_i[idx];
                    }
                }
                epi_bar();
            }
        }
    }
    __syncthreads();
    if (warp == 1) {
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" :: "r"(tmem), "r"(2 * TN) : "memory");
    }
}

// One thread per (row, 8 dimensions) of the padded matrix: FP32 -> BF16 hi
// and lo parts, written into the tiled, swizzled block layout. Row `i` of the
// output is input row order[i] (or i), rows past `rows` are zero.
__global__ void tile_split_kernel(const float *X, int64_t rows, int d, int nk, const int32_t *order,
                                  int64_t rows_pad, unsigned char *out) {
    const int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (idx >= rows_pad * nk * 8) return;
    const int64_t row = idx / (nk * 8);
    const int g = (int)(idx % (nk * 8));
    const int kc = g >> 3, c = g & 7;
    const int64_t src = row < rows ? (order ? (int64_t)order[row] : row) : -1;
    __align__(16) __nv_bfloat16 h[8];
    __align__(16) __nv_bfloat16 lo[8];
#pragma unroll
    for (int e = 0; e < 8; ++e) {
        const int k = kc * TK + c * 8 + e;
        const float v = (src >= 0 && k < d) ? X[src * d + k] : 0.f;
        h[e] = __float2bfloat16_rn(v);
        lo[e] = __float2bfloat16_rn(v - __bfloat162float(h[e]));
    }
    const int64_t tile = row >> 7;
    const int t = (int)(row & 127);
    unsigned char *blk = out + (tile * nk + kc) * (int64_t)STAGE;
    const uint32_t off = t * 128 + ((c ^ (t & 7)) << 4);
    *(uint4 *)(blk + off) = *(const uint4 *)h;
    *(uint4 *)(blk + CHUNK + off) = *(const uint4 *)lo;
}

__global__ void norms_kernel(const float *X, int64_t rows, int d, float *norm, float *rownorm) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= rows) return;
    const float *x = X + i * d;
    float s = 0.f;
    for (int j = 0; j < d; ++j) s = fmaf(x[j], x[j], s);
    norm[i] = s;
    rownorm[i] = sqrtf(s);
}

// Merge the per-item top-K1 lists of each valid query (one warp per sorted
// position) into one top-K1 list in the caller's query order. Lists are
// ascending in (distance, row) and hold distinct rows, so the position of
// an element in the merged list is its own index plus the number of
// elements of the other list that precede it.
__global__ void merge_parts_kernel(const float *part_d, const int32_t *part_i, const int32_t *part_n,
                                   const int32_t *item_begin, const int32_t *qorder, int64_t nv, int K1,
                                   float *cand_d, int32_t *cand_i, int32_t *cand_n) {
    __shared__ Cand buf[4][3][kMaxK1v2];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int64_t sp = blockIdx.x * (int64_t)4 + w;
    if (sp >= nv) return;
    const int64_t qt = sp / TM;
    const int row = (int)(sp % TM);
    Cand *A = buf[w][0], *B = buf[w][1], *C = buf[w][2];
    int na = 0;
    for (int it = item_begin[qt]; it < item_begin[qt + 1]; ++it) {
        const int64_t sub = (int64_t)it * TM + row;
        const int nb = part_n[sub];
        if (nb <= 0) continue;
        for (int e = lane; e < nb; e += 32)
            B[e] = Cand{part_d[sub * K1 + e], (uint32_t)part_i[sub * K1 + e]};
        __syncwarp();
        for (int i = lane; i < na; i += 32) {
            int lo = 0, hi = nb;   // number of B elements before A[i]
            while (lo < hi) {
                const int m = (lo + hi) >> 1;
                if (cand_less(B[m].d, B[m].id, A[i].d, A[i].id)) lo = m + 1; else hi = m;
            }
            if (i + lo < K1) C[i + lo] = A[i];
        }
        for (int j = lane; j < nb; j += 32) {
            int lo = 0, hi = na;   // number of A elements before B[j]
            while (lo < hi) {
                const int m = (lo + hi) >> 1;
                if (cand_less(A[m].d, A[m].id, B[j].d, B[j].id)) lo = m + 1; else hi = m;
            }
            if (j + lo < K1) C[j + lo] = B[j];
        }
        __syncwarp();
        Cand *t = A; A = C; C = t;
        na = min(K1, na + nb);
    }
    const int32_t o = qorder[sp];
    for (int e = lane; e < na; e += 32) {
        cand_d[(int64_t)o * K1 + e] = A[e].d;
        cand_i[(int64_t)o * K1 + e] = (int32_t)A[e].id;
    }
    if (lane == 0) cand_n[o] = na;
}

}  // namespace

// Exact FP32 re-rank of the candidate lists and certificate. The queries left
// uncertified go to `leftover` when it is given, else through the exact SIMT
// pass here.
static esg_status certify_and_redo(const float *base, int64_t n, int32_t d, int metric, const float *queries,
                                   int64_t nq, const int64_t *l, const int64_t *r, int32_t k, int K1,
                                   const float *cand_d, const int32_t *cand_i, const int32_t *cand_n,
                                   const float *qrow, const float *xmax, int32_t *redo, const int32_t *err,
                                   int64_t *out_ids, float *out_dist, int32_t *out_count, cudaStream_t stream,
                                   std::vector<int64_t> *leftover = nullptr) {
    rerank_certify_kernel<<<ceil_div_i(nq, 4), 128, 0, stream>>>(
        base, queries, d, metric, nq, k, K1, cand_d, cand_i, cand_n, qrow, xmax, out_ids, out_dist, out_count, redo);
    cudaError_t ce = cudaGetLastError();
    if (ce != cudaSuccess) { esg_set_error(cudaGetErrorString(ce)); return ESG_ERR_CUDA; }
    std::vector<int32_t> h_redo(nq);
    int32_t h_err = 0;
    ce = cudaMemcpyAsync(h_redo.data(), redo, sizeof(int32_t) * nq, cudaMemcpyDeviceToHost, stream);
    if (ce == cudaSuccess) ce = cudaMemcpyAsync(&h_err, err, sizeof(int32_t), cudaMemcpyDeviceToHost, stream);
    if (ce == cudaSuccess) ce = cudaStreamSynchronize(stream);
    if (ce != cudaSuccess) { esg_set_error(cudaGetErrorString(ce)); return ESG_ERR_CUDA; }
    if (h_err) { esg_set_error("tensor-core brute force: an mbarrier wait timed out"); return ESG_ERR_TIMEOUT; }
    std::vector<int64_t> idx;
    for (int64_t i = 0; i < nq; ++i) if (h_redo[i]) idx.push_back(i);
    const char *dbg = getenv("ESG_BF_STATS");
    if (dbg && *dbg == '1')
        fprintf(stderr, "tensor-core brute force: %lld of %lld queries left uncertified (list of %d)\n",
                (long long)idx.size(), (long long)nq, K1);
    if (leftover) { leftover->swap(idx); return ESG_OK; }
    if (idx.empty()) return ESG_OK;
    return esg_bruteforce_redo(base, n, d, metric, queries, nq, l, r, k, idx, out_ids, out_dist, out_count, stream);
}

// Shared-memory plan of the pipelined kernel for a dimension and list length:
// the query tile resident when that leaves room for two point stages, else
// streamed with the point chunks (stages of 64 KB); ESG_ERR_UNSUPPORTED when
// not even two streamed stages fit.
static esg_status bf2_smem(int32_t d, int K1, int max_smem, int *S, size_t *smem, int *stream_a) {
    if (K1 > kMaxK1v2 || d < 1) return ESG_ERR_UNSUPPORTED;
    const int nk = (d + TK - 1) / TK;
    const size_t common = 1024 + (size_t)TM * kTS * 4 + 8 * TN * 4 + (size_t)TM * K1 * 8 + 6 * TM * 4 + 8 * 4 +
                          8 * (2 * kMaxStages + 8) + 16;
    const size_t resident = common + (size_t)nk * STAGE;
    if ((size_t)max_smem >= resident + 2 * (size_t)STAGE) {
        *stream_a = 0;
        *S = (int)std::min<size_t>(kMaxStages, ((size_t)max_smem - resident) / STAGE);
        *smem = resident + (size_t)*S * STAGE;
        return ESG_OK;
    }
    if ((size_t)max_smem < common + 4 * (size_t)STAGE) return ESG_ERR_UNSUPPORTED;
    *stream_a = 1;
    *S = (int)std::min<size_t>(kMaxStages, ((size_t)max_smem - common) / (2 * STAGE));
    *smem = common + (size_t)*S * 2 * STAGE;
    return ESG_OK;
}

// The point side, prepared once per call: tiled BF16 splits, squared norms,
// row norms and their maximum.
struct PreparedX {
    const unsigned char *xs;
    const float *xnorm, *xrow, *xmax;
};

__global__ void gather_subset_kernel(const float *Q, const int64_t *l, const int64_t *r, int d,
                                     const int64_t *idx, int64_t m, float *Qg, int64_t *lg, int64_t *rg) {
    const int64_t i = blockIdx.x;
    if (i >= m) return;
    const int64_t q = idx[i];
    for (int j = threadIdx.x; j < d; j += blockDim.x) Qg[i * d + j] = Q[q * d + j];
    if (threadIdx.x == 0) { lg[i] = l[q]; rg[i] = r[q]; }
}

__global__ void scatter_subset_kernel(const int64_t *idx, int64_t m, int k, const int64_t *ids_g,
                                      const float *dist_g, const int32_t *cnt_g, int64_t *ids, float *dist,
                                      int32_t *cnt) {
    const int64_t i = blockIdx.x;
    if (i >= m) return;
    const int64_t q = idx[i];
    for (int j = threadIdx.x; j < k; j += blockDim.x) {
        ids[q * k + j] = ids_g[i * k + j];
        dist[q * k + j] = dist_g[i * k + j];
    }
    if (threadIdx.x == 0) cnt[q] = cnt_g[i];
}

// Host clock (ms) for the ESG_BF_STATS=1 phase report.
static double bf_host_ms() {
    return std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now().time_since_epoch()).count();
}
static bool bf_stats() {
    const char *dbg = getenv("ESG_BF_STATS");
    return dbg && *dbg == '1';
}

struct Bf2Plan;
static esg_status bf2_queries(const PreparedX &X, const float *base, int64_t n, int32_t d, int metric,
                              const float *queries, int64_t nq, const int64_t *l, const int64_t *r, int32_t k,
                              int K1, int64_t *out_ids, float *out_dist, int32_t *out_count, cudaStream_t stream,
                              Bf2Plan *given = nullptr);

// Queries whose list of K1 candidates could not be certified run again with
// the longest list that fits the kernel (their own plan, a few query tiles), and
// through the exact SIMT kernel if they are still uncertified.
static esg_status bf2_escalate(const PreparedX &X, const float *base, int64_t n, int32_t d, int metric,
                               const float *queries, int64_t nq, const int64_t *l, const int64_t *r, int32_t k,
                               int K1, const std::vector<int64_t> &idx, int64_t *out_ids, float *out_dist,
                               int32_t *out_count, cudaStream_t stream) {
    int dev = 0, max_smem = 0, S = 0;
    size_t smem = 0;
    ESG_CUDA_TRY(cudaGetDevice(&dev));
    ESG_CUDA_TRY(cudaDeviceGetAttribute(&max_smem, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
    int K2 = kMaxK1v2;   // the longest list that fits
    int sa_mode = 0;
    while (K2 > K1 && bf2_smem(d, K2, max_smem, &S, &smem, &sa_mode) != ESG_OK) --K2;
    if (K2 <= K1)
        return esg_bruteforce_redo(base, n, d, metric, queries, nq, l, r, k, idx, out_ids, out_dist, out_count, stream);
    const int64_t m = (int64_t)idx.size();
    auto al = [](size_t x) { return (x + 255) & ~(size_t)255; };
    const size_t bytes = al(sizeof(int64_t) * m) + al(sizeof(float) * m * d) + 2 * al(sizeof(int64_t) * m) +
                         al(sizeof(int64_t) * m * k) + al(sizeof(float) * m * k) + al(sizeof(int32_t) * m);
    unsigned char *sc = nullptr;
    ESG_CUDA_TRY(esg_malloc_async((void **)&sc, bytes, stream));
    unsigned char *p = sc;
    int64_t *didx = (int64_t *)p; p += al(sizeof(int64_t) * m);
    float *Qg = (float *)p; p += al(sizeof(float) * m * d);
    int64_t *lg = (int64_t *)p; p += al(sizeof(int64_t) * m);
    int64_t *rg = (int64_t *)p; p += al(sizeof(int64_t) * m);
    int64_t *ig = (int64_t *)p; p += al(sizeof(int64_t) * m * k);
    float *dg = (float *)p; p += al(sizeof(float) * m * k);
    int32_t *cg = (int32_t *)p;
    esg_status st = ESG_OK;
    cudaError_t ce = cudaMemcpyAsync(didx, idx.data(), sizeof(int64_t) * m, cudaMemcpyHostToDevice, stream);
    if (ce == cudaSuccess) {
        gather_subset_kernel<<<(unsigned)m, 128, 0, stream>>>(queries, l, r, d, didx, m, Qg, lg, rg);
        ce = cudaGetLastError();
    }
    if (ce != cudaSuccess) { esg_set_error(cudaGetErrorString(ce)); st = ESG_ERR_CUDA; }
    if (st == ESG_OK) st = bf2_queries(X, base, n, d, metric, Qg, m, lg, rg, k, K2, ig, dg, cg, stream);
    if (st == ESG_OK) {
        scatter_subset_kernel<<<(unsigned)m, 128, 0, stream>>>(didx, m, k, ig, dg, cg, out_ids, out_dist, out_count);
        ce = cudaGetLastError();
        if (ce != cudaSuccess) { esg_set_error(cudaGetErrorString(ce)); st = ESG_ERR_CUDA; }
    }
    // the host index vector must outlive the copy above
    const cudaError_t se = cudaStreamSynchronize(stream);
    if (st == ESG_OK && se != cudaSuccess) { esg_set_error(cudaGetErrorString(se)); st = ESG_ERR_CUDA; }
    cudaFreeAsync(sc, stream);
    return st;
}

// One pass of the pipelined kernel over a batch of queries against the
// prepared points, then merge, re-rank, certificate and escalation.
// Cuts the sequence of covered point tiles (query tile by query tile) into G
// contiguous shares of about equal estimated cost. A share's cost is its
// number of tiles plus `restart` for every (query, work item) pair in which
// the query covers at least one of the item's tiles: a row list starts empty
// at each item, and while it fills the epilogue inserts many candidates per
// tile. Per-CTA clock counters at d = 128 (two 64-wide K chunks) put a list
// start at about six tiles of MMA and filter time (the later insertions did
// not improve the fit). The epilogue work does not grow with d while a tile's
// MMA work does, and the longer MMA time per tile also hides more of the
// burst: the weight 6.25 (2 / nk)^2 tiles fits the best measured weights at
// d = 128 (6.25) and d = 768 (0 to 0.5, where equal shares are as good).
// Each cut inside a query tile costs the restarts of the lists of the queries
// that span it. The shares are chosen greedily: each CTA takes about the
// remaining cost over the remaining CTAs; every later pass adds the restart
// cost of the previous pass's later cuts to the remaining cost, and the pass
// with the smallest largest share is kept. `lt`/`rt` are the first and last
// covered tile of each sorted query; `cut` receives G + 1 positions.
constexpr double kRestart2 = 6.25;   // one list start, in tiles, at two K chunks
constexpr int kSharePasses = 2;      // greedy passes (the first without restart look-ahead)

static void bf2_shares(const std::vector<int32_t> &tiles, const std::vector<int64_t> &qt_first,
                       const std::vector<int32_t> &lt, const std::vector<int32_t> &rt, int64_t G,
                       double restart, std::vector<int64_t> &cut) {
    const int64_t T = (int64_t)tiles.size(), nqt = (int64_t)qt_first.size() - 1;
    const int64_t nv = (int64_t)lt.size();
    cut.assign(G + 1, T);
    cut[0] = 0;
    if (G <= 1 || nqt <= 0) return;
    // estimated cost of tiles [t0, t1) of query tile qt, run as one item
    auto cost = [&](int64_t qt, int64_t t0, int64_t t1) -> double {
        if (t1 <= t0) return 0.0;
        const int32_t a = tiles[t0], b = tiles[t1 - 1];
        const int32_t *lq = lt.data() + qt * TM, *rq = rt.data() + qt * TM;
        const int ns = (int)(std::min(nv, (qt + 1) * TM) - qt * TM);
        int nover = 0;
        for (int s = 0; s < ns; ++s) nover += rq[s] >= a && lq[s] <= b;
        return (double)(t1 - t0) + restart * nover;
    };
    std::vector<double> pre(nqt + 1, 0.0);   // prefix sums of whole query tiles
    for (int64_t qt = 0; qt < nqt; ++qt) pre[qt + 1] = pre[qt] + cost(qt, qt_first[qt], qt_first[qt + 1]);
    // about the largest e in [lo, hi] with f(e) = cost(qt, t0, e) <= budget,
    // given f(lo) = flo <= budget < f(hi) = fhi: interpolation steps
    // alternating with bisection, stopping within 1 % of the budget; f(e) in *fe
    auto last_within = [&](int64_t qt, int64_t t0, int64_t lo, int64_t hi, double flo, double fhi, double budget,
                           double *fe) {
        for (int step = 0; hi - lo > 1 && fhi - flo > 1e-2 * budget; ++step) {
            int64_t mid = lo + (hi - lo) / 2;
            if (step % 2 == 0) mid = lo + (int64_t)((budget - flo) / (fhi - flo) * (double)(hi - lo));
            mid = std::min(std::max(mid, lo + 1), hi - 1);
            const double fm = cost(qt, t0, mid);
            if (fm <= budget) { lo = mid; flo = fm; } else { hi = mid; fhi = fm; }
        }
        *fe = flo;
        return lo;
    };
    // one greedy pass: CTA c takes about (remaining cost + later[c]) / (G - c);
    // returns the largest share's cost, the heads (cost from each cut to the
    // end of its query tile) in `head`
    std::vector<double> head(G, 0.0);
    auto greedy = [&](const std::vector<double> &later, std::vector<int64_t> &cu) {
        cu.assign(G + 1, T);
        cu[0] = 0;
        int64_t t = 0, qt = 0;
        double worst = 0.0;
        for (int64_t c = 0; c < G; ++c) {
            while (qt_first[qt + 1] <= t) ++qt;
            const int64_t qend = qt_first[qt + 1];
            const double h = t == qt_first[qt] ? pre[qt + 1] - pre[qt] : cost(qt, t, qend);
            head[c] = h;
            const double rest = h + pre[nqt] - pre[qt + 1];
            if (c + 1 == G) { worst = std::max(worst, rest); break; }
            const double target = (rest + later[c]) / (double)(G - c);
            int64_t e;
            double share;
            if (h > target) {
                e = last_within(qt, t, t, qend, 0.0, h, target, &share);
            } else {
                // the query tile the cut falls in, then the position inside it
                const double rem = target - h;
                const int64_t qe = std::upper_bound(pre.begin() + qt + 1, pre.end(), pre[qt + 1] + rem) - pre.begin() - 1;
                if (qe >= nqt) {
                    e = T;
                    share = rest;
                } else {
                    double part = 0.0;
                    e = last_within(qe, qt_first[qe], qt_first[qe], qt_first[qe + 1], 0.0, pre[qe + 1] - pre[qe],
                                    rem - (pre[qe] - pre[qt + 1]), &part);
                    share = h + (pre[qe] - pre[qt + 1]) + part;
                }
            }
            if (e < t + 1 || e > T - (G - c - 1)) {
                e = std::min(std::max(e, t + 1), T - (G - c - 1));
                const int64_t qe = std::upper_bound(qt_first.begin(), qt_first.end(), e - 1) - qt_first.begin() - 1;
                share = qe == qt ? cost(qt, t, e) : h + (pre[qe] - pre[qt + 1]) + cost(qe, qt_first[qe], e);
            }
            worst = std::max(worst, share);
            cu[c + 1] = e;
            t = e;
        }
        return worst;
    };
    std::vector<double> later(G, 0.0);
    std::vector<int64_t> cur, nxt;
    double best = greedy(later, cur);
    cut = cur;
    for (int pass = 1; pass < kSharePasses; ++pass) {
        // restart cost of each cut of the previous pass (the next share's head
        // plus the query tile's cost up to the cut, minus the whole query
        // tile), summed over the later cuts
        for (int64_t c = G - 2; c >= 0; --c) {
            const int64_t t = cur[c + 1];
            double o = 0.0;
            if (t < T) {
                const int64_t qt = std::upper_bound(qt_first.begin(), qt_first.end(), t) - qt_first.begin() - 1;
                if (t > qt_first[qt]) o = head[c + 1] + cost(qt, qt_first[qt], t) - (pre[qt + 1] - pre[qt]);
            }
            later[c] = later[c + 1] + o;
        }
        const double w = greedy(later, nxt);
        if (w < best) { best = w; cut = nxt; }
        cur.swap(nxt);
    }
}

// Host work plan of the pipelined kernel for the valid queries of host
// ranges hl/hr over n points at dimension d, for `sms` CTAs: queries sorted
// by (log2 width, l, index) and tiled by 128, the rows of each full query tile
// interleaved over the four TMEM lane quarters, the point tiles each query
// tile covers in one sequence, cut into `G` shares (bf2_shares) and into work
// items at query-tile boundaries. ESG_ERR_UNSUPPORTED past 2^31 covered tiles.
struct Bf2Plan {
    std::vector<int32_t> order;        // sorted position -> caller's query index (valid queries)
    std::vector<int32_t> tiles;        // covered point tiles, query tile by query tile
    std::vector<int64_t> qt_first;     // [nqt + 1] first position of each query tile in `tiles`
    std::vector<WorkItem> items;       // in query-tile order, each CTA's items contiguous
    std::vector<int32_t> item_begin;   // [nqt + 1] first item of each query tile
    std::vector<int32_t> cta_first;    // [G + 1] first item of each CTA
    int64_t nv = 0, nqt = 0, total_tiles = 0, G = 0, largest = 0;
};

static esg_status bf2_plan(const int64_t *hl, const int64_t *hr, int64_t nq, int64_t n, int32_t d, int64_t sms,
                           Bf2Plan &P) {
    // sort key floor(log2 width) << 40 | l (l < 2^31), ties by query index:
    // a stable LSD radix sort by bytes of the key over the valid queries in
    // index order
    struct Key { uint64_t k; int32_t i; };
    std::vector<Key> keys, tmp;
    keys.reserve(nq);
    uint64_t kmax = 0;
    for (int64_t i = 0; i < nq; ++i)
        if (hl[i] >= 0 && hl[i] <= hr[i] && hr[i] < n) {
            const uint64_t wb = 63 - __builtin_clzll((unsigned long long)(hr[i] - hl[i] + 1));
            keys.push_back(Key{(wb << 40) | (uint64_t)hl[i], (int32_t)i});
            kmax = std::max(kmax, keys.back().k);
        }
    tmp.resize(keys.size());
    for (int sh = 0; sh < 64 && (kmax >> sh) != 0; sh += 8) {
        size_t cnt[257] = {0};
        for (const Key &x : keys) ++cnt[((x.k >> sh) & 255) + 1];
        for (int b = 0; b < 256; ++b) cnt[b + 1] += cnt[b];
        for (const Key &x : keys) tmp[cnt[(x.k >> sh) & 255]++] = x;
        keys.swap(tmp);
    }
    std::vector<int32_t> &order = P.order;
    order.resize(keys.size());
    for (size_t s = 0; s < keys.size(); ++s) order[s] = keys[s].i;
    const int64_t nv = (int64_t)order.size();
    const int64_t nqt = (nv + TM - 1) / TM;
    const int nk = (d + TK - 1) / TK;
    std::vector<std::vector<std::pair<int64_t, int64_t>>> spans(nqt);
    int64_t total_tiles = 0;
    std::vector<std::pair<int64_t, int64_t>> iv;
    iv.reserve(TM);
    for (int64_t qt = 0; qt < nqt; ++qt) {
        iv.clear();
        for (int64_t s = qt * TM; s < std::min(nv, (qt + 1) * TM); ++s)
            iv.push_back({hl[order[s]] / TN, hr[order[s]] / TN});
        if (!std::is_sorted(iv.begin(), iv.end())) std::sort(iv.begin(), iv.end());
        for (auto &x : iv) {
            if (!spans[qt].empty() && x.first <= spans[qt].back().second + 1)
                spans[qt].back().second = std::max(spans[qt].back().second, x.second);
            else
                spans[qt].push_back(x);
        }
        for (auto &x : spans[qt]) total_tiles += x.second - x.first + 1;
    }
    // the rows of each full query tile interleaved over the four TMEM lane
    // quarters (sorted position s -> row (s mod 4) * 32 + s / 4): queries
    // with nearby ranges take their insertions in the same point tiles, and
    // an accumulator is free only when all four epilogue warp pairs are done
    for (int64_t qt = 0; qt < nv / TM; ++qt) {
        int32_t rows[TM];
        for (int i = 0; i < TM; ++i) rows[(i & 3) * 32 + (i >> 2)] = order[qt * TM + i];
        std::copy(rows, rows + TM, order.begin() + qt * TM);
    }
    if (total_tiles >= ((int64_t)1 << 31)) return ESG_ERR_UNSUPPORTED;
    // the covered tiles of all query tiles in one sequence (query tile by query
    // tile); CTA c runs the share [cut[c], cut[c + 1]) of it, shares of equal
    // estimated cost, cut into work items at query-tile boundaries (items in
    // query-tile order, each CTA's items contiguous)
    std::vector<int32_t> &tiles = P.tiles;
    tiles.resize(total_tiles);
    std::vector<int64_t> &qt_first = P.qt_first;
    qt_first.assign(nqt + 1, 0);
    int64_t pos = 0;
    for (int64_t qt = 0; qt < nqt; ++qt) {
        qt_first[qt] = pos;
        for (auto &x : spans[qt])
            for (int64_t t = x.first; t <= x.second; ++t) tiles[pos++] = (int32_t)t;
    }
    qt_first[nqt] = pos;
    const int64_t G = std::max<int64_t>(1, std::min<int64_t>(sms, total_tiles));
    std::vector<int64_t> cut;
    {
        std::vector<int32_t> lt(nv), rt(nv);
        for (int64_t s = 0; s < nv; ++s) { lt[s] = (int32_t)(hl[order[s]] / TN); rt[s] = (int32_t)(hr[order[s]] / TN); }
        bf2_shares(tiles, qt_first, lt, rt, G, kRestart2 * (2.0 / nk) * (2.0 / nk), cut);
    }
    std::vector<WorkItem> &items = P.items;
    items.clear();
    std::vector<int32_t> &item_begin = P.item_begin, &cta_first = P.cta_first;
    item_begin.assign(nqt + 1, 0);
    cta_first.assign(G + 1, 0);
    for (int64_t c = 0; c < G; ++c) {
        cta_first[c] = (int32_t)items.size();
        const int64_t t0 = cut[c], t1 = cut[c + 1];
        int64_t t = t0;
        int64_t qt = std::upper_bound(qt_first.begin(), qt_first.end(), t0) - qt_first.begin() - 1;
        while (t < t1) {
            while (qt_first[qt + 1] <= t) ++qt;
            const int64_t e = std::min(t1, qt_first[qt + 1]);
            items.push_back(WorkItem{(int32_t)qt, (int32_t)t, (int32_t)(e - t), 0});
            t = e;
        }
    }
    cta_first[G] = (int32_t)items.size();
    for (int64_t qt = 0, i = 0; qt <= nqt; ++qt) {   // first item of each query tile
        while (i < (int64_t)items.size() && items[i].qtile < qt) ++i;
        item_begin[qt] = (int32_t)i;
    }
    P.largest = 0;
    for (int64_t c = 0; c < G; ++c) P.largest = std::max(P.largest, cut[c + 1] - cut[c]);
    P.nv = nv;
    P.nqt = nqt;
    P.total_tiles = total_tiles;
    P.G = G;
    return ESG_OK;
}

// `given`: a plan already made for these ranges (it is consumed), or null.
static esg_status bf2_queries(const PreparedX &X, const float *base, int64_t n, int32_t d, int metric,
                              const float *queries, int64_t nq, const int64_t *l, const int64_t *r, int32_t k,
                              int K1, int64_t *out_ids, float *out_dist, int32_t *out_count, cudaStream_t stream,
                              Bf2Plan *given) {
    if (nq == 0) return ESG_OK;
    const double h0 = bf_stats() ? bf_host_ms() : 0.0;
    const int nk = (d + TK - 1) / TK;
    int dev = 0, max_smem = 0, sms = 0, S = 0, stream_a = 0;
    size_t smem = 0;
    ESG_CUDA_TRY(cudaGetDevice(&dev));
    ESG_CUDA_TRY(cudaDeviceGetAttribute(&max_smem, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
    ESG_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    if (bf2_smem(d, K1, max_smem, &S, &smem, &stream_a) != ESG_OK) return ESG_ERR_UNSUPPORTED;

    // ---- host plan
    Bf2Plan P;
    if (given) {
        P = std::move(*given);
    } else {
        std::vector<int64_t> hl(nq), hr(nq);
        ESG_CUDA_TRY(cudaMemcpyAsync(hl.data(), l, sizeof(int64_t) * nq, cudaMemcpyDeviceToHost, stream));
        ESG_CUDA_TRY(cudaMemcpyAsync(hr.data(), r, sizeof(int64_t) * nq, cudaMemcpyDeviceToHost, stream));
        ESG_CUDA_TRY(cudaStreamSynchronize(stream));
        const esg_status pst = bf2_plan(hl.data(), hr.data(), nq, n, d, sms, P);
        if (pst != ESG_OK) return pst;
    }
    const std::vector<int32_t> &order = P.order, &tiles = P.tiles, &item_begin = P.item_begin,
                               &cta_first = P.cta_first;
    const std::vector<WorkItem> &items = P.items;
    const int64_t nv = P.nv, nqt = P.nqt, total_tiles = P.total_tiles, G = P.G, CH = P.largest;
    const int64_t n_items = (int64_t)items.size();

    // ---- query-side scratch
    auto al = [](size_t x) { return (x + 255) & ~(size_t)255; };
    const int64_t ni1 = std::max<int64_t>(n_items, 1);
    size_t bytes = al((size_t)std::max<int64_t>(nqt, 1) * nk * STAGE) + 2 * al(sizeof(float) * nq) +
                   al(sizeof(int32_t) * std::max<int64_t>(nv, 1)) + al(sizeof(WorkItem) * ni1) +
                   al(sizeof(int32_t) * std::max<int64_t>(total_tiles, 1)) + al(sizeof(int32_t) * (nqt + 1)) +
                   al(sizeof(int32_t) * (G + 1)) + 2 * al((size_t)4 * ni1 * K1 * TM) + al(sizeof(int32_t) * ni1 * TM) +
                   al((sizeof(float) + sizeof(int32_t)) * (size_t)nq * K1) + 3 * al(sizeof(int32_t) * nq) +
                   al(sizeof(int32_t) * 4);
    unsigned char *scratch = nullptr;
    ESG_CUDA_TRY(esg_malloc_async((void **)&scratch, bytes, stream));
    unsigned char *p = scratch;
    auto take = [&](size_t b) { unsigned char *q = p; p += al(b); return q; };
    unsigned char *qs = take((size_t)std::max<int64_t>(nqt, 1) * nk * STAGE);
    float *qnorm = (float *)take(sizeof(float) * nq);
    float *qrow = (float *)take(sizeof(float) * nq);
    int32_t *d_order = (int32_t *)take(sizeof(int32_t) * std::max<int64_t>(nv, 1));
    WorkItem *d_items = (WorkItem *)take(sizeof(WorkItem) * ni1);
    int32_t *d_tiles = (int32_t *)take(sizeof(int32_t) * std::max<int64_t>(total_tiles, 1));
    int32_t *d_ib = (int32_t *)take(sizeof(int32_t) * (nqt + 1));
    int32_t *d_cta = (int32_t *)take(sizeof(int32_t) * (G + 1));
    float *part_d = (float *)take((size_t)4 * ni1 * K1 * TM);
    int32_t *part_i = (int32_t *)take((size_t)4 * ni1 * K1 * TM);
    int32_t *part_n = (int32_t *)take(sizeof(int32_t) * ni1 * TM);
    float *cand_d = (float *)take(sizeof(float) * (size_t)nq * K1);
    int32_t *cand_i = (int32_t *)take(sizeof(int32_t) * (size_t)nq * K1);
    int32_t *cand_n = (int32_t *)take(sizeof(int32_t) * nq);
    int32_t *redo = (int32_t *)take(sizeof(int32_t) * nq);
    int32_t *err = (int32_t *)take(sizeof(int32_t) * 4);

    esg_status st = ESG_OK;
    cudaError_t ce = cudaMemsetAsync(err, 0, sizeof(int32_t) * 4, stream);
    if (ce == cudaSuccess) ce = cudaMemsetAsync(cand_n, 0xFF, sizeof(int32_t) * nq, stream);   // -1: invalid
    if (ce == cudaSuccess && nv > 0)
        ce = cudaMemcpyAsync(d_order, order.data(), sizeof(int32_t) * nv, cudaMemcpyHostToDevice, stream);
    if (ce == cudaSuccess && n_items > 0)
        ce = cudaMemcpyAsync(d_items, items.data(), sizeof(WorkItem) * n_items, cudaMemcpyHostToDevice, stream);
    if (ce == cudaSuccess && total_tiles > 0)
        ce = cudaMemcpyAsync(d_tiles, tiles.data(), sizeof(int32_t) * total_tiles, cudaMemcpyHostToDevice, stream);
    if (ce == cudaSuccess)
        ce = cudaMemcpyAsync(d_ib, item_begin.data(), sizeof(int32_t) * (nqt + 1), cudaMemcpyHostToDevice, stream);
    if (ce == cudaSuccess)
        ce = cudaMemcpyAsync(d_cta, cta_first.data(), sizeof(int32_t) * (G + 1), cudaMemcpyHostToDevice, stream);
    if (ce == cudaSuccess) {
        norms_kernel<<<ceil_div_i(nq, 256), 256, 0, stream>>>(queries, nq, d, qnorm, qrow);
        if (nqt > 0)
            tile_split_kernel<<<ceil_div_i(nqt * TM * nk * 8, 256), 256, 0, stream>>>(queries, nv, d, nk, d_order,
                                                                                     nqt * TM, qs);
        ce = cudaGetLastError();
    }
    if (ce == cudaSuccess) ce = cudaFuncSetAttribute(tc_knn2_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (ce == cudaSuccess && n_items > 0) {
        // MMA work issued: three 128 x 128 x 64 BF16 products per point tile and K chunk
        esg_prof_tensor_flops((double)total_tiles * nk * 3.0 * 2.0 * TM * TN * TK);
        // failure-detection hooks (host side): ESG_BF_WAIT_NS bounds each
        // pipeline wait, ESG_TEST_BF_STALL=1 makes every CTA's first wait one
        // that nothing completes
        const char *wn = getenv("ESG_BF_WAIT_NS");
        const char *stl = getenv("ESG_TEST_BF_STALL");
        const unsigned long long wait_ns = wn && *wn ? std::max(1ull, strtoull(wn, nullptr, 10)) : kWaitNs;
        Tc2Args a{X.xs, qs, X.xnorm, qnorm, l, r, d_order, d_items, d_tiles, d_cta, (int)n_items, nv, nk, metric, K1, S,
                  stream_a, n, part_d, part_i, part_n, err, wait_ns, (stl && atoi(stl) == 1) ? 1 : 0};
        const int pidx = esg_prof_begin(stream);
        tc_knn2_kernel<<<(unsigned)G, kThreads2, smem, stream>>>(a);
        ce = cudaGetLastError();
        esg_prof_end(pidx, stream);
        if (ce == cudaSuccess) {
            merge_parts_kernel<<<ceil_div_i(nv, 4), 128, 0, stream>>>(part_d, part_i, part_n, d_ib, d_order, nv, K1,
                                                                      cand_d, cand_i, cand_n);
            ce = cudaGetLastError();
        }
    }
    if (ce != cudaSuccess) { esg_set_error(cudaGetErrorString(ce)); st = ESG_ERR_CUDA; }
    const char *dbg = getenv("ESG_BF_STATS");
    if (dbg && *dbg == '1')
        fprintf(stderr, "tensor-core brute force (pipelined): %lld query tiles, %lld point tiles, %lld items, largest share %lld tiles, %d stages%s\n",
                (long long)nqt, (long long)total_tiles, (long long)n_items, (long long)CH, S,
                stream_a ? " (query tile streamed)" : "");
    std::vector<int64_t> left;
    const double h1 = bf_stats() ? bf_host_ms() : 0.0;
    if (st == ESG_OK)
        st = certify_and_redo(base, n, d, metric, queries, nq, l, r, k, K1, cand_d, cand_i, cand_n, qrow, X.xmax,
                              redo, err, out_ids, out_dist, out_count, stream, &left);
    cudaFreeAsync(scratch, stream);
    const double h2 = bf_stats() ? bf_host_ms() : 0.0;
    if (st == ESG_OK && !left.empty())
        st = bf2_escalate(X, base, n, d, metric, queries, nq, l, r, k, K1, left, out_ids, out_dist, out_count, stream);
    if (bf_stats())
        fprintf(stderr, "tensor-core brute force, host ms: plan + uploads + launches %.3f, until certified %.3f, "
                        "escalation %.3f\n", h1 - h0, h2 - h1, bf_host_ms() - h2);
    return st;
}

// Pipelined tensor-core path; ESG_ERR_UNSUPPORTED when the shape does not fit
// (k > 56, or shared memory for fewer than two stages). Each list keeps
// K1 = k + 12 approximate candidates (k + 8 where the longer list does not
// fit in shared memory): the certificate needs the exact k-th
// distance below the approximate K1-th minus the error bound, which holds for
// nearly every query, and a short list makes the epilogue's filter sharp; the
// few queries left uncertified run again with 64 candidates.
static esg_status bruteforce_tc_v2(const float *base, int64_t n, int32_t d, int metric, const float *queries,
                                   int64_t nq, const int64_t *l, const int64_t *r, int32_t k, int64_t *out_ids,
                                   float *out_dist, int32_t *out_count, cudaStream_t stream) {
    // k + 12 candidates, at least k + 8 (the longest list the kernel holds
    // caps it): at 1M x 128, 10k queries, k = 10, lists of k + 8 left 2 queries
    // uncertified and their second pass cost 0.75 ms of a 5.90 ms call; k + 12
    // certified all (5.52 ms), k + 16 and k + 24 made the epilogue slower
    // (5.83, 6.56 ms)
    if (k < 1 || k + 8 > kMaxK1v2 || n >= ((int64_t)1 << 31) || d < 1) return ESG_ERR_UNSUPPORTED;
    int K1 = std::min(k + 12, kMaxK1v2);
    int dev = 0, max_smem = 0, S = 0, stream_a = 0;
    size_t smem = 0;
    ESG_CUDA_TRY(cudaGetDevice(&dev));
    ESG_CUDA_TRY(cudaDeviceGetAttribute(&max_smem, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
    if (bf2_smem(d, K1, max_smem, &S, &smem, &stream_a) != ESG_OK) {
        K1 = k + 8;
        if (bf2_smem(d, K1, max_smem, &S, &smem, &stream_a) != ESG_OK) return ESG_ERR_UNSUPPORTED;
    }
    if (nq == 0) return ESG_OK;
    const double t0 = bf_stats() ? bf_host_ms() : 0.0;
    const int nk = (d + TK - 1) / TK;
    const int64_t xt = (n + TN - 1) / TN;
    // the ranges come to the host first, so that the host plan is made while
    // the GPU splits and swizzles the point matrix
    int sms = 0;
    ESG_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    std::vector<int64_t> hl(nq), hr(nq);
    ESG_CUDA_TRY(cudaMemcpyAsync(hl.data(), l, sizeof(int64_t) * nq, cudaMemcpyDeviceToHost, stream));
    ESG_CUDA_TRY(cudaMemcpyAsync(hr.data(), r, sizeof(int64_t) * nq, cudaMemcpyDeviceToHost, stream));
    ESG_CUDA_TRY(cudaStreamSynchronize(stream));
    auto al = [](size_t x) { return (x + 255) & ~(size_t)255; };
    const size_t bytes = al((size_t)xt * nk * STAGE) + 2 * al(sizeof(float) * n) + al(sizeof(float) * 4);
    unsigned char *scratch = nullptr;
    ESG_CUDA_TRY(esg_malloc_async((void **)&scratch, bytes, stream));
    unsigned char *p = scratch;
    unsigned char *xs = p; p += al((size_t)xt * nk * STAGE);
    float *xnorm = (float *)p; p += al(sizeof(float) * n);
    float *xrow = (float *)p; p += al(sizeof(float) * n);
    float *xmax = (float *)p;
    esg_status st = ESG_OK;
    cudaError_t ce = cudaMemsetAsync(xmax, 0, sizeof(float) * 4, stream);
    if (ce == cudaSuccess) {
        norms_kernel<<<ceil_div_i(n, 256), 256, 0, stream>>>(base, n, d, xnorm, xrow);
        max_kernel<<<152, 256, 0, stream>>>(xrow, n, xmax);
        tile_split_kernel<<<ceil_div_i(xt * TN * nk * 8, 256), 256, 0, stream>>>(base, n, d, nk, nullptr, xt * TN, xs);
        ce = cudaGetLastError();
    }
    if (ce != cudaSuccess) { esg_set_error(cudaGetErrorString(ce)); st = ESG_ERR_CUDA; }
    const double t1 = bf_stats() ? bf_host_ms() : 0.0;
    Bf2Plan P;
    if (st == ESG_OK) st = bf2_plan(hl.data(), hr.data(), nq, n, d, sms, P);
    if (bf_stats()) fprintf(stderr, "tensor-core brute force, host ms: ranges + point prep queued %.3f, plan %.3f\n",
                            t1 - t0, bf_host_ms() - t1);
    if (st == ESG_OK) {
        const PreparedX X{xs, xnorm, xrow, xmax};
        st = bf2_queries(X, base, n, d, metric, queries, nq, l, r, k, K1, out_ids, out_dist, out_count, stream, &P);
    }
    cudaFreeAsync(scratch, stream);
    return st;
}

// Tensor-core path of esg_bruteforce_filtered_knn; returns ESG_ERR_UNSUPPORTED
// when the shape is outside both versions (the caller then uses the SIMT kernel).
esg_status esg_bruteforce_tc(const float *base, int64_t n, int32_t d, int metric, const float *queries,
                             int64_t nq, const int64_t *l, const int64_t *r, int32_t k, int64_t *out_ids,
                             float *out_dist, int32_t *out_count, cudaStream_t stream) {
    return bruteforce_tc_v2(base, n, d, metric, queries, nq, l, r, k, out_ids, out_dist, out_count, stream);
}

esg_status esg_bruteforce_plan(int64_t n, int32_t d, const int64_t *l, const int64_t *r, int64_t nq,
                               int32_t ctas, int64_t *sizes, int32_t *order, int32_t *tiles, int32_t *items,
                               int32_t *cta_first) {
    if (n < 1 || n >= ((int64_t)1 << 31) - 1 || d < 1 || nq < 0 || nq >= ((int64_t)1 << 31) || ctas < 1 ||
        !sizes || (nq > 0 && (!l || !r))) {
        esg_set_error("esg_bruteforce_plan: bad argument");
        return ESG_ERR_INVALID_ARG;
    }
    Bf2Plan P;
    esg_status st = ESG_OK;
    try {
        st = bf2_plan(l, r, nq, n, d, ctas, P);
    } catch (...) { st = ESG_ERR_OOM; }
    if (st != ESG_OK) {
        if (st == ESG_ERR_UNSUPPORTED) esg_set_error("esg_bruteforce_plan: more than 2^31 covered point tiles");
        return st;
    }
    sizes[0] = P.nv;
    sizes[1] = P.total_tiles;
    sizes[2] = (int64_t)P.items.size();
    sizes[3] = P.G;
    if (order) std::copy(P.order.begin(), P.order.end(), order);
    if (tiles) std::copy(P.tiles.begin(), P.tiles.end(), tiles);
    if (items)
        for (size_t i = 0; i < P.items.size(); ++i) {
            items[4 * i] = P.items[i].qtile;
            items[4 * i + 1] = P.items[i].off;
            items[4 * i + 2] = P.items[i].cnt;
            items[4 * i + 3] = 0;
        }
    if (cta_first) std::copy(P.cta_first.begin(), P.cta_first.end(), cta_first);
    return ESG_OK;
}

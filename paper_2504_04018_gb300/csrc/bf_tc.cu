// Exact range-filtered k-NN on the 5th-generation tensor cores (tcgen05).
//
// Dot products q.x come from three BF16 MMAs per K step accumulated in FP32
// in tensor memory (split precision: q = q_hi + q_lo, x = x_hi + x_lo with
// BF16 parts, q.x ~ q_hi.x_hi + q_hi.x_lo + q_lo.x_hi; the dropped q_lo.x_lo
// and the split residuals are below 2^-17 relative). A CTA owns 128 queries
// (one TMEM lane each) and walks the union of their rank ranges in tiles of
// 128 points (128 TMEM columns). Operands are staged with cp.async into
// shared memory in the 128-byte-swizzled K-major layout the MMA descriptors
// name; one thread issues the MMAs and commits them to an mbarrier; all 128
// threads then read their row from TMEM, mask it by the query's range and
// keep the K1 = k' + 1 best approximate distances per query.
//
// A second kernel recomputes exact FP32 distances (direct form) of those
// candidates, sorts them, and certifies the result: with delta_q a bound on
// |approximate - exact| for every point of the range, the top k is proven
// when the exact k-th distance is below (K1-th approximate distance -
// delta_q). Queries without a certificate are recomputed by the exact SIMT
// brute force.
#include "esg_internal.cuh"

#include <algorithm>
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
constexpr int kMaxK1 = 72;
constexpr long kSpinLimit = 1L << 26;

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

// Bounded wait on an mbarrier phase; false when the limit ran out.
__device__ __forceinline__ bool mbar_wait(uint32_t mbar, uint32_t phase) {
    for (long it = 0; it < kSpinLimit; ++it) {
        uint32_t done = 0;
        asm volatile(
            "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}\n"
            : "=r"(done) : "r"(mbar), "r"(phase) : "memory");
        if (done) return true;
    }
    return false;
}

__device__ __forceinline__ void cp_async16(uint32_t dst, const void *src, bool valid) {
    const int sz = valid ? 16 : 0;   // zero-fill rows past the end
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" :: "r"(dst), "l"(src), "r"(sz) : "memory");
}

// 32 consecutive FP32 columns of this thread's TMEM lane.
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float *v) {
    uint32_t r[32];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
        "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
        "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
          "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
          "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]),
          "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]),
          "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

// Copy a 128-row x 64-element BF16 chunk (rows row0.., elements k0..k0+63 of
// a row-major [rows, d] matrix) into 128-byte-swizzled shared memory:
// 16-byte piece c of row t lands at t * 128 + ((c ^ (t & 7)) * 16).
__device__ __forceinline__ void load_chunk(uint32_t sdst, const __nv_bfloat16 *src, int64_t rows,
                                           int64_t row0, int d, int k0) {
    for (int idx = threadIdx.x; idx < TM * 8; idx += blockDim.x) {
        const int t = idx >> 3, c = idx & 7;
        const int64_t row = row0 + t;
        const bool ok = row >= 0 && row < rows;
        const __nv_bfloat16 *g = src + (ok ? row : 0) * (int64_t)d + k0 + c * 8;
        cp_async16(sdst + t * 128 + ((c ^ (t & 7)) << 4), g, ok);
    }
}

struct TcArgs {
    const __nv_bfloat16 *qhi, *qlo, *xhi, *xlo;   // [nq, d], [n, d]
    const float *qnorm, *xnorm;                    // squared norms (L2)
    const int64_t *l, *r;
    int64_t n, nq;
    int d, metric, K1;
    float *cand_d;      // [nq, K1] approximate distances (ascending)
    int32_t *cand_i;    // [nq, K1] rows
    int32_t *cand_n;    // [nq]
    int32_t *err;       // set when a bounded wait ran out
};

__global__ void __launch_bounds__(128, 1) tc_knn_kernel(TcArgs a) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    // 1024-byte aligned operand area: A hi/lo chunk, B hi/lo chunk
    unsigned char *base = (unsigned char *)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    unsigned char *sA_hi = base, *sA_lo = base + CHUNK, *sB_hi = base + 2 * CHUNK, *sB_lo = base + 3 * CHUNK;
    float *ld = (float *)(base + 4 * CHUNK);                       // [TM][K1 + 1] distances
    int32_t *li = (int32_t *)(ld + TM * (a.K1 + 1));               // [TM][K1 + 1] rows
    uint64_t *mbar = (uint64_t *)(li + TM * (a.K1 + 1) + 1);       // 8-byte aligned below
    mbar = (uint64_t *)(((uintptr_t)mbar + 7) & ~(uintptr_t)7);
    uint32_t *tmem_slot = (uint32_t *)(mbar + 1);
    __shared__ long long s_lo, s_hi;
    __shared__ int s_abort;

    const int tid = threadIdx.x, warp = tid >> 5;
    const int64_t q0 = (int64_t)blockIdx.x * TM;
    const int64_t qi = q0 + tid;
    int64_t my_lo = 1, my_hi = 0;
    if (qi < a.nq) {
        const int64_t l = a.l[qi], r = a.r[qi];
        if (l >= 0 && l <= r && r < a.n) { my_lo = l; my_hi = r; }
    }
    const float qn = (qi < a.nq && a.metric == ESG_L2SQ) ? a.qnorm[qi] : 0.f;
    const int K1 = a.K1;
    float *myd = ld + tid;        // column-interleaved: entry e at myd[e * TM]
    int32_t *myi = li + tid;
    int cnt = 0;
    float thr = INFINITY;
    int32_t thr_id = 0x7FFFFFFF;

    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" :: "r"(smem_u32(mbar)) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        s_lo = 0x7FFFFFFFFFFFFFFFLL; s_hi = -1; s_abort = 0;
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                     :: "r"(smem_u32(tmem_slot)), "r"(TN) : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = *tmem_slot;
    if (my_lo <= my_hi) {
        atomicMin(&s_lo, (long long)my_lo);
        atomicMax(&s_hi, (long long)my_hi);
    }
    __syncthreads();
    const int64_t ulo = s_lo, uhi = s_hi;
    uint32_t phase = 0;
    const int nk = a.d / TK;

    for (int64_t t0 = (uhi >= 0 ? ulo : 1); t0 <= uhi; t0 += TN) {
        // skip tiles no query of this CTA overlaps (uniform: barrier + OR)
        const bool overlaps = my_lo <= my_hi && my_lo <= t0 + TN - 1 && my_hi >= t0;
        if (!__syncthreads_or(overlaps)) continue;
        for (int kc = 0; kc < nk; ++kc) {
            load_chunk(smem_u32(sA_hi), a.qhi, a.nq, q0, a.d, kc * TK);
            load_chunk(smem_u32(sA_lo), a.qlo, a.nq, q0, a.d, kc * TK);
            load_chunk(smem_u32(sB_hi), a.xhi, a.n, t0, a.d, kc * TK);
            load_chunk(smem_u32(sB_lo), a.xlo, a.n, t0, a.d, kc * TK);
            asm volatile("cp.async.wait_all;" ::: "memory");
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
            __syncthreads();
            if (tid == 0) {
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                const uint32_t ah = smem_u32(sA_hi), al = smem_u32(sA_lo);
                const uint32_t bh = smem_u32(sB_hi), bl = smem_u32(sB_lo);
#pragma unroll
                for (int s = 0; s < TK / 16; ++s) {
                    const uint32_t off = s * 32;   // 16 BF16 along K inside the swizzled row
                    const uint32_t first = (kc == 0 && s == 0) ? 0u : 1u;
                    mma_bf16(tmem, sdesc(ah + off), sdesc(bh + off), first);
                    mma_bf16(tmem, sdesc(ah + off), sdesc(bl + off), 1u);
                    mma_bf16(tmem, sdesc(al + off), sdesc(bh + off), 1u);
                }
                mma_commit(smem_u32(mbar));
            }
            // the MMAs read the operand chunk: wait before overwriting it
            if (!mbar_wait(smem_u32(mbar), phase)) {
                if (tid == 0) { s_abort = 1; atomicExch(a.err, 1); }
            }
            phase ^= 1u;
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            __syncthreads();
            if (s_abort) break;
        }
        if (s_abort) break;
        // epilogue: this thread's row of the 128 x 128 tile (every lane of a
        // warp executes the tcgen05.ld; rows outside the tile ignore theirs)
        const bool active = my_lo <= my_hi && my_lo <= t0 + TN - 1 && my_hi >= t0;
        for (int c0 = 0; c0 < TN; c0 += 32) {
            float v[32];
            tmem_ld32(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0, v);
            if (!active) continue;
#pragma unroll 4
            for (int j = 0; j < 32; ++j) {
                const int64_t p = t0 + c0 + j;
                if (p < my_lo || p > my_hi) continue;
                const float dist = a.metric == ESG_L2SQ ? qn + __ldg(a.xnorm + p) - 2.f * v[j] : -v[j];
                const int32_t pid = (int32_t)p;
                if (cnt == K1 && !(dist < thr || (dist == thr && pid < thr_id))) continue;
                // insertion into the row's ascending list
                int e = cnt < K1 ? cnt : K1 - 1;
                while (e > 0) {
                    const float pd = myd[(e - 1) * TM];
                    const int32_t pi = myi[(e - 1) * TM];
                    if (pd < dist || (pd == dist && pi < pid)) break;
                    myd[e * TM] = pd;
                    myi[e * TM] = pi;
                    --e;
                }
                myd[e * TM] = dist;
                myi[e * TM] = pid;
                if (cnt < K1) ++cnt;
                if (cnt == K1) { thr = myd[(K1 - 1) * TM]; thr_id = myi[(K1 - 1) * TM]; }
            }
        }
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        __syncthreads();
    }
    if (qi < a.nq) {
        for (int e = 0; e < cnt; ++e) {
            a.cand_d[qi * K1 + e] = myd[e * TM];
            a.cand_i[qi * K1 + e] = myi[e * TM];
        }
        a.cand_n[qi] = (my_lo <= my_hi) ? cnt : -1;
    }
    __syncthreads();
    if (warp == 0) {
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" :: "r"(tmem), "r"(TN) : "memory");
    }
}

// FP32 -> (hi, lo) BF16 split and squared norms, one thread per row.
__global__ void split_rows_kernel(const float *X, int64_t rows, int d, __nv_bfloat16 *hi,
                                  __nv_bfloat16 *lo, float *norm, float *rownorm) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= rows) return;
    const float *x = X + i * d;
    float s = 0.f;
    for (int j = 0; j < d; ++j) {
        const float v = x[j];
        const __nv_bfloat16 h = __float2bfloat16_rn(v);
        hi[i * d + j] = h;
        lo[i * d + j] = __float2bfloat16_rn(v - __bfloat162float(h));
        s = fmaf(v, v, s);
    }
    if (norm) norm[i] = s;
    if (rownorm) rownorm[i] = sqrtf(s);
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

}  // namespace

// Tensor-core path of esg_bruteforce_filtered_knn; returns ESG_ERR_UNSUPPORTED
// when the shape is outside it (the caller then uses the SIMT kernel).
esg_status esg_bruteforce_tc(const float *base, int64_t n, int32_t d, int metric, const float *queries,
                             int64_t nq, const int64_t *l, const int64_t *r, int32_t k, int64_t *out_ids,
                             float *out_dist, int32_t *out_count, cudaStream_t stream) {
    if (d % TK != 0 || k < 1 || 2 * k + 8 > kMaxK1 || n >= ((int64_t)1 << 31)) return ESG_ERR_UNSUPPORTED;
    if (nq == 0) return ESG_OK;
    const int K1 = 2 * k + 8;
    // device scratch: BF16 splits, norms, candidates, flags
    const size_t nb = sizeof(__nv_bfloat16);
    size_t bytes = nb * (size_t)d * (2 * n + 2 * nq) + sizeof(float) * (2 * n + 2 * nq + 4) +
                   (sizeof(float) + sizeof(int32_t)) * (size_t)nq * K1 + sizeof(int32_t) * (2 * nq + 4);
    bytes += 8 * 256;
    unsigned char *scratch = nullptr;
    ESG_CUDA_TRY(cudaMallocAsync((void **)&scratch, bytes, stream));
    auto al = [](size_t x) { return (x + 255) & ~(size_t)255; };
    unsigned char *p = scratch;
    __nv_bfloat16 *xhi = (__nv_bfloat16 *)p; p += al(nb * n * d);
    __nv_bfloat16 *xlo = (__nv_bfloat16 *)p; p += al(nb * n * d);
    __nv_bfloat16 *qhi = (__nv_bfloat16 *)p; p += al(nb * nq * d);
    __nv_bfloat16 *qlo = (__nv_bfloat16 *)p; p += al(nb * nq * d);
    float *xnorm = (float *)p; p += al(sizeof(float) * n);
    float *xrow = (float *)p; p += al(sizeof(float) * n);
    float *qnorm = (float *)p; p += al(sizeof(float) * nq);
    float *qrow = (float *)p; p += al(sizeof(float) * nq);
    float *xmax = (float *)p; p += al(sizeof(float) * 4);
    float *cand_d = (float *)p; p += al(sizeof(float) * nq * K1);
    int32_t *cand_i = (int32_t *)p; p += al(sizeof(int32_t) * nq * K1);
    int32_t *cand_n = (int32_t *)p; p += al(sizeof(int32_t) * nq);
    int32_t *redo = (int32_t *)p; p += al(sizeof(int32_t) * nq);
    int32_t *err = (int32_t *)p;
    esg_status st = ESG_OK;
    cudaError_t ce = cudaMemsetAsync(xmax, 0, sizeof(float) * 4, stream);
    if (ce == cudaSuccess) ce = cudaMemsetAsync(err, 0, sizeof(int32_t), stream);
    if (ce == cudaSuccess) {
        split_rows_kernel<<<ceil_div_i(n, 256), 256, 0, stream>>>(base, n, d, xhi, xlo, xnorm, xrow);
        split_rows_kernel<<<ceil_div_i(nq, 256), 256, 0, stream>>>(queries, nq, d, qhi, qlo, qnorm, qrow);
        max_kernel<<<152, 256, 0, stream>>>(xrow, n, xmax);
        ce = cudaGetLastError();
    }
    const size_t smem = 1024 + 4 * CHUNK + (size_t)TM * (K1 + 1) * 8 + 64;
    if (ce == cudaSuccess) ce = cudaFuncSetAttribute(tc_knn_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (ce == cudaSuccess) {
        TcArgs a{qhi, qlo, xhi, xlo, qnorm, xnorm, l, r, n, nq, d, metric, K1, cand_d, cand_i, cand_n, err};
        const int pidx = esg_prof_begin(stream);
        tc_knn_kernel<<<(unsigned)((nq + TM - 1) / TM), 128, smem, stream>>>(a);
        ce = cudaGetLastError();
        esg_prof_end(pidx, stream);
    }
    if (ce == cudaSuccess) {
        rerank_certify_kernel<<<ceil_div_i(nq, 4), 128, 0, stream>>>(
            base, queries, d, metric, nq, k, K1, cand_d, cand_i, cand_n, qrow, xmax,
            out_ids, out_dist, out_count, redo);
        ce = cudaGetLastError();
    }
    if (ce != cudaSuccess) { esg_set_error(cudaGetErrorString(ce)); st = ESG_ERR_CUDA; }
    // queries without a certificate (or any aborted wait): exact SIMT pass
    if (st == ESG_OK) {
        std::vector<int32_t> h_redo(nq);
        int32_t h_err = 0;
        ce = cudaMemcpyAsync(h_redo.data(), redo, sizeof(int32_t) * nq, cudaMemcpyDeviceToHost, stream);
        if (ce == cudaSuccess) ce = cudaMemcpyAsync(&h_err, err, sizeof(int32_t), cudaMemcpyDeviceToHost, stream);
        if (ce == cudaSuccess) ce = cudaStreamSynchronize(stream);
        if (ce != cudaSuccess) { esg_set_error(cudaGetErrorString(ce)); st = ESG_ERR_CUDA; }
        if (st == ESG_OK && h_err) { esg_set_error("tensor-core brute force: an mbarrier wait timed out"); st = ESG_ERR_TIMEOUT; }
        if (st == ESG_OK) {
            std::vector<int64_t> idx;
            for (int64_t i = 0; i < nq; ++i) if (h_redo[i]) idx.push_back(i);
            const char *dbg = getenv("ESG_BF_STATS");
            if (dbg && *dbg == '1')
                fprintf(stderr, "tensor-core brute force: %lld of %lld queries recomputed\n",
                        (long long)idx.size(), (long long)nq);
            if (!idx.empty())
                st = esg_bruteforce_redo(base, n, d, metric, queries, nq, l, r, k, idx, out_ids, out_dist,
                                         out_count, stream);
        }
    }
    cudaFreeAsync(scratch, stream);
    return st;
}

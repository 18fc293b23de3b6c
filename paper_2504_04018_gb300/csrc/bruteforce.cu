// Exact range-filtered k-NN by brute force (Definitions 1 and 2).
//
// Tiled like a GEMM: a CTA owns 64 queries and walks the union of their rank
// ranges in tiles of 64 points, skipping tiles that no query of the CTA
// overlaps. Each 64 x 64 distance tile is computed from 32-dimension slices
// staged in shared memory (every thread a 4 x 4 block), masked by each
// query's range, and folded into a per-query sorted top-k list (candidates
// closer than the current k-th are sorted and merged by one warp).
// Distances: mode 0 = sum (q - x)^2 in the direct form, mode 1 = -<q, x>,
// mode 2 = |q|^2 + |x|^2 - 2 <q, x> from precomputed norms (graph build).
#include "esg_internal.cuh"

#include <algorithm>
#include <cstdlib>
#include <vector>

namespace {

constexpr int BQ = 64, BP = 64, BK = 32, PAD = 4;
constexpr int kSmemListMax = 128;

struct BfArgs {
    const float *base;
    int64_t n;
    int d;
    const float *queries;
    int64_t nq;
    const int64_t *l, *r;
    int k;
    int64_t *out_ids;
    float *out_dist;
    int32_t *out_count;
    const int64_t *id_map;   // optional: output id = id_map[row]
    int exclude_self;        // skip row == query index (graph build)
    const float *xnorm, *qnorm;  // mode 2
    Cand *glists;            // lists in global memory when k > kSmemListMax
};

__device__ __forceinline__ int merge_into(const Cand *A, int a, const Cand *B, int b, Cand *O, int C) {
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

template <int MODE>
__global__ void __launch_bounds__(256) bf_kernel(BfArgs a) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    float (*As)[BQ + PAD] = reinterpret_cast<float (*)[BQ + PAD]>(smem_raw);
    float (*Bs)[BP + PAD] = reinterpret_cast<float (*)[BP + PAD]>(smem_raw + sizeof(float) * BK * (BQ + PAD));
    float (*Ds)[BP + 1] = reinterpret_cast<float (*)[BP + 1]>(smem_raw + sizeof(float) * BK * (BQ + PAD) * 2);
    unsigned char *p = smem_raw + sizeof(float) * BK * (BQ + PAD) * 2 + sizeof(float) * BQ * (BP + 1);
    int64_t *qlo = reinterpret_cast<int64_t *>(p); p += sizeof(int64_t) * BQ;
    int64_t *qhi = reinterpret_cast<int64_t *>(p); p += sizeof(int64_t) * BQ;
    int *lens = reinterpret_cast<int *>(p); p += sizeof(int) * BQ;
    int *flag = reinterpret_cast<int *>(p); p += 16;
    Cand *batch = reinterpret_cast<Cand *>(p); p += sizeof(Cand) * 8 * 64;
    Cand *lists, *tmp;
    const int k = a.k;
    if (a.glists) {
        lists = a.glists + (size_t)blockIdx.x * (BQ + 8) * k;
        tmp = lists + (size_t)BQ * k;
    } else {
        lists = reinterpret_cast<Cand *>(p); p += sizeof(Cand) * BQ * k;
        tmp = reinterpret_cast<Cand *>(p);
    }
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int ty = tid >> 4, tx = tid & 15;
    const int64_t q0 = (int64_t)blockIdx.x * BQ;

    if (tid < BQ) {
        int64_t qi = q0 + tid;
        int64_t lo = 1, hi = 0;
        if (qi < a.nq) {
            int64_t l = a.l[qi], r = a.r[qi];
            if (l >= 0 && l <= r && r < a.n) { lo = l; hi = r; }
        }
        qlo[tid] = lo; qhi[tid] = hi; lens[tid] = 0;
    }
    __syncthreads();
    // union of the CTA's ranges
    int64_t ulo = INT64_MAX, uhi = -1;
    for (int i = 0; i < BQ; ++i) {
        if (qlo[i] <= qhi[i]) { ulo = min(ulo, qlo[i]); uhi = max(uhi, qhi[i]); }
    }
    const float4 *Q4 = reinterpret_cast<const float4 *>(a.queries);
    const float4 *X4 = reinterpret_cast<const float4 *>(a.base);
    const int nvec = a.d / 4;

    for (int64_t t0 = (uhi >= 0 ? ulo : 1); t0 <= uhi; t0 += BP) {
        const int64_t t1 = t0 + BP - 1;
        if (warp == 0) {
            bool ov = false;
            for (int i = lane; i < BQ; i += 32) ov |= (qlo[i] <= t1 && qhi[i] >= t0 && qlo[i] <= qhi[i]);
            unsigned b = __ballot_sync(0xffffffffu, ov);
            if (lane == 0) *flag = b != 0;
        }
        __syncthreads();
        if (!*flag) { __syncthreads(); continue; }

        float acc[4][4];
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
            for (int j = 0; j < 4; ++j) acc[i][j] = 0.f;

        for (int k0 = 0; k0 < a.d; k0 += BK) {
            // stage 64 x 32 query and point slices, transposed to [dim][row]
            for (int idx = tid; idx < BQ * (BK / 4); idx += 256) {
                int row = idx / (BK / 4), c4 = idx % (BK / 4);
                int v = k0 / 4 + c4;
                float4 x = make_float4(0.f, 0.f, 0.f, 0.f);
                if (q0 + row < a.nq && v < nvec) x = __ldg(Q4 + (q0 + row) * nvec + v);
                As[c4 * 4 + 0][row] = x.x; As[c4 * 4 + 1][row] = x.y;
                As[c4 * 4 + 2][row] = x.z; As[c4 * 4 + 3][row] = x.w;
                float4 y = make_float4(0.f, 0.f, 0.f, 0.f);
                if (t0 + row < a.n && v < nvec) y = __ldg(X4 + (t0 + row) * nvec + v);
                Bs[c4 * 4 + 0][row] = y.x; Bs[c4 * 4 + 1][row] = y.y;
                Bs[c4 * 4 + 2][row] = y.z; Bs[c4 * 4 + 3][row] = y.w;
            }
            __syncthreads();
#pragma unroll 8
            for (int kk = 0; kk < BK; ++kk) {
                float4 av = *reinterpret_cast<const float4 *>(&As[kk][ty * 4]);
                float4 bv = *reinterpret_cast<const float4 *>(&Bs[kk][tx * 4]);
                float aa[4] = {av.x, av.y, av.z, av.w};
                float bb[4] = {bv.x, bv.y, bv.z, bv.w};
#pragma unroll
                for (int i = 0; i < 4; ++i)
#pragma unroll
                    for (int j = 0; j < 4; ++j) {
                        if (MODE == 0) {
                            float df = aa[i] - bb[j];
                            acc[i][j] = fmaf(df, df, acc[i][j]);
                        } else {
                            acc[i][j] = fmaf(aa[i], bb[j], acc[i][j]);
                        }
                    }
            }
            __syncthreads();
        }
        // masked distances of the tile
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            int qr = ty * 4 + i;
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                int64_t pt = t0 + tx * 4 + j;
                bool ok = pt <= qhi[qr] && pt >= qlo[qr] && !(a.exclude_self && pt == q0 + qr);
                float v;
                if (MODE == 0) v = acc[i][j];
                else if (MODE == 1) v = -acc[i][j];
                else v = a.qnorm[min(q0 + qr, a.nq - 1)] + a.xnorm[min(pt, a.n - 1)] - 2.f * acc[i][j];
                Ds[qr][tx * 4 + j] = ok ? v : INFINITY;
            }
        }
        __syncthreads();
        // fold the tile into the per-query lists (warp w owns rows 8w..8w+7)
        Cand *wb = batch + warp * 64;
        for (int rr = 0; rr < BQ / 8; ++rr) {
            const int row = warp * (BQ / 8) + rr;
            Cand *L = lists + (size_t)row * k;
            const int len = lens[row];
            Cand thr = len < k ? Cand{INFINITY, ESG_NONE} : L[k - 1];
            Cand x0{Ds[row][lane], (uint32_t)(t0 + lane)};
            Cand x1{Ds[row][lane + 32], (uint32_t)(t0 + lane + 32)};
            bool p0 = x0.d < INFINITY && (len < k || cand_less(x0, thr));
            bool p1 = x1.d < INFINITY && (len < k || cand_less(x1, thr));
            unsigned b0 = __ballot_sync(0xffffffffu, p0), b1 = __ballot_sync(0xffffffffu, p1);
            if ((b0 | b1) == 0) continue;
            int c0 = __popc(b0), nb = c0 + __popc(b1);
            const unsigned below = (1u << lane) - 1;
            wb[lane] = Cand{INFINITY, ESG_NONE};
            wb[lane + 32] = Cand{INFINITY, ESG_NONE};
            __syncwarp();
            if (p0) wb[__popc(b0 & below)] = x0;
            if (p1) wb[c0 + __popc(b1 & below)] = x1;
            __syncwarp();
            warp_sort64(wb);
            Cand *T = tmp + (size_t)warp * k;
            int nl = merge_into(L, len, wb, nb, T, k);
            for (int i = lane; i < nl; i += 32) L[i] = T[i];
            if (lane == 0) lens[row] = nl;
            __syncwarp();
        }
        __syncthreads();
    }
    // write results
    for (int rr = 0; rr < BQ / 8; ++rr) {
        const int row = warp * (BQ / 8) + rr;
        const int64_t qi = q0 + row;
        if (qi >= a.nq) continue;
        const Cand *L = lists + (size_t)row * k;
        const int len = lens[row];
        for (int j = lane; j < k; j += 32) {
            int64_t id = -1;
            float dv = INFINITY;
            if (j < len) {
                id = (int64_t)L[j].id;
                if (a.id_map) id = a.id_map[id];
                dv = L[j].d;
            }
            a.out_ids[qi * k + j] = id;
            a.out_dist[qi * k + j] = dv;
        }
        if (lane == 0) a.out_count[qi] = len;
    }
}

}  // namespace

__global__ void row_norms_kernel(const float *X, int64_t n, int d, float *out) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float *x = X + i * d;
    float s = 0.f;
    for (int j = 0; j < d; ++j) s = fmaf(x[j], x[j], s);
    out[i] = s;
}

// mode: 0 = L2 direct, 1 = IP, 2 = L2 from norms (xnorm/qnorm required)
esg_status esg_launch_bruteforce_mode(int mode, const float *base, int64_t n, int32_t d,
                                      const float *queries, int64_t nq, const int64_t *l,
                                      const int64_t *r, int32_t k, int64_t *out_ids,
                                      float *out_dist, int32_t *out_count, const int64_t *id_map,
                                      int32_t exclude_self, const float *xnorm,
                                      const float *qnorm, cudaStream_t stream) {
    if (nq == 0) return ESG_OK;
    if (d % 4 != 0 || k < 1 || k > 1024) { esg_set_error("bruteforce: need d % 4 == 0 and 1 <= k <= 1024"); return ESG_ERR_INVALID_ARG; }
    const bool smem_lists = k <= kSmemListMax;
    size_t smem = sizeof(float) * BK * (BQ + PAD) * 2 + sizeof(float) * BQ * (BP + 1) +
                  sizeof(int64_t) * BQ * 2 + sizeof(int) * BQ + 16 + sizeof(Cand) * 8 * 64;
    if (smem_lists) smem += sizeof(Cand) * (size_t)(BQ + 8) * k;
    int64_t grid = (nq + BQ - 1) / BQ;
    Cand *glists = nullptr;
    if (!smem_lists) ESG_CUDA_TRY(esg_malloc_async((void **)&glists, sizeof(Cand) * (size_t)grid * (BQ + 8) * k, stream));
    BfArgs a{base, n, d, queries, nq, l, r, k, out_ids, out_dist, out_count, id_map, exclude_self,
             xnorm, qnorm, glists};
    void (*fn)(BfArgs) = mode == 0 ? bf_kernel<0> : (mode == 1 ? bf_kernel<1> : bf_kernel<2>);
    ESG_CUDA_TRY(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    fn<<<(unsigned)grid, 256, smem, stream>>>(a);
    ESG_CUDA_TRY(cudaGetLastError());
    if (glists) ESG_CUDA_TRY(cudaFreeAsync(glists, stream));
    return ESG_OK;
}

namespace {
__global__ void gather_queries_kernel(const float *Q, const int64_t *l, const int64_t *r, int d,
                                      const int64_t *idx, int64_t m, float *Qg, int64_t *lg, int64_t *rg) {
    const int64_t i = blockIdx.x;
    if (i >= m) return;
    const int64_t q = idx[i];
    for (int j = threadIdx.x; j < d; j += blockDim.x) Qg[i * d + j] = Q[q * d + j];
    if (threadIdx.x == 0) { lg[i] = l[q]; rg[i] = r[q]; }
}

__global__ void scatter_results_kernel(const int64_t *idx, int64_t m, int k, const int64_t *ids_g,
                                       const float *dist_g, const int32_t *cnt_g, int64_t *ids,
                                       float *dist, int32_t *cnt) {
    const int64_t i = blockIdx.x;
    if (i >= m) return;
    const int64_t q = idx[i];
    for (int j = threadIdx.x; j < k; j += blockDim.x) {
        ids[q * k + j] = ids_g[i * k + j];
        dist[q * k + j] = dist_g[i * k + j];
    }
    if (threadIdx.x == 0) cnt[q] = cnt_g[i];
}
}  // namespace

// Exact SIMT brute force for the listed queries only (results scattered into
// the full output arrays).
esg_status esg_bruteforce_redo(const float *base, int64_t n, int32_t d, int metric, const float *queries,
                               int64_t nq, const int64_t *l, const int64_t *r, int32_t k,
                               const std::vector<int64_t> &idx, int64_t *out_ids, float *out_dist,
                               int32_t *out_count, cudaStream_t stream) {
    (void)nq;
    const int64_t m = (int64_t)idx.size();
    if (m == 0) return ESG_OK;
    auto al = [](size_t x) { return (x + 255) & ~(size_t)255; };
    const size_t bytes = al(sizeof(int64_t) * m) + al(sizeof(float) * m * d) + 2 * al(sizeof(int64_t) * m) +
                         al(sizeof(int64_t) * m * k) + al(sizeof(float) * m * k) + al(sizeof(int32_t) * m);
    unsigned char *s = nullptr;
    ESG_CUDA_TRY(esg_malloc_async((void **)&s, bytes, stream));
    unsigned char *p = s;
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
        gather_queries_kernel<<<(unsigned)m, 128, 0, stream>>>(queries, l, r, d, didx, m, Qg, lg, rg);
        ce = cudaGetLastError();
    }
    if (ce != cudaSuccess) { esg_set_error(cudaGetErrorString(ce)); st = ESG_ERR_CUDA; }
    if (st == ESG_OK)
        st = esg_launch_bruteforce_mode(metric == ESG_IP ? 1 : 0, base, n, d, Qg, m, lg, rg, k, ig, dg, cg,
                                        nullptr, 0, nullptr, nullptr, stream);
    if (st == ESG_OK) {
        scatter_results_kernel<<<(unsigned)m, 128, 0, stream>>>(didx, m, k, ig, dg, cg, out_ids, out_dist, out_count);
        ce = cudaGetLastError();
        if (ce != cudaSuccess) { esg_set_error(cudaGetErrorString(ce)); st = ESG_ERR_CUDA; }
    }
    // the host vector must outlive the copy above
    cudaError_t se = cudaStreamSynchronize(stream);
    if (st == ESG_OK && se != cudaSuccess) { esg_set_error(cudaGetErrorString(se)); st = ESG_ERR_CUDA; }
    cudaFreeAsync(s, stream);
    return st;
}

esg_status esg_bruteforce_tc(const float *base, int64_t n, int32_t d, int metric, const float *queries,
                             int64_t nq, const int64_t *l, const int64_t *r, int32_t k, int64_t *out_ids,
                             float *out_dist, int32_t *out_count, cudaStream_t stream);

esg_status esg_launch_bruteforce(const float *base, int64_t n, int32_t d, int metric,
                                 const float *queries, int64_t nq, const int64_t *l,
                                 const int64_t *r, int32_t k, int64_t *out_ids, float *out_dist,
                                 int32_t *out_count, const int64_t *id_map, int32_t exclude_self,
                                 cudaStream_t stream) {
    // tensor-core path (split-precision BF16 MMAs, certified) when it applies
    const char *simt = getenv("ESG_BF_SIMT");
    if (!id_map && !exclude_self && !(simt && *simt == '1')) {
        esg_status st = esg_bruteforce_tc(base, n, d, metric, queries, nq, l, r, k, out_ids, out_dist,
                                          out_count, stream);
        if (st != ESG_ERR_UNSUPPORTED) return st;
    }
    return esg_launch_bruteforce_mode(metric == ESG_IP ? 1 : 0, base, n, d, queries, nq, l, r, k,
                                      out_ids, out_dist, out_count, id_map, exclude_self, nullptr,
                                      nullptr, stream);
}

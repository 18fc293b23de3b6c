// Learned search budget: a small MLP that predicts, per query, the beam
// width ef and an expansion budget needed to reach a recall target, trained
// on the GPU with this file's own forward, backward and Adam kernels from
// traces of the plain fixed-ef search. The paper has no learned component.
//
// Network (F = 9 features):  x_hat = (x - mu) / sigma,
//   h1 = relu(W1^T x_hat + b1) [64], h2 = relu(W2^T h1 + b2) [64],
//   y = W3^T h2 + b3 [2] = (log2 ef, log2 expansion budget).
// Loss: pinball (quantile q) averaged over rows and both outputs.
// Flat parameters: W1 [F*64] row-major, b1 [64], W2 [64*64], b2 [64],
// W3 [64*2], b3 [2].
//
// Features of a query (computed on the GPU from its range decomposition and
// the distances to its first piece's entry points):
//   0 log2 width, 1 number of pieces, 2/3 log2(node size / piece size) of
//   piece 0 / 1, 4 piece 0 is a graph piece, 5 log2 k, 6 min / mean entry
//   distance of piece 0 (1 for scans), 7 log2 node size of piece 0, 8 the
//   top-k gap of the first hop: (min(k, E)-th smallest - smallest entry
//   distance) / |mean entry distance| (0 for scans).
#include "esg_internal.cuh"
#include "decompose.cuh"

#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

constexpr int kF = ESG_MLP_FEATURES;
constexpr int kH = 64;
constexpr int kO = 2;
constexpr int kP = kF * kH + kH + kH * kH + kH + kH * kO + kO;

namespace {

struct MlpView {
    const float *W1, *b1, *W2, *b2, *W3, *b3;
};

__host__ __device__ inline MlpView view(const float *p) {
    MlpView v;
    v.W1 = p; p += kF * kH;
    v.b1 = p; p += kH;
    v.W2 = p; p += kH * kH;
    v.b2 = p; p += kH;
    v.W3 = p; p += kH * kO;
    v.b3 = p;
    return v;
}

// Forward pass of one row (params in shared memory); optionally keeps the
// pre-activations of both hidden layers.
__device__ inline void mlp_row(const float *sp, const float *xh, float *y, float *z1_out, float *z2_out) {
    const MlpView v = view(sp);
    float h1[kH];
#pragma unroll 4
    for (int j = 0; j < kH; ++j) {
        float s = v.b1[j];
#pragma unroll
        for (int i = 0; i < kF; ++i) s = fmaf(xh[i], v.W1[i * kH + j], s);
        if (z1_out) z1_out[j] = s;
        h1[j] = fmaxf(s, 0.f);
    }
    float acc0 = v.b3[0], acc1 = v.b3[1];
    for (int j = 0; j < kH; ++j) {
        float s = v.b2[j];
#pragma unroll 8
        for (int i = 0; i < kH; ++i) s = fmaf(h1[i], v.W2[i * kH + j], s);
        if (z2_out) z2_out[j] = s;
        const float h2 = fmaxf(s, 0.f);
        acc0 = fmaf(h2, v.W3[j * kO + 0], acc0);
        acc1 = fmaf(h2, v.W3[j * kO + 1], acc1);
    }
    y[0] = acc0;
    y[1] = acc1;
}

// Forward over B rows; stores y [B,2], z1 [B,64], z2 [B,64] when given.
__global__ void mlp_forward_kernel(const float *params, const float *X, const float *mu,
                                   const float *sigma, int64_t B, float *Y, float *Z1, float *Z2) {
    __shared__ float sp[kP];
    for (int i = threadIdx.x; i < kP; i += blockDim.x) sp[i] = params[i];
    __syncthreads();
    const int64_t b = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (b >= B) return;
    float xh[kF];
#pragma unroll
    for (int i = 0; i < kF; ++i) xh[i] = (X[b * kF + i] - mu[i]) / sigma[i];
    float y[2];
    mlp_row(sp, xh, y, Z1 ? Z1 + b * kH : nullptr, Z2 ? Z2 + b * kH : nullptr);
    Y[b * 2 + 0] = y[0];
    Y[b * 2 + 1] = y[1];
}

// Per-row error signals of the pinball loss: dY [B,2], dZ2 [B,64], dZ1 [B,64]
// (scaled by 1 / (B * 2), the mean over rows and outputs).
__global__ void mlp_delta_kernel(const float *params, const float *Y, const float *T, const float *Z1,
                                 const float *Z2, int64_t B, float q, float *dY, float *dZ2, float *dZ1,
                                 float *row_loss) {
    __shared__ float sp[kP];
    for (int i = threadIdx.x; i < kP; i += blockDim.x) sp[i] = params[i];
    __syncthreads();
    const int64_t b = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (b >= B) return;
    const MlpView v = view(sp);
    const float inv = 1.f / (float)(B * kO);
    float dy[kO], loss = 0.f;
#pragma unroll
    for (int o = 0; o < kO; ++o) {
        const float u = T[b * kO + o] - Y[b * kO + o];
        loss += fmaxf(q * u, (q - 1.f) * u);
        dy[o] = (u > 0.f ? -q : 1.f - q) * inv;
        dY[b * kO + o] = dy[o];
    }
    row_loss[b] = loss;
    float dz2[kH];
    for (int j = 0; j < kH; ++j) {
        const float g = dy[0] * v.W3[j * kO + 0] + dy[1] * v.W3[j * kO + 1];
        dz2[j] = Z2[b * kH + j] > 0.f ? g : 0.f;
        dZ2[b * kH + j] = dz2[j];
    }
    for (int i = 0; i < kH; ++i) {
        float g = 0.f;
#pragma unroll 8
        for (int j = 0; j < kH; ++j) g = fmaf(dz2[j], v.W2[i * kH + j], g);
        dZ1[b * kH + i] = Z1[b * kH + i] > 0.f ? g : 0.f;
    }
}

// Weight gradients as sums over rows (one thread per parameter, fixed row
// order: deterministic).
__global__ void mlp_wgrad_kernel(const float *X, const float *mu, const float *sigma, const float *Z1,
                                 const float *Z2, const float *dZ1, const float *dZ2, const float *dY,
                                 int64_t B, float *grad) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= kP) return;
    float g = 0.f;
    int o = t;
    if (o < kF * kH) {                       // W1[i][j] = sum_b xh[b,i] dZ1[b,j]
        const int i = o / kH, j = o % kH;
        for (int64_t b = 0; b < B; ++b) g = fmaf((X[b * kF + i] - mu[i]) / sigma[i], dZ1[b * kH + j], g);
    } else if ((o -= kF * kH) < kH) {        // b1
        for (int64_t b = 0; b < B; ++b) g += dZ1[b * kH + o];
    } else if ((o -= kH) < kH * kH) {        // W2[i][j] = sum_b relu(z1[b,i]) dZ2[b,j]
        const int i = o / kH, j = o % kH;
        for (int64_t b = 0; b < B; ++b) g = fmaf(fmaxf(Z1[b * kH + i], 0.f), dZ2[b * kH + j], g);
    } else if ((o -= kH * kH) < kH) {        // b2
        for (int64_t b = 0; b < B; ++b) g += dZ2[b * kH + o];
    } else if ((o -= kH) < kH * kO) {        // W3[i][o] = sum_b relu(z2[b,i]) dY[b,o]
        const int i = o / kO, oo = o % kO;
        for (int64_t b = 0; b < B; ++b) g = fmaf(fmaxf(Z2[b * kH + i], 0.f), dY[b * kO + oo], g);
    } else {                                 // b3
        o -= kH * kO;
        for (int64_t b = 0; b < B; ++b) g += dY[b * kO + o];
    }
    grad[t] = g;
}

// One Adam step; (1 - beta) is passed separately, rounded from its exact
// decimal value (1 - 0.999f in float32 would be off by 1.3e-5 relative).
__global__ void adam_kernel(float *p, const float *g, float *m, float *v, int n, float lr, float b1,
                            float omb1, float b2, float omb2, float eps, float c1, float c2) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float mi = b1 * m[i] + omb1 * g[i];
    const float vi = b2 * v[i] + omb2 * g[i] * g[i];
    m[i] = mi;
    v[i] = vi;
    p[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
}

// Features of each query (one warp per query; the entry points of the first
// piece are evaluated in parallel, 32 / E' lanes per entry with E' the next
// power of two >= E). With PREDICT the same warp then runs the network on
// its features (parameters in shared memory, two hidden units per lane) and
// writes the query's ef and expansion budget; invalid predictions fall back
// to the fixed beam width.
template <bool PREDICT>
__global__ void features_kernel(const float *X, int d, int metric, DecomposeSpec spec,
                                const int32_t *entries, int E, const float *queries, int64_t nq,
                                const int64_t *l, const int64_t *r, const int32_t *k, int32_t k_max,
                                float *feat, const float *blob, int ef_fixed, int ef_lo, int ef_hi,
                                int32_t *ef_q, int32_t *maxexp_q) {
    __shared__ float sp[PREDICT ? kP : 1];
    if (PREDICT) {
        for (int i = threadIdx.x; i < kP; i += blockDim.x) sp[i] = blob[i];
        __syncthreads();
    }
    const int lane = threadIdx.x & 31;
    const int64_t qi = blockIdx.x * (int64_t)(blockDim.x >> 5) + (threadIdx.x >> 5);
    if (qi >= nq) return;
    esg_piece pc[2];
    const int64_t lq = l[qi], rq = r[qi];
    const int np = esg_decompose_one(spec, lq, rq, pc);
    const int64_t n = spec.n;
    const int kk = k ? k[qi] : k_max;
    float f[kF];
    for (int i = 0; i < kF; ++i) f[i] = 0.f;
    if (np > 0) {
        // single precision throughout: FP64 is slow on this part and the
        // sizes (< 2^31) are exact enough as floats for network inputs
        f[0] = log2f((float)(rq - lq + 1));
        f[1] = (float)np;
        for (int s = 0; s < np; ++s)
            f[2 + s] = log2f((float)(pc[s].node_r - pc[s].node_l + 1)) - log2f((float)(pc[s].pr - pc[s].pl + 1));
        f[4] = pc[0].kind == ESG_PIECE_GRAPH ? 1.f : 0.f;
        f[5] = kk > 0 ? log2f((float)kk) : 0.f;
        f[7] = log2f((float)(pc[0].node_r - pc[0].node_l + 1));
        f[6] = 1.f;
        if (pc[0].kind == ESG_PIECE_GRAPH) {
            int ep = 1;
            while (ep < E) ep <<= 1;
            const int lpe = 32 / ep;                 // lanes per entry
            const int g = lane / lpe, sub = lane % lpe;
            int32_t v = -1;
            if (g < E) v = entries[(size_t)pc[0].heap * E + g];
            const bool ok = v >= 0 && v < n;
            const float4 *q4 = reinterpret_cast<const float4 *>(queries + qi * (int64_t)d);
            const float4 *x4 = reinterpret_cast<const float4 *>(X + (size_t)(ok ? v : 0) * d);
            float acc = 0.f;
            if (ok) {
                for (int j = sub; j < d / 4; j += lpe) {
                    const float4 a = __ldg(q4 + j), b = __ldg(x4 + j);
                    if (metric == ESG_L2SQ) {
                        const float t0 = a.x - b.x, t1 = a.y - b.y, t2 = a.z - b.z, t3 = a.w - b.w;
                        acc = fmaf(t0, t0, acc); acc = fmaf(t1, t1, acc);
                        acc = fmaf(t2, t2, acc); acc = fmaf(t3, t3, acc);
                    } else {
                        acc = fmaf(a.x, b.x, acc); acc = fmaf(a.y, b.y, acc);
                        acc = fmaf(a.z, b.z, acc); acc = fmaf(a.w, b.w, acc);
                    }
                }
            }
            for (int o = lpe >> 1; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
            const bool head = ok && sub == 0;
            const float dist = metric == ESG_L2SQ ? acc : -acc;
            float dmin = head ? dist : INFINITY, dsum = head ? dist : 0.f;
            int cnt = head ? 1 : 0;
            for (int o = 16; o > 0; o >>= 1) {
                dmin = fminf(dmin, __shfl_xor_sync(0xffffffffu, dmin, o));
                dsum += __shfl_xor_sync(0xffffffffu, dsum, o);
                cnt += __shfl_xor_sync(0xffffffffu, cnt, o);
            }
            // the min(k, cnt)-th smallest entry distance: the head lane whose
            // rank (entries before it in (distance, lane) order) is that minus one
            int rank = 0;
            for (int j = 0; j < 32; ++j) {
                const float dj = __shfl_sync(0xffffffffu, dist, j);
                const bool hj = __shfl_sync(0xffffffffu, head ? 1 : 0, j) != 0;
                rank += (hj && (dj < dist || (dj == dist && j < lane))) ? 1 : 0;
            }
            const int kth = min(max(kk, 1), max(cnt, 1)) - 1;
            const unsigned at = __ballot_sync(0xffffffffu, head && rank == kth);
            const float dk = at ? __shfl_sync(0xffffffffu, dist, __ffs(at) - 1) : dmin;
            if (cnt > 0) {
                const float mean = dsum / cnt;
                f[6] = fabsf(mean) > 1e-20f ? dmin / mean : 1.f;
                f[8] = fabsf(mean) > 1e-20f ? (dk - dmin) / fabsf(mean) : 0.f;
            }
        }
    }
    if (lane == 0)
        for (int i = 0; i < kF; ++i) feat[qi * kF + i] = f[i];
    if (!PREDICT) return;
    const MlpView v = view(sp);
    const float *mu = blob + kP, *sigma = blob + kP + kF, *margin = blob + kP + 2 * kF;
    float xh[kF];
#pragma unroll
    for (int i = 0; i < kF; ++i) xh[i] = (f[i] - __ldg(mu + i)) / __ldg(sigma + i);
    // hidden layer 1: units lane and lane + 32
    float h1a = v.b1[lane], h1b = v.b1[lane + 32];
#pragma unroll
    for (int i = 0; i < kF; ++i) {
        h1a = fmaf(xh[i], v.W1[i * kH + lane], h1a);
        h1b = fmaf(xh[i], v.W1[i * kH + lane + 32], h1b);
    }
    h1a = fmaxf(h1a, 0.f);
    h1b = fmaxf(h1b, 0.f);
    // hidden layer 2: units lane and lane + 32, inputs broadcast by shuffle
    float s2a = v.b2[lane], s2b = v.b2[lane + 32];
#pragma unroll 8
    for (int i = 0; i < 32; ++i) {
        const float hi = __shfl_sync(0xffffffffu, h1a, i);
        s2a = fmaf(hi, v.W2[i * kH + lane], s2a);
        s2b = fmaf(hi, v.W2[i * kH + lane + 32], s2b);
    }
#pragma unroll 8
    for (int i = 0; i < 32; ++i) {
        const float hi = __shfl_sync(0xffffffffu, h1b, i);
        s2a = fmaf(hi, v.W2[(i + 32) * kH + lane], s2a);
        s2b = fmaf(hi, v.W2[(i + 32) * kH + lane + 32], s2b);
    }
    const float h2a = fmaxf(s2a, 0.f), h2b = fmaxf(s2b, 0.f);
    float y0 = h2a * v.W3[lane * kO + 0] + h2b * v.W3[(lane + 32) * kO + 0];
    float y1 = h2a * v.W3[lane * kO + 1] + h2b * v.W3[(lane + 32) * kO + 1];
    for (int o = 16; o > 0; o >>= 1) {
        y0 += __shfl_xor_sync(0xffffffffu, y0, o);
        y1 += __shfl_xor_sync(0xffffffffu, y1, o);
    }
    y0 += v.b3[0];
    y1 += v.b3[1];
    if (lane == 0) {
        int ef = ef_fixed, mx = 0;
        if (isfinite(y0) && isfinite(y1)) {
            // the ef margin plus the offset of the query's class of k
            const float e = exp2f(fminf(fmaxf(y0 + margin[0] + margin[2 + esg_k_bucket(kk)], 0.f), 12.f));
            ef = (int)ceilf(e);
            ef = max(ef_lo, min(ef, ef_hi));
            const float x = exp2f(fminf(fmaxf(y1 + margin[1], 0.f), 20.f));
            mx = max(16, min((int)ceilf(x), 16 * ef + 256));
        }
        ef_q[qi] = max(ef, kk);
        maxexp_q[qi] = mx;   // 0 = default cap
    }
}

}  // namespace

// Shapes shared with the host code of the search and the ABI.
int esg_mlp_param_count() { return kP; }

esg_status esg_predict_budget(const esg_index *ix, int post_root, const float *queries, int64_t nq, const int64_t *l,
                              const int64_t *r, const int32_t *k, int32_t k_max, int ef_fixed,
                              float *feat, int32_t *ef_q, int32_t *maxexp_q, cudaStream_t stream) {
    features_kernel<true><<<ceil_div_i(nq, 4), 128, 0, stream>>>(
        ix->X, ix->d, ix->metric, esg_spec_of(ix, post_root), ix->entries, ix->E, queries, nq, l, r, k, k_max,
        feat, ix->mlp, ef_fixed, ix->mlp_ef_lo, ix->mlp_ef_hi, ef_q, maxexp_q);
    ESG_CUDA_TRY(cudaGetLastError());
    return ESG_OK;
}

extern "C" {

int32_t esg_mlp_num_params(void) { return kP; }

int32_t esg_mlp_num_features(void) { return kF; }

esg_status esg_mlp_forward(const float *params, const float *X, const float *mu, const float *sigma,
                           int64_t B, float *Y, esg_stream_t stream) {
    if (!params || !X || !mu || !sigma || !Y || B < 1) { esg_set_error("esg_mlp_forward: bad argument"); return ESG_ERR_INVALID_ARG; }
    mlp_forward_kernel<<<ceil_div_i(B, 128), 128, 0, (cudaStream_t)stream>>>(params, X, mu, sigma, B, Y,
                                                                            nullptr, nullptr);
    ESG_CUDA_TRY(cudaGetLastError());
    return ESG_OK;
}

esg_status esg_mlp_loss_grad(const float *params, const float *X, const float *T, const float *mu,
                             const float *sigma, int64_t B, float quantile, float *grad, float *loss,
                             esg_stream_t stream_v) {
    if (!params || !X || !T || !mu || !sigma || !grad || B < 1 || !(quantile > 0.f && quantile < 1.f)) {
        esg_set_error("esg_mlp_loss_grad: bad argument");
        return ESG_ERR_INVALID_ARG;
    }
    cudaStream_t stream = (cudaStream_t)stream_v;
    float *buf = nullptr;
    const size_t per = 2 + kH + kH + 2 + kH + kH + 1;   // Y, Z1, Z2, dY, dZ2, dZ1, row loss
    ESG_CUDA_TRY(esg_malloc_async((void **)&buf, sizeof(float) * per * B, stream));
    float *Y = buf, *Z1 = Y + 2 * B, *Z2 = Z1 + kH * B, *dY = Z2 + kH * B, *dZ2 = dY + 2 * B,
          *dZ1 = dZ2 + kH * B, *rl = dZ1 + kH * B;
    mlp_forward_kernel<<<ceil_div_i(B, 128), 128, 0, stream>>>(params, X, mu, sigma, B, Y, Z1, Z2);
    mlp_delta_kernel<<<ceil_div_i(B, 128), 128, 0, stream>>>(params, Y, T, Z1, Z2, B, quantile, dY, dZ2, dZ1, rl);
    mlp_wgrad_kernel<<<ceil_div_i(kP, 128), 128, 0, stream>>>(X, mu, sigma, Z1, Z2, dZ1, dZ2, dY, B, grad);
    esg_status st = ESG_OK;
    if (cudaGetLastError() != cudaSuccess) { esg_set_error("esg_mlp_loss_grad: launch failed"); st = ESG_ERR_CUDA; }
    if (st == ESG_OK && loss) {
        std::vector<float> h(B);
        if (cudaMemcpyAsync(h.data(), rl, sizeof(float) * B, cudaMemcpyDeviceToHost, stream) != cudaSuccess ||
            cudaStreamSynchronize(stream) != cudaSuccess) { esg_set_error("esg_mlp_loss_grad: copy"); st = ESG_ERR_CUDA; }
        double s = 0;
        for (int64_t b = 0; b < B; ++b) s += h[b];
        *loss = (float)(s / (double)(B * kO));
    }
    cudaFreeAsync(buf, stream);
    return st;
}

esg_status esg_mlp_adam_step(float *params, const float *grad, float *m, float *v, int32_t step, float lr,
                             esg_stream_t stream) {
    if (!params || !grad || !m || !v || step < 1 || !(lr > 0.f)) { esg_set_error("esg_mlp_adam_step: bad argument"); return ESG_ERR_INVALID_ARG; }
    const double b1 = 0.9, b2 = 0.999;
    adam_kernel<<<ceil_div_i(kP, 256), 256, 0, (cudaStream_t)stream>>>(
        params, grad, m, v, kP, lr, (float)b1, (float)(1.0 - b1), (float)b2, (float)(1.0 - b2), 1e-8f,
        (float)(1.0 - std::pow(b1, step)), (float)(1.0 - std::pow(b2, step)));
    ESG_CUDA_TRY(cudaGetLastError());
    return ESG_OK;
}

esg_status esg_query_features(const esg_index *ix, const float *queries, int64_t nq, const int64_t *l,
                              const int64_t *r, const int32_t *k, int32_t k_max, float *feat,
                              esg_stream_t stream) {
    if (!ix || nq < 0 || (nq > 0 && (!queries || !l || !r || !feat))) { esg_set_error("esg_query_features: bad argument"); return ESG_ERR_INVALID_ARG; }
    if (nq == 0) return ESG_OK;
    features_kernel<false><<<ceil_div_i(nq, 4), 128, 0, (cudaStream_t)stream>>>(
        ix->X, ix->d, ix->metric, esg_spec_of(ix, 0), ix->entries, ix->E, queries, nq, l, r, k, k_max, feat,
        nullptr, 0, 0, 0, nullptr, nullptr);
    ESG_CUDA_TRY(cudaGetLastError());
    return ESG_OK;
}

esg_status esg_query_budget(const esg_index *ix, const float *queries, int64_t nq, const int64_t *l,
                            const int64_t *r, const int32_t *k, int32_t k_max, int32_t ef_fixed,
                            int32_t *ef_out, int32_t *maxexp_out, esg_stream_t stream_v) {
    if (!ix || nq < 0 || nq >= kMaxBatch || k_max < 1 || k_max > 1024 || ef_fixed < 1 || ef_fixed > 1024 ||
        (nq > 0 && (!queries || !l || !r || !ef_out || !maxexp_out))) {
        esg_set_error("esg_query_budget: bad argument");
        return ESG_ERR_INVALID_ARG;
    }
    if (!ix->mlp_ready) { esg_set_error("esg_query_budget: no trained predictor"); return ESG_ERR_INVALID_ARG; }
    if (nq == 0) return ESG_OK;
    cudaStream_t stream = (cudaStream_t)stream_v;
    float *feat = nullptr;
    ESG_CUDA_TRY(esg_malloc_async((void **)&feat, sizeof(float) * nq * kF, stream));
    esg_status st = esg_predict_budget(ix, 0, queries, nq, l, r, k, k_max, ef_fixed, feat, ef_out, maxexp_out,
                                       stream);
    const cudaError_t fe = cudaFreeAsync(feat, stream);
    if (st == ESG_OK && fe != cudaSuccess) { esg_set_error(cudaGetErrorString(fe)); st = ESG_ERR_CUDA; }
    return st;
}

esg_status esg_predictor_set(esg_index *ix, const float *blob_host, int32_t ef_lo, int32_t ef_hi) {
    if (!ix || !blob_host || ef_lo < 1 || ef_hi < ef_lo || ef_hi > 1024) { esg_set_error("esg_predictor_set: bad argument"); return ESG_ERR_INVALID_ARG; }
    const size_t n = (size_t)esg_mlp_blob_floats();
    if (!ix->mlp) ESG_CUDA_TRY(esg_malloc((void **)&ix->mlp, sizeof(float) * n));
    ESG_CUDA_TRY(cudaMemcpy(ix->mlp, blob_host, sizeof(float) * n, cudaMemcpyHostToDevice));
    ix->mlp_host.assign(blob_host, blob_host + n);
    ix->mlp_ef_lo = ef_lo;
    ix->mlp_ef_hi = ef_hi;
    ix->mlp_ready = 1;
    return ESG_OK;
}

int32_t esg_mlp_blob_size(void) { return esg_mlp_blob_floats(); }

esg_status esg_predictor_get(const esg_index *ix, float *blob_host, int32_t *ef_lo, int32_t *ef_hi) {
    if (!ix) { esg_set_error("esg_predictor_get: bad argument"); return ESG_ERR_INVALID_ARG; }
    if (!ix->mlp_ready) { esg_set_error("no trained predictor"); return ESG_ERR_INVALID_ARG; }
    if (blob_host) std::memcpy(blob_host, ix->mlp_host.data(), sizeof(float) * ix->mlp_host.size());
    if (ef_lo) *ef_lo = ix->mlp_ef_lo;
    if (ef_hi) *ef_hi = ix->mlp_ef_hi;
    return ESG_OK;
}

}  // extern "C"

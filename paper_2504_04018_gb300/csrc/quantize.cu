// Low-precision copies of the rank-ordered vectors used for traversal:
// BF16 = round-to-nearest-even of the FP32 value; FP8-E4M3 with one FP32
// scale per row, s_i = max_j |x_ij| / 448 (the largest finite E4M3 value) and
// code_ij = saturating round-to-nearest-even of x_ij / s_i, so that
// x_ij ~= s_i * code_ij. Distances accumulate in FP32.
#include "esg_internal.cuh"

__global__ void to_bf16_kernel(const float *X, int64_t count, __nv_bfloat16 *out) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < count) out[i] = __float2bfloat16_rn(X[i]);
}

// One warp per row.
__global__ void to_fp8_kernel(const float *X, int64_t n, int d, __nv_fp8_e4m3 *out, float *scale) {
    int64_t row = blockIdx.x * (int64_t)(blockDim.x >> 5) + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    if (row >= n) return;
    const float *x = X + row * d;
    float m = 0.f;
    for (int j = lane; j < d; j += 32) m = fmaxf(m, fabsf(x[j]));
    for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
    const float s = m / 448.0f;
    for (int j = lane; j < d; j += 32) {
        float v = s > 0.f ? x[j] / s : 0.f;
        out[row * d + j].__x = __nv_cvt_float_to_fp8(v, __NV_SATFINITE, __NV_E4M3);
    }
    if (lane == 0) scale[row] = s;
}

esg_status esg_make_storage(esg_index *ix, cudaStream_t stream) {
    const int64_t count = ix->n * (int64_t)ix->d;
    if (ix->storage == ESG_BF16) {
        ESG_CUDA_TRY(esg_malloc((void **)&ix->Xb, sizeof(__nv_bfloat16) * count));
        to_bf16_kernel<<<ceil_div_i(count, 256), 256, 0, stream>>>(ix->X, count, ix->Xb);
        ESG_CUDA_TRY(cudaGetLastError());
    } else if (ix->storage == ESG_FP8E4M3) {
        ESG_CUDA_TRY(esg_malloc((void **)&ix->X8, sizeof(__nv_fp8_e4m3) * count));
        ESG_CUDA_TRY(esg_malloc((void **)&ix->scale8, sizeof(float) * ix->n));
        to_fp8_kernel<<<ceil_div_i(ix->n, 8), 256, 0, stream>>>(ix->X, ix->n, ix->d, ix->X8, ix->scale8);
        ESG_CUDA_TRY(cudaGetLastError());
    }
    ESG_CUDA_TRY(cudaStreamSynchronize(stream));
    return ESG_OK;
}

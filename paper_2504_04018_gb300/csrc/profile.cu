// Optional CUDA-event timing of the search kernels, for benchmarks: while
// enabled, each search call records an event pair around its main kernel on
// the call's stream and counts the kernels it launches.
#include "esg_internal.cuh"

#include <mutex>
#include <vector>

namespace {
std::mutex g_mu;
bool g_on = false;
std::vector<std::pair<cudaEvent_t, cudaEvent_t>> g_pairs;
size_t g_used = 0;
int64_t g_launches = 0;
double g_tensor_flops = 0.0;
}  // namespace

bool esg_prof_on() { return g_on; }

void esg_prof_tensor_flops(double flops) {
    if (!g_on) return;
    std::lock_guard<std::mutex> lk(g_mu);
    g_tensor_flops += flops;
}

void esg_prof_count(int64_t launches) {
    if (!g_on) return;
    std::lock_guard<std::mutex> lk(g_mu);
    g_launches += launches;
}

int esg_prof_begin(cudaStream_t stream) {
    if (!g_on) return -1;
    // no timing events inside a graph capture (they would belong to the graph)
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(stream, &cs) != cudaSuccess || cs != cudaStreamCaptureStatusNone) return -1;
    std::lock_guard<std::mutex> lk(g_mu);
    if (g_used == g_pairs.size()) {
        cudaEvent_t a, b;
        if (cudaEventCreate(&a) != cudaSuccess) return -1;
        if (cudaEventCreate(&b) != cudaSuccess) { cudaEventDestroy(a); return -1; }
        g_pairs.push_back({a, b});
    }
    int idx = (int)g_used++;
    cudaEventRecord(g_pairs[idx].first, stream);
    return idx;
}

void esg_prof_end(int idx, cudaStream_t stream) {
    if (idx < 0) return;
    std::lock_guard<std::mutex> lk(g_mu);
    cudaEventRecord(g_pairs[idx].second, stream);
}

extern "C" {

esg_status esg_profile_enable(int32_t on) {
    std::lock_guard<std::mutex> lk(g_mu);
    g_on = on != 0;
    g_used = 0;
    g_launches = 0;
    g_tensor_flops = 0.0;
    return ESG_OK;
}

esg_status esg_profile_read(double *kernel_ms, int64_t *kernel_launches, int64_t *timed_launches,
                            int32_t reset) {
    std::lock_guard<std::mutex> lk(g_mu);
    double total = 0.0;
    for (size_t i = 0; i < g_used; ++i) {
        cudaError_t e = cudaEventSynchronize(g_pairs[i].second);
        if (e != cudaSuccess) { esg_set_error(cudaGetErrorString(e)); return ESG_ERR_CUDA; }
        float ms = 0.f;
        e = cudaEventElapsedTime(&ms, g_pairs[i].first, g_pairs[i].second);
        if (e != cudaSuccess) { esg_set_error(cudaGetErrorString(e)); return ESG_ERR_CUDA; }
        total += ms;
    }
    if (kernel_ms) *kernel_ms = total;
    if (kernel_launches) *kernel_launches = g_launches;
    if (timed_launches) *timed_launches = (int64_t)g_used;
    if (reset) { g_used = 0; g_launches = 0; }
    return ESG_OK;
}

esg_status esg_profile_tensor_work(double *mma_flops, int32_t reset) {
    std::lock_guard<std::mutex> lk(g_mu);
    if (mma_flops) *mma_flops = g_tensor_flops;
    if (reset) g_tensor_flops = 0.0;
    return ESG_OK;
}

}  // extern "C"

// Search entry point that allocates no device memory.
//
// Some callers cannot call cudaMalloc (or cudaMallocAsync) when they search:
// a serving process whose GPU memory is owned entirely by another allocator
// (a framework's caching pool, a pre-partitioned budget), code that must not
// allocate on a latency-critical path, or code paths where an allocation
// would fail or block. esg_search_batch_noalloc runs the same search as
// esg_search_batch but takes its scratch memory from one fixed array in
// device global memory, declared below. That array is reserved in every GPU
// that loads this library and stays there until the process exits.
#include "esg_internal.cuh"

#include <mutex>

namespace {

constexpr size_t kNoAllocScratchBytes = (size_t)64 << 20;  // 64 MiB

// The shared scratch of every esg_search_batch_noalloc call on a device.
// Host code must not use this name as an address: the device address is
// fetched with cudaGetSymbolAddress for the current device.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

std::mutex g_mu;
constexpr int kMaxDevices = 64;
void *g_ptr[kMaxDevices] = {};

// Device address of the array on the current device. Outside stream capture
// every call looks it up again with that device current (the lookup queues
// no GPU work), so the address stays right when the device's context is torn
// down and made again (cudaDeviceReset), which reloads the module. A call on
// a capturing stream uses the address the last call outside capture found
// on that device, so the first call on a device must come before any capture.
esg_status scratch_address(cudaStream_t stream, void **out) {
    int dev = 0;
    ESG_CUDA_TRY(cudaGetDevice(&dev));
    if (dev < 0 || dev >= kMaxDevices) { esg_set_error("device ordinal out of range"); return ESG_ERR_UNSUPPORTED; }
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    ESG_CUDA_TRY(cudaStreamIsCapturing(stream, &cap));
    std::lock_guard<std::mutex> lk(g_mu);
    if (cap == cudaStreamCaptureStatusNone) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || p == nullptr) {
            esg_set_error(std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
            return ESG_ERR_CUDA;
        }
        g_ptr[dev] = p;
    } else if (g_ptr[dev] == nullptr) {
        esg_set_error("esg_search_batch_noalloc: the first call on a device must not be captured");
        return ESG_ERR_INVALID_ARG;
    }
    *out = g_ptr[dev];
    return ESG_OK;
}

}  // namespace

extern "C" esg_status esg_search_batch_noalloc(const esg_index *ix, const float *queries, int64_t nq,
                                               const int64_t *l, const int64_t *r, const int32_t *k,
                                               int32_t k_max, const esg_search_params *params,
                                               int64_t *out_ids, float *out_dist, int32_t *out_count,
                                               int32_t *out_status, int64_t *out_stats,
                                               esg_stream_t stream) {
    if (!ix || nq < 0 || nq >= kMaxBatch || k_max < 1 || k_max > 1024 ||
        (nq > 0 && (!queries || !l || !r || !out_ids || !out_dist || !out_count))) {
        esg_set_error("esg_search_batch_noalloc: bad argument");
        return ESG_ERR_INVALID_ARG;
    }
    if (((uintptr_t)queries) % 16 != 0) {
        esg_set_error("esg_search_batch_noalloc: queries must be 16-byte aligned");
        return ESG_ERR_INVALID_ARG;
    }
    SearchLaunch s;
    s.ix = ix; s.queries = queries; s.nq = nq; s.l = l; s.r = r; s.k = k; s.k_max = k_max;
    s.p = params ? *params : esg_search_params_default();
    if (esg_check_search_params(s.p, "esg_search_batch_noalloc") != ESG_OK) return ESG_ERR_INVALID_ARG;
    void *scratch = nullptr;
    esg_status st = scratch_address((cudaStream_t)stream, &scratch);
    if (st != ESG_OK || nq == 0) return st;
    s.out_ids = out_ids; s.out_dist = out_dist; s.out_count = out_count;
    s.out_status = out_status; s.out_stats = out_stats;
    SearchPlan plan;
    st = esg_search_prepare_capped(s, kNoAllocScratchBytes, plan);
    if (st != ESG_OK) return st;
    // the enqueue resets what must start cleared (work counter, overflow tables)
    return esg_search_enqueue(s, plan, scratch, (cudaStream_t)stream);
}

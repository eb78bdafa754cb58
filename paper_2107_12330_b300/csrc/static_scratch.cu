// static_scratch.cu -- a survey entry point that allocates no device memory.
//
// Some callers cannot allocate device memory at the point where they want a
// survey: latency-bound request loops that must never enter an allocator (an
// allocation can block on the driver or on other streams), and hosts whose
// device memory is carved up by another framework that owns every allocation.
// For them tripoll_survey_static runs the same survey kernels as
// tripoll_survey, but its scratch -- the accumulation record and the two
// work-item counters, which tripoll_survey allocates -- lives in the fixed
// array below, and a window is applied in place instead of through a
// compacted window view.
#include <mutex>

#include "common.cuh"

// 8 MiB of device scratch, present on every GPU that loads the library until
// the process exits.  Layout per call: the record words, then (at the next
// 256-byte boundary) the two 32-bit work-item counters.
constexpr size_t kStaticScratchBytes = size_t(8) << 20;
static __device__ __align__(256) unsigned char g_static_scratch[kStaticScratchBytes];

namespace tp {
namespace {

constexpr size_t kCounterBytes = 256;

constexpr int kMaxDevices = 64;
std::mutex g_scratch_mu;
void* g_scratch_addr[kMaxDevices] = {};

// Device address of g_static_scratch on the current device `dev`, looked up
// once per device (the host-side symbol is only a stand-in for it) and kept for
// the life of the process: the device's primary context must not be reset
// while the library is loaded.
int scratch_address(int dev, void** out) {
    if (dev < 0 || dev >= kMaxDevices) return fail(TRIPOLL_ERR_INVALID_ARG, "device index out of range");
    std::lock_guard<std::mutex> lk(g_scratch_mu);
    if (!g_scratch_addr[dev]) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_static_scratch);
        if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress(static scratch)");
        g_scratch_addr[dev] = p;
    }
    *out = g_scratch_addr[dev];
    return TRIPOLL_OK;
}

}  // namespace
}  // namespace tp

using namespace tp;

extern "C" int tripoll_survey_static(tripoll_graph_t g, uint32_t kind_mask, uint32_t t_lo, uint32_t t_hi,
                                     uint64_t* result, void* cuda_stream) {
    int rc = check_survey_args(g, kind_mask, t_lo, t_hi, result);
    if (rc) return rc;
    const uint64_t words = make_layout(kind_mask, g->Lv, g->Le, g->n, g->m).words * g->num_graphs;
    const uint64_t record_bytes = (words * 8 + 255) / 256 * 256;
    if (record_bytes + kCounterBytes > kStaticScratchBytes)
        return fail(TRIPOLL_ERR_NO_MEMORY, "survey result of " + std::to_string(words * 8) +
                                               " bytes exceeds the static scratch (8 MiB less 256 bytes)");
    int dev = 0;
    TP_CUDA(cudaGetDevice(&dev));
    if (dev != g->device) return fail(TRIPOLL_ERR_INVALID_ARG, "the graph's device is not the current device");
    void* base = nullptr;
    if ((rc = scratch_address(dev, &base))) return rc;
    cudaStream_t s = (cudaStream_t)cuda_stream;
    unsigned long long* acc = static_cast<unsigned long long*>(base);
    uint32_t* counters = reinterpret_cast<uint32_t*>(static_cast<unsigned char*>(base) + record_bytes);
    // the array keeps the previous call's contents: clear the record first
    TP_CUDA(cudaMemsetAsync(acc, 0, words * 8, s));
    if (g->n && (rc = launch_survey(g, kind_mask, t_lo, t_hi, 0, g->n, acc, counters, s, false))) return rc;
    TP_CUDA(cudaMemcpyAsync(result, acc, words * 8, cudaMemcpyDefault, s));
    if (!is_device_pointer(result)) TP_CUDA(cudaStreamSynchronize(s));
    return TRIPOLL_OK;
}

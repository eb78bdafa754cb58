// abi.cu -- the C entry points around the builder and the survey kernels:
// status text, argument checks, result buffers, statistics, export, shards.
#include <algorithm>
#include <atomic>
#include <mutex>
#include <string>
#include <vector>

#include "common.cuh"
#include "primitives.cuh"

namespace tp {

namespace {
thread_local std::string g_last_error;
std::atomic<uint64_t> g_launches{0};
}

void note_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }

void set_error(const std::string& msg) { g_last_error = msg; }

int fail(int status, const std::string& msg) {
    g_last_error = msg;
    return status;
}

int cuda_fail(cudaError_t e, const char* what) {
    g_last_error = std::string(what) + ": " + cudaGetErrorString(e);
    return e == cudaErrorMemoryAllocation ? TRIPOLL_ERR_NO_MEMORY : TRIPOLL_ERR_CUDA;
}

// ---- device memory ----------------------------------------------------------------------------

namespace {
std::mutex g_alloc_mu;
Allocator g_allocator;  // alloc == nullptr: the library's pool

constexpr int kMaxPoolDevices = 64;
std::mutex g_pool_mu;
cudaMemPool_t g_pool[kMaxPoolDevices] = {};

// The library's own stream-ordered pool on device `dev`, created on first use.  It keeps up to a
// quarter of the device's memory (at most 64 GiB) cached between calls, so that repeated builds
// and surveys do not return memory to the driver and map it again.
cudaError_t library_pool(int dev, cudaMemPool_t* out) {
    if (dev < 0 || dev >= kMaxPoolDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lk(g_pool_mu);
    if (!g_pool[dev]) {
        cudaMemPoolProps props = {};
        props.allocType = cudaMemAllocationTypePinned;
        props.handleTypes = cudaMemHandleTypeNone;
        props.location.type = cudaMemLocationTypeDevice;
        props.location.id = dev;
        cudaMemPool_t pool;
        cudaError_t e = cudaMemPoolCreate(&pool, &props);
        if (e != cudaSuccess) return e;
        size_t free_b = 0, total_b = 0;
        if (cudaMemGetInfo(&free_b, &total_b) == cudaSuccess) {
            uint64_t thr = std::min<uint64_t>(total_b / 4, 64ull << 30);
            cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr);
        }
        cudaGetLastError();
        g_pool[dev] = pool;
    }
    *out = g_pool[dev];
    return cudaSuccess;
}
}  // namespace

Allocator current_allocator() {
    std::lock_guard<std::mutex> lk(g_alloc_mu);
    return g_allocator;
}

cudaError_t dev_alloc(void** p, size_t bytes, cudaStream_t s, const Allocator& a) {
    *p = nullptr;
    if (a.alloc) {
        void* q = a.alloc(bytes, (void*)s, a.ctx);
        if (!q) return cudaErrorMemoryAllocation;
        if (reinterpret_cast<uintptr_t>(q) & 255u) {  // the stated alignment (vector loads rely on it)
            a.free(q, bytes, (void*)s, a.ctx);
            return cudaErrorMemoryAllocation;
        }
        *p = q;
        return cudaSuccess;
    }
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    cudaMemPool_t pool;
    if ((e = library_pool(dev, &pool)) != cudaSuccess) return e;
    return cudaMallocFromPoolAsync(p, bytes, pool, s);
}

void dev_free(void* p, size_t bytes, cudaStream_t s, const Allocator& a) {
    if (!p) return;
    if (a.alloc) a.free(p, bytes, (void*)s, a.ctx);
    else cudaFreeAsync(p, s);
}

void drop_block(tripoll_graph* g, void* ptr, cudaStream_t s) {
    for (size_t i = 0; i < g->blocks.size(); ++i)
        if (g->blocks[i].ptr == ptr) {
            dev_free(ptr, g->blocks[i].bytes, s, g->blocks[i].al);
            g->blocks.erase(g->blocks.begin() + i);
            return;
        }
}

// ---- survey plans ------------------------------------------------------------------------------

namespace {
std::mutex g_plan_mu;
tripoll_plan g_default_plan = {kWarpPlanQ, kItemInEdges, 4 * kBlockChunk, 1};
}  // namespace

tripoll_plan default_plan() {
    std::lock_guard<std::mutex> lk(g_plan_mu);
    return g_default_plan;
}

int check_plan(const tripoll_plan& p) {
    if (p.warp_max_dplus < 32 || p.warp_max_dplus > kWarpPlanMax)
        return fail(TRIPOLL_ERR_INVALID_ARG, "warp_max_dplus must lie in 32..256");
    if (p.block_item_in_edges < 256 || p.block_item_in_edges > kItemInEdges || p.block_item_in_edges % 256)
        return fail(TRIPOLL_ERR_INVALID_ARG, "block_item_in_edges must be a multiple of 256 in 256..2048");
    if (p.long_list_min_dplus < kBlockChunk || p.long_list_min_dplus > 65536)
        return fail(TRIPOLL_ERR_INVALID_ARG, "long_list_min_dplus must lie in 1024..65536");
    if (p.window_view > 1) return fail(TRIPOLL_ERR_INVALID_ARG, "window_view must be 0 or 1");
    return TRIPOLL_OK;
}

void swap_block(tripoll_graph* g, void* graph_ptr, Scratch& sc) {
    for (Block& b : g->blocks)
        if (b.ptr == graph_ptr) {
            std::swap(b.ptr, sc.ptr);
            std::swap(b.bytes, sc.bytes);
            std::swap(b.al, sc.al);
            return;
        }
}

bool is_device_pointer(const void* p) {
    cudaPointerAttributes attr;
    if (cudaPointerGetAttributes(&attr, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return attr.type == cudaMemoryTypeDevice || attr.type == cudaMemoryTypeManaged;
}

bool is_pinned_host_pointer(const void* p) {
    cudaPointerAttributes attr;
    if (cudaPointerGetAttributes(&attr, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return attr.type == cudaMemoryTypeHost;
}

int check_survey_args(const tripoll_graph* g, uint32_t kinds, uint32_t t_lo, uint32_t t_hi, const void* result) {
    if (!g) return fail(TRIPOLL_ERR_INVALID_ARG, "graph handle is NULL");
    if (!result) return fail(TRIPOLL_ERR_INVALID_ARG, "result is NULL");
    if (kinds == 0 || (kinds & ~TRIPOLL_ALL_KINDS)) return fail(TRIPOLL_ERR_INVALID_ARG, "bad kind mask");
    if (t_lo > t_hi) return fail(TRIPOLL_ERR_INVALID_ARG, "t_lo > t_hi");
    if ((kinds & (TRIPOLL_ELABEL_TRIPLES | TRIPOLL_MAX_ELABEL)) && !g->has_el)
        return fail(TRIPOLL_ERR_NO_EDGE_LABELS, "edge-label survey on a graph without edge labels");
    if ((kinds & (TRIPOLL_VERTEX_LOCAL | TRIPOLL_EDGE_LOCAL)) && g->graph_of)
        return fail(TRIPOLL_ERR_INVALID_ARG, "local counts are not available for batched graphs");
    return TRIPOLL_OK;
}

// Survey into `result` (device or host), pivots [p_lo, p_hi); ev as in launch_survey.
int survey_into(const tripoll_graph* g, uint32_t kinds, uint32_t t_lo, uint32_t t_hi, uint64_t p_lo, uint64_t p_hi,
                uint64_t* result, cudaStream_t s, cudaEvent_t* ev = nullptr) {
    int rc = check_survey_args(g, kinds, t_lo, t_hi, result);
    if (rc) return rc;
    const Layout lay = make_layout(kinds, g->Lv, g->Le, g->n, g->m);
    const uint64_t words = lay.words * g->num_graphs;
    const bool dev_result = is_device_pointer(result);
    Scratch acc, ctr;
    TP_CUDA(ctr.alloc(16, s));
    unsigned long long* a = reinterpret_cast<unsigned long long*>(result);
    if (!dev_result) {
        TP_CUDA(acc.alloc(words * 8, s));
        a = acc.as<unsigned long long>();
    }
    TP_CUDA(cudaMemsetAsync(a, 0, words * 8, s));
    if (p_hi > g->n) p_hi = g->n;
    if (p_lo < p_hi &&
        (rc = launch_survey(g, kinds, t_lo, t_hi, p_lo, p_hi, a, ctr.as<uint32_t>(), s, g->plan.window_view != 0, ev)))
        return rc;
    if (!dev_result) {
        TP_CUDA(cudaMemcpyAsync(result, a, words * 8, cudaMemcpyDeviceToHost, s));
        TP_CUDA(cudaStreamSynchronize(s));
    }
    return TRIPOLL_OK;
}

namespace {

// survey cost of each pivot position: the wedges rooted at it plus its out-edges
__global__ void pivot_cost_kernel(const uint64_t* __restrict__ off, uint64_t n, uint64_t* __restrict__ cost) {
    for (uint64_t p = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; p < n; p += (uint64_t)gridDim.x * blockDim.x) {
        uint64_t d = off[p + 1] - off[p];
        cost[p] = d * (d ? d - 1 : 0) / 2 + d;
    }
}

// bounds[i] = first position whose inclusive prefix cost exceeds total*i/parts
__global__ void cut_kernel(const uint64_t* __restrict__ prefix, uint64_t n, uint32_t parts, uint64_t* bounds) {
    uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i > parts) return;
    if (i == 0) { bounds[0] = 0; return; }
    if (i == parts) { bounds[parts] = n; return; }
    const uint64_t total = n ? prefix[n - 1] : 0;
    const unsigned __int128 target128 = (unsigned __int128)total * i / parts;
    const uint64_t target = (uint64_t)target128;
    uint64_t lo = 0, hi = n;
    while (lo < hi) {
        uint64_t mid = lo + ((hi - lo) >> 1);
        if (prefix[mid] <= target) lo = mid + 1; else hi = mid;
    }
    bounds[i] = lo;
}

// wedges of the window's subgraph: sum over pivots p of C(k, 2), k the
// number of in-window edges in Adj+(p)
__global__ void wedge_checks_kernel(const uint64_t* __restrict__ off, const uint32_t* __restrict__ ts, uint64_t n,
                                    uint32_t t_lo, uint32_t t_hi, unsigned long long* out) {
    unsigned long long w = 0;
    for (uint64_t p = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; p < n; p += (uint64_t)gridDim.x * blockDim.x) {
        unsigned long long k = 0;
        for (uint64_t e = off[p]; e < off[p + 1]; ++e) k += (ts[e] >= t_lo && ts[e] <= t_hi) ? 1u : 0u;
        w += k * (k ? k - 1 : 0) / 2;
    }
    for (int o = 16; o; o >>= 1) w += __shfl_xor_sync(0xffffffffu, w, o);
    if ((threadIdx.x & 31) == 0 && w) atomicAdd(out, w);
}

}  // namespace
}  // namespace tp

using namespace tp;

extern "C" int tripoll_wedge_checks(tripoll_graph_t g, uint32_t t_lo, uint32_t t_hi, uint64_t* out, void* cuda_stream) {
    if (!g || !out || t_lo > t_hi) return fail(TRIPOLL_ERR_INVALID_ARG, "bad wedge_checks arguments");
    cudaStream_t s = (cudaStream_t)cuda_stream;
    Scratch acc;
    TP_CUDA(acc.alloc(8, s));
    TP_CUDA(cudaMemsetAsync(acc.ptr, 0, 8, s));
    if (g->m) {
        wedge_checks_kernel<<<(unsigned)std::min<uint64_t>((g->n + 255) / 256, 148 * 32), 256, 0, s>>>(
            g->off, g->ts, g->n, t_lo, t_hi, acc.as<unsigned long long>()); ::tp::note_launch();
        TP_CUDA(cudaGetLastError());
    }
    TP_CUDA(cudaMemcpyAsync(out, acc.ptr, 8, cudaMemcpyDeviceToHost, s));
    TP_CUDA(cudaStreamSynchronize(s));
    return TRIPOLL_OK;
}

extern "C" int tripoll_set_allocator(tripoll_alloc_fn alloc, tripoll_free_fn free_fn, void* ctx) {
    if ((alloc == nullptr) != (free_fn == nullptr))
        return fail(TRIPOLL_ERR_INVALID_ARG, "alloc and free_fn must both be set or both be NULL");
    std::lock_guard<std::mutex> lk(g_alloc_mu);
    g_allocator.alloc = alloc;
    g_allocator.free = free_fn;
    g_allocator.ctx = alloc ? ctx : nullptr;
    return TRIPOLL_OK;
}

extern "C" const char* tripoll_status_string(int status) {
    switch (status) {
        case TRIPOLL_OK: return "ok";
        case TRIPOLL_ERR_INVALID_ARG: return "invalid argument";
        case TRIPOLL_ERR_VERTEX_RANGE: return "vertex id out of range";
        case TRIPOLL_ERR_LABEL_RANGE: return "label out of range";
        case TRIPOLL_ERR_NO_MEMORY: return "out of device memory or scratch budget";
        case TRIPOLL_ERR_CUDA: return "CUDA error";
        case TRIPOLL_ERR_TIMEOUT: return "timed out";
        case TRIPOLL_ERR_NO_EDGE_LABELS: return "graph has no edge labels";
        case TRIPOLL_ERR_NOT_FOUND: return "not found";
        default: return "unknown status";
    }
}

extern "C" const char* tripoll_last_error(void) { return g_last_error.c_str(); }

extern "C" uint64_t tripoll_launch_count(void) { return g_launches.load(); }

extern "C" uint64_t tripoll_result_words(uint32_t kind_mask, uint32_t num_vlabels, uint32_t num_elabels,
                                         uint64_t num_vertices, uint64_t num_edges) {
    return make_layout(kind_mask, num_vlabels ? num_vlabels : 1, num_elabels ? num_elabels : 1, num_vertices,
                       num_edges).words;
}

extern "C" int tripoll_survey(tripoll_graph_t g, uint32_t kind_mask, uint32_t t_lo, uint32_t t_hi, uint64_t* result,
                              void* cuda_stream) {
    return survey_into(g, kind_mask, t_lo, t_hi, 0, g ? g->n : 0, result, (cudaStream_t)cuda_stream);
}

extern "C" int tripoll_survey_range(tripoll_graph_t g, uint32_t kind_mask, uint32_t t_lo, uint32_t t_hi,
                                    uint64_t pivot_lo, uint64_t pivot_hi, uint64_t* result, void* cuda_stream) {
    if (pivot_lo > pivot_hi) return fail(TRIPOLL_ERR_INVALID_ARG, "pivot_lo > pivot_hi");
    return survey_into(g, kind_mask, t_lo, t_hi, pivot_lo, pivot_hi, result, (cudaStream_t)cuda_stream);
}

extern "C" int tripoll_survey_timed(tripoll_graph_t g, uint32_t kind_mask, uint32_t t_lo, uint32_t t_hi,
                                    uint64_t pivot_lo, uint64_t pivot_hi, uint64_t* result, float* phase_ms,
                                    void* cuda_stream) {
    if (!phase_ms) return fail(TRIPOLL_ERR_INVALID_ARG, "phase_ms is NULL");
    if (pivot_lo > pivot_hi) return fail(TRIPOLL_ERR_INVALID_ARG, "pivot_lo > pivot_hi");
    int rc = check_survey_args(g, kind_mask, t_lo, t_hi, result);
    if (rc) return rc;
    cudaStream_t s = (cudaStream_t)cuda_stream;
    cudaEvent_t ev[5] = {};
    struct Events {  // destroyed on every path
        cudaEvent_t* e;
        ~Events() {
            for (int k = 0; k < 5; ++k)
                if (e[k]) cudaEventDestroy(e[k]);
        }
    } guard{ev};
    for (int k = 0; k < 5; ++k) TP_CUDA(cudaEventCreate(&ev[k]));
    // phases that do not run still get their boundary recorded: an empty phase reads 0
    for (int k = 0; k < 5; ++k) TP_CUDA(cudaEventRecord(ev[k], s));
    if ((rc = survey_into(g, kind_mask, t_lo, t_hi, pivot_lo, pivot_hi, result, s, ev))) return rc;
    TP_CUDA(cudaStreamSynchronize(s));
    for (int k = 0; k < 4; ++k) TP_CUDA(cudaEventElapsedTime(&phase_ms[k], ev[k], ev[k + 1]));
    return TRIPOLL_OK;
}

extern "C" int tripoll_get_plan(tripoll_graph_t g, tripoll_plan* plan) {
    if (!g || !plan) return fail(TRIPOLL_ERR_INVALID_ARG, "NULL argument");
    *plan = g->plan;
    return TRIPOLL_OK;
}

static bool same_items(const tripoll_plan& a, const tripoll_plan& b) {
    return a.warp_max_dplus == b.warp_max_dplus && a.block_item_in_edges == b.block_item_in_edges &&
           a.long_list_min_dplus == b.long_list_min_dplus;
}

extern "C" int tripoll_set_plan(tripoll_graph_t g, const tripoll_plan* plan, void* cuda_stream) {
    if (!g || !plan) return fail(TRIPOLL_ERR_INVALID_ARG, "NULL argument");
    int rc = check_plan(*plan);
    if (rc) return rc;
    cudaStream_t s = (cudaStream_t)cuda_stream;
    const bool rebuild = !same_items(g->plan, *plan);
    g->plan = *plan;
    if (rebuild && (rc = build_plan(g, s))) return rc;
    TP_CUDA(cudaStreamSynchronize(s));
    return TRIPOLL_OK;
}

extern "C" int tripoll_set_default_plan(const tripoll_plan* plan) {
    tripoll_plan p = {kWarpPlanQ, kItemInEdges, 4 * kBlockChunk, 1};
    if (plan) {
        int rc = check_plan(*plan);
        if (rc) return rc;
        p = *plan;
    }
    std::lock_guard<std::mutex> lk(g_plan_mu);
    g_default_plan = p;
    return TRIPOLL_OK;
}

extern "C" int tripoll_tune(tripoll_graph_t g, uint32_t kind_mask, uint32_t t_lo, uint32_t t_hi, uint32_t reps,
                            tripoll_plan* best, float* best_ms, float* start_ms, void* cuda_stream) {
    int rc = check_survey_args(g, kind_mask, t_lo, t_hi, &kind_mask);
    if (rc) return rc;
    cudaStream_t s = (cudaStream_t)cuda_stream;
    reps = std::max(1u, reps);
    const uint64_t words = make_layout(kind_mask, g->Lv, g->Le, g->n, g->m).words * g->num_graphs;
    Scratch res;
    TP_CUDA(res.alloc(words * 8, s));
    cudaEvent_t e0, e1;
    TP_CUDA(cudaEventCreate(&e0));
    if (cudaEventCreate(&e1) != cudaSuccess) {
        cudaEventDestroy(e0);
        return fail(TRIPOLL_ERR_CUDA, "cudaEventCreate");
    }
    struct Events {
        cudaEvent_t a, b;
        ~Events() { cudaEventDestroy(a); cudaEventDestroy(b); }
    } guard{e0, e1};
    // median device time of `reps` surveys under plan P (g keeps P)
    auto time_plan = [&](const tripoll_plan& P, float* ms) -> int {
        int r = tripoll_set_plan(g, &P, s);
        if (r) return r;
        if ((r = survey_into(g, kind_mask, t_lo, t_hi, 0, g->n, res.as<uint64_t>(), s))) return r;
        std::vector<float> t;
        for (uint32_t k = 0; k < reps; ++k) {
            TP_CUDA(cudaEventRecord(e0, s));
            if ((r = survey_into(g, kind_mask, t_lo, t_hi, 0, g->n, res.as<uint64_t>(), s))) return r;
            TP_CUDA(cudaEventRecord(e1, s));
            TP_CUDA(cudaEventSynchronize(e1));
            float x = 0;
            TP_CUDA(cudaEventElapsedTime(&x, e0, e1));
            t.push_back(x);
        }
        std::sort(t.begin(), t.end());
        *ms = t[t.size() / 2];
        return TRIPOLL_OK;
    };
    tripoll_plan cur = g->plan;
    float cur_ms = 0;
    if ((rc = time_plan(cur, &cur_ms))) return rc;
    if (start_ms) *start_ms = cur_ms;
    const bool window = !(t_lo == 0 && t_hi == 0xFFFFFFFFu);
    const std::vector<uint32_t> cand[4] = {{32, 64, 128, 256}, {512, 1024, 2048}, {2048, 4096, 8192},
                                           window ? std::vector<uint32_t>{1, 0} : std::vector<uint32_t>{}};
    for (int f = 0; f < 4; ++f) {
        for (uint32_t v : cand[f]) {
            tripoll_plan P = cur;
            uint32_t* field[4] = {&P.warp_max_dplus, &P.block_item_in_edges, &P.long_list_min_dplus, &P.window_view};
            if (*field[f] == v) continue;
            *field[f] = v;
            float ms = 0;
            if ((rc = time_plan(P, &ms))) return rc;
            if (ms < cur_ms) {
                cur = P;
                cur_ms = ms;
            }
        }
    }
    if ((rc = tripoll_set_plan(g, &cur, s))) return rc;
    if (best) *best = cur;
    if (best_ms) *best_ms = cur_ms;
    return TRIPOLL_OK;
}

extern "C" int tripoll_partition_pivots(tripoll_graph_t g, uint32_t parts, uint64_t* bounds, void* cuda_stream) {
    if (!g || !bounds || parts == 0) return fail(TRIPOLL_ERR_INVALID_ARG, "bad partition arguments");
    cudaStream_t s = (cudaStream_t)cuda_stream;
    const uint64_t n = g->n;
    Scratch cost, prefix, tmp, cuts;
    TP_CUDA(cost.alloc((n + 1) * 8, s));
    TP_CUDA(prefix.alloc((n + 1) * 8, s));
    TP_CUDA(cuts.alloc((parts + 1) * 8ull, s));
    if (n) {
        pivot_cost_kernel<<<(unsigned)std::min<uint64_t>((n + 255) / 256, 148 * 64), 256, 0, s>>>(g->off, n,
                                                                                               cost.as<uint64_t>()); ::tp::note_launch();
        TP_CUDA(tmp.alloc(prim::scan_scratch_bytes(n), s));
        int rc;
        if ((rc = prim::scan<uint64_t, true>(prim::Load<uint64_t, uint64_t>{cost.as<uint64_t>(), n},
                                             prefix.as<uint64_t>(), n, tmp.ptr, s)))
            return rc;
    }
    cut_kernel<<<(parts + 1 + 255) / 256, 256, 0, s>>>(prefix.as<uint64_t>(), n, parts, cuts.as<uint64_t>()); ::tp::note_launch();
    TP_CUDA(cudaGetLastError());
    TP_CUDA(cudaMemcpyAsync(bounds, cuts.ptr, (parts + 1) * 8ull, cudaMemcpyDeviceToHost, s));
    TP_CUDA(cudaStreamSynchronize(s));
    return TRIPOLL_OK;
}

extern "C" int tripoll_graph_stats(tripoll_graph_t g, tripoll_graph_info* info) {
    if (!g || !info) return fail(TRIPOLL_ERR_INVALID_ARG, "NULL argument");
    *info = g->info;
    return TRIPOLL_OK;
}

extern "C" int tripoll_graph_export(tripoll_graph_t g, uint64_t* offsets, uint32_t* col, uint32_t* ts,
                                    uint8_t* elabel, uint32_t* order, void* cuda_stream) {
    if (!g) return fail(TRIPOLL_ERR_INVALID_ARG, "graph handle is NULL");
    if (elabel && !g->has_el) return fail(TRIPOLL_ERR_NO_EDGE_LABELS, "graph has no edge labels");
    cudaStream_t s = (cudaStream_t)cuda_stream;
    if (offsets) TP_CUDA(cudaMemcpyAsync(offsets, g->off, (g->n + 1) * 8, cudaMemcpyDeviceToHost, s));
    if (col && g->m) TP_CUDA(cudaMemcpyAsync(col, g->col, g->m * 4, cudaMemcpyDeviceToHost, s));
    if (ts && g->m) TP_CUDA(cudaMemcpyAsync(ts, g->ts, g->m * 4, cudaMemcpyDeviceToHost, s));
    if (elabel && g->m) TP_CUDA(cudaMemcpyAsync(elabel, g->el, g->m, cudaMemcpyDeviceToHost, s));
    if (order && g->n) TP_CUDA(cudaMemcpyAsync(order, g->order, g->n * 4, cudaMemcpyDeviceToHost, s));
    TP_CUDA(cudaStreamSynchronize(s));
    return TRIPOLL_OK;
}

extern "C" void tripoll_destroy(tripoll_graph_t g) {
    if (!g) return;
    free_graph_arrays(g);
    delete g;
}

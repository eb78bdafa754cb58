// common.cuh -- shared declarations of the survey library (status handling,
// the graph object, device helpers).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <utility>
#include <vector>

#include "../../include/tripoll.h"

namespace tp {

// ---- status / error detail -------------------------------------------------------------------

void set_error(const std::string& msg);
int fail(int status, const std::string& msg);
int cuda_fail(cudaError_t e, const char* what);

#define TP_CUDA(call)                                           \
    do {                                                        \
        cudaError_t tp_e_ = (call);                             \
        if (tp_e_ != cudaSuccess) return ::tp::cuda_fail(tp_e_, #call); \
    } while (0)

// ---- device memory owned by the library --------------------------------------------------------

// Every device allocation of the library goes through dev_alloc / dev_free.  By default the
// memory comes from a stream-ordered pool private to the library (one per device), so the
// caller's default pool and its settings are left as they are; tripoll_set_allocator installs
// the caller's functions instead.  An allocation remembers the allocator that made it and is
// returned to that one, even if another allocator has been installed since.
struct Allocator {
    tripoll_alloc_fn alloc = nullptr;  // null: the library's own pool
    tripoll_free_fn free = nullptr;
    void* ctx = nullptr;
};
Allocator current_allocator();
cudaError_t dev_alloc(void** p, size_t bytes, cudaStream_t s, const Allocator& a);
void dev_free(void* p, size_t bytes, cudaStream_t s, const Allocator& a);

// Stream-ordered temporary: freed on the stream when it goes out of scope.
struct Scratch {
    void* ptr = nullptr;
    size_t bytes = 0;
    cudaStream_t stream = nullptr;
    Allocator al;
    Scratch() = default;
    Scratch(const Scratch&) = delete;
    Scratch& operator=(const Scratch&) = delete;
    ~Scratch() { release(); }
    cudaError_t alloc(size_t n, cudaStream_t s) {
        release();
        stream = s;
        bytes = n ? n : 16;
        al = current_allocator();
        return dev_alloc(&ptr, bytes, s, al);
    }
    void release() {
        if (ptr) dev_free(ptr, bytes, stream, al);
        ptr = nullptr;
    }
    void swap(Scratch& o) {
        std::swap(ptr, o.ptr);
        std::swap(bytes, o.bytes);
        std::swap(stream, o.stream);
        std::swap(al, o.al);
    }
    template <class T> T* as() const { return static_cast<T*>(ptr); }
};

// A device array owned by a graph (released by free_graph_arrays).
struct Block {
    void* ptr = nullptr;
    size_t bytes = 0;
    Allocator al;
};

// Count of the library's own kernel launches (tripoll_launch_count).
void note_launch();

// Is p device-accessible memory (device or managed allocation)?
bool is_device_pointer(const void* p);
// Is p page-locked host memory (cudaHostAlloc or registered)?
bool is_pinned_host_pointer(const void* p);

// ---- the built graph G+ ------------------------------------------------------------------------

// In-edge record: the directed edge (p,q) of G+ at CSR position e, with
// end = one past the last position of Adj+(p), the edge's timestamp, and
// meta = edge label | (label of p) << 8.  Sorted by (q, p).
struct __align__(16) InEdge {
    uint32_t e;
    uint32_t end;
    uint32_t ts;
    uint32_t meta;
};

// A unit of survey work: middle vertex q, the part [qlo, qhi) of its out-list
// staged on chip, and the in-edges [in_lo, in_hi) of q whose pivot suffixes
// are checked against it.
struct __align__(16) WorkItem {
    uint32_t q;
    uint32_t qlo;     // offset into q's out-list
    uint32_t qlen;    // staged entries
    uint32_t in_lo;   // into in_edge[], absolute
    uint32_t in_hi;
    uint32_t flags;   // bit 0: chunked (restrict suffix to the staged value range)
    uint32_t vpos;    // the part's first CSR position, off[q] + qlo (in a window view's positions once translated)
    uint32_t pad;
};

struct GraphDev {
    uint64_t n = 0, m = 0;
    const uint64_t* off = nullptr;   // [n+1] out-list offsets, by position in <+
    const uint32_t* col = nullptr;   // [m] targets (positions), ascending per list
    const uint32_t* ts = nullptr;    // [m]
    const uint8_t* el = nullptr;     // [m] or null
    const uint8_t* vl = nullptr;     // [n] vertex label by position
    const uint32_t* deg = nullptr;   // [n] degree in the simple graph, by position
    const uint32_t* order = nullptr; // [n] input vertex id at each position
    const uint32_t* graph_of = nullptr; // [n] graph index by position (batched) or null
    const uint64_t* in_off = nullptr;   // [n+1]
    const InEdge* in_edge = nullptr;    // [m]
    // Window view: when set, col/ts/el above hold only the edges whose timestamp lies in the survey's
    // window (same order), and vidx tells where CSR position e of G+ (e in [0, m]) lands in it: word
    // vidx[e >> 5] holds the in-window edges before position 32 (e >> 5) and the in-window bits of
    // those 32 positions (view_pos).  off, in_off and in_edge stay those of G+ and are translated
    // through vidx.  (8 bytes per 32 edges: the index stays in L2 on large graphs.)
    const uint2* vidx = nullptr;        // [(m >> 5) + 1] or null
    const uint32_t* vorig = nullptr;    // [m] CSR position in G+ of each view entry (per-edge counts only)
    // The window view's in-edges: when set, in_edge above holds only the in-edge records whose edge lies in
    // the window (same order), with e and end already positions of the view, iidx tells where in-edge
    // record k of G+ lands among them (as vidx does for CSR positions), and vin_e gives the CSR position in
    // G+ of each one's edge (p,q).  Work items keep G+'s in-edge ranges and are translated through iidx.
    const uint2* iidx = nullptr;        // [(m >> 5) + 1] or null
    const uint32_t* vin_e = nullptr;    // [in-window in-edges]
};

}  // namespace tp

struct tripoll_graph {
    int device = 0;
    uint64_t n = 0, m = 0, m_in = 0;
    uint32_t num_graphs = 1;
    uint32_t Lv = 1, Le = 1;
    bool has_el = false;
    // per-graph vertex base in position space is not contiguous; batched builds keep
    // the input-vertex base of every graph for the local-count output
    uint64_t* graph_vbase = nullptr;  // device [num_graphs+1] (batched only)
    // device arrays
    uint64_t* off = nullptr;
    uint32_t* col = nullptr;
    uint32_t* ts = nullptr;
    uint8_t* el = nullptr;
    uint8_t* vl = nullptr;
    uint32_t* deg = nullptr;
    uint32_t* order = nullptr;
    uint32_t* graph_of = nullptr;
    uint64_t* in_off = nullptr;
    tp::InEdge* in_edge = nullptr;
    // survey plan (the thresholds of plan; see tripoll_plan)
    tripoll_plan plan{};
    tp::WorkItem* items_warp = nullptr;   // d+(q) <= plan.warp_max_dplus
    tp::WorkItem* items_block = nullptr;  // up to plan.long_list_min_dplus, parts of kBlockChunk
    tp::WorkItem* items_big = nullptr;    // longer out-lists, parts of kBigChunk
    // Edges by timestamp bucket (bucket b holds the timestamps t with t >> ts_shift == b), which bounds on the
    // host how many edges a window holds; filled on demand (tp::ts_histogram), empty until then.
    std::vector<uint64_t> ts_hist;
    uint32_t ts_shift = 0;
    uint64_t n_items_warp = 0, n_items_block = 0, n_items_big = 0;
    // statistics
    tripoll_graph_info info{};
    // every device array above, with the allocator that made it
    std::vector<tp::Block> blocks;

    tp::GraphDev dev() const {
        tp::GraphDev g;
        g.n = n; g.m = m; g.off = off; g.col = col; g.ts = ts; g.el = el; g.vl = vl; g.deg = deg;
        g.order = order; g.graph_of = graph_of; g.in_off = in_off; g.in_edge = in_edge;
        return g;
    }
};

namespace tp {
// survey plan limits shared by the builder and the survey kernels
constexpr uint32_t kWarpMaxQ = 64;      // entries of q's out-list a warp stages at a time
#ifndef TP_WARP_PLAN_Q
#define TP_WARP_PLAN_Q 128
#endif
constexpr uint32_t kWarpPlanQ = TP_WARP_PLAN_Q;  // middle vertices with d+(q) <= this go to the warp kernel
constexpr uint32_t kBlockChunk = 1024;  // on-chip staged entries of q's out-list per block item
constexpr uint32_t kBigChunk = 2048;    // the same for the large-table block kernel
constexpr uint32_t kWarpInEdges = 64;   // in-edges per warp item
constexpr uint32_t kBlockInEdges = 256; // in-edges a block stages at a time
constexpr uint32_t kItemInEdges = 2048; // in-edges per block item (staged kBlockInEdges at a time): the default
                                        // and the largest value the 32-bit on-chip sums allow
constexpr uint32_t kWarpPlanMax = 256;  // largest warp-item out-list the warp kernel's 32-bit sums allow
// The plan new graphs get (tripoll_set_default_plan), and the check of a plan's bounds.
tripoll_plan default_plan();
int check_plan(const tripoll_plan& p);
constexpr uint32_t kColPad = 8;         // col[] entries past m (0xFFFFFFFF) for 32-byte vector loads

// layout of one survey result record, in words (absent tables: ~0)
struct Layout {
    uint32_t o_count = ~0u, o_hist = ~0u, o_vtri = ~0u, o_etri = ~0u, o_joint = ~0u, o_maxel = ~0u,
             o_degtri = ~0u;
    uint64_t o_vlocal = ~0ull, o_elocal = ~0ull;
    uint64_t words = 0;
};
Layout make_layout(uint32_t kinds, uint32_t Lv, uint32_t Le, uint64_t n, uint64_t m);

// (Re)build g's work items under g->plan; items of an earlier plan are released.
int build_plan(tripoll_graph* g, cudaStream_t s);
// Return one of g's arrays to its allocator (stream-ordered on s) and forget it.
void drop_block(tripoll_graph* g, void* ptr, cudaStream_t s);
// Launch the survey kernels accumulating into `acc` (zeroed by the caller);
// counters: device uint32[4] of scratch.  With window_view, a window that is
// not [0, 0xFFFFFFFF] first compacts G+ to its in-window edges in pool memory
// (window_view_bytes of it); without, out-of-window edges are skipped in place.
// ev (optional, 5 events): recorded on s at the phase boundaries -- start, window
// view built, warp-item kernel done, block-item kernel done, long-list kernel done.
// multi (optional): several requests' windows surveyed at once -- lo, hi: their distinct lower and
// upper bounds, ascending, at most 64 each; [t_lo, t_hi] must be [lo[0], hi.back()]; acc holds
// lo.size() x hi.size() records of the kinds' layout (cell (i, j) at (i * hi.size() + j) * words);
// counters has 6 + lo.size() + hi.size() words.
struct MultiBounds {
    std::vector<uint32_t> lo, hi;
};
int launch_survey(const tripoll_graph* g, uint32_t kinds, uint32_t t_lo, uint32_t t_hi, uint64_t p_lo,
                  uint64_t p_hi, unsigned long long* acc, uint32_t* counters, cudaStream_t s,
                  bool window_view = true, cudaEvent_t* ev = nullptr, const MultiBounds* multi = nullptr);
// Survey `count` requests on one graph in one pass over the union of their windows (at most 64
// requests; no local-count kinds; not a batched graph).  results[k]: device or host, sized by
// tripoll_result_words(kinds[k], ...).  With window_view, the union window is compacted first.
// Asynchronous when every result is device memory (or sync_host is false: the caller orders its
// use of host results after the stream), else synchronises s.
int survey_many(const tripoll_graph* g, uint32_t count, const uint32_t* kinds, const uint32_t* t_lo,
                const uint32_t* t_hi, uint64_t* const* results, cudaStream_t s, bool window_view = true,
                bool sync_host = true);
// Device scratch survey_many takes for these requests (result records, bounds, window view).
uint64_t survey_many_bytes(const tripoll_graph* g, uint32_t count, const uint32_t* kinds, const uint32_t* t_lo,
                           const uint32_t* t_hi, bool window_view);
// Device scratch the window view of g takes for [t_lo, t_hi] (0 for the full window).
uint64_t window_view_bytes(const tripoll_graph* g, uint32_t kinds, uint32_t t_lo, uint32_t t_hi);
// Fill g->ts_hist (a few kernels over the timestamps, then a read-back; synchronises) unless it is filled
// already or g lives on another device than the current one (then window_view_bytes bounds by |E+|).
int ts_histogram(tripoll_graph* g);
// Allocate count elements of T for graph g on stream s (recorded in g->blocks).
template <class T> cudaError_t galloc(tripoll_graph* g, T** p, uint64_t count, cudaStream_t s) {
    Block b;
    b.bytes = (count ? count : 1) * sizeof(T);
    b.al = current_allocator();
    cudaError_t e = dev_alloc(&b.ptr, b.bytes, s, b.al);
    if (e != cudaSuccess) return e;
    g->blocks.push_back(b);
    *p = static_cast<T*>(b.ptr);
    return cudaSuccess;
}
// Exchange the graph's array at `graph_ptr` with the scratch buffer `s` (both stay owned).
void swap_block(tripoll_graph* g, void* graph_ptr, Scratch& s);
int check_survey_args(const tripoll_graph* g, uint32_t kinds, uint32_t t_lo, uint32_t t_hi, const void* result);
void free_graph_arrays(tripoll_graph* g);
}  // namespace tp

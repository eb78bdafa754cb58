// survey.cu -- the survey entry: result layout, work plan, window view, and
// the dispatch of a survey to the kernel instantiation its kinds need
// (survey_kernels.cuh; instantiated in survey_inst_*.cu).
#include <algorithm>
#include <map>
#include <mutex>
#include <tuple>

#include "survey_kernels.cuh"

namespace tp {
namespace sv {
#define TP_EXTERN_LAUNCH(F)                                                                               \
    extern template void launch_f<F>(const ItemLists&, const GraphDev&, const SurveyArgs&, cudaStream_t, \
                                     int, cudaEvent_t*);
TP_EXTERN_LAUNCH(0) TP_EXTERN_LAUNCH(1) TP_EXTERN_LAUNCH(2) TP_EXTERN_LAUNCH(3) TP_EXTERN_LAUNCH(4)
TP_EXTERN_LAUNCH(5) TP_EXTERN_LAUNCH(6) TP_EXTERN_LAUNCH(7) TP_EXTERN_LAUNCH(8) TP_EXTERN_LAUNCH(9)
TP_EXTERN_LAUNCH(10) TP_EXTERN_LAUNCH(11) TP_EXTERN_LAUNCH(12) TP_EXTERN_LAUNCH(13) TP_EXTERN_LAUNCH(14)
TP_EXTERN_LAUNCH(15) TP_EXTERN_LAUNCH(16) TP_EXTERN_LAUNCH(17) TP_EXTERN_LAUNCH(18) TP_EXTERN_LAUNCH(19)
TP_EXTERN_LAUNCH(20) TP_EXTERN_LAUNCH(21) TP_EXTERN_LAUNCH(22) TP_EXTERN_LAUNCH(23) TP_EXTERN_LAUNCH(24)
TP_EXTERN_LAUNCH(25) TP_EXTERN_LAUNCH(26) TP_EXTERN_LAUNCH(27) TP_EXTERN_LAUNCH(28) TP_EXTERN_LAUNCH(29)
TP_EXTERN_LAUNCH(30) TP_EXTERN_LAUNCH(31)
// several windows at once: timestamps always, any of labels, extras and the word cache
TP_EXTERN_LAUNCH(33) TP_EXTERN_LAUNCH(35) TP_EXTERN_LAUNCH(37) TP_EXTERN_LAUNCH(39) TP_EXTERN_LAUNCH(41)
TP_EXTERN_LAUNCH(43) TP_EXTERN_LAUNCH(45) TP_EXTERN_LAUNCH(47) TP_EXTERN_LAUNCH(49) TP_EXTERN_LAUNCH(51)
TP_EXTERN_LAUNCH(53) TP_EXTERN_LAUNCH(55) TP_EXTERN_LAUNCH(57) TP_EXTERN_LAUNCH(59) TP_EXTERN_LAUNCH(61)
TP_EXTERN_LAUNCH(63)
#undef TP_EXTERN_LAUNCH

// Resident blocks per SM of a kernel at a dynamic shared-memory size; cached
// per (kernel, size, device).  The kernel's dynamic shared-memory limit is
// raised once per (kernel, device) to the device's opt-in maximum, so launches
// of any size up to it stay valid whatever size was queried first.
int blocks_per_sm(const void* kernel, size_t smem) {
    static std::mutex mu;
    static std::map<std::tuple<const void*, size_t, int>, int> cache;
    static std::map<std::pair<const void*, int>, bool> raised;
    int dev = 0;
    cudaGetDevice(&dev);
    std::lock_guard<std::mutex> lk(mu);
    auto key = std::make_tuple(kernel, smem, dev);
    auto it = cache.find(key);
    if (it != cache.end()) return it->second;
    if (!raised[std::make_pair(kernel, dev)]) {
        int optin = 0;
        cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
        int static_bytes = 0;
        cudaFuncAttributes fa;
        if (cudaFuncGetAttributes(&fa, kernel) == cudaSuccess) static_bytes = (int)fa.sharedSizeBytes;
        cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, optin - static_bytes);
        raised[std::make_pair(kernel, dev)] = true;
    }
    int per = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, kernel, kBlockThreads, smem);
    per = std::max(per, 1);
    cache[key] = per;
    return per;
}

}  // namespace sv

using namespace sv;

Layout make_layout(uint32_t kinds, uint32_t Lv, uint32_t Le, uint64_t n, uint64_t m) {
    Layout L;
    uint64_t w = 0;
    if (kinds & TRIPOLL_COUNT) { L.o_count = (uint32_t)w; w += 1; }
    if (kinds & TRIPOLL_CLOSURE_HIST) { L.o_hist = (uint32_t)w; w += TRIPOLL_HIST_BINS; }
    if (kinds & TRIPOLL_VLABEL_TRIPLES) { L.o_vtri = (uint32_t)w; w += (uint64_t)Lv * Lv * Lv; }
    if (kinds & TRIPOLL_ELABEL_TRIPLES) { L.o_etri = (uint32_t)w; w += (uint64_t)Le * Le * Le; }
    if (kinds & TRIPOLL_OPEN_CLOSE_HIST) { L.o_joint = (uint32_t)w; w += TRIPOLL_HIST_BINS * TRIPOLL_HIST_BINS; }
    if (kinds & TRIPOLL_MAX_ELABEL) { L.o_maxel = (uint32_t)w; w += Le; }
    if (kinds & TRIPOLL_DEGREE_TRIPLES) {
        L.o_degtri = (uint32_t)w;
        w += (uint64_t)TRIPOLL_HIST_BINS * TRIPOLL_HIST_BINS * TRIPOLL_HIST_BINS;
    }
    if (kinds & TRIPOLL_VERTEX_LOCAL) { L.o_vlocal = w; w += n; }
    if (kinds & TRIPOLL_EDGE_LOCAL) { L.o_elocal = w; w += m; }
    L.words = w;
    return L;
}

namespace {

using namespace sv;

// ---- plan: work items per middle vertex ----------------------------------------------------

__device__ __forceinline__ uint64_t umin64(uint64_t a, uint64_t b) { return a < b ? a : b; }

// Items of middle vertex q: for each part of Adj+(q) staged at once (one part
// unless d+(q) exceeds the kernel's chunk), groups of at most `per` in-edges.
__device__ __forceinline__ void plan_shape(uint64_t dp, uint64_t di, const tripoll_plan& P, int& kind, uint64_t& chunk,
                                           uint64_t& per) {
    kind = dp <= P.warp_max_dplus ? 0 : (dp <= P.long_list_min_dplus ? 1 : 2);
    chunk = kind == 0 ? P.warp_max_dplus : (kind == 1 ? kBlockChunk : kBigChunk);
    per = kind == 0 ? kWarpInEdges : P.block_item_in_edges;
}

__global__ void plan_count_kernel(const uint64_t* __restrict__ off, const uint64_t* __restrict__ in_off, uint64_t n,
                                  tripoll_plan P, uint32_t* __restrict__ c0, uint32_t* __restrict__ c1, uint32_t* __restrict__ c2) {
    for (uint64_t q = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; q < n; q += (uint64_t)gridDim.x * blockDim.x) {
        const uint64_t dp = off[q + 1] - off[q], di = in_off[q + 1] - in_off[q];
        uint32_t cnt[3] = {0, 0, 0};
        if (dp > 0 && di > 0) {
            int kind;
            uint64_t chunk, per;
            plan_shape(dp, di, P, kind, chunk, per);
            cnt[kind] = (uint32_t)(((dp + chunk - 1) / chunk) * ((di + per - 1) / per));
        }
        c0[q] = cnt[0];
        c1[q] = cnt[1];
        c2[q] = cnt[2];
    }
}

__global__ void plan_fill_kernel(const uint64_t* __restrict__ off, const uint64_t* __restrict__ in_off, uint64_t n,
                                 tripoll_plan P, const uint32_t* __restrict__ o0, const uint32_t* __restrict__ o1,
                                 const uint32_t* __restrict__ o2, WorkItem* __restrict__ i0, WorkItem* __restrict__ i1,
                                 WorkItem* __restrict__ i2) {
    for (uint64_t q = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; q < n; q += (uint64_t)gridDim.x * blockDim.x) {
        const uint64_t dp = off[q + 1] - off[q], di = in_off[q + 1] - in_off[q];
        if (dp == 0 || di == 0) continue;
        int kind;
        uint64_t chunk, per;
        plan_shape(dp, di, P, kind, chunk, per);
        WorkItem* dst = kind == 0 ? i0 : (kind == 1 ? i1 : i2);
        uint32_t o = kind == 0 ? o0[q] : (kind == 1 ? o1[q] : o2[q]);
        const uint32_t ilo = (uint32_t)in_off[q];
        const bool chunked = dp > chunk;
        for (uint64_t c = 0; c < dp; c += chunk) {
            for (uint64_t s = 0; s < di; s += per) {
                WorkItem it;
                it.q = (uint32_t)q;
                it.qlo = (uint32_t)c;
                it.qlen = (uint32_t)umin64(chunk, dp - c);
                it.in_lo = ilo + (uint32_t)s;
                it.in_hi = ilo + (uint32_t)umin64(di, s + per);
                it.flags = chunked ? 1u : 0u;
                it.vpos = (uint32_t)(off[q] + c);
                it.pad = 0;
                dst[o++] = it;
            }
        }
    }
}

unsigned grid_n(uint64_t items) {
    uint64_t b = (items + 255) / 256;
    return (unsigned)std::max<uint64_t>(1, std::min<uint64_t>(b, 148u * 64u));
}

// ---- window view: G+ restricted to the edges in the window ----------------------------------
//
// A triangle is surveyed iff its three edges lie in the window, so the survey
// over [t_lo, t_hi] is the survey of the subgraph of in-window edges under the
// same order <+.  Compacting col/ts/el to that subgraph before the wedge
// checks removes the wedges (p,q),(p,r) whose (p,r) lies outside the window:
// with a window holding a fraction f of the edges, the checks drop from about
// f |W+| (in-place skipping of (p,q) and (q,r) only) to about f^2 |W+|.  The
// in-edge records are compacted the same way (their suffix bounds translated
// into view positions), and the warp kernel's work items are translated once,
// the items with nothing in the window left out.  One read-back of the counts
// sizes all of it.

// The window view's index, first part: per 32 CSR positions (a warp), the in-window bits (into
// vidx[w].y) and their count (the input of the scan that gives vidx[w].x).
__global__ void view_bits_kernel(const uint32_t* __restrict__ ts, uint64_t m, uint64_t words, uint32_t lo,
                                 uint32_t hi, uint2* __restrict__ vidx, uint32_t* __restrict__ cnt) {
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;  // a multiple of 32: warps stay aligned
    for (uint64_t e = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; e < words * 32; e += stride) {
        bool in = false;
        if (e < m) {
            const uint32_t t = ts[e];
            in = t >= lo && t <= hi;
        }
        const unsigned bits = __ballot_sync(0xffffffffu, in);
        if ((threadIdx.x & 31) == 0) {
            vidx[e >> 5].y = bits;
            cnt[e >> 5] = __popc(bits);
        }
    }
}

__global__ void view_prefix_kernel(const uint32_t* __restrict__ pre, uint64_t words, uint2* __restrict__ vidx) {
    for (uint64_t w = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; w < words; w += (uint64_t)gridDim.x * blockDim.x)
        vidx[w].x = pre[w];
}

__global__ void window_view_kernel(const uint32_t* __restrict__ col, const uint32_t* __restrict__ ts,
                                   const uint8_t* __restrict__ el, const uint2* __restrict__ vidx, uint64_t m,
                                   uint32_t lo, uint32_t hi, uint32_t* __restrict__ vcol, uint32_t* __restrict__ vts,
                                   uint8_t* __restrict__ vel, uint32_t* __restrict__ vorig) {
    for (uint64_t e = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; e < m; e += (uint64_t)gridDim.x * blockDim.x) {
        const uint32_t t = ts[e];
        if (t < lo || t > hi) continue;
        const uint2 w = vidx[e >> 5];
        const uint32_t p = w.x + __popc(w.y & ((1u << (e & 31u)) - 1u));
        vcol[p] = col[e];
        vts[p] = t;
        if (el) vel[p] = el[e];
        if (vorig) vorig[p] = (uint32_t)e;
    }
}

// The view's in-edges, first part: per 32 in-edge records, the in-window bits (into iidx[w].y) and
// their count (the input of the scan that gives iidx[w].x).
__global__ void in_view_bits_kernel(const InEdge* __restrict__ in_edge, uint64_t m, uint64_t words, uint32_t lo,
                                    uint32_t hi, uint2* __restrict__ iidx, uint32_t* __restrict__ cnt) {
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;  // a multiple of 32: warps stay aligned
    for (uint64_t k = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; k < words * 32; k += stride) {
        bool in = false;
        if (k < m) {
            const uint32_t t = in_edge[k].ts;
            in = t >= lo && t <= hi;
        }
        const unsigned bits = __ballot_sync(0xffffffffu, in);
        if ((threadIdx.x & 31) == 0) {
            iidx[k >> 5].y = bits;
            cnt[k >> 5] = __popc(bits);
        }
    }
}

// ... then the in-window records, in order, with e and end translated into the view's positions, and (for
// pivot ranges and the kinds that need it) the G+ position of each one's edge.
__global__ void in_view_kernel(const InEdge* __restrict__ in_edge, const uint2* __restrict__ iidx,
                               const uint2* __restrict__ vidx, uint64_t m, uint32_t lo, uint32_t hi,
                               InEdge* __restrict__ vin, uint32_t* __restrict__ vin_e) {
    for (uint64_t k = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; k < m; k += (uint64_t)gridDim.x * blockDim.x) {
        const InEdge ie = in_edge[k];
        if (ie.ts < lo || ie.ts > hi) continue;
        const uint32_t at = view_pos(iidx, (uint32_t)k);
        InEdge v;
        v.e = view_pos(vidx, ie.e);
        v.end = view_pos(vidx, ie.end);
        v.ts = ie.ts;
        v.meta = ie.meta;
        vin[at] = v;
        if (vin_e) vin_e[at] = ie.e;
    }
}

// Work items in a window view's positions: the staged part of Adj+(q) and the in-edge range translated
// through the two indexes, and keep[i] = 1 unless the item has no in-window entry or in-edge (it could
// close no triangle).
__global__ void view_items_kernel(const WorkItem* __restrict__ items, uint64_t n, const uint2* __restrict__ vidx,
                                  const uint2* __restrict__ iidx, WorkItem* __restrict__ out,
                                  uint32_t* __restrict__ keep) {
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n; i += (uint64_t)gridDim.x * blockDim.x) {
        WorkItem it = items[i];
        const uint32_t p0 = it.vpos;
        const uint32_t b0 = view_pos(vidx, p0);
        it.qlen = view_pos(vidx, p0 + it.qlen) - b0;
        it.vpos = b0;
        it.in_lo = view_pos(iidx, it.in_lo);
        it.in_hi = view_pos(iidx, it.in_hi);
        out[i] = it;
        keep[i] = (it.qlen > 0 && it.in_hi > it.in_lo) ? 1u : 0u;
    }
}

__global__ void scatter_items_kernel(const WorkItem* __restrict__ tmp, const uint32_t* __restrict__ keep,
                                     const uint32_t* __restrict__ at, uint64_t n, WorkItem* __restrict__ out) {
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n; i += (uint64_t)gridDim.x * blockDim.x)
        if (keep[i]) out[at[i]] = tmp[i];
}

uint64_t view_words(uint64_t m) { return (m >> 5) + 1; }
size_t window_scan_bytes(uint64_t m) { return prim::scan_scratch_bytes(view_words(m)); }
constexpr LaunchFn kLaunch[64] = {
    &launch_f<0>,  &launch_f<1>,  &launch_f<2>,  &launch_f<3>,  &launch_f<4>,  &launch_f<5>,  &launch_f<6>,
    &launch_f<7>,  &launch_f<8>,  &launch_f<9>,  &launch_f<10>, &launch_f<11>, &launch_f<12>, &launch_f<13>,
    &launch_f<14>, &launch_f<15>, &launch_f<16>, &launch_f<17>, &launch_f<18>, &launch_f<19>, &launch_f<20>,
    &launch_f<21>, &launch_f<22>, &launch_f<23>, &launch_f<24>, &launch_f<25>, &launch_f<26>, &launch_f<27>,
    &launch_f<28>, &launch_f<29>, &launch_f<30>, &launch_f<31>,
    // F_MULTI: only with F_TS (odd)
    nullptr, &launch_f<33>, nullptr, &launch_f<35>, nullptr, &launch_f<37>, nullptr, &launch_f<39>,
    nullptr, &launch_f<41>, nullptr, &launch_f<43>, nullptr, &launch_f<45>, nullptr, &launch_f<47>,
    nullptr, &launch_f<49>, nullptr, &launch_f<51>, nullptr, &launch_f<53>, nullptr, &launch_f<55>,
    nullptr, &launch_f<57>, nullptr, &launch_f<59>, nullptr, &launch_f<61>, nullptr, &launch_f<63>};

// ---- several requests in one pass: cell sums -------------------------------------------------
//
// rec holds A x B cell records of W words.  After these two sweeps, word w of record (x, y) is the
// sum of word w over the cells i >= x, j <= y: the tables of the request with window [L[x], H[y]].

__global__ void cells_prefix_j_kernel(unsigned long long* __restrict__ rec, uint32_t A, uint32_t B, uint64_t W) {
    for (uint64_t t = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; t < (uint64_t)A * W;
         t += (uint64_t)gridDim.x * blockDim.x) {
        const uint64_t i = t / W, w = t % W;
        unsigned long long acc = 0;
        for (uint32_t j = 0; j < B; ++j) {
            unsigned long long* p = rec + (i * B + j) * W + w;
            acc += *p;
            *p = acc;
        }
    }
}

__global__ void cells_suffix_i_kernel(unsigned long long* __restrict__ rec, uint32_t A, uint32_t B, uint64_t W) {
    for (uint64_t t = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; t < (uint64_t)B * W;
         t += (uint64_t)gridDim.x * blockDim.x) {
        const uint64_t j = t / W, w = t % W;
        unsigned long long acc = 0;
        for (uint32_t i = A; i-- > 0;) {
            unsigned long long* p = rec + ((uint64_t)i * B + j) * W + w;
            acc += *p;
            *p = acc;
        }
    }
}

// One copy per (request, table): len words from rec + src to out + dst.
struct TableCopy {
    uint64_t src, dst, len;
};

__global__ void gather_tables_kernel(const unsigned long long* __restrict__ rec, const TableCopy* __restrict__ copies,
                                     uint32_t n_copies, unsigned long long* __restrict__ out) {
    for (uint32_t c = blockIdx.x; c < n_copies; c += gridDim.x) {
        const TableCopy tc = copies[c];
        for (uint64_t k = threadIdx.x; k < tc.len; k += blockDim.x) out[tc.dst + k] = rec[tc.src + k];
    }
}

}  // namespace

int build_plan(tripoll_graph* g, cudaStream_t s) {
    const uint64_t n = g->n;
    Scratch c[3], o[3], tmp;
    for (int k = 0; k < 3; ++k) {
        TP_CUDA(c[k].alloc((n + 1) * 4, s));
        TP_CUDA(o[k].alloc((n + 1) * 4, s));
        TP_CUDA(cudaMemsetAsync(c[k].ptr, 0, (n + 1) * 4, s));
    }
    if (n)
        plan_count_kernel<<<grid_n(n), 256, 0, s>>>(g->off, g->in_off, n, g->plan, c[0].as<uint32_t>(), c[1].as<uint32_t>(),
                                                    c[2].as<uint32_t>()); ::tp::note_launch();
    TP_CUDA(cudaGetLastError());
    TP_CUDA(tmp.alloc(prim::scan_scratch_bytes(n + 1), s));
    uint32_t tot[3] = {0, 0, 0};
    int rc;
    for (int k = 0; k < 3; ++k) {
        if ((rc = prim::scan<uint32_t, false>(prim::Load<uint32_t, uint32_t>{c[k].as<uint32_t>(), n + 1},
                                              o[k].as<uint32_t>(), n + 1, tmp.ptr, s)))
            return rc;
        TP_CUDA(cudaMemcpyAsync(&tot[k], o[k].as<uint32_t>() + n, 4, cudaMemcpyDeviceToHost, s));
    }
    TP_CUDA(cudaStreamSynchronize(s));
    for (WorkItem** items : {&g->items_warp, &g->items_block, &g->items_big}) {  // an earlier plan's items
        if (*items) drop_block(g, *items, s);
        *items = nullptr;
    }
    g->n_items_warp = tot[0];
    g->n_items_block = tot[1];
    g->n_items_big = tot[2];
    TP_CUDA(galloc(g, &g->items_warp, std::max<uint64_t>(1, tot[0]), s));
    TP_CUDA(galloc(g, &g->items_block, std::max<uint64_t>(1, tot[1]), s));
    TP_CUDA(galloc(g, &g->items_big, std::max<uint64_t>(1, tot[2]), s));
    if (n)
        plan_fill_kernel<<<grid_n(n), 256, 0, s>>>(g->off, g->in_off, n, g->plan, o[0].as<uint32_t>(), o[1].as<uint32_t>(),
                                                   o[2].as<uint32_t>(), g->items_warp, g->items_block,
                                                   g->items_big); ::tp::note_launch();
    TP_CUDA(cudaGetLastError());
    return TRIPOLL_OK;
}

// Pool memory of a survey's window view: the two indexes and scan buffers by |E+|, the compacted arrays by
// the in-window edges -- bounded by the timestamp histogram when the graph has one, else by |E+|.
uint64_t window_view_bytes(const tripoll_graph* g, uint32_t kinds, uint32_t t_lo, uint32_t t_hi) {
    if ((t_lo == 0 && t_hi == 0xFFFFFFFFu) || !g->m) return 0;
    const uint64_t m = g->m;
    uint64_t mv = m;
    if (!g->ts_hist.empty()) {
        mv = 0;
        const uint64_t b0 = t_lo >> g->ts_shift, b1 = std::min<uint64_t>(t_hi >> g->ts_shift, g->ts_hist.size() - 1);
        for (uint64_t b = b0; b <= b1 && b < g->ts_hist.size(); ++b) mv += g->ts_hist[b];
    }
    const uint64_t r = 256;  // pool rounding per allocation
    const uint64_t w = view_words(m);
    uint64_t items = 0, it_max = 1;  // the translated item lists: temporaries, flags, positions, the lists
    for (uint64_t n : {g->n_items_warp}) {
        if (n) items += 2 * (n * sizeof(WorkItem) + r) + 2 * ((n + 1) * 4 + r);
        it_max = std::max(it_max, n + 1);
    }
    items += prim::scan_scratch_bytes(it_max) + r;
    return items + 2 * (w * 8 + r) + 4 * (w * 4 + r) + window_scan_bytes(m) + r + 2 * ((mv + kColPad) * 4 + r) +
           (g->el ? mv + kColPad + r : 0) + (std::max<uint64_t>(mv, 1) * sizeof(InEdge) + r) +
           (std::max<uint64_t>(mv, 1) * 4 + r) + ((kinds & TRIPOLL_EDGE_LOCAL) ? std::max<uint64_t>(mv, 1) * 4 + r : 0);
}

namespace {
constexpr uint32_t kTsBuckets = 4096;

__global__ void ts_max_kernel(const uint32_t* __restrict__ ts, uint64_t m, unsigned* __restrict__ out) {
    unsigned v = 0;
    for (uint64_t e = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; e < m; e += (uint64_t)gridDim.x * blockDim.x)
        v = max(v, ts[e]);
    for (int o = 16; o; o >>= 1) v = max(v, __shfl_xor_sync(0xffffffffu, v, o));
    if ((threadIdx.x & 31) == 0) atomicMax(out, v);
}

__global__ void ts_hist_kernel(const uint32_t* __restrict__ ts, uint64_t m, uint32_t shift,
                               unsigned long long* __restrict__ hist) {
    __shared__ uint32_t h[kTsBuckets];
    for (uint32_t i = threadIdx.x; i < kTsBuckets; i += blockDim.x) h[i] = 0;
    __syncthreads();
    for (uint64_t e = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; e < m; e += (uint64_t)gridDim.x * blockDim.x)
        atomicAdd(&h[min(ts[e] >> shift, kTsBuckets - 1)], 1u);
    __syncthreads();
    for (uint32_t i = threadIdx.x; i < kTsBuckets; i += blockDim.x)
        if (h[i]) atomicAdd(&hist[i], (unsigned long long)h[i]);
}
}  // namespace

int ts_histogram(tripoll_graph* g) {
    static std::mutex mu;
    std::lock_guard<std::mutex> lk(mu);
    if (!g->ts_hist.empty() || !g->m) return TRIPOLL_OK;
    int dev = -1;
    TP_CUDA(cudaGetDevice(&dev));
    if (dev != g->device) return TRIPOLL_OK;
    cudaStream_t s;
    TP_CUDA(cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking));
    Scratch buf;
    int rc = TRIPOLL_OK;
    unsigned tmax = 0;
    std::vector<uint64_t> h(kTsBuckets, 0);
    uint32_t shift = 0;
    do {
        cudaError_t e = buf.alloc(8 + kTsBuckets * 8, s);
        if (e == cudaSuccess) e = cudaMemsetAsync(buf.ptr, 0, 8 + kTsBuckets * 8, s);
        if (e != cudaSuccess) { rc = ::tp::cuda_fail(e, "timestamp histogram buffer"); break; }
        unsigned* mx = buf.as<unsigned>();
        unsigned long long* hist = reinterpret_cast<unsigned long long*>(buf.as<unsigned char>() + 8);
        ts_max_kernel<<<grid_n(g->m), 256, 0, s>>>(g->ts, g->m, mx); ::tp::note_launch();
        if (cudaMemcpyAsync(&tmax, mx, 4, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
            cudaStreamSynchronize(s) != cudaSuccess) { rc = fail(TRIPOLL_ERR_CUDA, "timestamp maximum"); break; }
        while (shift < 32 && (tmax >> shift) >= kTsBuckets) ++shift;  // kTsBuckets buckets cover [0, tmax]
        ts_hist_kernel<<<grid_n(g->m), 256, 0, s>>>(g->ts, g->m, shift, hist); ::tp::note_launch();
        if (cudaMemcpyAsync(h.data(), hist, kTsBuckets * 8, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
            cudaStreamSynchronize(s) != cudaSuccess) { rc = fail(TRIPOLL_ERR_CUDA, "timestamp histogram"); break; }
    } while (false);
    buf.release();
    cudaStreamSynchronize(s);
    cudaStreamDestroy(s);
    if (rc) return rc;
    g->ts_shift = shift;
    g->ts_hist.swap(h);
    return TRIPOLL_OK;
}

// Launch the survey kernels accumulating into `acc` (zeroed by the caller).
int launch_survey(const tripoll_graph* g, uint32_t kinds, uint32_t t_lo, uint32_t t_hi, uint64_t p_lo, uint64_t p_hi,
                  unsigned long long* acc, uint32_t* counters, cudaStream_t s, bool window_view, cudaEvent_t* ev,
                  const MultiBounds* multi) {
    const Layout lay = make_layout(kinds, g->Lv, g->Le, g->n, g->m);
    if (multi && (multi->lo.empty() || multi->hi.empty() || multi->lo.size() > kMultiMax ||
                  multi->hi.size() > kMultiMax || g->graph_of ||
                  (kinds & (TRIPOLL_VERTEX_LOCAL | TRIPOLL_EDGE_LOCAL))))
        return fail(TRIPOLL_ERR_INVALID_ARG, "several windows at once: 1..64 bounds, single graph, no local counts");
    SurveyArgs a;
    a.kinds = kinds;
    a.t_lo = t_lo;
    a.t_hi = t_hi;
    a.Lv = g->Lv;
    a.Le = g->Le;
    a.p_lo = p_lo;
    a.p_hi = p_hi;
    a.restricted = !(p_lo == 0 && p_hi >= g->n);
    a.e_lo = 0;
    a.e_hi = (uint32_t)g->m;
    if (a.restricted) {  // two offsets of the pivot range, read once on the host
        uint64_t ends[2] = {0, 0};
        TP_CUDA(cudaMemcpyAsync(&ends[0], g->off + p_lo, 8, cudaMemcpyDeviceToHost, s));
        TP_CUDA(cudaMemcpyAsync(&ends[1], g->off + p_hi, 8, cudaMemcpyDeviceToHost, s));
        TP_CUDA(cudaStreamSynchronize(s));
        a.e_lo = (uint32_t)ends[0];
        a.e_hi = (uint32_t)ends[1];
    }
    a.lay = lay;
    a.out = acc;
    a.counters = counters;
    // record prefix mirrored on chip: the tables that fit, never the local counts
    uint64_t sw = std::min(lay.o_vlocal, lay.o_elocal);
    if (sw == ~0ull) sw = lay.words;
    if (multi) sw = lay.words * multi->lo.size() * multi->hi.size();  // every cell's record
    if (g->graph_of) sw = 0;
    // a single record larger than the mirror: a dense prefix plus the word cache, in the same room
    const bool cache = sw > kSharedTableWords;
    a.s_words = (uint32_t)std::min<uint64_t>(sw, cache ? kCacheDenseWords : kSharedTableWords);
    {
        unsigned long kb = kBlockMoveLog2, kw = kWarpMoveLog2;
        if (const char* e = std::getenv("TRIPOLL_MIRROR_MOVE_LOG2")) {
            char* end = nullptr;
            const unsigned long v = std::strtoul(e, &end, 10);
            if (end != e) {
                kb = std::min(v, kb);
                kw = std::min(v, kw);
            }
        }
        a.move_block_log2 = (uint8_t)kb;
        a.move_warp_log2 = (uint8_t)kw;
        a.view_items = 0;
    }
    const bool window = !(t_lo == 0 && t_hi == 0xFFFFFFFFu);
    int F = 0;
    if (window || (kinds & (TRIPOLL_CLOSURE_HIST | TRIPOLL_OPEN_CLOSE_HIST))) F |= F_TS;
    if (kinds & (TRIPOLL_ELABEL_TRIPLES | TRIPOLL_MAX_ELABEL)) F |= F_EL;
    if (kinds & (TRIPOLL_VLABEL_TRIPLES | TRIPOLL_MAX_ELABEL)) F |= F_VL;
    if (kinds & (TRIPOLL_OPEN_CLOSE_HIST | TRIPOLL_MAX_ELABEL | TRIPOLL_DEGREE_TRIPLES | TRIPOLL_VERTEX_LOCAL |
                 TRIPOLL_EDGE_LOCAL))
        F |= F_EXTRA | F_TS;
    if (cache) F |= F_CACHE;
    if (multi) F |= F_MULTI | F_TS;
    int sms = 148;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, g->device);
    TP_CUDA(cudaMemsetAsync(counters, 0, 16, s));
    if (multi) {  // the bounds, read into shared memory by every block of the survey kernels
        std::vector<uint32_t> b;
        b.push_back((uint32_t)multi->lo.size());
        b.push_back((uint32_t)multi->hi.size());
        b.insert(b.end(), multi->lo.begin(), multi->lo.end());
        b.insert(b.end(), multi->hi.begin(), multi->hi.end());
        TP_CUDA(cudaMemcpyAsync(counters + 4, b.data(), b.size() * 4, cudaMemcpyHostToDevice, s));
    }
    mark(ev, 0, s);
    GraphDev gd = g->dev();
    // released (stream-ordered) after the kernels
    Scratch vx, vcnt, vpre, vcol, vts, vel, vorig, vtmp, ix, icnt, ipre, vin, vine, iscan, ilist[3];
    ItemLists L = {{g->items_warp, g->items_block, g->items_big}, {g->n_items_warp, g->n_items_block, g->n_items_big}};
    if (window && window_view && g->m) {
        const uint64_t m = g->m, words = view_words(m);
        TP_CUDA(vx.alloc(words * 8, s));
        TP_CUDA(vcnt.alloc(words * 4, s));
        TP_CUDA(vpre.alloc(words * 4, s));
        TP_CUDA(vtmp.alloc(window_scan_bytes(m), s));
        view_bits_kernel<<<grid_n(words * 32), 256, 0, s>>>(g->ts, m, words, t_lo, t_hi, vx.as<uint2>(),
                                                            vcnt.as<uint32_t>()); ::tp::note_launch();
        int rc;
        if ((rc = prim::scan<uint32_t, false>(prim::Load<uint32_t, uint32_t>{vcnt.as<uint32_t>(), words},
                                              vpre.as<uint32_t>(), words, vtmp.ptr, s)))
            return rc;
        view_prefix_kernel<<<grid_n(words), 256, 0, s>>>(vpre.as<uint32_t>(), words, vx.as<uint2>()); ::tp::note_launch();
        // the in-window in-edge records' index, with counts and prefixes of its own (vcnt and vpre keep
        // the edges' for the read-back below)
        TP_CUDA(ix.alloc(words * 8, s));
        TP_CUDA(icnt.alloc(words * 4, s));
        TP_CUDA(ipre.alloc(words * 4, s));
        in_view_bits_kernel<<<grid_n(words * 32), 256, 0, s>>>(g->in_edge, m, words, t_lo, t_hi, ix.as<uint2>(),
                                                               icnt.as<uint32_t>()); ::tp::note_launch();
        if ((rc = prim::scan<uint32_t, false>(prim::Load<uint32_t, uint32_t>{icnt.as<uint32_t>(), words},
                                              ipre.as<uint32_t>(), words, vtmp.ptr, s)))
            return rc;
        view_prefix_kernel<<<grid_n(words), 256, 0, s>>>(ipre.as<uint32_t>(), words, ix.as<uint2>()); ::tp::note_launch();
        // the warp kernel's work items in view positions, the empty ones marked for leaving out (the block
        // kernels translate their few large items themselves)
        const uint64_t n_it[3] = {g->n_items_warp, 0, 0};
        const WorkItem* its[3] = {g->items_warp, g->items_block, g->items_big};
        Scratch itmp[3], ikeep[3], iat[3];
        uint64_t it_max = 1;
        for (int k = 0; k < 3; ++k) it_max = std::max(it_max, n_it[k] + 1);
        TP_CUDA(iscan.alloc(prim::scan_scratch_bytes(it_max), s));
        for (int k = 0; k < 3; ++k) {
            if (!n_it[k]) continue;
            TP_CUDA(itmp[k].alloc(n_it[k] * sizeof(WorkItem), s));
            TP_CUDA(ikeep[k].alloc((n_it[k] + 1) * 4, s));
            TP_CUDA(iat[k].alloc((n_it[k] + 1) * 4, s));
            TP_CUDA(cudaMemsetAsync(ikeep[k].as<uint32_t>() + n_it[k], 0, 4, s));
            view_items_kernel<<<grid_n(n_it[k]), 256, 0, s>>>(its[k], n_it[k], vx.as<uint2>(), ix.as<uint2>(),
                                                              itmp[k].as<WorkItem>(), ikeep[k].as<uint32_t>()); ::tp::note_launch();
            if ((rc = prim::scan<uint32_t, false>(prim::Load<uint32_t, uint32_t>{ikeep[k].as<uint32_t>(), n_it[k] + 1},
                                                  iat[k].as<uint32_t>(), n_it[k] + 1, iscan.ptr, s)))
                return rc;
        }
        // one read-back sizes the view (the in-window edges: the last word's prefix and count; the same edges
        // are the in-window in-edges) and the item lists that are left
        uint32_t back[5] = {0, 0, 0, 0, 0};
        TP_CUDA(cudaMemcpyAsync(&back[0], vpre.as<uint32_t>() + words - 1, 4, cudaMemcpyDeviceToHost, s));
        TP_CUDA(cudaMemcpyAsync(&back[1], vcnt.as<uint32_t>() + words - 1, 4, cudaMemcpyDeviceToHost, s));
        for (int k = 0; k < 3; ++k)
            if (n_it[k]) TP_CUDA(cudaMemcpyAsync(&back[2 + k], iat[k].as<uint32_t>() + n_it[k], 4, cudaMemcpyDeviceToHost, s));
        TP_CUDA(cudaStreamSynchronize(s));
        const uint64_t mv = (uint64_t)back[0] + back[1];
        TP_CUDA(vcol.alloc((mv + kColPad) * 4, s));
        TP_CUDA(vts.alloc((mv + kColPad) * 4, s));
        if (g->el) TP_CUDA(vel.alloc(mv + kColPad, s));
        if (kinds & TRIPOLL_EDGE_LOCAL) TP_CUDA(vorig.alloc(std::max<uint64_t>(mv, 1) * 4, s));
        window_view_kernel<<<grid_n(m), 256, 0, s>>>(g->col, g->ts, g->el, vx.as<uint2>(), m, t_lo, t_hi,
                                                     vcol.as<uint32_t>(), vts.as<uint32_t>(),
                                                     g->el ? vel.as<uint8_t>() : nullptr,
                                                     vorig.as<uint32_t>()); ::tp::note_launch();
        TP_CUDA(cudaGetLastError());
        TP_CUDA(vin.alloc(std::max<uint64_t>(mv, 1) * sizeof(InEdge), s));
        const bool need_e = a.restricted || (F & F_EXTRA);  // the kernels read vin_e only then
        if (need_e) TP_CUDA(vine.alloc(std::max<uint64_t>(mv, 1) * 4, s));
        in_view_kernel<<<grid_n(m), 256, 0, s>>>(g->in_edge, ix.as<uint2>(), vx.as<uint2>(), m, t_lo, t_hi,
                                                 vin.as<InEdge>(), need_e ? vine.as<uint32_t>() : nullptr); ::tp::note_launch();
        for (int k = 0; k < 3; ++k) {
            if (!n_it[k]) continue;
            L.items[k] = nullptr;
            L.n[k] = back[2 + k];
            if (!L.n[k]) continue;
            TP_CUDA(ilist[k].alloc(L.n[k] * sizeof(WorkItem), s));
            scatter_items_kernel<<<grid_n(n_it[k]), 256, 0, s>>>(itmp[k].as<WorkItem>(), ikeep[k].as<uint32_t>(),
                                                                 iat[k].as<uint32_t>(), n_it[k],
                                                                 ilist[k].as<WorkItem>()); ::tp::note_launch();
            L.items[k] = ilist[k].as<WorkItem>();
        }
        TP_CUDA(cudaGetLastError());
        a.view_items = 1;
        gd.col = vcol.as<uint32_t>();
        gd.ts = vts.as<uint32_t>();
        gd.el = g->el ? vel.as<uint8_t>() : nullptr;
        gd.vidx = vx.as<uint2>();
        gd.vorig = vorig.as<uint32_t>();
        gd.in_edge = vin.as<InEdge>();
        gd.iidx = ix.as<uint2>();
        gd.vin_e = need_e ? vine.as<uint32_t>() : nullptr;
    }
    kLaunch[F](L, gd, a, s, sms, ev);
    TP_CUDA(cudaGetLastError());
    return TRIPOLL_OK;
}

// ---- several requests on one graph in one pass ----------------------------------------------

namespace {

// Tables of a layout present in `kinds`, as (offset, length) in words, in layout order.
void tables_of(uint32_t kinds, const Layout& L, uint32_t Lv, uint32_t Le, std::vector<std::pair<uint64_t, uint64_t>>* out) {
    const uint64_t H = TRIPOLL_HIST_BINS;
    if (kinds & TRIPOLL_COUNT) out->push_back({L.o_count, 1});
    if (kinds & TRIPOLL_CLOSURE_HIST) out->push_back({L.o_hist, H});
    if (kinds & TRIPOLL_VLABEL_TRIPLES) out->push_back({L.o_vtri, (uint64_t)Lv * Lv * Lv});
    if (kinds & TRIPOLL_ELABEL_TRIPLES) out->push_back({L.o_etri, (uint64_t)Le * Le * Le});
    if (kinds & TRIPOLL_OPEN_CLOSE_HIST) out->push_back({L.o_joint, H * H});
    if (kinds & TRIPOLL_MAX_ELABEL) out->push_back({L.o_maxel, Le});
    if (kinds & TRIPOLL_DEGREE_TRIPLES) out->push_back({L.o_degtri, H * H * H});
}

struct ManyPlan {
    uint32_t kinds = 0;  // union
    Layout lay;          // of the union
    MultiBounds b;
    std::vector<uint32_t> x, y;  // per request: index of its bounds
    uint64_t cells = 0, rec_words = 0, out_words = 0;
};

int plan_many(const tripoll_graph* g, uint32_t count, const uint32_t* kinds, const uint32_t* t_lo,
              const uint32_t* t_hi, ManyPlan* P) {
    if (!g || count == 0 || !kinds || !t_lo || !t_hi) return fail(TRIPOLL_ERR_INVALID_ARG, "bad request list");
    if (count > kMultiMax) return fail(TRIPOLL_ERR_INVALID_ARG, "at most 64 requests in one pass");
    if (g->graph_of) return fail(TRIPOLL_ERR_INVALID_ARG, "several requests at once need a single graph");
    for (uint32_t k = 0; k < count; ++k) {
        int rc = check_survey_args(g, kinds[k], t_lo[k], t_hi[k], kinds);  // (result pointers checked by the caller)
        if (rc) return rc;
        if (kinds[k] & (TRIPOLL_VERTEX_LOCAL | TRIPOLL_EDGE_LOCAL))
            return fail(TRIPOLL_ERR_INVALID_ARG, "local counts are surveyed one request at a time");
        P->kinds |= kinds[k];
        P->b.lo.push_back(t_lo[k]);
        P->b.hi.push_back(t_hi[k]);
        P->out_words += make_layout(kinds[k], g->Lv, g->Le, g->n, g->m).words;
    }
    for (auto* v : {&P->b.lo, &P->b.hi}) {
        std::sort(v->begin(), v->end());
        v->erase(std::unique(v->begin(), v->end()), v->end());
    }
    for (uint32_t k = 0; k < count; ++k) {
        P->x.push_back((uint32_t)(std::lower_bound(P->b.lo.begin(), P->b.lo.end(), t_lo[k]) - P->b.lo.begin()));
        P->y.push_back((uint32_t)(std::lower_bound(P->b.hi.begin(), P->b.hi.end(), t_hi[k]) - P->b.hi.begin()));
    }
    P->lay = make_layout(P->kinds, g->Lv, g->Le, g->n, g->m);
    P->cells = (uint64_t)P->b.lo.size() * P->b.hi.size();
    P->rec_words = P->cells * P->lay.words;
    if (P->rec_words >= (1ull << 31))
        return fail(TRIPOLL_ERR_NO_MEMORY, "too many windows x table words for one pass; split the requests");
    return TRIPOLL_OK;
}

uint64_t many_scratch_bytes(const tripoll_graph* g, const ManyPlan& P, bool window_view) {
    const uint64_t r = 256;
    return (P.rec_words * 8 + r) + ((6 + P.b.lo.size() + P.b.hi.size()) * 4 + r) + (P.out_words * 8 + r) +
           (P.x.size() * 8 * sizeof(TableCopy) + r) +
           (window_view ? window_view_bytes(g, P.kinds, P.b.lo.front(), P.b.hi.back()) : 0);
}

}  // namespace

uint64_t survey_many_bytes(const tripoll_graph* g, uint32_t count, const uint32_t* kinds, const uint32_t* t_lo,
                           const uint32_t* t_hi, bool window_view) {
    ManyPlan P;
    if (plan_many(g, count, kinds, t_lo, t_hi, &P)) return ~0ull;
    return many_scratch_bytes(g, P, window_view);
}

int survey_many(const tripoll_graph* g, uint32_t count, const uint32_t* kinds, const uint32_t* t_lo,
                const uint32_t* t_hi, uint64_t* const* results, cudaStream_t s, bool window_view, bool sync_host) {
    ManyPlan P;
    int rc = plan_many(g, count, kinds, t_lo, t_hi, &P);
    if (rc) return rc;
    if (!results) return fail(TRIPOLL_ERR_INVALID_ARG, "results is NULL");
    for (uint32_t k = 0; k < count; ++k)
        if (!results[k]) return fail(TRIPOLL_ERR_INVALID_ARG, "a result pointer is NULL");
    const uint32_t A = (uint32_t)P.b.lo.size(), B = (uint32_t)P.b.hi.size();
    const uint64_t W = P.lay.words;
    // copies of each request's tables out of its cell-sum record, into one packed output
    std::vector<TableCopy> copies;
    std::vector<uint64_t> out_off(count + 1, 0);
    for (uint32_t k = 0; k < count; ++k) {
        const Layout Lk = make_layout(kinds[k], g->Lv, g->Le, g->n, g->m);
        std::vector<std::pair<uint64_t, uint64_t>> tu, tk;
        tables_of(kinds[k], P.lay, g->Lv, g->Le, &tu);
        tables_of(kinds[k], Lk, g->Lv, g->Le, &tk);
        const uint64_t base = ((uint64_t)P.x[k] * B + P.y[k]) * W;
        for (size_t t = 0; t < tu.size(); ++t) copies.push_back({base + tu[t].first, out_off[k] + tk[t].first, tu[t].second});
        out_off[k + 1] = out_off[k] + Lk.words;
    }
    Scratch rec, ctr, outs, cps;
    TP_CUDA(rec.alloc(P.rec_words * 8, s));
    TP_CUDA(ctr.alloc((6 + A + B) * 4, s));
    TP_CUDA(outs.alloc(out_off[count] * 8, s));
    TP_CUDA(cps.alloc(copies.size() * sizeof(TableCopy), s));
    TP_CUDA(cudaMemsetAsync(rec.ptr, 0, P.rec_words * 8, s));
    TP_CUDA(cudaMemcpyAsync(cps.ptr, copies.data(), copies.size() * sizeof(TableCopy), cudaMemcpyHostToDevice, s));
    if (g->n && (rc = launch_survey(g, P.kinds, P.b.lo.front(), P.b.hi.back(), 0, g->n, rec.as<unsigned long long>(),
                                    ctr.as<uint32_t>(), s, window_view, nullptr, &P.b)))
        return rc;
    const unsigned grid_a = (unsigned)std::max<uint64_t>(1, std::min<uint64_t>((A * W + 255) / 256, 148u * 16u));
    const unsigned grid_b = (unsigned)std::max<uint64_t>(1, std::min<uint64_t>((B * W + 255) / 256, 148u * 16u));
    cells_prefix_j_kernel<<<grid_a, 256, 0, s>>>(rec.as<unsigned long long>(), A, B, W); note_launch();
    cells_suffix_i_kernel<<<grid_b, 256, 0, s>>>(rec.as<unsigned long long>(), A, B, W); note_launch();
    gather_tables_kernel<<<(unsigned)std::min<size_t>(copies.size(), 148u * 8u), 256, 0, s>>>(
        rec.as<unsigned long long>(), cps.as<TableCopy>(), (uint32_t)copies.size(), outs.as<unsigned long long>());
    note_launch();
    TP_CUDA(cudaGetLastError());
    bool host = false;
    for (uint32_t k = 0; k < count; ++k) {
        TP_CUDA(cudaMemcpyAsync(results[k], outs.as<unsigned long long>() + out_off[k], (out_off[k + 1] - out_off[k]) * 8,
                                cudaMemcpyDefault, s));
        host = host || !is_device_pointer(results[k]);
    }
    if (host && sync_host) TP_CUDA(cudaStreamSynchronize(s));
    return TRIPOLL_OK;
}

}  // namespace tp

extern "C" int tripoll_survey_many(tripoll_graph_t g, uint32_t count, const uint32_t* kind_masks, const uint32_t* t_lo,
                                   const uint32_t* t_hi, uint64_t* const* results, void* cuda_stream) {
    return tp::survey_many(g, count, kind_masks, t_lo, t_hi, results, (cudaStream_t)cuda_stream,
                           !g || g->plan.window_view != 0);
}

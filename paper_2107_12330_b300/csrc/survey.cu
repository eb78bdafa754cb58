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
    extern template void launch_f<F>(const tripoll_graph*, const GraphDev&, const SurveyArgs&, cudaStream_t, \
                                     int, cudaEvent_t*);
TP_EXTERN_LAUNCH(0) TP_EXTERN_LAUNCH(1) TP_EXTERN_LAUNCH(2) TP_EXTERN_LAUNCH(3) TP_EXTERN_LAUNCH(4)
TP_EXTERN_LAUNCH(5) TP_EXTERN_LAUNCH(6) TP_EXTERN_LAUNCH(7) TP_EXTERN_LAUNCH(8) TP_EXTERN_LAUNCH(9)
TP_EXTERN_LAUNCH(10) TP_EXTERN_LAUNCH(11) TP_EXTERN_LAUNCH(12) TP_EXTERN_LAUNCH(13) TP_EXTERN_LAUNCH(14)
TP_EXTERN_LAUNCH(15) TP_EXTERN_LAUNCH(16) TP_EXTERN_LAUNCH(17) TP_EXTERN_LAUNCH(18) TP_EXTERN_LAUNCH(19)
TP_EXTERN_LAUNCH(20) TP_EXTERN_LAUNCH(21) TP_EXTERN_LAUNCH(22) TP_EXTERN_LAUNCH(23) TP_EXTERN_LAUNCH(24)
TP_EXTERN_LAUNCH(25) TP_EXTERN_LAUNCH(26) TP_EXTERN_LAUNCH(27) TP_EXTERN_LAUNCH(28) TP_EXTERN_LAUNCH(29)
TP_EXTERN_LAUNCH(30) TP_EXTERN_LAUNCH(31)
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
__device__ __forceinline__ void plan_shape(uint64_t dp, uint64_t di, int& kind, uint64_t& chunk, uint64_t& per) {
    kind = dp <= kWarpPlanQ ? 0 : (dp <= 4 * kBlockChunk ? 1 : 2);
    chunk = kind == 0 ? kWarpPlanQ : (kind == 1 ? kBlockChunk : kBigChunk);
    per = kind == 0 ? kWarpInEdges : kItemInEdges;
}

__global__ void plan_count_kernel(const uint64_t* __restrict__ off, const uint64_t* __restrict__ in_off, uint64_t n,
                                  uint32_t* __restrict__ c0, uint32_t* __restrict__ c1, uint32_t* __restrict__ c2) {
    for (uint64_t q = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; q < n; q += (uint64_t)gridDim.x * blockDim.x) {
        const uint64_t dp = off[q + 1] - off[q], di = in_off[q + 1] - in_off[q];
        uint32_t cnt[3] = {0, 0, 0};
        if (dp > 0 && di > 0) {
            int kind;
            uint64_t chunk, per;
            plan_shape(dp, di, kind, chunk, per);
            cnt[kind] = (uint32_t)(((dp + chunk - 1) / chunk) * ((di + per - 1) / per));
        }
        c0[q] = cnt[0];
        c1[q] = cnt[1];
        c2[q] = cnt[2];
    }
}

__global__ void plan_fill_kernel(const uint64_t* __restrict__ off, const uint64_t* __restrict__ in_off, uint64_t n,
                                 const uint32_t* __restrict__ o0, const uint32_t* __restrict__ o1,
                                 const uint32_t* __restrict__ o2, WorkItem* __restrict__ i0, WorkItem* __restrict__ i1,
                                 WorkItem* __restrict__ i2) {
    for (uint64_t q = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; q < n; q += (uint64_t)gridDim.x * blockDim.x) {
        const uint64_t dp = off[q + 1] - off[q], di = in_off[q + 1] - in_off[q];
        if (dp == 0 || di == 0) continue;
        int kind;
        uint64_t chunk, per;
        plan_shape(dp, di, kind, chunk, per);
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
                it.pad0 = it.pad1 = 0;
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
// f |W+| (in-place skipping of (p,q) and (q,r) only) to about f^2 |W+|.

// 1 for CSR positions e < m whose timestamp lies in the window, 0 for e = m.
struct InWindow {
    const uint32_t* ts;
    uint64_t m;
    uint32_t lo, hi;
    __host__ __device__ uint32_t operator()(uint64_t e) const {
        return (e < m && ts[e] >= lo && ts[e] <= hi) ? 1u : 0u;
    }
};

__global__ void window_view_kernel(const uint32_t* __restrict__ col, const uint32_t* __restrict__ ts,
                                   const uint8_t* __restrict__ el, const uint32_t* __restrict__ newpos, uint64_t m,
                                   uint32_t lo, uint32_t hi, uint32_t* __restrict__ vcol, uint32_t* __restrict__ vts,
                                   uint8_t* __restrict__ vel, uint32_t* __restrict__ vorig) {
    for (uint64_t e = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; e < m; e += (uint64_t)gridDim.x * blockDim.x) {
        const uint32_t t = ts[e];
        if (t < lo || t > hi) continue;
        const uint32_t p = newpos[e];
        vcol[p] = col[e];
        vts[p] = t;
        if (el) vel[p] = el[e];
        if (vorig) vorig[p] = (uint32_t)e;
    }
}

size_t window_scan_bytes(uint64_t m) { return prim::scan_scratch_bytes(m + 1); }
constexpr LaunchFn kLaunch[32] = {
    &launch_f<0>,  &launch_f<1>,  &launch_f<2>,  &launch_f<3>,  &launch_f<4>,  &launch_f<5>,  &launch_f<6>,
    &launch_f<7>,  &launch_f<8>,  &launch_f<9>,  &launch_f<10>, &launch_f<11>, &launch_f<12>, &launch_f<13>,
    &launch_f<14>, &launch_f<15>, &launch_f<16>, &launch_f<17>, &launch_f<18>, &launch_f<19>, &launch_f<20>,
    &launch_f<21>, &launch_f<22>, &launch_f<23>, &launch_f<24>, &launch_f<25>, &launch_f<26>, &launch_f<27>,
    &launch_f<28>, &launch_f<29>, &launch_f<30>, &launch_f<31>};

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
        plan_count_kernel<<<grid_n(n), 256, 0, s>>>(g->off, g->in_off, n, c[0].as<uint32_t>(), c[1].as<uint32_t>(),
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
    g->n_items_warp = tot[0];
    g->n_items_block = tot[1];
    g->n_items_big = tot[2];
    TP_CUDA(galloc(g, &g->items_warp, std::max<uint64_t>(1, tot[0]), s));
    TP_CUDA(galloc(g, &g->items_block, std::max<uint64_t>(1, tot[1]), s));
    TP_CUDA(galloc(g, &g->items_big, std::max<uint64_t>(1, tot[2]), s));
    if (n)
        plan_fill_kernel<<<grid_n(n), 256, 0, s>>>(g->off, g->in_off, n, o[0].as<uint32_t>(), o[1].as<uint32_t>(),
                                                   o[2].as<uint32_t>(), g->items_warp, g->items_block,
                                                   g->items_big); ::tp::note_launch();
    TP_CUDA(cudaGetLastError());
    return TRIPOLL_OK;
}

uint64_t window_view_bytes(const tripoll_graph* g, uint32_t kinds, uint32_t t_lo, uint32_t t_hi) {
    if ((t_lo == 0 && t_hi == 0xFFFFFFFFu) || !g->m) return 0;
    const uint64_t m = g->m;
    const uint64_t r = 256;  // pool rounding per allocation
    return (m + 1) * 4 + r + 2 * ((m + kColPad) * 4 + r) + (g->el ? m + kColPad + r : 0) +
           ((kinds & TRIPOLL_EDGE_LOCAL) ? m * 4 + r : 0) + window_scan_bytes(m) + r;
}

// Launch the survey kernels accumulating into `acc` (zeroed by the caller).
int launch_survey(const tripoll_graph* g, uint32_t kinds, uint32_t t_lo, uint32_t t_hi, uint64_t p_lo, uint64_t p_hi,
                  unsigned long long* acc, uint32_t* counters, cudaStream_t s, bool window_view, cudaEvent_t* ev) {
    const Layout lay = make_layout(kinds, g->Lv, g->Le, g->n, g->m);
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
    int sms = 148;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, g->device);
    TP_CUDA(cudaMemsetAsync(counters, 0, 16, s));
    mark(ev, 0, s);
    GraphDev gd = g->dev();
    Scratch vpos, vcol, vts, vel, vorig, vtmp;  // released (stream-ordered) after the survey kernels
    if (window && window_view && g->m) {
        const uint64_t m = g->m;
        TP_CUDA(vpos.alloc((m + 1) * 4, s));
        TP_CUDA(vcol.alloc((m + kColPad) * 4, s));
        TP_CUDA(vts.alloc((m + kColPad) * 4, s));
        if (g->el) TP_CUDA(vel.alloc(m + kColPad, s));
        if (kinds & TRIPOLL_EDGE_LOCAL) TP_CUDA(vorig.alloc(m * 4, s));
        TP_CUDA(vtmp.alloc(window_scan_bytes(m), s));
        int rc;
        if ((rc = prim::scan<uint32_t, false>(InWindow{g->ts, m, t_lo, t_hi}, vpos.as<uint32_t>(), m + 1, vtmp.ptr, s)))
            return rc;
        window_view_kernel<<<grid_n(m), 256, 0, s>>>(g->col, g->ts, g->el, vpos.as<uint32_t>(), m, t_lo, t_hi,
                                                     vcol.as<uint32_t>(), vts.as<uint32_t>(),
                                                     g->el ? vel.as<uint8_t>() : nullptr,
                                                     vorig.as<uint32_t>()); ::tp::note_launch();
        TP_CUDA(cudaGetLastError());
        gd.col = vcol.as<uint32_t>();
        gd.ts = vts.as<uint32_t>();
        gd.el = g->el ? vel.as<uint8_t>() : nullptr;
        gd.newpos = vpos.as<uint32_t>();
        gd.vorig = vorig.as<uint32_t>();
    }
    kLaunch[F](g, gd, a, s, sms, ev);
    TP_CUDA(cudaGetLastError());
    return TRIPOLL_OK;
}

}  // namespace tp

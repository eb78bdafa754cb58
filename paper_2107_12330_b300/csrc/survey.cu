// survey.cu -- wedge checks and the survey fold (TriPoll Sec. 4.3-4.5, Alg. 1-4).
//
// Every triangle p <+ q <+ r of G+ is found exactly once as r in
// Adj+(p) ∩ Adj+(q) with r after q in Adj+(p) (Alg. 1).  The kernels here
// organise that intersection around the middle vertex q, the single-GPU form
// of the paper's pull phase (Sec. 4.4): the out-list of q, with the metadata
// of its edges (q,r) and the labels of the r, is staged once in shared memory
// as an open-addressing hash table, and then every in-edge (p,q) streams the
// suffix of Adj+(p) after q from HBM and probes each candidate r against it
// -- one probe per wedge (p,q,r), the wedge check of Sec. 3.  A hit is a
// triangle; its six metadata items (Sec. 3) are the (p,q) edge's (read once
// per in-edge), the (p,r) edge's (gathered at the hit position), and the
// (q,r) edge's plus vertex r's (from shared memory).
//
// Two kernels split the middle vertices by |Adj+(q)|: a warp-per-item kernel
// for short out-lists (each warp its own table) and a block-per-item kernel
// for long ones (tables of up to kBlockChunk entries; longer out-lists are cut
// into chunks and each in-edge's suffix is restricted to the chunk's value
// range).  Items carry at most a fixed number of in-edges so that dynamic
// scheduling (one atomic per item) keeps all SMs busy to the end.
//
// The fold aggregates hits inside a warp with __match_any_sync, then in
// shared memory, then with 64-bit global atomics once per block -- integer
// adds commute, so the result is exact and schedule-independent.
#include <cub/cub.cuh>

#include <algorithm>

#include "common.cuh"

namespace tp {

Layout make_layout(uint32_t kinds, uint32_t Lv, uint32_t Le, uint64_t n) {
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
    L.words = w;
    return L;
}

namespace {

constexpr uint32_t kEmpty = 0xFFFFFFFFu;
constexpr int kBlockThreads = 256;
constexpr int kWarps = kBlockThreads / 32;
constexpr uint32_t kSharedTableWords = 4096;  // on-chip mirror of the record prefix (32 KB)

// feature bits of a kernel instantiation
constexpr int F_TS = 1;     // timestamps (window or time kinds)
constexpr int F_EL = 2;     // edge labels
constexpr int F_VL = 4;     // vertex labels
constexpr int F_EXTRA = 8;  // joint table, max label, degree triples, local counts

struct SurveyArgs {
    uint32_t kinds;
    uint32_t t_lo, t_hi;
    uint32_t Lv, Le;
    uint32_t s_words;         // record words mirrored in shared memory (0 for batched graphs)
    uint64_t p_lo, p_hi;      // pivot range
    Layout lay;
    unsigned long long* out;  // accumulator: one record, or num_graphs records (batched)
    uint32_t* counters;       // [2] item counters of the two kernels
};

__device__ __forceinline__ uint32_t hash_slot(uint32_t r, int lg) {
    return (r * 2654435761u) >> (32 - lg);
}

// ceil(log2(d)) for d >= 2, and 0 for d in {0, 1}: the closing/opening-time bin (Alg. 4)
__device__ __forceinline__ uint32_t time_bin(uint32_t d) { return d <= 1u ? 0u : 32u - __clz(d - 1u); }

__device__ __forceinline__ void sort3(uint32_t& a, uint32_t& b, uint32_t& c) {
    uint32_t x = min(a, b), y = max(a, b);
    a = x; b = y;
    x = min(b, c); y = max(b, c);
    b = x; c = y;
    x = min(a, b); y = max(a, b);
    a = x; b = y;
}

// Add `amount` to word `w` of the record: shared mirror when w < s_words, else global.
__device__ __forceinline__ void rec_add(unsigned long long* s_tab, uint32_t s_words, unsigned long long* grec,
                                        uint64_t w, unsigned long long amount) {
    if (w < s_words) atomicAdd(&s_tab[w], amount);
    else atomicAdd(&grec[w], amount);
}

// Warp-aggregated increment of word `w` for the lanes in `mask` (the calling lanes).
__device__ __forceinline__ void warp_add(unsigned mask, unsigned long long* s_tab, uint32_t s_words,
                                         unsigned long long* grec, uint64_t w) {
    unsigned grp = __match_any_sync(mask, w);
    int leader = __ffs(grp) - 1;
    if ((int)(threadIdx.x & 31) == leader) rec_add(s_tab, s_words, grec, w, (unsigned long long)__popc(grp));
}

struct TriMeta {
    uint32_t t_pq, t_pr, t_qr;
    uint32_t e_pq, e_pr, e_qr;  // edge labels
    uint32_t l_p, l_q, l_r;     // vertex labels
    uint32_t d_p, d_q, d_r;     // degrees (F_EXTRA)
    uint32_t p, q, r;           // positions (F_EXTRA local counts)
};

// Fold the lanes with `keep` set (called by the whole warp).
template <int F>
__device__ __forceinline__ void fold_warp(bool keep, const TriMeta& t, const SurveyArgs& a, unsigned long long* s_tab,
                                          unsigned long long* grec, unsigned long long& cnt,
                                          const uint32_t* __restrict__ order) {
    const unsigned km = __ballot_sync(0xffffffffu, keep);
    if (!km) return;
    if (!keep) return;
    cnt += 1;
    const Layout& L = a.lay;
    uint32_t t1 = t.t_pq, t2 = t.t_pr, t3 = t.t_qr;
    if (F & F_TS) sort3(t1, t2, t3);
    if (L.o_hist != ~0u) warp_add(km, s_tab, a.s_words, grec, L.o_hist + time_bin(t3 - t1));
    if ((F & F_VL) && L.o_vtri != ~0u) {
        uint32_t x = t.l_p, y = t.l_q, z = t.l_r;
        sort3(x, y, z);
        warp_add(km, s_tab, a.s_words, grec, L.o_vtri + (x * a.Lv + y) * a.Lv + z);
    }
    if ((F & F_EL) && L.o_etri != ~0u) {
        uint32_t x = t.e_pq, y = t.e_pr, z = t.e_qr;
        sort3(x, y, z);
        warp_add(km, s_tab, a.s_words, grec, L.o_etri + (x * a.Le + y) * a.Le + z);
    }
    if (F & F_EXTRA) {
        if (L.o_joint != ~0u)
            rec_add(s_tab, a.s_words, grec, L.o_joint + time_bin(t2 - t1) * TRIPOLL_HIST_BINS + time_bin(t3 - t1), 1);
        if (L.o_maxel != ~0u && t.l_p != t.l_q && t.l_q != t.l_r && t.l_p != t.l_r)
            rec_add(s_tab, a.s_words, grec, L.o_maxel + max(t.e_pq, max(t.e_pr, t.e_qr)), 1);
        if (L.o_degtri != ~0u) {
            uint32_t x = time_bin(t.d_p), y = time_bin(t.d_q), z = time_bin(t.d_r);
            sort3(x, y, z);
            rec_add(s_tab, a.s_words, grec,
                    L.o_degtri + (x * TRIPOLL_HIST_BINS + y) * TRIPOLL_HIST_BINS + z, 1);
        }
        if (L.o_vlocal != ~0ull) {
            atomicAdd(&grec[L.o_vlocal + order[t.p]], 1ull);
            atomicAdd(&grec[L.o_vlocal + order[t.q]], 1ull);
            atomicAdd(&grec[L.o_vlocal + order[t.r]], 1ull);
        }
    }
}

__device__ __forceinline__ bool in_window(uint32_t t, uint32_t lo, uint32_t hi) { return t >= lo && t <= hi; }

// One warp scans the suffix [j0, end) of Adj+(p) against the staged table of q.
// Values outside [vlo, vhi] are skipped (chunked tables); the suffix is sorted.
template <int F>
__device__ __forceinline__ void scan_suffix(const GraphDev& g, const SurveyArgs& a, uint32_t e_pq, uint32_t j0,
                                            uint32_t end, uint32_t p, uint32_t q, uint32_t l_q, uint32_t d_q,
                                            uint32_t vhi, const uint32_t* s_key, const uint16_t* s_pos16,
                                            const uint8_t* s_pos8, int lg, const uint32_t* s_ts,
                                            const uint8_t* s_el, const uint8_t* s_vl, const uint32_t* s_deg,
                                            unsigned long long* s_tab, unsigned long long* grec,
                                            unsigned long long& cnt) {
    const int lane = threadIdx.x & 31;
    const uint32_t tmask = (1u << lg) - 1u;
    TriMeta t = {};
    t.t_pq = (F & F_TS) ? __ldg(&g.ts[e_pq]) : 0u;
    t.e_pq = (F & F_EL) ? __ldg(&g.el[e_pq]) : 0u;
    t.l_p = (F & F_VL) ? __ldg(&g.vl[p]) : 0u;
    t.l_q = l_q;
    t.d_p = (F & F_EXTRA) ? __ldg(&g.deg[p]) : 0u;
    t.d_q = d_q;
    t.p = p;
    t.q = q;
    if ((F & F_TS) && !in_window(t.t_pq, a.t_lo, a.t_hi)) return;  // no triangle through (p,q) qualifies
    for (uint32_t base = j0; base < end; base += 128) {
        uint32_t rr[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            uint32_t j = base + k * 32 + lane;
            rr[k] = j < end ? __ldg(&g.col[j]) : kEmpty;
        }
        bool past = false;
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            uint32_t r = rr[k];
            int pos = -1;
            if (r != kEmpty && r <= vhi) {
                uint32_t h = hash_slot(r, lg);
                while (true) {
                    uint32_t key = s_key[h];
                    if (key == r) { pos = s_pos16 ? (int)s_pos16[h] : (int)s_pos8[h]; break; }
                    if (key == kEmpty) break;
                    h = (h + 1) & tmask;
                }
            }
            if (r != kEmpty && r > vhi) past = true;
            bool hit = pos >= 0;
            if (__any_sync(0xffffffffu, hit)) {
                bool keep = hit;
                if (hit) {
                    uint32_t j = base + k * 32 + lane;
                    t.r = r;
                    if (F & F_TS) {
                        t.t_pr = __ldg(&g.ts[j]);
                        t.t_qr = s_ts[pos];
                        keep = in_window(t.t_pr, a.t_lo, a.t_hi) && in_window(t.t_qr, a.t_lo, a.t_hi);
                    }
                    if (F & F_EL) { t.e_pr = __ldg(&g.el[j]); t.e_qr = s_el[pos]; }
                    if (F & F_VL) t.l_r = s_vl[pos];
                    if (F & F_EXTRA) t.d_r = s_deg[pos];
                }
                fold_warp<F>(keep, t, a, s_tab, grec, cnt, g.order);
            }
        }
        if (__any_sync(0xffffffffu, past)) break;
    }
}

// Largest-first helper: first index in [lo, hi) with col[idx] >= v.
__device__ __forceinline__ uint32_t lower_bound_col(const uint32_t* __restrict__ col, uint32_t lo, uint32_t hi,
                                                    uint32_t v) {
    while (lo < hi) {
        uint32_t mid = lo + ((hi - lo) >> 1);
        if (__ldg(&col[mid]) < v) lo = mid + 1; else hi = mid;
    }
    return lo;
}

__device__ __forceinline__ unsigned long long* record_of(const GraphDev& g, const SurveyArgs& a, uint32_t q) {
    return g.graph_of ? a.out + (uint64_t)g.graph_of[q] * a.lay.words : a.out;
}

__device__ void flush_shared(unsigned long long* s_tab, uint32_t s_words, unsigned long long* out) {
    for (uint32_t w = threadIdx.x; w < s_words; w += blockDim.x)
        if (s_tab[w]) atomicAdd(&out[w], s_tab[w]);
}

__device__ void flush_count(unsigned long long cnt, const SurveyArgs& a, unsigned long long* s_tab,
                            unsigned long long* grec) {
    for (int o = 16; o; o >>= 1) cnt += __shfl_xor_sync(0xffffffffu, cnt, o);
    if ((threadIdx.x & 31) == 0 && cnt && a.lay.o_count != ~0u) rec_add(s_tab, a.s_words, grec, a.lay.o_count, cnt);
}

// ---- block kernel: one item per block at a time ---------------------------------------------

template <int F>
__global__ void __launch_bounds__(kBlockThreads) survey_block_kernel(GraphDev g, const WorkItem* __restrict__ items,
                                                                     uint32_t n_items, SurveyArgs a) {
    extern __shared__ __align__(16) unsigned char smem[];
    unsigned long long* s_tab = reinterpret_cast<unsigned long long*>(smem);
    uint32_t* s_key = reinterpret_cast<uint32_t*>(smem + a.s_words * 8);
    uint32_t* s_ts = s_key + 2 * kBlockChunk;
    uint32_t* s_deg = s_ts + kBlockChunk;
    uint16_t* s_pos = reinterpret_cast<uint16_t*>(s_deg + kBlockChunk);
    uint8_t* s_el = reinterpret_cast<uint8_t*>(s_pos + 2 * kBlockChunk);
    uint8_t* s_vl = s_el + kBlockChunk;
    __shared__ uint32_t s_item;

    for (uint32_t w = threadIdx.x; w < a.s_words; w += blockDim.x) s_tab[w] = 0;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    unsigned long long cnt = 0;
    unsigned long long* grec_prev = nullptr;

    while (true) {
        if (threadIdx.x == 0) s_item = atomicAdd(&a.counters[1], 1u);
        __syncthreads();  // also: previous item's table no longer in use
        const uint32_t it = s_item;
        if (it >= n_items) break;
        const WorkItem item = items[it];
        const uint32_t q = item.q;
        unsigned long long* grec = record_of(g, a, q);
        if (grec != grec_prev && grec_prev) {  // batched: counts belong to the previous graph
            flush_count(cnt, a, s_tab, grec_prev);
            cnt = 0;
        }
        grec_prev = grec;
        const uint32_t qbase = (uint32_t)g.off[q] + item.qlo;
        const uint32_t len = item.qlen;
        int lg = 5;
        while ((1u << lg) < 2 * len) ++lg;
        const uint32_t tsize = 1u << lg;
        for (uint32_t i = threadIdx.x; i < tsize; i += blockDim.x) s_key[i] = kEmpty;
        __syncthreads();
        for (uint32_t i = threadIdx.x; i < len; i += blockDim.x) {
            const uint32_t r = __ldg(&g.col[qbase + i]);
            uint32_t h = hash_slot(r, lg);
            while (true) {
                uint32_t old = atomicCAS(&s_key[h], kEmpty, r);
                if (old == kEmpty) { s_pos[h] = (uint16_t)i; break; }
                h = (h + 1) & (tsize - 1);
            }
            if (F & F_TS) s_ts[i] = __ldg(&g.ts[qbase + i]);
            if (F & F_EL) s_el[i] = __ldg(&g.el[qbase + i]);
            if (F & F_VL) s_vl[i] = __ldg(&g.vl[r]);
            if (F & F_EXTRA) s_deg[i] = __ldg(&g.deg[r]);
        }
        __syncthreads();
        const bool chunked = item.flags & 1u;
        const uint32_t vlo = chunked ? __ldg(&g.col[qbase]) : 0u;
        const uint32_t vhi = chunked ? __ldg(&g.col[qbase + len - 1]) : 0xFFFFFFFEu;
        const uint32_t l_q = (F & F_VL) ? __ldg(&g.vl[q]) : 0u;
        const uint32_t d_q = (F & F_EXTRA) ? __ldg(&g.deg[q]) : 0u;
        for (uint32_t k = item.in_lo + warp; k < item.in_hi; k += kWarps) {
            const InEdge ie = g.in_edge[k];
            if (ie.p < a.p_lo || ie.p >= a.p_hi) continue;
            uint32_t j0 = ie.e + 1;
            if (chunked) {
                uint32_t jj = 0;
                if (lane == 0) jj = lower_bound_col(g.col, j0, ie.end, vlo);
                j0 = __shfl_sync(0xffffffffu, jj, 0);
            }
            scan_suffix<F>(g, a, ie.e, j0, ie.end, ie.p, q, l_q, d_q, vhi, s_key, s_pos, nullptr, lg, s_ts, s_el,
                           s_vl, s_deg, s_tab, grec, cnt);
        }
    }
    if (grec_prev) flush_count(cnt, a, s_tab, grec_prev);
    __syncthreads();
    flush_shared(s_tab, a.s_words, a.out);
}

// ---- warp kernel: one item per warp at a time ------------------------------------------------

constexpr uint32_t kWTable = 2 * kWarpMaxQ;
struct WarpSmem {
    uint32_t key[kWTable];
    uint32_t ts[kWarpMaxQ];
    uint32_t deg[kWarpMaxQ];
    uint8_t pos[kWTable];
    uint8_t el[kWarpMaxQ];
    uint8_t vl[kWarpMaxQ];
};

template <int F>
__global__ void __launch_bounds__(kBlockThreads) survey_warp_kernel(GraphDev g, const WorkItem* __restrict__ items,
                                                                    uint32_t n_items, SurveyArgs a) {
    extern __shared__ __align__(16) unsigned char smem[];
    unsigned long long* s_tab = reinterpret_cast<unsigned long long*>(smem);
    WarpSmem* ws_all = reinterpret_cast<WarpSmem*>(smem + ((a.s_words * 8 + 15) & ~15u));
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    WarpSmem& ws = ws_all[warp];
    for (uint32_t w = threadIdx.x; w < a.s_words; w += blockDim.x) s_tab[w] = 0;
    __syncthreads();
    unsigned long long cnt = 0;
    unsigned long long* grec_prev = nullptr;

    while (true) {
        uint32_t it = 0;
        if (lane == 0) it = atomicAdd(&a.counters[0], 1u);
        it = __shfl_sync(0xffffffffu, it, 0);
        if (it >= n_items) break;
        const WorkItem item = items[it];
        const uint32_t q = item.q;
        unsigned long long* grec = record_of(g, a, q);
        if (grec != grec_prev && grec_prev) {
            flush_count(cnt, a, s_tab, grec_prev);
            cnt = 0;
        }
        grec_prev = grec;
        const uint32_t qbase = (uint32_t)g.off[q];
        const uint32_t len = item.qlen;
        int lg = 2;
        while ((1u << lg) < 2 * len) ++lg;
        const uint32_t tsize = 1u << lg;
        __syncwarp();
        for (uint32_t i = lane; i < tsize; i += 32) ws.key[i] = kEmpty;
        __syncwarp();
        for (uint32_t i = lane; i < len; i += 32) {
            const uint32_t r = __ldg(&g.col[qbase + i]);
            uint32_t h = hash_slot(r, lg);
            while (true) {
                uint32_t old = atomicCAS(&ws.key[h], kEmpty, r);
                if (old == kEmpty) { ws.pos[h] = (uint8_t)i; break; }
                h = (h + 1) & (tsize - 1);
            }
            if (F & F_TS) ws.ts[i] = __ldg(&g.ts[qbase + i]);
            if (F & F_EL) ws.el[i] = __ldg(&g.el[qbase + i]);
            if (F & F_VL) ws.vl[i] = __ldg(&g.vl[r]);
            if (F & F_EXTRA) ws.deg[i] = __ldg(&g.deg[r]);
        }
        __syncwarp();
        const uint32_t l_q = (F & F_VL) ? __ldg(&g.vl[q]) : 0u;
        const uint32_t d_q = (F & F_EXTRA) ? __ldg(&g.deg[q]) : 0u;
        for (uint32_t k = item.in_lo; k < item.in_hi; ++k) {
            const InEdge ie = g.in_edge[k];
            if (ie.p < a.p_lo || ie.p >= a.p_hi) continue;
            scan_suffix<F>(g, a, ie.e, ie.e + 1, ie.end, ie.p, q, l_q, d_q, 0xFFFFFFFEu, ws.key, nullptr, ws.pos, lg,
                           ws.ts, ws.el, ws.vl, ws.deg, s_tab, grec, cnt);
        }
    }
    if (grec_prev) flush_count(cnt, a, s_tab, grec_prev);
    __syncthreads();
    flush_shared(s_tab, a.s_words, a.out);
}

// ---- plan: work items per middle vertex ----------------------------------------------------

__device__ __forceinline__ uint64_t umin64(uint64_t a, uint64_t b) { return a < b ? a : b; }

__global__ void plan_count_kernel(const uint64_t* __restrict__ off, const uint64_t* __restrict__ in_off, uint64_t n,
                                  uint32_t* __restrict__ cw, uint32_t* __restrict__ cb) {
    for (uint64_t q = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; q < n; q += (uint64_t)gridDim.x * blockDim.x) {
        uint64_t dp = off[q + 1] - off[q], di = in_off[q + 1] - in_off[q];
        uint32_t w = 0, b = 0;
        if (dp > 0 && di > 0) {
            if (dp <= kWarpMaxQ) {
                w = (uint32_t)((di + kWarpInEdges - 1) / kWarpInEdges);
            } else {
                uint64_t chunks = (dp + kBlockChunk - 1) / kBlockChunk;
                uint64_t groups = (di + kBlockInEdges - 1) / kBlockInEdges;
                b = (uint32_t)(chunks * groups);
            }
        }
        cw[q] = w;
        cb[q] = b;
    }
}

__global__ void plan_fill_kernel(const uint64_t* __restrict__ off, const uint64_t* __restrict__ in_off, uint64_t n,
                                 const uint32_t* __restrict__ ow, const uint32_t* __restrict__ ob,
                                 WorkItem* __restrict__ iw, WorkItem* __restrict__ ib) {
    for (uint64_t q = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; q < n; q += (uint64_t)gridDim.x * blockDim.x) {
        uint64_t dp = off[q + 1] - off[q], di = in_off[q + 1] - in_off[q];
        if (dp == 0 || di == 0) continue;
        const uint32_t ilo = (uint32_t)in_off[q];
        if (dp <= kWarpMaxQ) {
            uint32_t o = ow[q];
            for (uint64_t s = 0; s < di; s += kWarpInEdges) {
                WorkItem it;
                it.q = (uint32_t)q; it.qlo = 0; it.qlen = (uint32_t)dp;
                it.in_lo = ilo + (uint32_t)s;
                it.in_hi = ilo + (uint32_t)umin64(di, s + kWarpInEdges);
                it.flags = 0; it.pad0 = it.pad1 = 0;
                iw[o++] = it;
            }
        } else {
            uint32_t o = ob[q];
            const bool chunked = dp > kBlockChunk;
            for (uint64_t c = 0; c < dp; c += kBlockChunk) {
                for (uint64_t s = 0; s < di; s += kBlockInEdges) {
                    WorkItem it;
                    it.q = (uint32_t)q; it.qlo = (uint32_t)c;
                    it.qlen = (uint32_t)umin64(kBlockChunk, dp - c);
                    it.in_lo = ilo + (uint32_t)s;
                    it.in_hi = ilo + (uint32_t)umin64(di, s + kBlockInEdges);
                    it.flags = chunked ? 1u : 0u; it.pad0 = it.pad1 = 0;
                    ib[o++] = it;
                }
            }
        }
    }
}

unsigned grid_n(uint64_t items) {
    uint64_t b = (items + 255) / 256;
    return (unsigned)std::max<uint64_t>(1, std::min<uint64_t>(b, 148u * 64u));
}

template <int F>
void launch_f(const tripoll_graph* g, const SurveyArgs& a, cudaStream_t s, int sms) {
    GraphDev gd = g->dev();
    if (g->n_items_warp) {
        size_t sm = ((a.s_words * 8 + 15) & ~15u) + kWarps * sizeof(WarpSmem);
        cudaFuncSetAttribute(survey_warp_kernel<F>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        int per = 0;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, survey_warp_kernel<F>, kBlockThreads, sm);
        uint64_t blocks = (uint64_t)std::max(per, 1) * sms;
        blocks = std::min<uint64_t>(blocks, (g->n_items_warp + kWarps - 1) / kWarps);
        survey_warp_kernel<F><<<(unsigned)blocks, kBlockThreads, sm, s>>>(gd, g->items_warp,
                                                                         (uint32_t)g->n_items_warp, a); ::tp::note_launch();
    }
    if (g->n_items_block) {
        size_t sm = a.s_words * 8 + (2 * kBlockChunk) * 4 + kBlockChunk * 4 * 2 + (2 * kBlockChunk) * 2 +
                    kBlockChunk * 2;
        cudaFuncSetAttribute(survey_block_kernel<F>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        int per = 0;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, survey_block_kernel<F>, kBlockThreads, sm);
        uint64_t blocks = (uint64_t)std::max(per, 1) * sms;
        blocks = std::min<uint64_t>(blocks, g->n_items_block);
        survey_block_kernel<F><<<(unsigned)blocks, kBlockThreads, sm, s>>>(gd, g->items_block,
                                                                          (uint32_t)g->n_items_block, a); ::tp::note_launch();
    }
}

using LaunchFn = void (*)(const tripoll_graph*, const SurveyArgs&, cudaStream_t, int);
constexpr LaunchFn kLaunch[16] = {&launch_f<0>,  &launch_f<1>,  &launch_f<2>,  &launch_f<3>,
                                  &launch_f<4>,  &launch_f<5>,  &launch_f<6>,  &launch_f<7>,
                                  &launch_f<8>,  &launch_f<9>,  &launch_f<10>, &launch_f<11>,
                                  &launch_f<12>, &launch_f<13>, &launch_f<14>, &launch_f<15>};

}  // namespace

int build_plan(tripoll_graph* g, cudaStream_t s) {
    const uint64_t n = g->n;
    Scratch cw, cb, ow, ob, tmp;
    TP_CUDA(cw.alloc((n + 1) * 4, s));
    TP_CUDA(cb.alloc((n + 1) * 4, s));
    TP_CUDA(ow.alloc((n + 1) * 4, s));
    TP_CUDA(ob.alloc((n + 1) * 4, s));
    TP_CUDA(cudaMemsetAsync(cw.ptr, 0, (n + 1) * 4, s));
    TP_CUDA(cudaMemsetAsync(cb.ptr, 0, (n + 1) * 4, s));
    if (n) plan_count_kernel<<<grid_n(n), 256, 0, s>>>(g->off, g->in_off, n, cw.as<uint32_t>(), cb.as<uint32_t>()); ::tp::note_launch();
    TP_CUDA(cudaGetLastError());
    size_t tb = 0;
    TP_CUDA(cub::DeviceScan::ExclusiveSum(nullptr, tb, cw.as<uint32_t>(), ow.as<uint32_t>(), n + 1, s));
    TP_CUDA(tmp.alloc(tb, s));
    TP_CUDA(cub::DeviceScan::ExclusiveSum(tmp.ptr, tb, cw.as<uint32_t>(), ow.as<uint32_t>(), n + 1, s));
    TP_CUDA(cub::DeviceScan::ExclusiveSum(tmp.ptr, tb, cb.as<uint32_t>(), ob.as<uint32_t>(), n + 1, s));
    uint32_t tot[2] = {0, 0};
    TP_CUDA(cudaMemcpyAsync(&tot[0], ow.as<uint32_t>() + n, 4, cudaMemcpyDeviceToHost, s));
    TP_CUDA(cudaMemcpyAsync(&tot[1], ob.as<uint32_t>() + n, 4, cudaMemcpyDeviceToHost, s));
    TP_CUDA(cudaStreamSynchronize(s));
    g->n_items_warp = tot[0];
    g->n_items_block = tot[1];
    TP_CUDA(cudaMalloc((void**)&g->items_warp, std::max<uint64_t>(1, tot[0]) * sizeof(WorkItem)));
    TP_CUDA(cudaMalloc((void**)&g->items_block, std::max<uint64_t>(1, tot[1]) * sizeof(WorkItem)));
    if (n)
        plan_fill_kernel<<<grid_n(n), 256, 0, s>>>(g->off, g->in_off, n, ow.as<uint32_t>(), ob.as<uint32_t>(),
                                                   g->items_warp, g->items_block); ::tp::note_launch();
    TP_CUDA(cudaGetLastError());
    return TRIPOLL_OK;
}

// Launch the survey kernels accumulating into `acc` (zeroed by the caller).
int launch_survey(const tripoll_graph* g, uint32_t kinds, uint32_t t_lo, uint32_t t_hi, uint64_t p_lo, uint64_t p_hi,
                  unsigned long long* acc, uint32_t* counters, cudaStream_t s) {
    const Layout lay = make_layout(kinds, g->Lv, g->Le, g->n);
    SurveyArgs a;
    a.kinds = kinds;
    a.t_lo = t_lo;
    a.t_hi = t_hi;
    a.Lv = g->Lv;
    a.Le = g->Le;
    a.p_lo = p_lo;
    a.p_hi = p_hi;
    a.lay = lay;
    a.out = acc;
    a.counters = counters;
    // record prefix mirrored on chip: the tables that fit, never the local counts
    uint64_t sw = lay.o_vlocal != ~0ull ? lay.o_vlocal : lay.words;
    if (g->graph_of) sw = 0;
    a.s_words = (uint32_t)std::min<uint64_t>(sw, kSharedTableWords);
    const bool window = !(t_lo == 0 && t_hi == 0xFFFFFFFFu);
    int F = 0;
    if (window || (kinds & (TRIPOLL_CLOSURE_HIST | TRIPOLL_OPEN_CLOSE_HIST))) F |= F_TS;
    if (kinds & (TRIPOLL_ELABEL_TRIPLES | TRIPOLL_MAX_ELABEL)) F |= F_EL;
    if (kinds & (TRIPOLL_VLABEL_TRIPLES | TRIPOLL_MAX_ELABEL)) F |= F_VL;
    if (kinds & (TRIPOLL_OPEN_CLOSE_HIST | TRIPOLL_MAX_ELABEL | TRIPOLL_DEGREE_TRIPLES | TRIPOLL_VERTEX_LOCAL))
        F |= F_EXTRA | F_TS;
    int sms = 148;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, g->device);
    TP_CUDA(cudaMemsetAsync(counters, 0, 8, s));
    kLaunch[F](g, a, s, sms);
    TP_CUDA(cudaGetLastError());
    return TRIPOLL_OK;
}

}  // namespace tp

// survey_kernels.cuh -- wedge checks and the survey fold (TriPoll Sec. 4.3-4.5, Alg. 1-4).
//
// Every triangle p <+ q <+ r of G+ is found exactly once as r in
// Adj+(p) ∩ Adj+(q) with r after q in Adj+(p) (Alg. 1).  The kernels here
// organise that intersection around the middle vertex q, the single-GPU form
// of the paper's pull phase (Sec. 4.4): the out-list of q, with the metadata
// of its edges (q,r) and the labels of the r, is staged once in shared memory
// as an open-addressing hash table, and then every in-edge (p,q) streams the
// suffix of Adj+(p) after q from HBM and probes each candidate r against it
// -- one probe per wedge (p,q,r), the wedge check of Sec. 3.  (A block item
// whose staged out-list spans few positions uses a rank bitmap over the span
// instead of the hash table.)  A hit is a triangle; its six metadata items
// (Sec. 3) are the (p,q) edge's (read once per in-edge), the (p,r) edge's
// (gathered at the hit position), and the (q,r) edge's plus vertex r's (from
// shared memory).
//
// Three kernels split the middle vertices by |Adj+(q)|: a warp-per-item kernel
// for out-lists of up to kWarpPlanQ entries (each warp its own table, staging
// kWarpMaxQ entries of the window view at a time), a block-per-item kernel for
// longer ones, staged kBlockChunk entries at a time, and the same block kernel
// with kBigChunk-entry tables for the longest (a longer out-list is cut into
// parts, and each in-edge's segment is restricted to the part's value range by
// binary search).  Inside an item the in-edges' segments form one flat index
// space of units of 8 consecutive candidates that warps split evenly and walk
// 32 units at a time: consecutive lanes read consecutive 32-byte units of the
// suffixes (coalesced), and no lane idles however skewed the suffix lengths
// are.  Triangles outside the time window are pruned before any probe: a survey
// with a window runs on a view of G+ holding only its in-window edges (the
// window view, built in survey.cu); without a view (the allocation-free survey) in-edges
// (p,q) outside the window get empty segments and entries (q,r) outside it are
// not inserted.
//
// Hits are queued per warp and folded 32 at a time, one per lane.  Table words
// that fit the block's on-chip mirror of the result record get one 32-bit
// shared-memory atomic per lane (the hardware resolves equal addresses); the
// mirror is moved into the 64-bit record with global atomics rarely, and once
// per block at its end.  Words outside the mirror (batched graphs, tables past
// its size) are first merged across the warp with __match_any_sync, then
// added through the block's word cache (records past the mirror, F_CACHE) or
// with one 64-bit global atomic per distinct word.  Integer adds commute, so
// the result is exact and schedule-independent.
//
// The kernels are templates over the features a survey needs (F_*); each
// survey_inst_*.cu file instantiates the launch of a quarter of the feature
// combinations, so that they compile in parallel, and survey.cu dispatches.
#pragma once

#include <cstdlib>

#include "common.cuh"
#include "primitives.cuh"

namespace tp {
namespace sv {

constexpr uint32_t kEmpty = 0xFFFFFFFFu;
constexpr int kBlockThreads = 256;
constexpr int kWarps = kBlockThreads / 32;
constexpr uint32_t kSharedTableWords = 4096;  // on-chip mirror of the record prefix (16 KB)
// The mirror holds 32-bit partial sums: 32-bit shared-memory atomics cost less than 64-bit ones.
// It is moved into the 64-bit record (each word exchanged with 0) often enough that no word
// can reach 2^32.  A word gains at most one per hit, and an item has at most (staged entries)
// x (in-edges) hits: 2^11 x 2^11 for block items, 2^8 x 2^6 for warp items (a plan's warp items
// hold out-lists of at most 256 entries).  So a block of a block kernel moves it after every 2^9
// items it takes (< 2^31 between moves), and each of the 8 warps of a warp-kernel block after every
// 2^14 items it takes (< 8 x 2^28 = 2^31).  The
// environment variable TRIPOLL_MIRROR_MOVE_LOG2 = k moves it every 2^k items instead when k is
// smaller (tests use it to exercise the moves on small graphs).
constexpr uint32_t kBlockMoveLog2 = 9, kWarpMoveLog2 = 14;
static_assert(kBlockMoveLog2 + 11 + 11 < 32 && kWarpMoveLog2 + 8 + 6 + 3 < 32, "mirror words stay below 2^32");
static_assert(kWarpPlanMax <= (1u << 8) && kItemInEdges <= (1u << 11) && kBigChunk <= (1u << 11),
              "the plan bounds that the move periods assume");
using MirrorWord = uint32_t;

// feature bits of a kernel instantiation
constexpr int F_TS = 1;     // timestamps (window or time kinds)
constexpr int F_EL = 2;     // edge labels
constexpr int F_VL = 4;     // vertex labels
constexpr int F_EXTRA = 8;  // joint table, max label, degree triples, local counts
constexpr int F_CACHE = 16; // record larger than the on-chip mirror: a word cache in front of global atomics
constexpr int F_MULTI = 32; // several requests' windows at once: one record per cell of their bounds

// Several requests in one pass (F_MULTI).  The distinct lower bounds L[0] < ... < L[A-1] and upper
// bounds H[0] < ... < H[B-1] of the requests' windows cut the (earliest, latest) timestamp plane of
// the triangles into A x B cells; a triangle with earliest timestamp t1 and latest t3 is counted in
// cell (i, j), i the last lower bound <= t1 and j the first upper bound >= t3, whose record holds
// all tables of the union of the requests' kinds.  The request with window [L[x], H[y]] takes
// exactly the triangles of the cells i >= x, j <= y, so its tables are that block's sum.  The bounds
// live in shared memory ahead of the mirror: A, B, then L and H (kMultiMax each).
constexpr uint32_t kMultiMax = 64;
constexpr uint32_t kMultiWords = 4 + 2 * kMultiMax;
template <int F> __host__ __device__ constexpr uint32_t multi_bytes() { return (F & F_MULTI) ? kMultiWords * 4 : 0; }

// Word cache (F_CACHE).  A record too large for the dense mirror keeps its first kCacheDenseWords
// words dense on chip and puts a small open-addressing cache (word -> 32-bit count) in front of
// the 64-bit global atomics for the rest: a word takes a slot on its first increment and keeps it
// for the life of the block, so hot words (the common label or degree triples) are counted on
// chip instead of serialising on one L2 address; a word that finds no slot within kCacheProbes
// probes goes to global memory directly.  Slot values move into the record on the mirror's
// schedule (so they stay below 2^32) and when the block ends.
constexpr uint32_t kCacheLog2 = 10;
constexpr uint32_t kCacheSlots = 1u << kCacheLog2;
constexpr uint32_t kCacheProbes = 8;
constexpr uint32_t kCacheDenseWords = kSharedTableWords - 2 * kCacheSlots;  // same room as the plain mirror

struct SurveyArgs {
    uint32_t kinds;
    uint32_t t_lo, t_hi;
    uint32_t Lv, Le;
    uint32_t s_words;         // record words mirrored in shared memory (0 for batched graphs)
    uint64_t p_lo, p_hi;      // pivot range
    uint32_t e_lo, e_hi;      // its CSR positions [off[p_lo], off[p_hi])
    bool restricted;          // pivot range is not all of [0, n)
    // log2 of the items between moves of the shared mirror into the record: a block of a block
    // kernel, a warp of the warp kernel.  (These sit in what would otherwise be padding: a larger
    // argument block measurably slowed the survey kernels.)
    uint8_t move_block_log2, move_warp_log2;
    // the warp kernel's items hold window-view positions already (vpos, qlen, in_lo, in_hi), none empty
    uint8_t view_items;
    Layout lay;  // (the argument block keeps 4 bytes of padding after the flags)
    unsigned long long* out;  // accumulator: one record, or num_graphs records (batched)
    uint32_t* counters;       // item counters of the three kernels; F_MULTI: [4] A, [5] B, then the bounds
};
static_assert(sizeof(SurveyArgs) == 128, "kernel argument block of the survey kernels");

// The work item lists a survey launch runs (warp, block, long-list kernels): the graph's, or for the
// warp kernel their translation into a window view's positions with the empty items left out.
struct ItemLists {
    const WorkItem* items[3];
    uint64_t n[3];
};

// Resident blocks per SM of a kernel at a dynamic shared-memory size (survey.cu).
int blocks_per_sm(const void* kernel, size_t smem);

namespace {  // the kernels: every translation unit that launches them has its own copy


// Home slot of r in a table of `size` slots: a multiplicative hash scaled to size.
__device__ __forceinline__ uint32_t hash_slot(uint32_t r, uint32_t size) {
    return __umulhi(r * 2654435761u, size);
}

// The word cache sits right after the dense mirror (F_CACHE): keys, then values.
__device__ __forceinline__ uint32_t* cache_keys(MirrorWord* s_tab, uint32_t s_words) {
    return s_tab + ((s_words + 3) & ~3u);
}

// Move the shared mirror (and the word cache's counts) into the record, by one warp while the
// others keep adding to it.
template <int F>
__device__ __forceinline__ void move_mirror_warp(MirrorWord* s_tab, uint32_t s_words, unsigned long long* out) {
    for (uint32_t w = threadIdx.x & 31; w < s_words; w += 32) {
        const MirrorWord v = atomicExch(&s_tab[w], 0u);
        if (v) atomicAdd(&out[w], (unsigned long long)v);
    }
    if (F & F_CACHE) {
        uint32_t* key = cache_keys(s_tab, s_words);
        uint32_t* val = key + kCacheSlots;
        for (uint32_t i = threadIdx.x & 31; i < kCacheSlots; i += 32) {
            const uint32_t v = atomicExch(&val[i], 0u);
            if (v) atomicAdd(&out[key[i]], (unsigned long long)v);
        }
    }
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

// Add `amount` to word `w` of the record: shared mirror when w < s_words, else (F_CACHE) the word
// cache, else global.  The cache is used only for a single record (grec is the accumulator base).
template <int F>
__device__ __forceinline__ void rec_add(MirrorWord* s_tab, uint32_t s_words, unsigned long long* grec,
                                        uint64_t w, unsigned long long amount) {
    if (w < s_words) {
        atomicAdd(&s_tab[w], (MirrorWord)amount);  // amount <= 32 here
        return;
    }
    if (F & F_CACHE) {
        volatile uint32_t* key = cache_keys(s_tab, s_words);
        uint32_t* val = const_cast<uint32_t*>(key) + kCacheSlots;
        const uint32_t ww = (uint32_t)w;
        uint32_t h = (ww * 2654435761u) >> (32 - kCacheLog2);
        for (uint32_t p = 0; p < kCacheProbes; ++p) {
            uint32_t k = key[h];
            if (k == kEmpty) {
                k = atomicCAS(const_cast<uint32_t*>(&key[h]), kEmpty, ww);
                if (k == kEmpty) __threadfence_block();  // the key is visible before its count
            }
            if (k == kEmpty || k == ww) {
                atomicAdd(&val[h], (uint32_t)amount);
                return;
            }
            h = (h + 1) & (kCacheSlots - 1);
        }
    }
    atomicAdd(&grec[w], amount);
}

// Increment of word `w` by each lane in `mask` (the calling lanes).  When all of their words are
// in the shared mirror, plain 32-bit shared atomics (the hardware resolves equal addresses) cost
// less than merging equal words first; other words are merged within the warp first.
template <int F>
__device__ __forceinline__ void warp_add(unsigned mask, MirrorWord* s_tab, uint32_t s_words,
                                         unsigned long long* grec, uint64_t w) {
    if (__all_sync(mask, w < s_words)) {
        atomicAdd(&s_tab[w], 1u);
        return;
    }
    unsigned grp = __match_any_sync(mask, w);
    int leader = __ffs(grp) - 1;
    if ((int)(threadIdx.x & 31) == leader) rec_add<F>(s_tab, s_words, grec, w, (unsigned long long)__popc(grp));
}

struct TriMeta {
    uint32_t t_pq, t_pr, t_qr;
    uint32_t e_pq, e_pr, e_qr;  // edge labels
    uint32_t l_p, l_q, l_r;     // vertex labels
    uint32_t d_p, d_q, d_r;     // degrees (F_EXTRA)
    uint32_t p, q, r;           // positions (F_EXTRA local counts)
    uint32_t x_pq, x_pr, x_qr;  // CSR positions of the three edges in G+ (F_EXTRA edge counts)
    uint32_t qbase;             // CSR position (in the surveyed arrays) of the staged part of Adj+(q)
};

// Fold the lanes with `keep` set (called by the whole warp).
template <int F>
__device__ __forceinline__ void fold_warp(bool keep, const TriMeta& t, const SurveyArgs& a, MirrorWord* s_tab,
                                          unsigned long long* grec, unsigned long long& cnt,
                                          const uint32_t* __restrict__ order) {
    uint64_t cb = 0;  // first word of the triangle's cell record (F_MULTI)
    uint32_t t1 = t.t_pq, t2 = t.t_pr, t3 = t.t_qr;
    if (F & F_MULTI) {
        sort3(t1, t2, t3);
        const uint32_t* win = reinterpret_cast<const uint32_t*>(s_tab) - kMultiWords;
        const uint32_t A = win[0], B = win[1];
        const uint32_t* lo = win + 4;
        const uint32_t* hi = win + 4 + kMultiMax;
        uint32_t i = 0, j = 0;  // i: lower bounds <= t1; j: upper bounds < t3
        for (uint32_t step = kMultiMax; step; step >>= 1) {
            if (i + step <= A && lo[i + step - 1] <= t1) i += step;
            if (j + step <= B && hi[j + step - 1] < t3) j += step;
        }
        if (i == 0 || j == B) keep = false;  // in no request's window
        cb = ((uint64_t)(i - 1) * B + j) * a.lay.words;
    }
    const unsigned km = __ballot_sync(0xffffffffu, keep);
    if (!km) return;
    if (!keep) return;
    const Layout& L = a.lay;
    if (F & F_MULTI) {
        if (L.o_count != ~0u) warp_add<F>(km, s_tab, a.s_words, grec, cb + L.o_count);
    } else {
        cnt += 1;
        if (F & F_TS) sort3(t1, t2, t3);
    }
    if (L.o_hist != ~0u) warp_add<F>(km, s_tab, a.s_words, grec, cb + L.o_hist + time_bin(t3 - t1));
    if ((F & F_VL) && L.o_vtri != ~0u) {
        uint32_t x = t.l_p, y = t.l_q, z = t.l_r;
        sort3(x, y, z);
        warp_add<F>(km, s_tab, a.s_words, grec, cb + L.o_vtri + (x * a.Lv + y) * a.Lv + z);
    }
    if ((F & F_EL) && L.o_etri != ~0u) {
        uint32_t x = t.e_pq, y = t.e_pr, z = t.e_qr;
        sort3(x, y, z);
        warp_add<F>(km, s_tab, a.s_words, grec, cb + L.o_etri + (x * a.Le + y) * a.Le + z);
    }
    if (F & F_EXTRA) {
        if (L.o_joint != ~0u)
            rec_add<F>(s_tab, a.s_words, grec,
                       cb + L.o_joint + time_bin(t2 - t1) * TRIPOLL_HIST_BINS + time_bin(t3 - t1), 1);
        if (L.o_maxel != ~0u && t.l_p != t.l_q && t.l_q != t.l_r && t.l_p != t.l_r)
            rec_add<F>(s_tab, a.s_words, grec, cb + L.o_maxel + max(t.e_pq, max(t.e_pr, t.e_qr)), 1);
        if (L.o_degtri != ~0u) {
            uint32_t x = time_bin(t.d_p), y = time_bin(t.d_q), z = time_bin(t.d_r);
            sort3(x, y, z);
            rec_add<F>(s_tab, a.s_words, grec,
                       cb + L.o_degtri + (x * TRIPOLL_HIST_BINS + y) * TRIPOLL_HIST_BINS + z, 1);
        }
        if (!(F & F_MULTI)) {  // local counts are never surveyed several windows at once
            if (L.o_vlocal != ~0ull) {
                atomicAdd(&grec[L.o_vlocal + order[t.p]], 1ull);
                atomicAdd(&grec[L.o_vlocal + order[t.q]], 1ull);
                atomicAdd(&grec[L.o_vlocal + order[t.r]], 1ull);
            }
            if (L.o_elocal != ~0ull) {
                atomicAdd(&grec[L.o_elocal + t.x_pq], 1ull);
                atomicAdd(&grec[L.o_elocal + t.x_pr], 1ull);
                atomicAdd(&grec[L.o_elocal + t.x_qr], 1ull);
            }
        }
    }
}

__device__ __forceinline__ bool in_window(uint32_t t, uint32_t lo, uint32_t hi) { return t >= lo && t <= hi; }

// Position in the window view of CSR position e of G+: in-window edges before e.
__device__ __forceinline__ uint32_t view_pos(const uint2* __restrict__ vidx, uint32_t e) {
    const uint2 w = __ldg(&vidx[e >> 5]);
    return w.x + __popc(w.y & ((1u << (e & 31u)) - 1u));
}

// First index in [lo, hi) with col[idx] >= v.
__device__ __forceinline__ uint32_t lower_bound_col(const uint32_t* __restrict__ col, uint32_t lo, uint32_t hi,
                                                    uint32_t v) {
    while (lo < hi) {
        uint32_t mid = lo + ((hi - lo) >> 1);
        if (__ldg(&col[mid]) < v) lo = mid + 1; else hi = mid;
    }
    return lo;
}

// ---- on-chip table of Adj+(q) -------------------------------------------------------------

// Open-addressing hash table of the staged part of Adj+(q): key[] holds target
// positions r (kEmpty = free slot), pos[] the index of r in the staged arrays
// ts[] (timestamp of (q,r)), el[] (its label), vl[] (label of r), deg[] (d(r)).
template <class PosT>
struct QTable {
    uint32_t* key;
    PosT* pos;
    uint32_t* ts;
    uint32_t* deg;
    uint8_t* el;
    uint8_t* vl;
    uint32_t size;  // slots in use (view_table_size)
};

#ifndef TP_TABLE_FACTOR
#define TP_TABLE_FACTOR 3
#endif
constexpr uint32_t kTableFactor = TP_TABLE_FACTOR;  // table slots per staged entry

__device__ __forceinline__ uint32_t table_size(uint32_t len) { return max(kTableFactor * len, 4u); }

// Slots used for len staged entries out of cap: a window view stages only
// in-window entries, so its tables use the room left by the out-of-window
// ones: six times the slots per entry (load factor <= 1/18) while they fit,
// which makes a probe that finds its home slot taken by another key rare.
__device__ __forceinline__ uint32_t view_table_size(uint32_t len, bool view, uint32_t cap) {
    return view ? min(table_size(6 * len), cap) : table_size(len);
}

// Insert the entries [i0, len) step `stride` of the staged out-list part at
// CSR position qbase; entries whose (q,r) timestamp lies outside the window
// can close no surveyed triangle and are left out.
template <int F, class PosT>
__device__ __forceinline__ void table_fill(const GraphDev& g, const SurveyArgs& a, QTable<PosT> T, uint32_t qbase,
                                           uint32_t len, uint32_t i0, uint32_t stride) {
    for (uint32_t i = i0; i < len; i += stride) {
        uint32_t t = 0;
        if (F & F_TS) {
            t = __ldg(&g.ts[qbase + i]);
            if (!in_window(t, a.t_lo, a.t_hi)) continue;
        }
        const uint32_t r = __ldg(&g.col[qbase + i]);
        uint32_t h = hash_slot(r, T.size);
        while (true) {
            uint32_t old = atomicCAS(&T.key[h], kEmpty, r);
            if (old == kEmpty) { T.pos[h] = (PosT)i; break; }
            if (++h == T.size) h = 0;
        }
        if (F & F_TS) T.ts[i] = t;
        if (F & F_EL) T.el[i] = __ldg(&g.el[qbase + i]);
        if (F & F_VL) T.vl[i] = __ldg(&g.vl[r]);
        if (F & F_EXTRA) T.deg[i] = __ldg(&g.deg[r]);
    }
}

// Index of r among the staged entries, or -1, searching from slot h on.
template <class PosT>
__device__ __forceinline__ int table_find_from(const QTable<PosT>& T, uint32_t r, uint32_t h) {
    while (true) {
        const uint32_t key = T.key[h];
        if (key == r) return (int)T.pos[h];
        if (key == kEmpty) return -1;
        if (++h == T.size) h = 0;
    }
}

// The four candidates of a quad (act[i]: position i lies in the segment): the
// four home slots are read together, and only a home slot holding another
// key continues the search.
template <class PosT>
__device__ __forceinline__ void probe_quad(const QTable<PosT>& T, const uint32_t (&r)[4], const bool (&act)[4],
                                           int (&pos)[4]) {
    uint32_t h[4], key[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        h[i] = hash_slot(r[i], T.size);
        key[i] = act[i] ? T.key[h[i]] : kEmpty;
    }
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        pos[i] = -1;
        if (key[i] == kEmpty) continue;
        if (key[i] == r[i]) {
            pos[i] = (int)T.pos[h[i]];
            continue;
        }
        pos[i] = table_find_from(T, r[i], h[i] + 1 == T.size ? 0u : h[i] + 1);
    }
}

// Rank bitmap of a staged part of Adj+(q) whose values lie in [vlo, vlo + span): bit r - vlo is set
// for every staged r, and pre[w] counts the set bits of the words before w, so the staged index of a
// set bit (the entries are sorted and all staged) is pre[w] + the set bits below it in its word.  A
// block item uses it instead of the hash table when the span fits (span = 0: the hash table), which
// in the degree order is the common case: a middle vertex's out-neighbours have higher degree and sit
// together near the end of the order.
struct RankBitmap {
    const uint32_t* bm;
    const uint32_t* pre;
    uint32_t vlo, span;
};

__device__ __forceinline__ void probe_quad_bm(const RankBitmap& B, const uint32_t (&r)[4], const bool (&act)[4],
                                              int (&pos)[4]) {
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const uint32_t b = r[i] - B.vlo;  // below vlo wraps to >= span
        const uint32_t w = (act[i] && b < B.span) ? B.bm[b >> 5] : 0u;
        const uint32_t sh = b & 31u;
        pos[i] = ((w >> sh) & 1u) ? (int)(B.pre[b >> 5] + __popc(w & ((1u << sh) - 1u))) : -1;
    }
}

// ---- in-edges of the item, staged ------------------------------------------------------------

// Per in-edge (p,q) of the item: the segment [j0, jend) of Adj+(p) to check
// (positions after q, restricted to the staged value range of a chunked
// item), the (p,q) metadata, and the exclusive prefix pp of the segments'
// unit counts, a unit being kUnit consecutive positions starting at a multiple
// of kUnit: the item's wedge checks form one flat index space of units
// [0, pp[n_in]), each unit read with kUnit/4 16-byte loads.
#ifndef TP_UNIT_LOG
#define TP_UNIT_LOG 3
#endif
constexpr uint32_t kUnitLog = TP_UNIT_LOG;       // a unit: 2^kUnitLog consecutive positions from a multiple of it
constexpr uint32_t kUnit = 1u << kUnitLog;
constexpr int kUnitQuads = (int)(kUnit / 4);     // 16-byte loads per unit
static_assert(kColPad >= kUnit, "the padding of col[] covers the last unit of the last out-list");

struct InStage {
    uint32_t* j0;
    uint32_t* jend;
    uint32_t* tpq;
    uint32_t* meta;
    uint32_t* p;
    uint32_t* e;   // CSR position of (p,q) in G+ (F_EXTRA)
    uint32_t* pp;  // [n_in + 1]
};

__device__ __forceinline__ uint32_t upper_bound_col(const uint32_t* __restrict__ col, uint32_t lo, uint32_t hi,
                                                    uint32_t v) {
    while (lo < hi) {
        uint32_t mid = lo + ((hi - lo) >> 1);
        if (__ldg(&col[mid]) <= v) lo = mid + 1; else hi = mid;
    }
    return lo;
}

// Stage in-edge slot k (absolute record kk); returns its segment's unit count.
template <int F>
__device__ __forceinline__ uint32_t stage_in_edge(const GraphDev& g, const SurveyArgs& a, InStage S, uint32_t k,
                                                  uint32_t kk, bool chunked, uint32_t vlo, uint32_t vhi) {
    const InEdge ie = g.in_edge[kk];
    bool ok = true;
    // (p,q) outside the window: no triangle through it (the view's in-edges are all inside)
    if ((F & F_TS) && !g.iidx) ok = in_window(ie.ts, a.t_lo, a.t_hi);
    // the CSR position of (p,q) in G+
    const uint32_t eg = (g.iidx && (a.restricted || (F & F_EXTRA))) ? __ldg(&g.vin_e[kk]) : ie.e;
    // the pivot p owns CSR positions [off[p], off[p+1]): a pivot range is a position range
    if (a.restricted && (eg < a.e_lo || eg >= a.e_hi)) ok = false;
    uint32_t p = 0;
    if (F & F_EXTRA) {  // p itself: the last vertex whose out-list starts at or before e
        uint32_t lo = 0, hi = (uint32_t)g.n - 1;
        while (lo < hi) {
            const uint32_t mid = lo + ((hi - lo + 1) >> 1);
            if (__ldg(&g.off[mid]) <= eg) lo = mid; else hi = mid - 1;
        }
        p = lo;
    }
    uint32_t j0 = ie.e + 1, jend = ie.end;  // (a view in-edge record holds view positions already)
    if (ok && g.vidx && !g.iidx) {  // the suffix of Adj+(p) after q in the window view
        j0 = view_pos(g.vidx, ie.e) + 1;
        jend = view_pos(g.vidx, ie.end);
    }
    if (ok && chunked && j0 < jend) {
        j0 = lower_bound_col(g.col, j0, jend, vlo);
        jend = upper_bound_col(g.col, j0, jend, vhi);
    }
    S.j0[k] = j0;
    S.jend[k] = jend;
    S.tpq[k] = ie.ts;
    S.meta[k] = ie.meta;
    if (F & F_EXTRA) {
        S.p[k] = p;
        S.e[k] = eg;
    }
    return (ok && j0 < jend) ? ((jend + kUnit - 1) >> kUnitLog) - (j0 >> kUnitLog) : 0u;
}

// Last slot k in [lo, hi) with pp[k] <= f (pp non-decreasing, pp[lo] <= f).
__device__ __forceinline__ uint32_t seg_of(const uint32_t* pp, uint32_t lo, uint32_t hi, uint32_t f) {
    while (hi - lo > 1) {
        const uint32_t mid = (lo + hi) >> 1;
        if (pp[mid] <= f) lo = mid; else hi = mid;
    }
    return lo;
}

#ifndef TP_UNROLL
#define TP_UNROLL 1
#endif
constexpr int kUnroll = TP_UNROLL;  // units each lane has in flight per chunk
constexpr int kHitQ = 64;  // per-warp queue of hits awaiting the fold (< 32 left + 32 new)

// Per-warp queue of wedge checks that hit: CSR position of (p,r), and
// (staged index of r) | (in-edge slot) << 16.
struct HitQueue {
    uint32_t* idx;
    uint32_t* pk;
};

// Fold the `nq` queued hits from entry `head` on, one per lane (nq <= 32).  A queue entry is
// the CSR position of (p,r) and (staged index of r) | (in-edge slot) << 16.
template <int F, class PosT>
__device__ __forceinline__ void fold_queue(const GraphDev& g, const SurveyArgs& a, const QTable<PosT>& T,
                                           const InStage& S, const HitQueue& H, uint32_t head, uint32_t nq, TriMeta t,
                                           MirrorWord* s_tab, unsigned long long* grec,
                                           unsigned long long& cnt) {
    const uint32_t lane = threadIdx.x & 31;
    bool keep = lane < nq;
    if (keep) {
        const uint32_t idx = H.idx[head + lane], pk = H.pk[head + lane];
        const uint32_t pos = pk & 0xffffu, k = pk >> 16;
        t.t_pq = S.tpq[k];
        const uint32_t meta = S.meta[k];
        t.e_pq = meta & 0xffu;
        t.l_p = (meta >> 8) & 0xffu;
        if (F & F_TS) {
            t.t_pr = __ldg(&g.ts[idx]);
            t.t_qr = T.ts[pos];
            keep = in_window(t.t_pr, a.t_lo, a.t_hi);  // (p,q) and (q,r) were checked at staging
        }
        if (F & F_EL) { t.e_pr = __ldg(&g.el[idx]); t.e_qr = T.el[pos]; }
        if (F & F_VL) t.l_r = T.vl[pos];
        if (F & F_EXTRA) {
            t.r = __ldg(&g.col[idx]);
            t.p = S.p[k];
            t.d_p = __ldg(&g.deg[t.p]);
            t.d_r = T.deg[pos];
            // positions in G+ of (p,r) and (q,r): through the window view's map when surveying one
            t.x_pq = S.e[k];
            t.x_pr = g.vorig ? __ldg(&g.vorig[idx]) : idx;
            t.x_qr = g.vorig ? __ldg(&g.vorig[t.qbase + pos]) : t.qbase + pos;
        }
    }
    fold_warp<F>(keep, t, a, s_tab, grec, cnt, g.order);
}

// Fold the first 32 queued hits, all lanes active, and move the rest (nq - 32 < 32) to the front.
template <int F, class PosT>
__device__ __forceinline__ void fold_front(uint32_t& nq, const GraphDev& g, const SurveyArgs& a,
                                           const QTable<PosT>& T, const InStage& S, const HitQueue& H,
                                           const TriMeta& t, MirrorWord* s_tab, unsigned long long* grec,
                                           unsigned long long& cnt) {
    const uint32_t lane = threadIdx.x & 31;
    __syncwarp();
    fold_queue<F>(g, a, T, S, H, 0, 32, t, s_tab, grec, cnt);
    const uint32_t left = nq - 32;
    uint32_t mi = 0, mp = 0;
    if (lane < left) {
        mi = H.idx[32 + lane];
        mp = H.pk[32 + lane];
    }
    __syncwarp();
    if (lane < left) {
        H.idx[lane] = mi;
        H.pk[lane] = mp;
    }
    nq = left;
    __syncwarp();
}

// Queue the hits of this lane's quad -- pos[i] >= 0 for a hit at CSR position
// e0 + i of in-edge slot k -- and fold 32 queued hits whenever 32 are waiting.
// The warp's hits of a quad step enter the queue together (each lane writes its
// own after those of the lanes below it) when they fit; otherwise, one quad
// position at a time.  Called by the whole warp; nq (< 32 on entry and exit)
// is warp-uniform.
template <int F, class PosT>
__device__ __forceinline__ void push_quad(const int (&pos)[4], uint32_t e0, uint32_t k, uint32_t& nq,
                                          const GraphDev& g, const SurveyArgs& a, const QTable<PosT>& T,
                                          const InStage& S, const HitQueue& H, const TriMeta& t,
                                          MirrorWord* s_tab, unsigned long long* grec,
                                          unsigned long long& cnt) {
    const uint32_t lane = threadIdx.x & 31;
    const uint32_t lt = (1u << lane) - 1u;
    {
        uint32_t total = 0, below = 0;
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const unsigned b = __ballot_sync(0xffffffffu, pos[i] >= 0);
            total += __popc(b);
            below += __popc(b & lt);
        }
        if (total == 0) return;
        if (nq + total <= (uint32_t)kHitQ) {
            uint32_t slot = nq + below;
#pragma unroll
            for (int i = 0; i < 4; ++i)
                if (pos[i] >= 0) {
                    H.idx[slot] = e0 + i;
                    H.pk[slot] = (uint32_t)pos[i] | (k << 16);
                    ++slot;
                }
            nq += total;
            while (nq >= 32) fold_front<F>(nq, g, a, T, S, H, t, s_tab, grec, cnt);
            return;
        }
    }
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const unsigned b = __ballot_sync(0xffffffffu, pos[i] >= 0);
        if (!b) continue;
        if (pos[i] >= 0) {
            const uint32_t slot = nq + __popc(b & lt);
            H.idx[slot] = e0 + i;
            H.pk[slot] = (uint32_t)pos[i] | (k << 16);
        }
        nq += __popc(b);
        if (nq >= 32) fold_front<F>(nq, g, a, T, S, H, t, s_tab, grec, cnt);
    }
}

// The calling warp checks the flat unit indices [f_begin, f_end) of the item
// in consecutive chunks of 32*kUnroll units: lane l takes units f0 + 32u + l,
// so consecutive lanes read consecutive 32-byte units of a pivot suffix
// (coalesced), and each probes the unit's candidates r in the table of q, a
// 16-byte quad at a time.
// The in-edge slots a chunk spans are found from the previous chunk's with
// one ballot.  Hits are queued and folded 32 at a time, one per lane.
template <int F, bool BM, class PosT>
__device__ __forceinline__ void scan_flat(const GraphDev& g, const SurveyArgs& a, const QTable<PosT>& T,
                                          const RankBitmap& B, const InStage& S, const HitQueue& H, uint32_t n_in,
                                          uint32_t f_begin, uint32_t f_end, uint32_t qbase, uint32_t q, uint32_t l_q,
                                          uint32_t d_q, MirrorWord* s_tab, unsigned long long* grec,
                                          unsigned long long& cnt) {
    const uint32_t lane = threadIdx.x & 31;
    TriMeta t = {};
    t.l_q = l_q;
    t.d_q = d_q;
    t.q = q;
    t.qbase = qbase;
    uint32_t nq = 0;   // queued hits (warp-uniform)
    uint32_t klo = 0;  // slot holding the chunk's first unit
    {
        uint32_t kb = 0;
        if (lane == 0 && f_begin < f_end) kb = seg_of(S.pp, 0, n_in, f_begin);
        klo = __shfl_sync(0xffffffffu, kb, 0);
    }
    for (uint32_t f0 = f_begin; f0 < f_end; f0 += 32 * kUnroll) {
        // khi: first slot after klo whose prefix passes the chunk's last unit (pp[n_in] = total)
        const uint32_t fl = min(f0 + 32 * kUnroll - 1, f_end - 1);
        uint32_t khi = 0;
        for (uint32_t base = klo + 1;; base += 32) {
            const uint32_t sl = base + lane;
            const unsigned bm = __ballot_sync(0xffffffffu, sl > n_in || S.pp[sl] > fl);
            if (bm) {
                khi = base + __ffs(bm) - 1;
                break;
            }
        }
        uint4 v[kUnroll][kUnitQuads];
        uint32_t e0[kUnroll], lo[kUnroll], hi[kUnroll], ks[kUnroll];
#pragma unroll
        for (int u = 0; u < kUnroll; ++u) {
            const uint32_t f = f0 + 32 * u + lane;
            ks[u] = 0;
            lo[u] = 1;
            hi[u] = 0;  // empty unless f is in range
            e0[u] = 0;
            if (f < f_end) {
                const uint32_t k = seg_of(S.pp, klo, khi, f);
                const uint32_t j0 = S.j0[k];
                ks[u] = k;
                e0[u] = ((j0 >> kUnitLog) + (f - S.pp[k])) << kUnitLog;
                lo[u] = j0;
                hi[u] = S.jend[k];
#pragma unroll
                for (int c = 0; c < kUnitQuads; ++c)
                    v[u][c] = __ldg(reinterpret_cast<const uint4*>(g.col + e0[u]) + c);
            }
        }
#pragma unroll
        for (int u = 0; u < kUnroll; ++u) {
#pragma unroll
            for (int c = 0; c < kUnitQuads; ++c) {
                const uint32_t rr[4] = {v[u][c].x, v[u][c].y, v[u][c].z, v[u][c].w};
                const uint32_t ec = e0[u] + 4 * c;
                bool act[4];
#pragma unroll
                for (int i = 0; i < 4; ++i) act[i] = ec + i >= lo[u] && ec + i < hi[u];
                int pos[4];
                if (BM && B.span) probe_quad_bm(B, rr, act, pos);
                else probe_quad(T, rr, act, pos);
                push_quad<F>(pos, ec, ks[u], nq, g, a, T, S, H, t, s_tab, grec, cnt);
            }
        }
        klo = khi - 1;
    }
    if (nq) {
        __syncwarp();
        fold_queue<F>(g, a, T, S, H, 0, nq, t, s_tab, grec, cnt);
    }
    __syncwarp();
}

__device__ __forceinline__ unsigned long long* record_of(const GraphDev& g, const SurveyArgs& a, uint32_t q) {
    return g.graph_of ? a.out + (uint64_t)g.graph_of[q] * a.lay.words : a.out;
}

template <int F>
__device__ void flush_shared(MirrorWord* s_tab, uint32_t s_words, unsigned long long* out) {
    for (uint32_t w = threadIdx.x; w < s_words; w += blockDim.x)
        if (s_tab[w]) atomicAdd(&out[w], (unsigned long long)s_tab[w]);
    if (F & F_CACHE) {
        const uint32_t* key = cache_keys(s_tab, s_words);
        const uint32_t* val = key + kCacheSlots;
        for (uint32_t i = threadIdx.x; i < kCacheSlots; i += blockDim.x)
            if (val[i]) atomicAdd(&out[key[i]], (unsigned long long)val[i]);
    }
}

// Clear the mirror (and the word cache) at kernel start; load the requests' bounds (F_MULTI) from
// the counters array: counters[4] = A, counters[5] = B, then the A lower and B upper bounds.
template <int F>
__device__ void init_shared(MirrorWord* s_tab, uint32_t s_words, const uint32_t* __restrict__ counters) {
    if (F & F_MULTI) {
        uint32_t* win = reinterpret_cast<uint32_t*>(s_tab) - kMultiWords;
        const uint32_t A = counters[4], B = counters[5];
        for (uint32_t i = threadIdx.x; i < kMultiWords; i += blockDim.x) {
            uint32_t v = 0;
            if (i < 2) v = counters[4 + i];
            else if (i >= 4 && i < 4 + A) v = counters[6 + (i - 4)];
            else if (i >= 4 + kMultiMax && i < 4 + kMultiMax + B) v = counters[6 + A + (i - 4 - kMultiMax)];
            win[i] = v;
        }
    }
    for (uint32_t w = threadIdx.x; w < s_words; w += blockDim.x) s_tab[w] = 0;
    if (F & F_CACHE) {
        uint32_t* key = cache_keys(s_tab, s_words);
        for (uint32_t i = threadIdx.x; i < kCacheSlots; i += blockDim.x) {
            key[i] = kEmpty;
            key[kCacheSlots + i] = 0;
        }
    }
}

// Bytes of dynamic shared memory ahead of a kernel's own arrays: the mirror, and the cache.
template <int F>
__host__ __device__ constexpr uint32_t mirror_bytes(uint32_t s_words) {
    return (F & F_CACHE) ? ((s_words + 3) & ~3u) * 4 + 2 * kCacheSlots * 4 : (s_words * 4 + 15) & ~15u;
}

__device__ void flush_count(unsigned long long cnt, const SurveyArgs& a, MirrorWord* s_tab,
                            unsigned long long* grec) {
    for (int o = 16; o; o >>= 1) cnt += __shfl_xor_sync(0xffffffffu, cnt, o);
    if ((threadIdx.x & 31) == 0 && cnt && a.lay.o_count != ~0u) atomicAdd(&grec[a.lay.o_count], cnt);
}

// ---- block kernel: one item per block at a time ---------------------------------------------

// dynamic shared memory of the block kernel after the record mirror, for
// staged parts of up to CHUNK entries in a table of 3*CHUNK slots (the degree
// array of staged entries only for kinds that use degrees)
template <int F, uint32_t CHUNK>
constexpr size_t block_smem_fixed() {
    return kWarps * kHitQ * 8 + kTableFactor * CHUNK * 4 + CHUNK * 4 * ((F & F_EXTRA) ? 2 : 1) +
           kTableFactor * CHUNK * 2 +
           CHUNK * (((F & F_EL) ? 1 : 0) + ((F & F_VL) ? 1 : 0)) + kBlockInEdges * 4 * ((F & F_EXTRA) ? 6 : 4) +
           (kBlockInEdges + 1) * 4;
}

// CTR selects the item counter: 1 for the kBlockChunk list, 2 for the kBigChunk list.
template <int F, uint32_t CHUNK, int CTR>
__global__ void __launch_bounds__(kBlockThreads, CHUNK <= kBlockChunk ? 5 : 3)
    survey_block_kernel(GraphDev g, const WorkItem* __restrict__ items,
                                                                     uint32_t n_items, SurveyArgs a) {
    constexpr uint32_t kBlockTable = kTableFactor * CHUNK;
    // the rank bitmap and its prefix share the table's key array; each thread's words are consecutive
    constexpr uint32_t kBmPerThread = kBlockTable / 2 / kBlockThreads;
    constexpr uint32_t kBmWords = kBmPerThread * kBlockThreads;
    extern __shared__ __align__(16) unsigned char smem[];
    static_assert(kBlockThreads == prim::kThreads, "block scan width");
    __shared__ uint32_t scan_tmp[kWarps];
    __shared__ uint32_t s_item, s_total;

    MirrorWord* s_tab = reinterpret_cast<MirrorWord*>(smem + multi_bytes<F>());
    unsigned char* base = smem + multi_bytes<F>() + mirror_bytes<F>(a.s_words);
    QTable<uint16_t> T;
    T.key = reinterpret_cast<uint32_t*>(base);
    T.ts = T.key + kBlockTable;
    T.deg = T.ts + CHUNK;  // present only with F_EXTRA
    InStage S;
    S.j0 = T.deg + ((F & F_EXTRA) ? CHUNK : 0);
    S.jend = S.j0 + kBlockInEdges;
    S.tpq = S.jend + kBlockInEdges;
    S.meta = S.tpq + kBlockInEdges;
    S.p = S.meta + kBlockInEdges;  // present only with F_EXTRA
    S.e = S.p + ((F & F_EXTRA) ? kBlockInEdges : 0);  // present only with F_EXTRA
    S.pp = S.e + ((F & F_EXTRA) ? kBlockInEdges : 0);
    uint32_t* hq = S.pp + kBlockInEdges + 1;
    HitQueue H;
    H.idx = hq + (threadIdx.x >> 5) * 2 * kHitQ;
    H.pk = H.idx + kHitQ;
    T.pos = reinterpret_cast<uint16_t*>(hq + kWarps * 2 * kHitQ);
    T.el = reinterpret_cast<uint8_t*>(T.pos + kBlockTable);  // present only with F_EL
    T.vl = T.el + ((F & F_EL) ? CHUNK : 0);                  // present only with F_VL

    init_shared<F>(s_tab, a.s_words, a.counters);
    unsigned long long cnt = 0;
    unsigned long long* grec_prev = nullptr;
    uint32_t taken = 0;  // items this block has taken (block-uniform)

    while (true) {
        if (threadIdx.x == 0) s_item = atomicAdd(&a.counters[CTR], 1u);
        __syncthreads();  // also: the previous item's table and stage are no longer read
        if (s_item >= n_items) break;
        if ((++taken & ((1u << a.move_block_log2) - 1u)) == 0 && threadIdx.x < 32)
            move_mirror_warp<F>(s_tab, a.s_words, a.out);
        const uint32_t it = n_items - 1 - s_item;  // high positions first: the hubs' long items start early
        const WorkItem item = items[it];
        const uint32_t q = item.q;
        unsigned long long* grec = record_of(g, a, q);
        if (grec != grec_prev && grec_prev) {  // batched: counts belong to the previous graph
            flush_count(cnt, a, s_tab, grec_prev);
            cnt = 0;
        }
        grec_prev = grec;
        uint32_t qbase = item.vpos;
        uint32_t len = item.qlen;
        uint32_t in_lo = item.in_lo, in_hi = item.in_hi;
        if (g.vidx) {  // the item's part of Adj+(q) in the window view
            const uint32_t b0 = view_pos(g.vidx, qbase);
            len = view_pos(g.vidx, qbase + len) - b0;
            qbase = b0;
            if (g.iidx) {  // and its in-window in-edges
                in_lo = view_pos(g.iidx, in_lo);
                in_hi = view_pos(g.iidx, in_hi);
            }
            if (len == 0 || in_lo == in_hi) {  // no in-window (q,r) or (p,q): no triangle; s_item is read by
                __syncthreads();                // all before it changes
                continue;
            }
        }
        const bool chunked = item.flags & 1u;
        const uint32_t first = __ldg(&g.col[qbase]), last = __ldg(&g.col[qbase + len - 1]);
        const uint32_t vlo = chunked ? first : 0u;
        const uint32_t vhi = chunked ? last : 0xFFFFFFFFu;
        // a rank bitmap when the part's values span few positions and every entry is staged (a window view,
        // or no window); else the hash table
        RankBitmap B{T.key, T.key + kBmWords, first, last - first + 1};
        if (!(g.vidx || (a.t_lo == 0 && a.t_hi == 0xFFFFFFFFu)) || B.span > kBmWords * 32u) B.span = 0;
        if (B.span) {
            uint32_t* bm = T.key;
            uint32_t* pre = T.key + kBmWords;
            const uint32_t nw = (B.span + 31) >> 5;
            for (uint32_t w = threadIdx.x; w < nw; w += blockDim.x) bm[w] = 0;
            __syncthreads();
            for (uint32_t i = threadIdx.x; i < len; i += blockDim.x) {
                const uint32_t r = __ldg(&g.col[qbase + i]);
                atomicOr(&bm[(r - first) >> 5], 1u << ((r - first) & 31u));
                if (F & F_TS) T.ts[i] = __ldg(&g.ts[qbase + i]);
                if (F & F_EL) T.el[i] = __ldg(&g.el[qbase + i]);
                if (F & F_VL) T.vl[i] = __ldg(&g.vl[r]);
                if (F & F_EXTRA) T.deg[i] = __ldg(&g.deg[r]);
            }
            __syncthreads();
            // pre: set bits before each word; a thread takes kBmPerThread consecutive words
            const uint32_t w0 = threadIdx.x * kBmPerThread;
            uint32_t c = 0;
#pragma unroll
            for (uint32_t j = 0; j < kBmPerThread; ++j) c += (w0 + j < nw) ? __popc(bm[w0 + j]) : 0u;
            uint32_t total_bits;
            uint32_t run = prim::block_exclusive_scan(c, scan_tmp, &total_bits);
#pragma unroll
            for (uint32_t j = 0; j < kBmPerThread; ++j)
                if (w0 + j < nw) {
                    pre[w0 + j] = run;
                    run += __popc(bm[w0 + j]);
                }
        } else {
            T.size = view_table_size(len, g.vidx != nullptr, kBlockTable);
            const uint32_t tsize = T.size;
            for (uint32_t i = threadIdx.x; i < tsize; i += blockDim.x) T.key[i] = kEmpty;
            __syncthreads();
            table_fill<F>(g, a, T, qbase, len, threadIdx.x, blockDim.x);
        }
        const uint32_t l_q = (F & F_VL) ? __ldg(&g.vl[q]) : 0u;
        const uint32_t d_q = (F & F_EXTRA) ? __ldg(&g.deg[q]) : 0u;
        const uint32_t warp = threadIdx.x >> 5;
        // the table stays; the item's in-edges are staged and scanned kBlockInEdges at a time
        for (uint32_t g0 = in_lo; g0 < in_hi; g0 += kBlockInEdges) {
            if (g0 != in_lo) __syncthreads();  // the previous group's stage is no longer read
            const uint32_t n_in = min(kBlockInEdges, in_hi - g0);
            uint32_t np = 0;
            if (threadIdx.x < n_in) np = stage_in_edge<F>(g, a, S, threadIdx.x, g0 + threadIdx.x, chunked, vlo, vhi);
            uint32_t total;
            const uint32_t pre = prim::block_exclusive_scan(np, scan_tmp, &total);
            if (threadIdx.x < n_in) S.pp[threadIdx.x] = pre;
            if (threadIdx.x == 0) { S.pp[n_in] = total; s_total = total; }
            __syncthreads();
            const uint32_t f_begin = (uint32_t)(((uint64_t)s_total * warp) / kWarps);
            const uint32_t f_end = (uint32_t)(((uint64_t)s_total * (warp + 1)) / kWarps);
            scan_flat<F, true>(g, a, T, B, S, H, n_in, f_begin, f_end, qbase, q, l_q, d_q, s_tab, grec, cnt);
        }
    }
    if (grec_prev) flush_count(cnt, a, s_tab, grec_prev);
    __syncthreads();
    flush_shared<F>(s_tab, a.s_words, a.out);
}

// ---- warp kernel: one item per warp at a time ------------------------------------------------

constexpr uint32_t kWTable = kTableFactor * kWarpMaxQ;
struct __align__(16) WarpSmem {
    uint32_t key[kWTable];
    uint32_t ts[kWarpMaxQ];
    uint32_t deg[kWarpMaxQ];
    uint32_t j0[kWarpInEdges], jend[kWarpInEdges], tpq[kWarpInEdges], meta[kWarpInEdges], p[kWarpInEdges];
    uint32_t e[kWarpInEdges];
    uint32_t pp[kWarpInEdges + 1];
    uint32_t qidx[kHitQ], qpk[kHitQ];
    uint8_t pos[kWTable];
    uint8_t el[kWarpMaxQ];
    uint8_t vl[kWarpMaxQ];
};

// 5 resident blocks per SM, like the block kernel (the register cap that sets)
template <int F>
__global__ void __launch_bounds__(kBlockThreads, 5) survey_warp_kernel(GraphDev g, const WorkItem* __restrict__ items,
                                                                    uint32_t n_items, SurveyArgs a) {
    extern __shared__ __align__(16) unsigned char smem[];
    MirrorWord* s_tab = reinterpret_cast<MirrorWord*>(smem + multi_bytes<F>());
    WarpSmem* ws_all = reinterpret_cast<WarpSmem*>(smem + multi_bytes<F>() + mirror_bytes<F>(a.s_words));
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    WarpSmem& ws = ws_all[warp];
    init_shared<F>(s_tab, a.s_words, a.counters);
    __syncthreads();
    QTable<uint8_t> T;
    T.key = ws.key; T.pos = ws.pos; T.ts = ws.ts; T.deg = ws.deg; T.el = ws.el; T.vl = ws.vl;
    InStage S;
    S.j0 = ws.j0; S.jend = ws.jend; S.tpq = ws.tpq; S.meta = ws.meta; S.p = ws.p; S.e = ws.e; S.pp = ws.pp;
    unsigned long long cnt = 0;
    unsigned long long* grec_prev = nullptr;
    uint32_t taken = 0;  // items this warp has taken (warp-uniform)

    // each warp claims its next item while it surveys the current one
    uint32_t next = 0;
    if (lane == 0) next = atomicAdd(&a.counters[0], 1u);
    while (true) {
        const uint32_t it = __shfl_sync(0xffffffffu, next, 0);
        if (it >= n_items) break;
        if (lane == 0) next = atomicAdd(&a.counters[0], 1u);
        if ((++taken & ((1u << a.move_warp_log2) - 1u)) == 0) move_mirror_warp<F>(s_tab, a.s_words, a.out);
        const WorkItem item = items[it];
        const uint32_t q = item.q;
        unsigned long long* grec = record_of(g, a, q);
        if (grec != grec_prev && grec_prev) {
            flush_count(cnt, a, s_tab, grec_prev);
            cnt = 0;
        }
        grec_prev = grec;
        uint32_t qbase = item.vpos;
        uint32_t len = item.qlen;
        uint32_t in_lo = item.in_lo, in_hi = item.in_hi;
        if (g.vidx && !a.view_items) {  // Adj+(q) in the window view
            const uint32_t b0 = view_pos(g.vidx, qbase);
            len = view_pos(g.vidx, qbase + len) - b0;
            qbase = b0;
            if (g.iidx) {  // and its in-window in-edges
                in_lo = view_pos(g.iidx, in_lo);
                in_hi = view_pos(g.iidx, in_hi);
            }
            if (len == 0 || in_lo == in_hi) continue;  // no in-window (q,r) or (p,q): no triangle
        }
        const uint32_t l_q = (F & F_VL) ? __ldg(&g.vl[q]) : 0u;
        const uint32_t d_q = (F & F_EXTRA) ? __ldg(&g.deg[q]) : 0u;
        const uint32_t n_in = in_hi - in_lo;
        const bool chunked = len > kWarpMaxQ;
        // the out-list is staged kWarpMaxQ entries at a time (one part unless the window
        // leaves more in it); each part restricts the suffixes to its value range
        for (uint32_t c0 = 0; c0 < len; c0 += kWarpMaxQ) {
            const uint32_t clen = min(kWarpMaxQ, len - c0);
            T.size = view_table_size(clen, g.vidx != nullptr, kWTable);
            const uint32_t tsize = T.size;
            __syncwarp();
            for (uint32_t i = lane; i < tsize; i += 32) ws.key[i] = kEmpty;
            __syncwarp();
            table_fill<F>(g, a, T, qbase + c0, clen, lane, 32);
            const uint32_t vlo = chunked ? __ldg(&g.col[qbase + c0]) : 0u;
            const uint32_t vhi = chunked ? __ldg(&g.col[qbase + c0 + clen - 1]) : 0xFFFFFFFFu;
            uint32_t np0 = 0, np1 = 0;
            if ((uint32_t)lane < n_in) np0 = stage_in_edge<F>(g, a, S, lane, in_lo + lane, chunked, vlo, vhi);
            if ((uint32_t)lane + 32 < n_in)
                np1 = stage_in_edge<F>(g, a, S, lane + 32, in_lo + lane + 32, chunked, vlo, vhi);
            // exclusive prefix over slots 0..63 held as (lane, lane + 32)
            uint32_t x0 = np0, x1 = np1;
            for (int o = 1; o < 32; o <<= 1) {
                uint32_t y0 = __shfl_up_sync(0xffffffffu, x0, o), y1 = __shfl_up_sync(0xffffffffu, x1, o);
                if (lane >= o) { x0 += y0; x1 += y1; }
            }
            const uint32_t half = __shfl_sync(0xffffffffu, x0, 31);
            const uint32_t total = half + __shfl_sync(0xffffffffu, x1, 31);
            if ((uint32_t)lane < n_in) ws.pp[lane] = x0 - np0;
            if ((uint32_t)lane + 32 < n_in) ws.pp[lane + 32] = half + x1 - np1;
            if (lane == 0) ws.pp[n_in] = total;
            __syncwarp();
            HitQueue H;
            H.idx = ws.qidx;
            H.pk = ws.qpk;
            scan_flat<F, false>(g, a, T, RankBitmap{nullptr, nullptr, 0u, 0u}, S, H, n_in, 0, total, qbase + c0, q,
                                l_q, d_q, s_tab, grec, cnt);
        }
    }
    if (grec_prev) flush_count(cnt, a, s_tab, grec_prev);
    __syncthreads();
    flush_shared<F>(s_tab, a.s_words, a.out);
}

}  // namespace

// Record phase boundary k of a timed survey (no-op for an untimed one).
inline void mark(cudaEvent_t* ev, int k, cudaStream_t s) {
    if (ev) cudaEventRecord(ev[k], s);
}

template <int F>
void launch_f(const ItemLists& L, const GraphDev& gd, const SurveyArgs& a, cudaStream_t s, int sms,
              cudaEvent_t* ev) {
    mark(ev, 1, s);
    if (L.n[0]) {
        size_t sm = multi_bytes<F>() + mirror_bytes<F>(a.s_words) + kWarps * sizeof(WarpSmem);
        const int per = blocks_per_sm((const void*)survey_warp_kernel<F>, sm);
        uint64_t blocks = (uint64_t)per * sms;
        blocks = std::min<uint64_t>(blocks, (L.n[0] + kWarps - 1) / kWarps);
        survey_warp_kernel<F><<<(unsigned)blocks, kBlockThreads, sm, s>>>(gd, L.items[0],
                                                                         (uint32_t)L.n[0], a); ::tp::note_launch();
    }
    mark(ev, 2, s);
    if (L.n[1]) {
        size_t sm = multi_bytes<F>() + mirror_bytes<F>(a.s_words) + block_smem_fixed<F, kBlockChunk>();
        const int per = blocks_per_sm((const void*)survey_block_kernel<F, kBlockChunk, 1>, sm);
        uint64_t blocks = std::min<uint64_t>((uint64_t)per * sms, L.n[1]);
        survey_block_kernel<F, kBlockChunk, 1><<<(unsigned)blocks, kBlockThreads, sm, s>>>(
            gd, L.items[1], (uint32_t)L.n[1], a); ::tp::note_launch();
    }
    mark(ev, 3, s);
    if (L.n[2]) {
        size_t sm = multi_bytes<F>() + mirror_bytes<F>(a.s_words) + block_smem_fixed<F, kBigChunk>();
        const int per = blocks_per_sm((const void*)survey_block_kernel<F, kBigChunk, 2>, sm);
        uint64_t blocks = std::min<uint64_t>((uint64_t)per * sms, L.n[2]);
        survey_block_kernel<F, kBigChunk, 2><<<(unsigned)blocks, kBlockThreads, sm, s>>>(
            gd, L.items[2], (uint32_t)L.n[2], a); ::tp::note_launch();
    }
    mark(ev, 4, s);
}

using LaunchFn = void (*)(const ItemLists&, const GraphDev&, const SurveyArgs&, cudaStream_t, int, cudaEvent_t*);

}  // namespace sv
}  // namespace tp

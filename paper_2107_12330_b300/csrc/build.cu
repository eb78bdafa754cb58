// build.cu -- on-device construction of G+ (TriPoll Sec. 3 and Sec. 4.2).
//
// Steps, all on the caller's stream:
//   validate   ids < n (per graph when batched), labels < L
//   canon      (u,v) -> key (min,max) packed in 2b bits, loops -> sentinel key;
//              payload (ts << 8 | elabel)
//   sort       radix sort of (key, payload) pairs
//   dedup      min payload per key run: the chronologically first record of
//              each unordered pair (Sec. 5.2), edge label as tie-break
//   degree     d(v) of the simple graph
//   order      vertices sorted by (graph, degree, id): the order <+ of Sec. 3
//              with the id as tie-break, per graph when batched
//   orient     every edge directed from the <+ -smaller end; sorted by
//              (source position, target position): the out-lists Adj+ (CSR)
//              with timestamps and edge labels aligned to them (Adj+^m)
//   in-edges   16-byte records of the same edges, stably sorted by target: for
//              every middle vertex q the directed edges (p,q) that end at it
//   stats      |E+|, |W+| = sum C(d+,2), d+ max, ...
#include <algorithm>
#include <utility>
#include <vector>

#include "common.cuh"
#include "primitives.cuh"

namespace tp {
namespace {

constexpr int kThreads = 256;

unsigned grid_for(uint64_t items, unsigned cap = 148u * 64u) {
    uint64_t b = (items + kThreads - 1) / kThreads;
    if (b < 1) b = 1;
    return (unsigned)std::min<uint64_t>(b, cap);
}

int bits_for(uint64_t x) {  // bits to hold values 0..x
    int b = 1;
    while (b < 64 && (x >> b) != 0) ++b;
    return b;
}

__device__ __forceinline__ uint32_t graph_of_edge(const uint64_t* eoff, uint32_t G, uint64_t i) {
    // largest g with eoff[g] <= i
    uint32_t lo = 0, hi = G - 1;
    while (lo < hi) {
        uint32_t mid = (lo + hi + 1) >> 1;
        if (eoff[mid] <= i) lo = mid; else hi = mid - 1;
    }
    return lo;
}

// The records of a batch are grouped by graph, many to a graph.  Giving each block one contiguous
// range of records lets a thread find the graph of its first record by binary search once and then
// step forward over graph boundaries as its record index grows, instead of searching per record.
__device__ __forceinline__ void block_records(uint64_t m, uint64_t& lo, uint64_t& hi) {
    uint64_t per = (m + gridDim.x - 1) / gridDim.x;
    per = (per + blockDim.x - 1) / blockDim.x * blockDim.x;  // warps stay aligned to 32 records
    lo = min(m, (uint64_t)blockIdx.x * per);
    hi = min(m, lo + per);
}

struct GraphCursor {
    const uint64_t* eoff;  // G + 1 record offsets, eoff[G] = total records; null for one graph
    uint32_t g;
    __device__ GraphCursor(const uint64_t* e, uint32_t G, uint64_t i) : eoff(e), g(0) {
        if (e && G) g = graph_of_edge(e, G, i);
    }
    // graph of record i, for non-decreasing i below eoff[G]
    __device__ __forceinline__ uint32_t at(uint64_t i) {
        while (eoff[g + 1] <= i) ++g;
        return g;
    }
};

__global__ void validate_edges_kernel(const uint32_t* __restrict__ src, const uint32_t* __restrict__ dst,
                                      const uint8_t* __restrict__ el, uint64_t m, uint32_t n,
                                      const uint64_t* __restrict__ eoff, const uint32_t* __restrict__ nv,
                                      uint32_t G, uint32_t Le, unsigned* flags) {
    unsigned f = 0;
    uint64_t lo, hi;
    block_records(m, lo, hi);
    GraphCursor gc(eoff, G, lo + threadIdx.x);
    for (uint64_t i = lo + threadIdx.x; i < hi; i += blockDim.x) {
        uint32_t lim = n;
        if (eoff) lim = nv[gc.at(i)];
        if (src[i] >= lim || dst[i] >= lim) f |= 1u;
        if (el && el[i] >= Le) f |= 2u;
    }
    if (f) atomicOr(flags, f);
}

__global__ void validate_vl_kernel(const uint8_t* __restrict__ vl, uint64_t n, uint32_t Lv, unsigned* flags) {
    unsigned f = 0;
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n;
         i += (uint64_t)gridDim.x * blockDim.x)
        if (vl[i] >= Lv) f |= 4u;
    if (f) atomicOr(flags, f);
}

// Records of the sorts: the pair key in the low 2b bits of a 64-bit word and the payload
// (ts << 8 | elabel) split between the word and a value of type V (prim::rec_word).
template <class V>
__global__ void canon_kernel(const uint32_t* __restrict__ src, const uint32_t* __restrict__ dst,
                             const uint32_t* __restrict__ ts, const uint8_t* __restrict__ el, uint64_t m,
                             const uint64_t* __restrict__ eoff, const uint64_t* __restrict__ vbase, uint32_t G,
                             int b, uint64_t sentinel, uint64_t* __restrict__ key, V* __restrict__ val) {
    uint64_t lo, hi;
    block_records(m, lo, hi);
    GraphCursor gc(eoff, G, lo + threadIdx.x);
    for (uint64_t i = lo + threadIdx.x; i < hi; i += blockDim.x) {
        uint64_t u = src[i], v = dst[i];
        if (eoff) {
            uint64_t base = vbase[gc.at(i)];
            u += base;
            v += base;
        }
        uint64_t lo = u < v ? u : v, hi = u < v ? v : u;
        const uint64_t payload = ((uint64_t)ts[i] << 8) | (el ? el[i] : 0u);
        key[i] = prim::rec_word<V>((u == v) ? sentinel : ((lo << b) | hi), payload, 2 * b);
        val[i] = (V)payload;
    }
}

__global__ void unique_count_kernel(const uint64_t* ukey, const uint64_t* runs, uint64_t sentinel, uint64_t* m_out) {
    uint64_t r = *runs;
    if (r > 0 && ukey[r - 1] == sentinel) r -= 1;
    *m_out = r;
}

// Degrees of the simple graph.  Keys are sorted, so the lanes of a warp mostly
// share the smaller endpoint: those increments are aggregated per warp.
__global__ void degree_kernel(const uint64_t* __restrict__ ukey, uint64_t m, int b, uint32_t* __restrict__ deg) {
    const uint64_t mask = (1ull << b) - 1;
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t base = blockIdx.x * (uint64_t)blockDim.x; base < m; base += stride) {
        const uint64_t i = base + threadIdx.x;
        const bool ok = i < m;
        const uint64_t k = ok ? ukey[i] : 0;
        const unsigned act = __ballot_sync(0xffffffffu, ok);
        if (ok) {
            const uint32_t u = (uint32_t)(k >> b);
            const unsigned grp = __match_any_sync(act, u);
            if ((int)(threadIdx.x & 31) == __ffs(grp) - 1) atomicAdd(&deg[u], (uint32_t)__popc(grp));
            atomicAdd(&deg[k & mask], 1u);
        }
    }
}

__global__ void max_u32_kernel(const uint32_t* __restrict__ x, uint64_t n, unsigned* out) {
    unsigned mx = 0;
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n;
         i += (uint64_t)gridDim.x * blockDim.x)
        mx = max(mx, x[i]);
    for (int o = 16; o; o >>= 1) mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    if ((threadIdx.x & 31) == 0 && mx) atomicMax(out, mx);
}

__global__ void vertex_key_kernel(const uint32_t* __restrict__ deg, uint64_t n, const uint64_t* __restrict__ vbase,
                                  uint32_t G, int b, int bd, uint64_t* __restrict__ vkey) {
    for (uint64_t v = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; v < n;
         v += (uint64_t)gridDim.x * blockDim.x) {
        uint64_t g = 0;
        if (vbase) {  // largest g with vbase[g] <= v
            uint32_t lo = 0, hi = G - 1;
            while (lo < hi) {
                uint32_t mid = (lo + hi + 1) >> 1;
                if (vbase[mid] <= v) lo = mid; else hi = mid - 1;
            }
            g = lo;
        }
        vkey[v] = (g << (bd + b)) | ((uint64_t)deg[v] << b) | v;
    }
}

__global__ void rank_kernel(const uint64_t* __restrict__ vkey, uint64_t n, int b, uint32_t* __restrict__ rank,
                            uint32_t* __restrict__ order, const uint32_t* __restrict__ deg,
                            uint32_t* __restrict__ deg_pos, int gshift, uint32_t* __restrict__ graph_of) {
    const uint64_t mask = (1ull << b) - 1;
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n;
         i += (uint64_t)gridDim.x * blockDim.x) {
        uint64_t k = vkey[i];
        uint32_t v = (uint32_t)(k & mask);
        rank[v] = (uint32_t)i;
        order[i] = v;
        deg_pos[i] = deg[v];
        if (graph_of) graph_of[i] = (uint32_t)(k >> gshift);
    }
}

template <class V>
__global__ void orient_kernel(const uint64_t* __restrict__ ukey, const uint64_t* __restrict__ uval, uint64_t m, int b,
                              const uint32_t* __restrict__ rank, uint64_t* __restrict__ okey, V* __restrict__ oval) {
    const uint64_t mask = (1ull << b) - 1;
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < m;
         i += (uint64_t)gridDim.x * blockDim.x) {
        uint64_t k = ukey[i];
        uint64_t ru = rank[k >> b], rv = rank[k & mask];
        uint64_t s = ru < rv ? ru : rv, d = ru < rv ? rv : ru;
        const uint64_t payload = uval[i];
        okey[i] = prim::rec_word<V>((s << b) | d, payload, 2 * b);
        oval[i] = (V)payload;
    }
}

// Runs of equal ((key & kmask) >> shift) in keys sorted ascending: first[v] and last[v]
// get the run of value v as [first, last) (both left 0 for absent values), so
// that last - first counts the keys of v without atomics.
template <class K>
__global__ void run_ends_kernel(const K* __restrict__ key, uint64_t m, uint64_t kmask, int shift,
                                uint32_t* __restrict__ first, uint32_t* __restrict__ last) {
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < m;
         i += (uint64_t)gridDim.x * blockDim.x) {
        const uint64_t v = ((uint64_t)key[i] & kmask) >> shift;
        if (i == 0 || (((uint64_t)key[i - 1] & kmask) >> shift) != v) first[v] = (uint32_t)i;
        if (i + 1 == m || (((uint64_t)key[i + 1] & kmask) >> shift) != v) last[v] = (uint32_t)(i + 1);
    }
}

__global__ void run_count_kernel(const uint32_t* __restrict__ first, uint32_t* __restrict__ last_cnt, uint64_t n) {
    for (uint64_t v = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; v < n; v += (uint64_t)gridDim.x * blockDim.x)
        last_cnt[v] -= first[v];
}

// CSR arrays of G+ from the (source, target)-sorted edges, plus, in the same
// order, the in-edge record of every edge and the key of the in-edge order
// (the target alone: a stable sort on it keeps sources ascending).
template <class V>
__global__ void csr_fill_kernel(const uint64_t* __restrict__ okey, const V* __restrict__ oval, uint64_t m,
                                int b, const uint64_t* __restrict__ off, const uint8_t* __restrict__ vl,
                                uint32_t* __restrict__ col, uint32_t* __restrict__ ts, uint8_t* __restrict__ el,
                                InEdge* __restrict__ rec, uint32_t* __restrict__ ckey, uint32_t* __restrict__ cpos) {
    const uint64_t mask = (1ull << b) - 1;
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < m;
         i += (uint64_t)gridDim.x * blockDim.x) {
        const uint64_t w = okey[i];
        const uint64_t k = prim::rec_key<V>(w, 2 * b), v = prim::rec_payload<V>(w, oval[i], 2 * b);
        const uint32_t s = (uint32_t)(k >> b), d = (uint32_t)(k & mask);
        const uint32_t t = (uint32_t)(v >> 8), l = (uint32_t)(v & 0xffu);
        col[i] = d;
        ts[i] = t;
        if (el) el[i] = (uint8_t)l;
        InEdge ie;
        ie.e = (uint32_t)i;
        ie.end = (uint32_t)off[s + 1];
        ie.ts = t;
        ie.meta = l | ((uint32_t)vl[s] << 8);
        rec[i] = ie;
        ckey[i] = d;
        cpos[i] = (uint32_t)i;
    }
}

// The in-edge records in (target, source) order: record k is the CSR-order record at the position
// the sort of (target, position) pairs left at k.
__global__ void gather_in_edges_kernel(const InEdge* __restrict__ csr_rec, const uint32_t* __restrict__ pos,
                                       uint64_t m, InEdge* __restrict__ out) {
    for (uint64_t k = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; k < m; k += (uint64_t)gridDim.x * blockDim.x)
        out[k] = csr_rec[pos[k]];
}

__global__ void vlabel_pos_kernel(const uint8_t* __restrict__ vl, const uint32_t* __restrict__ order, uint64_t n,
                                  uint8_t* __restrict__ vl_pos) {
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n;
         i += (uint64_t)gridDim.x * blockDim.x)
        vl_pos[i] = vl ? vl[order[i]] : 0;
}

// stats[0] = wedges, [1] = q_list_words, [2] = dplus_max, [3] = degree_max
__global__ void stats_kernel(const uint64_t* __restrict__ off, const uint64_t* __restrict__ in_off,
                             const uint32_t* __restrict__ deg, uint64_t n, unsigned long long* stats) {
    unsigned long long w = 0, ql = 0, dm = 0, gm = 0;
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n;
         i += (uint64_t)gridDim.x * blockDim.x) {
        uint64_t dp = off[i + 1] - off[i];
        uint64_t di = in_off[i + 1] - in_off[i];
        w += dp * (dp ? dp - 1 : 0) / 2;
        ql += dp * di;
        dm = max(dm, (unsigned long long)dp);
        gm = max(gm, (unsigned long long)deg[i]);
    }
    for (int o = 16; o; o >>= 1) {
        w += __shfl_xor_sync(0xffffffffu, w, o);
        ql += __shfl_xor_sync(0xffffffffu, ql, o);
        dm = max(dm, __shfl_xor_sync(0xffffffffu, dm, o));
        gm = max(gm, __shfl_xor_sync(0xffffffffu, gm, o));
    }
    if ((threadIdx.x & 31) == 0) {
        if (w) atomicAdd(&stats[0], w);
        if (ql) atomicAdd(&stats[1], ql);
        if (dm) atomicMax(&stats[2], dm);
        if (gm) atomicMax(&stats[3], gm);
    }
}

// off[0..n] = exclusive prefix of the run lengths of (key >> shift) over m
// keys sorted ascending (first, cnt: scratch of n + 1 words; scr: scan scratch
// of prim::scan_scratch_bytes(n + 1)).
template <class K>
int out_offsets(const K* key, uint64_t m, uint64_t kmask, int shift, uint64_t n, uint32_t* first, uint32_t* cnt,
                uint64_t* off, void* scr, cudaStream_t s) {
    TP_CUDA(cudaMemsetAsync(first, 0, (n + 1) * 4, s));
    TP_CUDA(cudaMemsetAsync(cnt, 0, (n + 1) * 4, s));
    if (m) {
        run_ends_kernel<K><<<grid_for(m), kThreads, 0, s>>>(key, m, kmask, shift, first, cnt); ::tp::note_launch();
        if (n) { run_count_kernel<<<grid_for(n), kThreads, 0, s>>>(first, cnt, n); ::tp::note_launch(); }
        TP_CUDA(cudaGetLastError());
    }
    return prim::scan<uint64_t, false>(prim::Load<uint32_t, uint64_t>{cnt, n + 1}, off, n + 1, scr, s);
}

// Device copy of a caller array that may live in host memory.
// Large pageable host arrays are page-locked in place for the copy (a DMA
// straight from the caller's pages instead of the driver's bounce buffers) and
// released once the stream has consumed them; page-locked arrays are copied as
// they are.
struct Input {
    const void* dptr = nullptr;
    Scratch copy;
    const void* pinned = nullptr;
    cudaStream_t stream = nullptr;
    int bind(const void* p, size_t bytes, cudaStream_t s) {
        if (!p) { dptr = nullptr; return TRIPOLL_OK; }
        if (is_device_pointer(p)) { dptr = p; return TRIPOLL_OK; }
        TP_CUDA(copy.alloc(bytes, s));
        if (bytes >= (size_t(64) << 20) && !is_pinned_host_pointer(p)) {
            if (cudaHostRegister(const_cast<void*>(p), bytes, cudaHostRegisterReadOnly) == cudaSuccess) {
                pinned = p;
                stream = s;
            } else {
                cudaGetLastError();  // already pinned or not registrable: the plain copy below still works
            }
        }
        TP_CUDA(cudaMemcpyAsync(copy.ptr, p, bytes, cudaMemcpyHostToDevice, s));
        dptr = copy.ptr;
        return TRIPOLL_OK;
    }
    ~Input() {
        if (pinned) {
            cudaStreamSynchronize(stream);
            cudaHostUnregister(const_cast<void*>(pinned));
        }
    }
};

struct GraphGuard {  // frees a half-built graph on any error path, after the stream's work
    tripoll_graph* g;
    cudaStream_t s;
    GraphGuard(tripoll_graph* g_, cudaStream_t s_) : g(g_), s(s_) {}
    ~GraphGuard() {
        if (g) {
            cudaStreamSynchronize(s);
            free_graph_arrays(g);
            delete g;
        }
    }
    tripoll_graph* release() { tripoll_graph* r = g; g = nullptr; return r; }
};

struct DedupIn {
    const uint32_t *src, *dst, *ts;
    const uint8_t* el;
    uint64_t m_in;
    const uint64_t *eoff, *vbase;
    uint32_t G;
    int b;
    uint64_t sentinel;
    uint32_t* fault;
};

// Step 2 with records of value type V: canonical records, their sort by pair, and the minimum
// payload of every run of equal pairs -- the chronologically first record (Sec. 5.2), label as
// the tie-break.  ukey/uval receive the unique pairs (sentinel last, if any loops) and payloads
// as 64-bit words; *m the number of unique pairs without loops.
template <class V, class Release>
int dedup(const DedupIn& in, Release release_inputs, Scratch& ukey_d, Scratch& uval_d, uint64_t* m_out,
          cudaStream_t s) {
    const uint64_t m_in = in.m_in;
    const int kb = std::min(64, 2 * in.b);
    Scratch k0, k1, v0, v1, scr, runs;
    TP_CUDA(k0.alloc(m_in * 8, s));
    TP_CUDA(k1.alloc(m_in * 8, s));
    TP_CUDA(v0.alloc(m_in * sizeof(V), s));
    TP_CUDA(v1.alloc(m_in * sizeof(V), s));
    if (m_in)
        canon_kernel<V><<<grid_for(m_in), kThreads, 0, s>>>(in.src, in.dst, in.ts, in.el, m_in, in.eoff, in.vbase, in.G,
                                                            in.b, in.sentinel, k0.as<uint64_t>(), v0.as<V>()); ::tp::note_launch();
    TP_CUDA(cudaGetLastError());
    release_inputs();
    const uint64_t tiles = (m_in + prim::kTile - 1) / prim::kTile;
    TP_CUDA(scr.alloc(std::max(prim::sort_scratch_bytes(m_in), tiles * 12 + prim::scan_scratch_bytes(tiles) + 512), s));
    bool alt = false;
    int rc = prim::radix_sort<uint64_t, V>(k0.as<uint64_t>(), k1.as<uint64_t>(), v0.as<V>(), v1.as<V>(), m_in, kb,
                                           scr.ptr, in.fault, s, &alt);
    if (rc) return rc;
    Scratch& kc = alt ? k1 : k0;  // sorted
    Scratch& vc = alt ? v1 : v0;
    Scratch& ku = alt ? k0 : k1;  // the unique keys go here
    (alt ? v0 : v1).release();    // the value buffer not holding the sorted values
    TP_CUDA(uval_d.alloc(m_in * 8, s));
    TP_CUDA(runs.alloc(16, s));
    TP_CUDA(cudaMemsetAsync(runs.ptr, 0, 16, s));
    if (m_in) {
        uint32_t* heads = scr.as<uint32_t>();
        uint64_t* tbase = reinterpret_cast<uint64_t*>(scr.as<unsigned char>() + (tiles * 4 + 255) / 256 * 256);
        void* sscr = reinterpret_cast<unsigned char*>(tbase) + (tiles * 8 + 255) / 256 * 256;
        prim::run_heads_kernel<V><<<(unsigned)tiles, prim::kThreads, 0, s>>>(kc.as<uint64_t>(), m_in, kb, heads); ::tp::note_launch();
        if ((rc = prim::scan<uint64_t, false>(prim::Load<uint32_t, uint64_t>{heads, tiles}, tbase, tiles, sscr, s,
                                              runs.as<uint64_t>())))
            return rc;
        TP_CUDA(cudaMemsetAsync(uval_d.ptr, 0xFF, m_in * 8, s));
        prim::run_min_kernel<V><<<(unsigned)tiles, prim::kThreads, 0, s>>>(
            kc.as<uint64_t>(), vc.as<V>(), m_in, kb, tbase, ku.as<uint64_t>(),
            uval_d.as<unsigned long long>()); ::tp::note_launch();
        TP_CUDA(cudaGetLastError());
    }
    unique_count_kernel<<<1, 1, 0, s>>>(ku.as<uint64_t>(), runs.as<uint64_t>(), in.sentinel, runs.as<uint64_t>() + 1); ::tp::note_launch();
    TP_CUDA(cudaGetLastError());
    TP_CUDA(cudaMemcpyAsync(m_out, runs.as<uint64_t>() + 1, 8, cudaMemcpyDeviceToHost, s));
    TP_CUDA(cudaStreamSynchronize(s));
    ukey_d.swap(ku);  // keep the unique keys; the other buffers go back when this returns
    return TRIPOLL_OK;
}

struct OrientIn {
    tripoll_graph* g;
    uint64_t m, n;
    int b;
    const uint32_t* rank;
    uint32_t *first, *cnt;
    void *sort_scr, *scan_scr;
    uint32_t* fault;
    uint32_t* ckey;  // out: target of every edge in CSR order (the key of the in-edge sort)
    uint32_t* cpos;  // out: the CSR position of every edge (the value of the in-edge sort)
    InEdge* rec;     // out: the in-edge records in CSR order
};

// Step 5 with records of value type V: every unique pair directed from its <+ -smaller end, sorted
// by (source, target) position, out-list offsets, the CSR arrays with timestamps and labels
// aligned (Adj+^m, Sec. 4.2), and the in-edge records in CSR order.  Releases ukey/uval/rank.
template <class V>
int orient_csr(const OrientIn& o, Scratch& ukey_d, Scratch& uval_d, Scratch& rank_d, cudaStream_t s) {
    tripoll_graph* g = o.g;
    const uint64_t m = o.m;
    const int kb = std::min(64, 2 * o.b);
    Scratch ok0, ok1, ov0, ov1;
    TP_CUDA(ok0.alloc(m * 8, s));
    TP_CUDA(ok1.alloc(m * 8, s));
    TP_CUDA(ov0.alloc(m * sizeof(V), s));
    TP_CUDA(ov1.alloc(m * sizeof(V), s));
    if (m)
        orient_kernel<V><<<grid_for(m), kThreads, 0, s>>>(ukey_d.as<uint64_t>(), uval_d.as<uint64_t>(), m, o.b, o.rank,
                                                          ok0.as<uint64_t>(), ov0.as<V>()); ::tp::note_launch();
    TP_CUDA(cudaGetLastError());
    ukey_d.release();
    uval_d.release();
    rank_d.release();
    bool alt = false;
    int rc = prim::radix_sort<uint64_t, V>(ok0.as<uint64_t>(), ok1.as<uint64_t>(), ov0.as<V>(), ov1.as<V>(), m, kb,
                                           o.sort_scr, o.fault, s, &alt);
    if (rc) return rc;
    const uint64_t* okey = alt ? ok1.as<uint64_t>() : ok0.as<uint64_t>();
    const V* oval = alt ? ov1.as<V>() : ov0.as<V>();
    // offsets: out-list lengths from the runs of equal sources (m < 2^32: 32-bit counts are exact)
    const uint64_t kmask = kb >= 64 ? ~0ull : ((1ull << kb) - 1);
    if ((rc = out_offsets(okey, m, kmask, o.b, o.n, o.first, o.cnt, g->off, o.scan_scr, s))) return rc;
    if (m)
        csr_fill_kernel<V><<<grid_for(m), kThreads, 0, s>>>(okey, oval, m, o.b, g->off, g->vl, g->col, g->ts, g->el,
                                                            o.rec, o.ckey, o.cpos); ::tp::note_launch();
    TP_CUDA(cudaGetLastError());
    return TRIPOLL_OK;
}

int build_impl(const uint32_t* src_h, const uint32_t* dst_h, const uint32_t* ts_h, const uint8_t* el_h,
               uint64_t m_in, const uint8_t* vl_h, uint64_t n, uint32_t Lv, uint32_t Le,
               const uint64_t* edge_offsets, const uint32_t* num_vertices, uint32_t G,
               cudaStream_t s, tripoll_graph_t* out) {
    if (!out) return fail(TRIPOLL_ERR_INVALID_ARG, "out handle is NULL");
    if (m_in > 0 && (!src_h || !dst_h || !ts_h)) return fail(TRIPOLL_ERR_INVALID_ARG, "src/dst/ts NULL");
    if (Lv == 0 || Lv > 256) return fail(TRIPOLL_ERR_INVALID_ARG, "num_vlabels must be in 1..256");
    if (el_h && (Le == 0 || Le > 256)) return fail(TRIPOLL_ERR_INVALID_ARG, "num_elabels must be in 1..256");
    if (n > 0xFFFFFFFFull) return fail(TRIPOLL_ERR_INVALID_ARG, "too many vertices for 32-bit ids");
    if (m_in >= (1ull << 40)) return fail(TRIPOLL_ERR_INVALID_ARG, "too many edge records");
    const bool batched = edge_offsets != nullptr;

    int dev = 0;
    TP_CUDA(cudaGetDevice(&dev));
    Input src, dst, ts, el, vl;
    int rc;
    if ((rc = src.bind(src_h, m_in * 4, s)) || (rc = dst.bind(dst_h, m_in * 4, s)) ||
        (rc = ts.bind(ts_h, m_in * 4, s)) || (rc = el.bind(el_h, m_in, s)) || (rc = vl.bind(vl_h, n, s)))
        return rc;

    // batched: per-graph edge offsets and vertex bases on the device
    std::vector<uint64_t> vbase_h;
    Scratch eoff_d, nv_d, vbase_d;
    if (batched) {
        vbase_h.resize(G + 1);
        vbase_h[0] = 0;
        for (uint32_t i = 0; i < G; ++i) vbase_h[i + 1] = vbase_h[i] + num_vertices[i];
        TP_CUDA(eoff_d.alloc((G + 1) * 8ull, s));
        TP_CUDA(nv_d.alloc(G * 4ull, s));
        TP_CUDA(vbase_d.alloc((G + 1) * 8ull, s));
        TP_CUDA(cudaMemcpyAsync(eoff_d.ptr, edge_offsets, (G + 1) * 8ull, cudaMemcpyHostToDevice, s));
        TP_CUDA(cudaMemcpyAsync(nv_d.ptr, num_vertices, G * 4ull, cudaMemcpyHostToDevice, s));
        TP_CUDA(cudaMemcpyAsync(vbase_d.ptr, vbase_h.data(), (G + 1) * 8ull, cudaMemcpyHostToDevice, s));
    }
    const uint64_t* eoff = batched ? eoff_d.as<uint64_t>() : nullptr;
    const uint64_t* vbase = batched ? vbase_d.as<uint64_t>() : nullptr;

    // 1. validate
    Scratch flags_d;
    TP_CUDA(flags_d.alloc(64, s));
    TP_CUDA(cudaMemsetAsync(flags_d.ptr, 0, 64, s));
    if (m_in)
        validate_edges_kernel<<<grid_for(m_in), kThreads, 0, s>>>(
            (const uint32_t*)src.dptr, (const uint32_t*)dst.dptr, (const uint8_t*)el.dptr, m_in, (uint32_t)n,
            eoff, nv_d.as<uint32_t>(), G, Le, flags_d.as<unsigned>()); ::tp::note_launch();
    if (vl.dptr && n)
        validate_vl_kernel<<<grid_for(n), kThreads, 0, s>>>((const uint8_t*)vl.dptr, n, Lv, flags_d.as<unsigned>()); ::tp::note_launch();
    TP_CUDA(cudaGetLastError());
    unsigned flags = 0;
    TP_CUDA(cudaMemcpyAsync(&flags, flags_d.ptr, 4, cudaMemcpyDeviceToHost, s));
    TP_CUDA(cudaStreamSynchronize(s));
    if (flags & 1u) return fail(TRIPOLL_ERR_VERTEX_RANGE, "an edge endpoint is >= the vertex count");
    if (flags & 6u) return fail(TRIPOLL_ERR_LABEL_RANGE, "a label is >= its label count");

    const int b = bits_for(n ? n - 1 : 0);
    const uint64_t vmask = (1ull << b) - 1;
    const uint64_t sentinel = (2 * b >= 64) ? ~0ull : ((1ull << (2 * b)) - 1);

    tripoll_graph* g = new tripoll_graph();
    GraphGuard guard(g, s);
    g->device = dev;
    g->n = n;
    g->m_in = m_in;
    g->num_graphs = batched ? G : 1;
    g->Lv = Lv;
    g->Le = el_h ? Le : 1;
    g->has_el = el_h != nullptr;
    g->plan = default_plan();

    // 2. canonical records, sort, keep the minimum payload of each pair (the chronologically first record)
    uint32_t* fault = flags_d.as<uint32_t>() + 1;  // look-back waits of the radix sorts that gave up
    const bool packed = 2 * b + 8 <= 64;           // 12-byte records (prim::rec_word)
    uint64_t m = 0;
    Scratch ukey_d, uval_d;
    {
        const DedupIn in{(const uint32_t*)src.dptr, (const uint32_t*)dst.dptr, (const uint32_t*)ts.dptr,
                         (const uint8_t*)el.dptr, m_in, eoff, vbase, G, b, sentinel, fault};
        auto release_inputs = [&] { src.copy.release(); dst.copy.release(); ts.copy.release(); el.copy.release(); };
        rc = packed ? dedup<uint32_t>(in, release_inputs, ukey_d, uval_d, &m, s)
                    : dedup<uint64_t>(in, release_inputs, ukey_d, uval_d, &m, s);
        if (rc) return rc;
        if (m >= 0xFFFFFFFFull) return fail(TRIPOLL_ERR_INVALID_ARG, "more than 2^32-2 unique edges");
    }
    g->m = m;

    // 3. degrees
    Scratch deg_d;
    TP_CUDA(deg_d.alloc((n + 1) * 4, s));
    TP_CUDA(cudaMemsetAsync(deg_d.ptr, 0, (n + 1) * 4, s));
    if (m) degree_kernel<<<grid_for(m), kThreads, 0, s>>>(ukey_d.as<uint64_t>(), m, b, deg_d.as<uint32_t>()); ::tp::note_launch();
    TP_CUDA(cudaGetLastError());
    unsigned dmax = 0;
    {
        Scratch mx;
        TP_CUDA(mx.alloc(4, s));
        TP_CUDA(cudaMemsetAsync(mx.ptr, 0, 4, s));
        if (n) max_u32_kernel<<<grid_for(n), kThreads, 0, s>>>(deg_d.as<uint32_t>(), n, mx.as<unsigned>()); ::tp::note_launch();
        TP_CUDA(cudaGetLastError());
        TP_CUDA(cudaMemcpyAsync(&dmax, mx.ptr, 4, cudaMemcpyDeviceToHost, s));
        TP_CUDA(cudaStreamSynchronize(s));
    }

    // 4. the order <+ : sort vertices by (graph, degree, id)
    const int bd = bits_for(dmax);
    const int gb = batched ? bits_for(G ? G - 1 : 0) : 0;
    if (gb + bd + b > 64) return fail(TRIPOLL_ERR_INVALID_ARG, "graph/degree/id key exceeds 64 bits");
    Scratch rank_d;
    TP_CUDA(rank_d.alloc((n + 1) * 4, s));
    TP_CUDA(galloc(g, &g->order, n, s));
    TP_CUDA(galloc(g, &g->deg, n, s));
    if (batched) TP_CUDA(galloc(g, &g->graph_of, n, s));
    {
        Scratch a, c, tmp;
        TP_CUDA(a.alloc(n * 8, s));
        TP_CUDA(c.alloc(n * 8, s));
        if (n)
            vertex_key_kernel<<<grid_for(n), kThreads, 0, s>>>(deg_d.as<uint32_t>(), n, vbase, G, b, bd,
                                                               a.as<uint64_t>()); ::tp::note_launch();
        TP_CUDA(cudaGetLastError());
        const int end_bit = gb + bd + b;
        TP_CUDA(tmp.alloc(prim::sort_scratch_bytes(n), s));
        bool alt = false;
        if ((rc = prim::radix_sort<uint64_t, prim::NoValue>(a.as<uint64_t>(), c.as<uint64_t>(), nullptr, nullptr, n,
                                                            end_bit, tmp.ptr, fault, s, &alt)))
            return rc;
        const uint64_t* sorted = alt ? c.as<uint64_t>() : a.as<uint64_t>();
        if (n)
            rank_kernel<<<grid_for(n), kThreads, 0, s>>>(sorted, n, b, rank_d.as<uint32_t>(), g->order,
                                                         deg_d.as<uint32_t>(), g->deg, bd + b, g->graph_of); ::tp::note_launch();
        TP_CUDA(cudaGetLastError());
    }
    deg_d.release();

    // vertex labels in position order
    TP_CUDA(galloc(g, &g->vl, n, s));
    if (n)
        vlabel_pos_kernel<<<grid_for(n), kThreads, 0, s>>>((const uint8_t*)vl.dptr, g->order, n, g->vl); ::tp::note_launch();
    TP_CUDA(cudaGetLastError());

    // 5. orient + CSR of G+ (col padded by kColPad entries so 32-byte vector loads
    //    of the last out-lists stay inside the allocation)
    TP_CUDA(galloc(g, &g->off, n + 1, s));
    TP_CUDA(galloc(g, &g->col, m + kColPad, s));
    TP_CUDA(cudaMemsetAsync(g->col + m, 0xFF, kColPad * 4, s));
    TP_CUDA(galloc(g, &g->ts, m + kColPad, s));  // padded like col: 16-byte loads of the last quads
    if (g->has_el) TP_CUDA(galloc(g, &g->el, m + kColPad, s));
    TP_CUDA(galloc(g, &g->in_off, n + 1, s));
    TP_CUDA(galloc(g, &g->in_edge, m, s));
    {
        Scratch first, cnt, tmp, sscr, ck0, cp0, rec0;
        TP_CUDA(first.alloc((n + 1) * 4, s));
        TP_CUDA(cnt.alloc((n + 1) * 4, s));
        TP_CUDA(tmp.alloc(prim::sort_scratch_bytes(m), s));
        TP_CUDA(sscr.alloc(prim::scan_scratch_bytes(n + 1), s));
        TP_CUDA(ck0.alloc(m * 4, s));
        TP_CUDA(cp0.alloc(m * 4, s));
        TP_CUDA(rec0.alloc(m * sizeof(InEdge), s));
        // orientation, sort by (source, target), offsets, CSR arrays and the in-edge records in CSR order
        const OrientIn oin{g, m, n, b, rank_d.as<uint32_t>(), first.as<uint32_t>(), cnt.as<uint32_t>(), tmp.ptr,
                           sscr.ptr, fault, ck0.as<uint32_t>(), cp0.as<uint32_t>(), rec0.as<InEdge>()};
        rc = packed ? orient_csr<uint32_t>(oin, ukey_d, uval_d, rank_d, s) : orient_csr<uint64_t>(oin, ukey_d, uval_d, rank_d, s);
        if (rc) return rc;
        // a stable sort of (target, CSR position) pairs by target leaves the positions in (target, source)
        // order; the 16-byte records are then gathered once in that order
        Scratch ck1, cp1;
        TP_CUDA(ck1.alloc(m * 4, s));
        TP_CUDA(cp1.alloc(m * 4, s));
        const int tbits = std::min(32, b);
        bool ealt = false;
        if ((rc = prim::radix_sort<uint32_t, uint32_t>(ck0.as<uint32_t>(), ck1.as<uint32_t>(), cp0.as<uint32_t>(),
                                                         cp1.as<uint32_t>(), m, tbits, tmp.ptr, fault, s, &ealt)))
            return rc;
        if (m)
            gather_in_edges_kernel<<<grid_for(m), kThreads, 0, s>>>(rec0.as<InEdge>(),
                                                                    (ealt ? cp1 : cp0).as<uint32_t>(), m,
                                                                    g->in_edge); ::tp::note_launch();
        TP_CUDA(cudaGetLastError());
        // in-edge offsets from the runs of equal targets
        const uint32_t* ckey = ealt ? ck1.as<uint32_t>() : ck0.as<uint32_t>();
        if ((rc = out_offsets(ckey, m, ~0ull, 0, n, first.as<uint32_t>(), cnt.as<uint32_t>(), g->in_off, sscr.ptr, s)))
            return rc;
        // both lists must account for every edge before anything indexes with these offsets
        uint64_t ends[2] = {0, 0};
        TP_CUDA(cudaMemcpyAsync(&ends[0], g->off + n, 8, cudaMemcpyDeviceToHost, s));
        TP_CUDA(cudaMemcpyAsync(&ends[1], g->in_off + n, 8, cudaMemcpyDeviceToHost, s));
        TP_CUDA(cudaStreamSynchronize(s));
        if (ends[0] != m || ends[1] != m)
            return fail(TRIPOLL_ERR_CUDA, "internal: the out- or in-list offsets of G+ do not add up to its edges");
    }
    (void)vmask;

    // 6. batched: vertex base of every graph
    if (batched) {
        TP_CUDA(galloc(g, &g->graph_vbase, G + 1, s));
        TP_CUDA(cudaMemcpyAsync(g->graph_vbase, vbase_h.data(), (G + 1) * 8ull, cudaMemcpyHostToDevice, s));
    }

    // 7. statistics
    {
        Scratch st;
        TP_CUDA(st.alloc(32, s));
        TP_CUDA(cudaMemsetAsync(st.ptr, 0, 32, s));
        if (n)
            stats_kernel<<<grid_for(n), kThreads, 0, s>>>(g->off, g->in_off, g->deg, n,
                                                          st.as<unsigned long long>()); ::tp::note_launch();
        TP_CUDA(cudaGetLastError());
        uint64_t h[4];
        TP_CUDA(cudaMemcpyAsync(h, st.ptr, 32, cudaMemcpyDeviceToHost, s));
        TP_CUDA(cudaStreamSynchronize(s));
        tripoll_graph_info& in = g->info;
        in.num_vertices = n;
        in.num_input_edges = m_in;
        in.num_edges = m;
        in.wedges = h[0];
        in.q_list_words = h[1];
        in.dplus_max = h[2];
        in.degree_max = h[3];
        in.num_graphs = g->num_graphs;
        in.num_vlabels = Lv;
        in.num_elabels = g->has_el ? Le : 0;
    }

    // 8. the survey plan (work items)
    if ((rc = build_plan(g, s)) != TRIPOLL_OK) return rc;
    TP_CUDA(cudaStreamSynchronize(s));
    g->info.device_bytes = (n + 1) * 8 * 2 + m * (4 + 4 + (g->has_el ? 1 : 0) + sizeof(InEdge)) +
                           n * (1 + 4 + 4 + (batched ? 4 : 0)) +
                           (g->n_items_warp + g->n_items_block + g->n_items_big) * sizeof(WorkItem);
    *out = guard.release();
    return TRIPOLL_OK;
}

}  // namespace

// Arrays go back to their allocators in the order of the legacy default stream.
void free_graph_arrays(tripoll_graph* g) {
    for (const Block& b : g->blocks) dev_free(b.ptr, b.bytes, 0, b.al);
    g->blocks.clear();
    g->off = nullptr; g->col = nullptr; g->ts = nullptr; g->el = nullptr; g->vl = nullptr;
    g->deg = nullptr; g->order = nullptr; g->graph_of = nullptr; g->in_off = nullptr;
    g->in_edge = nullptr; g->items_warp = nullptr; g->items_block = nullptr; g->items_big = nullptr;
    g->graph_vbase = nullptr;
}

}  // namespace tp

extern "C" int tripoll_graph_create(const uint32_t* src, const uint32_t* dst, const uint32_t* ts,
                                    const uint8_t* elabel, uint64_t num_edges, const uint8_t* vlabel,
                                    uint32_t num_vertices, uint32_t num_vlabels, uint32_t num_elabels,
                                    void* cuda_stream, tripoll_graph_t* out) {
    return tp::build_impl(src, dst, ts, elabel, num_edges, vlabel, num_vertices, num_vlabels, num_elabels,
                          nullptr, nullptr, 0, (cudaStream_t)cuda_stream, out);
}

extern "C" int tripoll_batch_create(const uint32_t* src, const uint32_t* dst, const uint32_t* ts,
                                    const uint8_t* elabel, const uint64_t* edge_offsets, const uint8_t* vlabel,
                                    const uint32_t* num_vertices, uint32_t num_graphs, uint32_t num_vlabels,
                                    uint32_t num_elabels, void* cuda_stream, tripoll_graph_t* out) {
    if (!edge_offsets || !num_vertices || num_graphs == 0)
        return tp::fail(TRIPOLL_ERR_INVALID_ARG, "batched build needs edge_offsets, num_vertices, num_graphs > 0");
    if (edge_offsets[0] != 0) return tp::fail(TRIPOLL_ERR_INVALID_ARG, "edge_offsets[0] must be 0");
    uint64_t n = 0;
    for (uint32_t i = 0; i < num_graphs; ++i) {
        if (edge_offsets[i + 1] < edge_offsets[i])
            return tp::fail(TRIPOLL_ERR_INVALID_ARG, "edge_offsets must be non-decreasing");
        n += num_vertices[i];
    }
    if (n > 0xFFFFFFFFull) return tp::fail(TRIPOLL_ERR_INVALID_ARG, "too many vertices in the batch");
    return tp::build_impl(src, dst, ts, elabel, edge_offsets[num_graphs], vlabel, n, num_vlabels, num_elabels,
                          edge_offsets, num_vertices, num_graphs, (cudaStream_t)cuda_stream, out);
}

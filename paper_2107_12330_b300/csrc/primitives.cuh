// primitives.cuh -- device-wide building blocks of the graph builder and the
// survey plan: LSD radix sort (keys, or keys with values), minimum per run of
// equal keys, and exclusive / inclusive scans.  All integer, all stable or
// order-independent, all on the caller's stream.
//
// Radix sort.  One sweep per 8-bit digit, least significant first.  The digit
// counts of every pass come from one read of the keys up front; a pass in
// which all keys share one digit leaves the order unchanged and is skipped.
// In a sweep each block takes the next tile of kTile consecutive keys (a
// ticket from an atomic counter, so that every earlier tile has already
// started), ranks its keys by digit -- warp by warp, 32 keys at a time, with
// __match_any_sync and per-warp digit counters in shared memory, which keeps
// the order of equal digits (stable) -- and learns where each digit of its
// tile starts in the output by decoupled look-back: it publishes its digit
// counts, then adds up its predecessors' counts until it meets one that has
// published its inclusive prefix, and publishes its own.  The tile is staged
// in shared memory in digit order and written out in runs of equal digits,
// consecutive threads to consecutive addresses.  Every wait on a predecessor
// is bounded: past kSpinLimit polls the block records a fault bit, stops
// waiting and finishes its tile (the caller reports the fault as an error).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <type_traits>
#include <utility>

#include "common.cuh"

namespace tp {
namespace prim {
namespace {  // each translation unit that uses these gets its own copy of the kernels

constexpr int kThreads = 256;
constexpr int kWarps = kThreads / 32;
constexpr int kItems = 16;                // keys per thread per tile
constexpr int kTile = kThreads * kItems;  // keys per tile
constexpr int kRadix = 256;
constexpr uint64_t kFlagAggregate = 1ull << 62;  // the tile's own counts are published
constexpr uint64_t kFlagInclusive = 2ull << 62;  // counts of all tiles up to this one are published
constexpr uint64_t kValueMask = (1ull << 62) - 1;
constexpr uint32_t kSpinLimit = 1u << 22;
constexpr int kLookback = 8;  // predecessors a look-back round reads at once
constexpr uint32_t kFaultLookback = 1u;  // a look-back wait gave up

static_assert(kThreads == kRadix, "one thread per digit in the look-back");

__device__ __forceinline__ uint32_t lanemask_lt() {
    uint32_t m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}

// Digit of key k at bit `shift`, keeping only the bits below end_bit: bits above the sort key may
// carry other data (a record's payload), which must not take part in the order.
template <class K> __device__ __forceinline__ uint32_t digit_of(K k, int shift, int end_bit) {
    const int w = end_bit - shift;
    return (uint32_t)(k >> shift) & (w >= 8 ? 0xFFu : ((1u << w) - 1u));
}

// Exclusive prefix of one value per thread over the block (kThreads threads); *total gets the sum.
template <class T>
__device__ __forceinline__ T block_exclusive_scan(T v, T* s_warp /*[kWarps]*/, T* total) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    T x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const T y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) s_warp[warp] = x;
    __syncthreads();
    T before = 0, all = 0;
#pragma unroll
    for (int w = 0; w < kWarps; ++w) {
        const T t = s_warp[w];
        if (w < warp) before += t;
        all += t;
    }
    __syncthreads();
    *total = all;
    return before + x - v;
}

// ---- digit counts of all passes ---------------------------------------------------------------

template <class K>
__global__ void __launch_bounds__(kThreads) digit_count_kernel(const K* __restrict__ keys, uint64_t n, int passes,
                                                               int end_bit, uint32_t* __restrict__ counts /*[passes][256]*/) {
    __shared__ uint32_t h[8 * kRadix];
    for (int i = threadIdx.x; i < passes * kRadix; i += kThreads) h[i] = 0;
    __syncthreads();
    for (uint64_t i = blockIdx.x * (uint64_t)kThreads + threadIdx.x; i < n; i += (uint64_t)gridDim.x * kThreads) {
        const K k = keys[i];
        for (int p = 0; p < passes; ++p) atomicAdd(&h[p * kRadix + digit_of(k, 8 * p, end_bit)], 1u);
    }
    __syncthreads();
    for (int i = threadIdx.x; i < passes * kRadix; i += kThreads)
        if (h[i]) atomicAdd(&counts[i], h[i]);
}

// starts[p][d] = number of keys whose digit p is below d
__global__ void digit_start_kernel(const uint32_t* __restrict__ counts, uint32_t* __restrict__ starts) {
    __shared__ uint32_t s_warp[kWarps];
    uint32_t total;
    const uint32_t c = counts[blockIdx.x * kRadix + threadIdx.x];
    starts[blockIdx.x * kRadix + threadIdx.x] = block_exclusive_scan(c, s_warp, &total);
}

// ---- one sweep --------------------------------------------------------------------------------

struct NoValue {};

// 16-byte asynchronous global -> shared copy; bytes past src_bytes (< 16) are filled with zeros.
__device__ __forceinline__ void cp_async16(void* smem, const void* gmem, uint32_t src_bytes) {
    const uint32_t sa = (uint32_t)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(sa), "l"(gmem), "r"(src_bytes) : "memory");
}
__device__ __forceinline__ void cp_async_commit_and_wait_all() {
    asm volatile("cp.async.commit_group;\ncp.async.wait_all;\n" ::: "memory");
}

// Tile shape per key/value type: 8-byte values are staged in digit order for coalesced writes;
// 16-byte values go out straight from the prefetch buffer (staging them too would cost a block per SM).
#ifndef TP_SORT_KV_ITEMS
#define TP_SORT_KV_ITEMS 12  // keys per thread in a sweep that moves values
#endif
#ifndef TP_SORT_MIN_BLOCKS
#define TP_SORT_MIN_BLOCKS 3  // resident blocks per SM the sweep's register budget allows
#endif
#ifndef TP_SORT_STAGE16
#define TP_SORT_STAGE16 0  // stage 16-byte values in digit order too
#endif
#ifndef TP_SORT_STAGE8
#define TP_SORT_STAGE8 1  // stage values of up to 8 bytes in digit order
#endif
#ifndef TP_SORT_RANK_ATOMIC
#define TP_SORT_RANK_ATOMIC 1  // the ranking leader bumps its warp counter with one shared atomic
#endif
#ifndef TP_SORT_ITEMS16
#define TP_SORT_ITEMS16 TP_SORT_KV_ITEMS  // keys per thread in a sweep that moves 16-byte values
#endif
template <class K, class V> struct SweepShape {
    static constexpr bool kHasValues = !std::is_same<V, NoValue>::value;
    static constexpr int kItems = !kHasValues ? 16 : (sizeof(V) > 8 ? TP_SORT_ITEMS16 : TP_SORT_KV_ITEMS);
    static constexpr int kTile = kThreads * kItems;
    static constexpr bool kStageValues = kHasValues && (sizeof(V) <= 8 ? TP_SORT_STAGE8 : TP_SORT_STAGE16);
    static constexpr size_t kRawBytes = kHasValues ? (size_t)kTile * sizeof(V) : 0;
    static constexpr size_t kStageBytes = (size_t)kTile * (kStageValues && sizeof(V) > sizeof(K) ? sizeof(V) : sizeof(K));
    static constexpr size_t kSmem = kRawBytes + kStageBytes;
};

template <class K, class V>
__global__ void __launch_bounds__(kThreads, TP_SORT_MIN_BLOCKS) sweep_kernel(const K* __restrict__ kin, K* __restrict__ kout,
                                                            const V* __restrict__ vin, V* __restrict__ vout, uint64_t n,
                                                            int shift, int end_bit, const uint32_t* __restrict__ start,
                                                            unsigned long long* __restrict__ status, uint64_t tiles,
                                                            uint32_t* __restrict__ ticket, uint32_t* __restrict__ fault) {
    using Shape = SweepShape<K, V>;
    constexpr int kIt = Shape::kItems;
    constexpr int kT = Shape::kTile;
    extern __shared__ __align__(16) unsigned char smem[];  // [raw values in input order][stage]
    __shared__ uint32_t s_tile;
    // per-warp digit counts, then the tile-local position of each warp's first key of each digit
    __shared__ uint32_t s_whist[kWarps][kRadix];
    // output position of tile-local index 0 of each digit, modulo 2^32 (positions are below 2^32, so
    // base + index modulo 2^32 is the position even when the base itself wraps)
    __shared__ uint32_t s_gbase[kRadix];
    __shared__ uint32_t s_warp_tmp[kWarps];
    __shared__ uint8_t s_sdig[Shape::kStageValues ? kT : 1];  // digit of each staged (sorted) key

    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (threadIdx.x == 0) s_tile = atomicAdd(ticket, 1u);
    for (int w = 0; w < kWarps; ++w) s_whist[w][threadIdx.x] = 0;
    __syncthreads();
    const uint64_t tile = s_tile;
    const uint64_t base = tile * kT;
    const uint32_t nv = (uint32_t)min((uint64_t)kT, n - base);  // keys in this tile
    const uint32_t wofs = (uint32_t)warp * 32 * kIt;            // this warp's keys: base + wofs + 32 r + lane
    V* raw = reinterpret_cast<V*>(smem);
    if constexpr (Shape::kHasValues) {  // the tile's values, in flight while the keys are ranked
        const uint32_t bytes = nv * (uint32_t)sizeof(V);
        const char* src = reinterpret_cast<const char*>(vin + base);
        for (uint32_t c = threadIdx.x; c * 16 < bytes; c += kThreads)
            cp_async16(smem + 16 * c, src + 16 * c, min(16u, bytes - 16 * c));
    }

    // rank: digit groups of each 32-key round, counted per warp in arrival order (stable)
    K key[kIt];
    uint32_t rank[kIt];
    const uint32_t lt = lanemask_lt();
#pragma unroll
    for (int r = 0; r < kIt; ++r) {  // all loads first, so that they are in flight together
        const uint32_t j = wofs + 32 * r + lane;
        key[r] = j < nv ? kin[base + j] : K(0);
    }
#pragma unroll
    for (int r = 0; r < kIt; ++r) {
        const bool ok = wofs + 32 * r + lane < nv;
        const uint32_t d = ok ? digit_of(key[r], shift, end_bit) : (uint32_t)kRadix;  // past the end: a digit of its own
        const uint32_t peers = __match_any_sync(0xffffffffu, d);
        const int leader = __ffs(peers) - 1;
        uint32_t old = 0;
        if (lane == leader && ok) {
#if TP_SORT_RANK_ATOMIC
            old = atomicAdd(&s_whist[warp][d], (uint32_t)__popc(peers));
#else
            old = s_whist[warp][d];
            s_whist[warp][d] = old + __popc(peers);
#endif
        }
        rank[r] = __shfl_sync(0xffffffffu, old, leader) + __popc(peers & lt);
        __syncwarp();  // the next round's leaders (other lanes) read these counters
    }
    __syncthreads();

    // per digit (thread = digit): offsets of the warps within the tile's run of that digit
    const uint32_t dg = threadIdx.x;
    uint32_t cnt = 0, wofs_d[kWarps];
#pragma unroll
    for (int w = 0; w < kWarps; ++w) {
        wofs_d[w] = cnt;
        cnt += s_whist[w][dg];
    }
    uint32_t tile_total;
    const uint32_t dstart = block_exclusive_scan(cnt, s_warp_tmp, &tile_total);
#pragma unroll
    for (int w = 0; w < kWarps; ++w) s_whist[w][dg] = dstart + wofs_d[w];  // where warp w's keys of dg start

    // decoupled look-back: keys of digit dg in all earlier tiles.  Status words are [tile][digit]
    // (a warp reads 32 digits of one tile in one line), and each round reads the next kLookback
    // predecessors at once: a tile usually finds its nearest predecessor with an inclusive prefix
    // several tiles back (tiles start a few tens of ns apart, an L2 round trip takes hundreds), so
    // reading them one at a time would make the walk a chain of round trips.
    volatile unsigned long long* col = status + dg;  // digit dg of tile t at col[t * kRadix]
    unsigned long long excl = 0;
    if (tile == 0) {
        col[0] = kFlagInclusive | cnt;
    } else {
        col[tile * kRadix] = kFlagAggregate | cnt;
        uint64_t j = tile;  // predecessors below j are still to be read
        bool done = false;
        while (!done && j > 0) {
            unsigned long long st[kLookback];
#pragma unroll
            for (int i = 0; i < kLookback; ++i) st[i] = (j > (uint64_t)i) ? col[(j - 1 - i) * kRadix] : kFlagInclusive;
#pragma unroll
            for (int i = 0; i < kLookback; ++i) {
                if (done) break;
                unsigned long long v = st[i];
                uint32_t spins = 0;
                while ((v & ~kValueMask) == 0) {  // not published yet: wait for this one
                    if (++spins > kSpinLimit) {
                        atomicOr(fault, kFaultLookback);
                        v = kFlagInclusive;  // give up; the tile's writes stay inside its digits' ranges
                        break;
                    }
                    __nanosleep(spins < 64 ? 32 : 256);
                    v = col[(j - 1 - i) * kRadix];
                }
                excl += v & kValueMask;
                if ((v & ~kValueMask) == kFlagInclusive) done = true;
            }
            j = j > (uint64_t)kLookback ? j - kLookback : 0;
        }
        col[tile * kRadix] = kFlagInclusive | (excl + cnt);
    }
    s_gbase[dg] = (uint32_t)((unsigned long long)start[dg] + excl - dstart);
    __syncthreads();

    // stage the keys in digit order, then write them out in runs of equal digits
    K* sk = reinterpret_cast<K*>(smem + Shape::kRawBytes);
    uint32_t lpos[kIt];
#pragma unroll
    for (int r = 0; r < kIt; ++r) {
        lpos[r] = 0xFFFFFFFFu;
        if (wofs + 32 * r + lane < nv) {
            const uint32_t d = digit_of(key[r], shift, end_bit);
            lpos[r] = s_whist[warp][d] + rank[r];
            sk[lpos[r]] = key[r];
        }
    }
    __syncthreads();
#pragma unroll
    for (int r = 0; r < kIt; ++r) {
        const uint32_t j = threadIdx.x + r * kThreads;
        if (j < nv) {
            const K k = sk[j];
            const uint32_t d = digit_of(k, shift, end_bit);
            if constexpr (Shape::kStageValues) s_sdig[j] = (uint8_t)d;
            kout[s_gbase[d] + j] = k;
        }
    }
    if constexpr (Shape::kHasValues) {
        cp_async_commit_and_wait_all();
        if constexpr (Shape::kStageValues) {
            __syncthreads();  // prefetched values visible to all; the key stage is no longer read
            V* sv = reinterpret_cast<V*>(smem + Shape::kRawBytes);
#pragma unroll
            for (int r = 0; r < kIt; ++r)
                if (lpos[r] != 0xFFFFFFFFu) sv[lpos[r]] = raw[wofs + 32 * r + lane];
            __syncthreads();
#pragma unroll
            for (int r = 0; r < kIt; ++r) {
                const uint32_t j = threadIdx.x + r * kThreads;
                if (j < nv) vout[s_gbase[s_sdig[j]] + j] = sv[j];
            }
        } else {
            __syncthreads();  // every thread's prefetched chunks are complete and visible
#pragma unroll
            for (int r = 0; r < kIt; ++r)
                if (lpos[r] != 0xFFFFFFFFu)
                    vout[s_gbase[digit_of(key[r], shift, end_bit)] + lpos[r]] = raw[wofs + 32 * r + lane];
        }
    }
}

// Sort n keys (with values when vals != nullptr) by bits [0, end_bit) (bits above end_bit are carried
// along and ignored).  keys/vals hold the input;
// keys_alt/vals_alt are buffers of the same size (16-byte aligned).  On return *in_alt tells where
// the sorted data is (false: keys/vals, true: keys_alt/vals_alt).  scratch: device memory of
// sort_scratch_bytes(n).
inline size_t sort_scratch_bytes(uint64_t n) {
    constexpr int kMinItems = TP_SORT_KV_ITEMS < TP_SORT_ITEMS16 ? TP_SORT_KV_ITEMS : TP_SORT_ITEMS16;
    constexpr uint64_t kMinTile = kThreads * (kMinItems < 16 ? kMinItems : 16);  // the smallest tile of any shape
    const uint64_t tiles = (n + kMinTile - 1) / kMinTile;
    return 256 + 2 * 8 * kRadix * 4 + tiles * kRadix * 8 + 256;
}

template <class K, class V>
int radix_sort(K* keys, K* keys_alt, V* vals, V* vals_alt, uint64_t n, int end_bit, void* scratch,
               uint32_t* fault, cudaStream_t s, bool* in_alt) {
    using Shape = SweepShape<K, V>;
    *in_alt = false;
    if (n == 0 || end_bit <= 0) return TRIPOLL_OK;
    if (n >= (1ull << 32)) return fail(TRIPOLL_ERR_INVALID_ARG, "radix sort of 2^32 or more keys");
    if (Shape::kHasValues && ((reinterpret_cast<uintptr_t>(vals) | reinterpret_cast<uintptr_t>(vals_alt)) & 15))
        return fail(TRIPOLL_ERR_INVALID_ARG, "radix sort: value arrays must be 16-byte aligned");
    const int passes = (end_bit + 7) / 8;
    const uint64_t tiles = (n + Shape::kTile - 1) / Shape::kTile;
    unsigned char* p = static_cast<unsigned char*>(scratch);
    uint32_t* ticket = reinterpret_cast<uint32_t*>(p);              // [passes] one per pass
    uint32_t* counts = reinterpret_cast<uint32_t*>(p + 256);        // [8][256]
    uint32_t* starts = counts + 8 * kRadix;                         // [8][256]
    unsigned long long* status = reinterpret_cast<unsigned long long*>(p + 256 + 2 * 8 * kRadix * 4);
    TP_CUDA(cudaMemsetAsync(p, 0, 256 + 2 * 8 * kRadix * 4, s));
    {
        const unsigned grid = (unsigned)std::min<uint64_t>((n + kThreads * 8 - 1) / (kThreads * 8), 148u * 8u);
        digit_count_kernel<K><<<grid, kThreads, 0, s>>>(keys, n, passes, end_bit, counts); note_launch();
        digit_start_kernel<<<passes, kRadix, 0, s>>>(counts, starts); note_launch();
        TP_CUDA(cudaGetLastError());
    }
    uint32_t h_counts[8 * kRadix];
    TP_CUDA(cudaMemcpyAsync(h_counts, counts, passes * kRadix * 4, cudaMemcpyDeviceToHost, s));
    TP_CUDA(cudaStreamSynchronize(s));
    static_assert(Shape::kSmem <= 200 * 1024, "stage fits the opt-in shared memory");
    cudaFuncSetAttribute(sweep_kernel<K, V>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)Shape::kSmem);
    K* kcur = keys;
    K* knext = keys_alt;
    V* vcur = vals;
    V* vnext = vals_alt;
    for (int pass = 0; pass < passes; ++pass) {
        bool trivial = false;  // every key has the same digit: the order stays as it is
        for (int d = 0; d < kRadix; ++d)
            if (h_counts[pass * kRadix + d] == n) trivial = true;
        if (trivial) continue;
        TP_CUDA(cudaMemsetAsync(status, 0, tiles * kRadix * 8, s));
        sweep_kernel<K, V><<<(unsigned)tiles, kThreads, Shape::kSmem, s>>>(
            kcur, knext, vcur, vnext, n, 8 * pass, end_bit, starts + pass * kRadix, status, tiles, ticket + pass, fault);
        note_launch();
        TP_CUDA(cudaGetLastError());
        std::swap(kcur, knext);
        std::swap(vcur, vnext);
        *in_alt = !*in_alt;
    }
    // a look-back wait that gave up leaves the output incomplete: report it before anyone reads it
    uint32_t h_fault = 0;
    TP_CUDA(cudaMemcpyAsync(&h_fault, fault, 4, cudaMemcpyDeviceToHost, s));
    TP_CUDA(cudaStreamSynchronize(s));
    if (h_fault & kFaultLookback) return fail(TRIPOLL_ERR_TIMEOUT, "radix sort: a look-back wait gave up");
    return TRIPOLL_OK;
}

// ---- records: a key with a payload ------------------------------------------------------------
//
// The builder sorts records made of a key of kb bits and a 40-bit payload.  The key sits in the low
// kb bits of a 64-bit word; with a 32-bit value (keys of at most 56 bits) the payload's low 32 bits
// are the value and its top 8 bits sit above the key in the word, so that a record moves 12 bytes
// per sort pass; with a 64-bit value the value is the whole payload.  Sorts look only at bits
// [0, kb) of the word.

template <class V> __host__ __device__ __forceinline__ uint64_t rec_key(uint64_t w, int kb) {
    return kb >= 64 ? w : (w & ((1ull << kb) - 1));
}
template <class V> __host__ __device__ __forceinline__ uint64_t rec_payload(uint64_t w, V v, int kb) {
    if (sizeof(V) == 4) return ((w >> kb) << 32) | (uint64_t)v;  // kb <= 56 here
    return (uint64_t)v;
}
template <class V> __host__ __device__ __forceinline__ uint64_t rec_word(uint64_t key, uint64_t payload, int kb) {
    if (sizeof(V) == 4) return key | ((payload >> 32) << kb);
    return key;
}

// ---- minimum payload per run of equal keys ----------------------------------------------------
//
// Records sorted by key (equal keys adjacent).  ukey[r], uval[r] = the key of the r-th run and the
// minimum of its payloads; the number of runs comes from a scan of the tiles' head counts.  Warp w
// of a block walks the records [tile + 32 kItems w, +32 kItems) 32 at a time (lane = position), so
// loads and the writes of consecutive runs are coalesced.  In each round the lanes of one run are
// contiguous: a segmented minimum over shuffles leaves the round's part of every run in its last
// lane, which stores it when the run lies wholly in the round and otherwise combines it with
// atomicMin (uval must hold ~0 there beforehand: the caller fills uval with 0xFF bytes).

template <class V>
__global__ void __launch_bounds__(kThreads) run_heads_kernel(const uint64_t* __restrict__ words, uint64_t n, int kb,
                                                             uint32_t* __restrict__ tile_heads) {
    __shared__ uint32_t s_warp[kWarps];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const uint64_t lo = blockIdx.x * (uint64_t)kTile + (uint64_t)warp * 32 * kItems;
    uint32_t h = 0;
#pragma unroll 4
    for (int r = 0; r < kItems; ++r) {
        const uint64_t i = lo + 32 * r + lane;
        if (i < n && (i == 0 || rec_key<V>(words[i - 1], kb) != rec_key<V>(words[i], kb))) ++h;
    }
    uint32_t total;
    block_exclusive_scan(h, s_warp, &total);
    if (threadIdx.x == 0) tile_heads[blockIdx.x] = total;
}

template <class V>
__global__ void __launch_bounds__(kThreads) run_min_kernel(const uint64_t* __restrict__ words,
                                                           const V* __restrict__ vals, uint64_t n, int kb,
                                                           const uint64_t* __restrict__ tile_base,
                                                           uint64_t* __restrict__ ukey,
                                                           unsigned long long* __restrict__ uval) {
    __shared__ uint32_t s_wheads[kWarps];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const uint64_t lo = blockIdx.x * (uint64_t)kTile + (uint64_t)warp * 32 * kItems;
    const uint32_t lt = lanemask_lt(), le = lt | (1u << lane);
    uint64_t key[kItems];
    uint32_t heads = 0;  // head bits of the rounds, lane-wise (bit r: the key of round r starts a run)
    uint32_t wh = 0;     // heads of the whole warp segment
#pragma unroll
    for (int r = 0; r < kItems; ++r) {
        const uint64_t i = lo + 32 * r + lane;
        key[r] = i < n ? rec_key<V>(words[i], kb) : 0;
        const bool h = i < n && (i == 0 || rec_key<V>(words[i - 1], kb) != key[r]);
        heads |= (h ? 1u : 0u) << r;
        wh += __popc(__ballot_sync(0xffffffffu, h));
    }
    if (lane == 0) s_wheads[warp] = wh;
    __syncthreads();
    uint64_t run_base = tile_base[blockIdx.x];  // heads before this warp's segment
    for (int w = 0; w < warp; ++w) run_base += s_wheads[w];
#pragma unroll
    for (int r = 0; r < kItems; ++r) {
        const uint64_t i = lo + 32 * r + lane;
        const bool ok = i < n;
        const bool h = (heads >> r) & 1u;
        const uint32_t b = __ballot_sync(0xffffffffu, h);
        // run index: heads at positions <= i, minus one
        const uint64_t run = ok ? run_base + __popc(b & le) - 1 : ~0ull;
        run_base += __popc(b);
        unsigned long long mn = ok ? (unsigned long long)rec_payload<V>(words[i], vals[i], kb) : ~0ull;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const unsigned long long m2 = __shfl_up_sync(0xffffffffu, mn, o);
            const uint64_t r2 = __shfl_up_sync(0xffffffffu, run, o);
            if (lane >= o && r2 == run) mn = min(mn, m2);
        }
        const uint64_t next_run = __shfl_down_sync(0xffffffffu, run, 1);
        if (!ok) continue;
        if (h) ukey[run] = key[r];
        const bool last_lane = lane == 31 || next_run != run;
        if (!last_lane) continue;
        // the run ends here when the next position starts another run (or the records end)
        const bool ends = lane != 31 || i + 1 == n || rec_key<V>(words[i + 1], kb) != key[r];
        const bool starts = (b & le) != 0;  // its head lies in this round
        if (starts && ends) uval[run] = mn;
        else atomicMin(&uval[run], mn);
    }
}

// ---- scans --------------------------------------------------------------------------------------
//
// out[i] = sum of in(j) for j < i (exclusive) or j <= i (inclusive), i in [0, n), for an input
// functor in(i) -> T.  Three steps: tile sums, a one-block scan of the tile sums, then each tile
// scanned from its base.

template <class T, class F>
__global__ void __launch_bounds__(kThreads) tile_sum_kernel(F in, uint64_t n, T* __restrict__ sums) {
    __shared__ T s_warp[kWarps];
    const uint64_t lo = blockIdx.x * (uint64_t)kTile + (uint64_t)threadIdx.x * kItems;
    T x = 0;
    for (int r = 0; r < kItems; ++r)
        if (lo + r < n) x += in(lo + r);
    T total;
    block_exclusive_scan(x, s_warp, &total);
    if (threadIdx.x == 0) sums[blockIdx.x] = total;
}

template <class T>
__global__ void __launch_bounds__(kThreads) tile_base_kernel(T* __restrict__ sums, uint64_t tiles, T* total_out) {
    __shared__ T s_warp[kWarps];
    T carry = 0;
    for (uint64_t b = 0; b < tiles; b += kThreads) {
        const uint64_t i = b + threadIdx.x;
        const T v = i < tiles ? sums[i] : T(0);
        T total;
        const T ex = block_exclusive_scan(v, s_warp, &total);
        if (i < tiles) sums[i] = carry + ex;
        carry += total;
    }
    if (threadIdx.x == 0 && total_out) *total_out = carry;
}

template <class T, class F, bool kInclusive>
__global__ void __launch_bounds__(kThreads) tile_scan_kernel(F in, uint64_t n, const T* __restrict__ bases,
                                                             T* __restrict__ out) {
    __shared__ T s_warp[kWarps];
    const uint64_t lo = blockIdx.x * (uint64_t)kTile + (uint64_t)threadIdx.x * kItems;
    T v[kItems];
    T x = 0;
#pragma unroll
    for (int r = 0; r < kItems; ++r) {
        v[r] = lo + r < n ? in(lo + r) : T(0);
        x += v[r];
    }
    T total;
    T run = bases[blockIdx.x] + block_exclusive_scan(x, s_warp, &total);
#pragma unroll
    for (int r = 0; r < kItems; ++r) {
        if (lo + r < n) out[lo + r] = kInclusive ? run + v[r] : run;
        run += v[r];
    }
}

inline size_t scan_scratch_bytes(uint64_t n) { return ((n + kTile - 1) / kTile + 1) * 8 + 256; }

// Scan of n values in(0..n-1) into out; total (device, optional) gets the sum of all n.
template <class T, bool kInclusive, class F>
int scan(F in, T* out, uint64_t n, void* scratch, cudaStream_t s, T* total = nullptr) {
    const uint64_t tiles = (n + kTile - 1) / kTile;
    T* sums = static_cast<T*>(scratch);
    if (n == 0) {
        if (total) TP_CUDA(cudaMemsetAsync(total, 0, sizeof(T), s));
        return TRIPOLL_OK;
    }
    tile_sum_kernel<T, F><<<(unsigned)tiles, kThreads, 0, s>>>(in, n, sums); note_launch();
    tile_base_kernel<T><<<1, kThreads, 0, s>>>(sums, tiles, total); note_launch();
    tile_scan_kernel<T, F, kInclusive><<<(unsigned)tiles, kThreads, 0, s>>>(in, n, sums, out); note_launch();
    TP_CUDA(cudaGetLastError());
    return TRIPOLL_OK;
}

// in(i) = a[i] as T (0 past n_valid)
template <class S, class T> struct Load {
    const S* a;
    uint64_t n_valid;
    __device__ __forceinline__ T operator()(uint64_t i) const { return i < n_valid ? (T)a[i] : T(0); }
};

}  // namespace
}  // namespace prim
}  // namespace tp

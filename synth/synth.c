/*
 * synth.c -- seeded synthetic input generators.
 *
 * These produce the decorated temporal graphs that both the CPU oracle and the
 * CUDA survey path read: edge endpoints (R-MAT, Chung-Lu), edge timestamps,
 * vertex labels and edge labels.  Nothing here computes any part of the
 * triangle survey; the module only shapes inputs.
 *
 * Every random number is counter-based: draw i of substream s under seed k is
 * the (i+1)-th output of SplitMix64 (Steele, Lea & Flood, "Fast splittable
 * pseudorandom number generators", OOPSLA 2014) started from a per-(k, s)
 * state.  Any element can therefore be produced independently of the others,
 * so the OpenMP loops below give the same arrays for every thread count.
 *
 * The R-MAT recursion follows Chakrabarti, Zhan & Faloutsos (SDM 2004), the
 * generator the paper uses for its weak-scaling graphs (Sec. 5.2): one
 * quadrant choice per level, no noise and no vertex permutation.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>

#define SM64_GAMMA 0x9E3779B97F4A7C15ULL

/* SplitMix64's output function. */
static inline uint64_t sm64_mix(uint64_t z) {
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

/* Starting state of substream `stream` under `seed`. */
uint64_t synth_stream_key(uint64_t seed, uint64_t stream) {
    return sm64_mix(sm64_mix(seed + SM64_GAMMA) ^ (stream * 0xD1B54A32D192ED03ULL));
}

/* Draw i (0-based) of the substream whose starting state is `key`. */
static inline uint64_t draw(uint64_t key, uint64_t i) {
    return sm64_mix(key + (i + 1) * SM64_GAMMA);
}

/* Draw i of a SplitMix64 sequence whose state starts at `state` (exported so a
 * test can check it against the generator's published outputs). */
uint64_t synth_splitmix64_at(uint64_t state, uint64_t i) { return draw(state, i); }

uint64_t synth_draw(uint64_t seed, uint64_t stream, uint64_t i) {
    return draw(synth_stream_key(seed, stream), i);
}

/* Uniform double in [0, 1) from the top 53 bits. */
static inline double unit53(uint64_t x) { return (double)(x >> 11) * 0x1.0p-53; }

/* R-MAT edges: scale levels, quadrant probabilities a, b, c (d = 1 - a - b - c).
 * Level l of edge i uses draw i*scale + l of the substream. */
void synth_rmat(uint64_t seed, uint64_t stream, int scale, uint64_t m, double a, double b, double c,
                uint32_t* src, uint32_t* dst) {
    const uint64_t key = synth_stream_key(seed, stream);
    const double t0 = a, t1 = a + b, t2 = a + b + c;
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < (int64_t)m; ++i) {
        uint32_t u = 0, v = 0;
        for (int l = 0; l < scale; ++l) {
            const double x = unit53(draw(key, (uint64_t)i * (uint64_t)scale + (uint64_t)l));
            u <<= 1;
            v <<= 1;
            if (x < t0) {
            } else if (x < t1) {
                v |= 1u;
            } else if (x < t2) {
                u |= 1u;
            } else {
                u |= 1u;
                v |= 1u;
            }
        }
        src[i] = u;
        dst[i] = v;
    }
}

/* Uniform integers in [0, 2^bits) (bits in 0..32): the top `bits` bits of each draw. */
void synth_bits_u32(uint64_t seed, uint64_t stream, uint64_t count, int bits, uint32_t* out) {
    const uint64_t key = synth_stream_key(seed, stream);
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < (int64_t)count; ++i)
        out[i] = bits == 0 ? 0u : (uint32_t)(draw(key, (uint64_t)i) >> (64 - bits));
}

/* floor(U * horizon) with U uniform in [0,1): the points of a Poisson process on
 * [0, horizon) conditioned on their number are i.i.d. uniform. */
void synth_scaled_u32(uint64_t seed, uint64_t stream, uint64_t count, double horizon, uint32_t* out) {
    const uint64_t key = synth_stream_key(seed, stream);
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < (int64_t)count; ++i) {
        double t = floor(unit53(draw(key, (uint64_t)i)) * horizon);
        out[i] = (uint32_t)t;
    }
}

/* Uniform labels in {0..L-1} (1 <= L <= 256) by multiply-shift of the top 32 bits. */
void synth_uniform_u8(uint64_t seed, uint64_t stream, uint64_t count, uint32_t L, uint8_t* out) {
    const uint64_t key = synth_stream_key(seed, stream);
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < (int64_t)count; ++i)
        out[i] = (uint8_t)(((draw(key, (uint64_t)i) >> 32) * (uint64_t)L) >> 32);
}

/* Zipf labels over {0..K-1} (K <= 256): P(k) proportional to (k+1)^-s, by inverse CDF. */
void synth_zipf_u8(uint64_t seed, uint64_t stream, uint64_t count, uint32_t K, double s, uint8_t* out) {
    double cdf[256];
    double z = 0.0;
    for (uint32_t k = 0; k < K; ++k) z += pow((double)(k + 1), -s);
    double acc = 0.0;
    for (uint32_t k = 0; k < K; ++k) {
        acc += pow((double)(k + 1), -s) / z;
        cdf[k] = acc;
    }
    const uint64_t key = synth_stream_key(seed, stream);
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < (int64_t)count; ++i) {
        const double x = unit53(draw(key, (uint64_t)i));
        uint32_t k = 0;
        while (k + 1 < K && !(x < cdf[k])) ++k;
        out[i] = (uint8_t)k;
    }
}

/* Chung-Lu edges: n vertices with weights w_i = (i+1)^(-1/(gamma-1)); each of the
 * m samples draws both endpoints i.i.d. with probability proportional to w (draws
 * 2i and 2i+1), by binary search in the cumulative weights.  Loops and repeated
 * pairs are left in; the graph builder removes them like any other input. */
int synth_chung_lu(uint64_t seed, uint64_t stream, uint32_t n, double gamma, uint64_t m,
                   uint32_t* src, uint32_t* dst) {
    double* cdf = (double*)malloc((size_t)n * sizeof(double));
    if (!cdf) return -1;
    const double expo = -1.0 / (gamma - 1.0);
    double acc = 0.0;
    for (uint32_t i = 0; i < n; ++i) {
        acc += pow((double)i + 1.0, expo);
        cdf[i] = acc;
    }
    const double total = acc;
    const uint64_t key = synth_stream_key(seed, stream);
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < (int64_t)m; ++i) {
        for (int side = 0; side < 2; ++side) {
            const double x = unit53(draw(key, 2 * (uint64_t)i + (uint64_t)side)) * total;
            /* first index whose cumulative weight exceeds x */
            uint32_t lo = 0, hi = n - 1;
            while (lo < hi) {
                const uint32_t mid = lo + (hi - lo) / 2;
                if (cdf[mid] > x) hi = mid; else lo = mid + 1;
            }
            if (side == 0) src[i] = lo; else dst[i] = lo;
        }
    }
    free(cdf);
    return 0;
}

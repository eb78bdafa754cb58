/*
 * oracle.c -- TEST INFRASTRUCTURE: the plain, slow CPU oracle of the metadata
 * triangle survey.  Only the tests, the smoke check and the benchmark's CPU
 * baseline use it; the library never calls it.  It shares no code, header,
 * table or helper with the CUDA path.
 *
 * What it computes (TriPoll, Sec. 3 and Sec. 4.3, Alg. 1):
 *   1. The simple undirected graph G' of the input: records with u == v are
 *      dropped; all records of one unordered pair {u,v} become one edge whose
 *      metadata (ts, elabel) is the lexicographic minimum over the records:
 *      the earliest record survives (Sec. 5.2), label as the tie-break.
 *   2. Degrees d(v) in G' (Sec. 3).
 *   3. The degree order <+ : u <+ v iff d(u) < d(v), or d(u) == d(v) and
 *      tie(u) < tie(v) (Sec. 3).  tie is the vertex id (mode 0), a bijective
 *      32-bit mixer of the id (mode 1, the paper's "hash"), or mode 2 ignores
 *      degree and orders by id alone.  Every mode is a strict total order, so
 *      every triangle is found exactly once under any of them.
 *   4. The DODGr G+ : each edge directed from its <+ -smaller end; Adj+(p)
 *      sorted ascending in <+ and augmented with the edge's metadata record
 *      (Adj+^m, Sec. 4.2).
 *   5. For every pivot p and every q in Adj+(p): the r in Adj+(p) with q <+ r
 *      that are also in Adj+(q), by a two-pointer merge of the two sorted lists
 *      (Alg. 1; the intersection there is of Adj+(p) and Adj+(q)).
 *   6. The survey fold over meta(Delta_pqr) for each triangle whose three edge
 *      timestamps all lie in [t_lo, t_hi]:
 *        count += 1                                   (Alg. 2)
 *        hist[ceil(log2(t3 - t1))] += 1, 0 -> bin 0   (closing time, Alg. 4)
 *        joint[open][close] += 1                      (Alg. 4 joint table)
 *        vtri[a][b][c] += 1, (a,b,c) the sorted vertex labels
 *        etri[a][b][c] += 1, (a,b,c) the sorted edge labels
 *        maxel[max edge label] += 1 when the three vertex labels are pairwise
 *          distinct                                   (Alg. 3)
 *        degtri[(ceil log2 d) sorted triple] += 1     (Sec. 5.9)
 *        vlocal[p], vlocal[q], vlocal[r] += 1         (local counts, Sec. 5.3)
 *        elocal[pq], elocal[pr], elocal[qr] += 1      (local edge counts, Sec. 5.3;
 *          edges numbered in (min id, max id) order)
 *   Output arrays the caller passes as NULL are skipped.
 *
 * The pivots can be restricted to a range of positions in the <+ order, so
 * that a part of a big survey can be checked on its own.
 */
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define HIST_BINS 33

typedef struct {
    uint64_t* count;  /* [1] */
    uint64_t* hist;   /* [33] */
    uint64_t* vtri;   /* [Lv^3] */
    uint64_t* etri;   /* [Le^3] */
    uint64_t* joint;  /* [33*33], index open*33 + close */
    uint64_t* maxel;  /* [Le] */
    uint64_t* degtri; /* [33^3] */
    uint64_t* vlocal; /* [n], by input vertex id */
    uint64_t* elocal; /* [m], by unique edge in ascending (min id, max id) order */
} oracle_out;

typedef struct {
    uint64_t m;         /* unique undirected edges of G' */
    uint64_t wedges;    /* |W+| = sum_p C(d+(p), 2) */
    uint64_t dplus_max; /* max_p d+(p) */
    uint64_t dmax;      /* max_v d(v) */
} oracle_stats;

/* ceil(log2(x)) for x >= 1 by its definition (smallest k with 2^k >= x); x = 0 -> 0. */
static int ceil_log2(uint64_t x) {
    int k = 0;
    while (k < 64 && ((uint64_t)1 << k) < x) ++k;
    return k;
}

typedef struct {
    uint32_t u, v, ts;
    uint8_t el;
} rec_t;

static int cmp_rec(const void* a, const void* b) {
    const rec_t* x = (const rec_t*)a;
    const rec_t* y = (const rec_t*)b;
    if (x->u != y->u) return x->u < y->u ? -1 : 1;
    if (x->v != y->v) return x->v < y->v ? -1 : 1;
    if (x->ts != y->ts) return x->ts < y->ts ? -1 : 1;
    if (x->el != y->el) return x->el < y->el ? -1 : 1;
    return 0;
}

/* A bijection on 32-bit words (the MurmurHash3 finaliser): the deterministic
 * "hash" tie-break of Sec. 3. */
static uint32_t mix32(uint32_t h) {
    h ^= h >> 16;
    h *= 0x85EBCA6Bu;
    h ^= h >> 13;
    h *= 0xC2B2AE35u;
    h ^= h >> 16;
    return h;
}

typedef struct {
    const uint64_t* deg;
    int mode;
} order_ctx;

static order_ctx g_order; /* qsort has no context argument; set before each sort */

/* -1 if x <+ y, +1 if y <+ x (never 0 for x != y). */
static int order_cmp(uint32_t x, uint32_t y) {
    if (g_order.mode != 2) {
        if (g_order.deg[x] != g_order.deg[y]) return g_order.deg[x] < g_order.deg[y] ? -1 : 1;
        if (g_order.mode == 1) {
            uint32_t hx = mix32(x), hy = mix32(y);
            if (hx != hy) return hx < hy ? -1 : 1;
        }
    }
    if (x != y) return x < y ? -1 : 1;
    return 0;
}

static int cmp_vertex(const void* a, const void* b) {
    return order_cmp(*(const uint32_t*)a, *(const uint32_t*)b);
}

typedef struct {
    uint32_t pos; /* the target's position in the <+ order */
    uint32_t v;   /* the target's input id */
    uint64_t e;   /* index of the undirected edge in the unique edge table */
} adj_t;

static int cmp_adj(const void* a, const void* b) {
    const adj_t* x = (const adj_t*)a;
    const adj_t* y = (const adj_t*)b;
    return x->pos < y->pos ? -1 : (x->pos > y->pos ? 1 : 0);
}

typedef struct {
    /* graph */
    uint32_t n, Lv, Le;
    const uint32_t* ets;
    const uint8_t* eel;
    const uint8_t* vl;
    const uint64_t* deg;
    const uint64_t* adj_start; /* [n+1] into adj[], by position in <+ */
    const adj_t* adj;
    const uint32_t* vertex_at; /* input id at each position */
    uint32_t t_lo, t_hi;
    /* work: the pivot positions in [p_lo, p_hi) whose block of 256 is t mod stride */
    uint32_t p_lo, p_hi;
    uint32_t t, stride;
    /* outputs (private per thread) */
    oracle_out out;
} work_t;

static void sort3_u32(uint32_t* a, uint32_t* b, uint32_t* c) {
    uint32_t t;
    if (*a > *b) { t = *a; *a = *b; *b = t; }
    if (*b > *c) { t = *b; *b = *c; *c = t; }
    if (*a > *b) { t = *a; *a = *b; *b = t; }
}

/* The fold of one triangle (step 6). */
static void fold(const work_t* w, uint32_t p, uint32_t q, uint32_t r, uint64_t e_pq, uint64_t e_pr,
                 uint64_t e_qr) {
    uint32_t t1 = w->ets[e_pq], t2 = w->ets[e_pr], t3 = w->ets[e_qr];
    if (t1 < w->t_lo || t1 > w->t_hi || t2 < w->t_lo || t2 > w->t_hi || t3 < w->t_lo ||
        t3 > w->t_hi)
        return;
    sort3_u32(&t1, &t2, &t3);
    const oracle_out* o = &w->out;
    if (o->count) o->count[0] += 1;
    if (o->hist) o->hist[ceil_log2((uint64_t)(t3 - t1))] += 1;
    if (o->joint) o->joint[ceil_log2((uint64_t)(t2 - t1)) * HIST_BINS + ceil_log2((uint64_t)(t3 - t1))] += 1;
    uint32_t lp = w->vl ? w->vl[p] : 0, lq = w->vl ? w->vl[q] : 0, lr = w->vl ? w->vl[r] : 0;
    uint32_t ea = w->eel ? w->eel[e_pq] : 0, eb = w->eel ? w->eel[e_pr] : 0,
             ec = w->eel ? w->eel[e_qr] : 0;
    if (o->maxel && lp != lq && lq != lr && lp != lr) {
        uint32_t mx = ea > eb ? ea : eb;
        mx = mx > ec ? mx : ec;
        o->maxel[mx] += 1;
    }
    if (o->vtri) {
        uint32_t a = lp, b = lq, c = lr;
        sort3_u32(&a, &b, &c);
        o->vtri[((uint64_t)a * w->Lv + b) * w->Lv + c] += 1;
    }
    if (o->etri) {
        uint32_t a = ea, b = eb, c = ec;
        sort3_u32(&a, &b, &c);
        o->etri[((uint64_t)a * w->Le + b) * w->Le + c] += 1;
    }
    if (o->degtri) {
        uint32_t a = (uint32_t)ceil_log2(w->deg[p]), b = (uint32_t)ceil_log2(w->deg[q]),
                 c = (uint32_t)ceil_log2(w->deg[r]);
        sort3_u32(&a, &b, &c);
        o->degtri[((uint64_t)a * HIST_BINS + b) * HIST_BINS + c] += 1;
    }
    if (o->vlocal) {
        o->vlocal[p] += 1;
        o->vlocal[q] += 1;
        o->vlocal[r] += 1;
    }
    if (o->elocal) {
        o->elocal[e_pq] += 1;
        o->elocal[e_pr] += 1;
        o->elocal[e_qr] += 1;
    }
}

/* Step 5 for this thread's pivots of [p_lo, p_hi). */
static void* survey_pivots(void* arg) {
    work_t* w = (work_t*)arg;
    for (uint32_t pp = w->p_lo; pp < w->p_hi; ++pp) {
        if (((pp - w->p_lo) >> 8) % w->stride != w->t) continue;
        const uint32_t p = w->vertex_at[pp];
        const adj_t* P = w->adj + w->adj_start[pp];
        const uint64_t dp = w->adj_start[pp + 1] - w->adj_start[pp];
        for (uint64_t i = 0; i < dp; ++i) {
            const uint32_t qpos = P[i].pos;
            const uint32_t q = P[i].v;
            const adj_t* Q = w->adj + w->adj_start[qpos];
            const uint64_t dq = w->adj_start[qpos + 1] - w->adj_start[qpos];
            /* merge Adj+(p) after q with Adj+(q) */
            uint64_t a = i + 1, b = 0;
            while (a < dp && b < dq) {
                if (P[a].pos < Q[b].pos) {
                    ++a;
                } else if (P[a].pos > Q[b].pos) {
                    ++b;
                } else {
                    fold(w, p, q, P[a].v, P[i].e, P[a].e, Q[b].e);
                    ++a;
                    ++b;
                }
            }
        }
    }
    return NULL;
}

static void add_into(uint64_t* dst, const uint64_t* src, uint64_t len) {
    if (!dst) return;
    for (uint64_t i = 0; i < len; ++i) dst[i] += src[i];
}

/* Returns 0 on success, -1 on bad arguments, -2 on out-of-memory.
 * Output arrays are accumulated into (the caller zeroes them). */
int oracle_survey(const uint32_t* src, const uint32_t* dst, const uint32_t* ts, const uint8_t* el,
                  uint64_t m_in, const uint8_t* vl, uint32_t n, uint32_t Lv, uint32_t Le,
                  uint32_t t_lo, uint32_t t_hi, int order_mode, uint32_t pivot_lo,
                  uint32_t pivot_hi, int threads, const oracle_out* out, oracle_stats* stats) {
    if (Lv == 0 || Le == 0 || order_mode < 0 || order_mode > 2) return -1;
    for (uint64_t i = 0; i < m_in; ++i)
        if (src[i] >= n || dst[i] >= n || (el && el[i] >= Le)) return -1;
    if (vl)
        for (uint32_t v = 0; v < n; ++v)
            if (vl[v] >= Lv) return -1;
    if (pivot_hi > n) pivot_hi = n;
    if (threads < 1) threads = 1;

    /* 1. the simple graph G' */
    rec_t* rec = (rec_t*)malloc((m_in ? m_in : 1) * sizeof(rec_t));
    if (!rec) return -2;
    uint64_t k = 0;
    for (uint64_t i = 0; i < m_in; ++i) {
        if (src[i] == dst[i]) continue;
        rec[k].u = src[i] < dst[i] ? src[i] : dst[i];
        rec[k].v = src[i] < dst[i] ? dst[i] : src[i];
        rec[k].ts = ts[i];
        rec[k].el = el ? el[i] : 0;
        ++k;
    }
    qsort(rec, k, sizeof(rec_t), cmp_rec);
    uint64_t m = 0;
    for (uint64_t i = 0; i < k; ++i)
        if (i == 0 || rec[i].u != rec[i - 1].u || rec[i].v != rec[i - 1].v) rec[m++] = rec[i];

    uint32_t* eu = (uint32_t*)malloc((m ? m : 1) * sizeof(uint32_t));
    uint32_t* ev = (uint32_t*)malloc((m ? m : 1) * sizeof(uint32_t));
    uint32_t* ets = (uint32_t*)malloc((m ? m : 1) * sizeof(uint32_t));
    uint8_t* eel = (uint8_t*)malloc(m ? m : 1);
    uint64_t* deg = (uint64_t*)calloc((size_t)n + 1, sizeof(uint64_t));
    uint32_t* vertex_at = (uint32_t*)malloc(((size_t)n + 1) * sizeof(uint32_t));
    uint32_t* pos_of = (uint32_t*)malloc(((size_t)n + 1) * sizeof(uint32_t));
    uint64_t* adj_start = (uint64_t*)calloc((size_t)n + 2, sizeof(uint64_t));
    adj_t* adj = (adj_t*)malloc((m ? m : 1) * sizeof(adj_t));
    if (!eu || !ev || !ets || !eel || !deg || !vertex_at || !pos_of || !adj_start || !adj) {
        free(rec); free(eu); free(ev); free(ets); free(eel); free(deg); free(vertex_at);
        free(pos_of); free(adj_start); free(adj);
        return -2;
    }
    for (uint64_t i = 0; i < m; ++i) {
        eu[i] = rec[i].u;
        ev[i] = rec[i].v;
        ets[i] = rec[i].ts;
        eel[i] = rec[i].el;
    }
    free(rec);

    /* 2. degrees */
    for (uint64_t i = 0; i < m; ++i) {
        deg[eu[i]] += 1;
        deg[ev[i]] += 1;
    }

    /* 3. the order <+ : position of every vertex */
    for (uint32_t v = 0; v < n; ++v) vertex_at[v] = v;
    g_order.deg = deg;
    g_order.mode = order_mode;
    qsort(vertex_at, n, sizeof(uint32_t), cmp_vertex);
    for (uint32_t i = 0; i < n; ++i) pos_of[vertex_at[i]] = i;

    /* 4. G+ with augmented out-lists, indexed by the pivot's position */
    for (uint64_t i = 0; i < m; ++i) {
        uint32_t p = order_cmp(eu[i], ev[i]) < 0 ? eu[i] : ev[i];
        adj_start[pos_of[p] + 1] += 1;
    }
    for (uint32_t i = 0; i < n; ++i) adj_start[i + 1] += adj_start[i];
    uint64_t* fill = (uint64_t*)malloc(((size_t)n + 1) * sizeof(uint64_t));
    if (!fill) {
        free(eu); free(ev); free(ets); free(eel); free(deg); free(vertex_at); free(pos_of);
        free(adj_start); free(adj);
        return -2;
    }
    memcpy(fill, adj_start, ((size_t)n + 1) * sizeof(uint64_t));
    for (uint64_t i = 0; i < m; ++i) {
        int fwd = order_cmp(eu[i], ev[i]) < 0;
        uint32_t p = fwd ? eu[i] : ev[i], q = fwd ? ev[i] : eu[i];
        adj_t a;
        a.pos = pos_of[q];
        a.v = q;
        a.e = i;
        adj[fill[pos_of[p]]++] = a;
    }
    free(fill);
    uint64_t wedges = 0, dplus_max = 0, dmax = 0;
    for (uint32_t i = 0; i < n; ++i) {
        uint64_t d = adj_start[i + 1] - adj_start[i];
        qsort(adj + adj_start[i], d, sizeof(adj_t), cmp_adj);
        wedges += d * (d ? d - 1 : 0) / 2;
        if (d > dplus_max) dplus_max = d;
        if (deg[i] > dmax) dmax = deg[i];
    }
    if (stats) {
        stats->m = m;
        stats->wedges = wedges;
        stats->dplus_max = dplus_max;
        stats->dmax = dmax;
    }

    /* 5 + 6: pivots dealt to `threads` workers in interleaved blocks of 256, private outputs */
    const uint64_t lv3 = (uint64_t)Lv * Lv * Lv, le3 = (uint64_t)Le * Le * Le;
    const uint64_t dt3 = (uint64_t)HIST_BINS * HIST_BINS * HIST_BINS;
    work_t* works = (work_t*)calloc((size_t)threads, sizeof(work_t));
    pthread_t* tids = (pthread_t*)calloc((size_t)threads, sizeof(pthread_t));
    int rc = 0;
    if (!works || !tids) rc = -2;
    uint32_t lo = pivot_lo < pivot_hi ? pivot_lo : pivot_hi;
    for (int t = 0; t < threads && rc == 0; ++t) {
        work_t* w = &works[t];
        w->n = n; w->Lv = Lv; w->Le = Le;
        w->ets = ets; w->eel = el ? eel : NULL; w->vl = vl;
        w->deg = deg; w->adj_start = adj_start; w->adj = adj; w->vertex_at = vertex_at;
        w->t_lo = t_lo; w->t_hi = t_hi;
        w->p_lo = lo;
        w->p_hi = pivot_hi;
        w->t = (uint32_t)t;
        w->stride = (uint32_t)threads;
        if (t == 0) {
            w->out = *out; /* thread 0 accumulates straight into the caller's arrays */
        } else {
            w->out.count = out->count ? (uint64_t*)calloc(1, 8) : NULL;
            w->out.hist = out->hist ? (uint64_t*)calloc(HIST_BINS, 8) : NULL;
            w->out.vtri = out->vtri ? (uint64_t*)calloc(lv3, 8) : NULL;
            w->out.etri = out->etri ? (uint64_t*)calloc(le3, 8) : NULL;
            w->out.joint = out->joint ? (uint64_t*)calloc(HIST_BINS * HIST_BINS, 8) : NULL;
            w->out.maxel = out->maxel ? (uint64_t*)calloc(Le, 8) : NULL;
            w->out.degtri = out->degtri ? (uint64_t*)calloc(dt3, 8) : NULL;
            w->out.vlocal = out->vlocal ? (uint64_t*)calloc((size_t)n + 1, 8) : NULL;
            w->out.elocal = out->elocal ? (uint64_t*)calloc((size_t)m + 1, 8) : NULL;
            if ((out->count && !w->out.count) || (out->hist && !w->out.hist) ||
                (out->vtri && !w->out.vtri) || (out->etri && !w->out.etri) ||
                (out->joint && !w->out.joint) || (out->maxel && !w->out.maxel) ||
                (out->degtri && !w->out.degtri) || (out->vlocal && !w->out.vlocal) ||
                (out->elocal && !w->out.elocal))
                rc = -2;
        }
    }
    if (rc == 0) {
        for (int t = 1; t < threads; ++t) pthread_create(&tids[t], NULL, survey_pivots, &works[t]);
        survey_pivots(&works[0]);
        for (int t = 1; t < threads; ++t) pthread_join(tids[t], NULL);
        for (int t = 1; t < threads; ++t) {
            const oracle_out* o = &works[t].out;
            add_into(out->count, o->count, 1);
            add_into(out->hist, o->hist, HIST_BINS);
            add_into(out->vtri, o->vtri, lv3);
            add_into(out->etri, o->etri, le3);
            add_into(out->joint, o->joint, HIST_BINS * HIST_BINS);
            add_into(out->maxel, o->maxel, Le);
            add_into(out->degtri, o->degtri, dt3);
            add_into(out->vlocal, o->vlocal, n);
            add_into(out->elocal, o->elocal, m);
        }
    }
    for (int t = 1; works && t < threads; ++t) {
        oracle_out* o = &works[t].out;
        free(o->count); free(o->hist); free(o->vtri); free(o->etri); free(o->joint);
        free(o->maxel); free(o->degtri); free(o->vlocal);
        free(o->elocal);
    }
    free(works); free(tids);
    free(eu); free(ev); free(ets); free(eel); free(deg); free(vertex_at); free(pos_of);
    free(adj_start); free(adj);
    return rc;
}

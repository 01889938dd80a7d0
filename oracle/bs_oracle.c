/*
 * bs_oracle.c -- plain, slow CPU oracle of the block-decomposed sort.
 *
 * TEST INFRASTRUCTURE ONLY: loaded by the tests, the smoke check and the
 * benchmark's CPU-baseline leg; never by the product path.  It shares no code
 * with the CUDA library.
 *
 * Every function follows El-Nashar, "Parallel performance of MPI sorting
 * algorithms on dual-core processor Windows-based systems" (IJDPS 2(3),
 * 2011); the section, figure or step it restates is named beside it.
 * Readings taken where the paper is silent or garbled:
 *   - s = n/p when p does not divide n: balanced bounds floor(i*n/p).
 *   - merge ties: the left (lower-id) list wins, which makes merges stable.
 *   - Fig. 3 mixes 'start' and 'first': read as the standard top-down split
 *     [first, mid], [mid+1, last] with mid = (first+last)/2.
 *   - Fig. 4 names an undefined 's' in the pivot swap: read as 'start'.
 *   - Fig. 1's merge loop never advances 'step' and only pairs (even, even+1):
 *     read as odd-even compare-split rounds that alternate between
 *     (even, even+1) and (odd, odd+1) pairs, p rounds in all, over p blocks
 *     of equal capacity ceil(n/p) padded with +infinity sentinels.
 *   - Section 3.2.2's gather form: the master folds the sorted sub-lists into
 *     its list one after another, in id order.
 *
 * ORC_MUT (compile-time, default 0) plants one numbered mistake; the test
 * suite builds those variants to show that its pins catch each one.
 */
#include "bs_oracle.h"

#include <pthread.h>
#include <stdlib.h>
#include <string.h>

#ifndef ORC_MUT
#define ORC_MUT 0
#endif

/* ------------------------------------------------------------------------ */
/* Codec: order-preserving unsigned codes.  Integers: flip the sign bit.     */
/* Floating point (IEEE 754-2008 totalOrder, Sec. 5.10): negative patterns   */
/* are bit-inverted, non-negative ones get the sign bit set.                 */
/* ------------------------------------------------------------------------ */

static uint64_t enc_f32_bits(uint32_t b) {
#if ORC_MUT == 2
    return (uint64_t)(b | 0x80000000u); /* planted: negatives not inverted */
#else
    return (uint64_t)((b & 0x80000000u) ? ~b : (b | 0x80000000u));
#endif
}
static uint32_t dec_f32_bits(uint64_t c) {
    uint32_t u = (uint32_t)c;
    return (u & 0x80000000u) ? (u & 0x7fffffffu) : ~u;
}
static uint64_t enc_f64_bits(uint64_t b) {
    return (b & 0x8000000000000000ull) ? ~b : (b | 0x8000000000000000ull);
}
static uint64_t dec_f64_bits(uint64_t c) {
    return (c & 0x8000000000000000ull) ? (c & 0x7fffffffffffffffull) : ~c;
}

int orc_encode(const void *keys, int dtype, int64_t n, uint64_t *codes) {
    if (n < 0 || (n > 0 && (!keys || !codes))) return -1;
    for (int64_t i = 0; i < n; i++) {
        switch (dtype) {
        case ORC_I32: {
            uint32_t u;
            memcpy(&u, (const char *)keys + 4 * i, 4);
#if ORC_MUT == 8
            codes[i] = (uint64_t)u; /* planted: sign bit not flipped */
#else
            codes[i] = (uint64_t)(u ^ 0x80000000u);
#endif
            break;
        }
        case ORC_U32: {
            uint32_t u;
            memcpy(&u, (const char *)keys + 4 * i, 4);
            codes[i] = u;
            break;
        }
        case ORC_F32: {
            uint32_t u;
            memcpy(&u, (const char *)keys + 4 * i, 4);
            codes[i] = enc_f32_bits(u);
            break;
        }
        case ORC_I64: {
            uint64_t u;
            memcpy(&u, (const char *)keys + 8 * i, 8);
            codes[i] = u ^ 0x8000000000000000ull;
            break;
        }
        case ORC_U64: {
            uint64_t u;
            memcpy(&u, (const char *)keys + 8 * i, 8);
            codes[i] = u;
            break;
        }
        case ORC_F64: {
            uint64_t u;
            memcpy(&u, (const char *)keys + 8 * i, 8);
            codes[i] = enc_f64_bits(u);
            break;
        }
        default:
            return -2;
        }
    }
    return 0;
}

int orc_decode(const uint64_t *codes, int dtype, int64_t n, void *keys) {
    if (n < 0 || (n > 0 && (!keys || !codes))) return -1;
    for (int64_t i = 0; i < n; i++) {
        uint32_t u32;
        uint64_t u64;
        switch (dtype) {
        case ORC_I32:
            u32 = (uint32_t)codes[i] ^ 0x80000000u;
            memcpy((char *)keys + 4 * i, &u32, 4);
            break;
        case ORC_U32:
            u32 = (uint32_t)codes[i];
            memcpy((char *)keys + 4 * i, &u32, 4);
            break;
        case ORC_F32:
            u32 = dec_f32_bits(codes[i]);
            memcpy((char *)keys + 4 * i, &u32, 4);
            break;
        case ORC_I64:
            u64 = codes[i] ^ 0x8000000000000000ull;
            memcpy((char *)keys + 8 * i, &u64, 8);
            break;
        case ORC_U64:
            u64 = codes[i];
            memcpy((char *)keys + 8 * i, &u64, 8);
            break;
        case ORC_F64:
            u64 = dec_f64_bits(codes[i]);
            memcpy((char *)keys + 8 * i, &u64, 8);
            break;
        default:
            return -2;
        }
    }
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Scatter phase (Fig. 1): block i holds items [b_i, b_{i+1}).              */
/* ------------------------------------------------------------------------ */

int orc_block_bounds(int64_t n, int64_t p, int64_t *bounds) {
    if (n < 0 || p < 1 || !bounds) return -1;
    for (int64_t i = 0; i <= p; i++)
        bounds[i] = (int64_t)(((__int128)i * (__int128)n) / (__int128)p);
#if ORC_MUT == 3
    if (n > 0) bounds[p] = n - 1; /* planted: last item left out of the blocks */
#endif
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Records and the stable two-list merge.                                    */
/* ------------------------------------------------------------------------ */

typedef struct {
    uint64_t *code;
    uint64_t *val; /* may be NULL */
} recs;

static void rec_swap(recs r, int64_t i, int64_t j) {
    /* the exchange function of Fig. 2 */
    uint64_t t = r.code[i];
    r.code[i] = r.code[j];
    r.code[j] = t;
    if (r.val) {
        t = r.val[i];
        r.val[i] = r.val[j];
        r.val[j] = t;
    }
}

/*
 * Merge the sorted lists A = src[a0, a1) and B = src[b0, b1) into dst[d0..].
 * An A item is taken first when A <= B, so equal codes keep list order.
 */
static void merge_lists(recs src, int64_t a0, int64_t a1, int64_t b0, int64_t b1,
                        recs dst, int64_t d0) {
    int64_t i = a0, j = b0, k = d0;
    while (i < a1 && j < b1) {
#if ORC_MUT == 1
        int take_a = src.code[i] < src.code[j]; /* planted: ties go to B */
#else
        int take_a = src.code[i] <= src.code[j];
#endif
        int64_t s = take_a ? i++ : j++;
        dst.code[k] = src.code[s];
        if (dst.val) dst.val[k] = src.val[s];
        k++;
    }
    while (i < a1) {
        dst.code[k] = src.code[i];
        if (dst.val) dst.val[k] = src.val[i];
        i++, k++;
    }
#if ORC_MUT != 4 /* planted (4): the rest of B is dropped */
    while (j < b1) {
        dst.code[k] = src.code[j];
        if (dst.val) dst.val[k] = src.val[j];
        j++, k++;
    }
#endif
}

/* ------------------------------------------------------------------------ */
/* Sort phase: the three sequential sorts of Section 3.2.                    */
/* ------------------------------------------------------------------------ */

/* Fig. 3: top-down merge sort of r[first..last] (inclusive); tmp is the     */
/* duplicate list the paper notes merge sort needs (Section 3.3).            */
static void merge_sort_rec(recs r, recs tmp, int64_t first, int64_t last) {
    if (last <= first) return;
    int64_t mid = first + (last - first) / 2;
    merge_sort_rec(r, tmp, first, mid);
    merge_sort_rec(r, tmp, mid + 1, last);
    merge_lists(r, first, mid + 1, mid + 1, last + 1, tmp, first);
    memcpy(r.code + first, tmp.code + first, (size_t)(last - first + 1) * 8);
    if (r.val) memcpy(r.val + first, tmp.val + first, (size_t)(last - first + 1) * 8);
}

/* Fig. 2: bubble sort of r[lo, lo+s) by adjacent exchange on a strict '>'. */
static void bubble_sort(recs r, int64_t lo, int64_t s) {
    for (int64_t i = s - 2; i >= 0; i--) {
#if ORC_MUT == 5
        for (int64_t j = 0; j < i; j++) /* planted: inner bound one short */
#else
        for (int64_t j = 0; j <= i; j++)
#endif
            if (r.code[lo + j] > r.code[lo + j + 1]) rec_swap(r, lo + j, lo + j + 1);
    }
}

/* Fig. 4: quick sort of r[start, start+length): middle pivot swapped to the
 * front, partition on '< pivot', pivot swapped into place, recurse. */
static void quick_sort(recs r, int64_t start, int64_t length) {
    if (length <= 1) return;
    uint64_t pivot = r.code[start + length / 2];
    rec_swap(r, start, start + length / 2);
    int64_t pstart = start;
    for (int64_t i = start + 1; i < start + length; i++) {
        if (r.code[i] < pivot) {
            pstart++;
            rec_swap(r, i, pstart);
        }
    }
    rec_swap(r, start, pstart);
    quick_sort(r, start, pstart - start);
    quick_sort(r, pstart + 1, start + length - pstart - 1);
}

static int local_sort(recs r, recs tmp, int64_t lo, int64_t hi, int alg) {
    int64_t s = hi - lo;
    if (s <= 1) return 0;
    switch (alg) {
    case ORC_LOCAL_MERGE:
        merge_sort_rec(r, tmp, lo, hi - 1);
        return 0;
    case ORC_LOCAL_BUBBLE:
        bubble_sort(r, lo, s);
        return 0;
    case ORC_LOCAL_QUICK:
        quick_sort(r, lo, s);
        return 0;
    default:
        return -2;
    }
}

/* ------------------------------------------------------------------------ */
/* A tiny static thread pool: task t of ntasks runs on thread t % threads.   */
/* ------------------------------------------------------------------------ */

typedef void (*task_fn)(void *ctx, int64_t t);
typedef struct {
    task_fn fn;
    void *ctx;
    int64_t ntasks;
    int64_t tid;
    int64_t nthreads;
} pool_arg;

static void *pool_worker(void *p) {
    pool_arg *a = (pool_arg *)p;
    for (int64_t t = a->tid; t < a->ntasks; t += a->nthreads) a->fn(a->ctx, t);
    return NULL;
}

static void run_tasks(task_fn fn, void *ctx, int64_t ntasks, int threads) {
    if (threads <= 1 || ntasks <= 1) {
        for (int64_t t = 0; t < ntasks; t++) fn(ctx, t);
        return;
    }
    int64_t nt = threads < ntasks ? threads : ntasks;
    pthread_t *th = (pthread_t *)malloc(sizeof(pthread_t) * (size_t)nt);
    pool_arg *args = (pool_arg *)malloc(sizeof(pool_arg) * (size_t)nt);
    int64_t started = 0;
    for (int64_t i = 0; i < nt; i++) {
        args[i].fn = fn, args[i].ctx = ctx, args[i].ntasks = ntasks;
        args[i].tid = i, args[i].nthreads = nt;
        if (pthread_create(&th[i], NULL, pool_worker, &args[i]) != 0) break;
        started++;
    }
    /* any thread that failed to start: run its share here */
    for (int64_t i = started; i < nt; i++) pool_worker(&args[i]);
    for (int64_t i = 0; i < started; i++) pthread_join(th[i], NULL);
    free(th);
    free(args);
}

/* ------------------------------------------------------------------------ */
/* The paradigm of Fig. 1.                                                   */
/* ------------------------------------------------------------------------ */

typedef struct {
    recs r, tmp;
    const int64_t *b; /* bounds */
    int alg;
    int err;
} sort_ctx;

static void sort_block_task(void *c, int64_t i) {
    sort_ctx *s = (sort_ctx *)c;
    if (local_sort(s->r, s->tmp, s->b[i], s->b[i + 1], s->alg) != 0) s->err = 1;
}

typedef struct {
    recs src, dst;
    const int64_t *runs; /* run starts, nruns+1 entries */
    int64_t nruns;
} tree_ctx;

static void tree_pair_task(void *c, int64_t k) {
    tree_ctx *t = (tree_ctx *)c;
    int64_t ra = 2 * k, rb = 2 * k + 1;
    int64_t a0 = t->runs[ra], a1 = t->runs[ra + 1];
    if (rb < t->nruns) {
        merge_lists(t->src, a0, a1, a1, t->runs[rb + 1], t->dst, a0);
    } else {
#if ORC_MUT != 7 /* planted (7): an unpaired last run is not carried */
        merge_lists(t->src, a0, a1, a1, a1, t->dst, a0);
#endif
    }
}

/* Pairwise merge tree: runs (2k, 2k+1) merge each round until one is left. */
static void merge_tree(recs r, recs tmp, const int64_t *bounds, int64_t p, int threads) {
    int64_t nruns = p;
    int64_t *runs = (int64_t *)malloc(sizeof(int64_t) * (size_t)(p + 1));
    memcpy(runs, bounds, sizeof(int64_t) * (size_t)(p + 1));
    recs src = r, dst = tmp;
    while (nruns > 1) {
        tree_ctx c = {src, dst, runs, nruns};
        int64_t npairs = (nruns + 1) / 2;
        run_tasks(tree_pair_task, &c, npairs, threads);
        for (int64_t k = 0; k < npairs; k++) runs[k] = runs[2 * k];
        runs[npairs] = runs[nruns];
        nruns = npairs;
        recs t = src;
        src = dst;
        dst = t;
    }
    if (src.code != r.code) {
        int64_t n = bounds[p] - bounds[0];
        memcpy(r.code + bounds[0], src.code + bounds[0], (size_t)n * 8);
        if (r.val) memcpy(r.val + bounds[0], src.val + bounds[0], (size_t)n * 8);
    }
    free(runs);
}

/*
 * Odd-even compare-split (the reading of Fig. 1's merge phase).  The paper's
 * partition size s = n/p assumes equal blocks; p alternating rounds sort p
 * equal blocks, but not unequal ones (n = 4, p = 3 is a counterexample).  So
 * every block gets the capacity s = ceil(n/p): its items, then +infinity
 * sentinels (pad = 1) that order after every item.  Compare-split of blocks
 * (i, i+1): merge both by (pad, code), stably; the lower id keeps the first
 * s slots, the higher id the rest.  After p rounds the items fill the first
 * n slots in order.
 */
typedef struct {
    uint64_t *code, *val;
    uint8_t *pad;
} slots;

static void merge_split_slots(slots a, slots t, int64_t lo, int64_t mid, int64_t hi) {
    int64_t i = lo, j = mid, k = lo;
    while (i < mid || j < hi) {
        int take_a;
        if (j >= hi) take_a = 1;
        else if (i >= mid) take_a = 0;
        else if (a.pad[i] != a.pad[j]) take_a = a.pad[i] < a.pad[j];
        else take_a = a.code[i] <= a.code[j];
        int64_t s = take_a ? i++ : j++;
        t.code[k] = a.code[s];
        t.pad[k] = a.pad[s];
        if (t.val) t.val[k] = a.val[s];
        k++;
    }
    memcpy(a.code + lo, t.code + lo, (size_t)(hi - lo) * 8);
    memcpy(a.pad + lo, t.pad + lo, (size_t)(hi - lo));
    if (a.val) memcpy(a.val + lo, t.val + lo, (size_t)(hi - lo) * 8);
}

typedef struct {
    slots a, t;
    int64_t cap;   /* slots per block */
    int64_t first; /* lower id of the first pair this round */
} oe_ctx;

static void oddeven_pair_task(void *c, int64_t k) {
    oe_ctx *o = (oe_ctx *)c;
    int64_t i = o->first + 2 * k;
    merge_split_slots(o->a, o->t, i * o->cap, (i + 1) * o->cap, (i + 2) * o->cap);
}

static int merge_oddeven(recs r, const int64_t *bounds, int64_t p, int threads) {
    int64_t n = bounds[p] - bounds[0];
    int64_t cap = (n + p - 1) / p, m = cap * p;
    slots a, t;
    a.code = (uint64_t *)malloc((size_t)m * 8), t.code = (uint64_t *)malloc((size_t)m * 8);
    a.pad = (uint8_t *)malloc((size_t)m), t.pad = (uint8_t *)malloc((size_t)m);
    a.val = r.val ? (uint64_t *)malloc((size_t)m * 8) : NULL;
    t.val = r.val ? (uint64_t *)malloc((size_t)m * 8) : NULL;
    int ok = a.code && t.code && a.pad && t.pad && (!r.val || (a.val && t.val));
    if (ok) {
        for (int64_t i = 0; i < p; i++) {
            for (int64_t s = 0; s < cap; s++) {
                int64_t x = bounds[i] + s, y = i * cap + s;
                int real = x < bounds[i + 1];
                a.pad[y] = (uint8_t)!real;
                a.code[y] = real ? r.code[x] : ~0ull;
                if (a.val) a.val[y] = real ? r.val[x] : 0;
            }
        }
#if ORC_MUT == 6
        int64_t rounds = p - 1; /* planted: one round short */
#else
        int64_t rounds = p;
#endif
        for (int64_t step = 0; step < rounds; step++) {
            int64_t first = step & 1; /* even rounds (0,1),(2,3)..; odd rounds (1,2),(3,4).. */
            oe_ctx c = {a, t, cap, first};
            run_tasks(oddeven_pair_task, &c, (p - first) / 2, threads);
        }
        int64_t k = bounds[0];
        for (int64_t y = 0; y < m; y++) {
            if (a.pad[y]) continue;
            r.code[k] = a.code[y];
            if (r.val) r.val[k] = a.val[y];
            k++;
        }
    }
    free(a.code), free(t.code), free(a.pad), free(t.pad), free(a.val), free(t.val);
    return ok ? 0 : -3;
}

/* Gather form (Sec. 3.2.2): the master merges each received sub-list into
 * the list it holds, in id order. */
static void merge_gather(recs r, recs tmp, const int64_t *bounds, int64_t p) {
    for (int64_t i = 1; i < p; i++) {
        int64_t a0 = bounds[0], a1 = bounds[i], b1 = bounds[i + 1];
        merge_lists(r, a0, a1, a1, b1, tmp, a0);
        memcpy(r.code + a0, tmp.code + a0, (size_t)(b1 - a0) * 8);
        if (r.val) memcpy(r.val + a0, tmp.val + a0, (size_t)(b1 - a0) * 8);
    }
}

int orc_sort_records(uint64_t *codes, uint64_t *vals, int64_t n, int64_t p,
                     int local_alg, int form, int threads) {
    if (n < 0 || p < 1 || threads < 1) return -1;
    if (n > 0 && !codes) return -1;
    if (local_alg == ORC_LOCAL_QUICK && vals) return -1; /* quick sort is not stable */
    if (local_alg < ORC_LOCAL_MERGE || local_alg > ORC_LOCAL_QUICK) return -2;
    if (form < ORC_FORM_TREE || form > ORC_FORM_GATHER) return -2;
    if (n == 0) return 0;
    if (p > n) p = n;

    int64_t *bounds = (int64_t *)malloc(sizeof(int64_t) * (size_t)(p + 1));
    uint64_t *tc = (uint64_t *)malloc((size_t)n * 8);
    uint64_t *tv = vals ? (uint64_t *)malloc((size_t)n * 8) : NULL;
    if (!bounds || !tc || (vals && !tv)) {
        free(bounds), free(tc), free(tv);
        return -3;
    }
    orc_block_bounds(n, p, bounds);
    recs r = {codes, vals}, tmp = {tc, tv};

    /* sort phase: one task per block (an MPI process in the paper) */
    sort_ctx sc = {r, tmp, bounds, local_alg, 0};
    run_tasks(sort_block_task, &sc, p, threads);

    /* merge phase */
    if (p > 1) {
        if (form == ORC_FORM_TREE) merge_tree(r, tmp, bounds, p, threads);
        else if (form == ORC_FORM_ODDEVEN) {
            if (merge_oddeven(r, bounds, p, threads) != 0) sc.err = 1;
        }
        else merge_gather(r, tmp, bounds, p);
    }
    free(bounds), free(tc), free(tv);
    return sc.err ? -4 : 0;
}

typedef struct {
    recs r, tmp;
    const int64_t *off;
} seg_ctx;

static void sort_segment_task(void *c, int64_t s) {
    seg_ctx *g = (seg_ctx *)c;
    local_sort(g->r, g->tmp, g->off[s], g->off[s + 1], ORC_LOCAL_MERGE);
}

int orc_sort_segments(uint64_t *codes, uint64_t *vals, const int64_t *off,
                      int64_t S, int threads) {
    if (S < 0 || threads < 1 || (S > 0 && !off)) return -1;
    if (S == 0) return 0;
    for (int64_t s = 0; s < S; s++)
        if (off[s + 1] < off[s]) return -1;
    int64_t lo = off[0], hi = off[S];
    if (lo < 0 || (hi > lo && !codes)) return -1;
    uint64_t *tc = (uint64_t *)malloc((size_t)(hi > 0 ? hi : 1) * 8);
    uint64_t *tv = vals ? (uint64_t *)malloc((size_t)(hi > 0 ? hi : 1) * 8) : NULL;
    if (!tc || (vals && !tv)) {
        free(tc), free(tv);
        return -3;
    }
    seg_ctx g = {{codes, vals}, {tc, tv}, off};
    run_tasks(sort_segment_task, &g, S, threads);
    free(tc), free(tv);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Checkers.                                                                 */
/* ------------------------------------------------------------------------ */

int orc_is_nondecreasing(const uint64_t *codes, int64_t n) {
    for (int64_t i = 1; i < n; i++)
        if (codes[i - 1] > codes[i]) return 0;
    return 1;
}

/* Two unrelated 64-bit finalisers (MurmurHash3's fmix64 and a xorshift-
 * multiply mix); a sum of mixed codes is a commutative multiset hash. */
static uint64_t mix_a(uint64_t x) {
    x ^= x >> 33;
    x *= 0xff51afd7ed558ccdull;
    x ^= x >> 33;
    x *= 0xc4ceb9fe1a85ec53ull;
    x ^= x >> 33;
    return x;
}
static uint64_t mix_b(uint64_t x) {
    x += 0x632be59bd9b4e019ull;
    x ^= x >> 29;
    x *= 0xbf58476d1ce4e5b9ull;
    x ^= x >> 32;
    x *= 0x94d049bb133111ebull;
    x ^= x >> 29;
    return x;
}

uint64_t orc_multiset_hash(const uint64_t *codes, int64_t n, int which) {
    uint64_t h = 0;
    for (int64_t i = 0; i < n; i++) h += which ? mix_b(codes[i]) : mix_a(codes[i]);
    return h;
}

int orc_rank_bounds(const uint64_t *codes, int64_t n, uint64_t v, int64_t *n_less,
                    int64_t *n_leq) {
    if (!n_less || !n_leq || n < 0) return -1;
    int64_t lt = 0, le = 0;
    for (int64_t i = 0; i < n; i++) {
        lt += codes[i] < v;
        le += codes[i] <= v;
    }
    *n_less = lt;
    *n_leq = le;
    return 0;
}

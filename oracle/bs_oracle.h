/*
 * bs_oracle.h -- CPU oracle for the block-decomposed sort (test infrastructure).
 *
 * THIS IS TEST INFRASTRUCTURE, NOT PART OF THE PRODUCT PATH.  Only the tests,
 * the smoke check and the CPU-baseline leg of the benchmark may load it.  It
 * shares no code, header, table or constant with the CUDA library.
 *
 * What it computes: the scatter / sort / merge paradigm of El-Nashar (IJDPS
 * 2011), Section 3.2 and Figure 1, applied to records (code, payload):
 *   1. scatter: the n items are split into p blocks with balanced bounds
 *      b_i = floor(i*n/p)                        (Fig. 1, scatter phase)
 *   2. sort phase: every block is sorted by one of the paper's sequential
 *      sorts -- top-down merge sort (Fig. 3), bubble sort (Fig. 2) or
 *      quick sort (Fig. 4)                        (Fig. 1, sort phase)
 *   3. merge phase: sorted blocks are merged into one list, in one of three
 *      forms: a pairwise merge tree, the odd-even compare-split exchange read
 *      from Fig. 1's merge phase, or the gather-to-master fold of Section 3.2.2.
 * Keys are ordered by an order-preserving unsigned code (IEEE 754-2008
 * totalOrder for floating point), so every comparison is an integer one.
 *
 * Errors: every function returning int returns 0 on success and a negative
 * value on invalid arguments or allocation failure.
 */
#ifndef BS_ORACLE_H
#define BS_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* key dtypes understood by the oracle's own codec */
enum { ORC_I32 = 0, ORC_U32 = 1, ORC_F32 = 2, ORC_I64 = 3, ORC_U64 = 4, ORC_F64 = 5 };
/* local (sort-phase) algorithms: Fig. 3, Fig. 2, Fig. 4 */
enum { ORC_LOCAL_MERGE = 0, ORC_LOCAL_BUBBLE = 1, ORC_LOCAL_QUICK = 2 };
/* merge-phase forms: pairwise tree, odd-even compare-split (Fig. 1), gather fold (Sec. 3.2.2) */
enum { ORC_FORM_TREE = 0, ORC_FORM_ODDEVEN = 1, ORC_FORM_GATHER = 2 };

/* Codec: keys[n] of dtype -> codes[n] (uint64, order preserving); and back. */
int orc_encode(const void *keys, int dtype, int64_t n, uint64_t *codes);
int orc_decode(const uint64_t *codes, int dtype, int64_t n, void *keys);

/* Balanced scatter bounds b_0..b_p (p+1 values) for n items in p blocks. */
int orc_block_bounds(int64_t n, int64_t p, int64_t *bounds);

/*
 * The whole method on records: codes[n] and (optional, may be NULL) vals[n]
 * are sorted in place into nondecreasing code order.  With the merge-sort or
 * bubble local sort every form is stable (equal codes keep input order);
 * the quick-sort local sort is keys-only (vals must be NULL).
 * p >= 1 blocks (p > n is clamped to n); threads >= 1 worker threads.
 */
int orc_sort_records(uint64_t *codes, uint64_t *vals, int64_t n, int64_t p,
                     int local_sort, int merge_form, int threads);

/* Independent sorts of S segments [off[s], off[s+1]) of codes/vals (stable). */
int orc_sort_segments(uint64_t *codes, uint64_t *vals, const int64_t *off,
                      int64_t S, int threads);

/* Checkers on code arrays. */
int orc_is_nondecreasing(const uint64_t *codes, int64_t n);          /* 1 / 0 */
uint64_t orc_multiset_hash(const uint64_t *codes, int64_t n, int which); /* which = 0 or 1 */
/* number of codes < v and number of codes <= v (rank bounds of value v) */
int orc_rank_bounds(const uint64_t *codes, int64_t n, uint64_t v,
                    int64_t *n_less, int64_t *n_leq);

#ifdef __cplusplus
}
#endif
#endif

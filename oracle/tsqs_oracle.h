/*
 * tsqs_oracle.h -- CPU oracle for Triple State QuickSort (Muqaddas, arXiv 1505.00558).
 *
 * TEST INFRASTRUCTURE ONLY.  This library is the slow, single-threaded, obviously
 * correct reference that the CUDA path is checked against.  Only the test suite,
 * the smoke check in __graft_entry__.py and the cpu_baseline / reference legs of
 * bench.py may load it.  The product library (libtsqs) never links or calls it,
 * and the two share no source, header, table or helper.
 *
 * What it implements, in the paper's order and notation:
 *   - the pointer-based qsort replacement: an untyped array `base` of `n` elements of
 *     `ses` bytes and a comparator chosen by key kind (Section VII; the comparator
 *     sign convention of Section III);
 *   - one recursive stage: initialisation (III.A), State 1 (III.B), the choice of the
 *     next state by inequalities (1) and (2) (III.C), States 2L/2R (III.D),
 *     States 3L/3R with the temporary buffer tar (III.E), copy-back and placement of
 *     temp and p (III.F), recursion that excludes the =p run (III.F);
 *   - pivot selection by size tier: median of 3, median of 5, ninther, fifteenther
 *     (III.H), with the randomised inner sample positions of Section V.C driven by the
 *     Park-Miller generator;
 *   - the copy-based insertion sort for tiny parts (Section IV);
 *   - counters of comparisons and element copies (Section VI; virtual swaps are
 *     copies / 3 as in Section V.A);
 *   - two comparison baselines with a uniformly random pivot: a textbook Hoare
 *     quicksort that counts exchanges (the setting of eqs. (3) and (4)) and the
 *     two-way empty-slot juggling partition of Section II that counts copies
 *     (the model behind eq. (8)).
 *
 * Total order (the "cmp" the library is given): integers in numeric order; floats in
 * IEEE 754 totalOrder (-NaN < -inf < ... < -0 < +0 < ... < +inf < +NaN, NaNs ordered
 * by payload); 16-byte records {uint64 key, uint64 payload} ordered by (key, payload).
 * Two elements compare equal only when they are bitwise identical.
 */
#ifndef TSQS_ORACLE_H
#define TSQS_ORACLE_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Key kinds; the numbering matches the product C-ABI so tests can pass one value. */
enum {
    ORC_I32 = 1, ORC_U32 = 2, ORC_F32 = 3,
    ORC_I64 = 4, ORC_U64 = 5, ORC_F64 = 6,
    ORC_REC = 7
};

/* Pivot policies. */
enum {
    ORC_PIVOT_TIERED = 0,   /* med3 / med5 / ninther / fifteenther by size (III.H) */
    ORC_PIVOT_RANDOM = 1    /* one uniformly random element per stage             */
};

/* Indices into state_entries[]. */
enum {
    ORC_ST_STATE1 = 0,      /* a stage entered State 1                               */
    ORC_ST_2L, ORC_ST_2R, ORC_ST_3L, ORC_ST_3R,
    ORC_ST_INIT_SPECIAL,    /* pre-scan reached mid: every element right of mid > p */
    ORC_ST_EXIT_STATE1,     /* the stage ended while still in State 1               */
    ORC_NSTATES
};

typedef struct {
    int      ins_threshold;  /* parts of n <= ins_threshold go to insertion sort (>= 2) */
    int      pivot_policy;   /* ORC_PIVOT_*                                            */
    int      random_samples; /* 1: shift inner sample positions by the V.C draw         */
    int      med3_below;     /* med3 for n <  med3_below   (paper: 70)                  */
    int      med5_below;     /* med5 for n <  med5_below                               */
    int      ninther_below;  /* ninther for n < ninther_below, fifteenther above        */
    uint64_t seed;           /* Park-Miller state at the start of the call (not 0)      */
} orc_cfg;

typedef struct {
    uint64_t cmps;           /* comparator calls                                       */
    uint64_t moves;          /* element copies: into ar[], tar[], temp and p           */
    uint64_t swaps;          /* exchanges (classical Hoare baseline only)              */
    uint64_t stages;         /* partition stages                                       */
    uint64_t ins_parts;      /* parts finished by insertion sort                       */
    uint64_t max_depth;      /* deepest recursion level reached                        */
    uint64_t tar_peak;       /* most elements held in tar at once                      */
    uint64_t state_entries[ORC_NSTATES];
} orc_stats;

/* Fills *cfg with the defaults: ins_threshold 16, tiered pivots, random samples on,
 * tiers med3 < 70 <= med5 < 800 <= ninther < 40000 <= fifteenther, seed 1. */
void orc_default_cfg(orc_cfg *cfg);

/* Element size in bytes of a key kind, 0 if unknown. */
size_t orc_elem_size(int key_kind);

/* Three-way comparison of two elements: <0, 0, >0. */
int orc_compare(const void *x, const void *y, int key_kind);

/* Triple State QuickSort of base[0..n) in place.  cfg may be NULL (defaults); st may
 * be NULL.  Returns 0, or -1 on a bad key kind / allocation failure. */
int orc_tsqs_sort(void *base, size_t n, int key_kind, const orc_cfg *cfg, orc_stats *st);

/* Sorts each of nrows consecutive rows of n elements independently (one call per row,
 * one shared cfg and Park-Miller stream; stats accumulate, max_depth is a maximum). */
int orc_tsqs_sort_rows(void *base, size_t nrows, size_t n, int key_kind,
                       const orc_cfg *cfg, orc_stats *st);

/* Sorts each segment [offs[s], offs[s+1]) of base independently with orc_tsqs_sort,
 * spreading segments over `threads` POSIX threads (1 = on the calling thread). */
int orc_tsqs_sort_segments(void *base, const uint64_t *offs, size_t nseg, int key_kind,
                           int threads);

/* Late swapping for large elements (Section VIII.H): base holds n elements of es
 * bytes, each with a key of kind key_kind (ORC_I32..ORC_F64) at byte offset key_off.
 * Sorts the array of element pointers with Triple State QuickSort (keys decide, equal
 * keys keep their original order) and then moves every element into place along the
 * cycles of the permutation, one temporary element per cycle.  Reports the element
 * moves (n - fixed points + cycles) and the cycle count.  Returns 0, or -1 on bad
 * arguments or allocation failure. */
int orc_wide_sort(void *base, size_t n, size_t es, size_t key_off, int key_kind,
                  uint64_t *moves_out, uint64_t *cycles_out);

/* Textbook quicksort: uniformly random pivot per stage, Hoare partition that compares
 * every non-pivot element exactly once, no insertion sort.  Counts cmps and swaps
 * (exchanges of a misplaced pair; moving the pivot is not an exchange). */
int orc_classical_sort(void *base, size_t n, int key_kind, uint64_t seed, orc_stats *st);

/* Quicksort with the two-way empty-slot juggling partition of Section II and a
 * uniformly random pivot per stage.  Counts cmps and moves (copies into holes plus the
 * copy into and out of temp). */
int orc_juggle_sort(void *base, size_t n, int key_kind, uint64_t seed, orc_stats *st);

/* One Triple State stage on base[0..n) (n >= 3) with the pivot forced to index pi;
 * *lo / *hi receive the last index of the left part and the first of the right part. */
int orc_tsqs_stage(void *base, size_t n, int key_kind, size_t pi, orc_stats *st,
                   long long *lo, long long *hi);

/* Pivot selection alone (Section III.H tiers) on the part base[0..n), n >= 3, with
 * mid = (n-1)/2: sorts the tier's samples in place exactly as a stage would and
 * returns the pivot index (-1 on bad arguments).  Counts its cmps and moves in st. */
long long orc_choose_pivot(void *base, size_t n, int key_kind, const orc_cfg *cfg,
                           orc_stats *st);

/* One textbook Hoare stage (as in orc_classical_sort) with the pivot at index pi. */
int orc_hoare_stage(void *base, size_t n, int key_kind, size_t pi, orc_stats *st);

/* Median of three with orientation as in Section III.I: sorts the three elements
 * ar[i0], ar[i1], ar[i2] (as positioned) in place and returns +1 if they were already
 * ascending (x0 <= x1 <= x2), -1 if strictly descending (x0 > x1 > x2), 0 otherwise. */
int orc_median3(void *base, size_t i0, size_t i1, size_t i2, int key_kind, orc_stats *st);

/* Lower median of s keys: sorts a private copy and writes element (s-1)/2 to out. */
int orc_lower_median(const void *keys, size_t s, int key_kind, void *out);

/* Plain definition of one three-way partition of in[0..n) around the value *pivot:
 * out receives the elements < p in input order, then the elements == p, then the
 * elements > p in input order.  Writes the three counts. */
int orc_three_way_split(const void *in, void *out, size_t n, int key_kind,
                        const void *pivot, size_t *nlt, size_t *neq, size_t *ngt);

#ifdef __cplusplus
}
#endif
#endif /* TSQS_ORACLE_H */

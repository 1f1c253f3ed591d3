/*
 * tsqs_oracle.c -- CPU oracle for Triple State QuickSort (arXiv 1505.00558).
 *
 * TEST INFRASTRUCTURE ONLY: loaded by the tests, by __graft_entry__.smoke() and by
 * the CPU legs of bench.py.  The product path never links, loads or calls it.
 *
 * The code follows the paper's steps and names (ar, a, b, mid, p, pi, l, r, m, ml,
 * mr, temp, tar, i, lc, k, k2) but is written as one loop around a switch over
 * explicit states instead of the paper's goto labels, which the paper itself says is
 * an equivalent form (end of Section III.B).  The readings taken where the printed
 * algorithm omits a case are marked "Reading:" in the comments.
 *
 * Invariants used throughout one stage on [a, b] (n = b - a + 1 >= 3):
 *   - ar[a..l-1] < p and ar[r+1..b] > p;
 *   - two slots of ar[] are "holes" (their element lives in p or temp or was copied
 *     elsewhere); every element copy fills a hole and opens another one;
 *   - State 1: the run of equals is [ml, mr] with its hole at m (m is ml or mr),
 *     the second hole is at l or at r;
 *   - States 2L/3L (right side closed): r is always a hole; 2R/3R mirror this with l.
 */
#include "tsqs_oracle.h"

#include <pthread.h>
#include <stdlib.h>
#include <string.h>

typedef long long idx;   /* signed indices, like the paper's int, wide enough for 2^40 */

/* ------------------------------------------------------------------------------ */
/* Comparators: the "cmp" of Section III, fixed per key kind (Section VII).        */
/* ------------------------------------------------------------------------------ */

static int cmp_i32(const void *x, const void *y) {
    int32_t a, b; memcpy(&a, x, 4); memcpy(&b, y, 4);
    return (a > b) - (a < b);
}
static int cmp_u32(const void *x, const void *y) {
    uint32_t a, b; memcpy(&a, x, 4); memcpy(&b, y, 4);
    return (a > b) - (a < b);
}
static int cmp_i64(const void *x, const void *y) {
    int64_t a, b; memcpy(&a, x, 8); memcpy(&b, y, 8);
    return (a > b) - (a < b);
}
static int cmp_u64(const void *x, const void *y) {
    uint64_t a, b; memcpy(&a, x, 8); memcpy(&b, y, 8);
    return (a > b) - (a < b);
}
/* IEEE 754 totalOrder on a binary format, taken from its definition: a negative sign
 * orders below a positive one (so -0 < +0); among positives a larger magnitude field
 * (exponent and significand read as one unsigned number) is larger, among negatives it
 * is smaller.  NaNs fall at the ends, quiet above signalling, payloads in magnitude
 * order. */
static int cmp_f32(const void *x, const void *y) {
    uint32_t a, b; memcpy(&a, x, 4); memcpy(&b, y, 4);
    uint32_t sa = a >> 31, sb = b >> 31, ma = a & 0x7fffffffu, mb = b & 0x7fffffffu;
    if (sa != sb) return sa ? -1 : 1;
    if (ma == mb) return 0;
    if (!sa) return ma < mb ? -1 : 1;
    return ma > mb ? -1 : 1;
}
static int cmp_f64(const void *x, const void *y) {
    uint64_t a, b; memcpy(&a, x, 8); memcpy(&b, y, 8);
    uint64_t sa = a >> 63, sb = b >> 63;
    uint64_t ma = a & 0x7fffffffffffffffull, mb = b & 0x7fffffffffffffffull;
    if (sa != sb) return sa ? -1 : 1;
    if (ma == mb) return 0;
    if (!sa) return ma < mb ? -1 : 1;
    return ma > mb ? -1 : 1;
}
/* 16-byte record {uint64 key; uint64 payload}: lexicographic on (key, payload). */
static int cmp_rec(const void *x, const void *y) {
    uint64_t ka, kb, pa, pb;
    memcpy(&ka, x, 8); memcpy(&pa, (const char *)x + 8, 8);
    memcpy(&kb, y, 8); memcpy(&pb, (const char *)y + 8, 8);
    if (ka != kb) return ka < kb ? -1 : 1;
    return (pa > pb) - (pa < pb);
}

typedef int (*cmp_fn)(const void *, const void *);

static cmp_fn pick_cmp(int kind, size_t *ses) {
    switch (kind) {
    case ORC_I32: *ses = 4; return cmp_i32;
    case ORC_U32: *ses = 4; return cmp_u32;
    case ORC_F32: *ses = 4; return cmp_f32;
    case ORC_I64: *ses = 8; return cmp_i64;
    case ORC_U64: *ses = 8; return cmp_u64;
    case ORC_F64: *ses = 8; return cmp_f64;
    case ORC_REC: *ses = 16; return cmp_rec;
    default: *ses = 0; return NULL;
    }
}

size_t orc_elem_size(int key_kind) { size_t s; pick_cmp(key_kind, &s); return s; }

int orc_compare(const void *x, const void *y, int key_kind) {
    size_t s; cmp_fn f = pick_cmp(key_kind, &s);
    return f ? f(x, y) : 0;
}

void orc_default_cfg(orc_cfg *c) {
    c->ins_threshold = 16;
    c->pivot_policy = ORC_PIVOT_TIERED;
    c->random_samples = 1;
    c->med3_below = 70;          /* Section V.C: median of three for n < 70 */
    c->med5_below = 800;
    c->ninther_below = 40000;
    c->seed = 1;
}

/* ------------------------------------------------------------------------------ */
/* Sort context: the array, element size, comparator, counters and tar.            */
/* ------------------------------------------------------------------------------ */

typedef struct {
    char *ar;            /* base of the whole array                              */
    size_t ses;          /* element size in bytes                                */
    cmp_fn cmp;
    orc_cfg cfg;
    orc_stats *st;
    char *tar;           /* temporary buffer of Section III.E, allocated per call */
    char *p;             /* the pivot, kept outside the array (Fig. 1)           */
    char *temp;          /* the second element kept outside the array            */
    char *scratch;       /* one element of scratch for sample sorting            */
    uint64_t zgen;       /* Park-Miller state (Section V.C)                      */
    double dran;         /* the per-call draw in [0.5, 1.5)                      */
    idx forced_pi;       /* >= 0: pivot index for the next stage (single-stage API) */
} tctx;

#define AR(c, j)  ((c)->ar + (size_t)(j) * (c)->ses)
#define TAR(c, j) ((c)->tar + (size_t)(j) * (c)->ses)

static inline int ccmp(tctx *c, const void *x, const void *y) {
    c->st->cmps++;
    return c->cmp(x, y);
}
static inline void ccopy(tctx *c, void *dst, const void *src) {
    c->st->moves++;
    memcpy(dst, src, c->ses);
}

/* Park-Miller "minimal standard" generator, Section V.C / VI.
 * Reading: the printed modulus 2^31 and 32-bit product overflow are taken as the
 * Lehmer generator z <- 16807 z mod (2^31 - 1) in 64-bit arithmetic; the seed is a
 * fixed configuration value instead of clock() so that runs are reproducible. */
static const uint64_t PM_A = 16807u, PM_M = 2147483647u;
static uint64_t pm_next(uint64_t *z) {
    *z = (PM_A * *z) % PM_M;
    return *z;
}
static uint64_t pm_seed(uint64_t s) {
    s %= PM_M;
    return s ? s : 1;
}
/* A uniformly random index in [0, n) from one Park-Miller draw (the GenRandom2 idea). */
static idx pm_index(uint64_t *z, idx n) {
    double u = (double)pm_next(z) / (double)PM_M;      /* (0, 1) */
    idx k = (idx)(u * (double)n);
    return k >= n ? n - 1 : k;
}

/* ------------------------------------------------------------------------------ */
/* Median selection (Section III.H-I).                                              */
/* ------------------------------------------------------------------------------ */

static void cswap(tctx *c, idx i, idx j) {   /* three copies through scratch */
    ccopy(c, c->scratch, AR(c, i));
    ccopy(c, AR(c, i), AR(c, j));
    ccopy(c, AR(c, j), c->scratch);
}

/* Median of three with orientation.  Sorts ar[i0], ar[i1], ar[i2] in place so the
 * median ends at i1; +1 when they were ascending (x0 <= x1 <= x2), -1 when strictly
 * descending, 0 otherwise.  The decision tree tests x1 against x0 first, then x2, and
 * moves elements by copies through one scratch element (a rotation of three costs
 * four copies, a transposition three). */
static int med3(tctx *c, idx i0, idx i1, idx i2) {
    if (ccmp(c, AR(c, i1), AR(c, i0)) >= 0) {              /* x0 <= x1 */
        if (ccmp(c, AR(c, i2), AR(c, i0)) >= 0) {          /* x0 <= x2 */
            if (ccmp(c, AR(c, i2), AR(c, i1)) >= 0) return 1;   /* x0 <= x1 <= x2 */
            cswap(c, i1, i2);                              /* x0 <= x2 < x1 */
            return 0;
        }
        /* x2 < x0 <= x1: rotate to (x2, x0, x1) */
        ccopy(c, c->scratch, AR(c, i0));
        ccopy(c, AR(c, i0), AR(c, i2));
        ccopy(c, AR(c, i2), AR(c, i1));
        ccopy(c, AR(c, i1), c->scratch);
        return 0;
    }
    /* x1 < x0 */
    if (ccmp(c, AR(c, i2), AR(c, i1)) >= 0) {              /* x1 <= x2 */
        if (ccmp(c, AR(c, i2), AR(c, i0)) >= 0) {          /* x1 < x0 <= x2 */
            cswap(c, i0, i1);
        } else {                                           /* x1 <= x2 < x0: rotate */
            ccopy(c, c->scratch, AR(c, i0));
            ccopy(c, AR(c, i0), AR(c, i1));
            ccopy(c, AR(c, i1), AR(c, i2));
            ccopy(c, AR(c, i2), c->scratch);
        }
        return 0;
    }
    cswap(c, i0, i2);                                      /* x2 < x1 < x0 */
    return -1;
}

/* Sorts the elements at k ascending positions pos[0..k) in place (copy-based insertion
 * over the positions).  Reading: the paper's generated median-of-five decision tree is
 * not printed; any exact in-place ordering of the five samples yields the same median. */
static void sort_positions(tctx *c, const idx *pos, int k) {
    for (int s = 1; s < k; s++) {
        if (ccmp(c, AR(c, pos[s]), AR(c, pos[s - 1])) >= 0) continue;
        ccopy(c, c->scratch, AR(c, pos[s]));
        int j = s;
        ccopy(c, AR(c, pos[j]), AR(c, pos[j - 1]));
        j--;
        while (j > 0 && ccmp(c, c->scratch, AR(c, pos[j - 1])) < 0) {
            ccopy(c, AR(c, pos[j]), AR(c, pos[j - 1]));
            j--;
        }
        ccopy(c, AR(c, pos[j]), c->scratch);
    }
}

/* Inner sample shift of Section V.C for spacing s: floor(s * (dran - 1)), |shift| <= s/2,
 * so shifted samples never cross their neighbours. */
static idx inner_shift(tctx *c, idx s) {
    if (!c->cfg.random_samples) return 0;
    return (idx)((double)s * (c->dran - 1.0));
}

/* Chooses the pivot of [a, b] by the size tiers of Section III.H and returns its index.
 * Every tier sorts its samples in place so that the chosen median sits at mid. */
static idx choose_pivot(tctx *c, idx a, idx b, idx mid) {
    idx n = b - a + 1;
    if (c->cfg.pivot_policy == ORC_PIVOT_RANDOM)
        return a + pm_index(&c->zgen, n);
    if (n < c->cfg.med3_below) {                    /* small: median of (a, mid, b) */
        med3(c, a, mid, b);
        return mid;
    }
    if (n < c->cfg.med5_below) {                    /* medium: median of five */
        idx gap = c->cfg.random_samples ? (idx)((double)(n / 4) * c->dran) : n / 4;
        idx pos[5] = { a, a + gap, mid, b - gap, b };
        sort_positions(c, pos, 5);
        return mid;
    }
    if (n < c->cfg.ninther_below) {                 /* large: ninther */
        idx q[9], s = (n - 1) / 8, d = inner_shift(c, s);
        for (int k = 0; k < 9; k++) q[k] = a + (idx)(((long double)k * (n - 1)) / 8);
        for (int k = 1; k <= 3; k++) q[k] += d;     /* inner samples left of mid  */
        for (int k = 5; k <= 7; k++) q[k] -= d;     /* inner samples right of mid */
        med3(c, q[0], q[1], q[2]);
        med3(c, q[3], q[4], q[5]);
        med3(c, q[6], q[7], q[8]);
        med3(c, q[1], q[4], q[7]);
        return mid;                                 /* q[4] == mid */
    }
    {                                               /* very large: fifteenther */
        idx q[15], s = (n - 1) / 14, d = inner_shift(c, s);
        for (int k = 0; k < 15; k++) q[k] = a + (idx)(((long double)k * (n - 1)) / 14);
        for (int k = 1; k <= 6; k++) q[k] += d;
        for (int k = 8; k <= 13; k++) q[k] -= d;
        for (int g = 0; g < 5; g++) med3(c, q[3 * g], q[3 * g + 1], q[3 * g + 2]);
        idx m5[5] = { q[1], q[4], q[7], q[10], q[13] };
        sort_positions(c, m5, 5);
        return mid;                                 /* q[7] == mid */
    }
}

/* ------------------------------------------------------------------------------ */
/* Copy-based insertion sort of ar[lo..hi] (Section IV).                            */
/* ------------------------------------------------------------------------------ */

static void insertion_sort(tctx *c, idx lo, idx hi) {
    for (idx k = lo + 1; k <= hi; k++) {
        if (ccmp(c, AR(c, k), AR(c, k - 1)) >= 0) continue;
        idx j = k;
        ccopy(c, c->temp, AR(c, j));
        ccopy(c, AR(c, j), AR(c, j - 1));
        if (--j > lo) {
            while (ccmp(c, c->temp, AR(c, j - 1)) < 0) {
                ccopy(c, AR(c, j), AR(c, j - 1));
                if (--j == lo) break;
            }
        }
        ccopy(c, AR(c, j), c->temp);
    }
}

/* ------------------------------------------------------------------------------ */
/* One Triple State stage (Section III.A-F).                                        */
/* ------------------------------------------------------------------------------ */

enum {
    S_L_SCAN1, S_R_SCAN1, S_MR_SCAN1, S_ML_SCAN1,         /* State 1           */
    S_MLEFT_CHECKM, S_MRIGHT_CHECKM, S_MLEFT, S_MRIGHT,   /* choice, III.C     */
    S_2L_M, S_2L_M2, S_2L_L,                              /* State 2L          */
    S_2R_M, S_2R_M2, S_2R_R,                              /* State 2R          */
    S_3L_M, S_3L_M2, S_3L_M3, S_3L_M4, S_3L_L,            /* State 3L          */
    S_3R_M, S_3R_M2, S_3R_M3, S_3R_M4, S_3R_R,            /* State 3R          */
    S_EXIT3L, S_EXIT3R, S_EXIT2, S_DONE
};

/* Partitions ar[a..b] (b - a + 1 >= 3) around a sampled pivot.  On return ar[a..*lo]
 * holds the elements < p (plus temp if temp < p), ar[*hi..b] the elements > p (plus
 * temp if temp > p), and every slot strictly between holds an element equal to p. */
static void ts_stage(tctx *c, idx a, idx b, idx *lo, idx *hi) {
    orc_stats *st = c->st;
    idx mid = a + (b - a) / 2;
    idx pi = c->forced_pi >= 0 ? c->forced_pi : choose_pivot(c, a, b, mid);
    /* III.A: p leaves the array and slot mid becomes empty. */
    ccopy(c, c->p, AR(c, pi));
    if (pi != mid) ccopy(c, AR(c, pi), AR(c, mid));   /* Reading: no self-copy when pi == mid */
    char *P = c->p;
    idx l = a, r = b, m = mid, ml = mid, mr = mid, i = 0, k = 0, k2 = 0;
    int lc = 0, state, in_state1 = 1;
    st->stages++;
    st->state_entries[ORC_ST_STATE1]++;

    /* Pre-scan from the right for the first ar[r] <= p; it goes to temp, opening the
     * second hole. */
    while (ccmp(c, AR(c, r), P) > 0) {
        r--;
        if (r == mid) break;
    }
    if (r == mid) {
        /* Reading of the special case "r reached mid": every element right of mid is
         * > p, so the right side is closed with the empty run [mid, mid-1].  The second
         * hole is opened at l = a by moving ar[a] into temp; this is exactly the
         * situation MLEFT expects (holes at l and r, equals in [ml, r-1]). */
        st->state_entries[ORC_ST_INIT_SPECIAL]++;
        ccopy(c, c->temp, AR(c, l));
        state = S_MLEFT;
    } else {
        ccopy(c, c->temp, AR(c, r));
        state = S_L_SCAN1;
    }

    for (;;) {
        switch (state) {
        /* ---------------- State 1 (III.B): four cursors l, r, ml, mr ---------------- */
        case S_L_SCAN1:                      /* second hole at r; scan l rightwards  */
            while ((lc = ccmp(c, AR(c, l), P)) < 0) {
                l++;
                if (l == ml) { state = S_MRIGHT_CHECKM; goto next; }
            }
            if (lc == 0) {                   /* an equal joins the run at its hole m */
                ccopy(c, AR(c, m), AR(c, l));
                if (r - mr > ml - l) { mr++; state = S_MR_SCAN1; }   /* larger gap */
                else { ml--; state = (ml == l) ? S_MRIGHT : S_ML_SCAN1; }
            } else {                         /* a larger element fills the hole at r */
                ccopy(c, AR(c, r), AR(c, l));
                r--;
                state = (mr == r) ? S_MLEFT_CHECKM : S_R_SCAN1;
            }
            break;

        case S_R_SCAN1:                      /* second hole at l; scan r leftwards   */
            while ((lc = ccmp(c, AR(c, r), P)) > 0) {
                r--;
                if (mr == r) { state = S_MLEFT_CHECKM; goto next; }
            }
            if (lc == 0) {
                ccopy(c, AR(c, m), AR(c, r));
                if (r - mr > ml - l) { mr++; state = S_MR_SCAN1; }
                else { ml--; state = (ml == l) ? S_MRIGHT : S_ML_SCAN1; }
            } else {                         /* a smaller element fills the hole at l */
                ccopy(c, AR(c, l), AR(c, r));
                l++;
                state = (ml == l) ? S_MRIGHT_CHECKM : S_L_SCAN1;
            }
            break;

        case S_MR_SCAN1:                     /* run is full, holes at l and r: grow it right */
            while ((lc = ccmp(c, AR(c, mr), P)) == 0) {
                mr++;
                if (mr == r) { state = S_MLEFT; goto next; }
            }
            if (lc < 0) {
                ccopy(c, AR(c, l), AR(c, mr));
                l++;
                if (ml == l) { ccopy(c, AR(c, mr), AR(c, ml)); state = S_MRIGHT; }
                else { m = mr; state = S_L_SCAN1; }
            } else {
                ccopy(c, AR(c, r), AR(c, mr));
                r--;
                if (mr == r) state = S_MLEFT;
                else { m = mr; state = S_R_SCAN1; }
            }
            break;

        case S_ML_SCAN1:                     /* run is full, holes at l and r: grow it left */
            while ((lc = ccmp(c, AR(c, ml), P)) == 0) {
                ml--;
                if (ml == l) { state = S_MRIGHT; goto next; }
            }
            if (lc < 0) {
                ccopy(c, AR(c, l), AR(c, ml));
                l++;
                if (l == ml) state = S_MRIGHT;
                else { m = ml; state = S_L_SCAN1; }
            } else {
                ccopy(c, AR(c, r), AR(c, ml));
                r--;
                if (mr == r) { ccopy(c, AR(c, ml), AR(c, mr)); state = S_MLEFT; }
                else { m = ml; state = S_R_SCAN1; }
            }
            break;

        /* ---------------- Choosing the next state (III.C) ---------------- */
        case S_MLEFT_CHECKM:
            /* Reading of MLEFT_CHECKM: r has reached mr while the run still has its
             * hole at m.  If that hole is not at mr, the equal at mr moves into it, so
             * that r becomes the hole MLEFT expects. */
            if (m != mr) ccopy(c, AR(c, m), AR(c, mr));
            state = S_MLEFT;
            break;

        case S_MRIGHT_CHECKM:                /* mirror image of MLEFT_CHECKM */
            if (m != ml) ccopy(c, AR(c, m), AR(c, ml));
            state = S_MRIGHT;
            break;

        case S_MLEFT:                        /* right side closed: mr == r            */
            do {
                ml--;
                if (ml == l) { state = S_EXIT2; goto next; }
            } while ((lc = ccmp(c, AR(c, ml), P)) == 0);
            m = ml; ml++;
            /* inequality (1): few equals -> State 3L, many -> State 2L */
            in_state1 = 0;
            if ((mr - ml) <= (ml - l) / 4) { st->state_entries[ORC_ST_3L]++; state = S_3L_M2; }
            else { st->state_entries[ORC_ST_2L]++; state = S_2L_M2; }
            break;

        case S_MRIGHT:                       /* left side closed: ml == l             */
            do {
                mr++;
                if (mr == r) { state = S_EXIT2; goto next; }
            } while ((lc = ccmp(c, AR(c, mr), P)) == 0);
            m = mr; mr--;
            /* inequality (2) */
            in_state1 = 0;
            if ((mr - ml) <= (r - mr) / 4) { st->state_entries[ORC_ST_3R]++; state = S_3R_M2; }
            else { st->state_entries[ORC_ST_2R]++; state = S_2R_M2; }
            break;

        /* ---------------- State 2L (III.D): roll the run of equals left ---------------- */
        case S_2L_M:                         /* holes at l and r; m scans left        */
            while ((lc = ccmp(c, AR(c, m), P)) == 0) {
                m--;
                if (m == l) { state = S_EXIT2; goto next; }
            }
            /* fall through */
        case S_2L_M2:
            if (lc < 0) {
                ccopy(c, AR(c, l), AR(c, m));
                l++;
                state = (m == l) ? S_EXIT2 : S_2L_L;     /* holes now at m and r */
            } else {                          /* roll: > p to r, last equal into m */
                ccopy(c, AR(c, r), AR(c, m));
                r--;
                ccopy(c, AR(c, m), AR(c, r));
                m--;
                state = (m == l) ? S_EXIT2 : S_2L_M;
            }
            break;

        case S_2L_L:                         /* holes at m and r; l scans right       */
            while ((lc = ccmp(c, AR(c, l), P)) < 0) {
                l++;
                if (m == l) { state = S_EXIT2; goto next; }
            }
            if (lc == 0) {
                ccopy(c, AR(c, m), AR(c, l));
                m--;
            } else {
                ccopy(c, AR(c, r), AR(c, l));
                r--;
                ccopy(c, AR(c, m), AR(c, r));
                m--;
            }
            state = (m == l) ? S_EXIT2 : S_2L_M;
            break;

        /* ---------------- State 2R: mirror image of 2L ---------------- */
        case S_2R_M:                         /* holes at l and r; m scans right       */
            while ((lc = ccmp(c, AR(c, m), P)) == 0) {
                m++;
                if (m == r) { state = S_EXIT2; goto next; }
            }
            /* fall through */
        case S_2R_M2:
            if (lc > 0) {
                ccopy(c, AR(c, r), AR(c, m));
                r--;
                state = (m == r) ? S_EXIT2 : S_2R_R;     /* holes now at l and m */
            } else {
                ccopy(c, AR(c, l), AR(c, m));
                l++;
                ccopy(c, AR(c, m), AR(c, l));
                m++;
                state = (m == r) ? S_EXIT2 : S_2R_M;
            }
            break;

        case S_2R_R:                         /* holes at l and m; r scans left        */
            while ((lc = ccmp(c, AR(c, r), P)) > 0) {
                r--;
                if (m == r) { state = S_EXIT2; goto next; }
            }
            if (lc == 0) {
                ccopy(c, AR(c, m), AR(c, r));
                m++;
            } else {
                ccopy(c, AR(c, l), AR(c, r));
                l++;
                ccopy(c, AR(c, m), AR(c, l));
                m++;
            }
            state = (m == r) ? S_EXIT2 : S_2R_M;
            break;

        /* ---------------- State 3L (III.E): equals go to tar ---------------- */
        case S_3L_M:                         /* hole at l (and r); m scans left       */
            while ((lc = ccmp(c, AR(c, m), P)) == 0) {
        case S_3L_M3:
                ccopy(c, TAR(c, i), AR(c, m)); i++;
                m--;
                if (m == l) { state = S_EXIT3L; goto next; }
            }
            /* fall through */
        case S_3L_M2:
            if (lc < 0) {
        case S_3L_M4:
                ccopy(c, AR(c, l), AR(c, m));
                l++;
                state = (m == l) ? S_EXIT3L : S_3L_L;    /* hole now at m */
                break;
            }
            /* a run of elements > p ends at k = m; find where it starts */
            k = m;
            do {
                m--;
                if (m == l) break;
            } while ((lc = ccmp(c, AR(c, m), P)) > 0);
            k2 = m + 1;
            /* copy the run into the gap (k, r]; every slot r passes that still holds an
             * equal of the old run [ml, ...) is first saved to tar */
            if (k - m < r - k) {             /* the whole run fits */
                do {
                    ccopy(c, AR(c, r), AR(c, k2));
                    r--;
                    if (r >= ml) { ccopy(c, TAR(c, i), AR(c, r)); i++; }
                } while (++k2 <= k);
            } else {                         /* the gap fills first; the rest stays put */
                for (;;) {
                    ccopy(c, AR(c, r), AR(c, k2));
                    r--;
                    if (r >= ml) { ccopy(c, TAR(c, i), AR(c, r)); i++; }
                    else if (r <= k) { r = k2; break; }
                    k2++;
                }
            }
            if (m == l) state = S_EXIT3L;
            else if (lc == 0) state = S_3L_M3;
            else state = S_3L_M4;
            break;

        case S_3L_L:                         /* hole at m (and r); l scans right      */
            while ((lc = ccmp(c, AR(c, l), P)) < 0) {
                l++;
                if (m == l) { state = S_EXIT3L; goto next; }
            }
            if (lc == 0) {
                ccopy(c, TAR(c, i), AR(c, l)); i++;
                m--;
            } else {
                ccopy(c, AR(c, r), AR(c, l));
                r--;
                if (r >= ml) { ccopy(c, TAR(c, i), AR(c, r)); i++; }
                m--;
            }
            state = (m == l) ? S_EXIT3L : S_3L_M;
            break;

        /* ---------------- State 3R: mirror image of 3L ---------------- */
        case S_3R_M:                         /* hole at r (and l); m scans right      */
            while ((lc = ccmp(c, AR(c, m), P)) == 0) {
        case S_3R_M3:
                ccopy(c, TAR(c, i), AR(c, m)); i++;
                m++;
                if (m == r) { state = S_EXIT3R; goto next; }
            }
            /* fall through */
        case S_3R_M2:
            if (lc > 0) {
        case S_3R_M4:
                ccopy(c, AR(c, r), AR(c, m));
                r--;
                state = (m == r) ? S_EXIT3R : S_3R_R;
                break;
            }
            k = m;                           /* a run of elements < p starts at k */
            do {
                m++;
                if (m == r) break;
            } while ((lc = ccmp(c, AR(c, m), P)) < 0);
            k2 = m - 1;
            if (m - k < k - l) {
                do {
                    ccopy(c, AR(c, l), AR(c, k2));
                    l++;
                    if (l <= mr) { ccopy(c, TAR(c, i), AR(c, l)); i++; }
                } while (--k2 >= k);
            } else {
                for (;;) {
                    ccopy(c, AR(c, l), AR(c, k2));
                    l++;
                    if (l <= mr) { ccopy(c, TAR(c, i), AR(c, l)); i++; }
                    else if (l >= k) { l = k2; break; }
                    k2--;
                }
            }
            if (m == r) state = S_EXIT3R;
            else if (lc == 0) state = S_3R_M3;
            else state = S_3R_M4;
            break;

        case S_3R_R:                         /* hole at m (and l); r scans left       */
            while ((lc = ccmp(c, AR(c, r), P)) > 0) {
                r--;
                if (m == r) { state = S_EXIT3R; goto next; }
            }
            if (lc == 0) {
                ccopy(c, TAR(c, i), AR(c, r)); i++;
                m++;
            } else {
                ccopy(c, AR(c, l), AR(c, r));
                l++;
                if (l <= mr) { ccopy(c, TAR(c, i), AR(c, l)); i++; }
                m++;
            }
            state = (m == r) ? S_EXIT3R : S_3R_M;
            break;

        /* ---------------- Copy back (III.F) ---------------- */
        case S_EXIT3L:                       /* tar holds only equals of p */
            if ((uint64_t)i > st->tar_peak) st->tar_peak = (uint64_t)i;
            while (i > 0) { i--; m++; ccopy(c, AR(c, m), TAR(c, i)); }
            state = S_EXIT2;
            break;

        case S_EXIT3R:
            if ((uint64_t)i > st->tar_peak) st->tar_peak = (uint64_t)i;
            while (i > 0) { i--; m--; ccopy(c, AR(c, m), TAR(c, i)); }
            state = S_EXIT2;
            break;

        case S_EXIT2:                        /* the two holes are at l and r */
            if (in_state1) st->state_entries[ORC_ST_EXIT_STATE1]++;
            if ((lc = ccmp(c, c->temp, P)) >= 0) {
                ccopy(c, AR(c, r), c->temp);
                ccopy(c, AR(c, l), P);
                l--;
                if (lc == 0) r++;
            } else {
                ccopy(c, AR(c, l), c->temp);
                ccopy(c, AR(c, r), P);
                r++;
            }
            state = S_DONE;
            break;

        default:
            break;
        }
        if (state == S_DONE) break;
    next:;
    }
    *lo = l;
    *hi = r;
}

/* Recursion driver (Fig. 1): stages on parts larger than the insertion threshold,
 * recursing into the smaller side and looping on the larger (Reading: the paper does
 * not state an order; this one bounds the stack by log2 n). */
static void ts_sort_range(tctx *c, idx a, idx b, uint64_t depth) {
    idx small = c->cfg.ins_threshold < 2 ? 2 : c->cfg.ins_threshold;
    for (;;) {
        if (depth > c->st->max_depth) c->st->max_depth = depth;
        if (b - a + 1 <= small) {
            if (b > a) { c->st->ins_parts++; insertion_sort(c, a, b); }
            return;
        }
        idx l, r;
        ts_stage(c, a, b, &l, &r);
        depth++;
        if (l - a < b - r) {
            ts_sort_range(c, a, l, depth);
            a = r;
        } else {
            ts_sort_range(c, r, b, depth);
            b = l;
        }
    }
}

static int ctx_init_cmp(tctx *c, void *base, size_t n, size_t ses, cmp_fn cmp,
                        const orc_cfg *cfg, orc_stats *st) {
    memset(c, 0, sizeof(*c));
    c->cmp = cmp;
    c->ses = ses;
    if (!c->cmp || !c->ses) return -1;
    if (cfg) c->cfg = *cfg; else orc_default_cfg(&c->cfg);
    c->ar = (char *)base;
    c->st = st;
    /* Section III.G: tar is allocated once per call.  Reading: n elements instead of
     * n/2, so no input can overflow it; tar_peak reports what was used. */
    c->tar = (char *)malloc((n ? n : 1) * c->ses);
    c->p = (char *)malloc(3 * c->ses);
    if (!c->tar || !c->p) { free(c->tar); free(c->p); return -1; }
    c->temp = c->p + c->ses;
    c->scratch = c->p + 2 * c->ses;
    c->forced_pi = -1;
    c->zgen = pm_seed(c->cfg.seed);
    /* Section V.C: one draw per sort call, dran in [0.5, 1.5) */
    c->dran = 0.5 + (double)pm_next(&c->zgen) / (double)PM_M;
    return 0;
}

static int ctx_init(tctx *c, void *base, size_t n, int key_kind, const orc_cfg *cfg,
                    orc_stats *st) {
    size_t ses;
    cmp_fn f = pick_cmp(key_kind, &ses);
    return ctx_init_cmp(c, base, n, ses, f, cfg, st);
}

static void ctx_free(tctx *c) { free(c->tar); free(c->p); }

int orc_tsqs_sort(void *base, size_t n, int key_kind, const orc_cfg *cfg, orc_stats *st) {
    orc_stats local;
    if (!st) { memset(&local, 0, sizeof(local)); st = &local; }
    tctx c;
    if (ctx_init(&c, base, n, key_kind, cfg, st)) return -1;
    if (n > 1) ts_sort_range(&c, 0, (idx)n - 1, 0);
    ctx_free(&c);
    return 0;
}

int orc_tsqs_sort_rows(void *base, size_t nrows, size_t n, int key_kind,
                       const orc_cfg *cfg, orc_stats *st) {
    orc_stats local;
    if (!st) { memset(&local, 0, sizeof(local)); st = &local; }
    tctx c;
    if (ctx_init(&c, base, n, key_kind, cfg, st)) return -1;
    for (size_t row = 0; row < nrows; row++) {
        c.ar = (char *)base + row * n * c.ses;
        if (n > 1) ts_sort_range(&c, 0, (idx)n - 1, 0);
    }
    ctx_free(&c);
    return 0;
}

typedef struct {
    char *base; const uint64_t *offs; size_t nseg; int kind;
    size_t next; pthread_mutex_t mu; int err;
} seg_job;

static void *seg_worker(void *arg) {
    seg_job *j = (seg_job *)arg;
    size_t ses = orc_elem_size(j->kind);
    for (;;) {
        pthread_mutex_lock(&j->mu);
        size_t s = j->next++;
        pthread_mutex_unlock(&j->mu);
        if (s >= j->nseg) break;
        uint64_t lo = j->offs[s], hi = j->offs[s + 1];
        if (hi > lo && orc_tsqs_sort(j->base + lo * ses, (size_t)(hi - lo), j->kind, NULL, NULL))
            j->err = -1;
    }
    return NULL;
}

int orc_tsqs_sort_segments(void *base, const uint64_t *offs, size_t nseg, int key_kind,
                           int threads) {
    if (!orc_elem_size(key_kind)) return -1;
    seg_job j = { (char *)base, offs, nseg, key_kind, 0, PTHREAD_MUTEX_INITIALIZER, 0 };
    if (threads < 1) threads = 1;
    if (threads == 1) { seg_worker(&j); return j.err; }
    pthread_t *t = (pthread_t *)malloc(sizeof(pthread_t) * (size_t)threads);
    if (!t) return -1;
    int started = 0;
    for (int k = 0; k < threads; k++)
        if (pthread_create(&t[k], NULL, seg_worker, &j) == 0) started++;
        else break;
    if (started == 0) seg_worker(&j);
    for (int k = 0; k < started; k++) pthread_join(t[k], NULL);
    free(t);
    return j.err;
}

/* ------------------------------------------------------------------------------ */
/* Large elements: late swapping (Section VIII.H).  The array of element pointers is */
/* sorted by Triple State QuickSort (the pointed-to keys decide; equal keys keep     */
/* their original order, because the pointers themselves break the tie), then the    */
/* elements are moved into place by following the cycles of the permutation, each   */
/* cycle through one temporary element.                                              */
/* ------------------------------------------------------------------------------ */

static _Thread_local size_t g_wide_off;
static _Thread_local cmp_fn g_wide_key;

static int cmp_wide_ptr(const void *x, const void *y) {
    const char *px = *(const char *const *)x, *py = *(const char *const *)y;
    const int r = g_wide_key(px + g_wide_off, py + g_wide_off);
    if (r) return r;
    return px < py ? -1 : (px > py ? 1 : 0);
}

int orc_wide_sort(void *base, size_t n, size_t es, size_t key_off, int key_kind,
                  uint64_t *moves_out, uint64_t *cycles_out) {
    size_t ks;
    cmp_fn key = pick_cmp(key_kind, &ks);
    if (!key || key_kind == ORC_REC || key_off + ks > es) return -1;
    if (moves_out) *moves_out = 0;
    if (cycles_out) *cycles_out = 0;
    if (n < 2) return 0;
    char *b = (char *)base;
    char **ptr = (char **)malloc(n * sizeof(char *));
    unsigned char *placed = (unsigned char *)calloc(n, 1);
    char *tmp = (char *)malloc(es);
    if (!ptr || !placed || !tmp) { free(ptr); free(placed); free(tmp); return -1; }
    for (size_t i = 0; i < n; i++) ptr[i] = b + i * es;
    g_wide_off = key_off;
    g_wide_key = key;
    orc_stats st;
    memset(&st, 0, sizeof(st));
    tctx c;
    if (ctx_init_cmp(&c, ptr, n, sizeof(char *), cmp_wide_ptr, NULL, &st)) {
        free(ptr); free(placed); free(tmp); return -1;
    }
    ts_sort_range(&c, 0, (idx)n - 1, 0);
    ctx_free(&c);
    /* ptr[j] is the original place of the element that belongs at j */
    uint64_t moves = 0, cycles = 0;
    for (size_t i = 0; i < n; i++) {
        if (placed[i]) continue;
        placed[i] = 1;
        if (ptr[i] == b + i * es) continue;             /* already in place */
        cycles++;
        memcpy(tmp, b + i * es, es);
        moves++;
        size_t j = i;
        for (;;) {
            const size_t src = (size_t)(ptr[j] - b) / es;
            if (src == i) { memcpy(b + j * es, tmp, es); moves++; break; }
            memcpy(b + j * es, b + src * es, es);
            moves++;
            placed[src] = 1;
            j = src;
        }
    }
    if (moves_out) *moves_out = moves;
    if (cycles_out) *cycles_out = cycles;
    free(ptr); free(placed); free(tmp);
    return 0;
}

/* ------------------------------------------------------------------------------ */
/* Baselines with a uniformly random pivot.                                         */
/* ------------------------------------------------------------------------------ */

/* Textbook Hoare partitioning (the setting of eqs. (3) and (4)): the pivot is swapped
 * to a, i runs right over elements < p, j runs left over elements > p, the misplaced
 * pair is exchanged.  Each non-pivot element is compared with p exactly once, so a
 * stage of n elements makes n - 1 comparisons.  Only the exchanges of misplaced pairs
 * are counted as swaps (the convention under which (n-2)/6 exchanges per stage give
 * eq. (4)). */
static void classical_range(tctx *c, idx a, idx b) {
    while (b > a) {
        idx pi = a + pm_index(&c->zgen, b - a + 1);
        if (pi != a) {                                     /* move pivot out of the way */
            memcpy(c->scratch, AR(c, a), c->ses);
            memcpy(AR(c, a), AR(c, pi), c->ses);
            memcpy(AR(c, pi), c->scratch, c->ses);
        }
        memcpy(c->p, AR(c, a), c->ses);
        idx i = a + 1, j = b;
        for (;;) {
            while (i <= j && ccmp(c, AR(c, i), c->p) < 0) i++;
            if (i > j) break;                              /* ar[i] >= p is classified */
            while (j > i && ccmp(c, AR(c, j), c->p) > 0) j--;
            if (j == i) break;
            memcpy(c->scratch, AR(c, i), c->ses);          /* exchange the misplaced pair */
            memcpy(AR(c, i), AR(c, j), c->ses);
            memcpy(AR(c, j), c->scratch, c->ses);
            c->st->swaps++;
            i++; j--;
        }
        /* ar[a+1..i-1] <= p, ar[i..b] >= p: the pivot goes to i-1 */
        if (i - 1 != a) {
            memcpy(AR(c, a), AR(c, i - 1), c->ses);
            memcpy(AR(c, i - 1), c->p, c->ses);
        }
        c->st->stages++;
        idx lo_n = i - 1 - a, hi_n = b - i + 1;
        if (lo_n < hi_n) { classical_range(c, a, i - 2); a = i; }
        else { classical_range(c, i, b); b = i - 2; }
    }
}

int orc_classical_sort(void *base, size_t n, int key_kind, uint64_t seed, orc_stats *st) {
    orc_stats local;
    if (!st) { memset(&local, 0, sizeof(local)); st = &local; }
    orc_cfg cfg; orc_default_cfg(&cfg); cfg.seed = seed;
    tctx c;
    if (ctx_init(&c, base, n, key_kind, &cfg, st)) return -1;
    if (n > 1) classical_range(&c, 0, (idx)n - 1);
    ctx_free(&c);
    return 0;
}

/* Section II: the first ar[r] <= p goes to temp, leaving an empty slot that juggles
 * between l and r as misplaced elements are copied into it; temp returns at the end.
 * The pivot element leaves the array first (p), the stage excludes the pivot and temp
 * as the paper's exit does, and recursion covers [a, l] and [r, b]. */
static void juggle_range(tctx *c, idx a, idx b) {
    while (b - a + 1 >= 2) {
        idx pi = a + pm_index(&c->zgen, b - a + 1);
        /* The pivot is swapped to b and excluded from the scan (not counted as moves:
         * the eq. (8) model charges only the hole copies and the temp round trip). */
        if (pi != b) {
            memcpy(c->scratch, AR(c, b), c->ses);
            memcpy(AR(c, b), AR(c, pi), c->ses);
            memcpy(AR(c, pi), c->scratch, c->ses);
        }
        memcpy(c->p, AR(c, b), c->ses);
        idx l = a, r = b - 1;
        c->st->stages++;
        /* pre-scan from the right */
        while (r >= l && ccmp(c, AR(c, r), c->p) > 0) r--;
        if (r < l) {                                      /* every element > p */
            /* pivot is the minimum: put it at a, recurse on (a, b] */
            memcpy(c->scratch, AR(c, a), c->ses);
            memcpy(AR(c, a), c->p, c->ses);
            memcpy(AR(c, b), c->scratch, c->ses);
            a = a + 1;
            continue;
        }
        ccopy(c, c->temp, AR(c, r));                      /* the empty slot is at r */
        /* main loop: hole alternates; invariant ar[a..l) <= p, ar(r..b-1] >= p */
        for (;;) {
            while (l < r && ccmp(c, AR(c, l), c->p) <= 0) l++;
            if (l >= r) break;
            ccopy(c, AR(c, r), AR(c, l)); r--;            /* hole moves to l */
            while (l < r && ccmp(c, AR(c, r), c->p) >= 0) r--;
            if (l >= r) { r = l; break; }                 /* hole at l == r */
            ccopy(c, AR(c, l), AR(c, r)); l++;            /* hole moves to r */
        }
        /* the hole is at r (== l): temp (<= p) goes back into it */
        ccopy(c, AR(c, r), c->temp);
        /* ar[a..r] <= p, ar[r+1..b-1] >= p: swap the pivot to r+1 */
        idx q = r + 1;
        if (q != b) {
            memcpy(AR(c, b), AR(c, q), c->ses);
            memcpy(AR(c, q), c->p, c->ses);
        }
        if (q - a < b - q) { juggle_range(c, a, q - 1); a = q + 1; }
        else { juggle_range(c, q + 1, b); b = q - 1; }
    }
}

int orc_juggle_sort(void *base, size_t n, int key_kind, uint64_t seed, orc_stats *st) {
    orc_stats local;
    if (!st) { memset(&local, 0, sizeof(local)); st = &local; }
    orc_cfg cfg; orc_default_cfg(&cfg); cfg.seed = seed;
    tctx c;
    if (ctx_init(&c, base, n, key_kind, &cfg, st)) return -1;
    if (n > 1) juggle_range(&c, 0, (idx)n - 1);
    ctx_free(&c);
    return 0;
}

/* One stage only, with the pivot at index pi (n >= 3).  Returns the bounds of the
 * two parts through lo (last index of the left part) and hi (first of the right). */
int orc_tsqs_stage(void *base, size_t n, int key_kind, size_t pi, orc_stats *st,
                   long long *lo, long long *hi) {
    orc_stats local;
    if (!st) { memset(&local, 0, sizeof(local)); st = &local; }
    if (n < 3 || pi >= n) return -1;
    tctx c;
    if (ctx_init(&c, base, n, key_kind, NULL, st)) return -1;
    c.forced_pi = (idx)pi;
    idx l, r;
    ts_stage(&c, 0, (idx)n - 1, &l, &r);
    ctx_free(&c);
    if (lo) *lo = l;
    if (hi) *hi = r;
    return 0;
}

/* Pivot selection alone on base[0..n): the tier choice of Section III.H for a part
 * [0, n-1] with mid = (n-1)/2, under cfg (NULL = defaults).  The samples are sorted in
 * place as in a stage; returns the pivot index, or -1 on bad arguments. */
long long orc_choose_pivot(void *base, size_t n, int key_kind, const orc_cfg *cfg,
                           orc_stats *st) {
    orc_stats local;
    if (!st) { memset(&local, 0, sizeof(local)); st = &local; }
    if (n < 3) return -1;
    tctx c;
    if (ctx_init(&c, base, n, key_kind, cfg, st)) return -1;
    idx b = (idx)n - 1, mid = b / 2;
    idx pi = choose_pivot(&c, 0, b, mid);
    ctx_free(&c);
    return (long long)pi;
}

/* One textbook Hoare stage with the pivot at index pi; counts cmps and exchanges. */
int orc_hoare_stage(void *base, size_t n, int key_kind, size_t pi, orc_stats *st) {
    orc_stats local;
    if (!st) { memset(&local, 0, sizeof(local)); st = &local; }
    if (n < 2 || pi >= n) return -1;
    tctx c;
    if (ctx_init(&c, base, n, key_kind, NULL, st)) return -1;
    idx a = 0, b = (idx)n - 1;
    if ((idx)pi != a) {
        memcpy(c.scratch, AR(&c, a), c.ses);
        memcpy(AR(&c, a), AR(&c, pi), c.ses);
        memcpy(AR(&c, pi), c.scratch, c.ses);
    }
    memcpy(c.p, AR(&c, a), c.ses);
    idx i = a + 1, j = b;
    for (;;) {
        while (i <= j && ccmp(&c, AR(&c, i), c.p) < 0) i++;
        if (i > j) break;
        while (j > i && ccmp(&c, AR(&c, j), c.p) > 0) j--;
        if (j == i) break;
        memcpy(c.scratch, AR(&c, i), c.ses);
        memcpy(AR(&c, i), AR(&c, j), c.ses);
        memcpy(AR(&c, j), c.scratch, c.ses);
        st->swaps++;
        i++; j--;
    }
    ctx_free(&c);
    return 0;
}

/* ------------------------------------------------------------------------------ */
/* Plain definitions used as per-step references.                                   */
/* ------------------------------------------------------------------------------ */

int orc_median3(void *base, size_t i0, size_t i1, size_t i2, int key_kind, orc_stats *st) {
    orc_stats local;
    if (!st) { memset(&local, 0, sizeof(local)); st = &local; }
    tctx c;
    if (ctx_init(&c, base, 3, key_kind, NULL, st)) return -2;
    int o = med3(&c, (idx)i0, (idx)i1, (idx)i2);
    ctx_free(&c);
    return o;
}

int orc_lower_median(const void *keys, size_t s, int key_kind, void *out) {
    size_t ses = orc_elem_size(key_kind);
    if (!ses || s == 0) return -1;
    char *tmp = (char *)malloc(s * ses);
    if (!tmp) return -1;
    memcpy(tmp, keys, s * ses);
    /* insertion sort of the copy: s is a sample size, and this keeps the routine
     * free of global state */
    for (size_t k = 1; k < s; k++) {
        for (size_t j = k; j > 0 && orc_compare(tmp + j * ses, tmp + (j - 1) * ses, key_kind) < 0; j--) {
            char t[16];
            memcpy(t, tmp + j * ses, ses);
            memcpy(tmp + j * ses, tmp + (j - 1) * ses, ses);
            memcpy(tmp + (j - 1) * ses, t, ses);
        }
    }
    memcpy(out, tmp + ((s - 1) / 2) * ses, ses);
    free(tmp);
    return 0;
}

int orc_three_way_split(const void *in, void *out, size_t n, int key_kind,
                        const void *pivot, size_t *nlt, size_t *neq, size_t *ngt) {
    size_t ses = orc_elem_size(key_kind);
    if (!ses) return -1;
    const char *src = (const char *)in;
    char *dst = (char *)out;
    size_t lt = 0, eq = 0, gt = 0;
    for (size_t j = 0; j < n; j++) {
        int c = orc_compare(src + j * ses, pivot, key_kind);
        if (c < 0) lt++; else if (c == 0) eq++; else gt++;
    }
    size_t wl = 0, we = lt, wg = lt + eq;
    for (size_t j = 0; j < n; j++) {
        int c = orc_compare(src + j * ses, pivot, key_kind);
        char *d = c < 0 ? dst + (wl++) * ses : c == 0 ? dst + (we++) * ses : dst + (wg++) * ses;
        memcpy(d, src + j * ses, ses);
    }
    if (nlt) *nlt = lt;
    if (neq) *neq = eq;
    if (ngt) *ngt = gt;
    return 0;
}

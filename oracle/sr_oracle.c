/*
 * sr_oracle.c -- the CPU oracle for the sort (TEST INFRASTRUCTURE ONLY).
 *
 * Only tests/, the smoke check in __graft_entry__.py and the CPU-baseline leg
 * of bench.py may load this library.  The GPU library never links, includes or
 * calls it, and it shares no code with the GPU path.
 *
 * Everything here is plain single-threaded C with the paper's generic interface
 * (Section 5: every method takes the array, its length, the item size and a
 * comparison function, like the C library's qsort), so every comparison goes
 * through one counted comparator call.
 *
 *   sro_isort        plain insertion sort: the brute-force definition of sorting.
 *   sro_mergesort    natural mergesort with the techniques of the paper's "mer6"
 *                    (Section 3: (a) reversed runs, (b) short runs grown by
 *                    insertion sort, (f) trimming, (g) galloping, (e2) the
 *                    half-down run list).  Stable.  The primary oracle.  The
 *                    "merge5" algorithm is the same without (b) (the paper's
 *                    mer5).
 *   sro_quicksort    the paper's hybrid quicksort "hyb2" (Section 4, techniques
 *                    (a)-(g), alpha = beta = 32, gamma = 2).
 *   sro_runs         Run(A): descents + 1 (Section 2).
 *   sro_mono         Mono(A): fewest monotone pieces (Section 2), greedy.
 *   sro_inversions   Inv(A) by the O(n^2) definition (Section 2).
 *   sro_rem          Rem(A): fewest items whose removal leaves a sorted list
 *                    (the measure Section 2 relates to k-exchange lists).
 *
 * The two sorts are written from the techniques as Section 3 and Section 4
 * state them, not from the listings of the appendices.
 *
 * Readings of places where the paper is garbled or silent:
 *   R3  Techniques (a) and (b) together: the input is cut into maximal runs,
 *       each either non-decreasing or non-increasing (the latter reversed,
 *       its blocks of equal items reversed first so they keep their order);
 *       a run shorter than minrun is then grown to minrun items by insertion
 *       sort.  Every run so made goes on the half-down list.
 *   R4  The 2-way split (technique (e)) is Hoare's: one scan advances past
 *       items < v, the other retreats past items > v, the stopped pair is
 *       exchanged; the equal items the scans stop on are counted for (g).
 *   R5  Technique (f): the B-suffix that is >= the last element of A is
 *       left in place (">=" trims more than ">" and gives the same result).
 *   R6  An ascending run is non-decreasing (Run(A) counts strict descents only).
 *   R7  float32 keys follow IEEE-754 totalOrder on the bit patterns
 *       (-0.0 < +0.0; bit-different equal values are distinct).
 *   R9  The pseudo-median of nine takes positions low + k*floor((n-1)/8),
 *       k = 0..8, so the ninth sample stays inside the range (the printed
 *       "every n/8th position" would read one past the end when 8 | n).
 *   R10 Galloping (g) starts after GALLOP_AFTER = 3 consecutive wins of one
 *       side, the count used by the worked example of Section 3; it then
 *       moves the winning side's whole block, found by probing 1, 3, 7, ...
 *       items ahead and finishing with a binary search.
 *   R11 minrun is not stated; MINRUN is the value whose comparison count on
 *       random integers comes closest to Table 4's 22.15 per item for mer6
 *       at n = 2,000,000: 14 gives 22.11 (8 gives 21.53, 16 gives 22.25).
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* ------------------------------------------------------------------ keys */

enum { SRO_I32 = 0, SRO_U32 = 1, SRO_F32 = 2, SRO_U64 = 3, SRO_I64 = 4 };

typedef int (*sro_cmp)(const void *, const void *);

static uint64_t g_cmp_count;

static int cmp_i32(const void *a, const void *b) {
    int32_t x, y;
    memcpy(&x, a, 4); memcpy(&y, b, 4);
    g_cmp_count++;
    return (x > y) - (x < y);
}
static int cmp_u32(const void *a, const void *b) {
    uint32_t x, y;
    memcpy(&x, a, 4); memcpy(&y, b, 4);
    g_cmp_count++;
    return (x > y) - (x < y);
}
/* IEEE-754 totalOrder on float32 bit patterns (reading R7): a set sign bit
 * orders below a clear one; among non-negative patterns a larger magnitude is
 * larger; among negative patterns a larger magnitude is smaller. */
static int cmp_f32(const void *a, const void *b) {
    uint32_t x, y;
    memcpy(&x, a, 4); memcpy(&y, b, 4);
    g_cmp_count++;
    uint32_t sx = x >> 31, sy = y >> 31;
    if (sx != sy) return sx ? -1 : 1;
    uint32_t mx = x & 0x7fffffffu, my = y & 0x7fffffffu;
    if (mx == my) return 0;
    if (sx == 0) return mx > my ? 1 : -1;
    return mx > my ? -1 : 1;
}
static int cmp_u64(const void *a, const void *b) {
    uint64_t x, y;
    memcpy(&x, a, 8); memcpy(&y, b, 8);
    g_cmp_count++;
    return (x > y) - (x < y);
}
static int cmp_i64(const void *a, const void *b) {
    int64_t x, y;
    memcpy(&x, a, 8); memcpy(&y, b, 8);
    g_cmp_count++;
    return (x > y) - (x < y);
}

static sro_cmp cmp_for(int kt) {
    switch (kt) {
    case SRO_I32: return cmp_i32;
    case SRO_U32: return cmp_u32;
    case SRO_F32: return cmp_f32;
    case SRO_U64: return cmp_u64;
    case SRO_I64: return cmp_i64;
    default: return 0;
    }
}
static size_t key_size(int kt) { return (kt == SRO_U64 || kt == SRO_I64) ? 8 : 4; }

uint64_t sro_cmp_count(void) { return g_cmp_count; }
void sro_cmp_reset(void) { g_cmp_count = 0; }

/* --------------------------------------------------------- merge tracing */
/* An optional log of what merge() did, so a test can replay the worked example
 * of Section 3 (which prefix was trimmed, which side was copied to the
 * temporary buffer, and how many items each gallop moved). */
enum { TR_TRIM_A = 1, TR_TRIM_B = 2, TR_COPY_A = 3, TR_COPY_B = 4,
       TR_GALLOP_A = 5, TR_GALLOP_B = 6 };
static int g_trace_on;
static int64_t g_trace[256];
static int g_trace_len;

static void trace(int ev, size_t count) {
    if (!g_trace_on || g_trace_len + 2 > 256) return;
    g_trace[g_trace_len++] = ev;
    g_trace[g_trace_len++] = (int64_t)count;
}
void sro_trace_enable(int on) { g_trace_on = on; g_trace_len = 0; }
int sro_trace_read(int64_t *out, int cap) {
    int k = g_trace_len < cap ? g_trace_len : cap;
    memcpy(out, g_trace, (size_t)k * sizeof(int64_t));
    return k;
}

/* ------------------------------------------------------------- helpers */

#define AT(base, i, es) ((char *)(base) + (size_t)(i) * (es))

static void swap_items(void *base, size_t i, size_t j, size_t es) {
    char tmp[64];
    char *p = AT(base, i, es), *q = AT(base, j, es);
    memcpy(tmp, p, es); memcpy(p, q, es); memcpy(q, tmp, es);
}

/* reverse base[lo..hi] (inclusive), as the appendix's reverse(). */
static void reverse_items(void *base, size_t lo, size_t hi, size_t es) {
    while (lo < hi) { swap_items(base, lo, hi, es); lo++; hi--; }
}

/* insertion sort of base[lo, hi) given that base[lo, mid) is already sorted
 * (technique (b)); stable: an item moves left only past strictly larger ones. */
static void isort_range(void *base, size_t lo, size_t mid, size_t hi, size_t es, sro_cmp cmp) {
    char x[64];
    if (mid <= lo) mid = lo + 1;
    for (size_t k = mid; k < hi; k++) {
        memcpy(x, AT(base, k, es), es);
        size_t j = k;
        while (j > lo && cmp(AT(base, j - 1, es), x) > 0) {
            memcpy(AT(base, j, es), AT(base, j - 1, es), es);
            j--;
        }
        memcpy(AT(base, j, es), x, es);
    }
}

/* first index in [lo, hi) whose item is > key (items sorted). */
static size_t upper_bound(const void *base, size_t lo, size_t hi, const void *key, size_t es, sro_cmp cmp) {
    while (lo < hi) {
        size_t mid = lo + (hi - lo) / 2;
        if (cmp(AT(base, mid, es), key) <= 0) lo = mid + 1; else hi = mid;
    }
    return lo;
}
/* first index in [lo, hi) whose item is >= key (items sorted). */
static size_t lower_bound(const void *base, size_t lo, size_t hi, const void *key, size_t es, sro_cmp cmp) {
    while (lo < hi) {
        size_t mid = lo + (hi - lo) / 2;
        if (cmp(AT(base, mid, es), key) < 0) lo = mid + 1; else hi = mid;
    }
    return lo;
}

/* Galloping search (technique (g)): the end of the prefix of the sorted range
 * [lo, hi) whose items are < key (strict) or <= key (not strict).  gallop_fwd
 * probes lo, lo+1, lo+3, lo+7, ... and gallop_rev probes hi-1, hi-2, hi-4, ...,
 * then a binary search finishes between the last two probes, so the cost grows
 * with the log of the distance moved, not of the range. */
static int in_prefix(const void *base, size_t p, const void *key, int strict, size_t es, sro_cmp cmp) {
    int c = cmp(AT(base, p, es), key);
    return strict ? c < 0 : c <= 0;
}
static size_t finish_search(const void *base, size_t a, size_t b, const void *key, int strict, size_t es, sro_cmp cmp) {
    while (a < b) {
        size_t mid = a + (b - a) / 2;
        if (in_prefix(base, mid, key, strict, es, cmp)) a = mid + 1; else b = mid;
    }
    return a;
}
static size_t gallop_fwd(const void *base, size_t lo, size_t hi, const void *key, int strict, size_t es, sro_cmp cmp) {
    if (lo >= hi || !in_prefix(base, lo, key, strict, es, cmp)) return lo;
    size_t good = lo, ofs = 1;
    while (lo + ofs < hi && in_prefix(base, lo + ofs, key, strict, es, cmp)) { good = lo + ofs; ofs = 2 * ofs + 1; }
    size_t bad = lo + ofs < hi ? lo + ofs : hi;
    return finish_search(base, good + 1, bad, key, strict, es, cmp);
}
static size_t gallop_rev(const void *base, size_t lo, size_t hi, const void *key, int strict, size_t es, sro_cmp cmp) {
    if (lo >= hi || in_prefix(base, hi - 1, key, strict, es, cmp)) return hi;
    size_t bad = hi - 1, ofs = 1, a = lo;
    while (ofs <= hi - 1 - lo) {
        size_t p = hi - 1 - ofs;
        if (in_prefix(base, p, key, strict, es, cmp)) { a = p + 1; break; }
        bad = p; ofs = 2 * ofs + 1;
    }
    return finish_search(base, a, bad, key, strict, es, cmp);
}

/* ---------------------------------------------------------------- merge */

#define GALLOP_AFTER 3   /* reading R10 */

/* Merge the sorted runs A = base[lo, mid) and B = base[mid, hi) into
 * base[lo, hi), stably (an A item precedes an equal B item).
 * Technique (f): the A-prefix that is <= B's first item and the B-suffix that
 * is >= A's last item are already in place; only the shorter of what remains
 * of A or B is copied to the temporary buffer.  Technique (g): after
 * GALLOP_AFTER wins in a row, a binary search moves the winner's whole block. */
static void merge_runs(void *base, size_t lo, size_t mid, size_t hi, size_t es, sro_cmp cmp, char *tmp) {
    if (lo >= mid || mid >= hi) return;
    size_t lo2 = upper_bound(base, lo, mid, AT(base, mid, es), es, cmp);
    trace(TR_TRIM_A, lo2 - lo);
    lo = lo2;
    if (lo == mid) return;                       /* A.last <= B.first: in order */
    size_t hi2 = lower_bound(base, mid, hi, AT(base, mid - 1, es), es, cmp);
    trace(TR_TRIM_B, hi - hi2);
    hi = hi2;
    size_t na = mid - lo, nb = hi - mid;

    if (na <= nb) {
        /* copy A to tmp, merge forwards; B stays in place. */
        trace(TR_COPY_A, na);
        memcpy(tmp, AT(base, lo, es), na * es);
        size_t i = 0, j = mid, k = lo;
        int wins_a = 0, wins_b = 0;
        while (i < na && j < hi) {
            if (wins_b >= GALLOP_AFTER) {
                /* move every B item < A[i]; then A[i] is next without a compare */
                size_t e = gallop_fwd(base, j, hi, tmp + i * es, 1, es, cmp);
                trace(TR_GALLOP_B, e - j);
                memmove(AT(base, k, es), AT(base, j, es), (e - j) * es);
                k += e - j; j = e;
                memcpy(AT(base, k, es), tmp + i * es, es); k++; i++;
                wins_b = 0; wins_a = 1;
            } else if (wins_a >= GALLOP_AFTER) {
                /* move every A item <= B[j]; then B[j] is next */
                size_t e = gallop_fwd(tmp, i, na, AT(base, j, es), 0, es, cmp);
                trace(TR_GALLOP_A, e - i);
                memcpy(AT(base, k, es), tmp + i * es, (e - i) * es);
                k += e - i; i = e;
                if (i < na) { memcpy(AT(base, k, es), AT(base, j, es), es); k++; j++; }
                wins_a = 0; wins_b = 1;
            } else if (cmp(AT(base, j, es), tmp + i * es) < 0) {
                memcpy(AT(base, k, es), AT(base, j, es), es); k++; j++;
                wins_b++; wins_a = 0;
            } else {
                memcpy(AT(base, k, es), tmp + i * es, es); k++; i++;
                wins_a++; wins_b = 0;
            }
        }
        if (i < na) memcpy(AT(base, k, es), tmp + i * es, (na - i) * es);
    } else {
        /* copy B to tmp, merge backwards; A stays in place. */
        trace(TR_COPY_B, nb);
        memcpy(tmp, AT(base, mid, es), nb * es);
        size_t i = mid, j = nb, k = hi;    /* one past the next item of each */
        int wins_a = 0, wins_b = 0;
        while (i > lo && j > 0) {
            if (wins_a >= GALLOP_AFTER) {
                /* move every A item > B[j-1] to the back; then B[j-1] is next */
                size_t e = gallop_rev(base, lo, i, tmp + (j - 1) * es, 0, es, cmp);
                trace(TR_GALLOP_A, i - e);
                memmove(AT(base, k - (i - e), es), AT(base, e, es), (i - e) * es);
                k -= i - e; i = e;
                memcpy(AT(base, k - 1, es), tmp + (j - 1) * es, es); k--; j--;
                wins_a = 0; wins_b = 1;
            } else if (wins_b >= GALLOP_AFTER) {
                /* move every B item >= A[i-1] to the back; then A[i-1] is next */
                size_t e = gallop_rev(tmp, 0, j, AT(base, i - 1, es), 1, es, cmp);
                trace(TR_GALLOP_B, j - e);
                memcpy(AT(base, k - (j - e), es), tmp + e * es, (j - e) * es);
                k -= j - e; j = e;
                if (j > 0) { memcpy(AT(base, k - 1, es), AT(base, i - 1, es), es); k--; i--; }
                wins_b = 0; wins_a = 1;
            } else if (cmp(AT(base, i - 1, es), tmp + (j - 1) * es) > 0) {
                memcpy(AT(base, k - 1, es), AT(base, i - 1, es), es); k--; i--;
                wins_a++; wins_b = 0;
            } else {
                memcpy(AT(base, k - 1, es), tmp + (j - 1) * es, es); k--; j--;
                wins_b++; wins_a = 0;
            }
        }
        if (j > 0) memcpy(AT(base, lo, es), tmp, j * es);
    }
}

/* ------------------------------------------------------------ mergesort */

#define MINRUN 14    /* reading R11 */

/* What a sort routine works on: the array, its item size, the comparison and
 * a temporary buffer of n items for the merges. */
typedef struct {
    char *base;
    size_t n, es;
    sro_cmp cmp;
    char *tmp;
} sorter;

/* Technique (a): the end of the run that starts at lo, turned ascending.  A
 * run that opens with a rise (or an equal pair) is the longest non-decreasing
 * stretch; one that opens with a strict fall is the longest non-increasing
 * stretch, which is reversed in place -- after every block of equal items in
 * it has been reversed on its own, so that equal items end up in their input
 * order again (stability). */
static size_t take_run(sorter *so, size_t lo) {
    size_t hi = lo + 1;
    if (hi >= so->n) return so->n;
    if (so->cmp(AT(so->base, lo, so->es), AT(so->base, hi, so->es)) <= 0) {
        while (hi + 1 < so->n && so->cmp(AT(so->base, hi, so->es), AT(so->base, hi + 1, so->es)) <= 0) hi++;
        return hi + 1;
    }
    size_t eq_from = hi;                 /* first item of the current block of equal items */
    for (;;) {
        int c = hi + 1 < so->n ? so->cmp(AT(so->base, hi, so->es), AT(so->base, hi + 1, so->es)) : -1;
        if (c != 0 && hi > eq_from) reverse_items(so->base, eq_from, hi, so->es);
        if (c < 0) break;                /* a rise (or the end): the run stops at hi */
        hi++;
        if (c > 0) eq_from = hi;
    }
    reverse_items(so->base, lo, hi, so->es);
    return hi + 1;
}

/* Technique (b): a run [lo, end) shorter than `minrun` grows to minrun items
 * (or to the end of the array) by insertion sort. */
static size_t grow_run(sorter *so, size_t lo, size_t end, size_t minrun) {
    if (end - lo >= minrun || end >= so->n) return end;
    size_t want = so->n - lo < minrun ? so->n : lo + minrun;
    isort_range(so->base, lo, end, want, so->es, so->cmp);
    return want;
}

/* Technique (e2), the half-down list: sorted runs side by side from the start
 * of the array; edge[0] = 0 and run i is [edge[i], edge[i+1]).  Each run on
 * the list is at most half as long as its predecessor. */
typedef struct {
    size_t edge[130];
    int runs;
} halfdown_list;

static void list_merge_top(sorter *so, halfdown_list *L) {
    size_t a = L->edge[L->runs - 2], m = L->edge[L->runs - 1], b = L->edge[L->runs];
    merge_runs(so->base, a, m, b, so->es, so->cmp, so->tmp);
    L->edge[L->runs - 1] = b;
    L->runs--;
}

/* Appends the run that ends at `end`, then restores the half-down property:
 * while the newest run is longer than half of the one before it, the two are
 * merged (which may in turn break the property one place further back). */
static void list_append(sorter *so, halfdown_list *L, size_t end) {
    L->edge[++L->runs] = end;
    while (L->runs >= 2) {
        size_t last = L->edge[L->runs] - L->edge[L->runs - 1];
        size_t before = L->edge[L->runs - 1] - L->edge[L->runs - 2];
        if (last <= before / 2) break;
        list_merge_top(so, L);
    }
}

/* Natural mergesort of Section 3: runs are taken from the input (a), short
 * ones grown to `minrun` (b; minrun <= 1 leaves them alone), kept on the
 * half-down list (e2), and merged with trimming (f) and galloping (g).  The
 * run lengths on the list fall by half at every step, so it holds at most
 * log2(n) + 2 runs.  With minrun = MINRUN this is the paper's mer6; with
 * minrun = 1, mer5.  Returns 0, or -1 if the temporary buffer cannot be had. */
static int mergesort_runs(void *base, size_t n, size_t es, sro_cmp cmp, size_t minrun) {
    if (n < 2) return 0;
    sorter so = {(char *)base, n, es, cmp, (char *)malloc(n * es)};
    if (!so.tmp) return -1;
    halfdown_list L;
    L.edge[0] = 0;
    L.runs = 0;
    for (size_t lo = 0; lo < n;) {
        size_t end = grow_run(&so, lo, take_run(&so, lo), minrun);
        list_append(&so, &L, end);
        lo = end;
    }
    while (L.runs > 1) list_merge_top(&so, &L);    /* what is left, last run first */
    free(so.tmp);
    return 0;
}

int sro_mergesort(void *base, size_t n, size_t es, sro_cmp cmp) {
    return mergesort_runs(base, n, es, cmp, MINRUN);
}

/* ------------------------------------------------------------ quicksort */

#define ALPHA 32
#define BETA 32
#define GAMMA 2

static int is_sorted_range(const void *base, size_t lo, size_t hi, size_t es, sro_cmp cmp) {
    for (size_t k = lo; k < hi; k++)
        if (cmp(AT(base, k, es), AT(base, k + 1, es)) > 0) return 0;
    return 1;
}

static size_t med3(const void *base, size_t a, size_t b, size_t c, size_t es, sro_cmp cmp) {
    const void *pa = AT(base, a, es), *pb = AT(base, b, es), *pc = AT(base, c, es);
    if (cmp(pa, pb) < 0) {
        if (cmp(pb, pc) < 0) return b;
        return cmp(pa, pc) < 0 ? c : a;
    }
    if (cmp(pb, pc) > 0) return b;
    return cmp(pa, pc) > 0 ? c : a;
}

/* technique (c), reading R9 */
static size_t pivot9(const void *base, size_t lo, size_t hi, size_t es, sro_cmp cmp) {
    size_t d = (hi - lo) / 8;
    size_t m1 = med3(base, lo, lo + d, lo + 2 * d, es, cmp);
    size_t m2 = med3(base, lo + 3 * d, lo + 4 * d, lo + 5 * d, es, cmp);
    size_t m3 = med3(base, lo + 6 * d, lo + 7 * d, lo + 8 * d, es, cmp);
    return med3(base, m1, m2, m3, es, cmp);
}

/* The outcome of splitting [lo, hi] around a pivot value v: the recursion
 * continues on [lo, left_end] and [right_begin, hi]; `equal_seen` counts the
 * items equal to v that the split met (technique (g)). */
typedef struct {
    long left_end, right_begin;
    long equal_seen;
} split_result;

/* 2-way split with the pivot left unplaced (technique (e)): afterwards
 * [lo, left_end] <= v and [left_end + 1, hi] >= v.  Two scans move towards
 * each other, each stopping at an item on the wrong side (or equal to v), and
 * the two stopped items change places.  A median pivot is never the unique
 * largest item of the range, so both parts are shorter than the range. */
static split_result split_two_way(sorter *so, long lo, long hi, const void *v) {
    split_result r = {0, 0, 0};
    long up = lo - 1, down = hi + 1;
    for (;;) {
        int c;
        do { up++; c = so->cmp(AT(so->base, up, so->es), v); } while (c < 0);
        r.equal_seen += c == 0;
        do { down--; c = so->cmp(AT(so->base, down, so->es), v); } while (c > 0);
        r.equal_seen += c == 0;
        if (up >= down) break;
        swap_items(so->base, (size_t)up, (size_t)down, so->es);
    }
    if (down >= hi || down < lo) abort();
    r.left_end = down;
    r.right_begin = down + 1;
    return r;
}

/* 3-way split (technique (d)): items equal to v are parked at both ends of
 * the range while the scans run, then moved next to each other in the middle,
 * where they take no further part.  Afterwards [lo, left_end] < v,
 * [right_begin, hi] > v and everything between equals v. */
static split_result split_three_way(sorter *so, long lo, long hi, const void *v) {
    split_result r = {0, 0, 0};
    long eq_lo = lo, up = lo;              /* [lo, eq_lo) == v, [eq_lo, up) < v */
    long down = hi, eq_hi = hi;            /* (down, eq_hi] > v, (eq_hi, hi] == v */
    for (;;) {
        int c;
        while (up <= down && (c = so->cmp(AT(so->base, up, so->es), v)) <= 0) {
            if (c == 0) { swap_items(so->base, (size_t)eq_lo, (size_t)up, so->es); eq_lo++; r.equal_seen++; }
            up++;
        }
        while (up <= down && (c = so->cmp(AT(so->base, down, so->es), v)) >= 0) {
            if (c == 0) { swap_items(so->base, (size_t)down, (size_t)eq_hi, so->es); eq_hi--; r.equal_seen++; }
            down--;
        }
        if (up > down) break;
        swap_items(so->base, (size_t)up, (size_t)down, so->es);
        up++;
        down--;
    }
    long less = up - eq_lo, more = eq_hi - down;
    /* the left block of equal items changes places with the end of the < part */
    long s = eq_lo - lo < less ? eq_lo - lo : less;
    for (long k = 0; k < s; k++) swap_items(so->base, (size_t)(lo + k), (size_t)(up - s + k), so->es);
    /* the right block with the start of the > part */
    s = hi - eq_hi < more ? hi - eq_hi : more;
    for (long k = 0; k < s; k++) swap_items(so->base, (size_t)(up + k), (size_t)(hi + 1 - s + k), so->es);
    r.left_end = lo + less - 1;
    r.right_begin = hi + 1 - more;
    return r;
}

/* Hybrid quicksort of Section 4 on [lo, hi] (inclusive): insertion sort for
 * fewer than ALPHA items (a), nothing to do on an already sorted range (f),
 * the median of three (b) or the pseudo-median of nine (c) as pivot, and a
 * split that is 2-way until a split meets more than GAMMA items equal to its
 * pivot, after which the ranges below use the 3-way split (g, d).  The
 * shorter part recurses; the longer one continues in the loop. */
static void quick_range(sorter *so, long lo, long hi, int three_way) {
    while (hi > lo) {
        long n = hi - lo + 1;
        if (n < ALPHA) { isort_range(so->base, (size_t)lo, (size_t)lo + 1, (size_t)hi + 1, so->es, so->cmp); return; }
        if (is_sorted_range(so->base, (size_t)lo, (size_t)hi, so->es, so->cmp)) return;
        size_t p = n < BETA ? med3(so->base, (size_t)lo, (size_t)(lo + (hi - lo) / 2), (size_t)hi, so->es, so->cmp)
                            : pivot9(so->base, (size_t)lo, (size_t)hi, so->es, so->cmp);
        char v[64];
        memcpy(v, AT(so->base, p, so->es), so->es);
        split_result r = three_way ? split_three_way(so, lo, hi, v) : split_two_way(so, lo, hi, v);
        if (!three_way && r.equal_seen > GAMMA) three_way = 1;
        if (r.left_end - lo < hi - r.right_begin) {
            quick_range(so, lo, r.left_end, three_way);
            lo = r.right_begin;
        } else {
            quick_range(so, r.right_begin, hi, three_way);
            hi = r.left_end;
        }
    }
}

int sro_quicksort(void *base, size_t n, size_t es, sro_cmp cmp) {
    sorter so = {(char *)base, n, es, cmp, NULL};
    if (n >= 2) quick_range(&so, 0, (long)n - 1, 0);
    return 0;
}

int sro_isort(void *base, size_t n, size_t es, sro_cmp cmp) {
    if (n >= 2) isort_range(base, 0, 1, n, es, cmp);
    return 0;
}

/* ------------------------------------------------------------- measures */

/* Run(A) = |{ i : a_i > a_{i+1} }| + 1 (Section 2); 0 for the empty array. */
uint64_t sro_runs(const void *base, size_t n, int kt) {
    sro_cmp cmp = cmp_for(kt);
    size_t es = key_size(kt);
    if (n == 0) return 0;
    uint64_t d = 0;
    for (size_t i = 0; i + 1 < n; i++)
        if (cmp(AT(base, i, es), AT(base, i + 1, es)) > 0) d++;
    return d + 1;
}

/* Mono(A): the fewest pieces w_1..w_k, each sorted or reversely sorted
 * (Section 2).  Taking the longest monotone prefix each time is optimal, since
 * any suffix of a monotone piece is monotone. */
uint64_t sro_mono(const void *base, size_t n, int kt) {
    sro_cmp cmp = cmp_for(kt);
    size_t es = key_size(kt);
    if (n == 0) return 0;
    uint64_t pieces = 1;
    int dir = 0;                     /* 0: piece so far is constant */
    for (size_t i = 0; i + 1 < n; i++) {
        int c = cmp(AT(base, i, es), AT(base, i + 1, es));
        if (c == 0) continue;
        int d = c < 0 ? 1 : -1;
        if (dir == 0) dir = d;
        else if (d != dir) { pieces++; dir = 0; }
    }
    return pieces;
}

/* Inv(A) = |{ (i, j) : i < j, a_i > a_j }| by its definition, O(n^2). */
uint64_t sro_inversions(const void *base, size_t n, int kt) {
    sro_cmp cmp = cmp_for(kt);
    size_t es = key_size(kt);
    uint64_t inv = 0;
    for (size_t i = 0; i < n; i++)
        for (size_t j = i + 1; j < n; j++)
            if (cmp(AT(base, i, es), AT(base, j, es)) > 0) inv++;
    return inv;
}

/* Rem(A): the fewest items whose removal leaves a non-decreasing list, i.e. n
 * minus the length of a longest non-decreasing subsequence, found by patience
 * sorting: tail[l] is the index of the smallest possible last item of a
 * non-decreasing subsequence of length l + 1 seen so far; each item replaces
 * the first tail greater than it (or extends the longest).  UINT64_MAX if the
 * work array cannot be allocated. */
uint64_t sro_rem(const void *base, size_t n, int kt) {
    sro_cmp cmp = cmp_for(kt);
    size_t es = key_size(kt);
    if (n == 0) return 0;
    size_t *tail = (size_t *)malloc(n * sizeof(size_t));
    if (!tail) return UINT64_MAX;
    size_t len = 0;
    for (size_t i = 0; i < n; i++) {
        size_t lo = 0, hi = len;
        while (lo < hi) {
            const size_t mid = lo + (hi - lo) / 2;
            if (cmp(AT(base, tail[mid], es), AT(base, i, es)) > 0) hi = mid;
            else lo = mid + 1;
        }
        tail[lo] = i;
        if (lo == len) len++;
    }
    free(tail);
    return (uint64_t)(n - len);
}

/* --------------------------------------------------------- entry points */

enum { SRO_ALGO_MERGE = 0, SRO_ALGO_QUICK = 1, SRO_ALGO_ISORT = 2, SRO_ALGO_MERGE5 = 3 };

static int run_algo(void *base, size_t n, size_t es, sro_cmp cmp, int algo) {
    switch (algo) {
    case SRO_ALGO_MERGE: return sro_mergesort(base, n, es, cmp);
    case SRO_ALGO_QUICK: return sro_quicksort(base, n, es, cmp);
    case SRO_ALGO_ISORT: return sro_isort(base, n, es, cmp);
    case SRO_ALGO_MERGE5: return mergesort_runs(base, n, es, cmp, 1);
    default: return -2;
    }
}

/* Sorts keys of type kt in place with the named algorithm. */
int sro_sort_keys(void *keys, size_t n, int kt, int algo) {
    sro_cmp cmp = cmp_for(kt);
    if (!cmp) return -2;
    return run_algo(keys, n, key_size(kt), cmp, algo);
}

/* Stable sort of (key, payload) pairs: the items are packed as key bytes
 * followed by the 4-byte payload, the comparator reads the key only, and a
 * stable algorithm (mergesort or insertion sort) keeps equal keys in input
 * order. */
int sro_sort_pairs(void *keys, uint32_t *vals, size_t n, int kt, int algo) {
    sro_cmp cmp = cmp_for(kt);
    if (!cmp) return -2;
    if (algo == SRO_ALGO_QUICK) return -2;    /* not stable */
    size_t ks = key_size(kt), es = ks + 4;
    char *items = (char *)malloc(n ? n * es : 1);
    if (!items) return -1;
    for (size_t i = 0; i < n; i++) {
        memcpy(items + i * es, (char *)keys + i * ks, ks);
        memcpy(items + i * es + ks, vals + i, 4);
    }
    int rc = run_algo(items, n, es, cmp, algo);
    for (size_t i = 0; i < n; i++) {
        memcpy((char *)keys + i * ks, items + i * es, ks);
        memcpy(vals + i, items + i * es + ks, 4);
    }
    free(items);
    return rc;
}

/* Sorts each segment [off[s], off[s+1]) on its own. */
int sro_sort_segmented(void *keys, const int64_t *off, size_t nseg, int kt, int algo) {
    sro_cmp cmp = cmp_for(kt);
    if (!cmp) return -2;
    size_t ks = key_size(kt);
    for (size_t s = 0; s < nseg; s++) {
        if (off[s + 1] < off[s]) return -3;
        int rc = run_algo((char *)keys + (size_t)off[s] * ks, (size_t)(off[s + 1] - off[s]), ks, cmp, algo);
        if (rc) return rc;
    }
    return 0;
}

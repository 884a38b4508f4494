/*
 * cch_oracle.c -- CPU oracle for the planar convex hull that CudaChain computes.
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the slow, plain reference that the
 * CUDA path is checked against.  Only the test suite, the smoke check and the
 * CPU-baseline leg of the benchmark may build, load or call it; the product
 * path never does.  It shares no code, header, table or helper with the CUDA
 * library.
 *
 * Two things live here:
 *
 *   1. oracle_hull_*: the DEFINITION of the output -- the vertex set of the
 *      strict convex hull (no collinear or duplicate points), reported as input
 *      indices in counter-clockwise order starting at the lexicographically
 *      smallest (x, then y) vertex, each vertex represented by the smallest
 *      input index among points with identical coordinates.  Computed with
 *      Andrew's monotone chain (the paper's reference [4], Sec. 1) on exact
 *      orientation predicates.
 *
 *   2. oracle_method_*: a sequential restatement of the paper's procedure
 *      (Sec. 2.1, steps 1-7; Table 1; Sec. 2.1.1 region rules; Fig. 2 SPA
 *      rules), emitting every intermediate set so that the GPU stages can be
 *      compared stage by stage.  Readings of silent or garbled passages:
 *        - region k <=> the point lies STRICTLY to the right of the directed
 *          quadrilateral edge E_k -> E_{k+1} (outside), first match in the
 *          order 1..4 (Sec. 2.1.1; the printed "left side" contradicts
 *          Fig. 1 for a counter-clockwise quadrilateral);
 *        - points on an edge, and the extremes themselves, fall in R0;
 *        - extremes: P_minx = lexmin(x,y), P_miny = lexmin(y,x),
 *          P_maxx = lexmax(x,y), P_maxy = lexmax(y,x), ties -> smallest index;
 *        - sorting is stable (equal keys keep index order);
 *        - SPA starts its running value t at the region's first extreme,
 *          tests every region point, discards only when strictly worse
 *          (Fig. 2 as printed) and otherwise sets t to the point's value;
 *        - the final hull of the simple polygon (step 7) is taken per chain
 *          with a strict left-turn stack, which yields the same unique hull
 *          as Melkman's algorithm on the polygon.
 *
 * Orientation predicate orient(a,b,c) = sign((b-a) x (c-a)):
 *   int32  -- exact in 128-bit integer arithmetic.
 *   double -- exact: the determinant is expanded into six products of input
 *             coordinates, each product is split exactly into a rounded part
 *             and its error term (fma), and the twelve resulting doubles are
 *             summed exactly with Shewchuk's Grow-Expansion (J. R. Shewchuk,
 *             "Adaptive Precision Floating-Point Arithmetic and Fast Robust
 *             Geometric Predicates", 1997, Sec. 2).  The sign of a
 *             non-overlapping expansion is the sign of its largest nonzero
 *             component.  Exact for coordinates that are 0 or of magnitude in
 *             [2^-400, 2^400]; must be compiled with -ffp-contract=off.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <math.h>

/* ------------------------------------------------------------------ */
/* exact orientation                                                    */
/* ------------------------------------------------------------------ */

int oracle_orient_i32(int32_t ax, int32_t ay, int32_t bx, int32_t by,
                      int32_t cx, int32_t cy)
{
    __int128 l = (__int128)((int64_t)bx - ax) * ((int64_t)cy - ay);
    __int128 r = (__int128)((int64_t)by - ay) * ((int64_t)cx - ax);
    __int128 d = l - r;
    return (d > 0) - (d < 0);
}

/* Knuth's TwoSum: s + e == a + b exactly. */
static void two_sum(double a, double b, double *s, double *e)
{
    double x = a + b;
    double bv = x - a;
    double av = x - bv;
    double br = b - bv;
    double ar = a - av;
    *s = x;
    *e = ar + br;
}

/* Grow-Expansion: add b to the non-overlapping expansion h[0..m) (smallest
 * magnitude first); the result has m+1 components. */
static int grow(double *h, int m, double b)
{
    double q = b;
    for (int i = 0; i < m; i++) {
        double s, e;
        two_sum(q, h[i], &s, &e);
        h[i] = e;
        q = s;
    }
    h[m] = q;
    return m + 1;
}

int oracle_orient_f64(double ax, double ay, double bx, double by,
                      double cx, double cy)
{
    /* det = bx*cy - bx*ay - ax*cy - by*cx + by*ax + ay*cx */
    double f[6][2] = {
        { bx,  cy}, {-bx,  ay}, {-ax,  cy},
        {-by,  cx}, { by,  ax}, { ay,  cx},
    };
    double h[13];
    int m = 0;
    for (int k = 0; k < 6; k++) {
        double p = f[k][0] * f[k][1];
        double e = fma(f[k][0], f[k][1], -p);
        m = grow(h, m, e);
        m = grow(h, m, p);
    }
    for (int i = m - 1; i >= 0; i--) {
        if (h[i] > 0) return 1;
        if (h[i] < 0) return -1;
    }
    return 0;
}

/* ------------------------------------------------------------------ */
/* typed point access                                                   */
/* ------------------------------------------------------------------ */

typedef struct {
    int dtype;           /* 1 = int32, 2 = double */
    const int32_t *pi;   /* [n,2] interleaved */
    const double *pd;
} pts_t;

static inline double px(const pts_t *P, int64_t i) { return P->dtype == 1 ? (double)P->pi[2*i] : P->pd[2*i]; }
static inline double py(const pts_t *P, int64_t i) { return P->dtype == 1 ? (double)P->pi[2*i+1] : P->pd[2*i+1]; }

/* Value comparison of one coordinate (c = 0 for x, 1 for y).  For doubles,
 * -0.0 and +0.0 compare equal; int32 values are exactly representable. */
static inline int cmpc(const pts_t *P, int64_t i, int64_t j, int c)
{
    if (P->dtype == 1) {
        int32_t a = P->pi[2*i+c], b = P->pi[2*j+c];
        return (a > b) - (a < b);
    } else {
        double a = P->pd[2*i+c], b = P->pd[2*j+c];
        return (a > b) - (a < b);
    }
}

static inline int same_point(const pts_t *P, int64_t i, int64_t j)
{
    return cmpc(P, i, j, 0) == 0 && cmpc(P, i, j, 1) == 0;
}

static inline int orient(const pts_t *P, int64_t a, int64_t b, int64_t c)
{
    if (P->dtype == 1)
        return oracle_orient_i32(P->pi[2*a], P->pi[2*a+1], P->pi[2*b], P->pi[2*b+1],
                                 P->pi[2*c], P->pi[2*c+1]);
    return oracle_orient_f64(P->pd[2*a], P->pd[2*a+1], P->pd[2*b], P->pd[2*b+1],
                             P->pd[2*c], P->pd[2*c+1]);
}

/* ------------------------------------------------------------------ */
/* merge sort of index arrays (stable; comparator on points)            */
/* ------------------------------------------------------------------ */

typedef int (*less_fn)(const pts_t *P, int64_t a, int64_t b, int mode);

static void msort(int64_t *a, int64_t *tmp, int64_t n, const pts_t *P,
                  less_fn less, int mode)
{
    if (n < 2) return;
    /* bottom-up, stable: take from the left run unless right < left */
    int64_t *src = a, *dst = tmp;
    for (int64_t w = 1; w < n; w *= 2) {
        for (int64_t lo = 0; lo < n; lo += 2 * w) {
            int64_t mid = lo + w < n ? lo + w : n;
            int64_t hi = lo + 2 * w < n ? lo + 2 * w : n;
            int64_t i = lo, j = mid, k = lo;
            while (i < mid && j < hi)
                dst[k++] = less(P, src[j], src[i], mode) ? src[j++] : src[i++];
            while (i < mid) dst[k++] = src[i++];
            while (j < hi) dst[k++] = src[j++];
        }
        int64_t *t = src; src = dst; dst = t;
    }
    if (src != a) memcpy(a, src, (size_t)n * sizeof(int64_t));
}

/* lexicographic (x, y) with index as the final key */
static int less_xy_idx(const pts_t *P, int64_t a, int64_t b, int mode)
{
    (void)mode;
    int c = cmpc(P, a, b, 0);
    if (c) return c < 0;
    c = cmpc(P, a, b, 1);
    if (c) return c < 0;
    return a < b;
}

/* ------------------------------------------------------------------ */
/* 1. the definition: Andrew's monotone chain                          */
/* ------------------------------------------------------------------ */

/* Returns h >= 0 and writes h indices to out (capacity >= n, >= 1). */
static int64_t hull_andrew(const pts_t *P, int64_t n, int32_t *out)
{
    if (n <= 0) return 0;
    int64_t *ord = malloc((size_t)n * sizeof(int64_t));
    int64_t *tmp = malloc((size_t)n * sizeof(int64_t));
    int64_t *stk = malloc((size_t)(2 * n + 2) * sizeof(int64_t));
    for (int64_t i = 0; i < n; i++) ord[i] = i;
    msort(ord, tmp, n, P, less_xy_idx, 0);
    /* drop later copies of identical coordinates: the first of each run has
     * the smallest index because the index is the last sort key */
    int64_t m = 0;
    for (int64_t i = 0; i < n; i++)
        if (m == 0 || !same_point(P, ord[m - 1], ord[i])) ord[m++] = ord[i];
    int64_t h = 0;
    if (m == 1) {
        out[0] = (int32_t)ord[0];
        h = 1;
    } else {
        int64_t t = 0;
        for (int64_t i = 0; i < m; i++) {               /* lower chain */
            while (t >= 2 && orient(P, stk[t - 2], stk[t - 1], ord[i]) <= 0) t--;
            stk[t++] = ord[i];
        }
        int64_t lower = t + 1;
        for (int64_t i = m - 2; i >= 0; i--) {          /* upper chain */
            while (t >= lower && orient(P, stk[t - 2], stk[t - 1], ord[i]) <= 0) t--;
            stk[t++] = ord[i];
        }
        h = t - 1;                                      /* last == first */
        for (int64_t i = 0; i < h; i++) out[i] = (int32_t)stk[i];
    }
    free(ord); free(tmp); free(stk);
    return h;
}

int64_t oracle_hull_i32(const int32_t *pts, int64_t n, int32_t *out)
{
    pts_t P = {1, pts, NULL};
    return hull_andrew(&P, n, out);
}

int64_t oracle_hull_f64(const double *pts, int64_t n, int32_t *out)
{
    pts_t P = {2, NULL, pts};
    return hull_andrew(&P, n, out);
}

/* ------------------------------------------------------------------ */
/* 2. the method, step by step (Sec. 2.1)                              */
/* ------------------------------------------------------------------ */

/* sort orders of Table 1: 1 = x asc, 2 = y asc, 3 = x desc, 4 = y desc;
 * ties keep index order (the index is the final key) */
static int less_region(const pts_t *P, int64_t a, int64_t b, int mode)
{
    int c;
    switch (mode) {
    case 1: c = cmpc(P, a, b, 0); break;
    case 2: c = cmpc(P, a, b, 1); break;
    case 3: c = -cmpc(P, a, b, 0); break;
    default: c = -cmpc(P, a, b, 1); break;
    }
    if (c) return c < 0;
    return a < b;
}

/*
 * Runs steps 1-7 on n >= 1 points.  Outputs (all caller-allocated):
 *   ext[4]        indices of P_minx, P_miny, P_maxx, P_maxy (= E1..E4)
 *   region[n]     0..4 per point (step 2, Sec. 2.1.1)
 *   r1_idx[n]     round-1 survivors, region-major, index order within a
 *                 region; r1_cnt[4] their counts
 *   sorted_idx[n] the same sets sorted per Table 1 (step 4)
 *   spa_idx[n]    SPA survivors in sorted order (step 5, Fig. 2);
 *                 spa_cnt[4]
 *   hull[n]       final hull (steps 6-7); returns its size h
 */
int64_t oracle_method(int dtype, const void *pts, int64_t n,
                      int32_t *ext, int8_t *region,
                      int32_t *r1_idx, int64_t *r1_cnt,
                      int32_t *sorted_idx,
                      int32_t *spa_idx, int64_t *spa_cnt,
                      int32_t *hull)
{
    pts_t P = {dtype, dtype == 1 ? (const int32_t *)pts : NULL,
               dtype == 2 ? (const double *)pts : NULL};
    if (n <= 0) {
        for (int k = 0; k < 4; k++) { r1_cnt[k] = 0; spa_cnt[k] = 0; ext[k] = -1; }
        return 0;
    }

    /* step 1: the four extreme points (lexicographic, smallest index) */
    int64_t e_minx = 0, e_miny = 0, e_maxx = 0, e_maxy = 0;
    for (int64_t i = 1; i < n; i++) {
        int cx = cmpc(&P, i, e_minx, 0), cy = cmpc(&P, i, e_minx, 1);
        if (cx < 0 || (cx == 0 && cy < 0)) e_minx = i;
        cx = cmpc(&P, i, e_maxx, 0); cy = cmpc(&P, i, e_maxx, 1);
        if (cx > 0 || (cx == 0 && cy > 0)) e_maxx = i;
        cy = cmpc(&P, i, e_miny, 1); cx = cmpc(&P, i, e_miny, 0);
        if (cy < 0 || (cy == 0 && cx < 0)) e_miny = i;
        cy = cmpc(&P, i, e_maxy, 1); cx = cmpc(&P, i, e_maxy, 0);
        if (cy > 0 || (cy == 0 && cx > 0)) e_maxy = i;
    }
    int64_t E[5] = {e_minx, e_miny, e_maxx, e_maxy, e_minx};
    for (int k = 0; k < 4; k++) ext[k] = (int32_t)E[k];

    /* steps 2-3: R_k = strictly outside edge E_k -> E_{k+1}, first match */
    for (int64_t i = 0; i < n; i++) {
        int r = 0;
        for (int k = 0; k < 4 && r == 0; k++)
            if (orient(&P, E[k], E[k + 1], i) < 0) r = k + 1;
        region[i] = (int8_t)r;
    }
    int64_t off = 0;
    for (int k = 0; k < 4; k++) {
        int64_t c = 0;
        for (int64_t i = 0; i < n; i++)
            if (region[i] == k + 1) r1_idx[off + c++] = (int32_t)i;
        r1_cnt[k] = c;
        off += c;
    }

    /* step 4: stable sort of each region by the Table 1 order */
    int64_t *a = malloc((size_t)(off > 0 ? off : 1) * sizeof(int64_t));
    int64_t *tmp = malloc((size_t)(off > 0 ? off : 1) * sizeof(int64_t));
    off = 0;
    for (int k = 0; k < 4; k++) {
        int64_t c = r1_cnt[k];
        for (int64_t j = 0; j < c; j++) a[off + j] = r1_idx[off + j];
        msort(a + off, tmp, c, &P, less_region, k + 1);
        for (int64_t j = 0; j < c; j++) sorted_idx[off + j] = (int32_t)a[off + j];
        off += c;
    }

    /* step 5: SPA (Fig. 2).  coord: y for R1/R3, x for R2/R4; a point is
     * interior when its coordinate is strictly above t (R1), below t (R2),
     * below t (R3), above t (R4). */
    int64_t soff = 0;
    off = 0;
    for (int k = 0; k < 4; k++) {
        int c_is_y = (k == 0 || k == 2);
        int cc = c_is_y ? 1 : 0;
        int drop_if_greater = (k == 0 || k == 3);
        int64_t tpt = E[k];                 /* t = coordinate of first point */
        int64_t kept = 0;
        for (int64_t j = 0; j < r1_cnt[k]; j++) {
            int64_t p = sorted_idx[off + j];
            int c = cmpc(&P, p, tpt, cc);
            int interior = drop_if_greater ? (c > 0) : (c < 0);
            if (!interior) {
                tpt = p;
                spa_idx[soff + kept++] = (int32_t)p;
            }
        }
        spa_cnt[k] = kept;
        soff += kept;
        off += r1_cnt[k];
    }

    /* steps 6-7: chain k = E_k, survivors, E_{k+1}; convex chain by a strict
     * left-turn stack, adjacent identical points dropped (first kept); the
     * polygon is the concatenation of the chains without their last point.
     * A chain whose two ends are the same point contributes nothing. */
    int64_t *stk = malloc((size_t)(soff + 8) * sizeof(int64_t));
    int64_t h = 0;
    soff = 0;
    for (int k = 0; k < 4; k++) {
        int64_t cnt = spa_cnt[k];
        if (E[k] != E[k + 1]) {
            int64_t t = 0;
            for (int64_t j = -1; j <= cnt; j++) {
                int64_t p = j < 0 ? E[k] : (j == cnt ? E[k + 1] : spa_idx[soff + j]);
                if (t > 0 && same_point(&P, stk[t - 1], p)) continue;
                while (t >= 2 && orient(&P, stk[t - 2], stk[t - 1], p) <= 0) t--;
                stk[t++] = p;
            }
            for (int64_t j = 0; j + 1 < t; j++) hull[h++] = (int32_t)stk[j];
        }
        soff += cnt;
    }
    if (h == 0) hull[h++] = (int32_t)E[0];  /* every point identical */
    free(a); free(tmp); free(stk);
    return h;
}

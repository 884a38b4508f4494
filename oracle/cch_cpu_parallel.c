/*
 * cch_cpu_parallel.c -- multi-core CPU baseline for the hull (OpenMP).
 *
 * TEST AND BENCHMARK INFRASTRUCTURE ONLY, like the oracle it includes: the
 * benchmark's CPU-baseline leg times it beside the single-thread oracle, and
 * the test suite checks that it returns exactly the oracle's hull.  The
 * product path never builds, loads or calls it.
 *
 * The classical multi-core route to the same output:
 *   1. the extreme points in eight directions (x, x + y, y, x - y, each way)
 *      by a parallel reduction;
 *   2. the Akl-Toussaint filter in parallel: the eight points, in the
 *      angular order of their directions, close a polygon; a point strictly
 *      to the left of every one of its edges is surrounded by it, so it lies
 *      strictly inside the hull of input points and is no hull vertex (this
 *      holds for any input points in any order: a wrong order only makes the
 *      filter drop less).  Every other point is kept, in index order; points
 *      on an edge or at a corner stay, so every copy of a hull vertex
 *      survives and the smallest index still represents it;
 *   3. a parallel merge sort of the survivors by (x, y, index): sorted chunks,
 *      then pairwise merges;
 *   4. Andrew's monotone chain over the sorted survivors, as in the oracle.
 * The exact predicates, comparisons and the sort step are the oracle's own
 * (this file includes its source); a floating-point filter decides the easy
 * orientations first.  The result is the oracle's hull exactly.
 */
#include "cch_oracle.c"

#include <omp.h>

/* Orientation with Shewchuk's floating-point filter in front of the
 * oracle's exact predicate: with the differences and products rounded, the
 * computed determinant has the true sign whenever its magnitude exceeds
 * (3 + 16 eps) eps (|detleft| + |detright|), eps = 2^-53 (Shewchuk, "Adaptive
 * precision floating-point arithmetic and fast robust geometric predicates",
 * 1997, orient2d stage A); otherwise the exact expansion decides.  int32
 * points go to the oracle's exact integer predicate directly. */
static inline int fast_orient(const pts_t *P, int64_t a, int64_t b, int64_t c)
{
    if (P->dtype == 1) return orient(P, a, b, c);
    const double ax = P->pd[2*a], ay = P->pd[2*a+1], bx = P->pd[2*b], by = P->pd[2*b+1];
    const double cx = P->pd[2*c], cy = P->pd[2*c+1];
    const double dl = (bx - ax) * (cy - ay), dr = (by - ay) * (cx - ax);
    const double det = dl - dr;
    const double bound = 3.3306690738754716e-16 * (fabs(dl) + fabs(dr));   /* (3 + 16 eps) eps */
    if (det > bound) return 1;
    if (-det > bound) return -1;
    return oracle_orient_f64(ax, ay, bx, by, cx, cy);
}

/* score of point i in direction e (counter-clockwise from -x): -x, -(x+y),
 * -y, x-y, x, x+y, y, y-x; the polygon's vertices maximise them */
static inline double dir_score(const pts_t *P, int64_t i, int e)
{
    const double x = px(P, i), y = py(P, i);
    switch (e) {
        case 0: return -x;
        case 1: return -(x + y);
        case 2: return -y;
        case 3: return x - y;
        case 4: return x;
        case 5: return x + y;
        case 6: return y;
        default: return y - x;
    }
}

/* merge of two sorted runs (stable, left first on ties) */
static void merge_runs(const int64_t *a, int64_t na, const int64_t *b, int64_t nb, int64_t *dst, const pts_t *P)
{
    int64_t i = 0, j = 0, k = 0;
    while (i < na && j < nb) dst[k++] = less_xy_idx(P, b[j], a[i], 0) ? b[j++] : a[i++];
    while (i < na) dst[k++] = a[i++];
    while (j < nb) dst[k++] = b[j++];
}

static int64_t parallel_hull(const pts_t *P, int64_t n, int32_t *out, int threads)
{
    if (n <= 0) return 0;
    if (threads <= 0) threads = omp_get_max_threads();
    if (threads > 256) threads = 256;

    /* 1. extremes (the team may be smaller than asked: use its real size) */
    int64_t ext[256][8];
    int team = 1;
    for (int t = 0; t < 256; t++)
        for (int e = 0; e < 8; e++) ext[t][e] = -1;
#pragma omp parallel num_threads(threads)
    {
        int t = omp_get_thread_num(), nt = omp_get_num_threads();
        if (t == 0) team = nt;
        int64_t lo = n * t / nt, hi = n * (t + 1) / nt;
        if (hi > lo) {
            int64_t b[8];
            double v[8];
            for (int e = 0; e < 8; e++) { b[e] = lo; v[e] = dir_score(P, lo, e); }
            for (int64_t i = lo + 1; i < hi; i++)
                for (int e = 0; e < 8; e++) {
                    const double d = dir_score(P, i, e);
                    if (d > v[e]) { v[e] = d; b[e] = i; }
                }
            for (int e = 0; e < 8; e++) ext[t][e] = b[e];
        }
    }
    int64_t Q[8];
    for (int e = 0; e < 8; e++) {
        Q[e] = -1;
        for (int t = 0; t < team; t++)
            if (ext[t][e] >= 0 && (Q[e] < 0 || dir_score(P, ext[t][e], e) > dir_score(P, Q[e], e)))
                Q[e] = ext[t][e];
    }

    /* 2. filter: drop what is strictly left of every edge of the closed
     * polygon Q[0..7] (edges between identical corners are skipped; fewer
     * than three edges leave nothing inside).  Every chunk lists its
     * survivors in index order in place, then copies them to its offset in
     * `sel`. */
    int live[8], nlive = 0;
    for (int k = 0; k < 8; k++) {
        live[k] = !same_point(P, Q[k], Q[(k + 1) & 7]);
        nlive += live[k];
    }
    int64_t *keep = malloc((size_t)n * sizeof(int64_t));
    int64_t *sel = malloc((size_t)n * sizeof(int64_t));
    int64_t cnt[257];
    for (int t = 0; t < 257; t++) cnt[t] = 0;
#pragma omp parallel num_threads(team)
    {
        int t = omp_get_thread_num(), nt = omp_get_num_threads();
        int64_t lo = n * t / nt, hi = n * (t + 1) / nt, c = 0;
        for (int64_t i = lo; i < hi; i++) {
            int inside = nlive >= 3;
            for (int k = 0; k < 8 && inside; k++)
                if (live[k] && fast_orient(P, Q[k], Q[(k + 1) & 7], i) <= 0) inside = 0;
            if (!inside) keep[lo + c++] = i;
        }
        cnt[t + 1] = c;
#pragma omp barrier
#pragma omp single
        {
            for (int q = 1; q <= nt; q++) cnt[q] += cnt[q - 1];
            team = nt;
        }
        memcpy(sel + cnt[t], keep + lo, (size_t)c * sizeof(int64_t));
    }
    const int64_t m = cnt[team];
    free(keep);
    threads = team;

    /* 3. parallel merge sort by (x, y, index) */
    int64_t *tmp = malloc((size_t)(m > 0 ? m : 1) * sizeof(int64_t));
    int64_t *keep_sorted = sel;
    int64_t bounds[257];
    for (int t = 0; t <= threads; t++) bounds[t] = m * t / threads;
#pragma omp parallel for num_threads(threads) schedule(static)
    for (int t = 0; t < threads; t++)
        msort(keep_sorted + bounds[t], tmp + bounds[t], bounds[t + 1] - bounds[t], P, less_xy_idx, 0);
    int64_t *src = keep_sorted, *dst = tmp;
    for (int w = 1; w < threads; w *= 2) {
#pragma omp parallel for num_threads(threads) schedule(dynamic, 1)
        for (int t = 0; t < threads; t += 2 * w) {
            int mid = t + w < threads ? t + w : threads, hi = t + 2 * w < threads ? t + 2 * w : threads;
            merge_runs(src + bounds[t], bounds[mid] - bounds[t], src + bounds[mid], bounds[hi] - bounds[mid],
                       dst + bounds[t], P);
        }
        int64_t *x = src; src = dst; dst = x;
    }

    /* 4. Andrew's monotone chain over the sorted survivors */
    int64_t u = 0;
    for (int64_t i = 0; i < m; i++)
        if (u == 0 || !same_point(P, src[u - 1], src[i])) src[u++] = src[i];
    int64_t h = 0;
    if (u == 1) {
        out[0] = (int32_t)src[0];
        h = 1;
    } else if (u > 1) {
        int64_t *stk = malloc((size_t)(2 * u + 2) * sizeof(int64_t));
        int64_t t = 0;
        for (int64_t i = 0; i < u; i++) {
            while (t >= 2 && fast_orient(P, stk[t - 2], stk[t - 1], src[i]) <= 0) t--;
            stk[t++] = src[i];
        }
        int64_t lower = t + 1;
        for (int64_t i = u - 2; i >= 0; i--) {
            while (t >= lower && fast_orient(P, stk[t - 2], stk[t - 1], src[i]) <= 0) t--;
            stk[t++] = src[i];
        }
        h = t - 1;
        for (int64_t i = 0; i < h; i++) out[i] = (int32_t)stk[i];
        free(stk);
    }
    free(sel);
    free(tmp);
    return h;
}

int64_t cpu_parallel_hull_i32(const int32_t *pts, int64_t n, int32_t *out, int threads)
{
    pts_t P = {1, pts, NULL};
    return parallel_hull(&P, n, out, threads);
}

int64_t cpu_parallel_hull_f64(const double *pts, int64_t n, int32_t *out, int threads)
{
    pts_t P = {2, NULL, pts};
    return parallel_hull(&P, n, out, threads);
}

int cpu_parallel_threads(void) { return omp_get_max_threads(); }

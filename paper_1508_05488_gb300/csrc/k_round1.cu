// k_round1.cu -- first round of discarding (Sec. 2.1 steps 1-3, Sec. 2.1.1).
//
//  k_extremes  one streaming pass over the points: the four lexicographic
//              extremes E1..E4 = P_minx, P_miny, P_maxx, P_maxy (smallest
//              index on ties) and the float64 domain check; the last CTA of
//              each set sets up its edges and bucket maps.
//  k_stairs    the SPA-dominance tables of a sample of each set (see below).
//  k_classify  second streaming pass, fed by a TMA ring of shared-memory
//              tiles: the quadrilateral test with region routing (first k
//              whose directed edge E_k -> E_{k+1} has the point strictly on
//              its right, i.e. outside) and the dominance prefilters; every
//              consumer warp compacts the survivors of its part of a tile
//              (a sub-slot) in place, in index order, and counts them per
//              region.  The shared-memory path and the multi-block path move
//              the survivors into region-major order themselves.
//
// Dominance prefilter.  SPA (Fig. 2) discards a point P of region R_r when a
// point Q of R_r before P in the Table 1 order has a strictly better compared
// coordinate (Fig. 3).  If Q is ANY input point strictly before P in the sort
// coordinate and strictly better in the compared one, Q itself lies in R_r
// (it is on the outer side of edge r and on the inner side of the earlier
// edges), so P is not an SPA survivor of the full set and dropping it early
// leaves the SPA survivors -- and the hull -- unchanged.  k_stairs buckets
// the staircase steps of a sample by the sort coordinate (monotone FP32 map)
// and keeps per bucket the best compared coordinate, as the order word of
// its FP32 view (the view is non-decreasing in the coordinate, so a strictly
// larger word means a strictly worse coordinate); the prefix minimum over
// lower buckets, seeded with the region's first extreme, gives for every
// bucket a word such that any region point of that bucket with a larger word
// is dominated by a sample point of a strictly lower bucket.
//
// Dominance box.  The same argument in all four quadrants at once: k_stairs
// also picks the sample point furthest into each quadrant (smallest x+y,
// y-x, -x-y, x-y).  A point strictly inside the box they span is strictly
// beaten in every quadrant -- in particular in the quadrant of whichever
// region it falls in, by a point of that region -- so it is neither a hull
// vertex nor an SPA survivor.  The test is four FP32 compares on the
// monotone views.
#include "cch_internal.cuh"

namespace cch {

template <int DT>
struct PointT;
template <>
struct PointT<DT_F64> { using T = double2; };
template <>
struct PointT<DT_I32> { using T = int2; };
template <>
struct PointT<DT_F32> { using T = double2; };   // widened

// Bytes a point takes in the input (float32: one word in each vector).
template <int DT>
constexpr int in_bytes() { return DT == DT_F64 ? 16 : 8; }

// ------------------------------------------------------------- keys

// Top word of 2^-126, read as FP32: a coordinate whose top word reads below
// it in magnitude is zero or below 2^-126 in magnitude, and gets the exact
// bookkeeping -- the lower end of the domain check (nonzero magnitudes below
// 2^-400 are out of range) and the smallest top-word magnitude of the set,
// zeros included, which tells a2 whether its short FP32 view is valid.
constexpr uint32_t kTinyTopBits = (1023u - 126u) << 20;
#define kTinyTopF __uint_as_float(kTinyTopBits)

// Order-preserving key of a float64 as 32-bit words (-0.0 -> +0.0).  Also
// folds the magnitude of a nonzero value into `amin` (top word), for the
// lower end of the domain check.
__device__ __forceinline__ void f64_key_words(uint64_t b, uint32_t& kh, uint32_t& kl, uint32_t& amin) {
  uint32_t h = (uint32_t)(b >> 32), l = (uint32_t)b;
  uint32_t a = h & 0x7FFFFFFFu;
  bool nz = (a | l) != 0;
  amin = min(amin, nz ? a : 0x7FFFFFFFu);
  h = nz ? h : 0u;
  uint32_t m = (uint32_t)((int32_t)h >> 31);
  kh = h ^ (m | 0x80000000u);
  kl = l ^ m;
}

// Top key word only (no domain bookkeeping).
__device__ __forceinline__ uint32_t f64_key_hi(uint64_t b) {
  uint32_t h = (uint32_t)(b >> 32), l = (uint32_t)b;
  if (((h & 0x7FFFFFFFu) | l) == 0) h = 0;
  return h ^ ((uint32_t)((int32_t)h >> 31) | 0x80000000u);
}

__device__ __forceinline__ uint64_t kw(uint32_t h, uint32_t l) { return ((uint64_t)h << 32) | l; }

// ------------------------------------------------------------------ a1

// Lexicographic minimum over (k1, k2, idx).  All four extremes are minima:
// E1 (kx, ky), E2 (ky, kx), E3 (~kx, ~ky), E4 (~ky, ~kx); int32 packs both
// 32-bit keys into k1.
struct Lex {
  uint64_t k1, k2;
  uint32_t idx;
};

__device__ __forceinline__ bool lex_less(const Lex& a, const Lex& b) {
  return a.k1 < b.k1 || (a.k1 == b.k1 && (a.k2 < b.k2 || (a.k2 == b.k2 && a.idx < b.idx)));
}
__device__ __forceinline__ void lex_min_into(Lex& a, const Lex& b) {
  if (lex_less(b, a)) a = b;
}
// Warp-wide minima in every lane, one warp reduction (redux) per 32-bit
// word: a 64-bit minimum takes its high word's minimum, then the low words'
// minimum over the lanes that hold it; the lexicographic minimum of
// (k1, k2, idx) goes word by word the same way.
__device__ __forceinline__ uint64_t u64_warp_min(uint64_t v) {
  const uint32_t hi = __reduce_min_sync(0xFFFFFFFFu, (uint32_t)(v >> 32));
  const uint32_t lo = __reduce_min_sync(0xFFFFFFFFu, (uint32_t)(v >> 32) == hi ? (uint32_t)v : 0xFFFFFFFFu);
  return kw(hi, lo);
}
__device__ __forceinline__ Lex lex_warp_min(const Lex& v) {
  const uint32_t w0 = (uint32_t)(v.k1 >> 32), w1 = (uint32_t)v.k1, w2 = (uint32_t)(v.k2 >> 32), w3 = (uint32_t)v.k2;
  const uint32_t m0 = __reduce_min_sync(0xFFFFFFFFu, w0);
  bool t = w0 == m0;
  const uint32_t m1 = __reduce_min_sync(0xFFFFFFFFu, t ? w1 : 0xFFFFFFFFu);
  t = t && w1 == m1;
  const uint32_t m2 = __reduce_min_sync(0xFFFFFFFFu, t ? w2 : 0xFFFFFFFFu);
  t = t && w2 == m2;
  const uint32_t m3 = __reduce_min_sync(0xFFFFFFFFu, t ? w3 : 0xFFFFFFFFu);
  t = t && w3 == m3;
  Lex r;
  r.k1 = kw(m0, m1);
  r.k2 = kw(m2, m3);
  r.idx = __reduce_min_sync(0xFFFFFFFFu, t ? v.idx : 0xFFFFFFFFu);
  return r;
}

template <int DT>
__device__ __forceinline__ void cand_keys(uint32_t xh, uint32_t xl, uint32_t yh, uint32_t yl, int e,
                                          uint64_t& k1, uint64_t& k2) {
  if constexpr (DT == DT_F64) {
    uint64_t kx = kw(xh, xl), ky = kw(yh, yl);
    switch (e) {
      case 0: k1 = kx; k2 = ky; break;
      case 1: k1 = ky; k2 = kx; break;
      case 2: k1 = ~kx; k2 = ~ky; break;
      default: k1 = ~ky; k2 = ~kx; break;
    }
  } else {
    switch (e) {
      case 0: k1 = kw(xh, yh); break;
      case 1: k1 = kw(yh, xh); break;
      case 2: k1 = kw(~xh, ~yh); break;
      default: k1 = kw(~yh, ~xh); break;
    }
    k2 = 0;
  }
}

// Key words of one point (int32: one word per coordinate, low words 0).
template <int DT>
__device__ __forceinline__ void a1_words(const typename PointT<DT>::T& p, uint32_t& xh, uint32_t& xl,
                                         uint32_t& yh, uint32_t& yl, uint32_t& amin) {
  if constexpr (DT == DT_F64) {
    f64_key_words((uint64_t)__double_as_longlong(p.x), xh, xl, amin);
    f64_key_words((uint64_t)__double_as_longlong(p.y), yh, yl, amin);
  } else {
    xh = (uint32_t)p.x ^ 0x80000000u;
    yh = (uint32_t)p.y ^ 0x80000000u;
    xl = yl = 0;
  }
}

// Whether a point can improve any of the four running minima: only the top
// 32 bits of each k1 are compared here; the full comparison runs in
// a1_update, which is rare (new minima, or ties of the top words).
__device__ __forceinline__ bool a1_maybe(uint32_t xh, uint32_t yh, const uint32_t th[4]) {
  return xh <= th[0] || yh <= th[1] || ~xh <= th[2] || ~yh <= th[3];
}

// Full update (indices grow within a thread: a strict order keeps the
// smallest index among equal keys).
template <int DT>
__device__ __forceinline__ void a1_update(uint32_t xh, uint32_t xl, uint32_t yh, uint32_t yl, uint32_t i,
                                          Lex best[4]) {
#pragma unroll
  for (int e = 0; e < 4; e++) {
    Lex c;
    cand_keys<DT>(xh, xl, yh, yl, e, c.k1, c.k2);
    if (c.k1 < best[e].k1 || (c.k1 == best[e].k1 && c.k2 < best[e].k2)) {
      best[e].k1 = c.k1;
      best[e].k2 = c.k2;
      best[e].idx = i;
    }
  }
}

// Thresholds shared by the warp: the smallest top word of each running
// minimum over the lanes.  A point whose top word exceeds the warp's cannot
// be the set's extreme, so only points at or below it take the full update;
// sharing the bound across the warp keeps that rare.
__device__ __forceinline__ void a1_thresholds(const Lex best[4], uint32_t th[4]) {
#pragma unroll
  for (int e = 0; e < 4; e++) th[e] = __reduce_min_sync(0xFFFFFFFFu, (uint32_t)(best[e].k1 >> 32));
}

// float64 filter on the top 32 bits of each coordinate read as an FP32
// number.  That reading is non-decreasing in the coordinate wherever it is
// not NaN and -0.0 and +0.0 compare equal; the largest magnitudes (from
// 2^1017 on) and Inf / NaN inputs read as +-Inf, ordered beyond every other
// reading, or as NaN, which the unordered tests below let through -- either
// way such a value reaches the exact update, becomes an extreme, and
// setup_set reports it.  A threshold is the top word of the warp's running bound
// turned back from key to bits: a point passes when its top word is at or
// beyond the bound's, so the exact keys still decide every tie.
__device__ __forceinline__ float a1_bound_f(uint32_t keyhi) {
  const uint32_t raw = (keyhi & 0x80000000u) ? (keyhi ^ 0x80000000u) : ~keyhi;
  return __uint_as_float(raw);
}
__device__ __forceinline__ void a1_thresholds_f(const Lex best[4], float thf[4]) {
#pragma unroll
  for (int e = 0; e < 4; e++) {
    const uint32_t t = __reduce_min_sync(0xFFFFFFFFu, (uint32_t)(best[e].k1 >> 32));
    thf[e] = a1_bound_f(e >= 2 ? ~t : t);
  }
}

// Bucket of the stairs map: monotone non-decreasing in u.
__device__ __forceinline__ int stair_bucket(float u, float lo, float scale) {
  float t = __fmul_rn(__fsub_rn(u, lo), scale);
  int b = __float2int_rd(t);
  return min(max(b, 0), kStairB - 1);
}

// Order-preserving unsigned key of a (non-NaN) float.
__device__ __forceinline__ uint32_t f32_order(float f) {
  const uint32_t u = __float_as_uint(f);
  return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}

// FP32 view of a point used by the filter and the stairs (truncated float64,
// rounded int32): monotone in each coordinate.  A float32 input is its own
// view (view_at reads it from the vectors).
template <int DT>
__device__ __forceinline__ void f32_view(const typename PointT<DT>::T& p, float& X, float& Y) {
  static_assert(DT != DT_F32, "float32 views come from view_at");
  if constexpr (DT == DT_F64) {
    X = f64_trunc_f32((uint64_t)__double_as_longlong(p.x));
    Y = f64_trunc_f32((uint64_t)__double_as_longlong(p.y));
  } else {
    X = __int2float_rn(p.x);
    Y = __int2float_rn(p.y);
  }
}

// FP32 view of input point i (set offset included).
template <int DT>
__device__ __forceinline__ void view_at(const Job& j, int64_t i, float& X, float& Y) {
  if constexpr (DT == DT_F32) {
    X = reinterpret_cast<const float*>(j.pts)[i];
    Y = j.ys[i];
  } else {
    f32_view<DT>(input_point<typename PointT<DT>::T>(j, i), X, Y);
  }
}

// The same FP32 view in three integer operations per coordinate, for sets
// whose coordinates all have magnitude in [2^-126, 2^60] (SF_SHORTVIEW): the
// exponent is rebiased on the signed top word (no borrow reaches the sign:
// the magnitude's top word is at least 0x38100000) and shifted with the three
// leading bits of the low word; the bits equal f64_trunc_f32's.
__device__ __forceinline__ float f64_view_short(uint64_t b) {
  const uint32_t hi = (uint32_t)(b >> 32), lo = (uint32_t)b;
  const uint32_t t = hi - 0x38000000u;
  return __uint_as_float(__funnelshift_l(lo, t, 3) | (hi & 0x80000000u));
}
template <int DT, bool SHORT>
__device__ __forceinline__ void f32_view_a2(const typename PointT<DT>::T& p, float& X, float& Y) {
  if constexpr (DT == DT_F64 && SHORT) {
    X = f64_view_short((uint64_t)__double_as_longlong(p.x));
    Y = f64_view_short((uint64_t)__double_as_longlong(p.y));
  } else {
    f32_view<DT>(p, X, Y);
  }
}

// Compared coordinate of region r (0..3) as the order word of its FP32 view
// in "smaller is better" form: R1 y, R2 -x, R3 -y, R4 x (-0.0 read as +0.0).
// The view is non-decreasing in the coordinate, so a strictly larger word
// means a strictly worse coordinate: the dominance tables hold these words.
__device__ __forceinline__ uint32_t cmp_view_order(float X, float Y, int r) {
  const float v = (r & 1) ? X : Y;
  return f32_order(__fadd_rn((r == 1 || r == 2) ? -v : v, 0.0f));
}

// Sort coordinate (FP32 view) of region r: R1 x asc, R2 y asc, R3 x desc, R4 y desc.
__device__ __forceinline__ float sort_u(float X, float Y, int r) {
  switch (r) {
    case 0: return X;
    case 1: return Y;
    case 2: return -X;
    default: return -Y;
  }
}

// FP32 filter of the directed edge a -> b (see setup_set): coefficients of
// orient(a, b, p) = A py - B px + C and the bound E on its FP32 evaluation
// error; a degenerate edge (a = b) is always "inside", without the filter
// (filt false) nothing is.
__device__ void edge_filter(double ax, double ay, double bx, double by, double xm, double ym, bool filt,
                            float& fA, float& fB, float& fC, float& fE) {
  const double u = 5.9604644775390625e-08;
  if (!filt) {
    fA = 0.f; fB = 0.f; fC = 0.f; fE = __int_as_float(0x7F800000);
  } else if (ax == bx && ay == by) {
    fA = 0.f; fB = 0.f; fC = 1.f; fE = 0.f;
  } else {
    double A = bx - ax, B = by - ay;
    double C = B * ax - A * ay;
    double Mc = fabs(B) * fabs(ax) + fabs(A) * fabs(ay);
    double E = 6.0 * u * (fabs(A) * ym + fabs(B) * xm + Mc)
             + (fabs(A) + fabs(B)) * 2.350988701644575e-38      // 2^-125
             + 3.5032461608120427e-45 * (xm + ym + 1.0);        // 2^-147
    fA = __double2float_rn(A);
    fB = __double2float_rn(B);
    fC = __double2float_rn(C);
    fE = __double2float_ru(E);
  }
}

// Edge set-up of one set once E1..E4 are known, run by one warp (every lane
// holds the set's extremes): lane k < 4 loads E_k, sets up edge k (octagon
// mode: finds D_k, and lane k < 8 sets up octagon edge k) and region k's
// stairs range; the flags, the same in every lane, are written by lane 0.
template <int DT>
__device__ void setup_set_warp(const Job& j, const Ws& w, int s, const SetDesc& sd, const Lex best[4],
                               uint32_t amin, uint32_t lomag, const uint64_t* dq) {
  SetCtl& c = w.ctl[s];
  using P = typename PointT<DT>::T;
  const int lane = threadIdx.x & 31;
  const int k1 = (lane + 1) & 3;
  const uint32_t myidx = lane == 0 ? best[0].idx : lane == 1 ? best[1].idx : lane == 2 ? best[2].idx : best[3].idx;
  P my{};
  if (lane < 4) my = input_point<P>(j, sd.off + myidx);
  P e[4];
#pragma unroll
  for (int k = 0; k < 4; k++) {
    e[k].x = __shfl_sync(0xFFFFFFFFu, my.x, k);
    e[k].y = __shfl_sync(0xFFFFFFFFu, my.y, k);
  }
  P nb;                                    // E_{k+1} on lane k
  nb.x = __shfl_sync(0xFFFFFFFFu, my.x, k1);
  nb.y = __shfl_sync(0xFFFFFFFFu, my.y, k1);
  if (lane == 0) {
    for (int k = 0; k < 4; k++) {
      c.ek1[k] = best[k].k1;
      c.ek2[k] = best[k].k2;
      c.eidx[k] = best[k].idx;
      c.ex[k] = (double)e[k].x;
      c.ey[k] = (double)e[k].y;
    }
  }
  uint32_t flags = 0;
  if constexpr (DT != DT_I32) {
    // NaN, Inf and huge values sort beyond every finite value, so they show
    // up among the extremes; tiny nonzero values were folded into amin.
    int st = 0;
    for (int k = 0; k < 4; k++) {
      for (int q = 0; q < 2; q++) {
        uint64_t b = (uint64_t)__double_as_longlong(q ? e[k].y : e[k].x);
        uint32_t ex = (uint32_t)(b >> 52) & 0x7FFu;
        if (ex == 0x7FFu) st = ST_NONFINITE;
        else if (ex > 1023u + 399u && st == 0) st = ST_RANGE;
      }
    }
    if (st == 0 && amin < ((1023u - 400u) << 20)) st = ST_RANGE;
    if (st) {
      if (lane == 0) c.status = st;
      return;
    }
  }
  for (int k = 0; k < 4; k++)
    if (best[k].idx == best[(k + 1) & 3].idx) flags |= SF_DEGEN0 << k;
  bool small = true;
  // E1 = P_minx, E3 = P_maxx, E2 = P_miny, E4 = P_maxy
  const double xm = fmax(fabs((double)e[0].x), fabs((double)e[2].x));
  const double ym = fmax(fabs((double)e[1].y), fabs((double)e[3].y));
  if constexpr (DT == DT_I32) {
    double spanx = (double)e[2].x - (double)e[0].x, spany = (double)e[3].y - (double)e[1].y;
    if (spanx >= 2147483648.0 || spany >= 2147483648.0) flags |= SF_WIDE;
  } else {
    const double lim = 1152921504606846976.0;  // 2^60
    small = xm <= lim && ym <= lim;
    if (small) flags |= SF_SMALL;
    // every coordinate of magnitude in [2^-126, 2^60]: the short FP32 view
    // (f32_view_short) equals f64_trunc_f32
    if (DT == DT_F64 && small && lomag >= kTinyTopBits) flags |= SF_SHORTVIEW;
  }
  const bool filt = small && !(j.opts & OPT_NO_FILTER);
  if (filt) flags |= SF_FILTER;
  // orient(a, b, p) = A py - B px + C with A = bx-ax, B = by-ay,
  // C = B ax - A ay.  The FP32 evaluation fma(A, Y, fma(-B, X, C)) on the
  // FP32 views X, Y (float64: significand-truncated, |X - x| < 2^-23 |x|;
  // int32: rounded to nearest, |X - x| <= 2^-24 |x|; float32: exact)
  // differs from the exact value by at most 5.01 u (|A| Ymax + |B| Xmax +
  // |B||ax| + |A||ay|) plus underflow terms, u = 2^-24; E below uses 6 u and
  // rounds up.  Without the filter every point takes the exact path
  // (E = inf); a degenerate edge is always "inside" (A = B = 0, C = 1, E = 0).
  if (lane < 4)
    edge_filter((double)my.x, (double)my.y, (double)nb.x, (double)nb.y, xm, ym, filt, c.fA[lane], c.fB[lane],
                c.fC[lane], c.fE[lane]);
  if (dq) {
    // Octagon (OPT_OCTAGON): vertex 2r is E_r, vertex 2r+1 the diagonal
    // extreme D_r when it lies strictly outside edge r (exact test), else
    // E_{r+1} (the edge D_r -> E_{r+1} is then degenerate).  Each kept D_r
    // is the extreme of its direction among the set's FP32 scores, so the
    // eight vertices in this order form a convex polygon inside the hull.
    double dx = (double)nb.x, dy = (double)nb.y;
    if (lane < 4) {
      const uint64_t dqr = dq[lane];
      int32_t didx = -1;
      if (!(flags & (SF_DEGEN0 << lane)) && dqr != ~0ull) {
        const uint32_t di = (uint32_t)dqr;
        const P d = input_point<P>(j, sd.off + di);
        int o;
        if constexpr (DT != DT_I32) o = orient_f64((double)my.x, (double)my.y, (double)nb.x, (double)nb.y, d.x, d.y);
        else o = orient_i32(my.x, my.y, nb.x, nb.y, d.x, d.y, true);
        if (o < 0) { dx = (double)d.x; dy = (double)d.y; didx = (int32_t)di; }
      }
      c.ovx[2 * lane] = (double)my.x;
      c.ovy[2 * lane] = (double)my.y;
      c.ovx[2 * lane + 1] = dx;
      c.ovy[2 * lane + 1] = dy;
      c.didx[lane] = didx;
    }
    // octagon edge k on lane k < 8: vertices k and k + 1 (vertex v is E_{v/2}
    // for even v, lane (v-1)/2's D for odd v)
    const int v0 = lane & 7, v1 = (lane + 1) & 7;
    const double ex0 = __shfl_sync(0xFFFFFFFFu, (double)my.x, v0 >> 1), ey0 = __shfl_sync(0xFFFFFFFFu, (double)my.y, v0 >> 1);
    const double dx0 = __shfl_sync(0xFFFFFFFFu, dx, v0 >> 1), dy0 = __shfl_sync(0xFFFFFFFFu, dy, v0 >> 1);
    const double ex1 = __shfl_sync(0xFFFFFFFFu, (double)my.x, v1 >> 1), ey1 = __shfl_sync(0xFFFFFFFFu, (double)my.y, v1 >> 1);
    const double dx1 = __shfl_sync(0xFFFFFFFFu, dx, v1 >> 1), dy1 = __shfl_sync(0xFFFFFFFFu, dy, v1 >> 1);
    if (lane < 8)
      edge_filter((v0 & 1) ? dx0 : ex0, (v0 & 1) ? dy0 : ey0, (v1 & 1) ? dx1 : ex1, (v1 & 1) ? dy1 : ey1, xm, ym,
                  filt, c.oA[lane], c.oB[lane], c.oC[lane], c.oE[lane]);
  }
  if (small && !(j.opts & OPT_NO_PREFILTER)) {
    flags |= SF_STAIRS;
    float X = 0.f, Y = 0.f;
    if (lane < 4) {
      if constexpr (DT == DT_F32) view_at<DT>(j, sd.off + myidx, X, Y);
      else f32_view<DT>(my, X, Y);
    }
    const float Xn = __shfl_sync(0xFFFFFFFFu, X, k1), Yn = __shfl_sync(0xFFFFFFFFu, Y, k1);
    // region r (lane r) runs from E_r to E_{r+1} along its sort coordinate
    if (lane < 4) {
      const float lo = sort_u(X, Y, lane), hi = sort_u(Xn, Yn, lane);
      c.slo[lane] = lo;
      c.shi[lane] = hi;
      c.sscale[lane] = hi > lo ? (float)kStairB / (hi - lo) : 0.f;
    }
  }
  if (lane == 0) c.flags = flags;
}

constexpr int kExtStages = 3;                          // TMA ring depth of a1
constexpr int kExtBlock = (kClsConsumers + 1) * 32;    // 8 consumer warps + a producer warp
constexpr int kExtTileBytes = 32768;                    // a1 tiles: 2048 float64 / 4096 int32 or float32 points
constexpr int kExtSmem = kExtStages * (kExtTileBytes + 32);

// Stage of a TMA ring: 16 bytes of slack, then the tile's points; float32
// input: the x half, 16 bytes of slack, the y half (`half` bytes from the
// stage start).
//
// Producer side of one tile: points [i0, i0 + np) of the input (set offset
// included) into `stage`, the bytes counted on `bar`.  Bulk copies want
// 16-byte aligned addresses and sizes, so the points before the first and
// after the last 16-byte boundary of a vector (int32: at most one each;
// float32: at most three each, per vector; float64: none, its input is
// 16-byte aligned) go by plain loads into the slack and the tile's ends.
// The number of leading points so moved (float32: x | y << 8) goes to
// *lead before the arrive that can complete the stage (a tile without bulk
// bytes completes on it): the consumers index the tile from 16 - that many
// points into the stage.  `keep` drops the evict-first hint.
__device__ __forceinline__ int f32_vec_part(const float* src, int np, unsigned char* dst, uint32_t& bytes,
                                            const float*& body) {
  const int mis = (int)(((uintptr_t)src >> 2) & 3u);
  const int head = min(mis ? 4 - mis : 0, np);
  const int rem = np - head;
  const int tail = rem & 3;
  float* d = reinterpret_cast<float*>(dst);
  for (int t = 0; t < head; t++) d[t - head] = src[t];
  for (int t = rem - tail; t < rem; t++) d[t] = src[head + t];
  bytes = (uint32_t)(rem - tail) * 4u;
  body = src + head;
  return head;
}

template <int DT>
__device__ __forceinline__ void stage_tile(const Job& j, int64_t i0, int np, unsigned char* stage, int half,
                                           uint64_t* bar, bool keep, int* lead) {
  if constexpr (DT == DT_F32) {
    const float *bx, *by;
    uint32_t nx, ny;
    const int hx = f32_vec_part(reinterpret_cast<const float*>(j.pts) + i0, np, stage + 16, nx, bx);
    const int hy = f32_vec_part(j.ys + i0, np, stage + half + 16, ny, by);
    *lead = hx | (hy << 8);
    mbar_arrive_tx(bar, nx + ny);
    if (nx) {
      if (keep) tma_load_1d(stage + 16, bx, nx, bar);
      else tma_load_1d_stream(stage + 16, bx, nx, bar);
    }
    if (ny) {
      if (keep) tma_load_1d(stage + half + 16, by, ny, bar);
      else tma_load_1d_stream(stage + half + 16, by, ny, bar);
    }
  } else {
    constexpr int PB = in_bytes<DT>();
    const char* src = reinterpret_cast<const char*>(j.pts) + i0 * PB;
    unsigned char* dst = stage + 16;
    int head = 0, tail = 0;
    if constexpr (DT == DT_I32) {
      head = ((uintptr_t)src & 15) ? 1 : 0;
      tail = (((np - head) * PB) & 15) ? 1 : 0;
      if (head) *reinterpret_cast<uint2*>(dst - PB) = *reinterpret_cast<const uint2*>(src);
      if (tail)
        *reinterpret_cast<uint2*>(dst + (np - 1 - head) * PB) = *reinterpret_cast<const uint2*>(src + (size_t)(np - 1) * PB);
    }
    const uint32_t bytes = (uint32_t)(np - head - tail) * PB;
    *lead = head;
    mbar_arrive_tx(bar, bytes);
    if (bytes) {
      if (keep) tma_load_1d(dst, src + head * PB, bytes, bar);
      else tma_load_1d_stream(dst, src + head * PB, bytes, bar);
    }
  }
}

// Barrier of the consumer warps only (the producer warp has left).
__device__ __forceinline__ void consumers_sync() {
  asm volatile("bar.sync 1, %0;" :: "r"(kClsConsumers * 32) : "memory");
}

// a1.  nchunk1 CTAs per set; CTA k takes the set's tiles k, k + nchunk1,
// k + 2 nchunk1, ... (all CTAs read close together in memory).  Warp 8
// streams them through a ring of shared-memory stages with 1-D TMA bulk
// copies (full/empty mbarriers); warps 0..7 each scan a contiguous eighth of
// every tile, so every thread meets its points in increasing index order.
// Diagonal extremes of the octagon mode (OPT_OCTAGON): per direction the
// point with the smallest FP32 score of its views -- lower left X + Y, lower
// right Y - X, upper right -X - Y, upper left X - Y -- ties to the smallest
// index, as (order word of the score) << 32 | index.  Any input point is a
// valid octagon vertex; the set-up keeps it only where it is strictly
// outside the quadrilateral's edge.
__device__ __forceinline__ void oct_update(uint64_t dq[4], float X, float Y, uint32_t i) {
  dq[0] = min(dq[0], ((uint64_t)f32_order(__fadd_rn(X, Y)) << 32) | i);
  dq[1] = min(dq[1], ((uint64_t)f32_order(__fsub_rn(Y, X)) << 32) | i);
  dq[2] = min(dq[2], ((uint64_t)f32_order(-__fadd_rn(X, Y)) << 32) | i);
  dq[3] = min(dq[3], ((uint64_t)f32_order(__fsub_rn(X, Y)) << 32) | i);
}

// Minimum / maximum that return NaN when either operand is NaN, so that a
// NaN coordinate shows up in a lane's running extremes.
__device__ __forceinline__ float fmin_nan(float a, float b) {
  float d;
  asm("min.NaN.f32 %0, %1, %2;" : "=f"(d) : "f"(a), "f"(b));
  return d;
}
__device__ __forceinline__ float fmax_nan(float a, float b) {
  float d;
  asm("max.NaN.f32 %0, %1, %2;" : "=f"(d) : "f"(a), "f"(b));
  return d;
}

template <int DT, bool OCT>
__global__ void __launch_bounds__(kExtBlock, 2) k_extremes(Job j, Ws w) {
  griddep_enter();
  using P = typename PointT<DT>::T;
  constexpr int PB = in_bytes<DT>();
  constexpr int TILE = kExtTileBytes / PB;
  constexpr int WPTS = TILE / kClsConsumers;
  constexpr int IW = WPTS / 32;
  constexpr int SB = kExtTileBytes + (DT == DT_F32 ? 32 : 16);
  constexpr int HALF = kExtTileBytes / 2 + 16;
  static_assert(SB * kExtStages <= kExtSmem, "a1 ring fits its allocation");
  extern __shared__ __align__(128) unsigned char smem[];
  __shared__ __align__(8) uint64_t full[kExtStages], empty[kExtStages];
  __shared__ int st_head[kExtStages];
  __shared__ Lex red[kClsConsumers][4];
  __shared__ uint32_t red_amin[kClsConsumers], red_lomag[kClsConsumers];
  __shared__ uint64_t red_dq[kClsConsumers][4];
  __shared__ int last;

  const int chunk = blockIdx.x;
  int s = 0;
  if (j.sets) {
    int lo = 0, hi = j.nsets - 1;
    while (lo < hi) {
      int mid = (lo + hi + 1) >> 1;
      if (j.sets[mid].chunk1 <= chunk) lo = mid; else hi = mid - 1;
    }
    s = lo;
  }
  const SetDesc sd = get_set(j, s);
  const int64_t tiles_set = (sd.n + TILE - 1) / TILE;
  const int64_t k0 = chunk - sd.chunk1, kstep = sd.nchunk1;
  const int ntile = k0 < tiles_set ? (int)((tiles_set - k0 + kstep - 1) / kstep) : 0;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  if (tid == 0) {
    for (int q = 0; q < kExtStages; q++) { mbar_init(&full[q], 1); mbar_init(&empty[q], kClsConsumers); }
    fence_mbar_init();
    fence_async_smem();
  }
  __syncthreads();

  if (warp == kClsConsumers) {
    // ---------------------------------------------------------- producer
    if (lane != 0) return;
    int issued = 0;
    bool ok = true;
    for (int it = 0; it < ntile; it++) {
      const int slot = it % kExtStages;
      if (it >= kExtStages) {
        uint32_t spins = 0;
        while (!mbar_try_wait(&empty[slot], (uint32_t)((it / kExtStages) - 1) & 1u))
          if (!spin_step(spins, w.ctr)) { ok = false; break; }
        if (!ok) break;
        fence_async_smem();
      }
      const int64_t i0 = (k0 + (int64_t)it * kstep) * TILE;
      const int np = (int)min((int64_t)TILE, sd.n - i0);
      stage_tile<DT>(j, sd.off + i0, np, smem + slot * SB, HALF, &full[slot], (sd.n - i0) * PB <= kL2KeepBytes,
                     &st_head[slot]);
      issued = it + 1;
    }
    // every tile is in flight: k_stairs may be scheduled (it reads none of
    // a1's results before its griddep_enter)
    griddep_release();
    if (!ok) {
      // a wait ran out: let the copies already issued land before exiting
      for (int it = max(0, issued - kExtStages); it < issued; it++) {
        uint32_t spins = 0;
        while (!mbar_try_wait(&full[it % kExtStages], (uint32_t)(it / kExtStages) & 1u))
          if (!spin_step(spins, w.ctr) && spins > kSpinLimit) break;
      }
    }
    return;
  }

  // ------------------------------------------------------------ consumers
  Lex best[4];
  uint32_t th[4];
  float thf[4];
#pragma unroll
  for (int k = 0; k < 4; k++) { best[k].k1 = ~0ull; best[k].k2 = ~0ull; best[k].idx = 0xFFFFFFFFu; th[k] = 0xFFFFFFFFu; }
  a1_thresholds_f(best, thf);
  uint32_t amin = 0x7FFFFFFFu;      // smallest top-word magnitude of a nonzero coordinate
  uint32_t lomag = 0x7FFFFFFFu;     // the same over every coordinate, zeros included (float64)
  uint64_t dqm[4] = {~0ull, ~0ull, ~0ull, ~0ull};   // OCT: diagonal extremes
  // set-local indices fit in 32 bits (n <= 2^30)
  for (int it = 0; it < ntile; it++) {
    const int slot = it % kExtStages;
    {
      uint32_t spins = 0;
      bool ok = true;
      while (!mbar_try_wait(&full[slot], (uint32_t)(it / kExtStages) & 1u))
        if (!spin_step(spins, w.ctr)) { ok = false; break; }
      if (!ok) break;
    }
    const int64_t t0 = (k0 + (int64_t)it * kstep) * TILE;
    const uint32_t i0 = (uint32_t)t0;
    const int np = (int)min((int64_t)TILE, sd.n - t0);
    const unsigned char* base = smem + slot * SB + 16 - st_head[slot] * PB;
    const int wb = warp * WPTS;
    if constexpr (!OCT && DT != DT_I32) {
      // Each lane first folds its items into running FP32 extremes (float64:
      // the top word read as FP32, the order of the filter below; float32:
      // the values), plus the smallest top-word magnitude (float64).  Only a
      // warp in which some lane's extremes reach the running bounds (ties and
      // NaN included), or in which a magnitude is tiny, rescans its items
      // with the exact keys: after the first tiles that is rare, so most
      // points cost one load and four min / max operations.
      const float* vx = reinterpret_cast<const float*>(smem + slot * SB + 16) - (st_head[slot] & 0xFF);
      const float* vy = reinterpret_cast<const float*>(smem + slot * SB + HALF + 16) - (st_head[slot] >> 8);
      const float inf = __int_as_float(0x7F800000);
      float mnx = inf, mny = inf, mxx = -inf, mxy = -inf, tmn = inf;
#pragma unroll
      for (int k = 0; k < IW; k++) {
        const int i = wb + k * 32 + lane;
        if (i < np) {
          float fx, fy;
          if constexpr (DT == DT_F64) {
            const uint4 q = *reinterpret_cast<const uint4*>(base + i * PB);
            fx = __uint_as_float(q.y);
            fy = __uint_as_float(q.w);
            tmn = fmin_nan(tmn, fmin_nan(fabsf(fx), fabsf(fy)));
          } else {
            fx = vx[i];
            fy = vy[i];
          }
          mnx = fmin_nan(mnx, fx);
          mny = fmin_nan(mny, fy);
          mxx = fmax_nan(mxx, fx);
          mxy = fmax_nan(mxy, fy);
        }
      }
      bool rare = !(mnx > thf[0]) | !(mny > thf[1]) | !(mxx < thf[2]) | !(mxy < thf[3]);
      if constexpr (DT == DT_F64) rare |= !(tmn >= kTinyTopF);
      if (__any_sync(0xFFFFFFFFu, rare)) {
        // the stage is still held: rescan the items
#pragma unroll 1
        for (int k = 0; k < IW; k++) {
          const int i = wb + k * 32 + lane;
          if (i >= np) continue;
          if constexpr (DT == DT_F64) {
            const uint4 q = *reinterpret_cast<const uint4*>(base + i * PB);
            const float fx = __uint_as_float(q.y), fy = __uint_as_float(q.w);
            if ((fabsf(fx) < kTinyTopF) | (fabsf(fy) < kTinyTopF)) {
              // zeros and tiny magnitudes: the exact lower end of the domain check
              uint32_t a = q.y & 0x7FFFFFFFu;
              if ((a | q.x) != 0) amin = min(amin, a);
              lomag = min(lomag, a);
              a = q.w & 0x7FFFFFFFu;
              if ((a | q.z) != 0) amin = min(amin, a);
              lomag = min(lomag, a);
            }
            if (!(fx > thf[0]) | !(fy > thf[1]) | !(fx < thf[2]) | !(fy < thf[3])) {
              uint32_t kxh, kxl, kyh, kyl, dummy = 0;
              f64_key_words(((uint64_t)q.y << 32) | q.x, kxh, kxl, dummy);
              f64_key_words(((uint64_t)q.w << 32) | q.z, kyh, kyl, dummy);
              a1_update<DT>(kxh, kxl, kyh, kyl, i0 + (uint32_t)i, best);
            }
          } else {
            const float X = vx[i], Y = vy[i];
            if (!(X > thf[0]) | !(Y > thf[1]) | !(X < thf[2]) | !(Y < thf[3]))
              a1_update<DT>(key_f32(X), 0u, key_f32(Y), 0u, i0 + (uint32_t)i, best);
          }
        }
        a1_thresholds_f(best, thf);
      }
      __syncwarp();
      if (lane == 0)   // the warp is done with the stage: release it to the producer
        asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" :: "r"(smem_addr(&empty[slot])) : "memory");
      continue;
    } else if constexpr (DT == DT_F32) {
      // octagon mode: exact 32-bit keys of the two vectors, as for int32
      const float* vx = reinterpret_cast<const float*>(smem + slot * SB + 16) - (st_head[slot] & 0xFF);
      const float* vy = reinterpret_cast<const float*>(smem + slot * SB + HALF + 16) - (st_head[slot] >> 8);
      uint32_t xh[IW], yh[IW];
      bool need = false;
#pragma unroll
      for (int k = 0; k < IW; k++) {
        const int i = wb + k * 32 + lane;
        if (i < np) {
          const float X = vx[i], Y = vy[i];
          xh[k] = key_f32(X);
          yh[k] = key_f32(Y);
          if constexpr (OCT) oct_update(dqm, X, Y, i0 + (uint32_t)i);
          need |= a1_maybe(xh[k], yh[k], th);
        } else {
          xh[k] = yh[k] = 0xFFFFFFFFu;
        }
      }
      __syncwarp();
      if (lane == 0)   // the warp is done with the stage: release it to the producer
        asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" :: "r"(smem_addr(&empty[slot])) : "memory");
      if (__any_sync(0xFFFFFFFFu, need)) {
#pragma unroll
        for (int k = 0; k < IW; k++) {
          const int i = wb + k * 32 + lane;
          if (i < np && a1_maybe(xh[k], yh[k], th)) a1_update<DT>(xh[k], 0u, yh[k], 0u, i0 + i, best);
        }
        a1_thresholds(best, th);
      }
      continue;
    } else if constexpr (DT == DT_F64) {
      // raw words; the filter and the small-magnitude test in FP32 on the
      // top words, the exact key work only where they fire
      uint32_t xh[IW], xl[IW], yh[IW], yl[IW];
      uint32_t passm = 0, tinym = 0;
#pragma unroll
      for (int k = 0; k < IW; k++) {
        const int i = wb + k * 32 + lane;
        if (i < np) {
          const uint4 q = *reinterpret_cast<const uint4*>(base + i * PB);
          xl[k] = q.x; xh[k] = q.y; yl[k] = q.z; yh[k] = q.w;
          if constexpr (OCT)
            oct_update(dqm, f64_trunc_f32(((uint64_t)q.y << 32) | q.x), f64_trunc_f32(((uint64_t)q.w << 32) | q.z),
                       i0 + (uint32_t)i);
          const float fx = __uint_as_float(q.y), fy = __uint_as_float(q.w);
          const bool pass = !(fx > thf[0]) | !(fy > thf[1]) | !(fx < thf[2]) | !(fy < thf[3]);
          const bool tiny = (fabsf(fx) < kTinyTopF) | (fabsf(fy) < kTinyTopF);
          passm |= (uint32_t)pass << k;
          tinym |= (uint32_t)tiny << k;
        } else {
          xh[k] = yh[k] = xl[k] = yl[k] = 0u;
        }
      }
      __syncwarp();
      if (lane == 0)   // the warp is done with the stage: release it to the producer
        asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" :: "r"(smem_addr(&empty[slot])) : "memory");
      // rare: zeros and tiny magnitudes (the exact lower end of the domain check)
      if (__any_sync(0xFFFFFFFFu, tinym != 0)) {
#pragma unroll
        for (int k = 0; k < IW; k++) {
          if ((tinym >> k) & 1u) {
            uint32_t a = xh[k] & 0x7FFFFFFFu;
            if ((a | xl[k]) != 0) amin = min(amin, a);
            lomag = min(lomag, a);
            a = yh[k] & 0x7FFFFFFFu;
            if ((a | yl[k]) != 0) amin = min(amin, a);
            lomag = min(lomag, a);
          }
        }
      }
      // rare: a warp-uniform branch keeps the full update out of the hot path
      if (__any_sync(0xFFFFFFFFu, passm != 0)) {
#pragma unroll
        for (int k = 0; k < IW; k++) {
          if ((passm >> k) & 1u) {
            uint32_t kxh, kxl, kyh, kyl, dummy = 0;
            f64_key_words(((uint64_t)xh[k] << 32) | xl[k], kxh, kxl, dummy);
            f64_key_words(((uint64_t)yh[k] << 32) | yl[k], kyh, kyl, dummy);
            a1_update<DT>(kxh, kxl, kyh, kyl, i0 + wb + k * 32 + lane, best);
          }
        }
        a1_thresholds_f(best, thf);
      }
      continue;
    } else {
      uint32_t xh[IW], xl[IW], yh[IW], yl[IW];
      bool need = false;
#pragma unroll
      for (int k = 0; k < IW; k++) {
        const int i = wb + k * 32 + lane;
        if (i < np) {
          const P p = *reinterpret_cast<const P*>(base + i * PB);
          a1_words<DT>(p, xh[k], xl[k], yh[k], yl[k], amin);
          if constexpr (OCT) {
            float X, Y;
            f32_view<DT>(p, X, Y);
            oct_update(dqm, X, Y, i0 + (uint32_t)i);
          }
          need |= a1_maybe(xh[k], yh[k], th);
        } else {
          xh[k] = yh[k] = 0xFFFFFFFFu;
          xl[k] = yl[k] = 0u;
        }
      }
      __syncwarp();
      if (lane == 0)   // the warp is done with the stage: release it to the producer
        asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" :: "r"(smem_addr(&empty[slot])) : "memory");
      // rare: a warp-uniform branch keeps the full update out of the hot path
      if (__any_sync(0xFFFFFFFFu, need)) {
#pragma unroll
        for (int k = 0; k < IW; k++) {
          const int i = wb + k * 32 + lane;
          if (i < np && a1_maybe(xh[k], yh[k], th)) a1_update<DT>(xh[k], xl[k], yh[k], yl[k], i0 + i, best);
        }
        a1_thresholds(best, th);
      }
    }
  }

  // the tile loops are done: k_stairs may be scheduled (it reads none of a1's
  // results before its griddep_enter)
  griddep_release();

  // reduction over the consumer warps, then over the warps' results in warp 0
  auto warp_reduce = [&]() {
#pragma unroll
    for (int k = 0; k < 4; k++) best[k] = lex_warp_min(best[k]);
    amin = __reduce_min_sync(0xFFFFFFFFu, amin);
    lomag = __reduce_min_sync(0xFFFFFFFFu, lomag);
    if constexpr (OCT) {
#pragma unroll
      for (int q = 0; q < 4; q++) dqm[q] = u64_warp_min(dqm[q]);
    }
  };
  auto warp0_gather = [&]() {
#pragma unroll
    for (int k = 0; k < 4; k++) {
      if (lane < kClsConsumers) best[k] = red[lane][k];
      else { best[k].k1 = ~0ull; best[k].k2 = ~0ull; best[k].idx = 0xFFFFFFFFu; }
    }
    amin = lane < kClsConsumers ? red_amin[lane] : 0x7FFFFFFFu;
    lomag = lane < kClsConsumers ? red_lomag[lane] : 0x7FFFFFFFu;
#pragma unroll
    for (int q = 0; q < 4; q++) dqm[q] = lane < kClsConsumers ? red_dq[lane][q] : ~0ull;
  };
  warp_reduce();
  if (lane == 0) {
#pragma unroll
    for (int k = 0; k < 4; k++) red[warp][k] = best[k];
    red_amin[warp] = amin;
    red_lomag[warp] = lomag;
#pragma unroll
    for (int q = 0; q < 4; q++) red_dq[warp][q] = dqm[q];
  }
  consumers_sync();
  if (warp == 0) {
    warp0_gather();
    warp_reduce();
  }
  if (tid == 0) {
    Part& pt = w.part[chunk];
    for (int k = 0; k < 4; k++) { pt.k1[k] = best[k].k1; pt.k2[k] = best[k].k2; pt.idx[k] = best[k].idx; }
    pt.bad = amin;
    pt.lomag = lomag;
    for (int k = 0; k < 4; k++) pt.dq[k] = dqm[k];
    __threadfence();
    last = atomicAdd(&w.ctl[s].arrive1, 1u) == (uint32_t)(sd.nchunk1 - 1);
  }
  consumers_sync();
  if (!last) return;

  // Last chunk of the set: reduce the set's partials, then warp 0 sets up
  // the set's edges while the other warps clear its sort histogram and
  // stairs table.
  __threadfence();
#pragma unroll
  for (int k = 0; k < 4; k++) { best[k].k1 = ~0ull; best[k].k2 = ~0ull; best[k].idx = 0xFFFFFFFFu; }
  amin = 0x7FFFFFFFu;
  lomag = 0x7FFFFFFFu;
  for (int k = 0; k < 4; k++) dqm[k] = ~0ull;
  auto fold = [&](const Part& pt) {
#pragma unroll
    for (int k = 0; k < 4; k++) {
      Lex v{pt.k1[k], pt.k2[k], pt.idx[k]};
      lex_min_into(best[k], v);
    }
    amin = min(amin, pt.bad);
    lomag = min(lomag, pt.lomag);
    if constexpr (OCT)
      for (int k = 0; k < 4; k++) dqm[k] = min(dqm[k], pt.dq[k]);
  };
  for (int q = threadIdx.x; q < sd.nchunk1; q += kClsConsumers * 32) fold(w.part[sd.chunk1 + q]);
  warp_reduce();
  consumers_sync();
  if (lane == 0) {
#pragma unroll
    for (int k = 0; k < 4; k++) red[warp][k] = best[k];
    red_amin[warp] = amin;
    red_lomag[warp] = lomag;
#pragma unroll
    for (int q = 0; q < 4; q++) red_dq[warp][q] = dqm[q];
  }
  consumers_sync();
  if (warp == 0) {
    // the eight warps' results, reduced so that every lane holds the set's
    warp0_gather();
    warp_reduce();
    setup_set_warp<DT>(j, w, s, sd, best, amin, lomag, OCT ? dqm : nullptr);
  } else {
    const int t = threadIdx.x - 32, nt = (kClsConsumers - 1) * 32;
    uint32_t* hist = w.hist + (size_t)s * kSortPasses * 256;
    for (int i = t; i < kSortPasses * 256; i += nt) hist[i] = 0;
    uint32_t* stt = w.stairs + (size_t)s * 4 * kStairB;
    for (int i = t; i < 4 * kStairB; i += nt) stt[i] = 0xFFFFFFFFu;
  }
}

// ------------------------------------------------------------ stairs

// Exclusive minimum of `v` over the lower threads of the same 64-thread
// region group (threads 64r .. 64r+63, two warps); sw holds one word per
// warp.  Ends with the CTA synchronised.
__device__ __forceinline__ uint32_t region_excl_min(uint32_t v, uint32_t* sw) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  uint32_t x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t y = __shfl_up_sync(0xFFFFFFFFu, x, o);
    if (lane >= o) x = min(x, y);
  }
  if (lane == 31) sw[warp] = x;
  __syncthreads();
  uint32_t ex = __shfl_up_sync(0xFFFFFFFFu, x, 1);
  if (lane == 0) ex = 0xFFFFFFFFu;
  if (warp & 1) ex = min(ex, sw[warp - 1]);
  __syncthreads();
  return ex;
}

// The float whose order word (f32_order) is k.
__device__ __forceinline__ float f32_unorder(uint32_t k) {
  return __uint_as_float((k & 0x80000000u) ? (k ^ 0x80000000u) : ~k);
}

// Bucket of u under the map (lo, scale) of NB buckets: non-decreasing in u.
template <int NB>
__device__ __forceinline__ int bucket_of(float u, float lo, float scale) {
  const int b = __float2int_rd(__fmul_rn(__fsub_rn(u, lo), scale));
  return min(max(b, 0), NB - 1);
}

// k_stairs: the dominance table of every set from the sample.  Each CTA
// takes kStairChunk sample points (eight per thread, loaded once and held in
// registers).  Before its griddep_enter it reads only input points, so it
// runs during a1's tail (a1 releases it once its tiles are in flight): pass
// 1 finds the chunk's extent and the quadrant extremes of the dominance box,
// pass 2 keeps, per region r and bucket of the chunk's own map
// (kStairLB buckets over the extent of the region's sort coordinate u =
// sort_u), the smallest (compared word v = cmp_view_order) << 32 | (order
// word of u), and the buckets whose v is below every lower bucket's are the
// chunk's staircase steps: sample points with their exact views.  After a1
// (regions, their maps E_r -> E_{r+1}, the cleared table) each step goes
// into the set's table at its bucket of the region's map; the last CTA of
// the set turns the bucket minima into exclusive prefix minima.  A step Q in
// a lower bucket than a region-r point P and with a smaller v beats P
// strictly in both coordinates, so P is no SPA survivor; every step is a
// sample point, so which steps reach the table only changes how much the
// prefilter drops.
template <int DT>
__global__ void __launch_bounds__(kThreads, 4) k_stairs(Job j, Ws w) {
  static_assert(kThreads == 4 * 64 && kStairB == 64 * 16 && kStairLB == 64 * 8, "64 threads per region");
  static_assert(kStairChunk % kThreads == 0, "whole points per thread");
  __shared__ uint64_t lt[4][kStairLB];
  __shared__ uint32_t sw[kWarps];
  __shared__ uint32_t sred[kWarps][4];
  __shared__ uint64_t sdq[kWarps][4];
  __shared__ int sidx[4];
  __shared__ float sqx[4], sqy[4];
  __shared__ int last;
  const int chunk = blockIdx.x;
  int s = 0;
  if (j.sets) {
    int lo = 0, hi = j.nsets - 1;
    while (lo < hi) {
      int mid = (lo + hi + 1) >> 1;
      if (j.sets[mid].chunk3 <= chunk) lo = mid; else hi = mid - 1;
    }
    s = lo;
  }
  if (j.opts & OPT_NO_PREFILTER) {   // uniform; the table is unused
    griddep_enter();   // every CTA exits after a1 has completed: a2 waits for k_stairs only
    return;
  }
  const SetDesc sd = get_set(j, s);
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  for (int i = tid; i < 4 * kStairLB; i += kThreads) (&lt[0][0])[i] = ~0ull;

  const int64_t m = stairs_sample(sd.n, j.tune);
  const int64_t c0 = sd.n - m + (int64_t)(chunk - sd.chunk3) * kStairChunk;
  const int64_t c1 = min(sd.n, c0 + kStairChunk);
  // the chunk's points, U per thread, held in registers for both passes
  constexpr int U = kStairChunk / kThreads;
  float vx[U], vy[U];
#pragma unroll
  for (int u = 0; u < U; u++) {
    const int64_t i = c0 + u * kThreads + tid;
    if (i < c1) view_at<DT>(j, sd.off + i, vx[u], vy[u]);
  }
  // pass 1: the chunk's extent and the quadrant extremes (per thread an FP32
  // score and the first point reaching it; smaller is further into the
  // quadrant: lower-left x+y, lower-right y-x, upper-right -x-y, upper-left x-y)
  const float inf = __int_as_float(0x7F800000);
  float ext[4] = {inf, -inf, inf, -inf};           // min x, max x, min y, max y
  float qs[4] = {inf, inf, inf, inf};
  int qi[4] = {-1, -1, -1, -1};                    // slot u * kThreads + tid of the best point
#pragma unroll
  for (int u = 0; u < U; u++) {
    if (c0 + u * kThreads + tid >= c1) continue;
    const float X = vx[u], Y = vy[u];
    ext[0] = fminf(ext[0], X); ext[1] = fmaxf(ext[1], X);
    ext[2] = fminf(ext[2], Y); ext[3] = fmaxf(ext[3], Y);
    const float sc[4] = {__fadd_rn(X, Y), __fsub_rn(Y, X), -__fadd_rn(X, Y), __fsub_rn(X, Y)};
#pragma unroll
    for (int q = 0; q < 4; q++)
      if (sc[q] < qs[q] || (qi[q] < 0 && !(sc[q] > qs[q]))) { qs[q] = sc[q]; qi[q] = u * kThreads + tid; }
  }
  // warp minima by order words (redux); the extent ignores NaN
  uint32_t eo[4];
#pragma unroll
  for (int k = 0; k < 4; k++) {
    const uint32_t o = f32_order(ext[k]);
    eo[k] = (k & 1) ? ~__reduce_min_sync(0xFFFFFFFFu, ~o) : __reduce_min_sync(0xFFFFFFFFu, o);
  }
  uint64_t dq[4];                                  // order word of the score << 32 | set-local index
#pragma unroll
  for (int q = 0; q < 4; q++)
    dq[q] = u64_warp_min(qi[q] < 0 ? ~0ull
                                   : ((uint64_t)f32_order(qs[q]) << 32) | (uint32_t)(c0 + qi[q]));
  if (lane == 0) {
#pragma unroll
    for (int k = 0; k < 4; k++) { sred[warp][k] = eo[k]; sdq[warp][k] = dq[k]; }
  }
  __syncthreads();
#pragma unroll
  for (int k = 0; k < 4; k++) {
    uint32_t v = sred[0][k];
#pragma unroll
    for (int q = 1; q < kWarps; q++) v = (k & 1) ? max(v, sred[q][k]) : min(v, sred[q][k]);
    ext[k] = f32_unorder(v);
  }
  // one atomic per quadrant and CTA (the set's words take one from every
  // CTA); the control words were cleared before a1, which leaves dq alone
  if (tid < 4) {
    uint64_t d = sdq[0][tid];
#pragma unroll
    for (int q = 1; q < kWarps; q++) d = min(d, sdq[q][tid]);
    if (d != ~0ull) atomicMax((unsigned long long*)&w.ctl[s].dq[tid], (unsigned long long)~d);
    sidx[tid] = d == ~0ull ? -1 : (int)((int64_t)(uint32_t)d - c0);   // the chunk's quadrant extreme
  }
  __syncthreads();
  // its owner publishes its view: a point that the chunk's quadrant extreme
  // of region r beats strictly in both coordinates is no step of region r
  // (R1 lower-left, R2 lower-right, R3 upper-right, R4 upper-left)
#pragma unroll
  for (int q = 0; q < 4; q++) {
    const int k = sidx[q];
#pragma unroll
    for (int u = 0; u < U; u++)
      if (k == u * kThreads + tid) { sqx[q] = vx[u]; sqy[q] = vy[u]; }
    if (k < 0 && tid == 0) { sqx[q] = __int_as_float(0x7FC00000); sqy[q] = sqx[q]; }   // NaN: beats nothing
  }
  // the chunk's map of region r: u over [a, b] (R1 x, R2 y, R3 -x, R4 -y);
  // an empty or unbounded extent puts everything into bucket 0
  float lo1[4], sc1[4];
#pragma unroll
  for (int r = 0; r < 4; r++) {
    const int e = (r & 1) ? 2 : 0;
    const float a = r < 2 ? ext[e] : -ext[e + 1], b = r < 2 ? ext[e + 1] : -ext[e];
    const float wd = __fsub_rn(b, a);
    lo1[r] = a;
    sc1[r] = (wd > 0.f && wd < inf) ? __fdiv_rn((float)kStairLB, wd) : 0.f;
  }
  __syncthreads();
  // pass 2: the smallest (v, u) per bucket (the shared word is read first:
  // most points change nothing)
#pragma unroll
  for (int u = 0; u < U; u++) {
    if (c0 + u * kThreads + tid >= c1) continue;
    const float X = vx[u], Y = vy[u];
#pragma unroll
    for (int r = 0; r < 4; r++) {
      const float qx = sqx[r], qy = sqy[r];
      const bool bx = (r == 0 || r == 3) ? (qx < X) : (qx > X);
      const bool by = r < 2 ? (qy < Y) : (qy > Y);
      if (bx && by) continue;
      const float su = sort_u(X, Y, r);
      const uint64_t e = ((uint64_t)cmp_view_order(X, Y, r) << 32) | f32_order(su);
      unsigned long long* slot = (unsigned long long*)&lt[r][bucket_of<kStairLB>(su, lo1[r], sc1[r])];
      if (e < *slot) atomicMin(slot, (unsigned long long)e);
    }
  }
  __syncthreads();
  // the chunk's steps: 64 threads per region, 8 buckets each
  const int rr = tid >> 6, ru = tid & 63;
  constexpr int Q = kStairLB / 64;
  uint64_t loc[Q];
  uint32_t stepm = 0;
  {
    uint32_t mn = 0xFFFFFFFFu;
#pragma unroll
    for (int q = 0; q < Q; q++) { loc[q] = lt[rr][ru * Q + q]; mn = min(mn, (uint32_t)(loc[q] >> 32)); }
    uint32_t ex = region_excl_min(mn, sw);
#pragma unroll
    for (int q = 0; q < Q; q++) {
      const uint32_t v = (uint32_t)(loc[q] >> 32);
      if (v < ex) { stepm |= 1u << q; ex = v; }
    }
  }

  griddep_enter();   // a1 has completed: the set's regions, maps and a cleared table
  const SetCtl& c = w.ctl[s];
  if (c.status != 0 || !(c.flags & SF_STAIRS)) return;   // uniform; table unused
  uint32_t* g = w.stairs + (size_t)s * 4 * kStairB;
  {
    // the table word is read first: most CTAs' steps are beaten by others'
    const float lo = c.slo[rr], sc = c.sscale[rr];
    int bk[Q];
    uint32_t cur[Q];
#pragma unroll
    for (int q = 0; q < Q; q++) {
      bk[q] = rr * kStairB + stair_bucket(f32_unorder((uint32_t)loc[q]), lo, sc);
      cur[q] = ((stepm >> q) & 1u) ? __ldcg(g + bk[q]) : 0u;
    }
#pragma unroll
    for (int q = 0; q < Q; q++)
      if ((uint32_t)(loc[q] >> 32) < cur[q]) atomicMin(g + bk[q], (uint32_t)(loc[q] >> 32));
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    last = atomicAdd(&w.ctl[s].arrive3, 1u) == (uint32_t)(sd.nchunk3 - 1);
  }
  __syncthreads();
  if (!last) return;
  __threadfence();
  // Last CTA of the set.  The table loads and the dominance box's loads are
  // issued together.
  uint4 tv[4];
  {
    const uint4* src = reinterpret_cast<const uint4*>(g + rr * kStairB + ru * 16);
#pragma unroll
    for (int q = 0; q < 4; q++) tv[q] = __ldcg(src + q);
  }
  // dominance box: a point strictly inside it is strictly beaten in all four
  // quadrants by sample points (Qll lower-left of it, Qlr lower-right, ...)
  if (threadIdx.x == 0) {
    const uint64_t d0 = *(volatile uint64_t*)&c.dq[0], d1 = *(volatile uint64_t*)&c.dq[1];
    const uint64_t d2 = *(volatile uint64_t*)&c.dq[2], d3 = *(volatile uint64_t*)&c.dq[3];
    if (d0 && d1 && d2 && d3) {
      float X[4], Y[4];
      const uint64_t d[4] = {d0, d1, d2, d3};
      for (int q = 0; q < 4; q++) view_at<DT>(j, sd.off + (uint32_t)~d[q], X[q], Y[q]);
      SetCtl& cw = w.ctl[s];
      cw.bx0 = fmaxf(X[0], X[3]);
      cw.bx1 = fminf(X[1], X[2]);
      cw.by0 = fmaxf(Y[0], Y[1]);
      cw.by1 = fminf(Y[2], Y[3]);
    }
  }
  // exclusive prefix minimum per region, seeded with the first extreme
  {
    uint32_t lv[16];
#pragma unroll
    for (int q = 0; q < 4; q++) { lv[4 * q] = tv[q].x; lv[4 * q + 1] = tv[q].y; lv[4 * q + 2] = tv[q].z; lv[4 * q + 3] = tv[q].w; }
    uint32_t mn = 0xFFFFFFFFu;
#pragma unroll
    for (int q = 0; q < 16; q++) mn = min(mn, lv[q]);
    float EX, EY;
    view_at<DT>(j, sd.off + c.eidx[rr], EX, EY);
    uint32_t ex = min(region_excl_min(mn, sw), cmp_view_order(EX, EY, rr));
    uint4 o[4];
#pragma unroll
    for (int q = 0; q < 16; q++) {
      const uint32_t v = lv[q];
      (&o[q >> 2].x)[q & 3] = ex;
      ex = min(ex, v);
    }
    uint4* dst = reinterpret_cast<uint4*>(g + rr * kStairB + ru * 16);
#pragma unroll
    for (int q = 0; q < 4; q++) dst[q] = o[q];
  }
}

// ------------------------------------------------------------------ a2

// Sort-plan step (single CTA, after a2): sort tiles per set.
__device__ void plan_sort(const Job& j, const Ws& w) {
  __shared__ uint32_t carry;
  __shared__ uint32_t wsum[kWarps];
  if (threadIdx.x == 0) carry = 0;
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int base = 0; base < j.nsets; base += kThreads) {
    int s = base + threadIdx.x;
    uint32_t t = 0;
    if (s < j.nsets && (w.ctl[s].flags & SF_BIG)) t = (w.ctl[s].s1 + kSortTile - 1) / kSortTile;
    uint32_t x = t;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      uint32_t y = __shfl_up_sync(0xFFFFFFFFu, x, o);
      if (lane >= o) x += y;
    }
    if (lane == 31) wsum[warp] = x;
    __syncthreads();
    uint32_t pre = carry;
    for (int q = 0; q < warp; q++) pre += wsum[q];
    if (s < j.nsets) w.sort_start[s] = pre + x - t;
    __syncthreads();
    if (threadIdx.x == kThreads - 1) carry = pre + x;
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    w.sort_start[j.nsets] = carry;
    w.ctr[CT_SORT_TOTAL] = carry;
  }
}

// Exact region test of one point (every edge: FP64 filter, then expansion
// arithmetic).  Kept out of line: only points the FP32 filter cannot decide
// get here.
__device__ __noinline__ int region_exact_f64(double px, double py, const double* ex, const double* ey,
                                             uint32_t flags) {
  for (int k = 0; k < 4; k++) {
    if (flags & (SF_DEGEN0 << k)) continue;
    int k1 = (k + 1) & 3;
    if (orient_f64(ex[k], ey[k], ex[k1], ey[k1], px, py) < 0) return k + 1;
  }
  return 0;
}

__device__ __noinline__ int region_exact_i32_wide(int px, int py, const double* ex, const double* ey,
                                                  uint32_t flags) {
  for (int k = 0; k < 4; k++) {
    if (flags & (SF_DEGEN0 << k)) continue;
    int k1 = (k + 1) & 3;
    if (orient_i32((int)ex[k], (int)ey[k], (int)ex[k1], (int)ey[k1], px, py, true) < 0) return k + 1;
  }
  return 0;
}

// Element r (0..3) of a four-element register array without dynamic
// indexing (which would move the array to local memory).
__device__ __forceinline__ float sel4(const float (&a)[4], int r) {
  return r == 0 ? a[0] : r == 1 ? a[1] : r == 2 ? a[2] : a[3];
}

// Table 1 sort key of a region-r point (r = 1..4): R1 x asc, R2 y asc,
// R3 x desc, R4 y desc, as an ascending order-preserving integer key.
template <int DT>
__device__ __forceinline__ uint64_t sort_key(const typename PointT<DT>::T& p, int r) {
  uint64_t kx, ky, m;
  if constexpr (DT != DT_I32) {
    kx = key_f64((uint64_t)__double_as_longlong(p.x));
    ky = key_f64((uint64_t)__double_as_longlong(p.y));
    m = ~0ull;
  } else {
    kx = key_i32(p.x);
    ky = key_i32(p.y);
    m = 0xFFFFFFFFull;
  }
  switch (r) {
    case 1: return kx;
    case 2: return ky;
    case 3: return kx ^ m;
    default: return ky ^ m;
  }
}

constexpr int kClsBlock = (kClsConsumers + 1) * 32;  // + one producer warp

// a2 stage bytes (the layout of stage_tile)
template <int DT>
constexpr int cls_stage_bytes() {
  return cls_tile(DT) * in_bytes<DT>() + (DT == DT_F32 ? 32 : 16);
}
template <int DT>
constexpr int cls_smem_bytes() {
  return kClsStages * cls_stage_bytes<DT>();
}

// Set parameters a consumer warp keeps in registers (the per-point filter);
// the rest lives in the warp's shared-memory copy (WarpParams).
struct ClsParams {
  float fA[4], fB[4], fC[4], fE[4];
  float bx0, bx1, by0, by1;           // dominance box (empty: never inside)
  uint32_t flags;
  int32_t status;
};
struct WarpParams {
  float slo[4], ssc[4];
  int ix[4], iy[4];
};

// Octagon mode: certainly strictly inside all eight octagon edges by their
// FP32 filters (oct[k] = A, -B, C, E of edge k, a shared-memory copy).
__device__ __forceinline__ bool oct_inside_f32(const float4* oct, float X, float Y) {
  bool in = true;
#pragma unroll
  for (int k = 0; k < 8; k++) {
    const float4 e = oct[k];
    in &= __fmaf_rn(e.x, Y, __fmaf_rn(e.y, X, e.z)) > e.w;
  }
  return in;
}

// Octagon mode, exact: strictly inside all eight edges (degenerate edges
// skipped), the FP32 filter deciding where it can.
template <int DT>
__device__ bool oct_inside_exact(const float4* oct, const SetCtl& c, float X, float Y,
                                 const typename PointT<DT>::T& p) {
#pragma unroll 1
  for (int k = 0; k < 8; k++) {
    const int k1 = (k + 1) & 7;
    const double ax = c.ovx[k], ay = c.ovy[k], bx = c.ovx[k1], by = c.ovy[k1];
    if (ax == bx && ay == by) continue;
    const float4 e = oct[k];
    const float d = __fmaf_rn(e.x, Y, __fmaf_rn(e.y, X, e.z));
    if (d > e.w) continue;
    if (d < -e.w) return false;
    int o;
    if constexpr (DT != DT_I32) o = orient_f64(ax, ay, bx, by, p.x, p.y);
    else o = orient_i32((int)ax, (int)ay, (int)bx, (int)by, p.x, p.y, true);
    if (o <= 0) return false;
  }
  return true;
}

// a2 pass 1 of a float64 tile slice (items k = 0 .. IW-1 of this lane, point
// wb + 32 k + lane): bit k of the result is set unless the point is certainly
// inside the quadrilateral (FP32 filter of the four edges) or strictly inside
// the dominance box; the point's FP32 view goes to vbw[32 k + lane].  SHORT
// selects the three-operation FP32 view.
template <bool SHORT, bool OCT, int IW>
__device__ __forceinline__ uint32_t a2_pass1_f64(const unsigned char* base, int wb, int lane, int npv,
                                                 const ClsParams& cp, uint2* vbw, const float4* oct) {
  uint32_t nim = 0;
#pragma unroll 4
  for (int k = 0; k < IW; k++) {
    const int i = wb + k * 32 + lane;
    if (i < npv) {
      const double2 p = *reinterpret_cast<const double2*>(base + i * 16);
      float X, Y;
      f32_view_a2<DT_F64, SHORT>(p, X, Y);
      vbw[k * 32 + lane] = make_uint2(__float_as_uint(X), __float_as_uint(Y));
      if constexpr (OCT) {
        nim |= (uint32_t)!oct_inside_f32(oct, X, Y) << k;
        continue;
      }
      const float d0 = __fmaf_rn(cp.fA[0], Y, __fmaf_rn(cp.fB[0], X, cp.fC[0]));
      const float d1 = __fmaf_rn(cp.fA[1], Y, __fmaf_rn(cp.fB[1], X, cp.fC[1]));
      const float d2 = __fmaf_rn(cp.fA[2], Y, __fmaf_rn(cp.fB[2], X, cp.fC[2]));
      const float d3 = __fmaf_rn(cp.fA[3], Y, __fmaf_rn(cp.fB[3], X, cp.fC[3]));
      const bool in = ((d0 > cp.fE[0]) & (d1 > cp.fE[1]) & (d2 > cp.fE[2]) & (d3 > cp.fE[3])) |
                      ((X > cp.bx0) & (X < cp.bx1) & (Y > cp.by0) & (Y < cp.by1));
      nim |= (uint32_t)(!in) << k;
    }
  }
  return nim;
}

// The same pass on a float32 tile slice (vx, vy: the stage's two halves).
// The values are their own FP32 views, and the view buffer keeps them: pass 2
// widens them again where it needs exact coordinates.
template <bool OCT, int IW>
__device__ __forceinline__ uint32_t a2_pass1_f32(const float* vx, const float* vy, int wb, int lane, int npv,
                                                 const ClsParams& cp, uint2* vbw, const float4* oct) {
  uint32_t nim = 0;
#pragma unroll 4
  for (int k = 0; k < IW; k++) {
    const int i = wb + k * 32 + lane;
    if (i < npv) {
      const float X = vx[i], Y = vy[i];
      vbw[k * 32 + lane] = make_uint2(__float_as_uint(X), __float_as_uint(Y));
      if constexpr (OCT) {
        nim |= (uint32_t)!oct_inside_f32(oct, X, Y) << k;
        continue;
      }
      const float d0 = __fmaf_rn(cp.fA[0], Y, __fmaf_rn(cp.fB[0], X, cp.fC[0]));
      const float d1 = __fmaf_rn(cp.fA[1], Y, __fmaf_rn(cp.fB[1], X, cp.fC[1]));
      const float d2 = __fmaf_rn(cp.fA[2], Y, __fmaf_rn(cp.fB[2], X, cp.fC[2]));
      const float d3 = __fmaf_rn(cp.fA[3], Y, __fmaf_rn(cp.fB[3], X, cp.fC[3]));
      const bool in = ((d0 > cp.fE[0]) & (d1 > cp.fE[1]) & (d2 > cp.fE[2]) & (d3 > cp.fE[3])) |
                      ((X > cp.bx0) & (X < cp.bx1) & (Y > cp.by0) & (Y < cp.by1));
      nim |= (uint32_t)(!in) << k;
    }
  }
  return nim;
}

// a2.  Warp-specialised: warp 8 acquires tiles (in increasing order) and
// streams them into a ring of shared-memory stages with 1-D TMA bulk copies
// (full/empty mbarriers); warps 0..7 each classify a contiguous eighth of the
// tile, so (warp, item, lane) is point order, and compact their survivors
// into their own sub-slot of the tile's record range (index order within the
// sub-slot) -- no block-wide barrier on the per-tile path.
template <int DT, bool OCT>
__global__ void __launch_bounds__(kClsBlock, 2) k_classify(Job j, Ws w) {
  griddep_enter();
  using P = typename PointT<DT>::T;
  constexpr int PB = in_bytes<DT>();
  constexpr int TILE = cls_tile(DT);
  static_assert(TILE % (32 * kClsConsumers) == 0, "a tile is a whole number of items per consumer lane");
  constexpr int WPTS = TILE / kClsConsumers;          // points per consumer warp
  constexpr int IW = WPTS / 32;                       // items per lane
  static_assert(IW <= 16, "pass-2 queue entries hold the item in 4 bits");
  constexpr int SB = cls_stage_bytes<DT>();           // stage bytes (the layout of stage_tile)
  constexpr int HALF = TILE * 4 + 16;                 // float32: offset of the y half
  extern __shared__ __align__(128) unsigned char smem[];
  __shared__ __align__(8) uint64_t full[kClsStages], empty[kClsStages];
  __shared__ int st_tile[kClsStages], st_set[kClsStages], st_head[kClsStages];
  __shared__ uint16_t wq[kClsConsumers][IW * 32];     // pass-2 queue: item << 5 | lane
  __shared__ uint2 vb[kClsConsumers][IW * 32];         // views (float64) / points (int32, float32) of the warp's slice
  __shared__ float4 woct[kClsConsumers][OCT ? 8 : 1];  // octagon mode: the edges' FP32 filters, per warp
  __shared__ WarpParams wpar[kClsConsumers];

  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  if (tid == 0) {
    for (int q = 0; q < kClsStages; q++) { mbar_init(&full[q], 1); mbar_init(&empty[q], kClsConsumers); }
    fence_mbar_init();
    fence_async_smem();
  }
  __syncthreads();

  if (warp == kClsConsumers) {
    // ---------------------------------------------------------- producer
    if (lane != 0) return;
    int issued = 0;
    bool ok = true;
    for (int it = 0;; it++) {
      const int slot = it % kClsStages;
      if (it >= kClsStages) {
        uint32_t spins = 0;
        while (!mbar_try_wait(&empty[slot], (uint32_t)((it / kClsStages) - 1) & 1u))
          if (!spin_step(spins, w.ctr)) { ok = false; break; }
        if (!ok) break;
        fence_async_smem();
      }
      // tiles from the last to the first: the first ones are still in L2
      // from a1
      const uint32_t tc = atomicAdd(w.ctr + CT_CLS_TILE, 1u);
      const uint32_t t = tc < (uint32_t)j.ntile2 ? (uint32_t)j.ntile2 - 1u - tc : tc;
      st_tile[slot] = (int)t;
      if (t >= (uint32_t)j.ntile2) {
        asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" :: "r"(smem_addr(&full[slot])) : "memory");
        break;
      }
      int s = 0;
      if (j.sets) {
        int lo = 0, hi = j.nsets - 1;
        while (lo < hi) {
          int mid = (lo + hi + 1) >> 1;
          if (j.sets[mid].tile2 <= (int)t) lo = mid; else hi = mid - 1;
        }
        s = lo;
      }
      st_set[slot] = s;
      const SetDesc sd = get_set(j, s);
      const int64_t i0 = (int64_t)(t - sd.tile2) * TILE;
      const int np = (int)min((int64_t)TILE, sd.n - i0);
      stage_tile<DT>(j, sd.off + i0, np, smem + slot * SB, HALF, &full[slot], false, &st_head[slot]);
      issued = it + 1;
    }
    if (!ok) {
      // a wait ran out: let the copies already issued land before exiting
      for (int it = max(0, issued - kClsStages); it < issued; it++) {
        uint32_t spins = 0;
        while (!mbar_try_wait(&full[it % kClsStages], (uint32_t)(it / kClsStages) & 1u))
          if (!spin_step(spins, w.ctr) && spins > kSpinLimit) break;
      }
    }
    return;
  }

  // ------------------------------------------------------------ consumers
  ClsParams cp{};
  int cur_set = -1;
  const uint32_t lt_mask = (1u << lane) - 1u;
  for (int it = 0;; it++) {
    const int slot = it % kClsStages;
    {
      uint32_t spins = 0;
      bool ok = true;
      while (!mbar_try_wait(&full[slot], (uint32_t)(it / kClsStages) & 1u))
        if (!spin_step(spins, w.ctr)) { ok = false; break; }
      if (!ok) break;
    }
    const int tile = st_tile[slot];
    if (tile >= j.ntile2) break;
    const int s = st_set[slot];
    const SetDesc sd = get_set(j, s);
    WarpParams& wp = wpar[warp];
    if (s != cur_set) {
      const SetCtl& c = w.ctl[s];
#pragma unroll
      for (int k = 0; k < 4; k++) {
        cp.fA[k] = c.fA[k]; cp.fB[k] = -c.fB[k]; cp.fC[k] = c.fC[k]; cp.fE[k] = c.fE[k];
      }
      if (lane < 4) {
        wp.slo[lane] = c.slo[lane]; wp.ssc[lane] = c.sscale[lane];
        wp.ix[lane] = (int)c.ex[lane]; wp.iy[lane] = (int)c.ey[lane];
      }
      if constexpr (OCT)
        if (lane < 8) woct[warp][lane] = make_float4(c.oA[lane], -c.oB[lane], c.oC[lane], c.oE[lane]);
      __syncwarp();
      cp.bx0 = c.bx0; cp.bx1 = c.bx1; cp.by0 = c.by0; cp.by1 = c.by1;
      cp.flags = c.flags;
      cp.status = c.status;
      cur_set = s;
    }
    const int64_t lt = tile - sd.tile2;
    const int64_t t0 = lt * TILE;
    const int np = (int)min((int64_t)TILE, sd.n - t0);
    const unsigned char* base = smem + slot * SB + 16 - st_head[slot] * PB;
    const int wb = warp * WPTS;                    // this warp's first point in the tile
    const int npv = cp.status != 0 ? 0 : np;
    const uint32_t* pre = w.stairs + (size_t)s * 4 * kStairB;
    const SetCtl& cg = w.ctl[s];
    const bool shortv = (cp.flags & SF_SHORTVIEW) != 0;

    // pass 1, every point: is it certainly inside the quadrilateral?
    // (float64: the FP32 filter's four edge tests; int32: the exact region).
    // Every point's FP32 view (float64) or the point itself (int32) goes to
    // the warp's view buffer, so that the stage can be released right after
    // this pass and the producer refills it while pass 2 runs.
    uint32_t nim = 0;                              // items that need pass 2
    uint2* vbw = vb[warp];
    if constexpr (DT == DT_F32) {
      const float* vx = reinterpret_cast<const float*>(smem + slot * SB + 16) - (st_head[slot] & 0xFF);
      const float* vy = reinterpret_cast<const float*>(smem + slot * SB + HALF + 16) - (st_head[slot] >> 8);
      nim = a2_pass1_f32<OCT, IW>(vx, vy, wb, lane, npv, cp, vbw, woct[warp]);
    } else if constexpr (DT == DT_F64) {
      nim = shortv ? a2_pass1_f64<true, OCT, IW>(base, wb, lane, npv, cp, vbw, woct[warp])
                   : a2_pass1_f64<false, OCT, IW>(base, wb, lane, npv, cp, vbw, woct[warp]);
    } else {
      // the same FP32 filter on the rounded views; the buffer keeps the
      // exact coordinates for pass 2
#pragma unroll 4
      for (int k = 0; k < IW; k++) {
        const int i = wb + k * 32 + lane;
        if (i < npv) {
          const P p = *reinterpret_cast<const P*>(base + i * PB);
          vbw[k * 32 + lane] = make_uint2((uint32_t)p.x, (uint32_t)p.y);
          const float X = __int2float_rn(p.x), Y = __int2float_rn(p.y);
          if constexpr (OCT) {
            nim |= (uint32_t)!oct_inside_f32(woct[warp], X, Y) << k;
          } else {
            const float d0 = __fmaf_rn(cp.fA[0], Y, __fmaf_rn(cp.fB[0], X, cp.fC[0]));
            const float d1 = __fmaf_rn(cp.fA[1], Y, __fmaf_rn(cp.fB[1], X, cp.fC[1]));
            const float d2 = __fmaf_rn(cp.fA[2], Y, __fmaf_rn(cp.fB[2], X, cp.fC[2]));
            const float d3 = __fmaf_rn(cp.fA[3], Y, __fmaf_rn(cp.fB[3], X, cp.fC[3]));
            const bool in = ((d0 > cp.fE[0]) & (d1 > cp.fE[1]) & (d2 > cp.fE[2]) & (d3 > cp.fE[3])) |
                            ((X > cp.bx0) & (X < cp.bx1) & (Y > cp.by0) & (Y < cp.by1));
            nim |= (uint32_t)(!in) << k;
          }
        }
      }
    }
    __syncwarp();
    if (lane == 0)   // the warp is done with the stage: release it to the producer
      asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" :: "r"(smem_addr(&empty[slot])) : "memory");

    // pass 2, dense over the warp's remaining points (a queue): region,
    // exact test where the filter was undecided, dominance prefilter.  The
    // queue lists the points in index order, so each round of 32 entries
    // compacts its survivors into the warp's sub-slot of the tile in order.
    // Only the rare exact test and the survivors' records read the point's
    // exact coordinates (float64: again from global memory).
    uint32_t rc01 = 0, rc23 = 0;                   // survivors of R1|R2, R3|R4 (16-bit fields)
    if (__any_sync(0xFFFFFFFFu, nim != 0)) {
      uint16_t* q = wq[warp];
      uint32_t nq = 0;
#pragma unroll
      for (int k = 0; k < IW; k++) {
        const bool o = (nim >> k) & 1u;
        const uint32_t b = __ballot_sync(0xFFFFFFFFu, o);
        if (o) {
          q[nq + __popc(b & lt_mask)] = (uint16_t)((k << 5) | lane);
        }
        nq += __popc(b);
      }
      __syncwarp();
      const int64_t ob = sd.off + t0 + wb;
      // float64: exact coordinates from global memory; float32: the views
      // are the values (widened where needed)
      const P* gp = DT == DT_F64 ? reinterpret_cast<const P*>(j.pts) + sd.off + t0 : nullptr;
      uint32_t run = 0;
      for (uint32_t e0 = 0; e0 < nq; e0 += 32) {
        const uint32_t e = e0 + lane;
        uint32_t r = 0;
        int i = 0;
        P p{};
        if (e < nq) {
          const uint32_t en = q[e];
          const int slot_i = (int)((en >> 5) & 15) * 32 + (int)(en & 31);
          i = wb + slot_i;
          const uint2 v = vbw[slot_i];
          float X, Y;
          if constexpr (DT != DT_I32) {
            X = __uint_as_float(v.x);
            Y = __uint_as_float(v.y);
            const float d0 = __fmaf_rn(cp.fA[0], Y, __fmaf_rn(cp.fB[0], X, cp.fC[0]));
            const float d1 = __fmaf_rn(cp.fA[1], Y, __fmaf_rn(cp.fB[1], X, cp.fC[1]));
            const float d2 = __fmaf_rn(cp.fA[2], Y, __fmaf_rn(cp.fB[2], X, cp.fC[2]));
            const float d3 = __fmaf_rn(cp.fA[3], Y, __fmaf_rn(cp.fB[3], X, cp.fC[3]));
            // first edge not certainly inside decides: outside -> region,
            // undecided -> exact test
            r = !(d3 > cp.fE[3]) ? (d3 < -cp.fE[3] ? 4u : 15u) : 0u;
            r = !(d2 > cp.fE[2]) ? (d2 < -cp.fE[2] ? 3u : 15u) : r;
            r = !(d1 > cp.fE[1]) ? (d1 < -cp.fE[1] ? 2u : 15u) : r;
            r = !(d0 > cp.fE[0]) ? (d0 < -cp.fE[0] ? 1u : 15u) : r;
            if (r == 15u) {
              if constexpr (DT == DT_F32) p = make_double2(widen_f32(X), widen_f32(Y));
              else p = gp[i];
              r = (uint32_t)region_exact_f64(p.x, p.y, cg.ex, cg.ey, cp.flags);
            }
          } else {
            // exact region in 64-bit (128-bit for wide spans) integers
            p.x = (int)v.x;
            p.y = (int)v.y;
            X = __int2float_rn(p.x);
            Y = __int2float_rn(p.y);
            if (cp.flags & SF_WIDE) {
              r = (uint32_t)region_exact_i32_wide(p.x, p.y, cg.ex, cg.ey, cp.flags);
            } else {
#pragma unroll
              for (int qq = 3; qq >= 0; qq--) {
                if (!(cp.flags & (SF_DEGEN0 << qq)) &&
                    orient_i32(wp.ix[qq], wp.iy[qq], wp.ix[(qq + 1) & 3], wp.iy[(qq + 1) & 3], p.x, p.y, false) < 0)
                  r = (uint32_t)qq + 1;
              }
            }
          }
          if constexpr (OCT) {
            if (r != 0) {
              if constexpr (DT == DT_F32) p = make_double2(widen_f32(X), widen_f32(Y));
              else if constexpr (DT == DT_F64) p = gp[i];
              if (oct_inside_exact<DT>(woct[warp], cg, X, Y, p)) r = 0;    // inside the octagon
            }
          }
          if (r != 0 && (cp.flags & SF_STAIRS)) {
            const int qr = (int)r - 1;
            const int bk = stair_bucket(sort_u(X, Y, qr), wp.slo[qr], wp.ssc[qr]);
            if (cmp_view_order(X, Y, qr) > __ldg(pre + qr * kStairB + bk)) r = 0;    // dominated
          }
          if constexpr (DT == DT_F32)
            if (r != 0) p = make_double2(widen_f32(X), widen_f32(Y));
        }
        const uint32_t b = __ballot_sync(0xFFFFFFFFu, r != 0);
        if (r != 0) {
          if constexpr (DT == DT_F64) p = gp[i];   // exact coordinates of a survivor
          const int64_t o = ob + run + __popc(b & lt_mask);
          w.keyB[o] = sort_key<DT>(p, (int)r);
          w.valB[o] = ((r - 1u) << 30) | (uint32_t)(t0 + i);
          if constexpr (DT != DT_I32) w.spvB[o] = spa_v_f64(p.x, p.y, (int)r - 1);
          else w.spvB[o] = spa_v_i32(p.x, p.y, (int)r - 1);
          const uint32_t inc = 1u << (((r - 1u) & 1u) * 16u);
          if (r <= 2u) rc01 += inc; else rc23 += inc;
        }
        run += __popc(b);
      }
      rc01 = __reduce_add_sync(0xFFFFFFFFu, rc01);
      rc23 = __reduce_add_sync(0xFFFFFFFFu, rc23);
    }
    if (lane == 0) {
      w.tcnt[(size_t)tile * kClsConsumers + warp] = (uint64_t)rc01 | ((uint64_t)rc23 << 32);
      uint32_t* pt = reinterpret_cast<uint32_t*>(w.ptot + sd.chunkP + (int)(lt / kPlanTiles));
      if (rc01 & 0xFFFFu) atomicAdd(pt + 0, rc01 & 0xFFFFu);
      if (rc01 >> 16) atomicAdd(pt + 1, rc01 >> 16);
      if (rc23 & 0xFFFFu) atomicAdd(pt + 2, rc23 & 0xFFFFu);
      if (rc23 >> 16) atomicAdd(pt + 3, rc23 >> 16);
    }
  }
}

// ------------------------------------------------------------ gather
//
// After a2 every (tile, consumer warp) sub-slot holds its survivors in place
// and a2 has added up every chunk's survivors per region (ptot).  k_gather
// runs one CTA per chunk: the set's region totals and the chunk's offsets
// come from ptot, the eight warps split the chunk's sub-slots, and every
// survivor moves to its region-major record, order kept.  The last CTA to
// finish decides per set between the shared-memory path (every region at
// most kSmallMax) and the multi-block sort, and plans both.

__global__ void __launch_bounds__(kThreads) k_gather(Job j, Ws w) {
  griddep_enter();
  constexpr int kChunkSub = kPlanTiles * kClsConsumers;     // sub-slots of a chunk
  constexpr int kPartSub = kChunkSub / kGatherSplit;         // sub-slots of a part of a dense chunk
  __shared__ uint32_t sh_tot[4], sh_cpre[4], sh_ct;
  __shared__ uint32_t wtot[kWarps][4], wpre[kWarps][4];
  __shared__ int sh_last;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int chunk = blockIdx.x / kGatherSplit, part = blockIdx.x % kGatherSplit;
  int s = 0;
  if (j.sets) {
    int lo = 0, hi = j.nsets - 1;
    while (lo < hi) {
      int mid = (lo + hi + 1) >> 1;
      if (j.sets[mid].chunkP <= chunk) lo = mid; else hi = mid - 1;
    }
    s = lo;
  }
  const SetDesc sd = get_set(j, s);
  const int lc = chunk - sd.chunkP;
  if (w.ctl[s].status == 0 && lc < sd.nchunkP) {      // uniform across the CTA
    if (warp == 0) {
      // region totals of the set and of its chunks before this one
      uint32_t t[4] = {0, 0, 0, 0}, p[4] = {0, 0, 0, 0};
      const uint4* pt = w.ptot + sd.chunkP;
      for (int k = lane; k < sd.nchunkP; k += 32) {
        const uint4 v = pt[k];
        t[0] += v.x; t[1] += v.y; t[2] += v.z; t[3] += v.w;
        if (k < lc) { p[0] += v.x; p[1] += v.y; p[2] += v.z; p[3] += v.w; }
      }
#pragma unroll
      for (int q = 0; q < 4; q++) {
        t[q] = __reduce_add_sync(0xFFFFFFFFu, t[q]);
        p[q] = __reduce_add_sync(0xFFFFFFFFu, p[q]);
      }
      if (lane == 0) {
        for (int q = 0; q < 4; q++) { sh_tot[q] = t[q]; sh_cpre[q] = p[q]; }
        const uint4 cv = pt[lc];
        sh_ct = cv.x + cv.y + cv.z + cv.w;
        if (lc == 0 && part == 0) {
          // the set's first chunk records its region totals and its path
          SetCtl& cs = w.ctl[s];
          bool big = false;
          for (int q = 0; q < 4; q++) { cs.cnt[q] = t[q]; big |= t[q] > (uint32_t)j.tune.small_max; }
          cs.s1 = t[0] + t[1] + t[2] + t[3];
          // the paper's chunked SPA reads the sorted records from global memory
          if ((j.opts & OPT_BLOCKED_SPA) && cs.s1 > 0) big = true;
          if (big) atomicOr(&cs.flags, (uint32_t)SF_BIG);
        }
      }
    }
    __syncthreads();
    // A chunk with few survivors is moved by its first CTA alone; a dense
    // one by all kGatherSplit CTAs of the chunk, each a part of its
    // sub-slots (the survivors of the earlier parts are counted first).
    const bool dense = sh_ct >= (uint32_t)kGatherDense;
    if (dense || part == 0) {                          // uniform across the CTA
      const int64_t nsub = (int64_t)sd.ntile2 * kClsConsumers;
      const int64_t cs0 = (int64_t)lc * kChunkSub;
      const int64_t a = dense ? cs0 + (int64_t)part * kPartSub : cs0;
      const int per_warp = (dense ? kPartSub : kChunkSub) / kWarps;
      const int64_t g0 = a + warp * per_warp;
      const int64_t g1 = min(g0 + per_warp, nsub);
      const uint64_t* tc = w.tcnt + (size_t)sd.tile2 * kClsConsumers;
      uint32_t mt[4] = {0, 0, 0, 0}, mp[4] = {0, 0, 0, 0};
      for (int64_t g = g0 + lane; g < g1; g += 32) {
        const uint64_t v = tc[g];
#pragma unroll
        for (int q = 0; q < 4; q++) mt[q] += (uint32_t)(v >> (16 * q)) & 0xFFFFu;
      }
      // the chunk's sub-slots before this CTA's part (none for part 0)
      for (int64_t g = cs0 + threadIdx.x; g < min(a, nsub); g += kThreads) {
        const uint64_t v = tc[g];
#pragma unroll
        for (int q = 0; q < 4; q++) mp[q] += (uint32_t)(v >> (16 * q)) & 0xFFFFu;
      }
#pragma unroll
      for (int q = 0; q < 4; q++) {
        mt[q] = __reduce_add_sync(0xFFFFFFFFu, mt[q]);
        mp[q] = __reduce_add_sync(0xFFFFFFFFu, mp[q]);
      }
      if (lane == 0)
        for (int q = 0; q < 4; q++) { wtot[warp][q] = mt[q]; wpre[warp][q] = mp[q]; }
      __syncthreads();
      uint32_t pos[4], roff[4], acc = 0;
#pragma unroll
      for (int q = 0; q < 4; q++) {
        pos[q] = sh_cpre[q];
        for (int v = 0; v < kWarps; v++) pos[q] += wpre[v][q];
        for (int v = 0; v < warp; v++) pos[q] += wtot[v][q];
        roff[q] = acc;
        acc += sh_tot[q];
      }
      if (g0 < g1) move_subslots(j, w, sd, s, g0, g1, -1, pos, roff);
    }
  }
  // last CTA: region totals of every set, the path of every set, the plans
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    sh_last = atomicAdd(w.ctr + CT_PLAN_DONE, 1u) == gridDim.x - 1;
  }
  __syncthreads();
  if (!sh_last) return;
  __threadfence();
  // last CTA: the plans of both sort paths over all sets (block-wide scans;
  // every set's region totals and path were recorded by its first chunk)
  plan_sort(j, w);
  __shared__ uint32_t carry;
  __shared__ uint32_t wsum[kWarps];
  if (threadIdx.x == 0) carry = 0;
  __syncthreads();
  for (int base = 0; base < j.nsets; base += kThreads) {
    const int s2 = base + threadIdx.x;
    uint32_t nseg = 0;
    if (s2 < j.nsets) {
      const SetCtl& c2 = w.ctl[s2];
      if (c2.status == 0 && !(c2.flags & SF_BIG))
        for (int r = 0; r < 4; r++) nseg += c2.cnt[r] != 0;
    }
    uint32_t x = nseg;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t y = __shfl_up_sync(0xFFFFFFFFu, x, o);
      if (lane >= o) x += y;
    }
    if (lane == 31) wsum[warp] = x;
    __syncthreads();
    uint32_t k = carry + x - nseg;
    for (int q = 0; q < warp; q++) k += wsum[q];
    if (nseg) {
      const SetCtl& c2 = w.ctl[s2];
      for (int r = 0; r < 4; r++)
        if (c2.cnt[r]) w.small_seg[k++] = (uint32_t)(4 * s2 + r);
    }
    __syncthreads();
    if (threadIdx.x == kThreads - 1) carry = k;
    __syncthreads();
  }
  if (threadIdx.x == 0) w.ctr[CT_SMALL_TOTAL] = carry;
}

template <int DT, bool OCT>
static void extremes_attr() {
  static bool once = [] {
    cudaFuncSetAttribute(k_extremes<DT, OCT>, cudaFuncAttributeMaxDynamicSharedMemorySize, kExtSmem);
    return true;
  }();
  (void)once;
}

int extremes_blocks_per_sm(int dtype) {
  int b = 0;
  if (dtype == DT_F64) {
    extremes_attr<DT_F64, false>();
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_extremes<DT_F64, false>, kExtBlock, kExtSmem);
  } else if (dtype == DT_F32) {
    extremes_attr<DT_F32, false>();
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_extremes<DT_F32, false>, kExtBlock, kExtSmem);
  } else {
    extremes_attr<DT_I32, false>();
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_extremes<DT_I32, false>, kExtBlock, kExtSmem);
  }
  return b > 0 ? b : 1;
}

template <int DT, bool OCT>
static void launch_extremes_t(const Job& j, const Ws& w, const Launch& L) {
  extremes_attr<DT, OCT>();
  launch_pdl(k_extremes<DT, OCT>, j.nchunk1, kExtBlock, kExtSmem, L.stream, j, w);
}

int launch_extremes(const Job& j, const Ws& w, const Launch& L) {
  if (j.nchunk1 == 0) return 0;
  const bool oct = (j.opts & OPT_OCTAGON) != 0;
  if (j.dtype == DT_F64) {
    if (oct) launch_extremes_t<DT_F64, true>(j, w, L);
    else launch_extremes_t<DT_F64, false>(j, w, L);
  } else if (j.dtype == DT_F32) {
    if (oct) launch_extremes_t<DT_F32, true>(j, w, L);
    else launch_extremes_t<DT_F32, false>(j, w, L);
  } else {
    if (oct) launch_extremes_t<DT_I32, true>(j, w, L);
    else launch_extremes_t<DT_I32, false>(j, w, L);
  }
  return 1;
}

int launch_stairs(const Job& j, const Ws& w, const Launch& L) {
  if (j.nchunk3 == 0) return 0;
  if (j.dtype == DT_F64) launch_pdl(k_stairs<DT_F64>, j.nchunk3, kThreads, 0, L.stream, j, w);
  else if (j.dtype == DT_F32) launch_pdl(k_stairs<DT_F32>, j.nchunk3, kThreads, 0, L.stream, j, w);
  else launch_pdl(k_stairs<DT_I32>, j.nchunk3, kThreads, 0, L.stream, j, w);
  return 1;
}

int launch_gather(const Job& j, const Ws& w, const Launch& L) {
  launch_pdl(k_gather, (j.nchunkP < 1 ? 1 : j.nchunkP) * kGatherSplit, kThreads, 0, L.stream, j, w);
  return 1;
}

template <int DT, bool OCT>
static void launch_classify_t(const Job& j, const Ws& w, const Launch& L, int grid) {
  static bool once = [] {
    cudaFuncSetAttribute(k_classify<DT, OCT>, cudaFuncAttributeMaxDynamicSharedMemorySize, cls_smem_bytes<DT>());
    return true;
  }();
  (void)once;
  launch_pdl(k_classify<DT, OCT>, grid, kClsBlock, cls_smem_bytes<DT>(), L.stream, j, w);
}

int launch_classify(const Job& j, const Ws& w, const Launch& L) {
  int grid = j.ntile2 < L.cls_grid ? j.ntile2 : L.cls_grid;
  if (grid < 1) grid = 1;
  const bool oct = (j.opts & OPT_OCTAGON) != 0;
  if (j.dtype == DT_F64) {
    if (oct) launch_classify_t<DT_F64, true>(j, w, L, grid);
    else launch_classify_t<DT_F64, false>(j, w, L, grid);
  } else if (j.dtype == DT_F32) {
    if (oct) launch_classify_t<DT_F32, true>(j, w, L, grid);
    else launch_classify_t<DT_F32, false>(j, w, L, grid);
  } else {
    if (oct) launch_classify_t<DT_I32, true>(j, w, L, grid);
    else launch_classify_t<DT_I32, false>(j, w, L, grid);
  }
  return 1;
}

}  // namespace cch

// cch_internal.cuh -- shared device-side definitions of the CudaChain hull
// pipeline (sm_103a).  Nothing here is visible through the C ABI.
//
// Pipeline (Sec. 2.1, steps 1-7), every stage a kernel, every set of points a
// "set" (a single hull is a batch of one):
//   a1  k_extremes      four lexicographic extremes + edge set-up (step 1)
//       k_stairs        dominance tables and box from a sample of each set;
//                       its sample pass runs during a1's tail
//   a2  k_classify      quadrilateral test, region routing and dominance
//                       prefilter; survivors compacted in place per tile
//                       (steps 2-3)
//       k_gather        survivors moved into region-major order; per set the
//                       choice between the two sort paths
//   a3+ k_small         per (set, region) in one CTA (or, for calls of a few
//   a4                  sets, an 8-CTA cluster): Table 1 sort and Fig. 2 SPA
//                       in shared memory (steps 4-5)
//       k_big           sets with a region above kSmallMax records: LSD radix
//                       sort and SPA as a segmented prefix-minimum scan, one
//                       cooperative persistent kernel (steps 4-5)
//   a5  k_chain_local + strictly convex chain per region (steps 6-7; the
//       k_chain_merge + paper's CPU Melkman stage is replaced by chunked
//       k_output        hulls merged by bridge walks) and the output
//                       compaction
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace cch {

// ------------------------------------------------------------------ status
enum : int {
  ST_OK = 0,
  ST_INVALID = -1,
  ST_DTYPE = -2,
  ST_NONFINITE = -3,
  ST_RANGE = -4,
  ST_NOMEM = -5,
  ST_CUDA = -6,
  ST_TIMEOUT = -7,
};

// Input formats.  DT_F32 (two float32 coordinate vectors) is read by the
// round-1 kernels only: every later stage sees its points widened exactly to
// float64 and runs the float64 code (the keys and SPA values it gets are the
// float64 ones of the widened points).
enum : int { DT_I32 = 1, DT_F64 = 2, DT_F32 = 3 };

// ------------------------------------------------------------------ sizes
constexpr int kThreads = 256;          // every kernel runs 256-thread CTAs
constexpr int kWarps = kThreads / 32;
// a2 tiles (points; a multiple of 32 x kClsConsumers): one TMA stage each
constexpr int kClsTileF64 = 2048;      // 32 KB
constexpr int kClsTileI32 = 4096;      // 32 KB
constexpr int kClsStages = 2;          // TMA ring depth of a2
constexpr int kClsConsumers = 8;       // consumer warps of a2: each tile has 8 sub-slots
// a2 tile of an input format: 32 KB of points (float32 vectors and int32
// pairs take 8 bytes a point, float64 pairs 16)
__host__ __device__ constexpr int cls_tile(int dtype) { return dtype == DT_F64 ? kClsTileF64 : kClsTileI32; }
constexpr int kClsMinTile = kClsTileF64 < kClsTileI32 ? kClsTileF64 : kClsTileI32;
// SPA-dominance prefilter ("stairs"): per region, the prefix minimum of the
// compared coordinate over buckets of the sort coordinate, built from a
// sample of the set.
constexpr int kStairB = 1024;          // buckets per region
constexpr int64_t kStairSample = int64_t(1) << 20;   // sample points per set (the last ones)
constexpr int kStairChunk = 2048;      // sample points per k_stairs CTA (eight per thread)
constexpr int kStairLB = 512;          // buckets per region of a k_stairs CTA's own table
constexpr int64_t kStairMin = 8192;    // smallest sample of a set
constexpr int kPlanTiles = 64;         // a2 tiles per survivor-count chunk
constexpr int kGatherSplit = 8;        // gather CTAs per chunk (all of them move a dense chunk)
constexpr int kGatherDense = 8192;     // survivors from which a chunk counts as dense
// a1 reads the last kL2KeepBytes of every set without the evict-first hint,
// so that they are still in L2 when k_stairs samples them (its sample is the
// set's tail) and when a2 starts (a2 hands out its tiles from the last to the
// first).
constexpr int64_t kL2KeepBytes = int64_t(48) << 20;
// Run-time choices of a call.  None of them changes a result (each only
// moves work between equivalent paths or resizes a sample that feeds an
// exact prefilter); the tuner (tune.cu) picks them per size bucket.
struct Tune {
  int32_t small_max;    // largest region of the shared-memory sort path (1 .. kSmallMax)
  int32_t stair_div;    // stairs sample m = min(n, stair_max, max(stair_min, n / stair_div))
  int32_t stair_min;
  int32_t stair_max;
  int32_t a1_len_min;   // smallest a1 chunk in points (a multiple of 1024)
  int32_t cls_per_sm;   // a2 CTAs per SM (1 or 2)
};
// Sample of a set: its last m points (the most recently streamed by a1).
__host__ __device__ inline int64_t stairs_sample(int64_t n, const Tune& t) {
  int64_t m = n / t.stair_div;
  if (m < t.stair_min) m = t.stair_min;
  if (m > t.stair_max) m = t.stair_max;
  return m < n ? m : n;
}
constexpr int kSortItems = 16;
constexpr int kSortTile = kThreads * kSortItems;    // 4096 records
constexpr int kSortPasses = 9;         // 8 key bytes + the region digit
// A set whose four regions each hold at most kSmallMax round-1 survivors is
// sorted and SPA-scanned by one CTA per region in shared memory.
constexpr int kSmallMax = 16384;
// kStairMin / kStairSample: the default sample is min(n, 2^20, max(8192, n / 16))
constexpr Tune kTuneDefault{kSmallMax, 16, (int32_t)kStairMin, (int32_t)kStairSample, 4096, 2};
constexpr int kSpaItems = 8;
constexpr int kSpaTile = kThreads * kSpaItems;      // 2048 records
constexpr int kChainItems = 16;
constexpr int kChainBlk = kThreads * kChainItems;   // 4096 chain positions
constexpr int kOutItems = 16;
constexpr int kOutTile = kThreads * kOutItems;      // 4096 chain positions
constexpr uint32_t kIdxMask = (1u << 30) - 1;       // record value: region<<30 | local index
constexpr int64_t kMaxSetPoints = int64_t(1) << 30;

// set flags
enum : uint32_t {
  SF_FILTER = 1u,       // f64: the FP32 filter of a2 is valid for this set
  SF_WIDE = 2u,         // i32: coordinate spans need 128-bit products
  SF_STAIRS = 4u,       // the dominance prefilter is active for this set
  SF_BIG = 8u,          // some region exceeds kSmallMax survivors: multi-CTA sort
  SF_SMALL = 256u,      // float64 set with every coordinate below 2^60: FP32 views valid
  SF_SHORTVIEW = 512u,  // float64 set with every coordinate's magnitude in [2^-126, 2^60]
  SF_LOCALOUT = 1024u,  // every chain of the set fits one chain block: k_chain_local writes the output
  SF_DEGEN0 = 16u,      // bit SF_DEGEN0 << k: E_k and E_{k+1} are the same point
};

// dynamic-tile and done counters (zeroed every call)
enum : int {
  CT_CLS_TILE = 0, CT_PLAN_DONE, CT_SMALL_TOTAL,
  CT_BIG_BAR,                          // grid barrier arrivals of the multi-block kernel
  CT_SORT_TILE0,                       // + pass
  CT_SPA_TILE = CT_SORT_TILE0 + kSortPasses,
  CT_OUT_TILE, CT_OUT_DONE,
  CT_SORT_TOTAL,                       // plan results
  CT_SPA_TOTAL,
  CT_CHAIN_TOTAL,
  CT_OUT_TOTAL,
  CT_ERR,                              // first device error (negative status)
  CT_COUNT
};

// Host-built description of one point set.
struct SetDesc {
  int64_t off;          // first point of the set; also the base of its records,
                        // chain slots (+8 per earlier set) and output slots
  int64_t n;            // number of points
  int32_t chunk1;       // first a1 chunk
  int32_t nchunk1;      // a1 chunks of this set
  int32_t tile2;        // first a2 tile
  int32_t ntile2;       // a2 tiles of this set
  int32_t chunk3;       // first stairs chunk
  int32_t nchunk3;      // stairs chunks of this set
  int32_t chunkP;       // first survivor-count chunk (kPlanTiles a2 tiles each)
  int32_t nchunkP;      // survivor-count chunks of this set
};

// Per-call launch description.  A single hull carries its descriptor inline;
// a batch points at a device array.
struct Job {
  const void* pts;      // [N,2] int32 or float64, device; DT_F32: the x vector, float[N]
  const float* ys;      // DT_F32: the y vector, float[N]; nullptr otherwise
  int64_t N;            // total points
  int32_t nsets;
  int32_t dtype;
  int32_t nchunk1;      // total a1 chunks
  int32_t ntile2;       // total a2 tiles
  int32_t nchunk3;      // total stairs chunks
  int32_t nchunkP;      // total survivor-count chunks
  int64_t chunk1_len;   // a1 chunk length (points), multiple of 256
  uint32_t epoch;       // look-back flag epoch of this call (1..0xFFFF)
  uint32_t opts;        // OPT_* bits
  Tune tune;            // run-time choices (the same results with any valid choice)
  const SetDesc* sets;  // device array, or nullptr -> use `one`
  SetDesc one;
  int32_t* out_idx;     // device
  int32_t* out_counts;  // device, [nsets]
  int32_t* r1_idx;      // stage hook (set 0, or nullptr): round-1 survivors, region-major
  int32_t* r1_region;   //   and their regions 1..4
};

enum : uint32_t {
  OPT_NO_FILTER = 1u,     // force the exact path for every f64 quadrilateral test
  OPT_NO_PREFILTER = 2u,  // keep every round-1 survivor (the paper's round 1 as printed)
  OPT_BLOCKED_SPA = 4u,   // stage output: the paper's chunked GPU SPA (Sec. 2.2.2); implies OPT_NO_PREFILTER
  OPT_OCTAGON = 8u,       // round 1 discards inside the extremes' octagon (Akl-Toussaint); implies OPT_NO_PREFILTER
};

__device__ __forceinline__ SetDesc get_set(const Job& j, int s) {
  return j.sets ? j.sets[s] : j.one;
}

// Result of a1 for one chunk.
struct Part {
  uint64_t k1[4], k2[4];
  uint32_t idx[4];
  uint32_t bad;          // smallest top-word magnitude of a nonzero coordinate (float64)
  uint32_t lomag;        // the same over every coordinate, zeros included
  uint64_t dq[4];        // OPT_OCTAGON: diagonal extremes, order word of the FP32 score << 32 | index
};

// Device-resident per-set state (zeroed every call).
struct SetCtl {
  uint64_t ek1[4], ek2[4];   // a1 lexicographic keys of E1..E4
  uint64_t dq[4];            // dominance points: ~(score key << 32 | index), largest wins
  double   ex[4], ey[4];     // E1..E4 coordinates (int32 widened exactly)
  float    fA[4], fB[4], fC[4], fE[4];   // FP32 filter of edge k (f64 only)
  uint32_t eidx[4];          // set-local indices of E1..E4
  int32_t  status;
  uint32_t flags;
  uint32_t arrive1;          // a1 chunk arrivals
  uint32_t s1;               // round-1 survivors (records)
  uint32_t cnt[4];           // records per region
  uint32_t s2[4];            // SPA survivors per region
  float    slo[4], shi[4], sscale[4];  // stairs bucket map of region r: b = (u - lo) * scale
  float    bx0, bx1, by0, by1;          // dominance box (FP32 views, open; empty when zero)
  uint32_t arrive3;          // stairs chunk arrivals
  uint32_t passes;           // radix passes the multi-block sort ran for this set
  uint32_t nloc;             // SF_LOCALOUT: chain blocks (= chains) of the set
  uint32_t arrive5;          // SF_LOCALOUT: chain blocks done
  uint32_t nal[4];           // SF_LOCALOUT: output points of chain r (its kept positions but the last)
  uint32_t sb[4];            // OPT_BLOCKED_SPA: points the chunked SPA keeps per region
  // OPT_OCTAGON: vertices E1 D1 E2 D2 E3 D3 E4 D4 (D_r = E_{r+1} where the diagonal
  // extreme adds nothing) and the FP32 filter of their eight edges
  int32_t  didx[4];           // set-local index of D_r, -1 where unused
  double   ovx[8], ovy[8];
  float    oA[8], oB[8], oC[8], oE[8];
};

// SPA prefix-minimum look-back status of one tile: value words published
// before the flag word (release / acquire).
struct SpaStat {
  uint64_t agg_min;
  uint64_t inc_min;
  uint32_t flag;             // tag << 16 | kind
  uint32_t pad;
};

// Workspace (device pointers), carved from one allocation.
struct Ws {
  SetCtl* ctl;               // [nsets]
  uint32_t* ctr;             // [CT_COUNT]
  Part* part;                // [nchunk1]
  uint4* ptot;               // [nchunkP] survivors per region of a survivor-count chunk (cleared per call)
  uint64_t* tcnt;            // [ntile2 * kClsConsumers] survivors of an a2 sub-slot per region (4 x u16)
  uint32_t* small_seg;       // [4 nsets] (set, region) segments of the shared-memory path
  uint64_t* keyA; uint32_t* valA;     // [N] records (sort ping)
  uint64_t* keyB; uint32_t* valB;     // [N] records (sort pong)
  uint64_t* spvA; uint64_t* spvB;     // [N] SPA value of each record (A: region-major, B: a2 tile slots)
  uint32_t* hist;            // [nsets][kSortPasses][256]
  uint64_t* st_sort;         // [max_sort_tiles][256] look-back words
  uint32_t* sort_start;      // [nsets + 1] first sort tile of each set
  SpaStat* st_spa;           // [max_spa_tiles]
  uint64_t* st_spa_cnt;      // [max_spa_tiles] survivor-count look-back words
  uint32_t* spa_start;       // [4 nsets + 1] first SPA tile of (set, region)
  void* cpts;                // [Nc] chain points (double2 / int2)
  uint32_t* cidx;            // [Nc] chain point indices (set-local)
  uint32_t* cprev; uint32_t* cnext;   // [Nc] chain links (chain-relative)
  uint8_t* calive;           // [Nc]
  uint32_t* chain_start;     // [4 nsets + 1] first chain block of (set, region)
  int32_t* blk_head; int32_t* blk_tail;   // [max_chain_blks]
  uint32_t* out_start;       // [4 nsets + 1] first output tile of (set, region)
  uint64_t* st_out;          // [max_out_tiles]
  uint32_t* stairs;          // [nsets][4][kStairB] bucket minima, then prefix minima
};

// Chain slots of (set s, region r) when the region's records start at `rbase`
// within the set (the sum of the earlier regions' counts).
__device__ __forceinline__ int64_t chain_base_at(const SetDesc& sd, int s, int r, uint32_t rbase) {
  return sd.off + 8 * (int64_t)s + 2 * r + rbase;
}

// Chain slots of (set s, region r): base + position, positions 0 .. L-1 with
// position 0 = E_r, L-1 = E_{r+1}, 1 .. L-2 the SPA survivors in order.
__device__ __forceinline__ int64_t chain_base(const SetDesc& sd, int s, const SetCtl& c, int r) {
  int64_t b = sd.off + 8 * (int64_t)s + 2 * r;
  for (int q = 0; q < r; q++) b += c.cnt[q];
  return b;
}

// Largest i in [0, n) with a[i] <= v (a non-decreasing, a[0] <= v).
__device__ __forceinline__ int seg_of(const uint32_t* a, int n, uint32_t v) {
  int lo = 0, hi = n - 1;
  while (lo < hi) {
    int mid = (lo + hi + 1) >> 1;
    if (a[mid] <= v) lo = mid; else hi = mid - 1;
  }
  return lo;
}

// ------------------------------------------------------------ order keys
// Order-preserving unsigned keys: a < b  <=>  key(a) < key(b).
__device__ __forceinline__ uint64_t key_f64(uint64_t b) {
  if (b == 0x8000000000000000ull) b = 0;                      // -0.0 == +0.0
  return (b >> 63) ? ~b : (b | 0x8000000000000000ull);
}
__device__ __forceinline__ uint64_t key_i32(int32_t v) {
  return (uint64_t)((uint32_t)v ^ 0x80000000u);
}

// Exact float32 -> float64 widening from the IEEE 754 encodings: the sign
// moves to bit 63, a normal exponent e becomes e - 127 + 1023, the 23-bit
// significand moves to the top of the 52-bit one; a subnormal m * 2^-149 is
// normalised (its leading 1 becomes the implicit bit); zero keeps its sign;
// Inf / NaN keep exponent all-ones and the payload.  Integer operations only.
__device__ __forceinline__ double widen_f32(float f) {
  const uint32_t u = __float_as_uint(f);
  const uint64_t sign = (uint64_t)(u >> 31) << 63;
  const uint32_t e = (u >> 23) & 0xFFu, m = u & 0x7FFFFFu;
  uint64_t bits;
  if (e == 0xFFu) {
    bits = sign | (0x7FFull << 52) | ((uint64_t)m << 29);
  } else if (e != 0) {
    bits = sign | ((uint64_t)(e + 896u) << 52) | ((uint64_t)m << 29);
  } else if (m == 0) {
    bits = sign;
  } else {
    const int p = 31 - __clz((int)m);                 // leading bit of m, 0..22
    bits = sign | ((uint64_t)(p + 874) << 52) | (((uint64_t)m << (52 - p)) & ((1ull << 52) - 1));
  }
  return __longlong_as_double((long long)bits);
}

// Order-preserving key of a float32 (-0.0 -> +0.0): the float64 key of its
// widening has the same order.
__device__ __forceinline__ uint32_t key_f32(float f) {
  uint32_t u = __float_as_uint(f);
  if ((u & 0x7FFFFFFFu) == 0) u = 0;
  return u ^ ((uint32_t)((int32_t)u >> 31) | 0x80000000u);
}

// Point i of the input (set offset included) in the type the stages compute
// in: float32 vectors widen to float64.
template <typename P>
__device__ __forceinline__ P input_point(const Job& j, int64_t i);
template <>
__device__ __forceinline__ double2 input_point<double2>(const Job& j, int64_t i) {
  if (j.ys) return make_double2(widen_f32(reinterpret_cast<const float*>(j.pts)[i]), widen_f32(j.ys[i]));
  return reinterpret_cast<const double2*>(j.pts)[i];
}
template <>
__device__ __forceinline__ int2 input_point<int2>(const Job& j, int64_t i) {
  return reinterpret_cast<const int2*>(j.pts)[i];
}

// a1 domain check of a float64 coordinate: 0, or 2^-400 <= |v| < 2^400.
// Returns 1 for NaN/Inf, 2 for other out-of-range values.
__device__ __forceinline__ uint32_t f64_bad(uint64_t b) {
  uint32_t e = (uint32_t)(b >> 52) & 0x7FFu;
  if (e == 0x7FFu) return 1u;
  if ((b << 1) == 0) return 0u;
  return (e < 1023u - 400u || e > 1023u + 399u) ? 2u : 0u;
}

// float64 -> float32 by truncating the significand (integer ops only; the
// caller guarantees |v| < 2^100).  The exponent is rebiased by subtracting
// (1023 - 127) << 20 from the top word, then the top word and the three
// leading bits of the low word are funnel-shifted into place; magnitudes
// below 2^-127 become +-0 (2^-127 .. 2^-126 come out as subnormals).  The map
// is monotone non-decreasing, and |v - t| < 2^-23 |v| for |v| >= 2^-126,
// |v - t| < 2^-126 below.
__device__ __forceinline__ float f64_trunc_f32(uint64_t b) {
  const uint32_t hi = (uint32_t)(b >> 32), lo = (uint32_t)b;
  const int t = (int)(hi & 0x7FFFFFFFu) - 0x38000000;
  const uint32_t sign = hi & 0x80000000u;
  return __uint_as_float(t < 0 ? sign : (sign | __funnelshift_l(lo, (uint32_t)t, 3)));
}

// --------------------------------------------------- exact orientation
// orient(a,b,c) = sign((b-a) x (c-a)).

__device__ __forceinline__ int sgn64(long long v) { return (v > 0) - (v < 0); }

__device__ __forceinline__ int orient_i32(int ax, int ay, int bx, int by, int cx, int cy, bool wide) {
  if (!wide) {
    // spans < 2^31: each difference fits in 32 bits, each product in 62
    int dx1 = bx - ax, dy1 = by - ay, dx2 = cx - ax, dy2 = cy - ay;
    long long d = (long long)dx1 * dy2 - (long long)dy1 * dx2;
    return sgn64(d);
  }
  long long dx1 = (long long)bx - ax, dy1 = (long long)by - ay;
  long long dx2 = (long long)cx - ax, dy2 = (long long)cy - ay;
  __int128 d = (__int128)dx1 * dy2 - (__int128)dy1 * dx2;
  return (d > 0) - (d < 0);
}

// Error-free transformations (never contracted: explicit _rn intrinsics).
__device__ __forceinline__ void ef_two_sum(double a, double b, double& s, double& e) {
  s = __dadd_rn(a, b);
  double bv = __dsub_rn(s, a);
  double av = __dsub_rn(s, bv);
  e = __dadd_rn(__dsub_rn(a, av), __dsub_rn(b, bv));
}
__device__ __forceinline__ void ef_two_prod(double a, double b, double& p, double& e) {
  p = __dmul_rn(a, b);
  e = __fma_rn(a, b, -p);
}

// Exact sign of the 2x2 determinant written as differences of expansions
// (Shewchuk 1997, orient2d): det = (ax-cx)(by-cy) - (ay-cy)(bx-cx).
// Every difference is split exactly into head + tail, the eight partial
// products exactly into value + error, and the sixteen terms are summed
// with Grow-Expansion; the sign is that of the largest nonzero component.
static __device__ __noinline__ int orient_f64_exact_tail(double ax, double ay, double bx, double by,
                                                  double cx, double cy) {
  double acx, acxt, bcx, bcxt, acy, acyt, bcy, bcyt;
  ef_two_sum(ax, -cx, acx, acxt);
  ef_two_sum(bx, -cx, bcx, bcxt);
  ef_two_sum(ay, -cy, acy, acyt);
  ef_two_sum(by, -cy, bcy, bcyt);
  const double L[4] = {acx, acx, acxt, acxt}, Lb[4] = {bcy, bcyt, bcy, bcyt};
  const double R[4] = {acy, acy, acyt, acyt}, Rb[4] = {bcx, bcxt, bcx, bcxt};
  double h[17];
  int m = 0;
#pragma unroll 1
  for (int k = 0; k < 8; k++) {
    double p, e;
    if (k < 4) ef_two_prod(L[k], Lb[k], p, e);
    else { ef_two_prod(R[k - 4], Rb[k - 4], p, e); p = -p; e = -e; }
    double q = e;
#pragma unroll 1
    for (int pass = 0; pass < 2; pass++) {
      for (int i = 0; i < m; i++) {
        double s, t;
        ef_two_sum(q, h[i], s, t);
        h[i] = t;
        q = s;
      }
      h[m++] = q;
      q = p;
    }
  }
  for (int i = m - 1; i >= 0; i--) {
    if (h[i] > 0) return 1;
    if (h[i] < 0) return -1;
  }
  return 0;
}

// Exact difference of two float64 values (0, or normal) as an integer times a
// power of two: v = q * 2^e.  A nonzero value is m * 2^(E - 1075) with its
// 53-bit significand m and biased exponent E; both operands are brought to
// the smaller exponent, which needs a left shift of the other significand by
// the exponent gap.  Returns false when the gap exceeds 9 bits (then the
// shifted significands could reach 2^63 and their difference overflow).
__device__ __forceinline__ bool diff_as_int(double a, double b, long long& q, int& e) {
  const uint64_t ba = (uint64_t)__double_as_longlong(a), bb = (uint64_t)__double_as_longlong(b);
  const bool za = (ba << 1) == 0, zb = (bb << 1) == 0;
  const int ea = (int)((ba >> 52) & 0x7FF), eb = (int)((bb >> 52) & 0x7FF);
  const long long ma = (long long)((ba & 0xFFFFFFFFFFFFFull) | (1ull << 52));
  const long long mb = (long long)((bb & 0xFFFFFFFFFFFFFull) | (1ull << 52));
  const long long sa = (ba >> 63) ? -ma : ma, sb = (bb >> 63) ? -mb : mb;
  if (za && zb) { q = 0; e = 0; return true; }
  if (za) { q = -sb; e = eb; return true; }
  if (zb) { q = sa; e = ea; return true; }
  const int emin = ea < eb ? ea : eb;
  const int ga = ea - emin, gb = eb - emin;
  if (ga > 9 || gb > 9) return false;
  q = sa * (1ll << ga) - sb * (1ll << gb);     // |q| < 2 * 2^62
  e = emin;
  return true;
}

// Bit length of a nonzero unsigned 128-bit value.
__device__ __forceinline__ int bitlen_u128(unsigned __int128 v) {
  const uint64_t hi = (uint64_t)(v >> 64), lo = (uint64_t)v;
  return hi ? 128 - __clzll((long long)hi) : 64 - __clzll((long long)lo);
}

// Exact orientation in integer arithmetic only (GB300's FP64 rate is a small
// fraction of its integer rate).  With the four coordinate differences exact
// as q_i * 2^e_i (diff_as_int), det = q1 q4 2^(e1+e4) - q2 q3 2^(e2+e3) with
// products of at most 126 bits: the signs decide unless both terms have the
// same sign, then the magnitudes are compared by bit length and, when the
// lengths agree, after aligning the exponents (a shift below the 128-bit
// width).  Returns false (no result) when a difference is not representable
// that way: the caller then takes the floating-point path.
static __device__ __noinline__ bool orient_f64_int(double ax, double ay, double bx, double by, double cx,
                                                   double cy, int& sign) {
  long long q1, q2, q3, q4;
  int e1, e2, e3, e4;
  // det = (ax - cx)(by - cy) - (ay - cy)(bx - cx)
  if (!diff_as_int(ax, cx, q1, e1) || !diff_as_int(by, cy, q4, e4) || !diff_as_int(ay, cy, q2, e2) ||
      !diff_as_int(bx, cx, q3, e3))
    return false;
  const __int128 p1 = (__int128)q1 * q4, p2 = (__int128)q2 * q3;
  const int s1 = (p1 > 0) - (p1 < 0), s2 = (p2 > 0) - (p2 < 0);
  if (s1 == 0 || s2 == 0 || s1 != s2) { sign = s1 != 0 ? s1 : -s2; return true; }
  const unsigned __int128 m1 = (unsigned __int128)(s1 > 0 ? p1 : -p1);
  const unsigned __int128 m2 = (unsigned __int128)(s2 > 0 ? p2 : -p2);
  const int E1 = e1 + e4, E2 = e2 + e3;
  const int L1 = bitlen_u128(m1) + E1, L2 = bitlen_u128(m2) + E2;
  int cmp;                                    // sign of |p1| 2^E1 - |p2| 2^E2
  if (L1 != L2) {
    cmp = L1 > L2 ? 1 : -1;
  } else {
    // equal lengths: the exponent gap is the bit-length gap (< 127)
    const unsigned __int128 a1 = E1 >= E2 ? m1 << (E1 - E2) : m1;
    const unsigned __int128 a2 = E2 > E1 ? m2 << (E2 - E1) : m2;
    cmp = a1 > a2 ? 1 : a1 < a2 ? -1 : 0;
  }
  sign = s1 > 0 ? cmp : -cmp;
  return true;
}

// Exact orientation: the integer path when the coordinate differences allow
// it (close points: the usual case for the near-degenerate triples that reach
// this point), else the FP64 filter with Shewchuk's bound
// (3 + 16 eps) eps (|l| + |r|), eps = 2^-53, then the expansion.  Valid for
// coordinates that are 0 or of magnitude in [2^-400, 2^400] (no underflow or
// overflow anywhere).
__device__ __forceinline__ int orient_f64(double ax, double ay, double bx, double by,
                                          double cx, double cy) {
  int sgn;
  if (orient_f64_int(ax, ay, bx, by, cx, cy, sgn)) return sgn;
  double l = __dmul_rn(__dsub_rn(ax, cx), __dsub_rn(by, cy));
  double r = __dmul_rn(__dsub_rn(ay, cy), __dsub_rn(bx, cx));
  double d = __dsub_rn(l, r);
  double bound = __dmul_rn(3.3306690738754716e-16, __dadd_rn(fabs(l), fabs(r)));
  if (d > bound) return 1;
  if (-d > bound) return -1;
  if (l == 0.0 && r == 0.0) return 0;
  return orient_f64_exact_tail(ax, ay, bx, by, cx, cy);
}

// FP32 filter of orient(a,b,c) for float64 points given their truncated FP32
// views A, B, C (f64_trunc_f32: |t - v| <= tau |v| + eta, tau = 2^-23,
// eta = 2^-126).  With the rounded differences u1 = Bx-Ax, v1 = By-Ay,
// u2 = Cx-Ax, v2 = Cy-Ay, U their largest magnitude, M the largest view
// magnitude, mu = 2^-24, each difference is within
//   ed = 2 tau M (1 + 3 tau) + 4 eta + 1.01 mu U
// of the exact one, and det = fma(u1, v2, -(v1 u2)) is within
//   E0 = 4 ed U + 2 ed^2 + mu U^2 + mu |det|   (+ 2^-149 for underflow)
// of the exact determinant (each bound with a (1 + 2 mu) slack).  Returns
// +1 / -1 when |det| (1 - 2 mu) exceeds 1.01 E0 (the factor covers the
// rounding of E0 itself), 0 when undecided.  Views outside [2^-60, 2^60] in
// magnitude are left undecided; the caller uses the filter only for sets
// whose coordinates are all below 2^60, where the views are valid.
__device__ __forceinline__ int orient_f32_filter(float2 A, float2 B, float2 C) {
  const float M = fmaxf(fmaxf(fmaxf(fabsf(A.x), fabsf(A.y)), fmaxf(fabsf(B.x), fabsf(B.y))),
                        fmaxf(fabsf(C.x), fabsf(C.y)));
  if (!(M >= 8.6736174e-19f && M <= 1.1529215e+18f)) return 0;
  const float u1 = __fsub_rn(B.x, A.x), v1 = __fsub_rn(B.y, A.y);
  const float u2 = __fsub_rn(C.x, A.x), v2 = __fsub_rn(C.y, A.y);
  const float U = fmaxf(fmaxf(fabsf(u1), fabsf(v1)), fmaxf(fabsf(u2), fabsf(v2)));
  const float det = __fmaf_rn(u1, v2, -__fmul_rn(v1, u2));
  const float mu = 5.9604645e-08f;                   // 2^-24
  const float ed = __fadd_rn(__fmul_rn(2.3841870e-07f, M),        // 2 tau (1 + 3 tau) M, rounded up
                             __fadd_rn(4.7020e-38f, __fmul_rn(6.0200692e-08f, U)));   // 4 eta + 1.01 mu U
  const float e0 = __fadd_rn(__fadd_rn(__fmul_rn(4.f, __fmul_rn(ed, U)), __fmul_rn(2.f, __fmul_rn(ed, ed))),
                             __fadd_rn(__fmul_rn(mu, __fmul_rn(U, U)), 5.6e-45f));
  const float lhs = __fmul_rn(fabsf(det), 0.99999988f);          // (1 - 2 mu), rounded down
  if (lhs > __fmul_rn(1.01f, e0)) return det > 0.f ? 1 : -1;
  return 0;
}

// Split of a float64 coordinate into two floats, x = h + l + d: h is the
// f64_trunc_f32 view (x with its 29 low significand bits cleared), l the
// float nearest to the cleared part x - h (an integer of 29 bits scaled by
// 2^(e - 1075), converted exactly up to one rounding), so |d| <= 2^-24 |x - h|
// <= 2^-47 |x|.  Defined for x = 0 and 2^-60 <= |x| <= 2^60; otherwise h is a
// NaN, which leaves every filter below undecided.
__device__ __forceinline__ float2 f64_split(double x) {
  const uint64_t b = (uint64_t)__double_as_longlong(x);
  if ((b << 1) == 0) return make_float2(0.f, 0.f);
  const uint32_t hw = (uint32_t)(b >> 32);
  const int e = (int)((hw >> 20) & 0x7FFu);
  if (e < 1023 - 60 || e > 1023 + 60) return make_float2(__int_as_float(0x7FC00000), 0.f);
  const float scale = __uint_as_float((uint32_t)(e - 1075 + 127) << 23);   // 2^(e-1075), normal
  const float lo = __fmul_rn(__uint2float_rn((uint32_t)b & 0x1FFFFFFFu), scale);
  return make_float2(f64_trunc_f32(b), (hw & 0x80000000u) ? -lo : lo);
}

// Second FP32 filter of orient(a,b,c), on split points (h.x, h.y, l.x, l.y)
// from f64_split.  A difference of two coordinates is taken as
// D = fl(fl(Ph - Ah) + fl(Pl - Al)); with mu = 2^-24, eta = 2^-149 and M the
// largest |h| of the three points, it is within
//   e = mu (|Ph - Ah| + |Pl - Al| + |D|) + 2^-46 (1 + 2^-22) M + 3 eta
// of the exact difference (each rounding is within mu of its result or eta
// absolute; the split errors add at most 2^-47 (|P| + |A|)).  With the four
// differences U1, V1, U2, V2 and their bounds e1..e4, det = fma(U1, V2,
// -fl(V1 U2)) is within
//   E = e1 |V2| + e4 |U1| + e1 e4 + e2 |U2| + e3 |V1| + e2 e3
//       + mu |V1 U2| + mu |det| + 2 eta
// of the exact determinant.  Returns its sign when |det| (1 - 2 mu) exceeds
// 1.01 E + 2^-146 (covering the rounding and underflow of evaluating E), else
// 0.  Unlike orient_f32_filter, whose error grows with the coordinates'
// magnitude, this one is relative to the differences, so it decides the
// nearly collinear triples of closely spaced points.
__device__ __forceinline__ int orient_split_filter(float4 A, float4 B, float4 C) {
  const float mu = 5.9604645e-08f;
  const float M = fmaxf(fmaxf(fmaxf(fabsf(A.x), fabsf(A.y)), fmaxf(fabsf(B.x), fabsf(B.y))),
                        fmaxf(fabsf(C.x), fabsf(C.y)));
  const float c0 = __fmaf_ru(1.4210859e-14f, M, 4.3e-45f);          // 2^-46 (1 + 2^-22) M + 3 eta
  float e1, e2, e3, e4;
  const float U1 = __fadd_rn(__fsub_rn(B.x, A.x), __fsub_rn(B.z, A.z));
  e1 = __fmaf_ru(mu, __fadd_ru(__fadd_ru(fabsf(__fsub_rn(B.x, A.x)), fabsf(__fsub_rn(B.z, A.z))), fabsf(U1)), c0);
  const float V1 = __fadd_rn(__fsub_rn(B.y, A.y), __fsub_rn(B.w, A.w));
  e2 = __fmaf_ru(mu, __fadd_ru(__fadd_ru(fabsf(__fsub_rn(B.y, A.y)), fabsf(__fsub_rn(B.w, A.w))), fabsf(V1)), c0);
  const float U2 = __fadd_rn(__fsub_rn(C.x, A.x), __fsub_rn(C.z, A.z));
  e3 = __fmaf_ru(mu, __fadd_ru(__fadd_ru(fabsf(__fsub_rn(C.x, A.x)), fabsf(__fsub_rn(C.z, A.z))), fabsf(U2)), c0);
  const float V2 = __fadd_rn(__fsub_rn(C.y, A.y), __fsub_rn(C.w, A.w));
  e4 = __fmaf_ru(mu, __fadd_ru(__fadd_ru(fabsf(__fsub_rn(C.y, A.y)), fabsf(__fsub_rn(C.w, A.w))), fabsf(V2)), c0);
  const float p = __fmul_rn(V1, U2);
  const float det = __fmaf_rn(U1, V2, -p);
  float E = __fmul_ru(e1, fabsf(V2));
  E = __fmaf_ru(e4, fabsf(U1), E);
  E = __fmaf_ru(e1, e4, E);
  E = __fmaf_ru(e2, fabsf(U2), E);
  E = __fmaf_ru(e3, fabsf(V1), E);
  E = __fmaf_ru(e2, e3, E);
  E = __fmaf_ru(mu, __fadd_ru(fabsf(p), fabsf(det)), E);
  E = __fmaf_ru(1.01f, E, 1.5e-44f);                                // + 2 eta + 2^-146 slack
  if (__fmul_rd(fabsf(det), 0.99999988f) > E) return det > 0.f ? 1 : -1;
  return 0;
}

// Split point (h.x, h.y, l.x, l.y) of f64_split.
__device__ __forceinline__ float4 f64_split4(double2 p) {
  const float2 x = f64_split(p.x), y = f64_split(p.y);
  return make_float4(x.x, y.x, x.y, y.y);
}

// Exact orientation of float64 points from their split forms: the view
// filter, then the split filter (when `filt`: coordinates below 2^60), then
// the FP64 filter and expansion arithmetic.
__device__ __forceinline__ int orient_f64_split(double2 a, double2 b, double2 c, float4 A, float4 B,
                                                float4 C, bool filt) {
  if (filt) {
    int o = orient_f32_filter(make_float2(A.x, A.y), make_float2(B.x, B.y), make_float2(C.x, C.y));
    if (o) return o;
    o = orient_split_filter(A, B, C);
    if (o) return o;
  }
  return orient_f64(a.x, a.y, b.x, b.y, c.x, c.y);
}


// ------------------------------------------------- memory-order helpers
__device__ __forceinline__ uint64_t ld_acq_u64(const uint64_t* p) {
  uint64_t v;
  asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ uint64_t ld_rlx_u64(const uint64_t* p) {
  uint64_t v;
  asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_rel_u64(uint64_t* p, uint64_t v) {
  asm volatile("st.release.gpu.global.u64 [%0], %1;" :: "l"(p), "l"(v) : "memory");
}
__device__ __forceinline__ uint32_t ld_acq_u32(const uint32_t* p) {
  uint32_t v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_rel_u32(uint32_t* p, uint32_t v) {
  asm volatile("st.release.gpu.global.u32 [%0], %1;" :: "l"(p), "r"(v) : "memory");
}

// Packed look-back word: [epoch:16 | kind:16 | value:32]; kind 1 = tile
// aggregate, 2 = inclusive prefix.  A word from an older call or pass has a
// different epoch/kind tag and reads as "not ready".
__device__ __forceinline__ uint64_t lb_pack(uint32_t tag, uint32_t kind, uint32_t v) {
  return ((uint64_t)((tag << 16) | kind) << 32) | v;
}

constexpr uint32_t kSpinLimit = 1u << 20;   // bounded waits (well under a second per wait)

__device__ __forceinline__ void record_error(uint32_t* ctr, int st) {
  atomicCAS(reinterpret_cast<int*>(ctr + CT_ERR), 0, st);
}

// One step of a bounded wait: false once the wait must be abandoned (its own
// limit ran out, recorded as ST_TIMEOUT, or another wait of the call already
// failed).
__device__ __forceinline__ bool spin_step(uint32_t& spins, uint32_t* ctr) {
  if (++spins > kSpinLimit) {
    record_error(ctr, ST_TIMEOUT);
    return false;
  }
  if ((spins & 63u) == 0 && *(volatile uint32_t*)(ctr + CT_ERR) != 0) return false;
  __nanosleep(64);
  return true;
}

// Warp-cooperative decoupled look-back over packed count words (sum).
// Called by all 32 lanes of one warp; returns the exclusive prefix of
// `tile` over tiles [first, tile).  Tiles before `first` count as zero.
__device__ __forceinline__ uint32_t lookback_sum(const uint64_t* st, int64_t tile, int64_t first,
                                                 uint32_t tag, uint32_t* ctr) {
  const int lane = threadIdx.x & 31;
  uint32_t excl = 0;
  int64_t base = tile - 1;
  uint32_t spins = 0;
  while (base >= first) {
    int64_t t = base - lane;
    uint64_t w = 0;
    uint32_t kind = 2;
    uint32_t v = 0;
    bool done = false;
    while (!done) {
      if (t >= first) {
        w = ld_acq_u64(st + t);
        uint32_t hi = (uint32_t)(w >> 32);
        kind = (hi >> 16) == tag ? (hi & 0xFFFFu) : 0u;
        v = (uint32_t)w;
      } else {
        kind = 2; v = 0;
      }
      done = __all_sync(0xFFFFFFFFu, kind != 0);
      if (!done) {
        bool go = spin_step(spins, ctr);   // identical in every lane
        if (!__all_sync(0xFFFFFFFFu, go)) return excl;
      }
    }
    uint32_t incl = __ballot_sync(0xFFFFFFFFu, kind == 2);
    int stop = incl ? __ffs(incl) - 1 : 31;
    uint32_t add = lane <= stop ? v : 0u;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) add += __shfl_xor_sync(0xFFFFFFFFu, add, o);
    excl += add;
    if (incl) break;
    base -= 32;
  }
  return excl;
}

// SPA value of a point of region r (0..3): the compared coordinate as an
// order-preserving key in "smaller is better" form -- R1 y, R2 -x, R3 -y,
// R4 x (Fig. 2: R1 keeps y <= t, R2 x >= t, R3 y >= t, R4 x <= t).
__device__ __forceinline__ uint64_t spa_v_f64(double x, double y, int r) {
  uint64_t kx = key_f64((uint64_t)__double_as_longlong(x));
  uint64_t ky = key_f64((uint64_t)__double_as_longlong(y));
  switch (r) {
    case 0: return ky;
    case 1: return ~kx;
    case 2: return ~ky;
    default: return kx;
  }
}
__device__ __forceinline__ uint64_t spa_v_i32(int x, int y, int r) {
  uint64_t kx = key_i32(x), ky = key_i32(y);
  switch (r) {
    case 0: return ky;
    case 1: return kx ^ 0xFFFFFFFFull;
    case 2: return ky ^ 0xFFFFFFFFull;
    default: return kx;
  }
}

// ------------------------------------------------------ TMA / mbarrier
__device__ __forceinline__ uint32_t smem_addr(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" :: "r"(smem_addr(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void fence_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ void fence_mbar_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void mbar_arrive_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;"
               :: "r"(smem_addr(bar)), "r"(bytes) : "memory");
}
// 1-D bulk copy global -> shared (both 16-byte aligned, bytes % 16 == 0),
// completion signalled on `bar` as transaction bytes.
__device__ __forceinline__ void tma_load_1d(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
               :: "r"(smem_addr(dst)), "l"(src), "r"(bytes), "r"(smem_addr(bar)) : "memory");
}
// The same copy with an L2 evict-first policy: for input that a1 and a2
// stream once, so that it does not push the small survivor buffers, tables,
// control words and kernel code of the later steps out of L2.
__device__ __forceinline__ void tma_load_1d_stream(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  uint64_t pol;
  asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(pol));
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes.L2::cache_hint [%0], [%1], %2, [%3], %4;"
               :: "r"(smem_addr(dst)), "l"(src), "r"(bytes), "r"(smem_addr(bar)), "l"(pol) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile("{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
               " selp.u32 %0, 1, 0, p;\n}" : "=r"(ok) : "r"(smem_addr(bar)), "r"(parity) : "memory");
  return ok != 0;
}

// ------------------------------------------------- round-1 survivor moves
// a2 leaves the survivors of every (tile, consumer warp) sub-slot in place:
// sub-slot g of a set (g = local tile * kClsConsumers + warp) holds
// sum(tcnt[g]) records in index order, regions mixed, at
// sd.off + g * (tile points / kClsConsumers) of keyB / valB / spvB.  Chunk c
// of a set is sub-slots [c, c + 1) * kPlanTiles * kClsConsumers; ptot holds
// its per-region totals.

// Warp-cooperative, order-preserving move of the region-`rsel` survivors
// (rsel < 0: all regions) of sub-slots [g0, g1) of set s to their
// region-major records: region q's next survivor goes to record
// sd.off + roff[q] + pos[q], and pos[q] advances.  pos and roff are the same
// in every lane.  With the stage hook set (set 0 only) the moved survivors
// are also listed in j.r1_idx / j.r1_region.
__device__ __forceinline__ void move_subslots(const Job& j, const Ws& w, const SetDesc& sd, int s,
                                              int64_t g0, int64_t g1, int rsel, uint32_t pos[4],
                                              const uint32_t roff[4]) {
  const int lane = threadIdx.x & 31;
  const uint32_t lt_mask = (1u << lane) - 1u;
  const int sub = cls_tile(j.dtype) / kClsConsumers;
  const uint64_t* tc = w.tcnt + (size_t)sd.tile2 * kClsConsumers;
  const bool hook = j.r1_idx != nullptr && s == 0;
  for (int64_t gs = g0; gs < g1; gs += 32) {
    const int64_t g = gs + lane;
    const uint64_t mine = g < g1 ? tc[g] : 0ull;
    uint32_t pre[4], tot[4];
#pragma unroll
    for (int q = 0; q < 4; q++) {
      const uint32_t c = (uint32_t)(mine >> (16 * q)) & 0xFFFFu;
      uint32_t x = c;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xFFFFFFFFu, x, o);
        if (lane >= o) x += y;
      }
      pre[q] = x - c;
      tot[q] = __shfl_sync(0xFFFFFFFFu, x, 31);
    }
    const uint32_t n = (uint32_t)(mine & 0xFFFFu) + (uint32_t)((mine >> 16) & 0xFFFFu) +
                       (uint32_t)((mine >> 32) & 0xFFFFu) + (uint32_t)(mine >> 48);
    const bool want = rsel < 0 ? n != 0 : ((mine >> (16 * rsel)) & 0xFFFFull) != 0;
    const int64_t src = sd.off + g * sub;
    if (__reduce_max_sync(0xFFFFFFFFu, want ? n : 0u) <= 8u) {
      // sparse step: every lane moves its own sub-slot's few records
      uint32_t b0 = pos[0] + pre[0], b1 = pos[1] + pre[1], b2 = pos[2] + pre[2], b3 = pos[3] + pre[3];
      const uint32_t nn = want ? n : 0u;
#pragma unroll 1
      for (uint32_t i0 = 0; i0 < nn; i0 += 4) {
        uint32_t val[4];
        uint64_t key[4], spv[4];
#pragma unroll
        for (int u = 0; u < 4; u++) {
          const bool ok = i0 + u < nn;
          val[u] = ok ? w.valB[src + i0 + u] : 0u;
          key[u] = ok ? w.keyB[src + i0 + u] : 0ull;
          spv[u] = ok ? w.spvB[src + i0 + u] : 0ull;
        }
#pragma unroll
        for (int u = 0; u < 4; u++) {
          if (i0 + u >= nn) continue;
          const int r = (int)(val[u] >> 30);
          if (rsel >= 0 && r != rsel) continue;
          const uint32_t p = r == 0 ? b0 : r == 1 ? b1 : r == 2 ? b2 : b3;
          const uint32_t ro = r == 0 ? roff[0] : r == 1 ? roff[1] : r == 2 ? roff[2] : roff[3];
          b0 += r == 0; b1 += r == 1; b2 += r == 2; b3 += r == 3;
          const int64_t o = sd.off + ro + p;
          w.keyA[o] = key[u];
          w.valA[o] = val[u];
          w.spvA[o] = spv[u];
          if (hook) {
            j.r1_idx[ro + p] = (int32_t)(val[u] & kIdxMask);
            j.r1_region[ro + p] = r + 1;
          }
        }
      }
    } else {
      // dense step: the whole warp moves one sub-slot at a time (coalesced)
      uint32_t busy = __ballot_sync(0xFFFFFFFFu, want);
      while (busy) {
        const int l = __ffs(busy) - 1;
        busy &= busy - 1;
        uint32_t b[4];
#pragma unroll
        for (int q = 0; q < 4; q++) b[q] = pos[q] + __shfl_sync(0xFFFFFFFFu, pre[q], l);
        const uint32_t nl = __shfl_sync(0xFFFFFFFFu, n, l);
        const int64_t sl = sd.off + (gs + l) * sub;
#pragma unroll 2
        for (uint32_t i0 = 0; i0 < nl; i0 += 32) {
          const uint32_t i = i0 + lane;
          const bool ok = i < nl;
          // the three loads do not wait on one another
          const uint32_t val = ok ? w.valB[sl + i] : 0u;
          const uint64_t key = ok ? w.keyB[sl + i] : 0ull;
          const uint64_t spv = ok ? w.spvB[sl + i] : 0ull;
          const int r = ok ? (int)(val >> 30) : -1;
          const bool mv = rsel < 0 ? ok : r == rsel;
#pragma unroll
          for (int q = 0; q < 4; q++) {
            if (rsel >= 0 && q != rsel) continue;
            const uint32_t bq = __ballot_sync(0xFFFFFFFFu, mv && r == q);
            if (mv && r == q) {
              const uint32_t p = b[q] + __popc(bq & lt_mask);
              const int64_t o = sd.off + roff[q] + p;
              w.keyA[o] = key;
              w.valA[o] = val;
              w.spvA[o] = spv;
              if (hook) {
                j.r1_idx[roff[q] + p] = (int32_t)(val & kIdxMask);
                j.r1_region[roff[q] + p] = q + 1;
              }
            }
            b[q] += __popc(bq);
          }
        }
      }
    }
#pragma unroll
    for (int q = 0; q < 4; q++) pos[q] += tot[q];
  }
}

// ------------------------------------------- programmatic dependent launch
// The pipeline's kernels are launched with programmatic stream serialization:
// a kernel may be set up while the previous kernel of its stream runs, and
// its CTAs start as that kernel's CTAs exit.  Each of them first waits for
// the previous kernel to complete and its writes to be visible (griddep_enter;
// it returns at once when there is no such dependency), touching no memory
// before, so only the launch latency and the tail of the previous kernel are
// overlapped.  (Letting successors be scheduled from the start of a kernel,
// griddepcontrol.launch_dependents, measured slower: their CTAs queue for
// resources the running kernel holds.)
__device__ __forceinline__ void griddep_enter() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
// The one exception: a1 lets k_stairs be scheduled once its tiles are in
// flight (griddep_release, from the producer after its last copy and from
// the consumers after their loops), and k_stairs reduces its sample --
// input points only -- before its griddep_enter, while a1's last CTA sets
// the set up.  Every k_stairs CTA passes its griddep_enter before it exits,
// so k_stairs completes after a1 and a2's wait covers both.
__device__ __forceinline__ void griddep_release() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

template <typename... KArgs, typename... Args>
inline cudaError_t launch_pdl(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t st,
                              Args... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kernel, args...);
}

// ------------------------------------------------------------ launchers
// (defined in the kernel translation units, called from the API)
struct Launch {
  cudaStream_t stream;
  int grid_cap;          // persistent-grid CTA cap (SMs x resident CTAs)
  int cls_grid;          // a2 CTAs (2 per SM)
};

// Each returns the number of kernels it launched.
int launch_extremes(const Job& j, const Ws& w, const Launch& L);
int launch_stairs(const Job& j, const Ws& w, const Launch& L);
int launch_classify(const Job& j, const Ws& w, const Launch& L);
int launch_gather(const Job& j, const Ws& w, const Launch& L);
int launch_small(const Job& j, const Ws& w, const Launch& L);
int launch_big(const Job& j, const Ws& w, const Launch& L);
int launch_chain(const Job& j, const Ws& w, const Launch& L);
// stage extraction (cch_hull_stages)
void launch_extract_spa(const Job& j, const Ws& w, int32_t* spa_idx, cudaStream_t st);
int launch_spa_blocked(const Job& j, const Ws& w, int32_t* spa_idx, cudaStream_t st);
int extremes_blocks_per_sm(int dtype);
void count_launches(uint64_t n);   // add to the library's launch counter (cch_launch_count)
Tune tune_for(int dtype, int64_t npts, int32_t nsets);   // run-time choices of a call (tune.cu)
int tune_bucket(int64_t npts, int32_t nsets);
void serve_release_pinned();   // free the server's pooled pinned host buffers

}  // namespace cch

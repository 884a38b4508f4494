// k_small.cu -- steps 4-5 (Table 1 sort, Fig. 2 SPA) for sets whose regions
// each hold at most kSmallMax round-1 survivors: one CTA per (set, region)
// segment, everything in shared memory.
//
//  1. Fine dominance filter.  Two bucket tables per region, each over a map
//     that is non-decreasing in its order key (FP32 view of the coordinate,
//     scaled linearly between the region's two extremes; for float64 sets
//     with coordinates beyond 2^60 the key bits themselves, shifted): table A
//     buckets the sort key and keeps the per-bucket minimum of the leading
//     32 bits of the SPA value, table B buckets the SPA value and keeps the
//     minimum of the sort key's.  Exclusive prefix minima over the buckets
//     (table A seeded with the region's first extreme) then drop every
//     candidate that some point strictly before it in the sort order beats
//     strictly in the SPA value: such a candidate is not an SPA survivor
//     (Fig. 2).  Table A alone is weak where the region's boundary runs
//     nearly parallel to the compared axis (near E_r, where many candidates
//     share a bucket of the sort key); table B covers that stretch.
//  2. Sort of the kept candidates (Table 1 order: key, then index).
//     Counting path: the kept candidates are counted per bucket, the counts
//     are scanned into bucket starts, and every candidate ranks itself among
//     the few others of its bucket by (key, index) -- the bucket map being
//     monotone, (bucket, rank) is the sorted order.  Radix path, taken when
//     a bucket holds more than kOccMax candidates (many equal or nearly
//     equal coordinates): a stable LSD radix sort over the key bytes that
//     vary (8-bit digits, warp-level ranking with match.any, one scatter of
//     16-bit positions through shared memory per pass) of the candidates in
//     index order.
//  3. SPA proper: exclusive prefix minimum of the exact SPA value over the
//     sorted order, seeded with the first extreme; the survivors go, in
//     order, to the region's chain slots.
//  Record path.  The candidates sit in index order, the sort visits them in
//  key order, so every later read of a candidate's key or SPA value is a
//  random gather from L2.  The keep test reads both in order anyway: it
//  also writes each kept candidate's record (key, SPA value, candidate
//  number), in keep order, to the (by then unused) second record buffers.
//  When at most kRecMax candidates are kept and the counting path applies,
//  the records come back into shared memory in one sequential copy, and
//  steps 2a and 3 read only shared memory; the output gathers only the
//  survivors' point indices.
//  Cluster form (CL = 8 CTAs per (set, region), for calls of a few sets, on
//  regions of at least kSplitMin candidates; smaller regions are left to the
//  leader CTA alone): every CTA of the cluster builds the two tables over
//  its own slice of the candidates, the copies are merged through distributed
//  shared memory (each CTA takes the minimum of one slice of the words over
//  the eight copies and writes it back to all of them), and every CTA takes
//  the prefix minima and runs the keep test on its slice, listing its kept
//  candidates, their bucket counts and index-order bits in the leader's
//  shared memory.  The leader then sorts and scans as above.
#include <cooperative_groups.h>
#include <type_traits>

#include "cch_internal.cuh"

namespace cch {

constexpr int kSmThreads = 512;
constexpr int kSmWarps = kSmThreads / 32;
constexpr int kSmItems = kSmallMax / kSmThreads;   // at most 32 candidates per thread
constexpr int kFineB = 16384;                      // fine buckets of the sort key per region
constexpr int kFineB2 = 8192;                      // fine buckets of the SPA value per region
constexpr int kOccMax = 32;                        // largest bucket the counting path ranks
constexpr int kRecMax = 4096;                      // most kept candidates the record path holds
constexpr int kSmCluster = 8;                      // CTAs per (set, region) in the cluster form
constexpr int kSmClusterSets = 4;                  // calls of at most this many sets take the cluster form
constexpr uint32_t kSplitMin = 4096;               // smallest region the cluster splits
// Dynamic shared memory, overlays of one 200 KB block (tables padded by one
// word in 32):
//   filter         table A u32 | table B u32 | kept-candidate list u16 (its
//                  tail reaches into sposA) ... bucket counts, then starts,
//                  u16 pairs, over sposB and the histograms
//   counting path  bucket members u16 from 0 (tables dead by then)
//   radix path     [0, 128K) keys u64 (tables, list and counts dead by then)
//   record path    membR u16 [0, 8K) | rk u64 [8K, 40K) | rv u64 [40K, 72K) |
//                  ri u32 [72K, 88K): the kept candidates' records (sort key,
//                  SPA value, candidate number) in keep order (at most
//                  kRecMax; the tables are dead by then)
//   both           [128K, 160K) sposA u16 (sorted positions) | [160K, 192K)
//                  sposB u16 | [192K, 200K) per-warp digit histograms;
//                  step 3 overwrites [0, 128K) with SPA values in sorted order
//                  (not on the record path) and lists the survivors in the
//                  free position buffer
constexpr size_t kSmSmem = (size_t)kSmallMax * (8 + 2 + 2) + (size_t)kSmWarps * 256 * 2;
constexpr int kPadA = kFineB + kFineB / 32;       // padded table words
constexpr int kPadB = kFineB2 + kFineB2 / 32;
constexpr int kPadC = kFineB / 2 + kFineB / 64;   // padded u16-pair count words
static_assert((size_t)(kPadA + kPadB) * 4 + (size_t)kSmallMax * 2 <= (size_t)kSmallMax * 10,
              "tables and the kept list end before the second position buffer");
static_assert((size_t)kPadC * 4 <= (size_t)kSmallMax * 2 + (size_t)kSmWarps * 256 * 2,
              "bucket counts fit the second position buffer and the histograms");
static_assert((size_t)kRecMax * (2 + 8 + 8 + 4) <= (size_t)(kPadA + kPadB) * 4,
              "records end before the kept-candidate list");

template <int DT>
__device__ __forceinline__ uint64_t spa_value_of(const typename std::conditional<DT == DT_F64, double2, int2>::type& p,
                                                 int r) {
  if constexpr (DT == DT_F64) return spa_v_f64(p.x, p.y, r);
  else return spa_v_i32(p.x, p.y, r);
}

// Table 1 sort key of a point for region r (0..3), as written by a2.
template <int DT>
__device__ __forceinline__ uint64_t region_sort_key(const typename std::conditional<DT == DT_F64, double2, int2>::type& p,
                                                    int r) {
  uint64_t kx, ky, msk;
  if constexpr (DT == DT_F64) {
    kx = key_f64((uint64_t)__double_as_longlong(p.x));
    ky = key_f64((uint64_t)__double_as_longlong(p.y));
    msk = ~0ull;
  } else {
    kx = key_i32(p.x);
    ky = key_i32(p.y);
    msk = 0xFFFFFFFFull;
  }
  switch (r) {
    case 0: return kx;
    case 1: return ky;
    case 2: return kx ^ msk;
    default: return ky ^ msk;
  }
}

// The point behind a record of region r: its sort key and SPA value are the
// order keys of its two coordinates (Table 1), so both invert exactly (a
// float64 -0.0 comes back as +0.0, the same coordinate).
template <int DT>
__device__ __forceinline__ typename std::conditional<DT == DT_F64, double2, int2>::type
point_from_keys(uint64_t key, uint64_t v, int r) {
  const bool kd = r >= 2, vd = r == 1 || r == 2;   // complemented keys
  typename std::conditional<DT == DT_F64, double2, int2>::type p;
  if constexpr (DT == DT_F64) {
    const uint64_t a = kd ? ~key : key, b = vd ? ~v : v;
    const double ca = __longlong_as_double((long long)((a >> 63) ? (a & 0x7FFFFFFFFFFFFFFFull) : ~a));
    const double cb = __longlong_as_double((long long)((b >> 63) ? (b & 0x7FFFFFFFFFFFFFFFull) : ~b));
    if (r & 1) { p.x = cb; p.y = ca; } else { p.x = ca; p.y = cb; }
  } else {
    const int ca = (int)((uint32_t)key ^ (kd ? 0xFFFFFFFFu : 0u) ^ 0x80000000u);
    const int cb = (int)((uint32_t)v ^ (vd ? 0xFFFFFFFFu : 0u) ^ 0x80000000u);
    if (r & 1) { p.x = cb; p.y = ca; } else { p.x = ca; p.y = cb; }
  }
  return p;
}

// FP32 view of the coordinate behind an order key (key_f64 / key_i32 of x or
// y, complemented when `desc`), negated when `desc`: non-decreasing in the key.
template <int DT>
__device__ __forceinline__ float key_view(uint64_t key, bool desc) {
  float v;
  if constexpr (DT == DT_F64) {
    const uint64_t k = desc ? ~key : key;                                 // key_f64 of the coordinate
    const uint64_t b = (k >> 63) ? (k & 0x7FFFFFFFFFFFFFFFull) : ~k;      // its bits
    v = f64_trunc_f32(b);
  } else {
    const uint32_t k = (uint32_t)key ^ (desc ? 0xFFFFFFFFu : 0u);
    v = __int2float_rn((int)(k ^ 0x80000000u));
  }
  return desc ? -v : v;
}

// The 32 leading significant bits of an order key (all of an int32 key).
template <int DT>
__device__ __forceinline__ uint32_t key_hi(uint64_t key) {
  return DT == DT_F64 ? (uint32_t)(key >> 32) : (uint32_t)key;
}

// Bucket map of an order key onto NB buckets between the keys of two
// points, non-decreasing in the key: the FP32 view scaled linearly, or (for
// float64 sets with coordinates beyond 2^60, whose FP32 views overflow) the
// key bits themselves, shifted.
template <int NB>
struct FineMap {
  uint64_t klo;
  float lo, sc;
  int shift;
  bool fp, desc;
  template <int DT>
  __device__ __forceinline__ void init(uint64_t ka, uint64_t kb, bool use_fp, bool dsc) {
    klo = ka;
    desc = dsc;
    fp = use_fp;
    const uint64_t span = kb > ka ? kb - ka : 0;
    shift = span == 0 ? 0 : max(0, 64 - __clzll((long long)span) - (31 - __clz(NB)));
    lo = key_view<DT>(ka, dsc);
    const float d = __fsub_rn(key_view<DT>(kb, dsc), lo);
    const float s = d > 0.f ? __fdiv_rn((float)NB, d) : 0.f;
    sc = s <= 1.0e38f ? s : 1.0e38f;
  }
  template <int DT>
  __device__ __forceinline__ uint32_t bucket(uint64_t key) const {
    if (fp) {
      const float t = __fmul_rn(__fsub_rn(key_view<DT>(key, desc), lo), sc);
      return (uint32_t)min(max(__float2int_rd(t), 0), NB - 1);
    }
    const uint64_t d = key > klo ? (key - klo) >> shift : 0ull;
    return (uint32_t)min(d, (uint64_t)(NB - 1));
  }
};

// Padded index of a table word: one spare word after every 32, so that a
// warp whose lanes walk contiguous per-thread chunks of 16 or 32 words hits
// 32 different banks at every step.
__device__ __forceinline__ uint32_t pad32(uint32_t b) { return b + (b >> 5); }

// Exclusive prefix minimum over a padded table of kSmThreads * PER words
// (thread t owns words t*PER .. t*PER+PER-1), seeded.
template <int PER>
__device__ __forceinline__ void prefix_min_excl(uint32_t* t, uint32_t seed, uint32_t* wsum) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  uint32_t loc = 0xFFFFFFFFu;
#pragma unroll
  for (int qq = 0; qq < PER; qq++) loc = min(loc, t[pad32(tid * PER + qq)]);
  uint32_t x = loc;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t y = __shfl_up_sync(0xFFFFFFFFu, x, o);
    if (lane >= o) x = min(x, y);
  }
  if (lane == 31) wsum[warp] = x;
  __syncthreads();
  uint32_t run = __shfl_up_sync(0xFFFFFFFFu, x, 1);
  if (lane == 0) run = 0xFFFFFFFFu;
  for (int qq = 0; qq < warp; qq++) run = min(run, wsum[qq]);
  run = min(run, seed);
#pragma unroll
  for (int qq = 0; qq < PER; qq++) {
    const uint32_t a = pad32(tid * PER + qq);
    const uint32_t v = t[a];
    t[a] = run;
    run = min(run, v);
  }
}

template <int DT, int CL>
__global__ void __launch_bounds__(kSmThreads, 1) k_small(Job j, Ws w) {
  griddep_enter();
  namespace cg = cooperative_groups;
  using P = typename std::conditional<DT == DT_F64, double2, int2>::type;
  extern __shared__ __align__(16) unsigned char smem[];
  uint32_t* vminA = reinterpret_cast<uint32_t*>(smem);                           // table A (padded)
  uint32_t* vminB = vminA + kPadA;                                               // table B (padded)
  uint16_t* klist = reinterpret_cast<uint16_t*>(vminB + kPadB);                  // kept candidates
  uint16_t* memb = reinterpret_cast<uint16_t*>(smem);                            // by bucket; tables dead
  uint64_t* skey = reinterpret_cast<uint64_t*>(smem);                            // [kSmallMax]
  uint16_t* sposA = reinterpret_cast<uint16_t*>(smem + (size_t)kSmallMax * 8);
  uint16_t* sposB = sposA + kSmallMax;
  uint32_t* bcnt = reinterpret_cast<uint32_t*>(sposB);                           // u16 pairs (padded)
  uint16_t* whist = sposB + kSmallMax;                                           // [kSmWarps][256]
  __shared__ uint32_t keepw[kSmallMax / 32];   // kept candidates, bit i%32 of word i/32
  __shared__ uint32_t doff[256];
  __shared__ uint32_t wsum[kSmWarps], wmx[kSmWarps];
  __shared__ uint64_t wor[kSmWarps], wand[kSmWarps], wmin[kSmWarps];
  __shared__ uint32_t sh_cnt[kSmWarps];
  __shared__ uint32_t sh_nk;

  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const uint32_t lt_mask = (1u << lane) - 1u;
  const uint32_t total = w.ctr[CT_SMALL_TOTAL];
  const uint32_t rank = blockIdx.x % CL;           // CTA within the cluster (clusters are consecutive CTAs)
  // the leader's lists (this CTA's own without a cluster)
  uint16_t* klistL = klist;
  uint32_t* bcntL = bcnt;
  uint32_t* keepwL = keepw;
  uint32_t* nkL = &sh_nk;
  if constexpr (CL > 1) {
    cg::cluster_group cl = cg::this_cluster();
    klistL = cl.map_shared_rank(klist, 0);
    bcntL = cl.map_shared_rank(bcnt, 0);
    keepwL = cl.map_shared_rank(keepw, 0);
    nkL = cl.map_shared_rank(&sh_nk, 0);
  }

  for (uint32_t q = blockIdx.x / CL; q < total; q += gridDim.x / CL) {
    const uint32_t g = w.small_seg[q];
    const int s = (int)(g >> 2), r = (int)(g & 3);
    const SetDesc sd = get_set(j, s);
    const SetCtl& c = w.ctl[s];
    const uint32_t m = c.cnt[r];
    uint32_t rbase = 0;
    for (int qq = 0; qq < r; qq++) rbase += c.cnt[qq];
    const uint64_t* kin = w.keyA + sd.off + rbase;
    const uint32_t* vin = w.valA + sd.off + rbase;
    const uint64_t* vv = w.spvA + sd.off + rbase;
    P e, e1;
    {
      const int r1 = (r + 1) & 3;
      if constexpr (DT == DT_F64) {
        e.x = c.ex[r]; e.y = c.ey[r]; e1.x = c.ex[r1]; e1.y = c.ey[r1];
      } else {
        e.x = (int)c.ex[r]; e.y = (int)c.ey[r]; e1.x = (int)c.ex[r1]; e1.y = (int)c.ey[r1];
      }
    }
    const uint64_t v0 = spa_value_of<DT>(e, r);
    // this CTA's candidates [lo, hi) (all of them without a cluster, or on a
    // region the cluster does not split -- the same decision in every CTA);
    // the slices start on multiples of 32 (one keepw word per warp and step)
    const bool split = CL > 1 && m >= kSplitMin;
    if (CL > 1 && !split && rank != 0) continue;
    const uint32_t chunk = split ? (m + CL * 32 - 1) / (CL * 32) * 32 : m;
    const uint32_t lo = min(m, rank * chunk), hi = min(m, lo + chunk);

    // ---- 1. fine dominance filter ------------------------------------
    // Table A: buckets of the sort key (every candidate's key lies between
    // those of E_r and E_{r+1}), per-bucket minimum of the SPA value.
    // Table B: buckets of the SPA value (between those of E_{r+1} and E_r),
    // per-bucket minimum of the sort key.  A candidate beaten in either
    // table by an entry of a strictly earlier bucket has a point strictly
    // before it in the sort order with a strictly smaller SPA value.
    FineMap<kFineB> fa;
    FineMap<kFineB2> fb;
    {
      const bool fp = DT == DT_I32 || (c.flags & SF_SMALL);
      fa.init<DT>(region_sort_key<DT>(e, r), region_sort_key<DT>(e1, r), fp, r >= 2);
      fb.init<DT>(spa_value_of<DT>(e1, r), v0, fp, r == 1 || r == 2);
    }
    for (int i = tid; i < kPadA + kPadB; i += kSmThreads) vminA[i] = 0xFFFFFFFFu;
    if (rank == 0) {
      for (int i = tid; i < kPadC; i += kSmThreads) bcnt[i] = 0u;
      for (int i = tid; i < kSmallMax / 32; i += kSmThreads) keepw[i] = 0u;
      if (tid == 0) sh_nk = 0;
    }
    if (split) cg::this_cluster().sync();   // the leader's tables and lists are clear
    else __syncthreads();
#pragma unroll 1
    for (uint32_t i0 = lo; i0 < hi; i0 += kSmThreads * 8) {
      uint64_t kk[8], va[8];
#pragma unroll
      for (int u = 0; u < 8; u++) {
        const uint32_t i = i0 + u * kSmThreads + tid;
        kk[u] = i < hi ? kin[i] : 0ull;
        va[u] = i < hi ? vv[i] : 0ull;
      }
#pragma unroll
      for (int u = 0; u < 8; u++) {
        if (i0 + u * kSmThreads + tid < hi) {
          atomicMin(&vminA[pad32(fa.bucket<DT>(kk[u]))], key_hi<DT>(va[u]));
          atomicMin(&vminB[pad32(fb.bucket<DT>(va[u]))], key_hi<DT>(kk[u]));
        }
      }
    }
    if (split) {
      // merge the cluster's tables: this CTA takes 16-byte groups [q0, q1)
      // of the (contiguous) two tables, minimum over the eight copies,
      // written back to every copy
      cg::cluster_group cl = cg::this_cluster();
      cl.sync();
      static_assert((kPadA + kPadB) % 4 == 0, "the tables are whole 16-byte groups");
      constexpr uint32_t W4 = (kPadA + kPadB) / 4, S4 = (W4 + CL - 1) / CL;
      const uint32_t q0 = rank * S4, q1 = min(W4, q0 + S4);
      uint4* t4 = reinterpret_cast<uint4*>(vminA);
      for (uint32_t x = q0 + tid; x < q1; x += kSmThreads) {
        uint4 v[CL];
#pragma unroll
        for (int c = 0; c < CL; c++) v[c] = cl.map_shared_rank(t4, c)[x];
        uint4 mn = v[0];
#pragma unroll
        for (int c = 1; c < CL; c++) {
          mn.x = min(mn.x, v[c].x); mn.y = min(mn.y, v[c].y);
          mn.z = min(mn.z, v[c].z); mn.w = min(mn.w, v[c].w);
        }
#pragma unroll
        for (int c = 0; c < CL; c++) cl.map_shared_rank(t4, c)[x] = mn;
      }
      cl.sync();
    } else {
      __syncthreads();
    }
    // exclusive prefix minima over the buckets; table A is seeded with E_r
    prefix_min_excl<kFineB / kSmThreads>(vminA, key_hi<DT>(v0), wsum);
    __syncthreads();
    prefix_min_excl<kFineB2 / kSmThreads>(vminB, 0xFFFFFFFFu, wmx);
    __syncthreads();
    // keep test: kept candidates are listed (any order), marked in keepw
    // (index order), counted per bucket of table A and their records
    // written in list order
    uint64_t* rkG = w.keyB + sd.off + rbase;
    uint64_t* rvG = w.spvB + sd.off + rbase;
    uint32_t* riG = w.valB + sd.off + rbase;
#pragma unroll 1
    for (uint32_t i0 = lo; i0 < hi; i0 += kSmThreads * 8) {
      uint64_t kk[8], va[8];
#pragma unroll
      for (int u = 0; u < 8; u++) {
        const uint32_t i = i0 + u * kSmThreads + tid;
        kk[u] = i < hi ? kin[i] : 0ull;
        va[u] = i < hi ? vv[i] : 0ull;
      }
#pragma unroll
      for (int u = 0; u < 8; u++) {
        const uint32_t i = i0 + u * kSmThreads + tid;
        bool keep = false;
        uint32_t b = 0;
        if (i < hi) {
          b = fa.bucket<DT>(kk[u]);
          keep = key_hi<DT>(va[u]) <= vminA[pad32(b)] &&
                 key_hi<DT>(kk[u]) <= vminB[pad32(fb.bucket<DT>(va[u]))];
        }
        const uint32_t bal = __ballot_sync(0xFFFFFFFFu, keep);
        if (bal) {
          uint32_t base = 0;
          if (lane == 0) {
            keepwL[(i0 + u * kSmThreads) / 32 + warp] = bal;
            base = atomicAdd(nkL, (uint32_t)__popc(bal));
          }
          base = __shfl_sync(0xFFFFFFFFu, base, 0);
          if (keep) {
            const uint32_t pos = base + __popc(bal & lt_mask);
            klistL[pos] = (uint16_t)i;
            atomicAdd(&bcntL[pad32(b >> 1)], 1u << ((b & 1u) * 16u));
            if (pos < kRecMax) { rkG[pos] = kk[u]; rvG[pos] = va[u]; riG[pos] = i; }
          }
        }
      }
    }
    if (split) {
      cg::this_cluster().sync();      // every kept candidate is listed at the leader
      if (rank != 0) continue;        // the leader sorts and scans
    } else {
      __syncthreads();
    }
    // exclusive scan of the bucket counts into bucket starts (in place, u16)
    uint32_t m2 = 0, maxocc = 0;
    {
      constexpr int wpt = kFineB / 2 / kSmThreads;    // count words per thread
      uint32_t loc[wpt];
      uint32_t sum = 0, mx = 0;
#pragma unroll
      for (int qq = 0; qq < wpt; qq++) {
        loc[qq] = bcnt[pad32(tid * wpt + qq)];
        const uint32_t a = loc[qq] & 0xFFFFu, b = loc[qq] >> 16;
        sum += a + b;
        mx = max(mx, max(a, b));
      }
      uint32_t x = sum;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xFFFFFFFFu, x, o);
        if (lane >= o) x += y;
      }
      mx = __reduce_max_sync(0xFFFFFFFFu, mx);
      if (lane == 31) wsum[warp] = x;
      if (lane == 0) wmx[warp] = mx;
      __syncthreads();
      uint32_t pre = x - sum;
      for (int qq = 0; qq < kSmWarps; qq++) {
        if (qq < warp) pre += wsum[qq];
        m2 += wsum[qq];
        maxocc = max(maxocc, wmx[qq]);
      }
#pragma unroll
      for (int qq = 0; qq < wpt; qq++) {
        const uint32_t a = loc[qq] & 0xFFFFu, b = loc[qq] >> 16;
        bcnt[pad32(tid * wpt + qq)] = pre | ((pre + a) << 16);
        pre += a + b;
      }
    }
    __syncthreads();

    uint16_t* pin = sposA;
    // record path: pin holds record numbers (keep order), else candidate
    // numbers (index order)
    const bool rec = maxocc <= kOccMax && m2 <= kRecMax;
    uint16_t* membR = reinterpret_cast<uint16_t*>(smem);
    uint64_t* rk = reinterpret_cast<uint64_t*>(smem + (size_t)kRecMax * 2);
    uint64_t* rv = rk + kRecMax;
    uint32_t* ri = reinterpret_cast<uint32_t*>(rv + kRecMax);
    if (rec) {
      // ---- 2a'. counting path on the records ----------------------------
      for (uint32_t t = tid; t < m2; t += kSmThreads) {
        rk[t] = rkG[t];
        rv[t] = rvG[t];
        ri[t] = riG[t];
      }
      __syncthreads();
#pragma unroll 1
      for (uint32_t t = tid; t < m2; t += kSmThreads) {
        const uint32_t b = fa.bucket<DT>(rk[t]);
        const uint32_t sh = (b & 1u) * 16u;
        const uint32_t old = atomicAdd(&bcnt[pad32(b >> 1)], 1u << sh);
        membR[(old >> sh) & 0xFFFFu] = (uint16_t)t;
      }
      __syncthreads();
      // rank within the bucket by (key, index)
#pragma unroll 1
      for (uint32_t t = tid; t < m2; t += kSmThreads) {
        const uint32_t x = membR[t];
        const uint64_t ki = rk[x];
        const uint32_t ii = ri[x];
        const uint32_t b = fa.bucket<DT>(ki);
        const uint32_t en = (bcnt[pad32(b >> 1)] >> ((b & 1u) * 16u)) & 0xFFFFu;
        const uint32_t st = b ? (bcnt[pad32((b - 1) >> 1)] >> (((b - 1) & 1u) * 16u)) & 0xFFFFu : 0u;
        uint32_t rkx = 0;
        for (uint32_t p = st; p < en; p++) {
          const uint32_t y = membR[p];
          if (y != x) {
            const uint64_t kj = rk[y];
            rkx += (kj < ki) || (kj == ki && ri[y] < ii);
          }
        }
        sposA[st + rkx] = (uint16_t)x;
      }
      __syncthreads();
    } else if (maxocc <= kOccMax) {
      // ---- 2a. counting path ------------------------------------------
      // scatter by bucket: the starts become cursors, then bucket ends
#pragma unroll 1
      for (uint32_t t = tid; t < m2; t += kSmThreads) {
        const uint32_t i = klist[t];
        const uint32_t b = fa.bucket<DT>(kin[i]);
        const uint32_t sh = (b & 1u) * 16u;
        const uint32_t old = atomicAdd(&bcnt[pad32(b >> 1)], 1u << sh);
        memb[(old >> sh) & 0xFFFFu] = (uint16_t)i;
      }
      __syncthreads();
      // rank within the bucket by (key, index); bucket b spans
      // [end(b-1), end(b)) of memb
#pragma unroll 1
      for (uint32_t t = tid; t < m2; t += kSmThreads) {
        const uint32_t i = memb[t];
        const uint64_t ki = kin[i];
        const uint32_t b = fa.bucket<DT>(ki);
        const uint32_t en = (bcnt[pad32(b >> 1)] >> ((b & 1u) * 16u)) & 0xFFFFu;
        const uint32_t st = b ? (bcnt[pad32((b - 1) >> 1)] >> (((b - 1) & 1u) * 16u)) & 0xFFFFu : 0u;
        uint32_t rk = 0;
        for (uint32_t p = st; p < en; p++) {
          const uint32_t jj = memb[p];
          if (jj != i) {
            const uint64_t kj = kin[jj];
            rk += (kj < ki) || (kj == ki && jj < i);
          }
        }
        sposA[st + rk] = (uint16_t)i;
      }
      __syncthreads();
    } else {
      // ---- 2b. radix path: candidates tid*32 .. +32 in index order -----
      const uint32_t c0 = tid * kSmItems;
      const uint32_t keep = keepw[tid];
      const uint32_t nk = __popc(keep);
      uint32_t cx = nk;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xFFFFFFFFu, cx, o);
        if (lane >= o) cx += y;
      }
      if (lane == 31) sh_cnt[warp] = cx;
      __syncthreads();
      uint32_t rank = cx - nk;
      for (int qq = 0; qq < warp; qq++) rank += sh_cnt[qq];
      uint64_t kor = 0, kand = ~0ull;
      for (int k = 0; k < kSmItems; k++) {
        if ((keep >> k) & 1u) {
          const uint64_t key = kin[c0 + k];
          skey[c0 + k] = key;
          sposA[rank++] = (uint16_t)(c0 + k);
          kor |= key;
          kand &= key;
        }
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        kor |= __shfl_xor_sync(0xFFFFFFFFu, kor, o);
        kand &= __shfl_xor_sync(0xFFFFFFFFu, kand, o);
      }
      if (lane == 0) { wor[warp] = kor; wand[warp] = kand; }
      __syncthreads();
      uint64_t diff;
      {
        uint64_t a = 0, b = ~0ull;
        for (int qq = 0; qq < kSmWarps; qq++) { a |= wor[qq]; b &= wand[qq]; }
        diff = a ^ b;   // bits that vary among the kept candidates
      }
      // the first nw warps own positions w*per*32 .. +per*32, item k of lane
      // l is position w*per*32 + k*32 + l, so (warp, item, lane) is position
      // order; few candidates -> few ranking warps (shorter digit prefixes)
      const int nw = (int)min((uint32_t)kSmWarps, max(1u, (m2 + 255) / 256));
      const int per = (int)((m2 + nw * 32 - 1) / (nw * 32));
      uint16_t* pout = sposB;
      for (int p = 0; p < 8; p++) {
        if (((diff >> (8 * p)) & 0xFFull) == 0) continue;     // uniform
        for (int i = tid; i < nw * 256; i += kSmThreads) whist[i] = 0;
        __syncthreads();
        uint32_t pr[kSmItems];     // pos | rank << 14 | digit << 24
        if (warp < nw) {
#pragma unroll
          for (int k = 0; k < kSmItems; k++) {
            if (k < per) {
              const uint32_t i = (uint32_t)(warp * per * 32 + k * 32 + lane);
              const bool ok = i < m2;
              const uint32_t pos = ok ? pin[i] : 0u;
              const uint32_t d = ok ? (uint32_t)(skey[pos] >> (8 * p)) & 0xFFu : 256u;
              const uint32_t peers = __match_any_sync(0xFFFFFFFFu, d);
              const uint32_t prior = d < 256 ? whist[warp * 256 + d] : 0u;
              __syncwarp();
              if (d < 256 && lane == __ffs(peers) - 1) whist[warp * 256 + d] = (uint16_t)(prior + __popc(peers));
              __syncwarp();
              pr[k] = pos | ((prior + __popc(peers & lt_mask)) << 14) | ((d & 0xFFu) << 24);
            }
          }
        }
        __syncthreads();
        if (tid < 256) {
          uint32_t run = 0;
          for (int qq = 0; qq < nw; qq++) {
            const uint32_t cc = whist[qq * 256 + tid];
            whist[qq * 256 + tid] = (uint16_t)run;
            run += cc;
          }
          uint32_t x = run;
#pragma unroll
          for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(0xFFFFFFFFu, x, o);
            if (lane >= o) x += y;
          }
          if (lane == 31) wsum[warp] = x;
          doff[tid] = x - run;
        }
        __syncthreads();
        if (tid < 256) {
          uint32_t pre = 0;
          for (int qq = 0; qq < warp; qq++) pre += wsum[qq];
          doff[tid] += pre;
        }
        __syncthreads();
        if (warp < nw) {
#pragma unroll
          for (int k = 0; k < kSmItems; k++) {
            if (k < per) {
              const uint32_t i = (uint32_t)(warp * per * 32 + k * 32 + lane);
              if (i < m2) {
                const uint32_t d = pr[k] >> 24;
                pout[doff[d] + whist[warp * 256 + d] + ((pr[k] >> 14) & 0x3FFu)] = (uint16_t)(pr[k] & 0x3FFFu);
              }
            }
          }
        }
        __syncthreads();
        uint16_t* t = pin; pin = pout; pout = t;
      }
    }

    // ---- 3. SPA over the sorted order (pin) ----------------------------
    const int per2 = (int)((m2 + kSmThreads - 1) / kSmThreads);
    const uint32_t i0 = tid * (uint32_t)per2;
    uint64_t tmin = ~0ull;
    if (rec) {
      for (int k = 0; k < per2; k++) {
        const uint32_t i = i0 + k;
        if (i < m2) tmin = min(tmin, rv[pin[i]]);
      }
    } else {
#pragma unroll 1
      for (int k0 = 0; k0 < per2; k0 += 4) {
        uint64_t va[4];
#pragma unroll
        for (int u = 0; u < 4; u++) {
          const uint32_t i = i0 + k0 + u;
          va[u] = (k0 + u < per2 && i < m2) ? vv[pin[i]] : ~0ull;
        }
#pragma unroll
        for (int u = 0; u < 4; u++) {
          const uint32_t i = i0 + k0 + u;
          if (k0 + u < per2 && i < m2) {
            skey[i] = va[u];
            tmin = min(tmin, va[u]);
          }
        }
      }
    }
    uint64_t x = tmin;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint64_t y = __shfl_up_sync(0xFFFFFFFFu, x, o);
      if (lane >= o) x = min(x, y);
    }
    uint64_t run = __shfl_up_sync(0xFFFFFFFFu, x, 1);
    if (lane == 0) run = ~0ull;
    if (lane == 31) wmin[warp] = x;
    __syncthreads();
    for (int qq = 0; qq < warp; qq++) run = min(run, wmin[qq]);
    run = min(run, v0);
    uint32_t keep2 = 0, n2 = 0;
    for (int k = 0; k < per2; k++) {
      const uint32_t i = i0 + k;
      if (i >= m2) break;
      const uint64_t v = rec ? rv[pin[i]] : skey[i];
      if (v <= run) { keep2 |= 1u << k; n2++; }
      run = min(run, v);
    }
    uint32_t cy = n2;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t y = __shfl_up_sync(0xFFFFFFFFu, cy, o);
      if (lane >= o) cy += y;
    }
    if (lane == 31) sh_cnt[warp] = cy;
    __syncthreads();
    uint32_t pre = cy - n2, tot = 0;
    for (int qq = 0; qq < kSmWarps; qq++) {
      if (qq < warp) pre += sh_cnt[qq];
      tot += sh_cnt[qq];
    }
    // survivors' record positions in order, then one parallel pass writes
    // the chain slots
    uint16_t* surv = pin == sposA ? sposB : sposA;
    for (int k = 0; k < per2; k++)
      if (keep2 & (1u << k)) surv[pre++] = pin[i0 + k];
    __syncthreads();
    {
      const int64_t cb = chain_base(sd, s, c, r) + 1;
      P* cp = reinterpret_cast<P*>(w.cpts);
      if (rec) {
#pragma unroll 1
        for (uint32_t t0 = 0; t0 < tot; t0 += kSmThreads * 8) {
          uint32_t idx[8];
#pragma unroll
          for (int u = 0; u < 8; u++) {
            const uint32_t t = t0 + u * kSmThreads + tid;
            idx[u] = t < tot ? vin[ri[surv[t]]] & kIdxMask : 0u;
          }
#pragma unroll
          for (int u = 0; u < 8; u++) {
            const uint32_t t = t0 + u * kSmThreads + tid;
            if (t < tot) {
              const uint32_t p = surv[t];
              w.cidx[cb + t] = idx[u];
              cp[cb + t] = point_from_keys<DT>(rk[p], rv[p], r);
            }
          }
        }
      } else {
#pragma unroll 1
        for (uint32_t t0 = 0; t0 < tot; t0 += kSmThreads * 4) {
          uint32_t idx[4];
          uint64_t kk[4], va[4];
#pragma unroll
          for (int u = 0; u < 4; u++) {
            const uint32_t t = t0 + u * kSmThreads + tid;
            const uint32_t p = t < tot ? surv[t] : 0u;
            idx[u] = t < tot ? vin[p] & kIdxMask : 0u;
            kk[u] = t < tot ? kin[p] : 0ull;
            va[u] = t < tot ? vv[p] : 0ull;
          }
#pragma unroll
          for (int u = 0; u < 4; u++) {
            const uint32_t t = t0 + u * kSmThreads + tid;
            if (t < tot) {
              w.cidx[cb + t] = idx[u];
              cp[cb + t] = point_from_keys<DT>(kk[u], va[u], r);
            }
          }
        }
      }
    }
    if (tid == 0) w.ctl[s].s2[r] = tot;
    __syncthreads();
  }
}

template <int DT, int CL>
static void small_attr() {
  static bool once = [] {
    cudaFuncSetAttribute(k_small<DT, CL>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmSmem);
    return true;
  }();
  (void)once;
}

// Clusters of kSmCluster CTAs that fit at once (0: none, or the query failed).
template <int DT>
static int small_clusters_resident() {
  static int n = [] {
    small_attr<DT, kSmCluster>();
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(kSmCluster * 64);
    cfg.blockDim = dim3(kSmThreads);
    cfg.dynamicSmemBytes = kSmSmem;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = kSmCluster;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    int c = 0;
    if (cudaOccupancyMaxActiveClusters(&c, k_small<DT, kSmCluster>, &cfg) != cudaSuccess) {
      cudaGetLastError();
      c = 0;
    }
    return c;
  }();
  return n;
}

template <int DT>
static void launch_small_t(const Job& j, const Ws& w, const Launch& L) {
  const int segs = 4 * j.nsets;
  const int ncl = j.nsets <= kSmClusterSets ? small_clusters_resident<DT>() : 0;
  if (ncl > 0) {
    small_attr<DT, kSmCluster>();
    const int nc = segs < ncl ? segs : ncl;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(nc * kSmCluster);
    cfg.blockDim = dim3(kSmThreads);
    cfg.dynamicSmemBytes = kSmSmem;
    cfg.stream = L.stream;
    cudaLaunchAttribute attr[2];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    attr[1].id = cudaLaunchAttributeClusterDimension;
    attr[1].val.clusterDim.x = kSmCluster;
    attr[1].val.clusterDim.y = 1;
    attr[1].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 2;
    cudaLaunchKernelEx(&cfg, k_small<DT, kSmCluster>, j, w);
    return;
  }
  int grid = segs;
  const int cap = L.grid_cap / 4;      // one 512-thread CTA per SM
  if (grid > cap) grid = cap;
  if (grid < 1) grid = 1;
  small_attr<DT, 1>();
  launch_pdl(k_small<DT, 1>, grid, kSmThreads, kSmSmem, L.stream, j, w);
}

int launch_small(const Job& j, const Ws& w, const Launch& L) {
  if (j.dtype != DT_I32) launch_small_t<DT_F64>(j, w, L);   // float32 input: the float64 stages
  else launch_small_t<DT_I32>(j, w, L);
  return 1;
}

}  // namespace cch

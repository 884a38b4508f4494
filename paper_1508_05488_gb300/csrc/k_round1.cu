// k_round1.cu -- first round of discarding (Sec. 2.1 steps 1-3, Sec. 2.1.1).
//
//  k_extremes  one streaming pass over the points: the four lexicographic
//              extremes E1..E4 = P_minx, P_miny, P_maxx, P_maxy (smallest
//              index on ties), the float64 domain check, and -- in the last
//              CTA of each set -- the edge set-up for the region test.
//  k_classify  second streaming pass: the quadrilateral test with region
//              routing (first k whose directed edge E_k -> E_{k+1} has the
//              point strictly on its right, i.e. outside), and stable
//              compaction of the survivors into one record stream per set
//              (warp ballots, block scan, decoupled look-back).
#include "cch_internal.cuh"

namespace cch {

// ------------------------------------------------------------------ a1

// Lexicographic minimum over (k1, k2, idx).  All four extremes are minima:
// E1 (kx, ky), E2 (ky, kx), E3 (~kx, ~ky), E4 (~ky, ~kx).
struct Lex {
  uint64_t k1, k2;
  uint32_t idx;
};

__device__ __forceinline__ bool lex_less(uint64_t a1, uint64_t a2, uint32_t ai,
                                         uint64_t b1, uint64_t b2, uint32_t bi) {
  return a1 < b1 || (a1 == b1 && (a2 < b2 || (a2 == b2 && ai < bi)));
}

__device__ __forceinline__ void lex_min_into(Lex& a, const Lex& b) {
  if (lex_less(b.k1, b.k2, b.idx, a.k1, a.k2, a.idx)) a = b;
}

__device__ __forceinline__ Lex lex_shfl(const Lex& v, int o) {
  Lex r;
  r.k1 = __shfl_xor_sync(0xFFFFFFFFu, v.k1, o);
  r.k2 = __shfl_xor_sync(0xFFFFFFFFu, v.k2, o);
  r.idx = __shfl_xor_sync(0xFFFFFFFFu, v.idx, o);
  return r;
}

template <int DT>
struct PointT;
template <>
struct PointT<DT_F64> { using T = double2; };
template <>
struct PointT<DT_I32> { using T = int2; };

// Keys of one point.  int32: the 32-bit keys of x and y are packed into k1
// (so one 64-bit compare orders (x, y)), k2 = 0.
template <int DT>
__device__ __forceinline__ void point_keys(const typename PointT<DT>::T& p, uint64_t kk[4][2],
                                           uint32_t& bad) {
  if constexpr (DT == DT_F64) {
    uint64_t bx = (uint64_t)__double_as_longlong(p.x), by = (uint64_t)__double_as_longlong(p.y);
    bad |= f64_bad(bx) | f64_bad(by);
    uint64_t kx = key_f64(bx), ky = key_f64(by);
    kk[0][0] = kx;  kk[0][1] = ky;
    kk[1][0] = ky;  kk[1][1] = kx;
    kk[2][0] = ~kx; kk[2][1] = ~ky;
    kk[3][0] = ~ky; kk[3][1] = ~kx;
  } else {
    uint64_t kx = key_i32(p.x), ky = key_i32(p.y);
    uint64_t nx = kx ^ 0xFFFFFFFFull, ny = ky ^ 0xFFFFFFFFull;
    kk[0][0] = (kx << 32) | ky; kk[0][1] = 0;
    kk[1][0] = (ky << 32) | kx; kk[1][1] = 0;
    kk[2][0] = (nx << 32) | ny; kk[2][1] = 0;
    kk[3][0] = (ny << 32) | nx; kk[3][1] = 0;
  }
}

// Edge set-up of one set, run by one thread once E1..E4 are known.
template <int DT>
__device__ void setup_set(const Job& j, const Ws& w, int s, const SetDesc& sd, const Lex best[4],
                          uint32_t bad) {
  SetCtl& c = w.ctl[s];
  if (bad) {
    c.status = (bad & 1u) ? ST_NONFINITE : ST_RANGE;
    return;
  }
  using P = typename PointT<DT>::T;
  const P* pts = reinterpret_cast<const P*>(j.pts) + sd.off;
  uint32_t flags = 0;
  for (int k = 0; k < 4; k++) {
    c.ek1[k] = best[k].k1;
    c.ek2[k] = best[k].k2;
    c.eidx[k] = best[k].idx;
    P p = pts[best[k].idx];
    c.ex[k] = (double)p.x;
    c.ey[k] = (double)p.y;
  }
  for (int k = 0; k < 4; k++)
    if (c.eidx[k] == c.eidx[(k + 1) & 3]) flags |= SF_DEGEN0 << k;
  if constexpr (DT == DT_I32) {
    // E1 = P_minx, E3 = P_maxx, E2 = P_miny, E4 = P_maxy
    double spanx = c.ex[2] - c.ex[0], spany = c.ey[3] - c.ey[1];
    if (spanx >= 2147483648.0 || spany >= 2147483648.0) flags |= SF_WIDE;
  } else {
    double xm = fmax(fabs(c.ex[0]), fabs(c.ex[2]));
    double ym = fmax(fabs(c.ey[1]), fabs(c.ey[3]));
    const double lim = 1152921504606846976.0;  // 2^60
    if (xm <= lim && ym <= lim && !(j.opts & OPT_NO_FILTER)) {
      flags |= SF_FILTER;
      // orient(a, b, p) = A py - B px + C with A = bx-ax, B = by-ay,
      // C = B ax - A ay.  The FP32 evaluation fma(A, Y, fma(-B, X, C)) on
      // significand-truncated X, Y differs from the exact value by at most
      // 5.01 u (|A| Ymax + |B| Xmax + |B||ax| + |A||ay|) plus underflow
      // terms, u = 2^-24; E below uses 6 u and rounds up.
      const double u = 5.9604644775390625e-08;
      for (int k = 0; k < 4; k++) {
        int k1 = (k + 1) & 3;
        double ax = c.ex[k], ay = c.ey[k], bx = c.ex[k1], by = c.ey[k1];
        double A = bx - ax, B = by - ay;
        double C = B * ax - A * ay;
        double Mc = fabs(B) * fabs(ax) + fabs(A) * fabs(ay);
        double E = 6.0 * u * (fabs(A) * ym + fabs(B) * xm + Mc)
                 + (fabs(A) + fabs(B)) * 2.350988701644575e-38      // 2^-125
                 + 3.5032461608120427e-45 * (xm + ym + 1.0);        // 2^-147
        c.fA[k] = __double2float_rn(A);
        c.fB[k] = __double2float_rn(B);
        c.fC[k] = __double2float_rn(C);
        c.fE[k] = __double2float_ru(E);
      }
    }
  }
  c.flags = flags;
}

template <int DT>
__global__ void __launch_bounds__(kThreads) k_extremes(Job j, Ws w) {
  using P = typename PointT<DT>::T;
  __shared__ Lex red[kWarps][4];
  __shared__ uint32_t red_bad[kWarps];
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
  const int64_t c0 = (int64_t)(chunk - sd.chunk1) * j.chunk1_len;
  const int64_t c1 = min(sd.n, c0 + j.chunk1_len);
  const P* pts = reinterpret_cast<const P*>(j.pts) + sd.off;

  Lex best[4];
#pragma unroll
  for (int k = 0; k < 4; k++) { best[k].k1 = ~0ull; best[k].k2 = ~0ull; best[k].idx = 0xFFFFFFFFu; }
  uint32_t bad = 0;

  constexpr int U = 4;
  for (int64_t base = c0; base < c1; base += (int64_t)kThreads * U) {
    P v[U];
#pragma unroll
    for (int u = 0; u < U; u++) {
      int64_t i = base + u * kThreads + threadIdx.x;
      if (i < c1) v[u] = __ldcs(pts + i);
    }
#pragma unroll
    for (int u = 0; u < U; u++) {
      int64_t i = base + u * kThreads + threadIdx.x;
      if (i < c1) {
        uint64_t kk[4][2];
        point_keys<DT>(v[u], kk, bad);
#pragma unroll
        for (int k = 0; k < 4; k++) {
          // indices grow within a thread: strict order keeps the smallest
          if (kk[k][0] < best[k].k1 || (kk[k][0] == best[k].k1 && kk[k][1] < best[k].k2)) {
            best[k].k1 = kk[k][0]; best[k].k2 = kk[k][1]; best[k].idx = (uint32_t)i;
          }
        }
      }
    }
  }

  // CTA reduction
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
#pragma unroll
    for (int k = 0; k < 4; k++) lex_min_into(best[k], lex_shfl(best[k], o));
    bad |= __shfl_xor_sync(0xFFFFFFFFu, bad, o);
  }
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (lane == 0) {
#pragma unroll
    for (int k = 0; k < 4; k++) red[warp][k] = best[k];
    red_bad[warp] = bad;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int q = 1; q < kWarps; q++) {
      for (int k = 0; k < 4; k++) lex_min_into(best[k], red[q][k]);
      bad |= red_bad[q];
    }
    Part& pt = w.part[chunk];
    for (int k = 0; k < 4; k++) { pt.k1[k] = best[k].k1; pt.k2[k] = best[k].k2; pt.idx[k] = best[k].idx; }
    pt.bad = bad;
    __threadfence();
    last = atomicAdd(&w.ctl[s].arrive1, 1u) == (uint32_t)(sd.nchunk1 - 1);
  }
  __syncthreads();
  if (!last) return;

  // Last chunk of the set: reduce the set's partials, clear its histogram
  // (accumulated by the sort later), set up its edges.
  __threadfence();
  uint32_t* hist = w.hist + (size_t)s * kSortPasses * 256;
  for (int i = threadIdx.x; i < kSortPasses * 256; i += kThreads) hist[i] = 0;
#pragma unroll
  for (int k = 0; k < 4; k++) { best[k].k1 = ~0ull; best[k].k2 = ~0ull; best[k].idx = 0xFFFFFFFFu; }
  bad = 0;
  for (int q = threadIdx.x; q < sd.nchunk1; q += kThreads) {
    const Part& pt = w.part[sd.chunk1 + q];
    for (int k = 0; k < 4; k++) {
      Lex v{pt.k1[k], pt.k2[k], pt.idx[k]};
      lex_min_into(best[k], v);
    }
    bad |= pt.bad;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
#pragma unroll
    for (int k = 0; k < 4; k++) lex_min_into(best[k], lex_shfl(best[k], o));
    bad |= __shfl_xor_sync(0xFFFFFFFFu, bad, o);
  }
  __syncthreads();
  if (lane == 0) {
#pragma unroll
    for (int k = 0; k < 4; k++) red[warp][k] = best[k];
    red_bad[warp] = bad;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int q = 1; q < kWarps; q++) {
      for (int k = 0; k < 4; k++) lex_min_into(best[k], red[q][k]);
      bad |= red_bad[q];
    }
    setup_set<DT>(j, w, s, sd, best, bad);
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
    if (s < j.nsets) t = (w.ctl[s].s1 + kSortTile - 1) / kSortTile;
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

// Region of one point: 1..4, or 0 inside / on the quadrilateral.
template <int DT>
struct EdgeCache {
  float fA[4], fB[4], fC[4], fE[4];
  double ex[4], ey[4];
  int ix[4], iy[4];
  uint32_t flags;
};

template <int DT>
__device__ __forceinline__ int region_of(const EdgeCache<DT>& e, const typename PointT<DT>::T& p) {
  if constexpr (DT == DT_F64) {
    if (e.flags & SF_FILTER) {
      uint64_t bx = (uint64_t)__double_as_longlong(p.x), by = (uint64_t)__double_as_longlong(p.y);
      float X = f64_trunc_f32(bx), Y = f64_trunc_f32(by);
#pragma unroll
      for (int k = 0; k < 4; k++) {
        if (e.flags & (SF_DEGEN0 << k)) continue;
        float d = __fmaf_rn(e.fA[k], Y, __fmaf_rn(-e.fB[k], X, e.fC[k]));
        if (d > e.fE[k]) continue;             // certainly left of (inside) edge k
        if (d < -e.fE[k]) return k + 1;        // certainly right (outside)
        int k1 = (k + 1) & 3;
        if (orient_f64(e.ex[k], e.ey[k], e.ex[k1], e.ey[k1], p.x, p.y) < 0) return k + 1;
      }
      return 0;
    }
#pragma unroll 1
    for (int k = 0; k < 4; k++) {
      if (e.flags & (SF_DEGEN0 << k)) continue;
      int k1 = (k + 1) & 3;
      if (orient_f64(e.ex[k], e.ey[k], e.ex[k1], e.ey[k1], p.x, p.y) < 0) return k + 1;
    }
    return 0;
  } else {
    const bool wide = (e.flags & SF_WIDE) != 0;
#pragma unroll
    for (int k = 0; k < 4; k++) {
      if (e.flags & (SF_DEGEN0 << k)) continue;
      int k1 = (k + 1) & 3;
      if (orient_i32(e.ix[k], e.iy[k], e.ix[k1], e.iy[k1], p.x, p.y, wide) < 0) return k + 1;
    }
    return 0;
  }
}

// Table 1 sort key of a region-r point: R1 x asc, R2 y asc, R3 x desc,
// R4 y desc (ascending order of the returned key).
template <int DT>
__device__ __forceinline__ uint64_t sort_key(const typename PointT<DT>::T& p, int r) {
  uint64_t kx, ky, m;
  if constexpr (DT == DT_F64) {
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

template <int DT>
__global__ void __launch_bounds__(kThreads) k_classify(Job j, Ws w) {
  using P = typename PointT<DT>::T;
  __shared__ int sh_tile;
  __shared__ int sh_set;
  __shared__ EdgeCache<DT> ec;
  __shared__ int32_t sh_status;
  __shared__ uint32_t cnt[kClsItems][kWarps];
  __shared__ uint32_t sh_excl, sh_agg;
  __shared__ int sh_last;

  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const uint32_t tag = j.epoch << 4;   // pass field 0
  if (threadIdx.x == 0) sh_set = -1;

  for (;;) {
    if (threadIdx.x == 0) sh_tile = (int)atomicAdd(w.ctr + CT_CLS_TILE, 1u);
    __syncthreads();
    const int tile = sh_tile;
    if (tile >= j.ntile2) break;
    int s = 0;
    if (j.sets) {
      int lo = 0, hi = j.nsets - 1;
      while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (j.sets[mid].tile2 <= tile) lo = mid; else hi = mid - 1;
      }
      s = lo;
    }
    const SetDesc sd = get_set(j, s);
    if (s != sh_set) {
      __syncthreads();
      if (threadIdx.x == 0) {
        const SetCtl& c = w.ctl[s];
        for (int k = 0; k < 4; k++) {
          ec.fA[k] = c.fA[k]; ec.fB[k] = c.fB[k]; ec.fC[k] = c.fC[k]; ec.fE[k] = c.fE[k];
          ec.ex[k] = c.ex[k]; ec.ey[k] = c.ey[k];
          ec.ix[k] = (int)c.ex[k]; ec.iy[k] = (int)c.ey[k];
        }
        ec.flags = c.flags;
        sh_status = c.status;
        sh_set = s;
      }
      __syncthreads();
    }
    if (sh_status != 0) { __syncthreads(); continue; }   // whole set skipped

    const int64_t lt = tile - sd.tile2;
    const int64_t t0 = lt * kClsTile;
    const P* pts = reinterpret_cast<const P*>(j.pts) + sd.off;

    P v[kClsItems];
#pragma unroll
    for (int it = 0; it < kClsItems; it++) {
      int64_t i = t0 + it * kThreads + threadIdx.x;
      if (i < sd.n) v[it] = pts[i];
    }
    uint64_t regs = 0;    // 4 bits per item
#pragma unroll
    for (int it = 0; it < kClsItems; it++) {
      int64_t i = t0 + it * kThreads + threadIdx.x;
      int r = 0;
      if (i < sd.n) r = region_of<DT>(ec, v[it]);
      regs |= (uint64_t)r << (4 * it);
      uint32_t b = __ballot_sync(0xFFFFFFFFu, r != 0);
      if (lane == 0) cnt[it][warp] = __popc(b);
    }
    __syncthreads();
    // exclusive scan over (item, warp) in point order
    if (threadIdx.x < 32) {
      uint32_t loc[kClsItems * kWarps / 32];
      uint32_t sum = 0;
#pragma unroll
      for (int q = 0; q < kClsItems * kWarps / 32; q++) {
        int f = lane * (kClsItems * kWarps / 32) + q;
        loc[q] = cnt[f / kWarps][f % kWarps];
        sum += loc[q];
      }
      uint32_t x = sum;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        uint32_t y = __shfl_up_sync(0xFFFFFFFFu, x, o);
        if (lane >= o) x += y;
      }
      uint32_t run = x - sum;
#pragma unroll
      for (int q = 0; q < kClsItems * kWarps / 32; q++) {
        int f = lane * (kClsItems * kWarps / 32) + q;
        cnt[f / kWarps][f % kWarps] = run;
        run += loc[q];
      }
      const uint32_t agg = __shfl_sync(0xFFFFFFFFu, x, 31);
      // decoupled look-back across the tiles of this set
      uint64_t* st = w.st2;
      uint32_t excl = 0;
      if (lt == 0) {
        if (lane == 0) st_rel_u64(st + tile, lb_pack(tag, 2, agg));
      } else {
        if (lane == 0) st_rel_u64(st + tile, lb_pack(tag, 1, agg));
        excl = lookback_sum(st, tile, sd.tile2, tag, w.ctr);
        if (lane == 0) st_rel_u64(st + tile, lb_pack(tag, 2, excl + agg));
      }
      if (lane == 0) {
        sh_excl = excl;
        sh_agg = agg;
        if (lt == sd.ntile2 - 1) w.ctl[s].s1 = excl + agg;
      }
    }
    __syncthreads();
    const uint32_t excl = sh_excl;
    uint64_t* keys = w.keyA + sd.off;
    uint32_t* vals = w.valA + sd.off;
    const uint32_t lt_mask = (1u << lane) - 1u;
#pragma unroll
    for (int it = 0; it < kClsItems; it++) {
      int r = (int)((regs >> (4 * it)) & 0xF);
      uint32_t b = __ballot_sync(0xFFFFFFFFu, r != 0);
      if (r != 0) {
        uint32_t pos = excl + cnt[it][warp] + __popc(b & lt_mask);
        int64_t i = t0 + it * kThreads + threadIdx.x;
        keys[pos] = sort_key<DT>(v[it], r);
        vals[pos] = ((uint32_t)(r - 1) << 30) | (uint32_t)i;
      }
    }
    __syncthreads();
  }

  // last CTA out: plan the sort
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    sh_last = atomicAdd(w.ctr + CT_CLS_DONE, 1u) == gridDim.x - 1;
  }
  __syncthreads();
  if (sh_last) {
    __threadfence();
    plan_sort(j, w);
  }
}

int extremes_blocks_per_sm(int dtype) {
  int b = 0;
  if (dtype == DT_F64) cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_extremes<DT_F64>, kThreads, 0);
  else cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_extremes<DT_I32>, kThreads, 0);
  return b > 0 ? b : 1;
}

void launch_extremes(const Job& j, const Ws& w, const Launch& L) {
  if (j.nchunk1 == 0) return;
  if (j.dtype == DT_F64) k_extremes<DT_F64><<<j.nchunk1, kThreads, 0, L.stream>>>(j, w);
  else k_extremes<DT_I32><<<j.nchunk1, kThreads, 0, L.stream>>>(j, w);
}

void launch_classify(const Job& j, const Ws& w, const Launch& L) {
  int grid = j.ntile2 < L.grid_cap ? j.ntile2 : L.grid_cap;
  if (grid < 1) grid = 1;
  if (j.dtype == DT_F64) k_classify<DT_F64><<<grid, kThreads, 0, L.stream>>>(j, w);
  else k_classify<DT_I32><<<grid, kThreads, 0, L.stream>>>(j, w);
}

}  // namespace cch

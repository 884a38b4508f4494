// k_small.cu -- steps 4-5 (Table 1 sort, Fig. 2 SPA) for sets whose regions
// each hold at most kSmallMax round-1 survivors: one CTA per (set, region)
// segment, everything in shared memory.
//
//  1. Fine dominance filter.  The region's sort keys are mapped to 16384
//     buckets by (key - kmin) >> shift (monotone, exact integer arithmetic),
//     the top 32 bits of every candidate's SPA value go into a per-bucket
//     minimum, and the exclusive prefix minimum over buckets (seeded with the
//     region's first extreme) is formed.  A candidate whose value exceeds
//     its bucket's prefix is beaten by a candidate with a strictly smaller
//     key, hence not an SPA survivor (Fig. 2), and is dropped.
//  2. The remaining candidates are sorted by a stable LSD radix sort over the
//     key bytes that vary (8-bit digits, warp-level ranking with match.any,
//     one scatter of 16-bit positions through shared memory per pass); equal
//     keys keep index order because a2 and the gather emit every region in
//     index order, and step 1 keeps that order.
//  3. SPA proper: exclusive prefix minimum of the exact SPA value over the
//     sorted order, seeded with the first extreme; the survivors go, in
//     order, to the region's chain slots.
#include <type_traits>

#include "cch_internal.cuh"

namespace cch {

constexpr int kSmThreads = 512;
constexpr int kSmWarps = kSmThreads / 32;
constexpr int kSmItems = kSmallMax / kSmThreads;   // at most 32 records per thread
constexpr int kFineB = 16384;                      // fine buckets per region
// keys (indexed by candidate) + two position buffers + per-warp histograms;
// the fine-bucket table aliases the two position buffers
constexpr size_t kSmSmem = (size_t)kSmallMax * (8 + 2 + 2) + (size_t)kSmWarps * 256 * 2;
static_assert((size_t)kFineB * 4 <= (size_t)kSmallMax * 4, "fine table must fit the position buffers");

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

// Fine bucket of a sort key (monotone; keys outside [klo, ...] clamp).
__device__ __forceinline__ uint32_t fine_bucket(uint64_t key, uint64_t klo, int shift) {
  const uint64_t d = key > klo ? (key - klo) >> shift : 0ull;
  return (uint32_t)min(d, (uint64_t)(kFineB - 1));
}

template <int DT>
__global__ void __launch_bounds__(kSmThreads, 1) k_small(Job j, Ws w) {
  using P = typename std::conditional<DT == DT_F64, double2, int2>::type;
  extern __shared__ __align__(16) unsigned char smem[];
  uint64_t* skey = reinterpret_cast<uint64_t*>(smem);          // key of candidate i; later SPA value of sorted position j
  uint16_t* sposA = reinterpret_cast<uint16_t*>(skey + kSmallMax);
  uint16_t* sposB = sposA + kSmallMax;
  uint16_t* whist = sposB + kSmallMax;                         // [kSmWarps][256]
  uint32_t* vmin = reinterpret_cast<uint32_t*>(sposA);         // [kFineB], steps 1 only
  __shared__ uint32_t doff[256];
  __shared__ uint32_t wsum[kSmWarps];
  __shared__ uint64_t wor[kSmWarps], wand[kSmWarps], wmin[kSmWarps];
  __shared__ uint32_t sh_cnt[kSmWarps];

  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const uint32_t lt_mask = (1u << lane) - 1u;
  const uint32_t total = w.ctr[CT_SMALL_TOTAL];

  for (uint32_t q = blockIdx.x; q < total; q += gridDim.x) {
    const uint32_t g = w.small_seg[q];
    const int s = (int)(g >> 2), r = (int)(g & 3);
    const SetDesc sd = get_set(j, s);
    const SetCtl& c = w.ctl[s];
    const uint32_t m = c.cnt[r];
    uint32_t rbase = 0;
    for (int qq = 0; qq < r; qq++) rbase += c.cnt[qq];
    const uint64_t* kin = w.keyA + sd.off + rbase;
    const uint32_t* vin = w.valA + sd.off + rbase;
    const P* pts = reinterpret_cast<const P*>(j.pts) + sd.off;
    P e;
    if constexpr (DT == DT_F64) { e.x = c.ex[r]; e.y = c.ey[r]; }
    else { e.x = (int)c.ex[r]; e.y = (int)c.ey[r]; }
    const uint64_t v0 = spa_value_of<DT>(e, r);

    // ---- 1. fine dominance filter ------------------------------------
    // every candidate's key lies between the sort keys of E_r and E_{r+1}
    const uint64_t* vv = w.spvA + sd.off + rbase;
    P e1;
    {
      const int r1 = (r + 1) & 3;
      if constexpr (DT == DT_F64) { e1.x = c.ex[r1]; e1.y = c.ey[r1]; }
      else { e1.x = (int)c.ex[r1]; e1.y = (int)c.ey[r1]; }
    }
    const uint64_t klo = region_sort_key<DT>(e, r), khi = region_sort_key<DT>(e1, r);
    const uint64_t span = khi > klo ? khi - klo : 0;
    const int shift = span == 0 ? 0 : max(0, 64 - __clzll((long long)span) - 14);
    for (int i = tid; i < kFineB; i += kSmThreads) vmin[i] = 0xFFFFFFFFu;
    __syncthreads();
    for (uint32_t i0 = 0; i0 < m; i0 += kSmThreads * 8) {
      uint64_t kk[8], va[8];
#pragma unroll
      for (int u = 0; u < 8; u++) {
        const uint32_t i = i0 + u * kSmThreads + tid;
        kk[u] = i < m ? kin[i] : 0ull;
        va[u] = i < m ? vv[i] : 0ull;
      }
#pragma unroll
      for (int u = 0; u < 8; u++) {
        if (i0 + u * kSmThreads + tid < m)
          atomicMin(&vmin[fine_bucket(kk[u], klo, shift)], (uint32_t)(va[u] >> 32));
      }
    }
    __syncthreads();
    {   // exclusive prefix minimum over the buckets, seeded with the first extreme
      constexpr int per = kFineB / kSmThreads;
      uint32_t loc = 0xFFFFFFFFu;
#pragma unroll
      for (int qq = 0; qq < per; qq++) loc = min(loc, vmin[tid * per + qq]);
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
      run = min(run, (uint32_t)(v0 >> 32));
#pragma unroll
      for (int qq = 0; qq < per; qq++) {
        const uint32_t t = vmin[tid * per + qq];
        vmin[tid * per + qq] = run;
        run = min(run, t);
      }
    }
    __syncthreads();
    // keep mask of the thread's candidates tid*32 .. +32 (index order)
    const uint32_t c0 = tid * kSmItems;
    uint32_t keep = 0;
    for (int k0 = 0; k0 < kSmItems; k0 += 8) {
      uint64_t kk[8], va[8];
#pragma unroll
      for (int u = 0; u < 8; u++) {
        const uint32_t i = c0 + k0 + u;
        kk[u] = i < m ? kin[i] : 0ull;
        va[u] = i < m ? vv[i] : 0ull;
      }
#pragma unroll
      for (int u = 0; u < 8; u++) {
        if (c0 + k0 + u < m && (uint32_t)(va[u] >> 32) <= vmin[fine_bucket(kk[u], klo, shift)])
          keep |= 1u << (k0 + u);
      }
    }
    // stable compaction of the kept candidates (the table is dead after this)
    const uint32_t nk = __popc(keep);
    uint32_t cx = nk;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t y = __shfl_up_sync(0xFFFFFFFFu, cx, o);
      if (lane >= o) cx += y;
    }
    if (lane == 31) sh_cnt[warp] = cx;
    __syncthreads();
    uint32_t rank = cx - nk, m2 = 0;
    for (int qq = 0; qq < kSmWarps; qq++) {
      if (qq < warp) rank += sh_cnt[qq];
      m2 += sh_cnt[qq];
    }
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

    // ---- 2. LSD radix sort of the kept candidates ----------------------
    // the first nw warps own positions w*per*32 .. +per*32, item k of lane l
    // is position w*per*32 + k*32 + l, so (warp, item, lane) is position
    // order; few candidates -> few ranking warps (shorter digit prefixes)
    const int nw = (int)min((uint32_t)kSmWarps, max(1u, (m2 + 255) / 256));
    const int per = (int)((m2 + nw * 32 - 1) / (nw * 32));
    uint16_t* pin = sposA;
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

    // ---- 3. SPA over the sorted order (pin) ----------------------------
    const int per2 = (int)((m2 + kSmThreads - 1) / kSmThreads);
    const uint32_t i0 = tid * (uint32_t)per2;
    uint64_t tmin = ~0ull;
    for (int k0 = 0; k0 < per2; k0 += 8) {
      uint64_t va[8];
#pragma unroll
      for (int u = 0; u < 8; u++) {
        const uint32_t i = i0 + k0 + u;
        va[u] = (k0 + u < per2 && i < m2) ? vv[pin[i]] : ~0ull;
      }
#pragma unroll
      for (int u = 0; u < 8; u++) {
        const uint32_t i = i0 + k0 + u;
        if (k0 + u < per2 && i < m2) {
          skey[i] = va[u];
          tmin = min(tmin, va[u]);
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
      const uint64_t v = skey[i];
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
    if (keep2) {
      const int64_t cb = chain_base(sd, s, c, r) + 1 + pre;
      P* cp = reinterpret_cast<P*>(w.cpts);
      uint32_t o = 0;
      for (int k = 0; k < per2; k++) {
        if (keep2 & (1u << k)) {
          const uint32_t idx = vin[pin[i0 + k]] & kIdxMask;
          w.cidx[cb + o] = idx;
          cp[cb + o] = pts[idx];
          o++;
        }
      }
    }
    if (tid == 0) w.ctl[s].s2[r] = tot;
    __syncthreads();
  }
}

int launch_small(const Job& j, const Ws& w, const Launch& L) {
  int grid = 4 * j.nsets;
  int cap = L.grid_cap / 4;            // one 512-thread CTA per SM
  if (grid > cap) grid = cap;
  if (grid < 1) grid = 1;
  if (j.dtype == DT_F64) {
    static bool once = [] {
      cudaFuncSetAttribute(k_small<DT_F64>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmSmem);
      return true;
    }();
    (void)once;
    k_small<DT_F64><<<grid, kSmThreads, kSmSmem, L.stream>>>(j, w);
  } else {
    static bool once = [] {
      cudaFuncSetAttribute(k_small<DT_I32>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmSmem);
      return true;
    }();
    (void)once;
    k_small<DT_I32><<<grid, kSmThreads, kSmSmem, L.stream>>>(j, w);
  }
  return 1;
}

}  // namespace cch

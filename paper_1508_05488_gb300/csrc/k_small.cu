// k_small.cu -- steps 4-5 (Table 1 sort, Fig. 2 SPA) for sets whose regions
// each hold at most kSmallMax round-1 survivors: one CTA per (set, region)
// segment, everything in shared memory.
//
// The segment's records (sort key, position) are sorted by a stable LSD radix
// sort over the key bytes that are not constant in the segment (8-bit digits,
// warp-level ranking with match.any, one scatter through shared memory per
// pass); equal keys keep index order because a2 and the gather emit every
// region in index order.  SPA is then an exclusive prefix minimum of the
// compared coordinate (seeded with the region's first extreme) over the
// sorted order, and the survivors are compacted, in order, into the region's
// chain slots.
#include <type_traits>

#include "cch_internal.cuh"

namespace cch {

constexpr int kSmThreads = 512;
constexpr int kSmWarps = kSmThreads / 32;
constexpr int kSmItems = kSmallMax / kSmThreads;   // 32 records per thread
// keys (fixed, original order) + two position buffers + per-warp histograms
constexpr size_t kSmSmem = (size_t)kSmallMax * (8 + 2 + 2) + (size_t)kSmWarps * 256 * 2;

template <int DT>
__global__ void __launch_bounds__(kSmThreads, 1) k_small(Job j, Ws w) {
  using P = typename std::conditional<DT == DT_F64, double2, int2>::type;
  extern __shared__ __align__(16) unsigned char smem[];
  uint64_t* skey = reinterpret_cast<uint64_t*>(smem);          // key of record i, later SPA value of sorted position i
  uint16_t* sposA = reinterpret_cast<uint16_t*>(skey + kSmallMax);
  uint16_t* sposB = sposA + kSmallMax;
  uint16_t* whist = sposB + kSmallMax;                         // [kSmWarps][256]
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

    uint64_t kor = 0, kand = ~0ull;
    for (uint32_t i = tid; i < m; i += kSmThreads) {
      const uint64_t k = kin[i];
      skey[i] = k;
      sposA[i] = (uint16_t)i;
      kor |= k;
      kand &= k;
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
      diff = a ^ b;   // bits that vary within the segment
    }

    // LSD passes over the varying key bytes; positions move between the two
    // buffers, (warp, item, lane) order = position order within a pass
    uint16_t* pin = sposA;
    uint16_t* pout = sposB;
    for (int p = 0; p < 8; p++) {
      if (((diff >> (8 * p)) & 0xFFull) == 0) continue;     // uniform
      for (int i = tid; i < kSmWarps * 256; i += kSmThreads) whist[i] = 0;
      __syncthreads();
      uint32_t pr[kSmItems];     // pos | rank << 14 | digit << 24
#pragma unroll
      for (int k = 0; k < kSmItems; k++) {
        const uint32_t i = warp * (kSmItems * 32) + k * 32 + lane;
        const bool ok = i < m;
        const uint32_t pos = ok ? pin[i] : 0u;
        const uint32_t d = ok ? (uint32_t)(skey[pos] >> (8 * p)) & 0xFFu : 256u;
        const uint32_t peers = __match_any_sync(0xFFFFFFFFu, d);
        const uint32_t prior = d < 256 ? whist[warp * 256 + d] : 0u;
        __syncwarp();
        if (d < 256 && lane == __ffs(peers) - 1) whist[warp * 256 + d] = (uint16_t)(prior + __popc(peers));
        __syncwarp();
        pr[k] = pos | ((prior + __popc(peers & lt_mask)) << 14) | ((d & 0xFFu) << 24);
      }
      __syncthreads();
      if (tid < 256) {
        uint32_t run = 0;
        for (int qq = 0; qq < kSmWarps; qq++) {
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
#pragma unroll
      for (int k = 0; k < kSmItems; k++) {
        const uint32_t i = warp * (kSmItems * 32) + k * 32 + lane;
        if (i < m) {
          const uint32_t d = pr[k] >> 24;
          pout[doff[d] + whist[warp * 256 + d] + ((pr[k] >> 14) & 0x3FFu)] = (uint16_t)(pr[k] & 0x3FFFu);
        }
      }
      __syncthreads();
      uint16_t* t = pin; pin = pout; pout = t;
    }

    // SPA over the sorted order (pin): thread t owns sorted positions t*32 .. +32
    const P* pts = reinterpret_cast<const P*>(j.pts) + sd.off;
    const uint32_t* vin = w.valA + sd.off + rbase;
    const uint32_t i0 = tid * kSmItems;
    uint64_t tmin = ~0ull;
#pragma unroll 8
    for (int k = 0; k < kSmItems; k++) {
      const uint32_t i = i0 + k;
      if (i < m) {
        const P p = pts[vin[pin[i]] & kIdxMask];
        uint64_t v;
        if constexpr (DT == DT_F64) v = spa_v_f64(p.x, p.y, r);
        else v = spa_v_i32(p.x, p.y, r);
        skey[i] = v;
        tmin = min(tmin, v);
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
    {
      uint64_t v0;
      if constexpr (DT == DT_F64) v0 = spa_v_f64(c.ex[r], c.ey[r], r);
      else v0 = spa_v_i32((int)c.ex[r], (int)c.ey[r], r);
      run = min(run, v0);
    }
    uint32_t keep = 0, nk = 0;
    for (int k = 0; k < kSmItems; k++) {
      const uint32_t i = i0 + k;
      if (i >= m) break;
      const uint64_t v = skey[i];
      if (v <= run) { keep |= 1u << k; nk++; }
      run = min(run, v);
    }
    uint32_t cx = nk;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t y = __shfl_up_sync(0xFFFFFFFFu, cx, o);
      if (lane >= o) cx += y;
    }
    if (lane == 31) sh_cnt[warp] = cx;
    __syncthreads();
    uint32_t pre = cx - nk, tot = 0;
    for (int qq = 0; qq < kSmWarps; qq++) {
      if (qq < warp) pre += sh_cnt[qq];
      tot += sh_cnt[qq];
    }
    if (keep) {
      const int64_t cb = chain_base(sd, s, c, r) + 1 + pre;
      P* cp = reinterpret_cast<P*>(w.cpts);
      uint32_t o = 0;
      for (int k = 0; k < kSmItems; k++) {
        if (keep & (1u << k)) {
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

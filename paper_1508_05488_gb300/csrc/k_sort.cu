// k_sort.cu -- per-region sort of the round-1 survivors (Sec. 2.1 step 4,
// Table 1), as one stable LSD radix sort per set.
//
// Records are (key u64, value u32): key = the Table 1 sort key of the point's
// region (x asc, y asc, x desc, y desc as an ascending order-preserving
// integer key), value = region << 30 | set-local index.  Eight byte passes
// over the key and a final pass over the region digit leave each set's
// records grouped by region and sorted by key, equal keys in index order
// (every pass is stable and a2 emits records in index order).
//
//  k_sort_hist  one read of all records: the 9 x 256 digit histograms of every
//               set; its last CTA plans the SPA tiles.
//  k_sort_pass  one pass: per tile, warp-level stable ranking
//               (match.any), a decoupled look-back per digit across the tiles
//               of the set, and a scatter into the other buffer.  A pass whose
//               digit is the same for every record of a set is skipped for
//               that set (the data stays in place; the buffer parity of the
//               remaining passes follows from the histograms).
#include "cch_internal.cuh"

namespace cch {

__device__ __forceinline__ uint32_t digit_of(uint64_t key, uint32_t val, int p) {
  return p < 8 ? (uint32_t)(key >> (8 * p)) & 0xFFu : (val >> 30);
}

// SPA plan (single CTA, after the histograms): SPA tiles per (set, region).
__device__ void plan_spa(const Job& j, const Ws& w) {
  __shared__ uint32_t carry;
  __shared__ uint32_t wsum[kWarps];
  if (threadIdx.x == 0) carry = 0;
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int nseg = 4 * j.nsets;
  for (int base = 0; base < nseg; base += kThreads) {
    int g = base + threadIdx.x;
    uint32_t t = 0;
    if (g < nseg) {
      const SetCtl& c = w.ctl[g >> 2];
      if (c.flags & SF_BIG) t = (c.cnt[g & 3] + kSpaTile - 1) / kSpaTile;
    }
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
    if (g < nseg) w.spa_start[g] = pre + x - t;
    __syncthreads();
    if (threadIdx.x == kThreads - 1) carry = pre + x;
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    w.spa_start[nseg] = carry;
    w.ctr[CT_SPA_TOTAL] = carry;
  }
}

__global__ void __launch_bounds__(kThreads) k_sort_hist(Job j, Ws w) {
  __shared__ uint32_t h[kSortPasses][256];
  __shared__ int sh_last;
  const int lane = threadIdx.x & 31;
  const uint32_t total = w.ctr[CT_SORT_TOTAL];
  if (total == 0) {          // no multi-block set: one CTA plans, no arrival count
    if (blockIdx.x == 0) plan_spa(j, w);
    return;
  }
  const int npass_key = j.dtype == DT_F64 ? 8 : 4;   // int32 keys have 4 zero bytes
  for (uint32_t tile = blockIdx.x; tile < total; tile += gridDim.x) {
    const int s = seg_of(w.sort_start, j.nsets, tile);
    const SetDesc sd = get_set(j, s);
    const uint32_t lt = tile - w.sort_start[s];
    const uint32_t n1 = w.ctl[s].s1;
    for (int q = threadIdx.x; q < kSortPasses * 256; q += kThreads) (&h[0][0])[q] = 0;
    __syncthreads();
    const uint32_t b0 = lt * kSortTile;
    const uint32_t b1 = min(n1, b0 + kSortTile);
    for (uint32_t i0 = b0; i0 < b1; i0 += kThreads) {
      uint32_t i = i0 + threadIdx.x;
      bool ok = i < b1;
      uint64_t key = ok ? w.keyA[sd.off + i] : 0;
      uint32_t val = ok ? w.valA[sd.off + i] : 0;
      const uint32_t act = __ballot_sync(0xFFFFFFFFu, ok);
      for (int p = 0; p < kSortPasses; p++) {
        if (p >= npass_key && p < 8) continue;
        uint32_t d = ok ? digit_of(key, val, p) : 0xFFFFFFFFu;
        uint32_t peers = __match_any_sync(0xFFFFFFFFu, d);
        if (ok && lane == __ffs(peers & act) - 1) atomicAdd(&h[p][d], __popc(peers));
      }
    }
    __syncthreads();
    uint32_t* gh = w.hist + (size_t)s * kSortPasses * 256;
    for (int q = threadIdx.x; q < kSortPasses * 256; q += kThreads) {
      uint32_t v = (&h[0][0])[q];
      int p = q >> 8;
      if (p >= npass_key && p < 8) {
        // constant zero byte: the first tile of the set records all records in bin 0
        if (lt == 0 && (q & 255) == 0) atomicAdd(gh + q, n1);
      } else if (v) {
        atomicAdd(gh + q, v);
      }
    }
    __syncthreads();
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    sh_last = atomicAdd(w.ctr + CT_HIST_DONE, 1u) == gridDim.x - 1;
  }
  __syncthreads();
  if (sh_last) {
    __threadfence();
    plan_spa(j, w);
  }
}

__global__ void __launch_bounds__(kThreads) k_sort_pass(Job j, Ws w, int p) {
  __shared__ uint32_t whist[kWarps][256];
  __shared__ uint32_t doff[256];
  __shared__ uint32_t gpre[256];
  __shared__ uint32_t wsum[kWarps];
  __shared__ uint32_t sh_tile;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const uint32_t lt_mask = (1u << lane) - 1u;
  const uint32_t total = w.ctr[CT_SORT_TOTAL];
  if (total == 0) return;
  const uint32_t tag = (j.epoch << 4) | (uint32_t)p;

  for (;;) {
    if (threadIdx.x == 0) sh_tile = atomicAdd(w.ctr + CT_SORT_TILE0 + p, 1u);
    __syncthreads();
    const uint32_t tile = sh_tile;
    if (tile >= total) break;
    const int s = seg_of(w.sort_start, j.nsets, tile);
    const SetDesc sd = get_set(j, s);
    const uint32_t first = w.sort_start[s];
    const uint32_t lt = tile - first;
    const uint32_t n1 = w.ctl[s].s1;
    const uint32_t* gh = w.hist + (size_t)s * kSortPasses * 256;

    // which earlier passes moved data (buffer parity), and whether this one does
    int par = 0;
    bool skip = false;
    for (int q = 0; q <= p; q++) {
      bool full = __syncthreads_or(gh[q * 256 + threadIdx.x] == n1) != 0;
      if (q < p) par ^= full ? 0 : 1;
      else skip = full;
    }
    if (skip) continue;   // uniform across the CTA
    const uint64_t* kin = par ? w.keyB : w.keyA;
    const uint32_t* vin = par ? w.valB : w.valA;
    uint64_t* kout = par ? w.keyA : w.keyB;
    uint32_t* vout = par ? w.valA : w.valB;

    // digit offsets within the set: exclusive scan of this pass's histogram
    {
      uint32_t c = gh[p * 256 + threadIdx.x];
      uint32_t x = c;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        uint32_t y = __shfl_up_sync(0xFFFFFFFFu, x, o);
        if (lane >= o) x += y;
      }
      if (lane == 31) wsum[warp] = x;
      for (int q = threadIdx.x; q < kWarps * 256; q += kThreads) (&whist[0][0])[q] = 0;
      __syncthreads();
      uint32_t pre = 0;
      for (int q = 0; q < warp; q++) pre += wsum[q];
      doff[threadIdx.x] = pre + x - c;
    }
    __syncthreads();

    // load: warp w owns records [w*512, w*512+512) of the tile, item k of
    // lane l is record w*512 + k*32 + l, so (warp, item, lane) is record order
    uint64_t key[kSortItems];
    uint32_t val[kSortItems];
    uint32_t dig[kSortItems];
    uint32_t rank[kSortItems];
    const uint32_t tbase = lt * kSortTile + warp * (kSortItems * 32);
#pragma unroll
    for (int k = 0; k < kSortItems; k++) {
      uint32_t i = tbase + k * 32 + lane;
      bool ok = i < n1;
      key[k] = ok ? kin[sd.off + i] : 0;
      val[k] = ok ? vin[sd.off + i] : 0;
      dig[k] = ok ? digit_of(key[k], val[k], p) : 256u;
    }
#pragma unroll
    for (int k = 0; k < kSortItems; k++) {
      uint32_t d = dig[k];
      uint32_t peers = __match_any_sync(0xFFFFFFFFu, d);
      uint32_t prior = d < 256 ? whist[warp][d] : 0u;
      __syncwarp();
      if (d < 256 && lane == __ffs(peers) - 1) whist[warp][d] = prior + __popc(peers);
      __syncwarp();
      rank[k] = prior + __popc(peers & lt_mask);
    }
    __syncthreads();
    // per digit: exclusive prefix over warps, tile count, look-back
    {
      const int d = threadIdx.x;
      uint32_t run = 0;
#pragma unroll
      for (int q = 0; q < kWarps; q++) {
        uint32_t c = whist[q][d];
        whist[q][d] = run;
        run += c;
      }
      uint64_t* st = w.st_sort + (size_t)tile * 256 + d;
      uint32_t excl = 0;
      if (lt == 0) {
        st_rel_u64(st, lb_pack(tag, 2, run));
      } else {
        st_rel_u64(st, lb_pack(tag, 1, run));
        int64_t t = (int64_t)tile - 1;
        uint32_t spins = 0;
        while (t >= (int64_t)first) {
          uint64_t v = ld_acq_u64(w.st_sort + (size_t)t * 256 + d);
          uint32_t hi = (uint32_t)(v >> 32);
          uint32_t kind = (hi >> 16) == tag ? (hi & 0xFFFFu) : 0u;
          if (kind == 0) {
            if (!spin_step(spins, w.ctr)) break;
            continue;
          }
          excl += (uint32_t)v;
          if (kind == 2) break;
          t--;
        }
        st_rel_u64(st, lb_pack(tag, 2, excl + run));
      }
      gpre[d] = doff[d] + excl;
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < kSortItems; k++) {
      uint32_t d = dig[k];
      uint32_t pos = d < 256 ? gpre[d] + whist[warp][d] + rank[k] : n1;
      if (pos < n1) {
        kout[sd.off + pos] = key[k];
        vout[sd.off + pos] = val[k];
      }
    }
    __syncthreads();
  }
}

int launch_sort(const Job& j, const Ws& w, const Launch& L) {
  int64_t tiles_max = j.N / kSortTile + j.nsets;
  int grid = (int)(tiles_max < L.grid_cap ? tiles_max : L.grid_cap);
  if (grid < 1) grid = 1;
  k_sort_hist<<<grid, kThreads, 0, L.stream>>>(j, w);
  int n = 1;
  for (int p = 0; p < kSortPasses; p++) {
    if (j.dtype == DT_I32 && p >= 4 && p < 8) continue;   // zero key bytes
    k_sort_pass<<<grid, kThreads, 0, L.stream>>>(j, w, p);
    n++;
  }
  return n;
}

}  // namespace cch

// k_big.cu -- per-region sort (Sec. 2.1 step 4, Table 1) and SPA (Sec. 2.1.2,
// Fig. 2; step 5) of the sets whose regions are too large for the
// shared-memory path, as one cooperative persistent kernel whose phases are
// separated by grid-wide barriers.  When no set needs it, one CTA writes the
// chain plan and the kernel ends: the common case costs one launch.
//
// Sort.  Records are (key u64, value u32): key = the Table 1 sort key of the
// point's region (x asc, y asc, x desc, y desc as an ascending
// order-preserving integer key), value = region << 30 | set-local index.
// Eight byte passes over the key and a final pass over the region digit leave
// each set's records grouped by region and sorted by key, equal keys in index
// order (every pass is stable and the gather emits records in index order).
//   histogram phase  one read of all records: the 9 x 256 digit histograms
//                    of every set.
//   pass phases      per tile, warp-level stable ranking (match.any), a
//                    decoupled look-back per digit across the tiles of the
//                    set, and a scatter into the other buffer.  A pass whose
//                    digit is the same for every record of a set is skipped
//                    for that set (the data stays in place; the buffer parity
//                    of the remaining passes follows from the histograms).
//
// SPA.  Fig. 2 walks each sorted region once, keeping a point unless its
// compared coordinate is strictly worse than the running value t, which
// starts at the region's first extreme and is updated by every kept point.
// Because a discarded point never lowers t, t before a point is the minimum
// over the first extreme and ALL earlier points; with the compared
// coordinate mapped to an order-preserving key v in "smaller is better" form
//     R1: v = key(y)   R2: v = ~key(x)   R3: v = ~key(y)   R4: v = key(x)
// a point survives iff  v <= min(v(E_r), exclusive prefix-min of v).  That
// is a segmented exclusive prefix-minimum scan (associative), run here with a
// decoupled look-back, followed by a stable compaction of the survivors into
// the region's chain slots (positions 1 .. s2).  The paper's own GPU version
// restarts t in each of 1024 chunks (Sec. 2.2.2), which keeps a superset; the
// scan keeps exactly the sequential set.
//
// The grid is launched cooperatively (every CTA resident), so the barriers
// and the look-backs always make progress; every wait is bounded and a
// timeout records CCH_ERR_TIMEOUT and ends the kernel.
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

template <int DT>
struct PtT;
template <>
struct PtT<DT_F64> { using T = double2; };
template <>
struct PtT<DT_I32> { using T = int2; };

template <int DT>
__device__ __forceinline__ uint64_t spa_value(const typename PtT<DT>::T& p, int r) {
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
    case 0: return ky;
    case 1: return kx ^ m;
    case 2: return ky ^ m;
    default: return kx;
  }
}

// Chain plan (single CTA, after SPA): chain blocks and output tiles per
// (set, region); output counts of sets that need no chain work.
__device__ void plan_chain(const Job& j, const Ws& w) {
  __shared__ uint32_t carry[2];
  __shared__ uint32_t wsum[2][kWarps];
  if (threadIdx.x < 2) carry[threadIdx.x] = 0;
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int nseg = 4 * j.nsets;
  for (int base = 0; base < nseg; base += kThreads) {
    int g = base + threadIdx.x;
    uint32_t tb = 0, to = 0;
    if (g < nseg) {
      const int s = g >> 2, r = g & 3;
      const SetDesc sd = get_set(j, s);
      const SetCtl& c = w.ctl[s];
      const uint32_t degen_all = (SF_DEGEN0 * 15u);
      if (c.status != 0) {
        if (r == 0) j.out_counts[s] = c.status;
      } else if (sd.n == 0) {
        if (r == 0) j.out_counts[s] = 0;
      } else if ((c.flags & degen_all) == degen_all) {
        // every point identical: the hull is the single point E1
        if (r == 0) { j.out_idx[sd.off] = (int32_t)c.eidx[0]; j.out_counts[s] = 1; }
      } else if (!(c.flags & (SF_DEGEN0 << r))) {
        uint32_t L = c.s2[r] + 2;
        tb = (L + kChainBlk - 1) / kChainBlk;
        to = (L - 1 + kOutTile - 1) / kOutTile;
      }
    }
    // A set whose chains each fit one chain block takes its output from
    // k_chain_local (the last of its chain blocks writes it): no output
    // tiles.  The four threads of a set are neighbouring lanes of one warp.
    {
      uint32_t f = tb <= 1u ? 1u : 0u;
      f &= __shfl_xor_sync(0xFFFFFFFFu, f, 1);   // every lane takes part in both shuffles
      f &= __shfl_xor_sync(0xFFFFFFFFu, f, 2);
      const bool fit = f != 0u;
      uint32_t nb = tb;
      nb += __shfl_xor_sync(0xFFFFFFFFu, nb, 1);
      nb += __shfl_xor_sync(0xFFFFFFFFu, nb, 2);
      if (g < nseg && fit && nb > 0) {
        to = 0;
        if ((g & 3) == 0) {
          SetCtl& cw = w.ctl[g >> 2];
          cw.flags |= SF_LOCALOUT;
          cw.nloc = nb;
        }
      }
    }
    uint32_t x = tb, y = to;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      uint32_t a = __shfl_up_sync(0xFFFFFFFFu, x, o);
      uint32_t b = __shfl_up_sync(0xFFFFFFFFu, y, o);
      if (lane >= o) { x += a; y += b; }
    }
    if (lane == 31) { wsum[0][warp] = x; wsum[1][warp] = y; }
    __syncthreads();
    uint32_t px = carry[0], py = carry[1];
    for (int q = 0; q < warp; q++) { px += wsum[0][q]; py += wsum[1][q]; }
    if (g < nseg) { w.chain_start[g] = px + x - tb; w.out_start[g] = py + y - to; }
    __syncthreads();
    if (threadIdx.x == kThreads - 1) { carry[0] = px + x; carry[1] = py + y; }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    w.chain_start[nseg] = carry[0];
    w.out_start[nseg] = carry[1];
    w.ctr[CT_CHAIN_TOTAL] = carry[0];
    w.ctr[CT_OUT_TOTAL] = carry[1];
  }
}

// Grid-wide barrier number `gen` (counted from 1 within a call).  Returns
// false (the same in every thread of the CTA) when the wait ran out.
__device__ __forceinline__ bool grid_sync(const Ws& w, uint32_t& gen) {
  __shared__ int sh_ok;
  __syncthreads();
  gen++;
  if (threadIdx.x == 0) {
    __threadfence();
    atomicAdd(w.ctr + CT_BIG_BAR, 1u);
    const uint32_t target = gen * gridDim.x;
    uint32_t spins = 0;
    int ok = 1;
    while (ld_acq_u32(w.ctr + CT_BIG_BAR) < target)
      if (!spin_step(spins, w.ctr)) { ok = 0; break; }
    __threadfence();
    sh_ok = ok;
  }
  __syncthreads();
  return sh_ok != 0;
}

// Histogram phase: every sort tile, strided over the grid.
__device__ void big_hist(const Job& j, const Ws& w, uint32_t total) {
  // A CTA adds up the histograms of all its tiles of a set in shared memory
  // (one shared atomic per record and digit: cheaper here than ranking equal
  // digits with match.any) and flushes them into the set's global histogram
  // once (the global atomics would otherwise queue on the same 2304 words
  // from every tile).
  __shared__ uint32_t h[kSortPasses][256];
  const int npass_key = j.dtype != DT_I32 ? 8 : 4;   // int32 keys have 4 zero bytes
  constexpr int kItems = kSortTile / kThreads;
  for (int q = threadIdx.x; q < kSortPasses * 256; q += kThreads) (&h[0][0])[q] = 0;
  __syncthreads();
  int cur = -1;            // set whose counts h holds (uniform across the CTA)
  bool cur_first = false;  // whether this CTA took that set's first tile
  auto flush = [&]() {
    uint32_t* gh = w.hist + (size_t)cur * kSortPasses * 256;
    const uint32_t n1 = w.ctl[cur].s1;
    for (int q = threadIdx.x; q < kSortPasses * 256; q += kThreads) {
      const uint32_t v = (&h[0][0])[q];
      const int p = q >> 8;
      if (p >= npass_key && p < 8) {
        // constant zero byte: the set's first tile records all records in bin 0
        if (cur_first && (q & 255) == 0) atomicAdd(gh + q, n1);
      } else if (v) {
        atomicAdd(gh + q, v);
      }
      (&h[0][0])[q] = 0;
    }
    __syncthreads();
  };
  for (uint32_t tile = blockIdx.x; tile < total; tile += gridDim.x) {
    const int s = seg_of(w.sort_start, j.nsets, tile);
    if (s != cur) {
      if (cur >= 0) flush();
      cur = s;
      cur_first = false;
    }
    const SetDesc sd = get_set(j, s);
    const uint32_t lt = tile - w.sort_start[s];
    if (lt == 0) cur_first = true;
    const uint32_t n1 = w.ctl[s].s1;
    const uint32_t b0 = lt * kSortTile;
    const uint32_t b1 = min(n1, b0 + kSortTile);
    uint64_t key[kItems];
    uint32_t val[kItems];
#pragma unroll
    for (int k = 0; k < kItems; k++) {      // the thread's records, loads in flight together
      const uint32_t i = b0 + k * kThreads + threadIdx.x;
      key[k] = i < b1 ? w.keyA[sd.off + i] : 0ull;
      val[k] = i < b1 ? w.valA[sd.off + i] : 0u;
    }
#pragma unroll
    for (int k = 0; k < kItems; k++) {
      const bool ok = b0 + k * kThreads + threadIdx.x < b1;
      for (int p = 0; p < kSortPasses; p++) {
        if (p >= npass_key && p < 8) continue;
        if (ok) atomicAdd(&h[p][digit_of(key[k], val[k], p)], 1u);
      }
    }
    __syncthreads();
  }
  if (cur >= 0) flush();
}

// One radix pass: tiles taken in order from the pass's counter.
__device__ void big_pass(const Job& j, const Ws& w, int p, uint32_t total) {
  __shared__ uint32_t whist[kWarps][256];
  __shared__ uint32_t doff[256];
  __shared__ uint32_t gpre[256];
  __shared__ uint32_t wsum[kWarps];
  __shared__ uint32_t sh_tile, sh_full;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const uint32_t lt_mask = (1u << lane) - 1u;
  const uint32_t tag = (j.epoch << 4) | (uint32_t)p;

  for (;;) {
    if (threadIdx.x == 0) {
      sh_tile = atomicAdd(w.ctr + CT_SORT_TILE0 + p, 1u);
      sh_full = 0;
    }
    __syncthreads();
    const uint32_t tile = sh_tile;
    if (tile >= total) break;
    const int s = seg_of(w.sort_start, j.nsets, tile);
    const SetDesc sd = get_set(j, s);
    const uint32_t first = w.sort_start[s];
    const uint32_t lt = tile - first;
    const uint32_t n1 = w.ctl[s].s1;
    const uint32_t* gh = w.hist + (size_t)s * kSortPasses * 256;

    // which earlier passes moved data (buffer parity), and whether this one
    // does: a pass whose digit histogram has all records in one bin moves
    // nothing.  Every thread reads its bin of passes 0..p at once, the CTA
    // ORs the bit masks.
    {
      uint32_t fm = 0;
      for (int q = 0; q <= p; q++) fm |= (gh[q * 256 + threadIdx.x] == n1 ? 1u : 0u) << q;
      fm = __reduce_or_sync(0xFFFFFFFFu, fm);
      if (lane == 0 && fm) atomicOr(&sh_full, fm);
    }
    __syncthreads();
    const uint32_t full = sh_full;
    const int par = __popc(~full & ((1u << p) - 1u)) & 1;
    const bool skip = (full >> p) & 1u;
    if (skip) continue;   // uniform across the CTA
    if (lt == 0 && threadIdx.x == 0) w.ctl[s].passes++;   // one CTA per (pass, set); passes are barrier-separated
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
        // Decoupled look-back over the digit's words of the predecessor
        // tiles, eight of them per step (their loads in flight together):
        // aggregates add up until an inclusive prefix ends the walk.  A
        // word packs tag, kind and value, so a relaxed load reads a
        // consistent triple.
        int64_t t = (int64_t)tile - 1;
        uint32_t spins = 0;
        while (t >= (int64_t)first) {
          constexpr int kLb = 8;
          uint64_t v[kLb];
#pragma unroll
          for (int u = 0; u < kLb; u++)
            v[u] = t - u >= (int64_t)first ? ld_rlx_u64(w.st_sort + (size_t)(t - u) * 256 + d)
                                           : lb_pack(tag, 2, 0);
          int used = 0;
          bool incl = false, stall = false;
#pragma unroll
          for (int u = 0; u < kLb; u++) {
            if (incl || stall) continue;
            const uint32_t hi = (uint32_t)(v[u] >> 32);
            const uint32_t kind = (hi >> 16) == tag ? (hi & 0xFFFFu) : 0u;
            if (kind == 0) { stall = true; continue; }
            excl += (uint32_t)v[u];
            used = u + 1;
            incl = kind == 2;
          }
          if (incl) break;
          t -= used;
          if (stall && !spin_step(spins, w.ctr)) break;
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

// SPA phase: tiles of (set, region) segments taken in order from a counter.
template <int DT>
__device__ void big_spa(const Job& j, const Ws& w) {
  using P = typename PtT<DT>::T;
  __shared__ uint32_t sh_tile;
  __shared__ uint64_t wmin[kWarps];
  __shared__ uint32_t wcnt[kWarps];
  __shared__ uint64_t sh_prefix;
  __shared__ uint32_t sh_excl;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const uint32_t total = w.ctr[CT_SPA_TOTAL];
  const uint32_t tag_min = (j.epoch << 4) | 10u, tag_cnt = (j.epoch << 4) | 11u;

  for (;;) {
    if (threadIdx.x == 0) sh_tile = atomicAdd(w.ctr + CT_SPA_TILE, 1u);
    __syncthreads();
    const uint32_t tile = sh_tile;
    if (tile >= total) break;
    const int g = seg_of(w.spa_start, 4 * j.nsets, tile);
    const int s = g >> 2, r = g & 3;
    const SetDesc sd = get_set(j, s);
    const SetCtl& c = w.ctl[s];
    const uint32_t first = w.spa_start[g];
    const uint32_t lt = tile - first;
    const uint32_t nr = c.cnt[r];
    const uint32_t* gh = w.hist + (size_t)s * kSortPasses * 256;
    int par = 0;
    for (int q = 0; q < kSortPasses; q++)
      par ^= __syncthreads_or(gh[q * 256 + threadIdx.x] == c.s1) ? 0 : 1;
    const uint32_t* vin = par ? w.valB : w.valA;
    uint32_t roff = 0;
    for (int q = 0; q < r; q++) roff += c.cnt[q];

    // thread t owns records lt*2048 + t*8 .. +8 (contiguous: in-thread scan)
    const uint32_t b0 = lt * kSpaTile + threadIdx.x * kSpaItems;
    uint32_t idx[kSpaItems];
    P pt[kSpaItems];
    uint64_t v[kSpaItems];
#pragma unroll
    for (int k = 0; k < kSpaItems; k++) {
      uint32_t i = b0 + k;
      idx[k] = i < nr ? (vin[sd.off + roff + i] & kIdxMask) : 0u;
    }
    uint64_t tmin = ~0ull;
#pragma unroll
    for (int k = 0; k < kSpaItems; k++) {
      uint32_t i = b0 + k;
      if (i < nr) {
        pt[k] = input_point<P>(j, sd.off + idx[k]);
        v[k] = spa_value<DT>(pt[k], r);
      } else {
        v[k] = ~0ull;
      }
      tmin = min(tmin, v[k]);
    }
    // exclusive prefix-min of thread minima within the tile
    uint64_t x = tmin;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      uint64_t y = __shfl_up_sync(0xFFFFFFFFu, x, o);
      if (lane >= o) x = min(x, y);
    }
    uint64_t texcl = __shfl_up_sync(0xFFFFFFFFu, x, 1);
    if (lane == 0) texcl = ~0ull;
    if (lane == 31) wmin[warp] = x;
    __syncthreads();
    for (int q = 0; q < warp; q++) texcl = min(texcl, wmin[q]);
    if (warp == 0) {
      uint64_t agg = ~0ull;
      for (int q = 0; q < kWarps; q++) agg = min(agg, wmin[q]);
      // start value: the region's first extreme
      const int k0 = r;
      P e;
      if constexpr (DT == DT_F64) { e.x = c.ex[k0]; e.y = c.ey[k0]; }
      else { e.x = (int)c.ex[k0]; e.y = (int)c.ey[k0]; }
      uint64_t excl = spa_value<DT>(e, r);
      SpaStat* st = w.st_spa + tile;
      if (lt == 0) {
        if (lane == 0) {
          st->inc_min = min(excl, agg);
          st_rel_u32(&st->flag, (tag_min << 16) | 2u);
        }
      } else {
        if (lane == 0) {
          st->agg_min = agg;
          st_rel_u32(&st->flag, (tag_min << 16) | 1u);
        }
        // warp-cooperative decoupled look-back: lane l reads tile base - l;
        // the minimum runs over the tiles up to the nearest inclusive prefix
        int64_t base = (int64_t)tile - 1;
        uint32_t spins = 0;
        while (base >= (int64_t)first) {
          const int64_t t = base - lane;
          uint32_t kind = 2u;
          if (t >= (int64_t)first) {
            const uint32_t f = ld_acq_u32(&w.st_spa[t].flag);
            kind = (f >> 16) == tag_min ? (f & 0xFFFFu) : 0u;
          }
          const uint32_t incl = __ballot_sync(0xFFFFFFFFu, kind == 2u);
          const int stop = incl ? __ffs(incl) - 1 : 31;
          const uint32_t upto = stop == 31 ? 0xFFFFFFFFu : (2u << stop) - 1u;
          if (__ballot_sync(0xFFFFFFFFu, kind == 0u) & upto) {
            const bool go = spin_step(spins, w.ctr);   // identical in every lane
            if (!__all_sync(0xFFFFFFFFu, go)) break;
            continue;
          }
          uint64_t v = ~0ull;
          if (lane <= stop && t >= (int64_t)first)
            v = kind == 2u ? *(volatile const uint64_t*)&w.st_spa[t].inc_min
                           : *(volatile const uint64_t*)&w.st_spa[t].agg_min;
#pragma unroll
          for (int o = 16; o > 0; o >>= 1) v = min(v, __shfl_xor_sync(0xFFFFFFFFu, v, o));
          excl = min(excl, v);
          if (incl) break;
          base -= 32;
        }
        if (lane == 0) {
          st->inc_min = min(excl, agg);
          st_rel_u32(&st->flag, (tag_min << 16) | 2u);
        }
      }
      if (lane == 0) sh_prefix = excl;
    }
    __syncthreads();
    uint64_t run = min(sh_prefix, texcl);
    uint32_t keep = 0, nkeep = 0;
#pragma unroll
    for (int k = 0; k < kSpaItems; k++) {
      if (b0 + k < nr && v[k] <= run) { keep |= 1u << k; nkeep++; }
      run = min(run, v[k]);
    }
    // stable compaction of the survivors
    uint32_t cx = nkeep;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      uint32_t y = __shfl_up_sync(0xFFFFFFFFu, cx, o);
      if (lane >= o) cx += y;
    }
    if (lane == 31) wcnt[warp] = cx;
    __syncthreads();
    uint32_t pre = cx - nkeep;
    for (int q = 0; q < warp; q++) pre += wcnt[q];
    if (warp == 0) {
      uint32_t agg = 0;
      for (int q = 0; q < kWarps; q++) agg += wcnt[q];
      uint64_t* stc = w.st_spa_cnt;
      uint32_t excl = 0;
      if (lt == 0) {
        if (lane == 0) st_rel_u64(stc + tile, lb_pack(tag_cnt, 2, agg));
      } else {
        if (lane == 0) st_rel_u64(stc + tile, lb_pack(tag_cnt, 1, agg));
        excl = lookback_sum(stc, tile, first, tag_cnt, w.ctr);
        if (lane == 0) st_rel_u64(stc + tile, lb_pack(tag_cnt, 2, excl + agg));
      }
      if (lane == 0) {
        sh_excl = excl;
        if (lt == (w.spa_start[g + 1] - first) - 1) w.ctl[s].s2[r] = excl + agg;
      }
    }
    __syncthreads();
    if (keep) {
      const int64_t cb = chain_base(sd, s, c, r) + 1 + sh_excl + pre;
      P* cp = reinterpret_cast<P*>(w.cpts);
      uint32_t o = 0;
#pragma unroll
      for (int k = 0; k < kSpaItems; k++) {
        if (keep & (1u << k)) {
          w.cidx[cb + o] = idx[k];
          cp[cb + o] = pt[k];
          o++;
        }
      }
    }
    __syncthreads();
  }
}

template <int DT>
__global__ void __launch_bounds__(kThreads) k_big(Job j, Ws w) {
  griddep_enter();
  const uint32_t total = w.ctr[CT_SORT_TOTAL];
  if (total == 0) {          // no multi-block set: one CTA plans the chains
    if (blockIdx.x == 0) plan_chain(j, w);
    return;
  }
  uint32_t gen = 0;
  if (blockIdx.x == 0) plan_spa(j, w);     // needs only the region counts
  big_hist(j, w, total);
  if (!grid_sync(w, gen)) return;
  for (int p = 0; p < kSortPasses; p++) {
    if (DT == DT_I32 && p >= 4 && p < 8) continue;   // zero key bytes
    big_pass(j, w, p, total);
    if (!grid_sync(w, gen)) return;
  }
  big_spa<DT>(j, w);
  if (!grid_sync(w, gen)) return;
  if (blockIdx.x == 0) plan_chain(j, w);
}

// ------------------------------------------- the paper's blocked SPA
//
// Comparison mode of cch_hull_stages (OPT_BLOCKED_SPA): SPA as the paper's
// GPU implementation runs it (Sec. 2.2.2): one thread block of 1024 threads
// per region, thread t checking the consecutive sorted points
// [t L, (t + 1) L), L = ceil(m / 1024), with Fig. 2's rule restarted at its
// chunk's first point (kept).  The region arrays of the paper hold the
// region's points only (the extremes are R0), so chunk 0 starts at its own
// first point too.  In this mode every set takes the multi-block sort, so
// the sorted records are in global memory; the chunked rule reads them
// after the pipeline and reports its survivors, while the hull itself comes
// from the exact sequential rule (a superset of its survivors would give the
// same hull).  Two kernels: the check (per record a keep byte, per region the
// count) and the stable compaction of the kept records' indices.
constexpr int kBlkThreads = 1024;

template <int DT>
__device__ __forceinline__ const uint32_t* sorted_vals(const Job& j, const Ws& w, const SetCtl& c) {
  const uint32_t* gh = w.hist;          // set 0
  int par = 0;
  for (int q = 0; q < kSortPasses; q++)
    par ^= __syncthreads_or(gh[q * 256 + (threadIdx.x & 255)] == c.s1) ? 0 : 1;
  return par ? w.valB : w.valA;
}

template <int DT>
__global__ void __launch_bounds__(kBlkThreads) k_spa_blocked(Job j, Ws w) {
  griddep_enter();
  using P = typename PtT<DT>::T;
  __shared__ uint32_t wsum[kBlkThreads / 32];
  const int r = blockIdx.x;                       // set 0, region r
  const SetDesc sd = get_set(j, 0);
  const SetCtl& c = w.ctl[0];
  if (c.status != 0 || !(c.flags & SF_BIG)) return;   // uniform
  const uint32_t* vin = sorted_vals<DT>(j, w, c);
  uint32_t roff = 0;
  for (int q = 0; q < r; q++) roff += c.cnt[q];
  const uint32_t m = c.cnt[r];
  const uint32_t L = (m + kBlkThreads - 1) / kBlkThreads;
  const uint32_t b0 = threadIdx.x * L, b1 = min(m, b0 + L);
  uint8_t* keep = reinterpret_cast<uint8_t*>(w.spvB) + sd.off + roff;
  uint64_t t = 0;
  uint32_t kept = 0;
  for (uint32_t i = b0; i < b1; i++) {
    const uint64_t v = spa_value<DT>(input_point<P>(j, sd.off + (vin[sd.off + roff + i] & kIdxMask)), r);
    const bool k = i == b0 || v <= t;              // Fig. 2: discard only the strictly worse
    if (k) { t = v; kept++; }
    keep[i] = k ? 1 : 0;
  }
  const uint32_t tot = __reduce_add_sync(0xFFFFFFFFu, kept);
  if ((threadIdx.x & 31) == 0) wsum[threadIdx.x >> 5] = tot;
  __syncthreads();
  if (threadIdx.x == 0) {
    uint32_t a = 0;
    for (int q = 0; q < kBlkThreads / 32; q++) a += wsum[q];
    w.ctl[0].sb[r] = a;
  }
}

template <int DT>
__global__ void __launch_bounds__(kBlkThreads) k_spa_blocked_out(Job j, Ws w, int32_t* spa_idx) {
  griddep_enter();
  __shared__ uint32_t wsum[kBlkThreads / 32];
  const int r = blockIdx.x;
  const SetDesc sd = get_set(j, 0);
  const SetCtl& c = w.ctl[0];
  if (c.status != 0 || !(c.flags & SF_BIG)) return;
  const uint32_t* vin = sorted_vals<DT>(j, w, c);
  uint32_t roff = 0, ooff = 0;
  for (int q = 0; q < r; q++) { roff += c.cnt[q]; ooff += c.sb[q]; }
  const uint32_t m = c.cnt[r];
  const uint32_t L = (m + kBlkThreads - 1) / kBlkThreads;
  const uint32_t b0 = threadIdx.x * L, b1 = min(m, b0 + L);
  const uint8_t* keep = reinterpret_cast<const uint8_t*>(w.spvB) + sd.off + roff;
  uint32_t n = 0;
  for (uint32_t i = b0; i < b1; i++) n += keep[i];
  // exclusive prefix of n over the block (thread order = chunk order)
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  uint32_t x = n;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t y = __shfl_up_sync(0xFFFFFFFFu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) wsum[warp] = x;
  __syncthreads();
  uint32_t pos = ooff + x - n;
  for (int q = 0; q < warp; q++) pos += wsum[q];
  for (uint32_t i = b0; i < b1; i++)
    if (keep[i]) spa_idx[pos++] = (int32_t)(vin[sd.off + roff + i] & kIdxMask);
}

int launch_spa_blocked(const Job& j, const Ws& w, int32_t* spa_idx, cudaStream_t st) {
  if (j.dtype != DT_I32) {   // float32 input: the float64 stages
    launch_pdl(k_spa_blocked<DT_F64>, 4, kBlkThreads, 0, st, j, w);
    launch_pdl(k_spa_blocked_out<DT_F64>, 4, kBlkThreads, 0, st, j, w, spa_idx);
  } else {
    launch_pdl(k_spa_blocked<DT_I32>, 4, kBlkThreads, 0, st, j, w);
    launch_pdl(k_spa_blocked_out<DT_I32>, 4, kBlkThreads, 0, st, j, w, spa_idx);
  }
  return 2;
}

int launch_big(const Job& j, const Ws& w, const Launch& L) {
  static int occ[3] = {0, 0, 0};
  const int k = j.dtype != DT_I32 ? 1 : 2;   // float32 input: the float64 stages
  void* fn = j.dtype != DT_I32 ? (void*)k_big<DT_F64> : (void*)k_big<DT_I32>;
  if (!occ[k]) {
    int b = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, fn, kThreads, 0) != cudaSuccess || b < 1) b = 1;
    occ[k] = b;
  }
  int64_t tiles_max = j.N / kSortTile + j.nsets;
  const int64_t spa_max = j.N / kSpaTile + 4 * (int64_t)j.nsets;
  if (spa_max > tiles_max) tiles_max = spa_max;
  int64_t cap = (int64_t)(L.grid_cap / 4) * occ[k];     // SMs x resident CTAs per SM
  if (cap > L.grid_cap) cap = L.grid_cap;
  int grid = (int)(tiles_max < cap ? tiles_max : cap);
  if (grid < 1) grid = 1;
  Job jj = j;
  Ws ww = w;
  void* args[] = {&jj, &ww};
  cudaLaunchCooperativeKernel(fn, dim3(grid), dim3(kThreads), args, 0, L.stream);
  return 1;
}

}  // namespace cch

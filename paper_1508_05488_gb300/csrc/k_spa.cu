// k_spa.cu -- second round of discarding: the Sorting-based Preprocessing
// Approach (Sec. 2.1.2, Fig. 2; step 5).
//
// Fig. 2 walks each sorted region once, keeping a point unless its compared
// coordinate is strictly worse than the running value t, which starts at the
// region's first extreme and is updated by every kept point.  Because a
// discarded point never lowers t, t before a point is the minimum over the
// first extreme and ALL earlier points; with the compared coordinate mapped
// to an order-preserving key v in "smaller is better" form
//     R1: v = key(y)   R2: v = ~key(x)   R3: v = ~key(y)   R4: v = key(x)
// a point survives iff  v <= min(v(E_r), exclusive prefix-min of v).
// That is a segmented exclusive prefix-minimum scan (associative), run here
// with a decoupled look-back, followed by a stable compaction of the
// survivors into the region's chain slots (positions 1 .. s2).  The paper's
// own GPU version restarts t in each of 1024 chunks (Sec. 2.2.2), which keeps
// a superset; the scan keeps exactly the sequential set.
#include "cch_internal.cuh"

namespace cch {

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

template <int DT>
__global__ void __launch_bounds__(kThreads) k_spa(Job j, Ws w) {
  using P = typename PtT<DT>::T;
  __shared__ uint32_t sh_tile;
  __shared__ uint64_t wmin[kWarps];
  __shared__ uint32_t wcnt[kWarps];
  __shared__ uint64_t sh_prefix;
  __shared__ uint32_t sh_excl;
  __shared__ int sh_last;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const uint32_t total = w.ctr[CT_SPA_TOTAL];
  if (total == 0) {          // no multi-block set: one CTA plans the chains
    if (blockIdx.x == 0) plan_chain(j, w);
    return;
  }
  const uint32_t tag_min = (j.epoch << 4) | 10u, tag_cnt = (j.epoch << 4) | 11u;
  const P* pts_all = reinterpret_cast<const P*>(j.pts);

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
    const P* pts = pts_all + sd.off;
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
        pt[k] = pts[idx[k]];
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
    if (threadIdx.x == 0) {
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
        st->inc_min = min(excl, agg);
        st_rel_u32(&st->flag, (tag_min << 16) | 2u);
      } else {
        st->agg_min = agg;
        st_rel_u32(&st->flag, (tag_min << 16) | 1u);
        int64_t t = (int64_t)tile - 1;
        uint32_t spins = 0;
        while (t >= (int64_t)first) {
          const SpaStat* q = w.st_spa + t;
          uint32_t f = ld_acq_u32(&q->flag);
          uint32_t kind = (f >> 16) == tag_min ? (f & 0xFFFFu) : 0u;
          if (kind == 0) {
            if (!spin_step(spins, w.ctr)) break;
            continue;
          }
          if (kind == 2) { excl = min(excl, *(volatile const uint64_t*)&q->inc_min); break; }
          excl = min(excl, *(volatile const uint64_t*)&q->agg_min);
          t--;
        }
        st->inc_min = min(excl, agg);
        st_rel_u32(&st->flag, (tag_min << 16) | 2u);
      }
      sh_prefix = excl;
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

  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    sh_last = atomicAdd(w.ctr + CT_SPA_DONE, 1u) == gridDim.x - 1;
  }
  __syncthreads();
  if (sh_last) {
    __threadfence();
    plan_chain(j, w);
  }
}

int launch_spa(const Job& j, const Ws& w, const Launch& L) {
  int64_t tiles_max = j.N / kSpaTile + 4 * (int64_t)j.nsets;
  int grid = (int)(tiles_max < L.grid_cap ? tiles_max : L.grid_cap);
  if (grid < 1) grid = 1;
  if (j.dtype == DT_F64) k_spa<DT_F64><<<grid, kThreads, 0, L.stream>>>(j, w);
  else k_spa<DT_I32><<<grid, kThreads, 0, L.stream>>>(j, w);
  return 1;
}

}  // namespace cch

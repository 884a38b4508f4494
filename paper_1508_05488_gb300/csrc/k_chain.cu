// k_chain.cu -- the simple polygon and its hull (Sec. 2.1 steps 6-7).
//
// Chain r of a set is E_r, the SPA survivors of region r in sorted order,
// E_{r+1}.  After SPA the chain is monotone in its Table 1 order (and in the
// other coordinate), so its part of the hull is the strictly convex chain
// obtained by keeping only left turns -- Andrew's monotone-chain pass in the
// frame of that order.  The paper runs Melkman's algorithm on the CPU for
// this step; here it runs on the device in three kernels:
//
//  k_chain_local  per block of 4096 chain positions: identical neighbours are
//                 dropped (the first index stays), every thread builds the
//                 convex chain of its 16 positions with a strict left-turn
//                 stack, and the 256 partial chains are merged pairwise in
//                 shared memory.  Partial chains are doubly linked lists.
//  k_chain_merge  merges the block chains of a region pairwise, level by
//                 level.  A merge walks the tail of the left chain backwards
//                 and the head of the right chain forwards until the bridge
//                 makes left turns at both ends; it costs O(1 + removed).
//  k_output       stable compaction of the surviving positions of the four
//                 chains of a set (each without its last point) into out_idx.
#include "cch_internal.cuh"

namespace cch {

template <int DT>
struct PT;
template <>
struct PT<DT_F64> { using T = double2; };
template <>
struct PT<DT_I32> { using T = int2; };

template <int DT>
__device__ __forceinline__ bool same_pt(const typename PT<DT>::T& a, const typename PT<DT>::T& b) {
  return a.x == b.x && a.y == b.y;   // value equality: -0.0 == +0.0
}

// Merge two adjacent convex chains given by (head, tail) into the left one.
// Links, flags, points and orientation go through the accessor (shared or
// global memory).
template <class A>
__device__ void merge_chains(A& acc, int& hl, int& tl, int hr, int tr) {
  if (hr < 0) return;
  if (hl < 0) { hl = hr; tl = tr; return; }
  int a = tl, b = hr;
  for (;;) {
    bool moved = false;
    while (a != hl && acc.orient(acc.prv(a), a, b) <= 0) {
      acc.kill(a);
      a = acc.prv(a);
      moved = true;
    }
    while (b != tr && acc.orient(a, b, acc.nxt(b)) <= 0) {
      acc.kill(b);
      b = acc.nxt(b);
      moved = true;
    }
    if (!moved) break;
  }
  acc.link(a, b);
  tl = tr;
}

// Orientation of three chain points: float64 through the FP32 filter on
// their views (when the set's coordinates allow), then exactly; int32
// exactly in 64/128-bit integers.
template <int DT>
__device__ __forceinline__ int orient_chain(const typename PT<DT>::T& a, const typename PT<DT>::T& b,
                                            const typename PT<DT>::T& c, float4 A, float4 B, float4 C,
                                            bool flag) {
  if constexpr (DT == DT_F64) return orient_f64_split(a, b, c, A, B, C, flag);
  else return orient_i32(a.x, a.y, b.x, b.y, c.x, c.y, flag);
}

template <int DT>
struct SmemAcc {
  typename PT<DT>::T* p;
  float4* f;          // FP32 split points (float64 only)
  uint16_t* pv;
  uint16_t* nx;
  uint8_t* al;
  bool flag;          // float64: filter usable; int32: wide products
  __device__ __forceinline__ int prv(int i) const { return pv[i]; }
  __device__ __forceinline__ int nxt(int i) const { return nx[i]; }
  __device__ __forceinline__ void kill(int i) { al[i] = 0; }
  __device__ __forceinline__ void link(int a, int b) { nx[a] = (uint16_t)b; pv[b] = (uint16_t)a; }
  __device__ __forceinline__ int orient(int i, int j, int k) const {
    if constexpr (DT == DT_F64) return orient_chain<DT>(p[i], p[j], p[k], f[i], f[j], f[k], flag);
    else return orient_chain<DT>(p[i], p[j], p[k], float4{}, float4{}, float4{}, flag);
  }
};

template <int DT>
struct GlobAcc {
  const typename PT<DT>::T* p;   // chain base applied
  uint32_t* pv;
  uint32_t* nx;
  uint8_t* al;
  bool flag;
  __device__ __forceinline__ int prv(int i) const { return (int)pv[i]; }
  __device__ __forceinline__ int nxt(int i) const { return (int)nx[i]; }
  __device__ __forceinline__ void kill(int i) { al[i] = 0; }
  __device__ __forceinline__ void link(int a, int b) { nx[a] = (uint32_t)b; pv[b] = (uint32_t)a; }
  __device__ __forceinline__ int orient(int i, int j, int k) const {
    const typename PT<DT>::T a = p[i], b = p[j], c = p[k];
    if constexpr (DT == DT_F64) return orient_chain<DT>(a, b, c, f64_split4(a), f64_split4(b), f64_split4(c), flag);
    else return orient_chain<DT>(a, b, c, float4{}, float4{}, float4{}, flag);
  }
};

// Asynchronous global -> shared copy of B (8 or 16) bytes, both B-aligned.
template <int B>
__device__ __forceinline__ void cp_async_copy(void* dst, const void* src) {
  static_assert(B == 8 || B == 16, "cp.async copies 8 or 16 bytes here");
  const uint32_t d = (uint32_t)__cvta_generic_to_shared(dst);
  if constexpr (B == 16) asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" :: "r"(d), "l"(src) : "memory");
  else asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" :: "r"(d), "l"(src) : "memory");
}

constexpr int kPeelRounds = 48;   // peeling rounds before the stack-and-merge fallback

// Exclusive prefix sum of one value per thread over the CTA; sh[kWarps]
// receives the total.  Ends with the CTA synchronised.
__device__ __forceinline__ int block_excl_sum(int v, int* sh) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  int x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int y = __shfl_up_sync(0xFFFFFFFFu, x, o);
    if (lane >= o) x += y;
  }
  __syncthreads();
  if (lane == 31) sh[warp] = x;
  __syncthreads();
  int pre = x - v, tot = 0;
  for (int q = 0; q < kWarps; q++) {
    if (q < warp) pre += sh[q];
    tot += sh[q];
  }
  __syncthreads();
  if (threadIdx.x == 0) sh[kWarps] = tot;
  __syncthreads();
  return pre;
}

// Positions i < m with al[i] != 0, in order, into out; returns their count.
__device__ __forceinline__ int block_compact(const uint8_t* al, int m, uint16_t* out, int* sh) {
  const int per = (m + kThreads - 1) / kThreads;
  const int i0 = threadIdx.x * per;
  int c = 0;
  for (int q = 0; q < per; q++) c += (i0 + q < m && al[i0 + q]) ? 1 : 0;
  int pre = block_excl_sum(c, sh);
  for (int q = 0; q < per; q++)
    if (i0 + q < m && al[i0 + q]) out[pre++] = (uint16_t)(i0 + q);
  const int n = sh[kWarps];
  __syncthreads();
  return n;
}

// Output of a set whose chains each fit one chain block (SF_LOCALOUT), by the
// last of its k_chain_local blocks: every block has left the indices of its
// chain's kept positions but the last (the next chain's first) compacted at
// the start of the chain's link slots (cprev) and their number in nal[r];
// the four lists are copied in order R1..R4 into out_idx (coalesced reads
// from L2: they were published before their blocks' arrival).
__device__ void chain_set_output(const Job& j, const Ws& w, const SetDesc& sd, int s, const SetCtl& c) {
  uint32_t off = 0;
#pragma unroll 1
  for (int r = 0; r < 4; r++) {
    const uint32_t nr = __ldcg(&c.nal[r]);
    const uint32_t* src = w.cprev + chain_base(sd, s, c, r);
    for (uint32_t k = threadIdx.x; k < nr; k += kThreads) j.out_idx[sd.off + off + k] = (int32_t)__ldcg(src + k);
    off += nr;
  }
  if (threadIdx.x == 0) j.out_counts[s] = (int32_t)off;
}

template <int DT>
constexpr size_t chain_local_smem() {
  return (size_t)kChainBlk * (sizeof(typename PT<DT>::T) + (DT == DT_F64 ? 16 : 0) + 2 + 2 + 2 + 1) +
         2 * kThreads * sizeof(int);
}

template <int DT>
__global__ void __launch_bounds__(kThreads) k_chain_local(Job j, Ws w) {
  griddep_enter();
  using P = typename PT<DT>::T;
  extern __shared__ __align__(16) unsigned char smem[];
  P* sp = reinterpret_cast<P*>(smem);
  float4* sf = reinterpret_cast<float4*>(sp + kChainBlk);              // split points (float64 only)
  uint16_t* pv = reinterpret_cast<uint16_t*>(DT == DT_F64 ? (void*)(sf + kChainBlk) : (void*)(sp + kChainBlk));
  uint16_t* nx = pv + kChainBlk;
  uint16_t* stk = nx + kChainBlk;
  int* gh = reinterpret_cast<int*>(stk + kChainBlk);
  int* gt = gh + kThreads;
  uint8_t* al = reinterpret_cast<uint8_t*>(gt + kThreads);
  __shared__ P pred;
  __shared__ int sh_cnt[kWarps + 1];
  __shared__ int sh_last;

  const uint32_t total = w.ctr[CT_CHAIN_TOTAL];
  P* cp = reinterpret_cast<P*>(w.cpts);
  for (uint32_t b = blockIdx.x; b < total; b += gridDim.x) {
    const int g = seg_of(w.chain_start, 4 * j.nsets, b);
    const int s = g >> 2, r = g & 3;
    const SetDesc sd = get_set(j, s);
    const SetCtl& c = w.ctl[s];
    const bool flag = DT == DT_F64 ? (c.flags & SF_SMALL) != 0 : (c.flags & SF_WIDE) != 0;
    const uint32_t lb = b - w.chain_start[g];
    const uint32_t L = c.s2[r] + 2;
    const int64_t cb = chain_base(sd, s, c, r);
    const uint32_t p0 = lb * kChainBlk;
    const int m = (int)min((uint32_t)kChainBlk, L - p0);
    // the block's points straight into shared memory (all copies in
    // flight at once); the chain's two extremes come from the set's record
    for (int i = threadIdx.x; i < m; i += kThreads) {
      const uint32_t p = p0 + i;
      if (p != 0 && p != L - 1) cp_async_copy<sizeof(P)>(&sp[i], &cp[cb + p]);
    }
    asm volatile("cp.async.wait_all;" ::: "memory");
    if (threadIdx.x < 2) {
      const uint32_t p = threadIdx.x == 0 ? 0u : L - 1;
      if (p >= p0 && p < p0 + (uint32_t)m) {
        const int k = p == 0 ? r : ((r + 1) & 3);
        P v;
        if constexpr (DT == DT_F64) { v.x = c.ex[k]; v.y = c.ey[k]; }
        else { v.x = (int)c.ex[k]; v.y = (int)c.ey[k]; }
        cp[cb + p] = v;
        w.cidx[cb + p] = c.eidx[k];
        sp[p - p0] = v;
      }
    }
    if constexpr (DT == DT_F64) {
      __syncthreads();
      for (int i = threadIdx.x; i < m; i += kThreads) sf[i] = f64_split4(sp[i]);
    }
    if (threadIdx.x == 0 && p0 > 0) pred = cp[cb + p0 - 1];
    __syncthreads();

    SmemAcc<DT> acc{sp, sf, pv, nx, al, flag};
    // identical neighbours: the first index stays
    for (int i = threadIdx.x; i < m; i += kThreads) {
      bool dup;
      if (i > 0) dup = same_pt<DT>(sp[i], sp[i - 1]);
      else dup = p0 > 0 && same_pt<DT>(sp[0], pred);
      al[i] = dup ? 0 : 1;
    }
    __syncthreads();
    // Peeling: every inner point of the block's current sequence that does
    // not make a strict left turn with its two current neighbours is no
    // strict vertex of the chain's hull (it lies on or inside the segment
    // between two chain points around it), so all of them go at once.  When
    // a round removes nothing the sequence is locally convex everywhere,
    // i.e. it is the block's convex chain.  The block's first and last points
    // stay (their neighbours lie in other blocks).
    uint16_t* cur = stk;
    uint16_t* nxt = nx;
    int n = block_compact(al, m, cur, sh_cnt);
    bool conv = false;
    for (int round = 0; round < kPeelRounds && !conv; round++) {
      const int per = (n + kThreads - 1) / kThreads;
      const int t0 = threadIdx.x * per;
      uint32_t keep = 0;
      for (int q = 0; q < per; q++) {
        const int t = t0 + q;
        if (t >= n) break;
        bool k = true;
        if (t > 0 && t < n - 1) k = acc.orient(cur[t - 1], cur[t], cur[t + 1]) > 0;
        keep |= (uint32_t)k << q;
      }
      const int nk = __popc(keep);
      int pre = block_excl_sum(nk, sh_cnt);
      const int n2 = sh_cnt[kWarps];
      for (int q = 0; q < per; q++) {
        const int t = t0 + q;
        if (t >= n) break;
        if ((keep >> q) & 1u) nxt[pre++] = cur[t];
        else al[cur[t]] = 0;
      }
      __syncthreads();
      conv = n2 == n;
      n = n2;
      uint16_t* tmp = cur; cur = nxt; nxt = tmp;
    }
    if (conv) {
      // links of the convex sequence (held in stk, so that nx is free)
      if (cur != stk) {
        for (int t = threadIdx.x; t < n; t += kThreads) stk[t] = cur[t];
        __syncthreads();
        cur = stk;
      }
      for (int t = threadIdx.x; t < n; t += kThreads) {
        const int i = cur[t];
        if (t > 0) pv[i] = cur[t - 1];
        if (t + 1 < n) nx[i] = cur[t + 1];
      }
      if (threadIdx.x == 0) {
        gh[0] = n ? cur[0] : -1;
        gt[0] = n ? cur[n - 1] : -1;
      }
    } else {
      // not converged: per thread a strict left-turn stack over its 16
      // positions (peeled points skipped), then pairwise merges
      __syncthreads();
      const int i0 = threadIdx.x * kChainItems;
      const int i1 = min(m, i0 + kChainItems);
      int top = 0;
      for (int i = i0; i < i1; i++) {
        if (!al[i]) continue;
        while (top >= 2 && acc.orient(stk[i0 + top - 2], stk[i0 + top - 1], i) <= 0) {
          al[stk[i0 + top - 1]] = 0;
          top--;
        }
        stk[i0 + top++] = (uint16_t)i;
      }
      for (int q = 0; q + 1 < top; q++) {
        nx[stk[i0 + q]] = stk[i0 + q + 1];
        pv[stk[i0 + q + 1]] = stk[i0 + q];
      }
      gh[threadIdx.x] = top ? stk[i0] : -1;
      gt[threadIdx.x] = top ? stk[i0 + top - 1] : -1;
      for (int step = 1; step < kThreads; step <<= 1) {
        __syncthreads();
        const int t = threadIdx.x;
        if ((t & (2 * step - 1)) == 0 && t + step < kThreads && (t + step) * kChainItems < m) {
          int hl = gh[t], tl = gt[t];
          merge_chains(acc, hl, tl, gh[t + step], gt[t + step]);
          gh[t] = hl;
          gt[t] = tl;
        }
      }
    }
    __syncthreads();
    if (c.flags & SF_LOCALOUT) {      // uniform: this block is all of chain r (p0 = 0, m = L)
      // the indices of the kept positions but the last, in order, at the
      // start of the chain's link slots (no merge or output pass follows)
      const int nout = block_compact(al, m - 1, stk, sh_cnt);
      for (int k = threadIdx.x; k < nout; k += kThreads) w.cprev[cb + k] = w.cidx[cb + stk[k]];
      __syncthreads();
      if (threadIdx.x == 0) {
        w.ctl[s].nal[r] = (uint32_t)nout;
        __threadfence();
        sh_last = atomicAdd(&w.ctl[s].arrive5, 1u) == c.nloc - 1u;
      }
      __syncthreads();
      if (sh_last) {
        __threadfence();
        chain_set_output(j, w, sd, s, c);
      }
      __syncthreads();
      continue;
    }
    for (int i = threadIdx.x; i < m; i += kThreads) {
      w.calive[cb + p0 + i] = al[i];
      if (al[i]) {
        w.cprev[cb + p0 + i] = p0 + pv[i];
        w.cnext[cb + p0 + i] = p0 + nx[i];
      }
    }
    if (threadIdx.x == 0) {
      w.blk_head[b] = gh[0] < 0 ? -1 : (int)(p0 + gh[0]);
      w.blk_tail[b] = gt[0] < 0 ? -1 : (int)(p0 + gt[0]);
    }
    __syncthreads();
  }
}

template <int DT>
__global__ void __launch_bounds__(kThreads) k_chain_merge(Job j, Ws w) {
  griddep_enter();
  using P = typename PT<DT>::T;
  const int nseg = 4 * j.nsets;
  for (int g = blockIdx.x; g < nseg; g += gridDim.x) {
    const uint32_t b0 = w.chain_start[g];
    const int B = (int)(w.chain_start[g + 1] - b0);
    if (B <= 1) continue;
    const int s = g >> 2, r = g & 3;
    const SetDesc sd = get_set(j, s);
    const SetCtl& c = w.ctl[s];
    const bool flag = DT == DT_F64 ? (c.flags & SF_SMALL) != 0 : (c.flags & SF_WIDE) != 0;
    const int64_t cb = chain_base(sd, s, c, r);
    GlobAcc<DT> acc{reinterpret_cast<const P*>(w.cpts) + cb, w.cprev + cb, w.cnext + cb, w.calive + cb, flag};
    for (int step = 1; step < B; step <<= 1) {
      for (int q = threadIdx.x; (int64_t)q * 2 * step < B; q += kThreads) {
        int left = q * 2 * step, right = left + step;
        if (right >= B) continue;
        int hl = w.blk_head[b0 + left], tl = w.blk_tail[b0 + left];
        merge_chains(acc, hl, tl, w.blk_head[b0 + right], w.blk_tail[b0 + right]);
        w.blk_head[b0 + left] = hl;
        w.blk_tail[b0 + left] = tl;
      }
      __syncthreads();
    }
  }
}

__global__ void __launch_bounds__(kThreads) k_output(Job j, Ws w) {
  griddep_enter();
  __shared__ uint32_t sh_tile;
  __shared__ int sh_last;
  __shared__ uint32_t cnt[kOutItems][kWarps];
  __shared__ uint32_t sh_excl;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const uint32_t total = w.ctr[CT_OUT_TOTAL];
  const uint32_t tag = (j.epoch << 4) | 12u;
  const uint32_t lt_mask = (1u << lane) - 1u;
  if (total == 0) {
    // every output was written before this kernel (by k_chain_local or the
    // chain plan): one CTA applies a device error of the call, if any
    if (blockIdx.x == 0) {
      const int err = (int)ld_acq_u32(w.ctr + CT_ERR);
      if (err != 0)
        for (int s = threadIdx.x; s < j.nsets; s += kThreads) j.out_counts[s] = err;
    }
    return;
  }
  for (;;) {
    if (threadIdx.x == 0) sh_tile = atomicAdd(w.ctr + CT_OUT_TILE, 1u);
    __syncthreads();
    const uint32_t tile = sh_tile;
    if (tile >= total) break;
    const int g = seg_of(w.out_start, 4 * j.nsets, tile);
    const int s = g >> 2, r = g & 3;
    const SetDesc sd = get_set(j, s);
    const SetCtl& c = w.ctl[s];
    const uint32_t lt = tile - w.out_start[g];
    const uint32_t first = w.out_start[4 * s];
    const uint32_t last = w.out_start[4 * s + 4] - 1;
    const uint32_t lim = c.s2[r] + 1;            // positions 0 .. L-2
    const int64_t cb = chain_base(sd, s, c, r);
    uint32_t keepm = 0;
#pragma unroll
    for (int k = 0; k < kOutItems; k++) {
      uint32_t p = lt * kOutTile + k * kThreads + threadIdx.x;
      bool keep = p < lim && w.calive[cb + p];
      uint32_t b = __ballot_sync(0xFFFFFFFFu, keep);
      if (lane == 0) cnt[k][warp] = __popc(b);
      keepm |= (keep ? 1u : 0u) << k;
    }
    __syncthreads();
    if (warp == 0) {
      constexpr int per = kOutItems * kWarps / 32;
      uint32_t loc[per];
      uint32_t sum = 0;
#pragma unroll
      for (int q = 0; q < per; q++) {
        int f = lane * per + q;
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
      for (int q = 0; q < per; q++) {
        int f = lane * per + q;
        cnt[f / kWarps][f % kWarps] = run;
        run += loc[q];
      }
      const uint32_t agg = __shfl_sync(0xFFFFFFFFu, x, 31);
      uint32_t excl = 0;
      if (tile == first) {
        if (lane == 0) st_rel_u64(w.st_out + tile, lb_pack(tag, 2, agg));
      } else {
        if (lane == 0) st_rel_u64(w.st_out + tile, lb_pack(tag, 1, agg));
        excl = lookback_sum(w.st_out, tile, first, tag, w.ctr);
        if (lane == 0) st_rel_u64(w.st_out + tile, lb_pack(tag, 2, excl + agg));
      }
      if (lane == 0) {
        sh_excl = excl;
        if (tile == last) j.out_counts[s] = (int32_t)(excl + agg);
      }
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < kOutItems; k++) {
      bool keep = (keepm >> k) & 1u;
      uint32_t b = __ballot_sync(0xFFFFFFFFu, keep);
      if (keep) {
        uint32_t p = lt * kOutTile + k * kThreads + threadIdx.x;
        uint32_t pos = sh_excl + cnt[k][warp] + __popc(b & lt_mask);
        j.out_idx[sd.off + pos] = (int32_t)w.cidx[cb + p];
      }
    }
    __syncthreads();
  }
  // last CTA out: a device-side error invalidates every result of the call
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    sh_last = atomicAdd(w.ctr + CT_OUT_DONE, 1u) == gridDim.x - 1;
  }
  __syncthreads();
  if (sh_last) {
    __threadfence();
    const int err = (int)ld_acq_u32(w.ctr + CT_ERR);
    if (err != 0)
      for (int s = threadIdx.x; s < j.nsets; s += kThreads) j.out_counts[s] = err;
  }
}

// ---------------------------------------------------- stage extraction
__global__ void k_extract_spa(Job j, Ws w, int32_t* spa_idx) {
  griddep_enter();
  const SetDesc sd = get_set(j, 0);
  const SetCtl& c = w.ctl[0];
  uint32_t o = 0;
  for (int r = 0; r < 4; r++) {
    const int64_t cb = chain_base(sd, 0, c, r);
    const uint32_t m = c.s2[r];
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < m; i += gridDim.x * blockDim.x)
      spa_idx[o + i] = (int32_t)w.cidx[cb + 1 + i];
    o += m;
  }
}

void launch_extract_spa(const Job& j, const Ws& w, int32_t* spa_idx, cudaStream_t st) {
  launch_pdl(k_extract_spa, 256, kThreads, 0, st, j, w, spa_idx);
}

int launch_chain(const Job& j, const Ws& w, const Launch& L) {
  int64_t blks_max = (j.N + 8 * (int64_t)j.nsets) / kChainBlk + 4 * (int64_t)j.nsets;
  int grid = (int)(blks_max < L.grid_cap ? blks_max : L.grid_cap);
  if (grid < 1) grid = 1;
  int gridm = 4 * j.nsets < L.grid_cap ? 4 * j.nsets : L.grid_cap;
  if (j.dtype != DT_I32) {   // float32 input: the float64 stages
    constexpr size_t sm = chain_local_smem<DT_F64>();
    static bool once = [] {
      cudaFuncSetAttribute(k_chain_local<DT_F64>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
      return true;
    }();
    (void)once;
    launch_pdl(k_chain_local<DT_F64>, grid, kThreads, sm, L.stream, j, w);
    launch_pdl(k_chain_merge<DT_F64>, gridm, kThreads, 0, L.stream, j, w);
  } else {
    constexpr size_t sm = chain_local_smem<DT_I32>();
    static bool once = [] {
      cudaFuncSetAttribute(k_chain_local<DT_I32>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
      return true;
    }();
    (void)once;
    launch_pdl(k_chain_local<DT_I32>, grid, kThreads, sm, L.stream, j, w);
    launch_pdl(k_chain_merge<DT_I32>, gridm, kThreads, 0, L.stream, j, w);
  }
  launch_pdl(k_output, grid, kThreads, 0, L.stream, j, w);
  return 3;
}

}  // namespace cch

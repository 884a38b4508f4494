// noalloc.cu -- cch_hull_noalloc: the hull of one small set with no device
// memory allocation at all.
//
// cch_hull takes its scratch workspace from cudaMalloc (once per stream, then
// reused).  Some callers cannot allow that: code that runs while a CUDA graph
// is being captured in a mode that forbids allocation, real-time or embedded
// callers that must fix their device-memory footprint at load time, and
// callers running inside a custom allocator (or its out-of-memory handler),
// where a nested cudaMalloc could deadlock or recurse.  This entry point
// serves them: its scratch is one file-scope __device__ array of fixed size,
// created when the library's device code is loaded and held by every GPU that
// loads it until the process exits.  It runs the same kernels as cch_hull, so
// its results are cch_hull's.
//
// Limits and rules (also in include/cch.h):
//   * at most kNoAllocMaxPoints points (sets of any larger size are rejected
//     with CCH_ERR_RANGE before anything is launched);
//   * every call on a device shares the one array and the array keeps the
//     last call's contents.  The array has one fixed layout, sized for the
//     largest call, so every buffer sits at the same place in every call.
//     The per-call control words are cleared by each call.  Look-back words
//     carry the call's epoch (1..4095) and read as "not ready" in any other
//     call; when the epoch wraps, the whole look-back region is cleared, so
//     no word of an earlier cycle can be taken for one of this call;
//   * calls whose work overlaps on the GPU (different streams, no ordering
//     between them) race on the shared array and give wrong results: order
//     them (one stream, or events);
//   * the first call on a device looks up the array's device address
//     (cudaGetSymbolAddress) and clears it; make that first call before any
//     stream capture.
#include <mutex>

#include "cch.h"
#include "cch_internal.cuh"

namespace cch {
namespace {

constexpr int64_t kNoAllocMaxPoints = int64_t(1) << 17;   // 131072 points
constexpr size_t kNoAllocBytes = size_t(12) << 20;        // 12 MiB

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];

constexpr int kMaxDevices = 64;
std::mutex g_na_mu;
char* g_na_ptr[kMaxDevices] = {};
uint32_t g_na_epoch[kMaxDevices] = {};
int g_na_sms[kMaxDevices] = {};

size_t na_up(size_t v) { return (v + 255) / 256 * 256; }

// Largest a1 chunk count and a2 tile count of any call: a1 chunks hold at
// least 4096 points, a2 tiles at least kClsMinTile.
constexpr int32_t kNaMaxChunk1 = (int32_t)((kNoAllocMaxPoints + 4095) / 4096);
constexpr int32_t kNaMaxTile2 = (int32_t)((kNoAllocMaxPoints + kClsMinTile - 1) / kClsMinTile);

// The one fixed layout of the array, sized for kNoAllocMaxPoints points and
// the largest chunk and tile counts, so that every buffer -- in particular
// the look-back words -- sits at the same address in every call, whatever its
// size or dtype (a call of fewer points uses a prefix of each buffer).
// Returns the bytes used; [0, ctl_bytes) is cleared by every call,
// [status_off, status_off + status_bytes) holds every look-back word.
size_t na_layout(char* base, Ws& w, size_t& ctl_bytes, size_t& status_off, size_t& status_bytes) {
  size_t o = 0;
  auto take = [&](size_t bytes) { size_t r = o; o = na_up(o + bytes); return base ? base + r : nullptr; };
  const int64_t n = kNoAllocMaxPoints;
  const int64_t nc = n + 8;
  const int64_t sort_tiles = n / kSortTile + 2;
  const int64_t spa_tiles = n / kSpaTile + 5;
  const int64_t chain_blks = nc / kChainBlk + 5;
  const int64_t out_tiles = nc / kOutTile + 5;
  w = Ws{};
  w.ctl = (SetCtl*)take(sizeof(SetCtl));
  w.ctr = (uint32_t*)take(sizeof(uint32_t) * CT_COUNT);
  w.ptot = (uint4*)take(16 * ((size_t)kNaMaxTile2 / kPlanTiles + 2));
  ctl_bytes = o;
  status_off = o;
  w.st_sort = (uint64_t*)take(8 * 256 * (size_t)sort_tiles);
  w.st_spa = (SpaStat*)take(sizeof(SpaStat) * (size_t)spa_tiles);
  w.st_spa_cnt = (uint64_t*)take(8 * (size_t)spa_tiles);
  w.st_out = (uint64_t*)take(8 * (size_t)out_tiles);
  status_bytes = o - status_off;
  w.part = (Part*)take(sizeof(Part) * (size_t)kNaMaxChunk1);
  w.tcnt = (uint64_t*)take(8 * 8 * (size_t)kNaMaxTile2);
  w.small_seg = (uint32_t*)take(16);
  w.keyA = (uint64_t*)take(8 * (size_t)n);
  w.keyB = (uint64_t*)take(8 * (size_t)n);
  w.valA = (uint32_t*)take(4 * (size_t)n);
  w.valB = (uint32_t*)take(4 * (size_t)n);
  w.spvA = (uint64_t*)take(8 * (size_t)n);
  w.spvB = (uint64_t*)take(8 * (size_t)n);
  w.hist = (uint32_t*)take(4 * (size_t)kSortPasses * 256);
  w.sort_start = (uint32_t*)take(8);
  w.spa_start = (uint32_t*)take(4 * 5);
  w.cpts = take(16 * (size_t)nc);
  w.cidx = (uint32_t*)take(4 * (size_t)nc);
  w.cprev = (uint32_t*)take(4 * (size_t)nc);
  w.cnext = (uint32_t*)take(4 * (size_t)nc);
  w.calive = (uint8_t*)take((size_t)nc);
  w.chain_start = (uint32_t*)take(4 * 5);
  w.blk_head = (int32_t*)take(4 * (size_t)chain_blks);
  w.blk_tail = (int32_t*)take(4 * (size_t)chain_blks);
  w.out_start = (uint32_t*)take(4 * 5);
  w.stairs = (uint32_t*)take(4 * 4 * (size_t)kStairB);
  return o;
}

}  // namespace
}  // namespace cch

using namespace cch;

extern "C" int cch_hull_noalloc(const void* points, int64_t n, int dtype, int32_t* out_idx,
                                int32_t* out_count, void* stream) {
  if (dtype != CCH_I32 && dtype != CCH_F64) return CCH_ERR_DTYPE;
  if (n < 0 || !out_idx || !out_count || (n > 0 && !points)) return CCH_ERR_INVALID;
  if ((uintptr_t)points % (dtype == CCH_F64 ? 16 : 8)) return CCH_ERR_INVALID;
  if (n > kNoAllocMaxPoints) return CCH_ERR_RANGE;
  cudaStream_t st = (cudaStream_t)stream;

  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return CCH_ERR_CUDA;

  // the same job description as cch_hull (one set)
  Job j{};
  j.pts = points;
  j.N = n;
  j.nsets = 1;
  j.dtype = dtype;
  j.out_idx = out_idx;
  j.out_counts = out_count;

  std::lock_guard<std::mutex> lk(g_na_mu);
  if (!g_na_sms[dev]) {
    int sms = 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms <= 0)
      return CCH_ERR_CUDA;
    g_na_sms[dev] = sms;
  }
  const int sms = g_na_sms[dev];
  const int target = sms * extremes_blocks_per_sm(dtype);
  int64_t len = (n + target - 1) / target;
  len = len < 4096 ? 4096 : (len + 1023) / 1024 * 1024;
  j.chunk1_len = len;
  j.nchunk1 = (int32_t)((n + len - 1) / len);
  j.ntile2 = (int32_t)((n + cls_tile(dtype) - 1) / cls_tile(dtype));
  j.tune = kTuneDefault;
  j.nchunk3 = n > 0 ? (int32_t)((stairs_sample(n, j.tune) + kStairChunk - 1) / kStairChunk) : 0;
  j.nchunkP = (j.ntile2 + kPlanTiles - 1) / kPlanTiles;
  j.sets = nullptr;
  j.one = SetDesc{0, n, 0, j.nchunk1, 0, j.ntile2, 0, j.nchunk3, 0, j.nchunkP};

  // set-up, once per device with that device current: the array's address
  if (!g_na_ptr[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) return CCH_ERR_CUDA;
    if (cudaMemsetAsync(p, 0, kNoAllocBytes, st) != cudaSuccess) return CCH_ERR_CUDA;
    g_na_ptr[dev] = (char*)p;
    g_na_epoch[dev] = 0;
  }
  Ws w;
  size_t ctl_bytes = 0, status_off = 0, status_bytes = 0;
  const size_t need = na_layout(g_na_ptr[dev], w, ctl_bytes, status_off, status_bytes);
  if (need > kNoAllocBytes) return CCH_ERR_RANGE;

  if (++g_na_epoch[dev] > 0xFFFu) {
    if (cudaMemsetAsync(g_na_ptr[dev] + status_off, 0, status_bytes, st) != cudaSuccess) return CCH_ERR_CUDA;
    g_na_epoch[dev] = 1;
  }
  j.epoch = g_na_epoch[dev];
  if (cudaMemsetAsync(g_na_ptr[dev], 0, ctl_bytes, st) != cudaSuccess) return CCH_ERR_CUDA;

  Launch L{st, sms * 4, 2 * sms};
  int nk = 0;
  nk += launch_extremes(j, w, L);
  nk += launch_stairs(j, w, L);
  nk += launch_classify(j, w, L);
  nk += launch_gather(j, w, L);
  nk += launch_small(j, w, L);
  nk += launch_big(j, w, L);
  nk += launch_chain(j, w, L);
  count_launches((uint64_t)nk);
  if (cudaGetLastError() != cudaSuccess) return CCH_ERR_CUDA;
  return CCH_OK;
}

// api.cu -- the C ABI (include/cch.h): argument checks, per-stream
// workspaces, launch planning and the kernel sequence of one call.
#include <algorithm>
#include <atomic>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <vector>

#include "cch.h"
#include "cch_internal.cuh"

namespace cch {
namespace {

constexpr size_t kAlign = 256;
size_t up(size_t v) { return (v + kAlign - 1) / kAlign * kAlign; }

struct Dims {
  int64_t N;
  int32_t nsets;
  int32_t nchunk1;
  int32_t ntile2;
  int64_t max_sort_tiles, max_spa_tiles, max_chain_blks, max_out_tiles, Nc;
};

Dims make_dims(int64_t N, int32_t nsets, int32_t nchunk1, int32_t ntile2) {
  Dims d;
  d.N = N;
  d.nsets = nsets;
  d.nchunk1 = nchunk1;
  d.ntile2 = ntile2;
  d.Nc = N + 8 * (int64_t)nsets;
  d.max_sort_tiles = N / kSortTile + nsets + 1;
  d.max_spa_tiles = N / kSpaTile + 4 * (int64_t)nsets + 1;
  d.max_chain_blks = d.Nc / kChainBlk + 4 * (int64_t)nsets + 1;
  d.max_out_tiles = d.Nc / kOutTile + 4 * (int64_t)nsets + 1;
  return d;
}

// Byte layout of a workspace; `base` null -> sizes only.
struct Layout {
  size_t total = 0;
  size_t ctl_bytes = 0;                  // ctl + ctr (cleared each call)
  size_t status_off = 0, status_bytes = 0;   // look-back words (cleared on epoch wrap)
  size_t sets_off = 0;
  Ws w{};
};

Layout layout(const Dims& d, char* base) {
  Layout L;
  size_t o = 0;
  auto take = [&](size_t bytes) { size_t r = o; o = up(o + bytes); return base ? base + r : nullptr; };
  L.w.ctl = (SetCtl*)take(sizeof(SetCtl) * d.nsets);
  L.w.ctr = (uint32_t*)take(sizeof(uint32_t) * CT_COUNT);
  L.w.ptot = (uint4*)take(16 * ((size_t)d.ntile2 / kPlanTiles + d.nsets + 1));
  L.ctl_bytes = o;
  L.status_off = o;
  L.w.st_sort = (uint64_t*)take(8 * 256 * (size_t)d.max_sort_tiles);
  L.w.st_spa = (SpaStat*)take(sizeof(SpaStat) * (size_t)d.max_spa_tiles);
  L.w.st_spa_cnt = (uint64_t*)take(8 * (size_t)d.max_spa_tiles);
  L.w.st_out = (uint64_t*)take(8 * (size_t)d.max_out_tiles);
  L.status_bytes = o - L.status_off;
  L.w.part = (Part*)take(sizeof(Part) * (size_t)std::max(d.nchunk1, 1));
  L.w.tcnt = (uint64_t*)take(8 * 8 * (size_t)std::max(d.ntile2, 1));
  L.w.small_seg = (uint32_t*)take(4 * 4 * (size_t)d.nsets);
  L.w.keyA = (uint64_t*)take(8 * (size_t)d.N);
  L.w.keyB = (uint64_t*)take(8 * (size_t)d.N);
  L.w.valA = (uint32_t*)take(4 * (size_t)d.N);
  L.w.valB = (uint32_t*)take(4 * (size_t)d.N);
  L.w.spvA = (uint64_t*)take(8 * (size_t)d.N);
  L.w.spvB = (uint64_t*)take(8 * (size_t)d.N);
  L.w.hist = (uint32_t*)take(4 * (size_t)kSortPasses * 256 * d.nsets);
  L.w.sort_start = (uint32_t*)take(4 * ((size_t)d.nsets + 1));
  L.w.spa_start = (uint32_t*)take(4 * (4 * (size_t)d.nsets + 1));
  L.w.cpts = take(16 * (size_t)d.Nc);
  L.w.cidx = (uint32_t*)take(4 * (size_t)d.Nc);
  L.w.cprev = (uint32_t*)take(4 * (size_t)d.Nc);
  L.w.cnext = (uint32_t*)take(4 * (size_t)d.Nc);
  L.w.calive = (uint8_t*)take((size_t)d.Nc);
  L.w.chain_start = (uint32_t*)take(4 * (4 * (size_t)d.nsets + 1));
  L.w.blk_head = (int32_t*)take(4 * (size_t)d.max_chain_blks);
  L.w.blk_tail = (int32_t*)take(4 * (size_t)d.max_chain_blks);
  L.w.out_start = (uint32_t*)take(4 * (4 * (size_t)d.nsets + 1));
  L.w.stairs = (uint32_t*)take(4 * 4 * (size_t)kStairB * d.nsets);
  L.sets_off = o;
  take(sizeof(SetDesc) * (size_t)d.nsets);
  L.total = o;
  return L;
}

struct Workspace {
  char* dev = nullptr;
  size_t bytes = 0;
  Dims cap{};
  uint32_t epoch = 0;
  SetDesc* host_sets = nullptr;      // pinned staging of the set table
  size_t host_sets_cap = 0;
  cudaEvent_t sets_done = nullptr;   // staging buffer free again
  void* h2d = nullptr;               // device copy of host points (cch_hull_host)
  size_t h2d_bytes = 0;
  int32_t* dcount = nullptr;         // device counts (cch_hull_host)
  int32_t* didx = nullptr;
  size_t didx_bytes = 0;
};

std::mutex g_mu;
std::map<cudaStream_t, Workspace*> g_ws;
std::atomic<uint64_t> g_launches{0};

// Optional stage timing: CUDA events around the stages of every call, read
// back (and summed) by cch_profile_read.
constexpr int kStages = 8;   // a1, stairs, a2, gather, small path, multi-block path, chain, blocked SPA
struct ProfRec { cudaEvent_t ev[kStages + 1]; uint32_t mask; };
uint32_t g_prof = 0;   // stages whose boundaries get events (bit k: stage k)
std::vector<ProfRec> g_prof_pending, g_prof_free;

cudaEvent_t* prof_begin(ProfRec& rec) {
  if (!g_prof) return nullptr;
  if (!g_prof_free.empty()) { rec = g_prof_free.back(); g_prof_free.pop_back(); }
  else for (auto& e : rec.ev) cudaEventCreate(&e);
  rec.mask = g_prof;
  return rec.ev;
}
int g_sms = 0;
int g_occ[4] = {0, 0, 0, 0};   // a1 CTAs per SM, by input format

int sm_count() {
  if (g_sms == 0) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&g_sms, cudaDevAttrMultiProcessorCount, dev);
    if (g_sms <= 0) g_sms = 1;
  }
  return g_sms;
}

bool fits(const Dims& c, const Dims& d) {
  return d.N <= c.N && d.nsets <= c.nsets && d.nchunk1 <= c.nchunk1 && d.ntile2 <= c.ntile2;
}

// Get (or grow) the workspace of `stream` for dims `d`.  Called with g_mu held.
int acquire(cudaStream_t stream, const Dims& d, Workspace** out) {
  Workspace*& ws = g_ws[stream];
  if (!ws) ws = new Workspace();
  if (!ws->dev || !fits(ws->cap, d)) {
    Dims c = d;
    if (ws->dev) {   // grow by at least 1.5x to amortise
      c.N = std::max(d.N, ws->cap.N + ws->cap.N / 2);
      c.nsets = std::max(d.nsets, ws->cap.nsets);
      c.nchunk1 = std::max(d.nchunk1, ws->cap.nchunk1);
      c.ntile2 = std::max(d.ntile2, ws->cap.ntile2);
      c = make_dims(c.N, c.nsets, c.nchunk1, (int32_t)std::max<int64_t>(c.ntile2, c.N / kClsMinTile + c.nsets + 1));
      if (cudaStreamSynchronize(stream) != cudaSuccess) return CCH_ERR_CUDA;
      cudaFree(ws->dev);
      ws->dev = nullptr;
    }
    Layout L = layout(c, nullptr);
    if (cudaMalloc(&ws->dev, L.total) != cudaSuccess) {
      cudaGetLastError();
      ws->dev = nullptr;
      return CCH_ERR_NOMEM;
    }
    if (cudaMemsetAsync(ws->dev, 0, L.total, stream) != cudaSuccess) return CCH_ERR_CUDA;
    ws->bytes = L.total;
    ws->cap = c;
    ws->epoch = 0;
  }
  *out = ws;
  return CCH_OK;
}

int a1_target(int dtype) {
  if (!g_occ[dtype]) g_occ[dtype] = extremes_blocks_per_sm(dtype);
  return sm_count() * g_occ[dtype];
}

int grid_cap() { return sm_count() * 4; }

// Launch the whole pipeline for the job; `sets_host` is the set table for a
// batch (nullptr for a single set).  `stages` hooks the stage extraction.
struct StageOut {
  int32_t* r1_idx;
  int32_t* r1_region;
  int32_t* spa_idx;
};

int run(Job& j, const std::vector<SetDesc>* sets_host, cudaStream_t stream, StageOut* stages,
        Workspace** ws_out) {
  Dims d = make_dims(j.N, j.nsets, j.nchunk1, j.ntile2);
  std::lock_guard<std::mutex> lk(g_mu);
  Workspace* ws = nullptr;
  int st = acquire(stream, d, &ws);
  if (st != CCH_OK) return st;
  Layout L = layout(ws->cap, ws->dev);
  if (++ws->epoch > 0xFFFu) {
    if (cudaMemsetAsync(ws->dev + L.status_off, 0, L.status_bytes, stream) != cudaSuccess) return CCH_ERR_CUDA;
    ws->epoch = 1;
  }
  j.epoch = ws->epoch;
  if (cudaMemsetAsync(ws->dev, 0, L.ctl_bytes, stream) != cudaSuccess) return CCH_ERR_CUDA;
  if (sets_host) {
    size_t bytes = sizeof(SetDesc) * sets_host->size();
    if (ws->host_sets_cap < sets_host->size()) {
      if (ws->host_sets) { cudaEventSynchronize(ws->sets_done); cudaFreeHost(ws->host_sets); }
      if (cudaMallocHost(&ws->host_sets, bytes) != cudaSuccess) { ws->host_sets = nullptr; ws->host_sets_cap = 0; return CCH_ERR_NOMEM; }
      ws->host_sets_cap = sets_host->size();
      if (!ws->sets_done) cudaEventCreateWithFlags(&ws->sets_done, cudaEventDisableTiming);
    } else if (ws->sets_done) {
      cudaEventSynchronize(ws->sets_done);
    }
    memcpy(ws->host_sets, sets_host->data(), bytes);
    SetDesc* dsets = reinterpret_cast<SetDesc*>(ws->dev + L.sets_off);
    if (cudaMemcpyAsync(dsets, ws->host_sets, bytes, cudaMemcpyHostToDevice, stream) != cudaSuccess) return CCH_ERR_CUDA;
    cudaEventRecord(ws->sets_done, stream);
    j.sets = dsets;
  }
  if (stages) { j.r1_idx = stages->r1_idx; j.r1_region = stages->r1_region; }
  Launch La{stream, grid_cap(), j.tune.cls_per_sm * sm_count()};
  ProfRec rec{};
  cudaEvent_t* ev = prof_begin(rec);
  int nk = 0;
  // event k marks the start of stage k (and the end of stage k - 1)
  auto mark = [&](int k) {
    if (ev && ((rec.mask >> k) & 1u || (k > 0 && (rec.mask >> (k - 1)) & 1u))) cudaEventRecord(ev[k], stream);
  };
  mark(0);
  nk += launch_extremes(j, L.w, La);
  mark(1);
  nk += launch_stairs(j, L.w, La);
  mark(2);
  nk += launch_classify(j, L.w, La);
  mark(3);
  nk += launch_gather(j, L.w, La);
  mark(4);
  nk += launch_small(j, L.w, La);
  mark(5);
  nk += launch_big(j, L.w, La);
  mark(6);
  nk += launch_chain(j, L.w, La);
  mark(7);
  if (stages) {
    if (j.opts & OPT_BLOCKED_SPA) nk += launch_spa_blocked(j, L.w, stages->spa_idx, stream);
    else { launch_extract_spa(j, L.w, stages->spa_idx, stream); nk++; }
  }
  mark(8);
  if (ev) g_prof_pending.push_back(rec);
  g_launches += (uint64_t)nk;
  if (cudaGetLastError() != cudaSuccess) return CCH_ERR_CUDA;
  if (ws_out) *ws_out = ws;
  return CCH_OK;
}

int check_common(const void* points, int64_t n, int dtype, const void* out_idx, const void* out_count) {
  if (dtype != CCH_I32 && dtype != CCH_F64) return CCH_ERR_DTYPE;
  if (n < 0 || !out_idx || !out_count) return CCH_ERR_INVALID;
  if (n > 0 && !points) return CCH_ERR_INVALID;
  if (n > kMaxSetPoints) return CCH_ERR_RANGE;
  uintptr_t a = (uintptr_t)points;
  if (a % (dtype == CCH_F64 ? 16 : 8)) return CCH_ERR_INVALID;
  return CCH_OK;
}

// Single-set job.
Job single_job(const void* points, int64_t n, int dtype, int32_t* out_idx, int32_t* out_count,
               uint32_t opts) {
  Job j{};
  j.pts = points;
  j.N = n;
  j.nsets = 1;
  j.dtype = dtype;
  j.opts = opts;
  j.tune = tune_for(dtype, n, 1);
  int target = a1_target(dtype);
  int64_t len = (n + target - 1) / std::max(target, 1);
  len = std::max<int64_t>(j.tune.a1_len_min, (len + 1023) / 1024 * 1024);
  j.chunk1_len = len;
  int32_t nch = (int32_t)((n + len - 1) / len);
  j.nchunk1 = nch;
  const int ct = cls_tile(dtype);
  j.ntile2 = (int32_t)((n + ct - 1) / ct);
  j.nchunk3 = n > 0 ? (int32_t)((stairs_sample(n, j.tune) + kStairChunk - 1) / kStairChunk) : 0;
  j.nchunkP = (j.ntile2 + kPlanTiles - 1) / kPlanTiles;
  j.sets = nullptr;
  j.one = SetDesc{0, n, 0, nch, 0, j.ntile2, 0, j.nchunk3, 0, j.nchunkP};
  j.out_idx = out_idx;
  j.out_counts = out_count;
  return j;
}

// ------------------------------------------------ float32 SoA input

}  // namespace

void count_launches(uint64_t n) { g_launches += n; }

}  // namespace cch

using namespace cch;

extern "C" {

const char* cch_status_string(int status) {
  switch (status) {
    case CCH_OK: return "ok";
    case CCH_ERR_INVALID: return "invalid argument";
    case CCH_ERR_DTYPE: return "unsupported dtype (use CCH_I32 or CCH_F64)";
    case CCH_ERR_NONFINITE: return "non-finite float64 coordinate";
    case CCH_ERR_RANGE: return "size or coordinate magnitude outside the supported range";
    case CCH_ERR_NOMEM: return "out of memory";
    case CCH_ERR_CUDA: return "CUDA runtime error";
    case CCH_ERR_TIMEOUT: return "bounded device wait expired";
    case CCH_ERR_BUSY: return "server queue full";
    case CCH_ERR_NOTFOUND: return "unknown ticket";
    default: return "unknown status";
  }
}

int cch_hull(const void* points, int64_t n, int dtype, int32_t* out_idx, int32_t* out_count,
             void* stream) {
  int st = check_common(points, n, dtype, out_idx, out_count);
  if (st != CCH_OK) return st;
  Job j = single_job(points, n, dtype, out_idx, out_count, 0);
  return run(j, nullptr, (cudaStream_t)stream, nullptr, nullptr);
}

int cch_hull_batched(const void* points, const int64_t* offsets, int32_t nsets, int dtype,
                     int32_t* out_idx, int32_t* out_counts, void* stream) {
  if (dtype != CCH_I32 && dtype != CCH_F64) return CCH_ERR_DTYPE;
  if (nsets < 0 || !offsets || !out_idx || !out_counts) return CCH_ERR_INVALID;
  if (nsets == 0) return CCH_OK;
  if (offsets[0] != 0) return CCH_ERR_INVALID;
  const int64_t N = offsets[nsets];
  if (N > 0x7FFFFFFFll) return CCH_ERR_RANGE;
  if (N > 0 && !points) return CCH_ERR_INVALID;
  if ((uintptr_t)points % (dtype == CCH_F64 ? 16 : 8)) return CCH_ERR_INVALID;
  std::vector<SetDesc> sets(nsets);
  const Tune tune = tune_for(dtype, N, nsets);
  int target = a1_target(dtype);
  int64_t len = std::max<int64_t>(tune.a1_len_min, ((N + target - 1) / std::max(target, 1) + 1023) / 1024 * 1024);
  int64_t nch = 0, nt = 0, n3 = 0, np_ = 0;
  const int ct = cls_tile(dtype);
  for (int32_t s = 0; s < nsets; s++) {
    int64_t n = offsets[s + 1] - offsets[s];
    if (n < 0) return CCH_ERR_INVALID;
    if (n > kMaxSetPoints) return CCH_ERR_RANGE;
    int32_t c = (int32_t)((n + len - 1) / len);
    int32_t t = (int32_t)((n + ct - 1) / ct);
    int32_t c3 = n > 0 ? (int32_t)((stairs_sample(n, tune) + kStairChunk - 1) / kStairChunk) : 0;
    int32_t cp = (t + kPlanTiles - 1) / kPlanTiles;
    sets[s] = SetDesc{offsets[s], n, (int32_t)nch, c, (int32_t)nt, t, (int32_t)n3, c3, (int32_t)np_, cp};
    nch += c;
    nt += t;
    n3 += c3;
    np_ += cp;
  }
  Job j{};
  j.pts = points;
  j.N = N;
  j.nsets = nsets;
  j.dtype = dtype;
  j.tune = tune;
  j.nchunk1 = (int32_t)nch;
  j.ntile2 = (int32_t)nt;
  j.nchunk3 = (int32_t)n3;
  j.nchunkP = (int32_t)np_;
  j.chunk1_len = len;
  j.out_idx = out_idx;
  j.out_counts = out_counts;
  return run(j, &sets, (cudaStream_t)stream, nullptr, nullptr);
}

int cch_hull_host(const void* points_host, int64_t n, int dtype, int32_t* out_idx_host,
                  int32_t* out_count, void* stream) {
  if (dtype != CCH_I32 && dtype != CCH_F64) return CCH_ERR_DTYPE;
  if (n < 0 || !out_idx_host || !out_count || (n > 0 && !points_host)) return CCH_ERR_INVALID;
  if (n > kMaxSetPoints) return CCH_ERR_RANGE;
  cudaStream_t s = (cudaStream_t)stream;
  const size_t pbytes = (size_t)n * (dtype == CCH_F64 ? 16 : 8);
  void* dpts = nullptr;
  int32_t* dcount = nullptr;
  int32_t* didx = nullptr;
  {
    std::lock_guard<std::mutex> lk(g_mu);
    Workspace*& ws = g_ws[s];
    if (!ws) ws = new Workspace();
    if (ws->h2d_bytes < pbytes) {
      if (ws->h2d) { cudaStreamSynchronize(s); cudaFree(ws->h2d); }
      ws->h2d = nullptr;
      ws->h2d_bytes = 0;
      if (cudaMalloc(&ws->h2d, pbytes) != cudaSuccess) { cudaGetLastError(); return CCH_ERR_NOMEM; }
      ws->h2d_bytes = pbytes;
    }
    size_t ib = 4 * (size_t)std::max<int64_t>(n, 1);
    if (ws->didx_bytes < ib) {
      if (ws->didx) { cudaStreamSynchronize(s); cudaFree(ws->didx); }
      ws->didx = nullptr;
      ws->didx_bytes = 0;
      if (cudaMalloc(&ws->didx, ib) != cudaSuccess) { cudaGetLastError(); return CCH_ERR_NOMEM; }
      ws->didx_bytes = ib;
    }
    if (!ws->dcount && cudaMalloc(&ws->dcount, 16) != cudaSuccess) { cudaGetLastError(); return CCH_ERR_NOMEM; }
    dpts = ws->h2d;
    dcount = ws->dcount;
    didx = ws->didx;
  }
  if (pbytes && cudaMemcpyAsync(dpts, points_host, pbytes, cudaMemcpyHostToDevice, s) != cudaSuccess)
    return CCH_ERR_CUDA;
  int st = cch_hull(dpts, n, dtype, didx, dcount, stream);
  if (st != CCH_OK) return st;
  if (cudaMemcpyAsync(out_count, dcount, 4, cudaMemcpyDeviceToHost, s) != cudaSuccess) return CCH_ERR_CUDA;
  if (cudaStreamSynchronize(s) != cudaSuccess) return CCH_ERR_CUDA;
  if (*out_count < 0) return *out_count;
  if (*out_count > 0 &&
      cudaMemcpyAsync(out_idx_host, didx, 4 * (size_t)*out_count, cudaMemcpyDeviceToHost, s) != cudaSuccess)
    return CCH_ERR_CUDA;
  if (cudaStreamSynchronize(s) != cudaSuccess) return CCH_ERR_CUDA;
  return CCH_OK;
}

int cch_hull_f32soa(const float* x, const float* y, int64_t n, int32_t* out_idx, int32_t* out_count,
                    void* stream) {
  if (n < 0 || !out_idx || !out_count || (n > 0 && (!x || !y))) return CCH_ERR_INVALID;
  if ((((uintptr_t)x | (uintptr_t)y) & 3u) != 0) return CCH_ERR_INVALID;
  if (n > kMaxSetPoints) return CCH_ERR_RANGE;
  Job j = single_job(x, n, DT_F32, out_idx, out_count, 0);
  j.ys = y;
  return run(j, nullptr, (cudaStream_t)stream, nullptr, nullptr);
}

int cch_hull_stages(const void* points, int64_t n, int dtype, uint32_t opts, int32_t* r1_idx,
                    int32_t* r1_region, int32_t* spa_idx, int64_t* counts_host, int32_t* out_idx,
                    int32_t* out_count, void* stream) {
  int st = check_common(points, n, dtype, out_idx, out_count);
  if (st != CCH_OK) return st;
  if (!r1_idx || !r1_region || !spa_idx || !counts_host) return CCH_ERR_INVALID;
  if (opts & ~(uint32_t)(OPT_NO_FILTER | OPT_NO_PREFILTER | OPT_BLOCKED_SPA | OPT_OCTAGON)) return CCH_ERR_INVALID;
  if (opts & (OPT_BLOCKED_SPA | OPT_OCTAGON)) opts |= OPT_NO_PREFILTER;   // the paper's round 1 (or its octagon form)
  Job j = single_job(points, n, dtype, out_idx, out_count, opts);
  StageOut so{r1_idx, r1_region, spa_idx};
  Workspace* ws = nullptr;
  cudaStream_t s = (cudaStream_t)stream;
  st = run(j, nullptr, s, &so, &ws);
  if (st != CCH_OK) return st;
  SetCtl c;
  uint32_t ctr[CT_COUNT];
  Layout L = layout(ws->cap, ws->dev);
  if (cudaMemcpyAsync(&c, L.w.ctl, sizeof(SetCtl), cudaMemcpyDeviceToHost, s) != cudaSuccess) return CCH_ERR_CUDA;
  if (cudaMemcpyAsync(ctr, L.w.ctr, sizeof(ctr), cudaMemcpyDeviceToHost, s) != cudaSuccess) return CCH_ERR_CUDA;
  if (cudaStreamSynchronize(s) != cudaSuccess) return CCH_ERR_CUDA;
  counts_host[0] = c.s1;
  for (int r = 0; r < 4; r++) counts_host[1 + r] = c.cnt[r];
  for (int r = 0; r < 4; r++) counts_host[5 + r] = (opts & OPT_BLOCKED_SPA) ? c.sb[r] : c.s2[r];
  counts_host[9] = c.status != 0 ? c.status : (int32_t)ctr[CT_ERR];
  counts_host[10] = c.passes;
  for (int r = 0; r < 4; r++) counts_host[11 + r] = (opts & OPT_OCTAGON) ? c.didx[r] : -1;
  counts_host[15] = 0;
  return CCH_OK;
}

int cch_profile(int enable) {
  std::lock_guard<std::mutex> lk(g_mu);
  g_prof = enable != 0 ? (1u << kStages) - 1u : 0u;
  return CCH_OK;
}

int cch_profile_stages(uint32_t mask) {
  std::lock_guard<std::mutex> lk(g_mu);
  g_prof = mask & ((1u << kStages) - 1u);
  return CCH_OK;
}

int cch_profile_read(double* stage_ms, int max_stages, int64_t* calls) {
  std::lock_guard<std::mutex> lk(g_mu);
  if (!stage_ms || max_stages < 0) return CCH_ERR_INVALID;
  for (int k = 0; k < max_stages; k++) stage_ms[k] = 0.0;
  int64_t n = 0;
  for (auto& rec : g_prof_pending) {
    int last = 0;
    for (int k = 0; k < kStages; k++)
      if ((rec.mask >> k) & 1u) last = k + 1;
    if (cudaEventSynchronize(rec.ev[last]) != cudaSuccess) return CCH_ERR_CUDA;
    for (int k = 0; k < kStages && k < max_stages; k++) {
      if (!((rec.mask >> k) & 1u)) continue;
      float ms = 0.f;
      cudaEventElapsedTime(&ms, rec.ev[k], rec.ev[k + 1]);
      stage_ms[k] += ms;
    }
    g_prof_free.push_back(rec);
    n++;
  }
  g_prof_pending.clear();
  if (calls) *calls = n;
  return kStages;
}

uint64_t cch_launch_count(void) { return g_launches.load(); }

namespace cch {
namespace {
// One thread waits on a flag that nothing sets, with the library's bounded
// wait; the error word it records is the result.
__global__ void k_selftest_wait(uint32_t* words, int32_t* status) {
  uint32_t* flag = words + CT_COUNT;
  uint32_t spins = 0;
  while (ld_acq_u32(flag) == 0)
    if (!spin_step(spins, words)) break;
  *status = (int32_t)ld_acq_u32(words + CT_ERR);
}
}  // namespace
}  // namespace cch

int cch_selftest_wait(int32_t* status_dev, void* stream) {
  if (!status_dev) return CCH_ERR_INVALID;
  static uint32_t* words = nullptr;           // CT_COUNT error words + the flag
  {
    std::lock_guard<std::mutex> lk(g_mu);
    if (!words && cudaMalloc(&words, sizeof(uint32_t) * (CT_COUNT + 1)) != cudaSuccess) {
      cudaGetLastError();
      words = nullptr;
      return CCH_ERR_NOMEM;
    }
  }
  cudaStream_t st = (cudaStream_t)stream;
  if (cudaMemsetAsync(words, 0, sizeof(uint32_t) * (CT_COUNT + 1), st) != cudaSuccess) return CCH_ERR_CUDA;
  k_selftest_wait<<<1, 1, 0, st>>>(words, status_dev);
  g_launches += 1;
  return cudaGetLastError() == cudaSuccess ? CCH_OK : CCH_ERR_CUDA;
}

size_t cch_workspace_bytes(int64_t n, int dtype) {
  if (n < 0 || (dtype != CCH_I32 && dtype != CCH_F64)) return 0;
  int target = 1216;
  int64_t len = std::max<int64_t>(4096, ((n + target - 1) / target + 1023) / 1024 * 1024);
  Dims d = make_dims(n, 1, (int32_t)((n + len - 1) / len), (int32_t)((n + cls_tile(dtype) - 1) / cls_tile(dtype)));
  return layout(d, nullptr).total;
}

void cch_release_workspace(void) {
  std::lock_guard<std::mutex> lk(g_mu);
  cudaDeviceSynchronize();
  serve_release_pinned();
  for (auto& kv : g_ws) {
    Workspace* ws = kv.second;
    if (ws->dev) cudaFree(ws->dev);
    if (ws->host_sets) cudaFreeHost(ws->host_sets);
    if (ws->sets_done) cudaEventDestroy(ws->sets_done);
    if (ws->h2d) cudaFree(ws->h2d);
    if (ws->dcount) cudaFree(ws->dcount);
    if (ws->didx) cudaFree(ws->didx);
    delete ws;
  }
  g_ws.clear();
}

}  // extern "C"

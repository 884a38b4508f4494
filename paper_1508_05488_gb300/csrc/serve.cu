// serve.cu -- the hull server of include/cch.h.
//
// Requests are copied at submit into pinned host memory from a pool (several
// threads share large copies; the caller keeps no obligation), queued, and
// admitted in arrival order by a scheduler thread whenever a stream slot is
// free and the device-memory budget still covers them; everything admitted
// together runs as one cch_hull_batched call on that slot's stream.  While a
// batch runs on one slot, requests arriving meanwhile form the next batch on
// another, so their copies and kernels overlap on the device (continuous
// batching).  A batch moves through three stages:
//   1. upload (one copy per request, straight from its pinned buffer),
//      cch_hull_batched, a scan and gather that packs the hulls of
//      all sets into one array, and the download of the hull sizes;
//   2. once the sizes are on the host, the download of the packed hulls;
//   3. the results are handed to their requests (host memory, kept until
//      cch_serve_release) and the batch's budget share is returned.
// Every result is that of cch_hull on the request alone: the batched path
// runs the same kernels per set.
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <thread>
#include <vector>

#include "cch.h"
#include "cch_internal.cuh"

namespace cch {
namespace {

using Clock = std::chrono::steady_clock;

// Exclusive prefix of the hull sizes of a batch (negative sizes are error
// codes and count as 0) and their total; one CTA.
__global__ void k_hull_scan(const int32_t* counts, int32_t nsets, int64_t* hoff, int64_t* total) {
  __shared__ int64_t wsum[kWarps];
  __shared__ int64_t carry;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (threadIdx.x == 0) carry = 0;
  __syncthreads();
  for (int base = 0; base < nsets; base += kThreads) {
    const int s = base + threadIdx.x;
    const int64_t c = s < nsets ? (int64_t)max(counts[s], 0) : 0;
    int64_t x = c;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int64_t y = __shfl_up_sync(0xFFFFFFFFu, x, o);
      if (lane >= o) x += y;
    }
    if (lane == 31) wsum[warp] = x;
    __syncthreads();
    int64_t pre = carry;
    for (int q = 0; q < warp; q++) pre += wsum[q];
    if (s < nsets) hoff[s] = pre + x - c;
    __syncthreads();
    if (threadIdx.x == kThreads - 1) carry = pre + x;
    __syncthreads();
  }
  if (threadIdx.x == 0) *total = carry;
}

// Pack the hulls: set s's counts[s] indices from out_idx + offs[s] to
// dst + hoff[s].
__global__ void k_hull_pack(const int32_t* out_idx, const int64_t* offs, const int32_t* counts,
                            const int64_t* hoff, int32_t nsets, int32_t* dst) {
  for (int s = blockIdx.x; s < nsets; s += gridDim.x) {
    const int32_t c = counts[s];
    for (int i = threadIdx.x; i < c; i += blockDim.x) dst[hoff[s] + i] = out_idx[offs[s] + i];
  }
}

// Buffers by power-of-two size class, reused across requests and servers:
// pinned host memory (pinning costs far more than copying into it) for
// requests submitted from the host, device memory for requests submitted
// from the device (their resident copies).  Freed by cch_release_workspace.
class BufPool {
 public:
  explicit BufPool(bool device) : device_(device) {}
  void* get(size_t bytes, size_t& cls) {
    cls = size_t(1) << 16;
    while (cls < bytes) cls <<= 1;
    {
      std::lock_guard<std::mutex> lk(mu_);
      auto& v = free_[cls];
      if (!v.empty()) { void* p = v.back(); v.pop_back(); return p; }
    }
    void* p = nullptr;
    const cudaError_t e = device_ ? cudaMalloc(&p, cls) : cudaMallocHost(&p, cls);
    if (e != cudaSuccess) { cudaGetLastError(); return nullptr; }
    return p;
  }
  void put(void* p, size_t cls) {
    if (!p) return;
    std::lock_guard<std::mutex> lk(mu_);
    free_[cls].push_back(p);
  }
  void release() {
    std::lock_guard<std::mutex> lk(mu_);
    for (auto& kv : free_)
      for (void* p : kv.second) {
        if (device_) cudaFree(p);
        else cudaFreeHost(p);
      }
    free_.clear();
  }
 private:
  bool device_;
  std::mutex mu_;
  std::map<size_t, std::vector<void*>> free_;
};

// memcpy, split over a few threads when large.
void copy_in(void* dst, const void* src, size_t bytes) {
  constexpr size_t kSlice = size_t(8) << 20;
  const int parts = (int)std::min<size_t>(8, bytes / kSlice);
  if (parts <= 1) { memcpy(dst, src, bytes); return; }
  const size_t step = (bytes + parts - 1) / parts;
  std::vector<std::thread> th;
  for (int k = 1; k < parts; k++) {
    const size_t a = k * step, b = std::min(bytes, a + step);
    th.emplace_back([=] { memcpy((char*)dst + a, (const char*)src + a, b - a); });
  }
  memcpy(dst, src, std::min(bytes, step));
  for (auto& t : th) t.join();
}

BufPool g_pinned(false);   // host copies of host-submitted requests
BufPool g_devbuf(true);    // resident copies of device-submitted requests

struct Request {
  uint64_t ticket = 0;
  int64_t n = 0;
  void* pts = nullptr;               // copy of the input until its batch has read it: pinned
  size_t pts_cls = 0;                // host memory, or device memory when `dev`
  bool dev = false;
  Clock::time_point t_submit;
  int32_t status = CCH_OK;
  int32_t count = 0;
  std::vector<int32_t> idx;          // the hull (host)
  double latency_ms = 0.0;
};

// Device or pinned host buffer that only grows.
struct Buf {
  void* p = nullptr;
  size_t cap = 0;
  bool host = false;
  bool ensure(size_t bytes) {
    if (bytes <= cap) return true;
    release();
    const size_t want = std::max(bytes, cap + cap / 2);
    const cudaError_t e = host ? cudaMallocHost(&p, want) : cudaMalloc(&p, want);
    if (e != cudaSuccess) { cudaGetLastError(); p = nullptr; cap = 0; return false; }
    cap = want;
    return true;
  }
  void release() {
    if (p) { if (host) cudaFreeHost(p); else cudaFree(p); }
    p = nullptr;
    cap = 0;
  }
};

struct Slot {
  cudaStream_t st = nullptr;
  cudaEvent_t ev = nullptr;
  int stage = 0;                     // 0 idle, 1 kernels + sizes, 2 packed hulls
  std::vector<Request*> reqs;
  std::vector<int64_t> offs;
  size_t need = 0;                   // budget share of the batch
  Buf d_pts, d_out, d_counts, d_offs, d_hoff, d_hull;
  Buf h_offs{nullptr, 0, true}, h_counts{nullptr, 0, true},
      h_total{nullptr, 0, true}, h_hull{nullptr, 0, true};
};

}  // namespace

void serve_release_pinned() {
  g_pinned.release();
  g_devbuf.release();
}

}  // namespace cch

using namespace cch;

struct cch_server {
  cch_serve_config cfg{};
  int device = 0;
  std::mutex mu;
  std::condition_variable cv;
  bool stop = false;
  std::thread worker;
  std::deque<Request*> pending;
  std::deque<Request*> done;                 // finished, not yet polled
  std::map<uint64_t, Request*> finished;     // polled or not, until released
  std::vector<Slot> slots;
  size_t reserved = 0;                       // budget held by batches in flight
  uint64_t next_ticket = 1;
  bool started = false;
  Clock::time_point t_first, t_last;
  std::vector<double> latencies;
  int64_t nfinished = 0;
  BufPool& pinned = g_pinned;
  std::mutex submit_mu;                      // guards submit_ev
  cudaEvent_t submit_ev = nullptr;           // completion of a device submit's copy
  BufPool& devbuf = g_devbuf;
  void put_input(Request* r) {
    (r->dev ? devbuf : pinned).put(r->pts, r->pts_cls);
    r->pts = nullptr;
  }

  size_t point_bytes() const { return cfg.dtype == CCH_F64 ? 16 : 8; }
  // device bytes a batch of `npts` points in `nsets` sets holds while it runs
  size_t need_of(int64_t npts, int64_t nsets) const {
    return (size_t)npts * (point_bytes() + 4 + 4) + (size_t)nsets * 32 + 4096 +
           cch_workspace_bytes(npts, cfg.dtype);
  }

  void launch(Slot& sl);
  void advance(Slot& sl);
  void finish(Slot& sl, int status);
  void loop();
};

void cch_server::finish(Slot& sl, int status) {
  if (status != CCH_OK) cudaStreamSynchronize(sl.st);   // no copy may still read a pinned input
  for (Request* r : sl.reqs) put_input(r);
  const Clock::time_point now = Clock::now();
  const int32_t* counts = static_cast<const int32_t*>(sl.h_counts.p);
  const int32_t* hull = static_cast<const int32_t*>(sl.h_hull.p);
  int64_t h0 = 0;
  std::lock_guard<std::mutex> lk(mu);
  for (size_t i = 0; i < sl.reqs.size(); i++) {
    Request* r = sl.reqs[i];
    if (status != CCH_OK) {
      r->status = status;
      r->count = 0;
    } else if (counts[i] < 0) {
      r->status = counts[i];
      r->count = 0;
    } else {
      r->status = CCH_OK;
      r->count = counts[i];
      r->idx.assign(hull + h0, hull + h0 + counts[i]);
      h0 += counts[i];
    }
    r->latency_ms = std::chrono::duration<double, std::milli>(now - r->t_submit).count();
    latencies.push_back(r->latency_ms);
    finished[r->ticket] = r;
    done.push_back(r);
    nfinished++;
  }
  t_last = now;
  reserved -= sl.need;
  sl.need = 0;
  sl.reqs.clear();
  sl.stage = 0;
}

// Stage 1 of a batch (scheduler thread, no lock held).
void cch_server::launch(Slot& sl) {
  const int32_t nsets = (int32_t)sl.reqs.size();
  const int64_t N = sl.offs[nsets];
  const size_t pb = point_bytes();
  const bool ok = sl.d_pts.ensure(std::max<size_t>(N * pb, 16)) && sl.d_out.ensure(std::max<size_t>(N * 4, 4)) &&
                  sl.d_counts.ensure(4 * (size_t)nsets) && sl.d_offs.ensure(8 * (size_t)(nsets + 1)) &&
                  sl.d_hoff.ensure(8 * (size_t)nsets + 8) && sl.d_hull.ensure(std::max<size_t>(N * 4, 4)) &&
                  sl.h_offs.ensure(8 * (size_t)(nsets + 1)) && sl.h_counts.ensure(4 * (size_t)nsets) &&
                  sl.h_total.ensure(8);
  if (!ok) { finish(sl, CCH_ERR_NOMEM); return; }
  memcpy(sl.h_offs.p, sl.offs.data(), 8 * (size_t)(nsets + 1));
  int st = CCH_OK;
  for (int32_t i = 0; i < nsets && st == CCH_OK; i++) {
    const Request* r = sl.reqs[i];
    if (r->n && cudaMemcpyAsync(static_cast<unsigned char*>(sl.d_pts.p) + sl.offs[i] * pb, r->pts, (size_t)r->n * pb,
                                r->dev ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, sl.st) != cudaSuccess)
      st = CCH_ERR_CUDA;
  }
  if (st == CCH_OK &&
      cudaMemcpyAsync(sl.d_offs.p, sl.h_offs.p, 8 * (size_t)(nsets + 1), cudaMemcpyHostToDevice, sl.st) != cudaSuccess)
    st = CCH_ERR_CUDA;
  if (st == CCH_OK)
    st = cch_hull_batched(sl.d_pts.p, sl.offs.data(), nsets, cfg.dtype, static_cast<int32_t*>(sl.d_out.p),
                          static_cast<int32_t*>(sl.d_counts.p), sl.st);
  if (st == CCH_OK) {
    k_hull_scan<<<1, kThreads, 0, sl.st>>>(static_cast<const int32_t*>(sl.d_counts.p), nsets,
                                           static_cast<int64_t*>(sl.d_hoff.p),
                                           static_cast<int64_t*>(sl.d_hoff.p) + nsets);
    const int grid = std::min<int>(nsets, 1024);
    k_hull_pack<<<grid, kThreads, 0, sl.st>>>(static_cast<const int32_t*>(sl.d_out.p),
                                              static_cast<const int64_t*>(sl.d_offs.p),
                                              static_cast<const int32_t*>(sl.d_counts.p),
                                              static_cast<const int64_t*>(sl.d_hoff.p), nsets,
                                              static_cast<int32_t*>(sl.d_hull.p));
    if (cudaMemcpyAsync(sl.h_counts.p, sl.d_counts.p, 4 * (size_t)nsets, cudaMemcpyDeviceToHost, sl.st) != cudaSuccess ||
        cudaMemcpyAsync(sl.h_total.p, static_cast<int64_t*>(sl.d_hoff.p) + nsets, 8, cudaMemcpyDeviceToHost, sl.st) !=
            cudaSuccess ||
        cudaEventRecord(sl.ev, sl.st) != cudaSuccess)
      st = CCH_ERR_CUDA;
  }
  if (st != CCH_OK) { cudaStreamSynchronize(sl.st); cudaGetLastError(); finish(sl, st); return; }
  sl.stage = 1;
}

// Next stage of a batch whose event has completed (scheduler thread).
void cch_server::advance(Slot& sl) {
  if (sl.stage == 1) {
    for (Request* r : sl.reqs) put_input(r);
    const int64_t total = *static_cast<const int64_t*>(sl.h_total.p);
    if (total > 0) {
      if (!sl.h_hull.ensure(4 * (size_t)total)) { finish(sl, CCH_ERR_NOMEM); return; }
      if (cudaMemcpyAsync(sl.h_hull.p, sl.d_hull.p, 4 * (size_t)total, cudaMemcpyDeviceToHost, sl.st) != cudaSuccess ||
          cudaEventRecord(sl.ev, sl.st) != cudaSuccess) {
        finish(sl, CCH_ERR_CUDA);
        return;
      }
      sl.stage = 2;
      return;
    }
  }
  finish(sl, CCH_OK);
}

void cch_server::loop() {
  cudaSetDevice(device);
  std::unique_lock<std::mutex> lk(mu);
  for (;;) {
    bool moved = false;
    // finished stages
    for (auto& sl : slots) {
      if (sl.stage == 0) continue;
      const cudaError_t q = cudaEventQuery(sl.ev);
      if (q == cudaErrorNotReady) continue;
      lk.unlock();
      if (q == cudaSuccess) advance(sl);
      else { cudaGetLastError(); finish(sl, CCH_ERR_CUDA); }
      lk.lock();
      moved = true;
    }
    // new batches: arrival order, while a slot is free and the budget holds
    for (auto& sl : slots) {
      if (sl.stage != 0 || pending.empty()) continue;
      int64_t npts = 0;
      size_t k = 0;
      while (k < pending.size() && k < (size_t)cfg.max_batch) {
        const int64_t n2 = npts + pending[k]->n;
        if (n2 > 0x7FFFFFFFll || reserved + need_of(n2, (int64_t)k + 1) > cfg.budget_bytes) break;
        npts = n2;
        k++;
      }
      if (k == 0) break;   // the head waits for budget to come back
      sl.reqs.assign(pending.begin(), pending.begin() + k);
      pending.erase(pending.begin(), pending.begin() + k);
      sl.offs.assign(k + 1, 0);
      for (size_t i = 0; i < k; i++) sl.offs[i + 1] = sl.offs[i] + sl.reqs[i]->n;
      sl.need = need_of(npts, (int64_t)k);
      reserved += sl.need;
      sl.stage = 1;                     // taken (launch may finish it at once)
      lk.unlock();
      launch(sl);
      lk.lock();
      moved = true;
    }
    bool busy = false;
    for (auto& sl : slots) busy |= sl.stage != 0;
    if (stop && !busy && pending.empty()) break;
    if (moved) continue;
    if (busy) {
      lk.unlock();
      std::this_thread::sleep_for(std::chrono::microseconds(20));
      lk.lock();
    } else {
      cv.wait(lk, [&] { return stop || !pending.empty(); });
    }
  }
}

extern "C" int cch_serve_create(const cch_serve_config* cfg, cch_server** out) {
  if (!cfg || !out) return CCH_ERR_INVALID;
  if (cfg->dtype != CCH_I32 && cfg->dtype != CCH_F64) return CCH_ERR_DTYPE;
  if (cfg->num_streams < 0 || cfg->max_pending < 0 || cfg->max_batch < 0) return CCH_ERR_INVALID;
  cch_server* s = new cch_server();
  s->cfg = *cfg;
  if (!s->cfg.budget_bytes) s->cfg.budget_bytes = size_t(64) << 30;
  if (!s->cfg.num_streams) s->cfg.num_streams = 4;
  if (!s->cfg.max_pending) s->cfg.max_pending = 65536;
  if (!s->cfg.max_batch) s->cfg.max_batch = 4096;
  if (cudaGetDevice(&s->device) != cudaSuccess) { delete s; return CCH_ERR_CUDA; }
  s->slots.resize(s->cfg.num_streams);
  if (cudaEventCreateWithFlags(&s->submit_ev, cudaEventDisableTiming) != cudaSuccess) { delete s; return CCH_ERR_CUDA; }
  for (auto& sl : s->slots) {
    if (cudaStreamCreateWithFlags(&sl.st, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&sl.ev, cudaEventDisableTiming) != cudaSuccess) {
      for (auto& q : s->slots) {
        if (q.st) cudaStreamDestroy(q.st);
        if (q.ev) cudaEventDestroy(q.ev);
      }
      cudaEventDestroy(s->submit_ev);
      delete s;
      return CCH_ERR_CUDA;
    }
  }
  s->worker = std::thread([s] { s->loop(); });
  *out = s;
  return CCH_OK;
}

namespace {
int serve_check(cch_server* srv, const void* points, int64_t n, uint64_t* ticket) {
  if (!srv || !ticket || n < 0 || (n > 0 && !points)) return CCH_ERR_INVALID;
  if (n > kMaxSetPoints) return CCH_ERR_RANGE;
  if (srv->need_of(n, 1) > srv->cfg.budget_bytes) return CCH_ERR_RANGE;
  return CCH_OK;
}

// Queue a request whose input copy is complete.
int serve_enqueue(cch_server* srv, Request* r, uint64_t* ticket) {
  {
    std::lock_guard<std::mutex> lk(srv->mu);
    if (srv->stop || srv->pending.size() >= (size_t)srv->cfg.max_pending) {
      srv->put_input(r);
      const int code = srv->stop ? CCH_ERR_INVALID : CCH_ERR_BUSY;
      delete r;
      return code;
    }
    r->ticket = srv->next_ticket++;
    r->t_submit = Clock::now();
    if (!srv->started) { srv->started = true; srv->t_first = r->t_submit; }
    srv->pending.push_back(r);
    *ticket = r->ticket;
  }
  srv->cv.notify_one();
  return CCH_OK;
}
}  // namespace

extern "C" int cch_serve_submit(cch_server* srv, const void* points, int64_t n, uint64_t* ticket) {
  int st = serve_check(srv, points, n, ticket);
  if (st != CCH_OK) return st;
  Request* r = new Request();
  r->n = n;
  if (n) {
    const size_t bytes = (size_t)n * srv->point_bytes();
    r->pts = srv->pinned.get(bytes, r->pts_cls);
    if (!r->pts) { delete r; return CCH_ERR_NOMEM; }
    copy_in(r->pts, points, bytes);
  }
  return serve_enqueue(srv, r, ticket);
}

extern "C" int cch_serve_submit_device(cch_server* srv, const void* points, int64_t n, void* stream,
                                       uint64_t* ticket) {
  int st = serve_check(srv, points, n, ticket);
  if (st != CCH_OK) return st;
  if ((uintptr_t)points % srv->point_bytes()) return CCH_ERR_INVALID;
  Request* r = new Request();
  r->n = n;
  r->dev = true;
  if (n) {
    const size_t bytes = (size_t)n * srv->point_bytes();
    r->pts = srv->devbuf.get(bytes, r->pts_cls);
    if (!r->pts) { delete r; return CCH_ERR_NOMEM; }
    // ordered after the caller's work on `stream`; complete before return,
    // so the caller may reuse or free its buffer at once
    cudaStream_t cs = (cudaStream_t)stream;
    std::lock_guard<std::mutex> lk(srv->submit_mu);
    if (cudaMemcpyAsync(r->pts, points, bytes, cudaMemcpyDeviceToDevice, cs) != cudaSuccess ||
        cudaEventRecord(srv->submit_ev, cs) != cudaSuccess || cudaEventSynchronize(srv->submit_ev) != cudaSuccess) {
      cudaGetLastError();
      srv->put_input(r);
      delete r;
      return CCH_ERR_CUDA;
    }
  }
  return serve_enqueue(srv, r, ticket);
}

extern "C" int cch_serve_poll(cch_server* srv, cch_done* done, int max, int* n_done) {
  if (!srv || !n_done || max < 0 || (max > 0 && !done)) return CCH_ERR_INVALID;
  std::lock_guard<std::mutex> lk(srv->mu);
  int k = 0;
  while (k < max && !srv->done.empty()) {
    Request* r = srv->done.front();
    srv->done.pop_front();
    done[k].ticket = r->ticket;
    done[k].status = r->status;
    done[k].count = r->count;
    done[k].idx = r->idx.empty() ? nullptr : r->idx.data();
    done[k].latency_ms = r->latency_ms;
    k++;
  }
  *n_done = k;
  return CCH_OK;
}

extern "C" int cch_serve_release(cch_server* srv, uint64_t ticket) {
  if (!srv) return CCH_ERR_INVALID;
  std::lock_guard<std::mutex> lk(srv->mu);
  auto it = srv->finished.find(ticket);
  if (it == srv->finished.end()) return CCH_ERR_NOTFOUND;
  Request* r = it->second;
  // a result not yet polled stays in the done queue: drop it there too
  auto d = std::find(srv->done.begin(), srv->done.end(), r);
  if (d != srv->done.end()) srv->done.erase(d);
  srv->finished.erase(it);
  delete r;
  return CCH_OK;
}

extern "C" int cch_serve_stats(cch_server* srv, double* p50_ms, double* p99_ms, double* hulls_per_s,
                               int64_t* finished) {
  if (!srv) return CCH_ERR_INVALID;
  std::lock_guard<std::mutex> lk(srv->mu);
  std::vector<double> v = srv->latencies;
  auto pct = [&](double q) {
    if (v.empty()) return 0.0;
    const size_t k = std::min(v.size() - 1, (size_t)(q * (double)(v.size() - 1) + 0.5));
    std::nth_element(v.begin(), v.begin() + k, v.end());
    return v[k];
  };
  if (p50_ms) *p50_ms = pct(0.50);
  if (p99_ms) *p99_ms = pct(0.99);
  if (hulls_per_s) {
    const double sec = srv->nfinished ? std::chrono::duration<double>(srv->t_last - srv->t_first).count() : 0.0;
    *hulls_per_s = sec > 0 ? (double)srv->nfinished / sec : 0.0;
  }
  if (finished) *finished = srv->nfinished;
  return CCH_OK;
}

extern "C" int cch_serve_destroy(cch_server* srv) {
  if (!srv) return CCH_ERR_INVALID;
  {
    std::lock_guard<std::mutex> lk(srv->mu);
    srv->stop = true;
  }
  srv->cv.notify_one();
  if (srv->worker.joinable()) srv->worker.join();
  for (auto& sl : srv->slots) {
    cudaStreamSynchronize(sl.st);
    for (Buf* b : {&sl.d_pts, &sl.d_out, &sl.d_counts, &sl.d_offs, &sl.d_hoff, &sl.d_hull, &sl.h_offs,
                   &sl.h_counts, &sl.h_total, &sl.h_hull})
      b->release();
    cudaEventDestroy(sl.ev);
    cudaStreamDestroy(sl.st);
  }
  cudaEventDestroy(srv->submit_ev);
  for (auto& kv : srv->finished) delete kv.second;
  for (Request* r : srv->pending) { srv->put_input(r); delete r; }
  delete srv;
  return CCH_OK;
}

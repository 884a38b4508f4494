// tune.cu -- run-time choices per size bucket (struct Tune), their table and
// JSON cache, and the tuner that measures candidates on the caller's batch.
//
// A call's choices come from the table entry of its key: the GPU (name and
// SM count), the dtype, whether it is a batch of several sets, and the size
// bucket floor(log2(mean points per set)).  Without an entry the defaults
// apply.  No choice changes a result: each only moves work between
// equivalent paths (the shared-memory or the multi-block sort, the a1 chunk
// length, the a2 grid) or resizes the sample behind an exact prefilter.
#include <algorithm>
#include <array>
#include <climits>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <tuple>
#include <vector>

#include "cch.h"
#include "cch_internal.cuh"

namespace cch {
namespace {

struct Key {
  std::string gpu;
  int sms, dtype, batched, bucket;
  bool operator<(const Key& o) const {
    return std::tie(gpu, sms, dtype, batched, bucket) < std::tie(o.gpu, o.sms, o.dtype, o.batched, o.bucket);
  }
};

std::mutex g_tmu;
std::map<Key, Tune> g_table;
std::map<int, std::pair<std::string, int>> g_ident;   // device -> (name, SMs)

bool device_identity(std::string& name, int& sms) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) { cudaGetLastError(); return false; }
  auto it = g_ident.find(dev);
  if (it == g_ident.end()) {
    cudaDeviceProp p;
    if (cudaGetDeviceProperties(&p, dev) != cudaSuccess) { cudaGetLastError(); return false; }
    it = g_ident.emplace(dev, std::make_pair(std::string(p.name), p.multiProcessorCount)).first;
  }
  name = it->second.first;
  sms = it->second.second;
  return true;
}

Tune default_tune(bool batched) {
  Tune t = kTuneDefault;
  if (batched) t.a1_len_min = 16384;
  return t;
}

bool valid(const Tune& t) {
  return t.small_max >= 1 && t.small_max <= kSmallMax && t.stair_div >= 1 && t.stair_min >= 1 &&
         t.stair_min <= t.stair_max && t.stair_max <= (1 << 24) && t.a1_len_min >= 4096 &&
         t.a1_len_min <= (1 << 26) && t.a1_len_min % 1024 == 0 && (t.cls_per_sm == 1 || t.cls_per_sm == 2);
}

Tune from_c(const cch_tune_params& p) {
  return Tune{p.small_max, p.stair_div, p.stair_min, p.stair_max, p.a1_len_min, p.cls_per_sm};
}
void to_c(const Tune& t, cch_tune_params& p) {
  p.small_max = t.small_max; p.stair_div = t.stair_div; p.stair_min = t.stair_min;
  p.stair_max = t.stair_max; p.a1_len_min = t.a1_len_min; p.cls_per_sm = t.cls_per_sm;
}

// --------------------------------------------------------- JSON cache
// {"cch_tune": 1, "entries": [{"gpu": "...", "sms": 152, "dtype": 2,
//  "batched": 1, "bucket": 16, "small_max": ..., ...}, ...]}

std::string json_str(const std::string& s) {
  std::string o = "\"";
  for (char c : s) {
    if (c == '"' || c == '\\') o += '\\';
    o += c;
  }
  return o + "\"";
}

// Minimal parser for the cache's own format: objects of string and integer
// members inside the "entries" array.  Returns false on malformed input.
struct Parser {
  const std::string& s;
  size_t i = 0;
  void ws() { while (i < s.size() && (s[i] == ' ' || s[i] == '\n' || s[i] == '\r' || s[i] == '\t')) i++; }
  bool lit(char c) { ws(); if (i < s.size() && s[i] == c) { i++; return true; } return false; }
  bool str(std::string& out) {
    ws();
    if (i >= s.size() || s[i] != '"') return false;
    i++;
    out.clear();
    while (i < s.size() && s[i] != '"') {
      if (s[i] == '\\') { if (++i >= s.size()) return false; }
      out += s[i++];
    }
    if (i >= s.size()) return false;
    i++;
    return true;
  }
  bool integer(long long& v) {
    ws();
    size_t j = i;
    if (j < s.size() && s[j] == '-') j++;
    if (j >= s.size() || s[j] < '0' || s[j] > '9') return false;
    while (j < s.size() && s[j] >= '0' && s[j] <= '9') j++;
    if (j - i > 18) return false;            // beyond any value the cache holds
    v = std::stoll(s.substr(i, j - i));
    i = j;
    return true;
  }
  // one entry object: member name -> value
  bool entry(std::string& gpu, std::map<std::string, long long>& ints) {
    if (!lit('{')) return false;
    if (lit('}')) return true;
    for (;;) {
      std::string k;
      if (!str(k) || !lit(':')) return false;
      ws();
      if (i < s.size() && s[i] == '"') {
        std::string v;
        if (!str(v)) return false;
        if (k == "gpu") gpu = v;
      } else {
        long long v;
        if (!integer(v)) return false;
        ints[k] = v;
      }
      if (lit(',')) continue;
      return lit('}');
    }
  }
};

}  // namespace

int tune_bucket(int64_t npts, int32_t nsets) {
  const int64_t mean = nsets > 0 ? npts / nsets : npts;
  int b = 0;
  while ((int64_t(1) << (b + 1)) <= mean && b < 62) b++;
  return b;
}

Tune tune_for(int dtype, int64_t npts, int32_t nsets) {
  std::lock_guard<std::mutex> lk(g_tmu);
  const bool batched = nsets > 1;
  std::string gpu;
  int sms = 0;
  if (g_table.empty() || !device_identity(gpu, sms)) return default_tune(batched);
  auto it = g_table.find(Key{gpu, sms, dtype, batched ? 1 : 0, tune_bucket(npts, nsets)});
  return it == g_table.end() ? default_tune(batched) : it->second;
}

}  // namespace cch

using namespace cch;

extern "C" {

int cch_tune_bucket(int64_t npts, int32_t nsets) { return tune_bucket(npts, nsets); }

static int tune_key(const char* gpu, int32_t sms, int32_t dtype, int32_t batched, int32_t bucket, Key& k) {
  if (dtype != CCH_I32 && dtype != CCH_F64) return CCH_ERR_DTYPE;
  if ((batched != 0 && batched != 1) || bucket < 0 || bucket > 62) return CCH_ERR_INVALID;
  if (gpu) {
    if (sms <= 0) return CCH_ERR_INVALID;
    k = Key{gpu, sms, dtype, batched, bucket};
    return CCH_OK;
  }
  std::string name;
  int n = 0;
  if (!device_identity(name, n)) return CCH_ERR_CUDA;
  k = Key{name, n, dtype, batched, bucket};
  return CCH_OK;
}

int cch_tune_set(const char* gpu, int32_t sms, int32_t dtype, int32_t batched, int32_t bucket,
                 const cch_tune_params* p) {
  if (!p) return CCH_ERR_INVALID;
  const Tune t = from_c(*p);
  if (!valid(t)) return CCH_ERR_INVALID;
  std::lock_guard<std::mutex> lk(g_tmu);
  Key k;
  const int st = tune_key(gpu, sms, dtype, batched, bucket, k);
  if (st != CCH_OK) return st;
  g_table[k] = t;
  return CCH_OK;
}

int cch_tune_get(const char* gpu, int32_t sms, int32_t dtype, int32_t batched, int32_t bucket,
                 cch_tune_params* p) {
  if (!p) return CCH_ERR_INVALID;
  std::lock_guard<std::mutex> lk(g_tmu);
  Key k;
  const int st = tune_key(gpu, sms, dtype, batched, bucket, k);
  if (st != CCH_OK) return st;
  auto it = g_table.find(k);
  to_c(it == g_table.end() ? default_tune(batched != 0) : it->second, *p);
  return it == g_table.end() ? CCH_ERR_NOTFOUND : CCH_OK;
}

int cch_tune_clear(void) {
  std::lock_guard<std::mutex> lk(g_tmu);
  g_table.clear();
  return CCH_OK;
}

int cch_tune_save(const char* path) {
  if (!path) return CCH_ERR_INVALID;
  std::string o = "{\"cch_tune\": 1, \"entries\": [";
  {
    std::lock_guard<std::mutex> lk(g_tmu);
    bool first = true;
    for (const auto& kv : g_table) {
      const Key& k = kv.first;
      const Tune& t = kv.second;
      char buf[1024];
      snprintf(buf, sizeof buf,
               "%s\n  {\"gpu\": %s, \"sms\": %d, \"dtype\": %d, \"batched\": %d, \"bucket\": %d, "
               "\"small_max\": %d, \"stair_div\": %d, \"stair_min\": %d, \"stair_max\": %d, "
               "\"a1_len_min\": %d, \"cls_per_sm\": %d}",
               first ? "" : ",", json_str(k.gpu).c_str(), k.sms, k.dtype, k.batched, k.bucket, t.small_max,
               t.stair_div, t.stair_min, t.stair_max, t.a1_len_min, t.cls_per_sm);
      o += buf;
      first = false;
    }
  }
  o += "\n]}\n";
  FILE* f = fopen(path, "w");
  if (!f) return CCH_ERR_INVALID;
  const bool ok = fwrite(o.data(), 1, o.size(), f) == o.size();
  return (fclose(f) == 0 && ok) ? CCH_OK : CCH_ERR_INVALID;
}

int cch_tune_load(const char* path) {
  if (!path) return CCH_ERR_INVALID;
  FILE* f = fopen(path, "r");
  if (!f) return CCH_ERR_NOTFOUND;
  std::string s;
  char buf[4096];
  size_t got;
  while ((got = fread(buf, 1, sizeof buf, f)) > 0) s.append(buf, got);
  fclose(f);
  Parser ps{s};
  std::vector<std::pair<Key, Tune>> entries;
  const size_t at = s.find("\"entries\"");
  if (at == std::string::npos) return CCH_ERR_INVALID;
  ps.i = at + 9;
  if (!ps.lit(':') || !ps.lit('[')) return CCH_ERR_INVALID;
  if (!ps.lit(']')) {
    for (;;) {
      std::string gpu;
      std::map<std::string, long long> v;
      if (!ps.entry(gpu, v)) return CCH_ERR_INVALID;
      const char* need[] = {"sms", "dtype", "batched", "bucket", "small_max", "stair_div",
                            "stair_min", "stair_max", "a1_len_min", "cls_per_sm"};
      for (const char* n : need)
        if (!v.count(n) || v[n] < INT32_MIN || v[n] > INT32_MAX) return CCH_ERR_INVALID;
      const Key k{gpu, (int)v["sms"], (int)v["dtype"], (int)v["batched"], (int)v["bucket"]};
      const Tune t{(int32_t)v["small_max"], (int32_t)v["stair_div"], (int32_t)v["stair_min"],
                   (int32_t)v["stair_max"], (int32_t)v["a1_len_min"], (int32_t)v["cls_per_sm"]};
      if (gpu.empty() || k.sms <= 0 || (k.dtype != CCH_I32 && k.dtype != CCH_F64) ||
          (k.batched != 0 && k.batched != 1) || k.bucket < 0 || k.bucket > 62 || !valid(t))
        return CCH_ERR_INVALID;
      entries.emplace_back(k, t);
      if (ps.lit(',')) continue;
      if (!ps.lit(']')) return CCH_ERR_INVALID;
      break;
    }
  }
  std::lock_guard<std::mutex> lk(g_tmu);
  for (auto& e : entries) g_table[e.first] = e.second;   // the whole file parsed: merge it
  return CCH_OK;
}

// Coordinate descent over the candidate values of each choice, timed on the
// caller's own batch (CUDA events on its stream, one untimed call per
// candidate first); the fastest choice of every knob is kept in turn.  The
// result is stored in the table under this call's key and returned.
int cch_autotune_batched(const void* points, const int64_t* offsets, int32_t nsets, int32_t dtype,
                         int32_t* out_idx, int32_t* out_counts, void* stream, int32_t reps,
                         cch_tune_params* best) {
  if (nsets <= 0 || !offsets || reps <= 0) return CCH_ERR_INVALID;
  const int64_t N = offsets[nsets];
  cudaStream_t st = (cudaStream_t)stream;
  const int bucket = tune_bucket(N, nsets);
  const int batched = nsets > 1 ? 1 : 0;
  cch_tune_params cur;
  int rc = cch_tune_get(nullptr, 0, dtype, batched, bucket, &cur);
  if (rc != CCH_OK && rc != CCH_ERR_NOTFOUND) return rc;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) return CCH_ERR_CUDA;
  auto measure = [&](const cch_tune_params& p, float& ms) -> int {
    int r = cch_tune_set(nullptr, 0, dtype, batched, bucket, &p);
    if (r != CCH_OK) return r;
    r = cch_hull_batched(points, offsets, nsets, dtype, out_idx, out_counts, stream);
    if (r != CCH_OK) return r;
    cudaEventRecord(e0, st);
    for (int k = 0; k < reps && r == CCH_OK; k++)
      r = cch_hull_batched(points, offsets, nsets, dtype, out_idx, out_counts, stream);
    cudaEventRecord(e1, st);
    if (r != CCH_OK) return r;
    if (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess)
      return CCH_ERR_CUDA;
    return CCH_OK;
  };
  const std::vector<int32_t> small_max = {16384, 8192, 4096};
  const std::vector<std::array<int32_t, 3>> stairs = {
      {16, 8192, 1 << 20}, {32, 4096, 1 << 19}, {8, 16384, 1 << 21}, {64, 2048, 1 << 18}};
  const std::vector<int32_t> a1_len = {16384, 65536, 262144, 4096};
  const std::vector<int32_t> cls = {2, 1};
  float best_ms = 0.f;
  rc = measure(cur, best_ms);
  for (int knob = 0; knob < 4 && rc == CCH_OK; knob++) {
    const size_t nv = knob == 0 ? small_max.size() : knob == 1 ? stairs.size() : knob == 2 ? a1_len.size()
                                                                                            : cls.size();
    for (size_t v = 0; v < nv && rc == CCH_OK; v++) {
      cch_tune_params c = cur;
      if (knob == 0) c.small_max = small_max[v];
      else if (knob == 1) { c.stair_div = stairs[v][0]; c.stair_min = stairs[v][1]; c.stair_max = stairs[v][2]; }
      else if (knob == 2) c.a1_len_min = a1_len[v];
      else c.cls_per_sm = cls[v];
      if (memcmp(&c, &cur, sizeof c) == 0) continue;
      float ms = 0.f;
      rc = measure(c, ms);
      if (rc == CCH_OK && ms < best_ms) { best_ms = ms; cur = c; }
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (rc != CCH_OK) return rc;
  rc = cch_tune_set(nullptr, 0, dtype, batched, bucket, &cur);
  if (best) *best = cur;
  return rc;
}

}  // extern "C"

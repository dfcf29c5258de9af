// Autotuner of launch geometries (tune.h) and its C ABI (dfm_autotune,
// dfm_autotune_report).
#include <algorithm>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <tuple>

#include "dfm_internal.cuh"
#include "tune.h"

namespace dfm {
namespace tune {
namespace {

struct Entry {
  Geometry best;
  std::vector<Geometry> tried;
};

auto key_tuple(const Key& k) { return std::make_tuple(k.kind, k.nb, k.prec, k.w, k.rgl, k.trans, k.nrows, k.device); }

struct KeyLess {
  bool operator()(const Key& a, const Key& b) const { return key_tuple(a) < key_tuple(b); }
};

std::mutex g_mu;
std::map<Key, Entry, KeyLess> g_cache;
int g_mode = 1;  // 0: fixed default geometries, 1: tune on first use

constexpr int kTimedLaunches = 2;

}  // namespace

int choose(const Key& key, cudaStream_t st, const std::vector<Geometry>& cands, const Geometry& fallback,
           const std::function<int(int, int)>& launch, Geometry* out) {
  {
    std::lock_guard<std::mutex> lk(g_mu);
    if (g_mode == 0 || cands.size() < 2) {
      *out = fallback;
      return DFM_OK;
    }
    auto it = g_cache.find(key);
    if (it != g_cache.end()) {
      *out = it->second.best;
      return DFM_OK;
    }
  }
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  DFM_CUDA_CHECK(cudaStreamIsCapturing(st, &cap));
  if (cap != cudaStreamCaptureStatusNone) {  // no timing inside a graph capture
    *out = fallback;
    return DFM_OK;
  }
  cudaEvent_t e0, e1;
  DFM_CUDA_CHECK(cudaEventCreate(&e0));
  cudaError_t ce = cudaEventCreate(&e1);
  if (ce != cudaSuccess) {
    cudaEventDestroy(e0);
    return cuda_error(ce, "autotune: cudaEventCreate");
  }
  Entry ent;
  int rc = DFM_OK;
  for (const Geometry& c : cands) {
    rc = launch(c.rpt, c.stages);  // warm-up (first use of the shared-memory size)
    if (rc) break;
    ce = cudaEventRecord(e0, st);
    for (int i = 0; i < kTimedLaunches && rc == DFM_OK && ce == cudaSuccess; ++i) rc = launch(c.rpt, c.stages);
    if (ce == cudaSuccess) ce = cudaEventRecord(e1, st);
    if (ce == cudaSuccess) ce = cudaEventSynchronize(e1);
    float ms = 0.f;
    if (ce == cudaSuccess) ce = cudaEventElapsedTime(&ms, e0, e1);
    if (rc || ce != cudaSuccess) break;
    ent.tried.push_back(Geometry{c.rpt, c.stages, ms / kTimedLaunches});
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (rc) return rc;
  if (ce != cudaSuccess) return cuda_error(ce, "autotune: timing");
  ent.best = *std::min_element(ent.tried.begin(), ent.tried.end(),
                               [](const Geometry& a, const Geometry& b) { return a.ms < b.ms; });
  // the caller's launch with the chosen geometry follows; its output replaces the candidates'
  {
    std::lock_guard<std::mutex> lk(g_mu);
    g_cache[key] = ent;
  }
  *out = ent.best;
  return DFM_OK;
}

}  // namespace tune
}  // namespace dfm

extern "C" int dfm_autotune(int mode) {
  using namespace dfm::tune;
  if (mode < 0 || mode > 2) return dfm::set_error(DFM_ERR_ARG, "dfm_autotune: mode must be 0, 1 or 2");
  std::lock_guard<std::mutex> lk(g_mu);
  if (mode == 2) {
    g_cache.clear();
    mode = 1;
  }
  g_mode = mode;
  return DFM_OK;
}

extern "C" int64_t dfm_autotune_report(char* buf, int64_t len) {
  using namespace dfm::tune;
  std::string s = "[";
  {
    std::lock_guard<std::mutex> lk(g_mu);
    bool first = true;
    for (const auto& kv : g_cache) {
      const Key& k = kv.first;
      char head[256];
      std::snprintf(head, sizeof head,
                    "%s{\"kernel\": \"%s\", \"nb\": %d, \"precision\": %d, \"rhs_per_group\": %d, \"groups\": %d, "
                    "\"transpose\": %d, \"rows\": %lld, \"device\": %d, \"chosen\": {\"rows_per_tile\": %d, "
                    "\"stages\": %d, \"ms\": %.5f}, \"tried\": [",
                    first ? "" : ", ", k.kind == 0 ? "hop_frag" : "other", k.nb, k.prec, k.w, k.rgl, k.trans,
                    (long long)k.nrows, k.device, kv.second.best.rpt, kv.second.best.stages, kv.second.best.ms);
      s += head;
      for (size_t i = 0; i < kv.second.tried.size(); ++i) {
        const Geometry& g = kv.second.tried[i];
        char t[96];
        std::snprintf(t, sizeof t, "%s[%d, %d, %.5f]", i ? ", " : "", g.rpt, g.stages, g.ms);
        s += t;
      }
      s += "]}";
      first = false;
    }
  }
  s += "]";
  const int64_t need = (int64_t)s.size() + 1;
  if (buf && len > 0) {
    const int64_t n = std::min<int64_t>(len - 1, (int64_t)s.size());
    std::memcpy(buf, s.data(), (size_t)n);
    buf[n] = '\0';
  }
  return need;
}

// Launch counting and optional per-kernel CUDA-event timing.
//
// The benchmark reports the device time of the dominant kernels measured on
// the stream they run on; when timing is enabled every timed launch site
// records an event pair around its kernel.  Events come from a pool that is
// reused after dfm_stats_reset, so steady-state timing allocates nothing.
#include <atomic>
#include <mutex>
#include <vector>

#include "dfm_internal.cuh"

namespace dfm {
namespace {
std::atomic<long long> g_launches{0};
std::atomic<int> g_timing{0};
std::mutex g_mu;
struct Rec {
  int kernel;
  int e0, e1;
};
std::vector<cudaEvent_t> g_pool;
std::vector<Rec> g_recs;
size_t g_next = 0;

int take_event() {
  if (g_next == g_pool.size()) {
    cudaEvent_t e;
    if (cudaEventCreate(&e) != cudaSuccess) return -1;
    g_pool.push_back(e);
  }
  return (int)g_next++;
}
}  // namespace

void count_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }

KernelTimer::KernelTimer(int kernel, cudaStream_t st) : kernel_(kernel), st_(st), e0_(-1) {
  if (!g_timing.load(std::memory_order_relaxed)) return;
  std::lock_guard<std::mutex> lk(g_mu);
  e0_ = take_event();
  if (e0_ >= 0) cudaEventRecord(g_pool[e0_], st_);
}

KernelTimer::~KernelTimer() {
  if (e0_ < 0) return;
  std::lock_guard<std::mutex> lk(g_mu);
  const int e1 = take_event();
  if (e1 < 0) return;
  cudaEventRecord(g_pool[e1], st_);
  g_recs.push_back(Rec{kernel_, e0_, e1});
}

}  // namespace dfm

using namespace dfm;

extern "C" long long dfm_launch_count(void) { return g_launches.load(); }

extern "C" int dfm_stats_enable(int on) {
  g_timing.store(on ? 1 : 0);
  return DFM_OK;
}

extern "C" int dfm_stats_reset(void) {
  std::lock_guard<std::mutex> lk(g_mu);
  g_recs.clear();
  g_next = 0;
  return DFM_OK;
}

extern "C" int dfm_kernel_stats(int kernel, int64_t* launches, double* total_ms) {
  if (!launches || !total_ms) return set_error(DFM_ERR_ARG, "dfm_kernel_stats: NULL argument");
  std::lock_guard<std::mutex> lk(g_mu);
  int64_t n = 0;
  double ms = 0.0;
  for (const Rec& r : g_recs) {
    if (r.kernel != kernel) continue;
    cudaError_t e = cudaEventSynchronize(g_pool[r.e1]);
    if (e != cudaSuccess) return cuda_error(e, "dfm_kernel_stats: cudaEventSynchronize");
    float t = 0.f;
    e = cudaEventElapsedTime(&t, g_pool[r.e0], g_pool[r.e1]);
    if (e != cudaSuccess) return cuda_error(e, "dfm_kernel_stats: cudaEventElapsedTime");
    ms += t;
    ++n;
  }
  *launches = n;
  *total_ms = ms;
  return DFM_OK;
}

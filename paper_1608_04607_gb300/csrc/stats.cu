// Launch counting and optional per-kernel CUDA-event timing.
//
// The benchmark reports the device time of the dominant kernels measured on
// the stream they run on; when timing is enabled a timed launch site records
// an event pair around its kernel, at every launch or every n-th launch of
// that kernel.  Events come from a pool that is reused after dfm_stats_reset,
// so steady-state timing allocates nothing.
#include <atomic>
#include <mutex>
#include <vector>

#include "dfm_internal.cuh"

namespace dfm {
namespace {
std::atomic<long long> g_launches{0};
std::atomic<int> g_timing{0};  // 0: off, n >= 1: every n-th launch of a kernel
std::mutex g_mu;
long long g_count[DFM_KERNEL_COUNT] = {};  // launches per kernel while timing was on
struct Rec {
  int kernel;
  int e0, e1;
  int weight;  // launches the event pair spans (a replayed graph: all its nodes)
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

// launches recorded into a graph under capture are counted when it is replayed
thread_local bool t_capturing = false;

void set_capturing(bool on) { t_capturing = on; }

void count_launch() {
  if (!t_capturing) g_launches.fetch_add(1, std::memory_order_relaxed);
}

void count_launches(long long n) { g_launches.fetch_add(n, std::memory_order_relaxed); }

KernelTimer::KernelTimer(int kernel, cudaStream_t st, int weight)
    : kernel_(kernel), st_(st), e0_(-1), weight_(weight) {
  const int every = g_timing.load(std::memory_order_relaxed);
  if (!every || t_capturing || kernel < 0 || kernel >= DFM_KERNEL_COUNT) return;
  std::lock_guard<std::mutex> lk(g_mu);
  const long long before = g_count[kernel];
  g_count[kernel] += weight;
  // a single launch is timed every n-th time; a replayed graph every time
  if (weight == 1 && before % every != 0) return;
  e0_ = take_event();
  if (e0_ >= 0) cudaEventRecord(g_pool[e0_], st_);
}

KernelTimer::~KernelTimer() {
  if (e0_ < 0) return;
  std::lock_guard<std::mutex> lk(g_mu);
  const int e1 = take_event();
  if (e1 < 0) return;
  cudaEventRecord(g_pool[e1], st_);
  g_recs.push_back(Rec{kernel_, e0_, e1, weight_});
}

}  // namespace dfm

using namespace dfm;

extern "C" long long dfm_launch_count(void) { return g_launches.load(); }

extern "C" int dfm_stats_enable(int on) {
  if (on < 0) return set_error(DFM_ERR_ARG, "dfm_stats_enable: negative sampling interval");
  g_timing.store(on);
  return DFM_OK;
}

extern "C" int dfm_stats_reset(void) {
  std::lock_guard<std::mutex> lk(g_mu);
  g_recs.clear();
  g_next = 0;
  for (long long& c : g_count) c = 0;
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
    n += r.weight;
  }
  const int64_t all = (kernel >= 0 && kernel < DFM_KERNEL_COUNT) ? g_count[kernel] : n;
  *launches = all;
  *total_ms = n ? ms * (double)all / (double)n : 0.0;
  return DFM_OK;
}

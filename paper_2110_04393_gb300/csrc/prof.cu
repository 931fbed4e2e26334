// Live measurement hooks: CUDA events around the grouped-GEMM launches (on the
// caller's stream) and a count of every kernel this library launches. Off by
// default; enabled by the benchmark through tt_prof_enable.
#include <atomic>
#include <mutex>

#include "kernels.cuh"
#include "prof.cuh"

namespace ttr {

namespace {
struct Prof {
  std::mutex mu;
  bool on = false;
  std::vector<cudaEvent_t> pool;
  size_t used = 0;
  double flops = 0.0;
  int64_t gemm_launches = 0;
};
Prof& P() {
  static Prof p;
  return p;
}
std::atomic<int64_t> g_launches{0};
}  // namespace

void prof_count_launch(int n) { g_launches.fetch_add(n, std::memory_order_relaxed); }

bool prof_gemm_begin(cudaStream_t s, cudaEvent_t* e0) {
  Prof& p = P();
  std::lock_guard<std::mutex> g(p.mu);
  if (!p.on) return false;
  while (p.pool.size() < p.used + 2) {
    cudaEvent_t e;
    if (cudaEventCreate(&e) != cudaSuccess) return false;
    p.pool.push_back(e);
  }
  *e0 = p.pool[p.used];
  cudaEventRecord(*e0, s);
  return true;
}

void prof_gemm_end(cudaStream_t s, double flops) {
  Prof& p = P();
  std::lock_guard<std::mutex> g(p.mu);
  cudaEventRecord(p.pool[p.used + 1], s);
  p.used += 2;
  p.flops += flops;
  p.gemm_launches += 1;
}

}  // namespace ttr

using namespace ttr;

extern "C" {

int tt_prof_enable(int on) {
  Prof& p = P();
  std::lock_guard<std::mutex> g(p.mu);
  p.on = (on != 0);
  return TT_OK;
}

int tt_prof_reset(void) {
  Prof& p = P();
  std::lock_guard<std::mutex> g(p.mu);
  p.used = 0;
  p.flops = 0.0;
  p.gemm_launches = 0;
  g_launches.store(0);
  return TT_OK;
}

int tt_prof_read(double* gemm_ms, double* gemm_flops, int64_t* gemm_launches, int64_t* kernel_launches) {
  Prof& p = P();
  std::lock_guard<std::mutex> g(p.mu);
  double ms = 0.0;
  for (size_t i = 0; i + 1 < p.used; i += 2) {
    if (cudaEventSynchronize(p.pool[i + 1]) != cudaSuccess) {
      set_error("tt_prof_read: event synchronize failed");
      return TT_ECUDA;
    }
    float t = 0.f;
    if (cudaEventElapsedTime(&t, p.pool[i], p.pool[i + 1]) != cudaSuccess) {
      set_error("tt_prof_read: elapsed time failed");
      return TT_ECUDA;
    }
    ms += t;
  }
  if (gemm_ms) *gemm_ms = ms;
  if (gemm_flops) *gemm_flops = p.flops;
  if (gemm_launches) *gemm_launches = p.gemm_launches;
  if (kernel_launches) *kernel_launches = g_launches.load();
  return TT_OK;
}

}  // extern "C"

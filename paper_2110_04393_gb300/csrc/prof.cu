// Live measurement hooks: CUDA events around the grouped-GEMM launches (on the
// caller's stream) and a count of every kernel this library launches. Off by
// default; enabled by the benchmark through tt_prof_enable.
#include <atomic>
#include <mutex>

#include "plan.cuh"
#include "prof.cuh"

namespace ttr {

namespace {
struct Prof {
  std::mutex mu;
  bool on = false;
  std::vector<cudaEvent_t> pool;
  std::vector<int> kinds;          // kind of each recorded pair
  size_t used = 0;
  double flops[kProfKinds] = {0.0, 0.0};
  int64_t count[kProfKinds] = {0, 0};
  double replay_ms[kProfKinds] = {0.0, 0.0};
};
Prof& P() {
  static Prof p;
  return p;
}
std::atomic<int64_t> g_launches{0};
thread_local std::vector<ProfPair>* t_sink = nullptr;
thread_local int64_t t_sink_launches = 0;
thread_local cudaEvent_t t_sink_e0 = nullptr;
}  // namespace

void prof_count_launch(int n) {
  if (t_sink) {
    t_sink_launches += n;
    return;
  }
  g_launches.fetch_add(n, std::memory_order_relaxed);
}

void prof_capture_begin(std::vector<ProfPair>* sink) {
  t_sink = sink;
  t_sink_launches = 0;
}
int64_t prof_capture_end() {
  t_sink = nullptr;
  return t_sink_launches;
}
bool prof_on() {
  Prof& p = P();
  std::lock_guard<std::mutex> g(p.mu);
  return p.on;
}

int prof_replayed(const std::vector<ProfPair>& pairs, int64_t launches) {
  Prof& p = P();
  std::lock_guard<std::mutex> g(p.mu);
  if (!p.on) return TT_OK;
  for (const auto& q : pairs) {
    float t = 0.f;
    if (cudaEventElapsedTime(&t, q.e0, q.e1) != cudaSuccess) {
      set_error("profiling: elapsed time of a replayed event pair failed");
      return TT_ECUDA;
    }
    p.replay_ms[q.kind] += t;
    p.flops[q.kind] += q.flops;
    p.count[q.kind] += 1;
  }
  g_launches.fetch_add(launches, std::memory_order_relaxed);
  return TT_OK;
}

bool prof_gemm_begin(cudaStream_t s, cudaEvent_t* e0) { return prof_begin(s, e0); }
void prof_gemm_end(cudaStream_t s, double flops) { prof_end(s, 0, flops); }

bool prof_begin(cudaStream_t s, cudaEvent_t* e0) {
  if (t_sink) {
    if (!prof_on()) return false;
    cudaEvent_t e;
    if (cudaEventCreate(&e) != cudaSuccess) return false;
    // an event node of the graph (a plain record in a capture is only a dependency)
    cudaEventRecordWithFlags(e, s, cudaEventRecordExternal);
    t_sink_e0 = e;
    *e0 = e;
    return true;
  }
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

void prof_end(cudaStream_t s, int kind, double flops) {
  if (t_sink) {
    cudaEvent_t e;
    if (cudaEventCreate(&e) != cudaSuccess) return;
    cudaEventRecordWithFlags(e, s, cudaEventRecordExternal);
    t_sink->push_back(ProfPair{t_sink_e0, e, flops, kind});
    return;
  }
  Prof& p = P();
  std::lock_guard<std::mutex> g(p.mu);
  cudaEventRecord(p.pool[p.used + 1], s);
  if (p.kinds.size() < (p.used + 2) / 2) p.kinds.resize((p.used + 2) / 2);
  p.kinds[p.used / 2] = kind;
  p.used += 2;
  p.flops[kind] += flops;
  p.count[kind] += 1;
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
  for (int k = 0; k < kProfKinds; ++k) {
    p.flops[k] = 0.0;
    p.count[k] = 0;
    p.replay_ms[k] = 0.0;
  }
  g_launches.store(0);
  return TT_OK;
}

// Sum of the eager event pairs of one kind plus the replayed ones.
static int kind_ms(Prof& p, int kind, double* out) {
  double ms = p.replay_ms[kind];
  for (size_t i = 0; i + 1 < p.used; i += 2) {
    if (p.kinds[i / 2] != kind) continue;
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
  *out = ms;
  return TT_OK;
}

int tt_prof_read(double* gemm_ms, double* gemm_flops, int64_t* gemm_launches, int64_t* kernel_launches) {
  Prof& p = P();
  std::lock_guard<std::mutex> g(p.mu);
  double ms = 0.0;
  TTR_TRY(kind_ms(p, 0, &ms));
  if (gemm_ms) *gemm_ms = ms;
  if (gemm_flops) *gemm_flops = p.flops[0];
  if (gemm_launches) *gemm_launches = p.count[0];
  if (kernel_launches) *kernel_launches = g_launches.load();
  return TT_OK;
}

int tt_prof_read_kind(int32_t kind, double* ms, double* flops, int64_t* launches) {
  if (kind < 0 || kind >= kProfKinds) {
    set_error("tt_prof_read_kind: kind must be 0 (contraction groups) or 1 (QR passes)");
    return TT_EINVAL;
  }
  Prof& p = P();
  std::lock_guard<std::mutex> g(p.mu);
  double t = 0.0;
  TTR_TRY(kind_ms(p, kind, &t));
  if (ms) *ms = t;
  if (flops) *flops = p.flops[kind];
  if (launches) *launches = p.count[kind];
  return TT_OK;
}

}  // extern "C"

// Host-side schedule: a list of stream-ordered launch items plus one table of
// GEMM descriptors uploaded once per call (internal to the library).
#pragma once
#include <functional>

#include "kernels.cuh"

namespace ttr {

struct Schedule {
  std::vector<GemmDesc> descs;
  std::vector<std::function<int(cudaStream_t, const GemmDesc*)>> items;
  std::vector<std::vector<double>> host_keep;   // host sources of H2D copies
  int64_t pbuf_need = 0;                        // split-K partial doubles needed by the largest group
  double* pbuf = nullptr;                       // partial buffer (null while sizing)
  int64_t cnt_need = 0;                         // split-K counters needed by the largest group
  int* cnt = nullptr;                           // counters (zeroed once per call, self-resetting)

  void gemm(std::vector<GemmDesc> g) {
    if (g.empty()) return;
    int64_t tiles = 0, pb = 0, cn = 0;
    gemm_prepare(g, &tiles, &pb, &cn, 2 * num_sms(), pbuf, cnt);
    if (pb > pbuf_need) pbuf_need = pb;
    if (cn > cnt_need) cnt_need = cn;
    const size_t off = descs.size();
    const int n = int(g.size());
    double flops = 0.0;
    for (const auto& d : g) flops += 2.0 * double(d.M) * double(d.N) * double(d.K) * double(d.batch);
    descs.insert(descs.end(), g.begin(), g.end());
    items.push_back([=](cudaStream_t s, const GemmDesc* d) { return gemm_launch(d + off, n, tiles, flops, s); });
  }
  // Device status word of one run (zeroed at its start): kernels OR in
  // DEV_TIMEOUT when a bounded wait gives up and DEV_QR_FAIL when a thin QR
  // could not produce an orthonormal basis; the entry points read it back and
  // turn it into TT_ETIMEOUT / TT_ESINGULAR.
  int* dev_status = nullptr;
  int64_t acc_need = 0, ex_need = 0;            // emulated-GEMM accumulators / exponent tags (largest group)
  long long* acc = nullptr;                     // zeroed once per call, left zero by every group
  int* ex = nullptr;                            // zeroed once per call, tagged by epoch
  int64_t plane_need = 0;                       // digit-plane bytes (largest group)
  uint8_t* planes = nullptr;
  int tc_epoch = 0;
  // Group run by the emulated FP64 GEMM on the tensor cores (s digits).
  void gemm_tc(std::vector<GemmDesc> g, int s) {
    if (g.empty()) return;
    double flops = 0.0;
    for (const auto& d : g) flops += 2.0 * double(d.M) * double(d.N) * double(d.K) * double(d.batch);
    TcPlan tp;
    gemm_tc_prepare(g, s, num_sms(), &tp, acc, ex, cnt, planes);
    if (tp.plane_bytes > plane_need) plane_need = tp.plane_bytes;
    if (tp.acc_words > acc_need) acc_need = tp.acc_words;
    if (tp.ex_ints > ex_need) ex_need = tp.ex_ints;
    if (tp.counters > cnt_need) cnt_need = tp.counters;
    const int epoch = ++tc_epoch;
    const size_t off = descs.size();
    const int n = int(g.size());
    descs.insert(descs.end(), g.begin(), g.end());
    int** errp = &dev_status;
    items.push_back([=](cudaStream_t st, const GemmDesc* d) {
      return gemm_tc_launch(d + off, n, tp, s, epoch, flops, *errp, st);
    });
  }
  void add(std::function<int(cudaStream_t)> f) {
    items.push_back([f](cudaStream_t s, const GemmDesc*) { return f(s); });
  }
  // Copy descriptors live in the same uploaded table as raw bytes after the GEMM
  // descriptors would complicate alignment; they get their own device region.
  std::vector<Copy3> copies;
  Copy3* d_copies = nullptr;     // bound by plan_execute
  void copy3(std::vector<Copy3> g) {
    if (g.empty()) return;
    int64_t t = 0;
    for (auto& c : g) { c.begin = t; t += c.n0 * c.n1 * c.n2; }
    const size_t off = copies.size();
    const int n = int(g.size());
    copies.insert(copies.end(), g.begin(), g.end());
    Copy3** base = &d_copies;
    items.push_back([=](cudaStream_t s, const GemmDesc*) { return copy3_launch(*base + off, n, t, s); });
  }
  // Copy of host values into device memory, run every time the schedule runs.
  // Eager runs copy from the kept host vector; a captured (graph) run copies
  // from upload_dev, the pristine device copies laid out in upload order.
  // Returns the upload's offset (doubles) in that layout.
  size_t upload_total = 0;
  const double* upload_dev = nullptr;
  const uint64_t* seed_dev = nullptr;           // graph runs: sketch seed read on the device
  size_t upload(double* dst, std::vector<double> v) {
    host_keep.push_back(std::move(v));
    const size_t idx = host_keep.size() - 1, off = upload_total, n = host_keep.back().size();
    upload_total += n;
    const Schedule* self = this;
    add([self, dst, idx, off, n](cudaStream_t s) -> int {
      if (!dst || n == 0) return int(TT_OK);
      if (self->upload_dev)
        TTR_CHECK_CUDA(cudaMemcpyAsync(dst, self->upload_dev + off, n * sizeof(double), cudaMemcpyDeviceToDevice, s));
      else
        TTR_CHECK_CUDA(
            cudaMemcpyAsync(dst, self->host_keep[idx].data(), n * sizeof(double), cudaMemcpyHostToDevice, s));
      return int(TT_OK);
    });
    return off;
  }
};

inline GemmDesc gdesc(const double* A, int64_t a_rs, int64_t a_cs, const double* B, int64_t b_rs, int64_t b_cs,
                      double* C, int64_t c_rs, int64_t c_cs, int64_t M, int64_t N, int64_t K, double alpha = 1.0,
                      double beta = 0.0) {
  GemmDesc d{};
  d.A = A; d.B = B; d.C = C;
  d.a_rs = a_rs; d.a_cs = a_cs; d.b_rs = b_rs; d.b_cs = b_cs; d.c_rs = c_rs; d.c_cs = c_cs;
  d.M = M; d.N = N; d.K = K;
  d.alpha = alpha; d.beta = beta;
  d.batch = 1; d.ksplit = 1;
  return d;
}

// Runs a planner twice: once to size the workspace, once to bind real pointers
// and execute. build(Arena&, Schedule&) must take arena regions in the same
// order on both passes.
using BuildFn = std::function<int(Arena&, Schedule&)>;
int plan_workspace_bytes(const BuildFn& build, size_t* bytes);
// host_status (may be null): receives the run's device status word by a
// stream-ordered copy enqueued after the last item (valid once the stream has
// been synchronized); see status_code.
int plan_execute(const BuildFn& build, void* workspace, size_t ws_bytes, cudaStream_t s, int* host_status = nullptr);
// Maps a device status word to a tt_status (TT_OK for 0), setting the error text.
int status_code(int bits, const char* who);
// Test hook: bits armed by tt_debug_inject_device_status, consumed (and
// disarmed) by the next read-back of a device status word.
int take_injected_status();

// A schedule captured once into a CUDA graph and replayed (no host planning or
// per-kernel launch cost on replay). The graph owns nothing: the plan keeps the
// workspace, the schedule (whose items hold the device pointers) and the
// pristine copies of the uploads. prologue / epilogue add nodes before and
// after the schedule (may be empty).
struct ProfPair {
  cudaEvent_t e0, e1;
  double flops;
  int kind;
};
struct GraphPlan {
  Schedule* sc = nullptr;
  Schedule* probe = nullptr;           // sizing pass (region sizes for the per-run resets)
  void* ws = nullptr;
  size_t ws_bytes = 0;
  double* pristine = nullptr;
  uint64_t* seed_dev = nullptr;
  GemmDesc* d_descs = nullptr;
  cudaGraphExec_t exec = nullptr;
  int64_t kernels = 0;                 // kernel launches per replay
  std::vector<ProfPair> prof;          // GEMM event pairs, when captured with profiling on
};
using StageFn = std::function<int(cudaStream_t)>;
int plan_capture(const BuildFn& build, const StageFn& prologue, const StageFn& epilogue, cudaStream_t st,
                 GraphPlan* gp);
int plan_replay(GraphPlan& gp, cudaStream_t st);
void plan_free(GraphPlan* gp);
// The pieces of plan_capture, for graphs holding several schedules:
// plan_prepare sizes, allocates, builds and uploads the static tables (no
// capture); plan_emit issues prologue, resets, items and epilogue on a stream
// (inside a capture); capture_graph captures body on a fresh stream and
// instantiates the graph (exec), collecting profiling pairs and launches.
int plan_prepare(const BuildFn& build, GraphPlan* gp);
int plan_emit(GraphPlan& gp, const StageFn& prologue, const StageFn& epilogue, cudaStream_t cs);
int capture_graph(const std::function<int(cudaStream_t)>& body, cudaGraphExec_t* exec, std::vector<ProfPair>* prof,
                  int64_t* kernels);

}  // namespace ttr

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
  int* tc_err = nullptr;                        // device flag of the tensor-core GEMMs
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
    int** errp = &tc_err;
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
  // H2D copy of host values kept alive by the schedule.
  void upload(double* dst, std::vector<double> v) {
    host_keep.push_back(std::move(v));
    const std::vector<double>* src = &host_keep.back();
    const size_t bytes = src->size() * sizeof(double);
    const double* hp = src->data();
    add([dst, hp, bytes](cudaStream_t s) -> int {
      if (!dst || bytes == 0) return int(TT_OK);
      TTR_CHECK_CUDA(cudaMemcpyAsync(dst, hp, bytes, cudaMemcpyHostToDevice, s));
      return int(TT_OK);
    });
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
int plan_execute(const BuildFn& build, void* workspace, size_t ws_bytes, cudaStream_t s);

}  // namespace ttr

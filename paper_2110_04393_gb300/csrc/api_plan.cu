// C ABI: the randomized rounding of a sum (Algorithm 7, with the tolerance
// truncation of Section 3.2 when tol > 0) captured once into a CUDA graph for
// fixed sizes, summand ranks, sketch ranks, tolerance and precision, then
// replayed for any core data, coefficients and sketch seed.
//
// A replay is one pinned host-to-device copy of the run's arguments (core and
// output pointers, seed, coefficients) and one graph launch. The graph gathers
// the summand cores into plan-owned buffers, runs the whole schedule (every
// kernel, copy and reset of the eager entry point, in the same order, so the
// results are bit-wise those of tt_round_sum_rand with the same seed) and
// scatters the rounded cores to the caller's buffers, sized on the device from
// the decided ranks. Only the tolerance mode waits for the stream, to return
// the ranks.
#include <algorithm>
#include <cstring>
#include <string>

#include "plan.cuh"
#include "problem.cuh"
#include "prof.cuh"

namespace ttr {

int build_sum_rand_batch(const std::vector<SumProblem>& Ps, const uint64_t* seeds_dev, int digits, int qr_ctas,
                         const std::vector<std::vector<double*>>& outs, Arena& ar, Schedule& sc);
int build_sum_rand(const SumProblem& P, const double* const* sketch_in, uint64_t seed, double tol, int digits,
                   double* const* out, Arena& ar, Schedule& sc, int64_t** rk_dev, size_t* coeff_off,
                   const double* coeff_dev, int sketch_digits);
int mixed_digits(double tol, int N);

namespace {

constexpr int64_t kCopyBlock = 4096;      // elements per copy block

struct CopyBlock {
  int64_t core;
  int64_t begin, end;
};

__global__ void __launch_bounds__(256) gather_kernel(const CopyBlock* blocks, const double* const* src,
                                                     const int64_t* off, double* dst) {
  const CopyBlock b = blocks[blockIdx.x];
  const double* sp = src[b.core];
  double* dp = dst + off[b.core];
  for (int64_t e = b.begin + threadIdx.x; e < b.end; e += blockDim.x) dp[e] = __ldg(sp + e);
}

// rk (device, may be null): decided ranks; core n holds rk[n] * dims[n] * rk[n+1] values
__global__ void __launch_bounds__(256) scatter_kernel(const CopyBlock* blocks, const double* src, const int64_t* off,
                                                      double* const* dst, const int64_t* rk, const int64_t* dims) {
  const CopyBlock b = blocks[blockIdx.x];
  const int64_t n = b.core;
  const int64_t cnt = rk ? rk[n] * dims[n] * rk[n + 1] : b.end;
  const int64_t end = b.end < cnt ? b.end : cnt;
  const double* sp = src + off[n];
  double* dp = dst[n];
  for (int64_t e = b.begin + threadIdx.x; e < end; e += blockDim.x) dp[e] = sp[e];
}

std::vector<CopyBlock> copy_blocks(const std::vector<int64_t>& sizes) {
  std::vector<CopyBlock> v;
  for (size_t c = 0; c < sizes.size(); ++c)
    for (int64_t b = 0; b < sizes[c]; b += kCopyBlock) v.push_back({int64_t(c), b, std::min(sizes[c], b + kCopyBlock)});
  return v;
}

// One sum rounding inside a graph: plan-owned inputs / outputs, the prepared
// schedule and the copy tables; its run arguments live at stage_off in a
// staging block shared by all problems of the graph.
struct SumUnit {
  SumProblem P;
  double tol = 0.0;
  int digits = 0;
  int sketch_digits = -1;
  double* in_buf = nullptr;
  double* out_buf = nullptr;
  std::vector<double*> outs;
  int64_t* rk_dev = nullptr;
  size_t coeff_off = 0;
  GraphPlan gp;
  void* tables = nullptr;
  CopyBlock* gblocks = nullptr;
  CopyBlock* sblocks = nullptr;
  int64_t* in_off = nullptr;
  int64_t* out_off = nullptr;
  int64_t* dims = nullptr;
  int ngb = 0, nsb = 0;
  size_t stage_off = 0;
  std::vector<int64_t> h_in_off, h_out_off;   // packed host layout (elements)
  int64_t in_total = 0, out_total = 0;
  double* land_in = nullptr;                  // device landing of the host input copy
  double* land_out = nullptr;                 // device source of the host output copy
  int* h_status = nullptr;                    // pinned slot receiving the replay's device status word
};

size_t unit_stage_bytes(int N, int K) {
  return sizeof(double*) * (size_t(K) * N + N) + sizeof(uint64_t) + sizeof(double) * K;
}

void unit_free(SumUnit* u) {
  plan_free(&u->gp);
  if (u->in_buf) cudaFree(u->in_buf);
  if (u->out_buf) cudaFree(u->out_buf);
  if (u->tables) cudaFree(u->tables);
  if (u->land_in) cudaFree(u->land_in);
  if (u->land_out) cudaFree(u->land_out);
  u->land_in = u->land_out = nullptr;
  u->in_buf = u->out_buf = nullptr;
  u->tables = nullptr;
}

// Validates, allocates, uploads the copy tables and prepares the schedule.
int unit_init(SumUnit* u, int32_t N, int32_t K, const int64_t* dims, const int64_t* ranks, const int64_t* ells,
              double tol, int32_t precision) {
  TTR_TRY(validate_sum(N, K, dims, ranks, nullptr, nullptr, ells, false, &u->P));
  SumProblem& P = u->P;
  u->tol = tol;
  u->digits = (precision != TT_PREC_FP64) ? mixed_digits(tol, N) : 0;
  u->sketch_digits = (precision == TT_PREC_MIXED_FULL) ? u->digits : -1;
  std::vector<int64_t> in_sizes, in_off, out_sizes, out_off;
  int64_t tot = 0;
  for (int j = 0; j < K; ++j)
    for (int n = 1; n <= N; ++n) {
      in_off.push_back(tot);
      in_sizes.push_back(P.r(j, n - 1) * P.I[n - 1] * P.r(j, n));
      tot += in_sizes.back();
    }
  const int64_t in_total = tot;
  tot = 0;
  for (int n = 1; n <= N; ++n) {
    out_off.push_back(tot);
    out_sizes.push_back(P.ell[n - 1] * P.I[n - 1] * P.ell[n]);
    tot += out_sizes.back();
  }
  const int64_t out_total = tot;
  u->h_in_off = in_off;
  u->h_out_off = out_off;
  u->in_total = in_total;
  u->out_total = out_total;
  if (cudaMalloc(&u->in_buf, sizeof(double) * std::max<int64_t>(in_total, 1)) != cudaSuccess ||
      cudaMalloc(&u->out_buf, sizeof(double) * std::max<int64_t>(out_total, 1)) != cudaSuccess) {
    cudaGetLastError();
    set_error("plan: buffer allocation failed");
    return TT_ENOMEM;
  }
  P.cores.assign(size_t(K) * N, nullptr);
  for (int j = 0; j < K; ++j)
    for (int n = 1; n <= N; ++n) P.cores[size_t(j) * N + (n - 1)] = u->in_buf + in_off[size_t(j) * N + (n - 1)];
  u->outs.resize(N);
  for (int n = 0; n < N; ++n) u->outs[n] = u->out_buf + out_off[n];
  const auto gb = copy_blocks(in_sizes), sb = copy_blocks(out_sizes);
  u->ngb = int(gb.size());
  u->nsb = int(sb.size());
  const size_t gbb = align256(sizeof(CopyBlock) * std::max<size_t>(gb.size(), 1));
  const size_t sbb = align256(sizeof(CopyBlock) * std::max<size_t>(sb.size(), 1));
  const size_t tb_bytes = gbb + sbb + align256(sizeof(int64_t) * in_off.size()) +
                          align256(sizeof(int64_t) * out_off.size()) + align256(sizeof(int64_t) * N);
  if (cudaMalloc(&u->tables, tb_bytes) != cudaSuccess) {
    cudaGetLastError();
    set_error("plan: table allocation failed");
    return TT_ENOMEM;
  }
  char* t = static_cast<char*>(u->tables);
  u->gblocks = reinterpret_cast<CopyBlock*>(t);
  t += gbb;
  u->sblocks = reinterpret_cast<CopyBlock*>(t);
  t += sbb;
  u->in_off = reinterpret_cast<int64_t*>(t);
  t += align256(sizeof(int64_t) * in_off.size());
  u->out_off = reinterpret_cast<int64_t*>(t);
  t += align256(sizeof(int64_t) * out_off.size());
  u->dims = reinterpret_cast<int64_t*>(t);
  if ((!gb.empty() && cudaMemcpy(u->gblocks, gb.data(), sizeof(CopyBlock) * gb.size(), cudaMemcpyHostToDevice)) ||
      (!sb.empty() && cudaMemcpy(u->sblocks, sb.data(), sizeof(CopyBlock) * sb.size(), cudaMemcpyHostToDevice)) ||
      cudaMemcpy(u->in_off, in_off.data(), sizeof(int64_t) * in_off.size(), cudaMemcpyHostToDevice) ||
      cudaMemcpy(u->out_off, out_off.data(), sizeof(int64_t) * out_off.size(), cudaMemcpyHostToDevice) ||
      cudaMemcpy(u->dims, P.I.data(), sizeof(int64_t) * N, cudaMemcpyHostToDevice)) {
    set_error("plan: table upload failed");
    return TT_ECUDA;
  }
  BuildFn build = [u](Arena& ar, Schedule& sc) {
    return build_sum_rand(u->P, nullptr, 0, u->tol, u->digits, u->outs.data(), ar, sc, &u->rk_dev, &u->coeff_off,
                          nullptr, u->sketch_digits);
  };
  return plan_prepare(build, &u->gp);
}

// Prologue / epilogue of a unit whose staging starts at `stage` (device).
StageFn unit_prologue(SumUnit* u, const char* stage) {
  const int N = u->P.N, K = u->P.K;
  const double* const* d_src = reinterpret_cast<const double* const*>(stage);
  const uint64_t* d_seed = reinterpret_cast<const uint64_t*>(stage + sizeof(double*) * (size_t(K) * N + N));
  const double* d_coeffs = reinterpret_cast<const double*>(stage + sizeof(double*) * (size_t(K) * N + N) + 8);
  return [u, d_src, d_seed, d_coeffs, K](cudaStream_t s) -> int {
    TTR_CHECK_CUDA(cudaMemcpyAsync(u->gp.seed_dev, d_seed, sizeof(uint64_t), cudaMemcpyDeviceToDevice, s));
    if (u->gp.pristine)
      TTR_CHECK_CUDA(cudaMemcpyAsync(u->gp.pristine + u->coeff_off, d_coeffs, sizeof(double) * K,
                                     cudaMemcpyDeviceToDevice, s));
    if (u->ngb > 0) {
      TTR_PREFER_SHARED(gather_kernel);
      gather_kernel<<<unsigned(u->ngb), 256, 0, s>>>(u->gblocks, d_src, u->in_off, u->in_buf);
      TTR_CHECK_LAUNCH();
      prof_count_launch(1);
    }
    return int(TT_OK);
  };
}
StageFn unit_epilogue(SumUnit* u, const char* stage) {
  const int N = u->P.N, K = u->P.K;
  double* const* d_dst = reinterpret_cast<double* const*>(stage + sizeof(double*) * size_t(K) * N);
  return [u, d_dst](cudaStream_t s) -> int {
    if (u->nsb > 0) {
      TTR_PREFER_SHARED(scatter_kernel);
      scatter_kernel<<<unsigned(u->nsb), 256, 0, s>>>(u->sblocks, u->out_buf, u->out_off, d_dst,
                                                      u->tol > 0.0 ? u->rk_dev : nullptr, u->dims);
      TTR_CHECK_LAUNCH();
      prof_count_launch(1);
    }
    if (u->h_status)
      TTR_CHECK_CUDA(cudaMemcpyAsync(u->h_status, u->gp.sc->dev_status, sizeof(int), cudaMemcpyDeviceToHost, s));
    return int(TT_OK);
  };
}

// Host side of a unit's staging: core pointers, output pointers, seed, coefficients.
int unit_fill_stage(const SumUnit* u, char* hs, const double* const* cores, const double* coeffs, uint64_t seed,
                    double* const* out) {
  const int N = u->P.N, K = u->P.K;
  for (size_t i = 0; i < size_t(K) * N; ++i)
    if (!cores[i]) {
      set_error("plan run: null core pointer");
      return TT_EINVAL;
    }
  for (int n = 0; n < N; ++n)
    if (!out[n]) {
      set_error("plan run: null output core pointer");
      return TT_EINVAL;
    }
  std::memcpy(hs, cores, sizeof(double*) * size_t(K) * N);
  std::memcpy(hs + sizeof(double*) * size_t(K) * N, out, sizeof(double*) * N);
  std::memcpy(hs + sizeof(double*) * (size_t(K) * N + N), &seed, sizeof(uint64_t));
  double* hc = reinterpret_cast<double*>(hs + sizeof(double*) * (size_t(K) * N + N) + 8);
  for (int j = 0; j < K; ++j) hc[j] = coeffs ? coeffs[j] : 1.0;
  return TT_OK;
}

// Graph of several units on `width` parallel chains (unit b on chain b mod width).
struct UnitGraph {
  std::vector<SumUnit*> units;
  size_t stage_bytes = 0;
  void* d_stage = nullptr;
  void* h_stage = nullptr;
  int64_t* h_rk = nullptr;       // all units' ranks (sum of N_b + 1)
  int* h_status = nullptr;       // one device status word per unit (pinned)
  std::vector<size_t> rk_off;
  cudaEvent_t staged = nullptr;
  cudaGraphExec_t exec = nullptr;
  std::vector<ProfPair> prof;
  int64_t kernels = 0;
  int width = 1;
};

void unit_graph_free(UnitGraph* g) {
  if (g->exec) cudaGraphExecDestroy(g->exec);
  for (auto& q : g->prof) {
    cudaEventDestroy(q.e0);
    cudaEventDestroy(q.e1);
  }
  for (SumUnit* u : g->units) {
    unit_free(u);
    delete u;
  }
  g->units.clear();
  if (g->d_stage) cudaFree(g->d_stage);
  if (g->h_stage) cudaFreeHost(g->h_stage);
  if (g->h_rk) cudaFreeHost(g->h_rk);
  if (g->h_status) cudaFreeHost(g->h_status);
  if (g->staged) cudaEventDestroy(g->staged);
  *g = UnitGraph{};
}

// Staging layout, then one capture: fork into width chains, every unit's
// prologue / schedule / epilogue on its chain, join.
int unit_graph_capture(UnitGraph* g, int width) {
  g->width = std::max(1, std::min<int>(width, int(g->units.size())));
  size_t off = 0, rk = 0;
  for (SumUnit* u : g->units) {
    u->stage_off = off;
    off += align256(unit_stage_bytes(u->P.N, u->P.K));
    g->rk_off.push_back(rk);
    rk += size_t(u->P.N) + 1;
  }
  g->stage_bytes = std::max<size_t>(off, 256);
  if (cudaMalloc(&g->d_stage, g->stage_bytes) != cudaSuccess ||
      cudaMallocHost(&g->h_stage, g->stage_bytes) != cudaSuccess ||
      cudaMallocHost(reinterpret_cast<void**>(&g->h_rk), sizeof(int64_t) * std::max<size_t>(rk, 1)) != cudaSuccess ||
      cudaMallocHost(reinterpret_cast<void**>(&g->h_status), sizeof(int) * g->units.size()) != cudaSuccess ||
      cudaEventCreateWithFlags(&g->staged, cudaEventDisableTiming) != cudaSuccess) {
    cudaGetLastError();
    set_error("plan: staging allocation failed");
    return TT_ENOMEM;
  }
  std::memset(g->h_stage, 0, g->stage_bytes);
  for (size_t b = 0; b < g->units.size(); ++b) {
    g->h_status[b] = 0;
    g->units[b]->h_status = g->h_status + b;
  }
  const char* ds = static_cast<const char*>(g->d_stage);
  auto body = [&](cudaStream_t cs) -> int {
    if (g->width == 1) {
      for (SumUnit* u : g->units)
        TTR_TRY(plan_emit(u->gp, unit_prologue(u, ds + u->stage_off), unit_epilogue(u, ds + u->stage_off), cs));
      return int(TT_OK);
    }
    std::vector<cudaStream_t> chains(g->width, nullptr);
    std::vector<cudaEvent_t> ev(g->width + 1, nullptr);
    int rc = TT_OK;
    for (auto& e : ev)
      if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess) rc = TT_ECUDA;
    for (auto& c : chains)
      if (cudaStreamCreateWithFlags(&c, cudaStreamNonBlocking) != cudaSuccess) rc = TT_ECUDA;
    if (rc == TT_OK && cudaEventRecord(ev[g->width], cs) != cudaSuccess) rc = TT_ECUDA;
    for (int w = 0; rc == TT_OK && w < g->width; ++w)
      if (cudaStreamWaitEvent(chains[w], ev[g->width], 0) != cudaSuccess) rc = TT_ECUDA;
    for (size_t b = 0; rc == TT_OK && b < g->units.size(); ++b) {
      SumUnit* u = g->units[b];
      rc = plan_emit(u->gp, unit_prologue(u, ds + u->stage_off), unit_epilogue(u, ds + u->stage_off),
                     chains[b % size_t(g->width)]);
    }
    for (int w = 0; rc == TT_OK && w < g->width; ++w) {
      if (cudaEventRecord(ev[w], chains[w]) != cudaSuccess || cudaStreamWaitEvent(cs, ev[w], 0) != cudaSuccess)
        rc = TT_ECUDA;
    }
    if (rc == TT_ECUDA) set_error("plan: fork / join of the capture failed");
    for (auto& e : ev)
      if (e) cudaEventDestroy(e);
    for (auto& c : chains)
      if (c) cudaStreamDestroy(c);
    return rc;
  };
  return capture_graph(body, &g->exec, &g->prof, &g->kernels);
}

// Device status of the last replay (valid once its stream has been synchronized).
int unit_graph_status(const UnitGraph* g, const char* who) {
  int bits = 0;
  for (size_t b = 0; b < g->units.size(); ++b) bits |= g->h_status[b];
  return status_code(bits, who);
}

// One replay: staging copy, graph launch, rank read-back (tolerance units).
// The replay's device status words land in the pinned h_status slots; with a
// tolerance (the call waits) they are turned into the return status.
int unit_graph_run(UnitGraph* g, cudaStream_t s, int64_t* const* out_ranks) {
  TTR_CHECK_CUDA(cudaMemcpyAsync(g->d_stage, g->h_stage, g->stage_bytes, cudaMemcpyHostToDevice, s));
  TTR_CHECK_CUDA(cudaEventRecord(g->staged, s));
  TTR_CHECK_CUDA(cudaGraphLaunch(g->exec, s));
  {
    // test hook: overwrite unit 0's device status word after the replay and read it again
    static thread_local int inj = 0;
    inj = take_injected_status();
    if (inj != 0) {
      SumUnit* u0 = g->units[0];
      TTR_CHECK_CUDA(cudaMemcpyAsync(u0->gp.sc->dev_status, &inj, sizeof(int), cudaMemcpyHostToDevice, s));
      TTR_CHECK_CUDA(cudaStreamSynchronize(s));
      TTR_CHECK_CUDA(cudaMemcpyAsync(u0->h_status, u0->gp.sc->dev_status, sizeof(int), cudaMemcpyDeviceToHost, s));
    }
  }
  bool synced = false;
  bool any_tol = false;
  for (SumUnit* u : g->units) any_tol = any_tol || u->tol > 0.0;
  if (any_tol) {
    for (size_t b = 0; b < g->units.size(); ++b) {
      SumUnit* u = g->units[b];
      if (u->tol > 0.0)
        TTR_CHECK_CUDA(cudaMemcpyAsync(g->h_rk + g->rk_off[b], u->rk_dev, sizeof(int64_t) * (u->P.N + 1),
                                       cudaMemcpyDeviceToHost, s));
    }
    TTR_CHECK_CUDA(cudaStreamSynchronize(s));
    synced = true;
    TTR_TRY(unit_graph_status(g, "plan replay"));
  }
  for (size_t b = 0; b < g->units.size(); ++b) {
    SumUnit* u = g->units[b];
    for (int n = 0; n <= u->P.N; ++n) out_ranks[b][n] = u->tol > 0.0 ? g->h_rk[g->rk_off[b] + n] : u->P.ell[n];
  }
  if (prof_on()) {
    if (!synced) TTR_CHECK_CUDA(cudaStreamSynchronize(s));
    TTR_TRY(prof_replayed(g->prof, g->kernels));
  }
  return TT_OK;
}

// ---------------------------------------------------------------------------
// Fused batches: groups of consecutive problems, each rounded by one schedule
// of grouped launches (build_sum_rand_batch); one gather and one scatter
// launch per group; the groups run on parallel branches of one graph.
struct FusedUnit {
  std::vector<SumProblem> P;
  std::vector<std::vector<double*>> outs;
  int digits = 0, qr_ctas = 8;
  double* in_buf = nullptr;
  double* out_buf = nullptr;
  void* tables = nullptr;
  CopyBlock* gblocks = nullptr;
  CopyBlock* sblocks = nullptr;
  int64_t* in_off = nullptr;
  int64_t* out_off = nullptr;
  int ngb = 0, nsb = 0;
  size_t src0 = 0, dst0 = 0, b0 = 0;     // first core pointer, output pointer and seed of the group
  GraphPlan gp;
  int* h_status = nullptr;
};

struct FusedGraph {
  std::vector<FusedUnit*> units;
  int B = 0;
  size_t n_src = 0, n_dst = 0;           // pointers staged per run
  size_t stage_bytes = 0;
  void* d_stage = nullptr;
  void* h_stage = nullptr;
  int* h_status = nullptr;
  cudaEvent_t staged = nullptr;
  cudaGraphExec_t exec = nullptr;
  std::vector<ProfPair> prof;
  int64_t kernels = 0;
  std::vector<std::vector<int64_t>> ell;   // per problem, the clamped sketch ranks
  std::vector<int> N, K;
};

void fused_free(FusedGraph* g) {
  if (g->exec) cudaGraphExecDestroy(g->exec);
  for (auto& q : g->prof) {
    cudaEventDestroy(q.e0);
    cudaEventDestroy(q.e1);
  }
  for (FusedUnit* u : g->units) {
    plan_free(&u->gp);
    if (u->in_buf) cudaFree(u->in_buf);
    if (u->out_buf) cudaFree(u->out_buf);
    if (u->tables) cudaFree(u->tables);
    delete u;
  }
  g->units.clear();
  if (g->d_stage) cudaFree(g->d_stage);
  if (g->h_stage) cudaFreeHost(g->h_stage);
  if (g->h_status) cudaFreeHost(g->h_status);
  if (g->staged) cudaEventDestroy(g->staged);
  *g = FusedGraph{};
}

int fused_unit_init(FusedUnit* u, const std::vector<SumProblem>& probs, size_t b0, size_t b1, size_t src0,
                    size_t dst0, int digits, int qr_ctas, const uint64_t* seeds_dev) {
  u->P.assign(probs.begin() + b0, probs.begin() + b1);
  u->digits = digits;
  u->qr_ctas = qr_ctas;
  u->src0 = src0;
  u->dst0 = dst0;
  u->b0 = b0;
  std::vector<int64_t> in_sizes, in_off, out_sizes, out_off;
  int64_t it = 0, ot = 0;
  for (const SumProblem& P : u->P) {
    for (int j = 0; j < P.K; ++j)
      for (int n = 1; n <= P.N; ++n) {
        in_off.push_back(it);
        in_sizes.push_back(P.r(j, n - 1) * P.I[n - 1] * P.r(j, n));
        it += in_sizes.back();
      }
    for (int n = 1; n <= P.N; ++n) {
      out_off.push_back(ot);
      out_sizes.push_back(P.ell[n - 1] * P.I[n - 1] * P.ell[n]);
      ot += out_sizes.back();
    }
  }
  if (cudaMalloc(&u->in_buf, sizeof(double) * std::max<int64_t>(it, 1)) != cudaSuccess ||
      cudaMalloc(&u->out_buf, sizeof(double) * std::max<int64_t>(ot, 1)) != cudaSuccess) {
    cudaGetLastError();
    set_error("batch plan: buffer allocation failed");
    return TT_ENOMEM;
  }
  size_t ci = 0, oi = 0;
  u->outs.clear();
  for (SumProblem& P : u->P) {
    P.cores.assign(size_t(P.K) * P.N, nullptr);
    for (size_t c = 0; c < size_t(P.K) * P.N; ++c) P.cores[c] = u->in_buf + in_off[ci++];
    std::vector<double*> o(P.N);
    for (int n = 0; n < P.N; ++n) o[n] = u->out_buf + out_off[oi++];
    u->outs.push_back(o);
  }
  const auto gb = copy_blocks(in_sizes), sb = copy_blocks(out_sizes);
  u->ngb = int(gb.size());
  u->nsb = int(sb.size());
  const size_t gbb = align256(sizeof(CopyBlock) * std::max<size_t>(gb.size(), 1));
  const size_t sbb = align256(sizeof(CopyBlock) * std::max<size_t>(sb.size(), 1));
  const size_t iob = align256(sizeof(int64_t) * std::max<size_t>(in_off.size(), 1));
  const size_t oob = align256(sizeof(int64_t) * std::max<size_t>(out_off.size(), 1));
  if (cudaMalloc(&u->tables, gbb + sbb + iob + oob) != cudaSuccess) {
    cudaGetLastError();
    set_error("batch plan: table allocation failed");
    return TT_ENOMEM;
  }
  char* t = static_cast<char*>(u->tables);
  u->gblocks = reinterpret_cast<CopyBlock*>(t);
  u->sblocks = reinterpret_cast<CopyBlock*>(t + gbb);
  u->in_off = reinterpret_cast<int64_t*>(t + gbb + sbb);
  u->out_off = reinterpret_cast<int64_t*>(t + gbb + sbb + iob);
  if ((!gb.empty() && cudaMemcpy(u->gblocks, gb.data(), sizeof(CopyBlock) * gb.size(), cudaMemcpyHostToDevice)) ||
      (!sb.empty() && cudaMemcpy(u->sblocks, sb.data(), sizeof(CopyBlock) * sb.size(), cudaMemcpyHostToDevice)) ||
      (!in_off.empty() &&
       cudaMemcpy(u->in_off, in_off.data(), sizeof(int64_t) * in_off.size(), cudaMemcpyHostToDevice)) ||
      (!out_off.empty() &&
       cudaMemcpy(u->out_off, out_off.data(), sizeof(int64_t) * out_off.size(), cudaMemcpyHostToDevice))) {
    set_error("batch plan: table upload failed");
    return TT_ECUDA;
  }
  BuildFn build = [u, seeds_dev](Arena& ar, Schedule& sc) {
    return build_sum_rand_batch(u->P, seeds_dev, u->digits, u->qr_ctas, u->outs, ar, sc);
  };
  return plan_prepare(build, &u->gp);
}

int fused_create(FusedGraph* g, int32_t B, const tt_sum_problem* probs, int32_t precision, int width, int qr_ctas) {
  std::vector<SumProblem> P(B);
  for (int b = 0; b < B; ++b) {
    const int rc = validate_sum(probs[b].N, probs[b].K, probs[b].dims, probs[b].ranks, nullptr, nullptr,
                                probs[b].ells, false, &P[b]);
    if (rc != TT_OK) {
      set_error("tt_batch_plan_create: problem " + std::to_string(b) + ": " + tt_last_error());
      return rc;
    }
    g->ell.push_back(P[b].ell);
    g->N.push_back(P[b].N);
    g->K.push_back(P[b].K);
    g->n_src += size_t(P[b].K) * P[b].N;
    g->n_dst += size_t(P[b].N);
  }
  g->B = B;
  int maxN = 1;
  for (const auto& p : P) maxN = std::max(maxN, p.N);
  const int digits = (precision != TT_PREC_FP64) ? mixed_digits(0.0, maxN) : 0;
  g->stage_bytes = align256(sizeof(double*) * (g->n_src + g->n_dst) + sizeof(uint64_t) * size_t(B));
  const int nu = std::max(1, std::min(width, B));
  if (cudaMalloc(&g->d_stage, g->stage_bytes) != cudaSuccess ||
      cudaMallocHost(&g->h_stage, g->stage_bytes) != cudaSuccess ||
      cudaMallocHost(reinterpret_cast<void**>(&g->h_status), sizeof(int) * size_t(nu)) != cudaSuccess ||
      cudaEventCreateWithFlags(&g->staged, cudaEventDisableTiming) != cudaSuccess) {
    cudaGetLastError();
    set_error("batch plan: staging allocation failed");
    return TT_ENOMEM;
  }
  std::memset(g->h_stage, 0, g->stage_bytes);
  const char* ds = static_cast<const char*>(g->d_stage);
  const uint64_t* seeds = reinterpret_cast<const uint64_t*>(ds + sizeof(double*) * (g->n_src + g->n_dst));
  size_t src = 0, dst = 0;
  for (int u = 0; u < nu; ++u) {
    const size_t b0 = size_t(B) * u / nu, b1 = size_t(B) * (u + 1) / nu;
    FusedUnit* fu = new FusedUnit;
    g->units.push_back(fu);
    fu->h_status = g->h_status + u;
    *fu->h_status = 0;
    TTR_TRY(fused_unit_init(fu, P, b0, b1, src, dst, digits, qr_ctas, seeds + b0));
    for (size_t b = b0; b < b1; ++b) {
      src += size_t(P[b].K) * P[b].N;
      dst += size_t(P[b].N);
    }
  }
  auto emit = [g, ds](FusedUnit* u, cudaStream_t cs) -> int {
    const double* const* srcp = reinterpret_cast<const double* const*>(ds) + u->src0;
    double* const* dstp = reinterpret_cast<double* const*>(ds + sizeof(double*) * g->n_src) + u->dst0;
    StageFn pro = [u, srcp](cudaStream_t s) -> int {
      if (u->ngb > 0) {
        TTR_PREFER_SHARED(gather_kernel);
        gather_kernel<<<unsigned(u->ngb), 256, 0, s>>>(u->gblocks, srcp, u->in_off, u->in_buf);
        TTR_CHECK_LAUNCH();
        prof_count_launch(1);
      }
      return int(TT_OK);
    };
    StageFn epi = [u, dstp](cudaStream_t s) -> int {
      if (u->nsb > 0) {
        TTR_PREFER_SHARED(scatter_kernel);
        scatter_kernel<<<unsigned(u->nsb), 256, 0, s>>>(u->sblocks, u->out_buf, u->out_off, dstp, nullptr, nullptr);
        TTR_CHECK_LAUNCH();
        prof_count_launch(1);
      }
      TTR_CHECK_CUDA(cudaMemcpyAsync(u->h_status, u->gp.sc->dev_status, sizeof(int), cudaMemcpyDeviceToHost, s));
      return int(TT_OK);
    };
    return plan_emit(u->gp, pro, epi, cs);
  };
  auto body = [&](cudaStream_t cs) -> int {
    if (g->units.size() == 1) return emit(g->units[0], cs);
    const int w = int(g->units.size());
    std::vector<cudaStream_t> chains(w, nullptr);
    std::vector<cudaEvent_t> ev(w + 1, nullptr);
    int rc = TT_OK;
    for (auto& e : ev)
      if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess) rc = TT_ECUDA;
    for (auto& c : chains)
      if (cudaStreamCreateWithFlags(&c, cudaStreamNonBlocking) != cudaSuccess) rc = TT_ECUDA;
    if (rc == TT_OK && cudaEventRecord(ev[w], cs) != cudaSuccess) rc = TT_ECUDA;
    for (int i = 0; rc == TT_OK && i < w; ++i)
      if (cudaStreamWaitEvent(chains[i], ev[w], 0) != cudaSuccess) rc = TT_ECUDA;
    for (int i = 0; rc == TT_OK && i < w; ++i) rc = emit(g->units[i], chains[i]);
    for (int i = 0; rc == TT_OK && i < w; ++i)
      if (cudaEventRecord(ev[i], chains[i]) != cudaSuccess || cudaStreamWaitEvent(cs, ev[i], 0) != cudaSuccess)
        rc = TT_ECUDA;
    if (rc == TT_ECUDA) set_error("batch plan: fork / join of the capture failed");
    for (auto& e : ev)
      if (e) cudaEventDestroy(e);
    for (auto& c : chains)
      if (c) cudaStreamDestroy(c);
    return rc;
  };
  return capture_graph(body, &g->exec, &g->prof, &g->kernels);
}

int fused_status(const FusedGraph* g, const char* who) {
  int bits = 0;
  for (size_t u = 0; u < g->units.size(); ++u) bits |= g->h_status[u];
  return status_code(bits, who);
}

int fused_run(FusedGraph* g, const double* const* cores, const uint64_t* seeds, double* const* out,
              int64_t* out_ranks, cudaStream_t s) {
  TTR_CHECK_CUDA(cudaEventSynchronize(g->staged));
  char* hs = static_cast<char*>(g->h_stage);
  for (size_t i = 0; i < g->n_src; ++i)
    if (!cores[i]) {
      set_error("tt_batch_plan_run: null core pointer");
      return TT_EINVAL;
    }
  for (size_t i = 0; i < g->n_dst; ++i)
    if (!out[i]) {
      set_error("tt_batch_plan_run: null output core pointer");
      return TT_EINVAL;
    }
  std::memcpy(hs, cores, sizeof(double*) * g->n_src);
  std::memcpy(hs + sizeof(double*) * g->n_src, out, sizeof(double*) * g->n_dst);
  uint64_t* hsd = reinterpret_cast<uint64_t*>(hs + sizeof(double*) * (g->n_src + g->n_dst));
  for (int b = 0; b < g->B; ++b) hsd[b] = seeds ? seeds[b] : uint64_t(b);
  TTR_CHECK_CUDA(cudaMemcpyAsync(g->d_stage, g->h_stage, g->stage_bytes, cudaMemcpyHostToDevice, s));
  TTR_CHECK_CUDA(cudaEventRecord(g->staged, s));
  TTR_CHECK_CUDA(cudaGraphLaunch(g->exec, s));
  {
    static thread_local int inj = 0;
    inj = take_injected_status();
    if (inj != 0) {
      FusedUnit* u0 = g->units[0];
      TTR_CHECK_CUDA(cudaMemcpyAsync(u0->gp.sc->dev_status, &inj, sizeof(int), cudaMemcpyHostToDevice, s));
      TTR_CHECK_CUDA(cudaStreamSynchronize(s));
      TTR_CHECK_CUDA(cudaMemcpyAsync(u0->h_status, u0->gp.sc->dev_status, sizeof(int), cudaMemcpyDeviceToHost, s));
    }
  }
  size_t ri = 0;
  for (int b = 0; b < g->B; ++b)
    for (int n = 0; n <= g->N[b]; ++n) out_ranks[ri++] = g->ell[b][n];
  if (prof_on()) {
    TTR_CHECK_CUDA(cudaStreamSynchronize(s));
    TTR_TRY(prof_replayed(g->prof, g->kernels));
  }
  return TT_OK;
}

}  // namespace
}  // namespace ttr

using namespace ttr;

struct tt_sum_plan {
  UnitGraph g;
};
struct tt_batch_plan {
  UnitGraph g;
  FusedGraph f;
  bool fused = false;
  std::vector<int> N, K;
};

extern "C" {

int tt_sum_plan_create(int32_t N, int32_t K, const int64_t* dims, const int64_t* ranks, const int64_t* ells,
                       double tol, int32_t precision, tt_sum_plan** plan, void* stream) {
  if (!plan) {
    set_error("tt_sum_plan_create: null plan pointer");
    return TT_EINVAL;
  }
  *plan = nullptr;
  if (precision != TT_PREC_FP64 && precision != TT_PREC_MIXED && precision != TT_PREC_MIXED_FULL) {
    set_error("tt_sum_plan_create: unknown precision mode");
    return TT_EINVAL;
  }
  tt_sum_plan* p = new tt_sum_plan;
  SumUnit* u = new SumUnit;
  p->g.units.push_back(u);
  int rc = unit_init(u, N, K, dims, ranks, ells, tol, precision);
  if (rc == TT_OK) rc = unit_graph_capture(&p->g, 1);
  if (rc != TT_OK) {
    unit_graph_free(&p->g);
    delete p;
    return rc;
  }
  (void)stream;
  *plan = p;
  return TT_OK;
}

int tt_sum_plan_run(tt_sum_plan* p, const double* const* cores, const double* coeffs, uint64_t seed,
                    double* const* out, int64_t* out_ranks, void* stream) {
  if (!p || !cores || !out || !out_ranks) {
    set_error("tt_sum_plan_run: null argument");
    return TT_EINVAL;
  }
  TTR_CHECK_CUDA(cudaEventSynchronize(p->g.staged));   // the previous staging copy left the pinned block
  SumUnit* u = p->g.units[0];
  TTR_TRY(unit_fill_stage(u, static_cast<char*>(p->g.h_stage) + u->stage_off, cores, coeffs, seed, out));
  int64_t* const rk[1] = {out_ranks};
  return unit_graph_run(&p->g, static_cast<cudaStream_t>(stream), rk);
}

int tt_sum_plan_host_layout(const tt_sum_plan* p, int64_t* in_offsets, int64_t* out_offsets, int64_t* in_total,
                            int64_t* out_total) {
  if (!p) {
    set_error("tt_sum_plan_host_layout: null plan");
    return TT_EINVAL;
  }
  const SumUnit* u = p->g.units[0];
  if (in_offsets) std::copy(u->h_in_off.begin(), u->h_in_off.end(), in_offsets);
  if (out_offsets) std::copy(u->h_out_off.begin(), u->h_out_off.end(), out_offsets);
  if (in_total) *in_total = u->in_total;
  if (out_total) *out_total = u->out_total;
  return TT_OK;
}

int tt_sum_plan_run_host(tt_sum_plan* p, const double* h_in, const double* coeffs, uint64_t seed, double* h_out,
                         int64_t* out_ranks, void* stream) {
  if (!p || !h_in || !h_out || !out_ranks) {
    set_error("tt_sum_plan_run_host: null argument");
    return TT_EINVAL;
  }
  SumUnit* u = p->g.units[0];
  const cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (!u->land_in) {
    if (cudaMalloc(&u->land_in, sizeof(double) * std::max<int64_t>(u->in_total, 1)) != cudaSuccess ||
        cudaMalloc(&u->land_out, sizeof(double) * std::max<int64_t>(u->out_total, 1)) != cudaSuccess) {
      cudaGetLastError();
      set_error("tt_sum_plan_run_host: landing buffer allocation failed");
      return TT_ENOMEM;
    }
  }
  const int N = u->P.N, K = u->P.K;
  std::vector<const double*> cores(size_t(K) * N);
  std::vector<double*> outs(N);
  for (size_t i = 0; i < cores.size(); ++i) cores[i] = u->land_in + u->h_in_off[i];
  for (int n = 0; n < N; ++n) outs[n] = u->land_out + u->h_out_off[n];
  TTR_CHECK_CUDA(cudaEventSynchronize(p->g.staged));
  TTR_TRY(unit_fill_stage(u, static_cast<char*>(p->g.h_stage) + u->stage_off, cores.data(), coeffs, seed,
                          outs.data()));
  if (u->in_total > 0)
    TTR_CHECK_CUDA(cudaMemcpyAsync(u->land_in, h_in, sizeof(double) * u->in_total, cudaMemcpyHostToDevice, s));
  int64_t* const rk[1] = {out_ranks};
  TTR_TRY(unit_graph_run(&p->g, s, rk));
  if (u->out_total > 0)
    TTR_CHECK_CUDA(cudaMemcpyAsync(h_out, u->land_out, sizeof(double) * u->out_total, cudaMemcpyDeviceToHost, s));
  TTR_CHECK_CUDA(cudaStreamSynchronize(s));
  return unit_graph_status(&p->g, "tt_sum_plan_run_host");
}

int tt_sum_plan_status(tt_sum_plan* p, void* stream) {
  if (!p) {
    set_error("tt_sum_plan_status: null plan");
    return TT_EINVAL;
  }
  TTR_CHECK_CUDA(cudaStreamSynchronize(static_cast<cudaStream_t>(stream)));
  return unit_graph_status(&p->g, "tt_sum_plan_run");
}

int tt_sum_plan_destroy(tt_sum_plan* p) {
  if (!p) return TT_OK;
  cudaDeviceSynchronize();
  unit_graph_free(&p->g);
  delete p;
  return TT_OK;
}

int64_t tt_sum_plan_launches(const tt_sum_plan* p) { return p ? p->g.kernels : 0; }

int tt_batch_plan_create_sched(int32_t B, const tt_sum_problem* probs, int32_t precision,
                               const tt_batch_schedule* sched, tt_batch_plan** plan, void* stream) {
  if (!plan || B < 1 || !probs || !sched || sched->width < 1) {
    set_error("tt_batch_plan_create: need B >= 1 problems, a schedule with width >= 1 and a plan pointer");
    return TT_EINVAL;
  }
  *plan = nullptr;
  if (precision != TT_PREC_FP64 && precision != TT_PREC_MIXED) {
    set_error("tt_batch_plan_create: unknown precision mode");
    return TT_EINVAL;
  }
  const int width = sched->width;
  // fused grouped launches need fixed ranks and target ranks the batched QR takes
  bool can_fuse = true;
  for (int b = 0; b < B; ++b) {
    if (probs[b].tol > 0.0) can_fuse = false;
    if (probs[b].ells)
      for (int n = 1; n < probs[b].N; ++n)
        if (probs[b].ells[n] > 96) can_fuse = false;
  }
  if (sched->fused == 1 && !can_fuse) {
    set_error("tt_batch_plan_create: the fused schedule needs fixed ranks (tol <= 0) and target ranks <= 96");
    return TT_EUNSUPPORTED;
  }
  if (sched->fused != 0 && can_fuse) {
    tt_batch_plan* p = new tt_batch_plan;
    p->fused = true;
    const int rc = fused_create(&p->f, B, probs, precision, width, sched->qr_ctas > 0 ? sched->qr_ctas : 8);
    if (rc != TT_OK) {
      fused_free(&p->f);
      delete p;
      return rc;
    }
    (void)stream;
    *plan = p;
    return TT_OK;
  }
  tt_batch_plan* p = new tt_batch_plan;
  int rc = TT_OK;
  for (int b = 0; rc == TT_OK && b < B; ++b) {
    SumUnit* u = new SumUnit;
    p->g.units.push_back(u);
    rc = unit_init(u, probs[b].N, probs[b].K, probs[b].dims, probs[b].ranks, probs[b].ells, probs[b].tol,
                   precision);
    if (rc != TT_OK) set_error("tt_batch_plan_create: problem " + std::to_string(b) + ": " + tt_last_error());
    p->N.push_back(probs[b].N);
    p->K.push_back(probs[b].K);
  }
  if (rc == TT_OK) rc = unit_graph_capture(&p->g, width);
  if (rc != TT_OK) {
    unit_graph_free(&p->g);
    delete p;
    return rc;
  }
  (void)stream;
  *plan = p;
  return TT_OK;
}

int tt_batch_plan_create(int32_t B, const tt_sum_problem* probs, int32_t precision, int32_t width,
                         tt_batch_plan** plan, void* stream) {
  tt_batch_schedule sc{width, 8, -1};
  return tt_batch_plan_create_sched(B, probs, precision, &sc, plan, stream);
}

int tt_batch_plan_run(tt_batch_plan* p, const double* const* cores, const uint64_t* seeds, double* const* out,
                      int64_t* out_ranks, void* stream) {
  if (!p || !cores || !out || !out_ranks) {
    set_error("tt_batch_plan_run: null argument");
    return TT_EINVAL;
  }
  if (p->fused) return fused_run(&p->f, cores, seeds, out, out_ranks, static_cast<cudaStream_t>(stream));
  TTR_CHECK_CUDA(cudaEventSynchronize(p->g.staged));
  std::vector<int64_t*> rk(p->g.units.size());
  size_t ci = 0, oi = 0, ri = 0;
  for (size_t b = 0; b < p->g.units.size(); ++b) {
    SumUnit* u = p->g.units[b];
    TTR_TRY(unit_fill_stage(u, static_cast<char*>(p->g.h_stage) + u->stage_off, cores + ci, nullptr,
                            seeds ? seeds[b] : uint64_t(b), out + oi));
    rk[b] = out_ranks + ri;
    ci += size_t(u->P.K) * u->P.N;
    oi += size_t(u->P.N);
    ri += size_t(u->P.N) + 1;
  }
  return unit_graph_run(&p->g, static_cast<cudaStream_t>(stream), rk.data());
}

int tt_batch_plan_status(tt_batch_plan* p, void* stream) {
  if (!p) {
    set_error("tt_batch_plan_status: null plan");
    return TT_EINVAL;
  }
  TTR_CHECK_CUDA(cudaStreamSynchronize(static_cast<cudaStream_t>(stream)));
  if (p->fused) return fused_status(&p->f, "tt_batch_plan_run");
  return unit_graph_status(&p->g, "tt_batch_plan_run");
}

int tt_batch_plan_destroy(tt_batch_plan* p) {
  if (!p) return TT_OK;
  cudaDeviceSynchronize();
  if (p->fused) fused_free(&p->f);
  else unit_graph_free(&p->g);
  delete p;
  return TT_OK;
}

int64_t tt_batch_plan_launches(const tt_batch_plan* p) { return p ? (p->fused ? p->f.kernels : p->g.kernels) : 0; }
int tt_batch_plan_is_fused(const tt_batch_plan* p) { return p && p->fused ? 1 : 0; }

}  // extern "C"

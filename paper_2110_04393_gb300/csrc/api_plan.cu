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

int build_sum_rand(const SumProblem& P, const double* const* sketch_in, uint64_t seed, double tol, int digits,
                   double* const* out, Arena& ar, Schedule& sc, int64_t** rk_dev, size_t* coeff_off);
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

}  // namespace
}  // namespace ttr

using namespace ttr;

struct tt_sum_plan {
  SumProblem P;
  double tol = 0.0;
  int digits = 0;
  double* in_buf = nullptr;
  double* out_buf = nullptr;
  std::vector<double*> outs;
  int64_t* rk_dev = nullptr;
  size_t coeff_off = 0;
  GraphPlan gp;
  // static device tables: gather / scatter blocks, offsets, mode sizes
  void* tables = nullptr;
  CopyBlock* gblocks = nullptr;
  CopyBlock* sblocks = nullptr;
  int64_t* in_off = nullptr;
  int64_t* out_off = nullptr;
  int64_t* dims = nullptr;
  int ngb = 0, nsb = 0;
  // per-run arguments: [src pointers K*N | dst pointers N | seed | coefficients K]
  size_t stage_bytes = 0;
  void* d_stage = nullptr;
  void* h_stage = nullptr;
  int64_t* h_rk = nullptr;
  cudaEvent_t staged = nullptr;
};

static void sum_plan_free(tt_sum_plan* p) {
  if (!p) return;
  plan_free(&p->gp);
  if (p->in_buf) cudaFree(p->in_buf);
  if (p->out_buf) cudaFree(p->out_buf);
  if (p->tables) cudaFree(p->tables);
  if (p->d_stage) cudaFree(p->d_stage);
  if (p->h_stage) cudaFreeHost(p->h_stage);
  if (p->h_rk) cudaFreeHost(p->h_rk);
  if (p->staged) cudaEventDestroy(p->staged);
  delete p;
}

extern "C" {

int tt_sum_plan_create(int32_t N, int32_t K, const int64_t* dims, const int64_t* ranks, const int64_t* ells,
                       double tol, int32_t precision, tt_sum_plan** plan, void* stream) {
  if (!plan) {
    set_error("tt_sum_plan_create: null plan pointer");
    return TT_EINVAL;
  }
  *plan = nullptr;
  if (precision != TT_PREC_FP64 && precision != TT_PREC_MIXED) {
    set_error("tt_sum_plan_create: unknown precision mode");
    return TT_EINVAL;
  }
  tt_sum_plan* p = new tt_sum_plan;
  int rc = validate_sum(N, K, dims, ranks, nullptr, nullptr, ells, false, &p->P);
  if (rc != TT_OK) {
    delete p;
    return rc;
  }
  SumProblem& P = p->P;
  p->tol = tol;
  p->digits = (precision == TT_PREC_MIXED) ? mixed_digits(tol, N) : 0;
  auto fail = [&](int code, const std::string& msg) {
    if (!msg.empty()) set_error("tt_sum_plan_create: " + msg);
    sum_plan_free(p);
    return code;
  };
  // plan-owned inputs (summand cores packed) and outputs (capacity l_{n-1} I_n l_n)
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
  if (cudaMalloc(&p->in_buf, sizeof(double) * std::max<int64_t>(in_total, 1)) != cudaSuccess ||
      cudaMalloc(&p->out_buf, sizeof(double) * std::max<int64_t>(out_total, 1)) != cudaSuccess) {
    cudaGetLastError();
    return fail(TT_ENOMEM, "buffer allocation failed");
  }
  P.cores.assign(size_t(K) * N, nullptr);
  for (int j = 0; j < K; ++j)
    for (int n = 1; n <= N; ++n) P.cores[size_t(j) * N + (n - 1)] = p->in_buf + in_off[size_t(j) * N + (n - 1)];
  p->outs.resize(N);
  for (int n = 0; n < N; ++n) p->outs[n] = p->out_buf + out_off[n];

  // static tables
  const auto gb = copy_blocks(in_sizes), sb = copy_blocks(out_sizes);
  p->ngb = int(gb.size());
  p->nsb = int(sb.size());
  const size_t tb_bytes = align256(sizeof(CopyBlock) * std::max<size_t>(gb.size(), 1)) +
                          align256(sizeof(CopyBlock) * std::max<size_t>(sb.size(), 1)) +
                          align256(sizeof(int64_t) * in_off.size()) + align256(sizeof(int64_t) * out_off.size()) +
                          align256(sizeof(int64_t) * N);
  if (cudaMalloc(&p->tables, tb_bytes) != cudaSuccess) {
    cudaGetLastError();
    return fail(TT_ENOMEM, "table allocation failed");
  }
  char* t = static_cast<char*>(p->tables);
  p->gblocks = reinterpret_cast<CopyBlock*>(t);
  t += align256(sizeof(CopyBlock) * std::max<size_t>(gb.size(), 1));
  p->sblocks = reinterpret_cast<CopyBlock*>(t);
  t += align256(sizeof(CopyBlock) * std::max<size_t>(sb.size(), 1));
  p->in_off = reinterpret_cast<int64_t*>(t);
  t += align256(sizeof(int64_t) * in_off.size());
  p->out_off = reinterpret_cast<int64_t*>(t);
  t += align256(sizeof(int64_t) * out_off.size());
  p->dims = reinterpret_cast<int64_t*>(t);
  if ((!gb.empty() && cudaMemcpy(p->gblocks, gb.data(), sizeof(CopyBlock) * gb.size(), cudaMemcpyHostToDevice)) ||
      (!sb.empty() && cudaMemcpy(p->sblocks, sb.data(), sizeof(CopyBlock) * sb.size(), cudaMemcpyHostToDevice)) ||
      cudaMemcpy(p->in_off, in_off.data(), sizeof(int64_t) * in_off.size(), cudaMemcpyHostToDevice) ||
      cudaMemcpy(p->out_off, out_off.data(), sizeof(int64_t) * out_off.size(), cudaMemcpyHostToDevice) ||
      cudaMemcpy(p->dims, P.I.data(), sizeof(int64_t) * N, cudaMemcpyHostToDevice))
    return fail(TT_ECUDA, "table upload failed");

  // per-run staging
  p->stage_bytes = sizeof(double*) * (size_t(K) * N + N) + sizeof(uint64_t) + sizeof(double) * K;
  if (cudaMalloc(&p->d_stage, p->stage_bytes) != cudaSuccess ||
      cudaMallocHost(&p->h_stage, p->stage_bytes) != cudaSuccess ||
      cudaMallocHost(reinterpret_cast<void**>(&p->h_rk), sizeof(int64_t) * (N + 1)) != cudaSuccess ||
      cudaEventCreateWithFlags(&p->staged, cudaEventDisableTiming) != cudaSuccess) {
    cudaGetLastError();
    return fail(TT_ENOMEM, "staging allocation failed");
  }
  std::memset(p->h_stage, 0, p->stage_bytes);
  char* ds = static_cast<char*>(p->d_stage);
  const double* const* d_src = reinterpret_cast<const double* const*>(ds);
  double* const* d_dst = reinterpret_cast<double* const*>(ds + sizeof(double*) * size_t(K) * N);
  const uint64_t* d_seed = reinterpret_cast<const uint64_t*>(ds + sizeof(double*) * (size_t(K) * N + N));
  const double* d_coeffs = reinterpret_cast<const double*>(ds + sizeof(double*) * (size_t(K) * N + N) + 8);

  BuildFn build = [p](Arena& ar, Schedule& sc) {
    return build_sum_rand(p->P, nullptr, 0, p->tol, p->digits, p->outs.data(), ar, sc, &p->rk_dev, &p->coeff_off);
  };
  GraphPlan* gpp = &p->gp;
  const int Kc = K;
  StageFn prologue = [p, gpp, d_src, d_seed, d_coeffs, Kc](cudaStream_t s) -> int {
    TTR_CHECK_CUDA(cudaMemcpyAsync(gpp->seed_dev, d_seed, sizeof(uint64_t), cudaMemcpyDeviceToDevice, s));
    if (gpp->pristine)
      TTR_CHECK_CUDA(cudaMemcpyAsync(gpp->pristine + p->coeff_off, d_coeffs, sizeof(double) * Kc,
                                     cudaMemcpyDeviceToDevice, s));
    if (p->ngb > 0) {
      gather_kernel<<<unsigned(p->ngb), 256, 0, s>>>(p->gblocks, d_src, p->in_off, p->in_buf);
      TTR_CHECK_LAUNCH();
      prof_count_launch(1);
    }
    return int(TT_OK);
  };
  StageFn epilogue = [p, d_dst](cudaStream_t s) -> int {
    if (p->nsb > 0) {
      scatter_kernel<<<unsigned(p->nsb), 256, 0, s>>>(p->sblocks, p->out_buf, p->out_off, d_dst,
                                                      p->tol > 0.0 ? p->rk_dev : nullptr, p->dims);
      TTR_CHECK_LAUNCH();
      prof_count_launch(1);
    }
    return int(TT_OK);
  };
  rc = plan_capture(build, prologue, epilogue, static_cast<cudaStream_t>(stream), &p->gp);
  if (rc != TT_OK) return fail(rc, "");
  *plan = p;
  return TT_OK;
}

int tt_sum_plan_run(tt_sum_plan* p, const double* const* cores, const double* coeffs, uint64_t seed,
                    double* const* out, int64_t* out_ranks, void* stream) {
  if (!p || !cores || !out || !out_ranks) {
    set_error("tt_sum_plan_run: null argument");
    return TT_EINVAL;
  }
  const SumProblem& P = p->P;
  const int N = P.N, K = P.K;
  for (size_t i = 0; i < size_t(K) * N; ++i)
    if (!cores[i]) {
      set_error("tt_sum_plan_run: null core pointer");
      return TT_EINVAL;
    }
  for (int n = 0; n < N; ++n)
    if (!out[n]) {
      set_error("tt_sum_plan_run: null output core pointer");
      return TT_EINVAL;
    }
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  // the previous run's staging copy must have left the pinned buffer
  TTR_CHECK_CUDA(cudaEventSynchronize(p->staged));
  char* hs = static_cast<char*>(p->h_stage);
  std::memcpy(hs, cores, sizeof(double*) * size_t(K) * N);
  std::memcpy(hs + sizeof(double*) * size_t(K) * N, out, sizeof(double*) * N);
  std::memcpy(hs + sizeof(double*) * (size_t(K) * N + N), &seed, sizeof(uint64_t));
  double* hc = reinterpret_cast<double*>(hs + sizeof(double*) * (size_t(K) * N + N) + 8);
  for (int j = 0; j < K; ++j) hc[j] = coeffs ? coeffs[j] : 1.0;
  TTR_CHECK_CUDA(cudaMemcpyAsync(p->d_stage, p->h_stage, p->stage_bytes, cudaMemcpyHostToDevice, s));
  TTR_CHECK_CUDA(cudaEventRecord(p->staged, s));
  TTR_TRY(plan_replay(p->gp, s));
  if (p->tol > 0.0) {
    TTR_CHECK_CUDA(cudaMemcpyAsync(p->h_rk, p->rk_dev, sizeof(int64_t) * (N + 1), cudaMemcpyDeviceToHost, s));
    TTR_CHECK_CUDA(cudaStreamSynchronize(s));
    for (int n = 0; n <= N; ++n) out_ranks[n] = p->h_rk[n];
  } else {
    for (int n = 0; n <= N; ++n) out_ranks[n] = P.ell[n];
  }
  if (prof_on()) {
    TTR_CHECK_CUDA(cudaStreamSynchronize(s));
    TTR_TRY(prof_replayed(p->gp.prof, p->gp.kernels));
  }
  return TT_OK;
}

int tt_sum_plan_destroy(tt_sum_plan* p) {
  if (p) cudaDeviceSynchronize();
  sum_plan_free(p);
  return TT_OK;
}

int64_t tt_sum_plan_launches(const tt_sum_plan* p) { return p ? p->gp.kernels : 0; }

}  // extern "C"

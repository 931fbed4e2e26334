// C ABI: planner + stream-ordered execution of the randomized roundings.
//
// tt_round_sum_rand follows Algorithm 7 (Section 3.4):
//   RL sweep (Algorithm 3 per summand, shared sketch), n = N..2:
//     Z^{(j)}   = V(Y^{(j)}_n) W^{(j)}_n                 (one grouped GEMM, all j)
//     W^{(j)}_{n-1} = H(Z^{(j)}) H(Omega_n)^T            (one grouped split-K GEMM)
//   LR sweep, n = 1..N-1 (M_0 = the summand coefficients):
//     X_n(:, i, :) = [M^{(j)}_{n-1} Y^{(j)}_n(:, i, :)]_j (batched over i and j)
//     Y_n = V(X_n) [W^{(1)}_n; ...; W^{(K)}_n]           (GEMM)
//     V(Xout_n) = Q of TSQR(Y_n)                         (thin Householder QR)
//     [M^{(1)}_n ... M^{(K)}_n] = Q^T V(X_n)             (split-K GEMM)
//   last core: X_N = sum_j M^{(j)}_{N-1} Y^{(j)}_N, i.e. V(X_N) times a column of ones.
// With tol > 0 the left-orthogonal result is truncated right to left
// (Section 3.2 with Algorithm 2's loop mirrored): per bond TSQR of H(X_n)^T,
// the eps-rule on R, then X_n := (Q G1)^T and X_{n-1} := X_{n-1} G2.
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstring>
#include <string>

#include "plan.cuh"
#include "prof.cuh"
#include "qr.cuh"
#include "problem.cuh"

namespace ttr {

static thread_local std::string g_err;
// the all-reduce hook of the current tt_round_sum_rand_sharded call (this thread)
static thread_local tt_allreduce_fn g_allreduce = nullptr;
static thread_local void* g_allreduce_ctx = nullptr;
void set_error(const std::string& msg) { g_err = msg; }

// Arena regions plus the schedule's own regions (partials, descriptors,
// counters, copy descriptors, error flag, emulated-GEMM accumulators,
// exponent tags and digit planes), each 256-byte aligned.
static size_t schedule_bytes(const Arena& a, const Schedule& s) {
  return a.used + align256(size_t(std::max<int64_t>(s.pbuf_need, 1)) * sizeof(double)) +
         align256(std::max<size_t>(s.descs.size(), 1) * sizeof(GemmDesc)) +
         align256(size_t(std::max<int64_t>(s.cnt_need, 1)) * sizeof(int)) +
         align256(std::max<size_t>(s.copies.size(), 1) * sizeof(Copy3)) + align256(sizeof(int)) +
         align256(size_t(std::max<int64_t>(s.acc_need, 1)) * sizeof(long long)) +
         align256(size_t(std::max<int64_t>(s.ex_need, 1)) * sizeof(int)) +
         align256(size_t(std::max<int64_t>(s.plane_need, 1))) + 512;
}

int plan_workspace_bytes(const BuildFn& build, size_t* bytes) {
  Arena a;
  a.sizing = true;
  Schedule s;
  TTR_TRY(build(a, s));
  *bytes = schedule_bytes(a, s);
  return TT_OK;
}

// Takes the schedule's own regions from the arena (sizes from the sizing pass).
static GemmDesc* bind_schedule_regions(Arena& a, const Schedule& probe, Schedule& s) {
  s.pbuf = a.take<double>(size_t(std::max<int64_t>(probe.pbuf_need, 1)));
  GemmDesc* d_descs = a.take<GemmDesc>(std::max<size_t>(probe.descs.size(), 1));
  s.cnt = a.take<int>(size_t(std::max<int64_t>(probe.cnt_need, 1)));
  s.d_copies = a.take<Copy3>(std::max<size_t>(probe.copies.size(), 1));
  s.dev_status = a.take<int>(1);
  s.acc = a.take<long long>(size_t(std::max<int64_t>(probe.acc_need, 1)));
  s.ex = a.take<int>(size_t(std::max<int64_t>(probe.ex_need, 1)));
  s.planes = a.take<uint8_t>(size_t(std::max<int64_t>(probe.plane_need, 1)));
  return d_descs;
}

// Zeroes what must start at zero on every run (counters, flags, emulated-GEMM
// accumulators and exponent tags).
static int reset_schedule_regions(const Schedule& probe, const Schedule& s, cudaStream_t st) {
  cudaError_t e = cudaMemsetAsync(s.cnt, 0, size_t(std::max<int64_t>(probe.cnt_need, 1)) * sizeof(int), st);
  if (e == cudaSuccess) e = cudaMemsetAsync(s.dev_status, 0, sizeof(int), st);
  if (e == cudaSuccess && probe.acc_need > 0)
    e = cudaMemsetAsync(s.acc, 0, size_t(probe.acc_need) * sizeof(long long), st);
  if (e == cudaSuccess && probe.ex_need > 0) e = cudaMemsetAsync(s.ex, 0, size_t(probe.ex_need) * sizeof(int), st);
  if (e != cudaSuccess) {
    set_error(std::string("counter reset: ") + cudaGetErrorString(e));
    return TT_ECUDA;
  }
  return TT_OK;
}

static std::atomic<int> g_inject{0};

int take_injected_status() { return g_inject.exchange(0); }

int status_code(int bits, const char* who) {
  if (bits == 0) return TT_OK;
  if (bits & DEV_TIMEOUT) {
    set_error(std::string(who) + ": a bounded device wait gave up (outputs are not valid)");
    return TT_ETIMEOUT;
  }
  if (bits & DEV_QR_FAIL) {
    set_error(std::string(who) + ": a thin QR above the Householder fallback limit could not orthogonalize a block");
    return TT_ESINGULAR;
  }
  set_error(std::string(who) + ": unknown device status " + std::to_string(bits));
  return TT_ECUDA;
}

// Enqueues the read-back of a run's device status word into *host (after the
// armed test injection, if any, overwrote the device word).
static int enqueue_status_read(int* dev, int* host, cudaStream_t st) {
  static thread_local int inj_src = 0;
  inj_src = take_injected_status();
  if (inj_src != 0) {
    cudaError_t e = cudaMemcpyAsync(dev, &inj_src, sizeof(int), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) {
      set_error(std::string("status injection: ") + cudaGetErrorString(e));
      return TT_ECUDA;
    }
  }
  TTR_CHECK_CUDA(cudaMemcpyAsync(host, dev, sizeof(int), cudaMemcpyDeviceToHost, st));
  return TT_OK;
}

int plan_execute(const BuildFn& build, void* workspace, size_t ws_bytes, cudaStream_t st, int* host_status) {
  size_t need = 0;
  Schedule probe;
  {
    Arena a;
    a.sizing = true;
    TTR_TRY(build(a, probe));
    need = schedule_bytes(a, probe);
  }
  void* ws = workspace;
  bool owned = false;
  if (ws == nullptr) {
    if (need > 0) {
      cudaError_t e = cudaMallocAsync(&ws, need, st);
      if (e != cudaSuccess) {
        set_error(std::string("workspace allocation of ") + std::to_string(need) + " bytes failed: " +
                  cudaGetErrorString(e));
        return TT_ENOMEM;
      }
      owned = true;
    }
  } else if (ws_bytes < need) {
    set_error("workspace too small: need " + std::to_string(need) + " bytes, got " + std::to_string(ws_bytes));
    return TT_ENOMEM;
  } else if ((reinterpret_cast<uintptr_t>(ws) & 255) != 0) {
    set_error("workspace must be 256-byte aligned");
    return TT_EINVAL;
  }
  Arena a;
  a.sizing = false;
  a.base = static_cast<char*>(ws);
  a.cap = need;
  Schedule s;
  GemmDesc* d_descs = bind_schedule_regions(a, probe, s);
  int rc = reset_schedule_regions(probe, s, st);
  if (rc == TT_OK) rc = build(a, s);
  if (rc == TT_OK && !s.descs.empty()) {
    cudaError_t e = cudaMemcpyAsync(d_descs, s.descs.data(), s.descs.size() * sizeof(GemmDesc),
                                    cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess) {
      set_error(std::string("descriptor upload: ") + cudaGetErrorString(e));
      rc = TT_ECUDA;
    }
  }
  if (rc == TT_OK && !s.copies.empty()) {
    cudaError_t e = cudaMemcpyAsync(s.d_copies, s.copies.data(), s.copies.size() * sizeof(Copy3),
                                    cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess) {
      set_error(std::string("copy descriptor upload: ") + cudaGetErrorString(e));
      rc = TT_ECUDA;
    }
  }
  for (size_t i = 0; rc == TT_OK && i < s.items.size(); ++i) rc = s.items[i](st, d_descs);
  if (rc == TT_OK && host_status) rc = enqueue_status_read(s.dev_status, host_status, st);
  if (owned) cudaFreeAsync(ws, st);
  return rc;
}

void plan_free(GraphPlan* gp) {
  if (gp->exec) cudaGraphExecDestroy(gp->exec);
  for (auto& q : gp->prof) {
    cudaEventDestroy(q.e0);
    cudaEventDestroy(q.e1);
  }
  gp->prof.clear();
  if (gp->ws) cudaFree(gp->ws);
  if (gp->pristine) cudaFree(gp->pristine);
  if (gp->seed_dev) cudaFree(gp->seed_dev);
  delete gp->sc;
  delete gp->probe;
  *gp = GraphPlan{};
}

int plan_prepare(const BuildFn& build, GraphPlan* gp) {
  *gp = GraphPlan{};
  auto fail = [&](int rc) {
    plan_free(gp);
    return rc;
  };
  gp->probe = new Schedule;
  size_t need = 0;
  {
    Arena a;
    a.sizing = true;
    const int rc = build(a, *gp->probe);
    if (rc != TT_OK) return fail(rc);
    need = schedule_bytes(a, *gp->probe);
  }
  if (cudaMalloc(&gp->ws, std::max<size_t>(need, 256)) != cudaSuccess ||
      cudaMalloc(&gp->seed_dev, 256) != cudaSuccess) {
    cudaGetLastError();
    set_error("plan: workspace allocation of " + std::to_string(need) + " bytes failed");
    return fail(TT_ENOMEM);
  }
  gp->ws_bytes = need;
  Arena a;
  a.sizing = false;
  a.base = static_cast<char*>(gp->ws);
  a.cap = need;
  gp->sc = new Schedule;
  Schedule& s = *gp->sc;
  gp->d_descs = bind_schedule_regions(a, *gp->probe, s);
  s.seed_dev = gp->seed_dev;
  int rc = build(a, s);
  if (rc != TT_OK) return fail(rc);
  // static tables and the pristine copies of the uploads, before any capture
  if (!s.descs.empty() &&
      cudaMemcpy(gp->d_descs, s.descs.data(), s.descs.size() * sizeof(GemmDesc), cudaMemcpyHostToDevice) !=
          cudaSuccess) {
    set_error("plan: descriptor upload failed");
    return fail(TT_ECUDA);
  }
  if (!s.copies.empty() &&
      cudaMemcpy(s.d_copies, s.copies.data(), s.copies.size() * sizeof(Copy3), cudaMemcpyHostToDevice) !=
          cudaSuccess) {
    set_error("plan: copy descriptor upload failed");
    return fail(TT_ECUDA);
  }
  if (s.upload_total > 0) {
    if (cudaMalloc(&gp->pristine, s.upload_total * sizeof(double)) != cudaSuccess) {
      cudaGetLastError();
      set_error("plan: upload buffer allocation failed");
      return fail(TT_ENOMEM);
    }
    size_t off = 0;
    for (const auto& v : s.host_keep) {
      if (!v.empty() &&
          cudaMemcpy(gp->pristine + off, v.data(), v.size() * sizeof(double), cudaMemcpyHostToDevice) != cudaSuccess) {
        set_error("plan: upload copy failed");
        return fail(TT_ECUDA);
      }
      off += v.size();
    }
    s.upload_dev = gp->pristine;
  }
  return TT_OK;
}

int plan_emit(GraphPlan& gp, const StageFn& prologue, const StageFn& epilogue, cudaStream_t cs) {
  int rc = TT_OK;
  if (prologue) rc = prologue(cs);
  if (rc == TT_OK) rc = reset_schedule_regions(*gp.probe, *gp.sc, cs);
  for (size_t i = 0; rc == TT_OK && i < gp.sc->items.size(); ++i) rc = gp.sc->items[i](cs, gp.d_descs);
  if (rc == TT_OK && epilogue) rc = epilogue(cs);
  return rc;
}

int capture_graph(const std::function<int(cudaStream_t)>& body, cudaGraphExec_t* exec, std::vector<ProfPair>* prof,
                  int64_t* kernels) {
  cudaStream_t cs;
  if (cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking) != cudaSuccess) {
    set_error("plan: capture stream creation failed");
    return TT_ECUDA;
  }
  prof_capture_begin(prof);
  cudaError_t ce = cudaStreamBeginCapture(cs, cudaStreamCaptureModeRelaxed);
  if (ce != cudaSuccess) {
    prof_capture_end();
    cudaStreamDestroy(cs);
    set_error(std::string("plan: begin capture: ") + cudaGetErrorString(ce));
    return TT_ECUDA;
  }
  int rc = body(cs);
  cudaGraph_t graph = nullptr;
  ce = cudaStreamEndCapture(cs, &graph);
  *kernels = prof_capture_end();
  cudaStreamDestroy(cs);
  if (rc == TT_OK && ce != cudaSuccess) {
    set_error(std::string("plan: end capture: ") + cudaGetErrorString(ce));
    rc = TT_ECUDA;
  }
  if (rc == TT_OK) {
    ce = cudaGraphInstantiate(exec, graph, 0);
    if (ce != cudaSuccess) {
      set_error(std::string("plan: graph instantiation: ") + cudaGetErrorString(ce));
      rc = TT_ECUDA;
    }
  }
  if (graph) cudaGraphDestroy(graph);
  cudaGetLastError();
  return rc;
}

int plan_capture(const BuildFn& build, const StageFn& prologue, const StageFn& epilogue, cudaStream_t st,
                 GraphPlan* gp) {
  TTR_TRY(plan_prepare(build, gp));
  GraphPlan* g = gp;
  const int rc = capture_graph([&](cudaStream_t cs) { return plan_emit(*g, prologue, epilogue, cs); }, &gp->exec,
                               &gp->prof, &gp->kernels);
  if (rc != TT_OK) {
    plan_free(gp);
    return rc;
  }
  (void)st;
  return TT_OK;
}

int plan_replay(GraphPlan& gp, cudaStream_t st) {
  TTR_CHECK_CUDA(cudaGraphLaunch(gp.exec, st));
  return TT_OK;
}

std::vector<int64_t> clamp_rank_vector(const std::vector<int64_t>& I, const int64_t* r) {
  const int N = int(I.size());
  std::vector<int64_t> ell(r, r + N + 1);
  ell[0] = 1;
  ell[N] = 1;
  for (int n = 1; n < N; ++n) ell[n] = std::min(std::max<int64_t>(ell[n], 1), ell[n - 1] * I[n - 1]);
  for (int n = N - 1; n >= 1; --n) ell[n] = std::min(ell[n], ell[n + 1] * I[n]);
  return ell;
}

int validate_sum(int32_t N, int32_t K, const int64_t* dims, const int64_t* ranks, const double* const* cores,
                        const double* coeffs, const int64_t* ells, bool need_cores, SumProblem* P) {
  if (N < 1 || K < 1 || !dims || !ranks || !ells || (need_cores && !cores)) {
    set_error("invalid arguments: need N >= 1, K >= 1 and non-null dims/ranks/ells/cores");
    return TT_EINVAL;
  }
  P->N = N;
  P->K = K;
  P->I.assign(dims, dims + N);
  P->R.assign(ranks, ranks + size_t(K) * (N + 1));
  for (int n = 0; n < N; ++n)
    if (P->I[n] < 1) { set_error("mode sizes must be positive"); return TT_EINVAL; }
  for (int j = 0; j < K; ++j) {
    if (P->r(j, 0) != 1 || P->r(j, N) != 1) { set_error("summand ranks must start and end with 1"); return TT_EINVAL; }
    for (int n = 0; n <= N; ++n)
      if (P->r(j, n) < 1) { set_error("ranks must be positive"); return TT_EINVAL; }
  }
  P->S.assign(N + 1, 0);
  P->off.assign(size_t(K) * (N + 1), 0);
  for (int n = 0; n <= N; ++n) {
    int64_t acc = 0;
    for (int j = 0; j < K; ++j) {
      P->off[size_t(j) * (N + 1) + n] = acc;
      acc += P->r(j, n);
    }
    P->S[n] = acc;
  }
  if (need_cores) {
    P->cores.assign(cores, cores + size_t(K) * N);
    for (auto* c : P->cores)
      if (!c) { set_error("null core pointer"); return TT_EINVAL; }
  } else {
    P->cores.assign(size_t(K) * N, nullptr);
  }
  P->coeffs.assign(K, 1.0);
  if (coeffs) P->coeffs.assign(coeffs, coeffs + K);
  // target ranks: l_0 = l_N = 1, l_n <= min(l_{n-1} I_n, I_{n+1} l_{n+1})
  P->ell.assign(ells, ells + N + 1);
  P->ell[0] = 1;
  P->ell[N] = 1;
  for (int n = 1; n < N; ++n)
    if (P->ell[n] < 1) { set_error("target ranks must be positive"); return TT_EINVAL; }
  for (int n = 1; n < N; ++n) P->ell[n] = std::min(P->ell[n], P->ell[n - 1] * P->I[n - 1]);
  for (int n = N - 1; n >= 1; --n) P->ell[n] = std::min(P->ell[n], P->ell[n + 1] * P->I[n]);
  for (int n = 1; n < N; ++n)
    if (P->ell[n] > TT_MAX_RANK) {
      set_error("target rank " + std::to_string(P->ell[n]) + " above the supported maximum " +
                std::to_string(TT_MAX_RANK));
      return TT_EUNSUPPORTED;
    }
  return TT_OK;
}

// ---------------------------------------------------------------------------
// Right-to-left truncation of a left-orthogonal TT held in caller buffers
// (padded layout (l_{n-1}, I_n, l_n)); decided ranks land in rk[0..N] (device).
struct TruncBufs {
  double* eps;      // [2]: eps, ||X||
  int64_t* rk;      // [N+1]
  double* Qt;       // max m*k
  double* Rb;       // k*k
  double* G1;
  double* G2;
  double* sig;
  double* tmp;      // max core size
};

// tol <= 0: no tolerance (ranks capped by max_rank only); max_rank <= 0: no cap.
int plan_truncation(Arena& ar, Schedule& sc, int N, const std::vector<int64_t>& I, const std::vector<int64_t>& ell,
                    double tol, double* const* out, int64_t** rk_out, int64_t max_rank) {
  TruncBufs b;
  int64_t qmax = 1, kmax = 1, cmax = 1;
  for (int n = 2; n <= N; ++n) {
    const int64_t m = I[n - 1] * ell[n], k = ell[n - 1];
    qmax = std::max(qmax, m * k);
    kmax = std::max(kmax, k);
  }
  for (int n = 1; n <= N; ++n) cmax = std::max(cmax, ell[n - 1] * I[n - 1] * ell[n]);
  b.eps = ar.take<double>(2);
  b.rk = ar.take<int64_t>(N + 1);
  b.Qt = ar.take<double>(qmax);
  b.Rb = ar.take<double>(kmax * kmax);
  b.G1 = ar.take<double>(kmax * kmax);
  b.G2 = ar.take<double>(kmax * kmax);
  b.sig = ar.take<double>(kmax);
  b.tmp = ar.take<double>(cmax);
  *rk_out = b.rk;
  std::vector<std::pair<int64_t, int>> shapes;
  for (int n = 2; n <= N; ++n) shapes.push_back({I[n - 1] * ell[n], int(ell[n - 1])});
  const QrPool pool = qr_pool_reserve(ar, shapes);
  double* sbig = ar.take<double>(std::max<size_t>(svd_scratch_doubles(int(kmax)), 1));

  {   // int64 ranks staged through a double-sized host buffer
    std::vector<int64_t> tmp(ell.begin(), ell.end());
    std::vector<double> raw(N + 1);
    std::memcpy(raw.data(), tmp.data(), sizeof(int64_t) * (N + 1));
    sc.upload(reinterpret_cast<double*>(b.rk), raw);
  }
  if (tol > 0.0)
    sc.add([=](cudaStream_t s) -> int {
      return norm_eps_launch(out[N - 1], ell[N - 1] * I[N - 1], tol, N, b.eps, s);
    });
  const double* epsp = tol > 0.0 ? b.eps : nullptr;
  for (int n = N; n >= 2; --n) {
    const int64_t m = I[n - 1] * ell[n], k = ell[n - 1];
    const int rcap = int(max_rank > 0 ? std::min<int64_t>(max_rank, k) : k);
    double* Xn = out[n - 1];
    double* Xp = out[n - 2];
    const int64_t mp = ell[n - 2] * I[n - 2];
    // With a tolerance the QR may certify that nothing can be cut at this bond
    // and apply the bond's update itself; the general steps below then skip.
    const QrBufs qb = qr_view(pool, m, int(k));
    QrCert cert{epsp, rcap, b.rk ? b.rk + (n - 1) : nullptr, Xn, Xp, mp};
    qr_plan(sc, qb, Xn, 1, m, b.Qt, k, 1, b.Rb, true, epsp ? &cert : nullptr);
    const int* skip = epsp ? qr_cert_flag(qb) : nullptr;
    sc.add([=](cudaStream_t s) -> int {
      return svd_trunc_launch(int(k), b.Rb, epsp, rcap, b.G1, b.G2, b.sig, b.rk + (n - 1), s, sbig, skip);
    });
    // new H(X_n) = (Q G1)^T : column-major m x k view of core n, and
    // V(X_{n-1}) G2 into scratch (copied over V(X_{n-1}) next): independent
    // products, one grouped launch
    GemmDesc g1 = gdesc(b.Qt, k, 1, b.G1, k, 1, Xn, 1, m, m, k, k);
    g1.skip = skip;
    GemmDesc g2 = gdesc(Xp, k, 1, b.G2, k, 1, b.tmp, k, 1, mp, k, k);
    g2.skip = skip;
    sc.gemm({g1, g2});
    sc.add([=](cudaStream_t s) -> int { return copy_if_launch(Xp, b.tmp, mp * k, skip, s); });
  }
  // compact every core to its decided ranks
  for (int n = 1; n <= N; ++n) {
    double* Xn = out[n - 1];
    const int64_t r0 = ell[n - 1], In = I[n - 1], r1 = ell[n];
    sc.add([=](cudaStream_t s) -> int {
      if (!Xn) return int(TT_OK);
      TTR_CHECK_CUDA(cudaMemcpyAsync(b.tmp, Xn, sizeof(double) * r0 * In * r1, cudaMemcpyDeviceToDevice, s));
      return compact_core_launch(b.tmp, Xn, r0, In, r1, b.rk + (n - 1), b.rk + n, s);
    });
  }
  return TT_OK;
}

// ---------------------------------------------------------------------------
// bf16 digits of the Algorithm 3 contractions in the mixed path (14 bits).
constexpr int kSketchDigits = 2;

int build_sum_rand(const SumProblem& P, const double* const* sketch_in, uint64_t seed, double tol, int digits,
                   double* const* out, Arena& ar, Schedule& sc, int64_t** rk_dev, size_t* coeff_off,
                   const double* coeff_dev, int sketch_digits) {
  // digits == 0: every contraction in FP64. Else every contraction runs on the
  // tensor cores (emulated GEMM): the core updates and projections with
  // `digits` bf16 digits, the partial contractions of Algorithm 3 with
  // sketch_digits (< 0: kSketchDigits). Their rounding errors only change the
  // sketch (the sketched core stays in the range of the unfolding), which is
  // harmless as long as the sum does not cancel: for a sum far smaller than
  // its summands (a Gram-Schmidt combination) or a fixed-sketch rounding that
  // is differentiated, callers pass sketch_digits = digits.
  const int dw = digits > 0 ? (sketch_digits < 0 ? kSketchDigits : sketch_digits) : 0;
  auto big = [&](std::vector<GemmDesc> g) {
    if (digits > 0) sc.gemm_tc(std::move(g), digits); else sc.gemm(std::move(g));
  };
  auto sketchy = [&](std::vector<GemmDesc> g) {
    if (dw > 0) sc.gemm_tc(std::move(g), dw); else sc.gemm(std::move(g));
  };
  const int N = P.N, K = P.K;
  const auto& I = P.I;
  const auto& S = P.S;
  const auto& ell = P.ell;
  auto In = [&](int n) { return I[n - 1]; };   // 1-based mode size

  // ---- workspace
  std::vector<double*> W(N + 1, nullptr);
  for (int n = 1; n <= N; ++n) W[n] = ar.take<double>(S[n] * ell[n]);
  int64_t zmax = 1, xmax = 1, ymax = 1, mmax = 1;
  for (int n = 2; n <= N; ++n) zmax = std::max(zmax, S[n - 1] * In(n) * ell[n]);
  for (int n = 1; n <= N; ++n) xmax = std::max(xmax, ell[n - 1] * In(n) * S[n]);
  for (int n = 1; n < N; ++n) ymax = std::max(ymax, ell[n - 1] * In(n) * ell[n]);
  for (int n = 0; n < N; ++n) mmax = std::max(mmax, ell[n] * S[n]);
  double* Z = ar.take<double>(zmax);
  double* X = ar.take<double>(xmax);
  double* Ys = ar.take<double>(ymax);
  double* Mb[2] = {ar.take<double>(mmax), ar.take<double>(mmax)};
  std::vector<const double*> sk(N + 1, nullptr);
  std::vector<double*> skw(N + 1, nullptr);
  for (int n = 2; n <= N; ++n) {
    if (sketch_in) {
      sk[n] = sketch_in[n - 1];
    } else {
      skw[n] = ar.take<double>(ell[n - 1] * In(n) * ell[n]);
      sk[n] = skw[n];
    }
  }
  std::vector<std::pair<int64_t, int>> shapes;
  for (int n = 1; n < N; ++n) shapes.push_back({ell[n - 1] * In(n), int(ell[n])});
  const QrPool pool = qr_pool_reserve(ar, shapes);

  // ---- set-up: counters, W_N = ones, M_0 = coefficients, sketch
  sc.add([=](cudaStream_t s) -> int { return fill_launch(W[N], S[N] * ell[N], 1.0, s); });
  if (coeff_dev) {
    // coefficients computed on the device by earlier steps of the schedule
    double* m0 = Mb[0];
    const int Kc = K;
    sc.add([m0, coeff_dev, Kc](cudaStream_t s) -> int {
      if (m0) TTR_CHECK_CUDA(cudaMemcpyAsync(m0, coeff_dev, sizeof(double) * Kc, cudaMemcpyDeviceToDevice, s));
      return int(TT_OK);
    });
  } else {
    const size_t off = sc.upload(Mb[0], P.coeffs);
    if (coeff_off) *coeff_off = off;
  }
  if (!sketch_in) {
    for (int n = 2; n <= N; ++n) {
      double* dst = skw[n];
      const int64_t a = ell[n - 1], b = In(n), c = ell[n];
      const Schedule* scp = &sc;
      sc.add([=](cudaStream_t s) -> int { return sketch_launch(dst, a, b, c, n - 1, seed, scp->seed_dev, s); });
    }
  }

  // ---- right-to-left partial contractions (Algorithm 3 for every summand).
  // The sketch is shared, so the second product of all summands is one GEMM of
  // the stacked H(Z^(j)) (S_{n-1} x I_n l_n) with H(Omega_n)^T.
  for (int n = N; n >= 2; --n) {
    std::vector<GemmDesc> ga;
    for (int j = 0; j < K; ++j) {
      const int64_t r0 = P.r(j, n - 1), r1 = P.r(j, n);
      double* Zj = Z ? Z + P.o(j, n - 1) * In(n) * ell[n] : nullptr;
      const double* Wj = W[n] ? W[n] + P.o(j, n) * ell[n] : nullptr;
      ga.push_back(gdesc(P.core(j, n), r1, 1, Wj, ell[n], 1, Zj, ell[n], 1, r0 * In(n), ell[n], r1));
    }
    sketchy(ga);
    sketchy({gdesc(Z, In(n) * ell[n], 1, sk[n], 1, In(n) * ell[n], W[n - 1], ell[n - 1], 1, S[n - 1], ell[n - 1],
                   In(n) * ell[n])});
  }

  // ---- left-to-right sweep
  for (int n = 1; n <= N; ++n) {
    const double* Mp = Mb[(n - 1) & 1];
    double* Mn = Mb[n & 1];
    std::vector<GemmDesc> gc;
    for (int j = 0; j < K; ++j) {
      const int64_t r0 = P.r(j, n - 1), r1 = P.r(j, n);
      if (digits > 0) {
        // one product per summand: rows (i, c) of H(Y^(j)_n)^T, columns a
        GemmDesc d = gdesc(P.core(j, n), 1, In(n) * r1, Mp ? Mp + P.o(j, n - 1) : nullptr, 1, S[n - 1],
                           X ? X + P.o(j, n) : nullptr, S[n], In(n) * S[n], In(n) * r1, ell[n - 1], r0);
        d.c_rdiv = r1;
        d.c_rs2 = 1;
        gc.push_back(d);
      } else {
        GemmDesc d = gdesc(Mp ? Mp + P.o(j, n - 1) : nullptr, S[n - 1], 1, P.core(j, n), In(n) * r1, 1,
                           X ? X + P.o(j, n) : nullptr, In(n) * S[n], 1, ell[n - 1], r1, r0);
        d.batch = int32_t(In(n));
        d.a_bs = 0;
        d.b_bs = r1;
        d.c_bs = S[n];
        gc.push_back(d);
      }
    }
    if (digits > 0) sc.gemm_tc(gc, digits); else sc.gemm(gc);
    double* dst = (n < N) ? Ys : out[N - 1];
    big({gdesc(X, S[n], 1, W[n], ell[n], 1, dst, ell[n], 1, ell[n - 1] * In(n), ell[n], S[n])});
    if (P.allreduce) {
      // summand-sharded rounding: the sketch (and the last core) of this rank's
      // summands is summed over the ranks before the QR, which every rank then
      // repeats on identical data
      const tt_allreduce_fn fn = P.allreduce;
      void* ctx = P.allreduce_ctx;
      const size_t cnt = size_t(ell[n - 1] * In(n) * ell[n]);
      sc.add([fn, ctx, dst, cnt](cudaStream_t s) -> int {
        if (!dst) return int(TT_OK);
        const int rc = fn(dst, cnt, static_cast<void*>(s), ctx);
        if (rc != 0) {
          set_error("the all-reduce callback of the sharded rounding returned " + std::to_string(rc));
          return TT_ECUDA;
        }
        return int(TT_OK);
      });
    }
    if (n == N) break;
    const int64_t m = ell[n - 1] * In(n), k = ell[n];
    double* Qn = out[n - 1];
    qr_plan(sc, qr_view(pool, m, int(k)), Ys, k, 1, Qn, k, 1, nullptr);
    big({gdesc(Qn, 1, k, X, S[n], 1, Mn, S[n], 1, k, S[n], m)});
  }

  if (tol > 0.0) TTR_TRY(plan_truncation(ar, sc, N, I, ell, tol, out, rk_dev, 0));
  return TT_OK;
}

// ---------------------------------------------------------------------------
// Many independent sum roundings (fixed ranks) rounded together: the same
// steps as build_sum_rand for every problem, but each step is ONE grouped
// launch over all problems (the Algorithm 3 products of every summand of every
// problem, then every sketch, every core update, ...), and the thin QRs of a
// step run as one batched Cholesky-QR chain. Problems of different orders are
// aligned at their last core in the right-to-left sweep and at their first core
// in the left-to-right sweep. seeds_dev: B device seeds (sketches drawn on the
// device); outs[b]: problem b's N_b output cores (l_{n-1} I_n l_n doubles).
int build_sum_rand_batch(const std::vector<SumProblem>& Ps, const uint64_t* seeds_dev, int digits, int qr_ctas,
                         const std::vector<std::vector<double*>>& outs, Arena& ar, Schedule& sc) {
  const int B = int(Ps.size());
  const int dw = digits > 0 ? kSketchDigits : 0;
  auto group = [&](std::vector<GemmDesc> g, int d) {
    if (g.empty()) return;
    if (d > 0) sc.gemm_tc(std::move(g), d); else sc.gemm(std::move(g));
  };
  struct Buf {
    std::vector<double*> W, skw;
    double *Z, *X, *Ys, *Mb[2];
    double *q0, *q1, *qg, *qr;    // thin-QR scratch, reused by every bond
  };
  std::vector<Buf> bf(B);
  int maxN = 0;
  int64_t wn_tot = 0, m0_tot = 0;
  std::vector<int64_t> mmax(B, 1);
  for (int b = 0; b < B; ++b) {
    const SumProblem& P = Ps[b];
    maxN = std::max(maxN, P.N);
    wn_tot += P.S[P.N] * P.ell[P.N];
    for (int n = 0; n < P.N; ++n) mmax[b] = std::max(mmax[b], P.ell[n] * P.S[n]);
    m0_tot += mmax[b];
  }
  // W_N (= ones) and M_0 (= the unit coefficients) of all problems live in two
  // contiguous blocks filled once
  double* wn_all = ar.take<double>(size_t(std::max<int64_t>(wn_tot, 1)));
  double* m0_all = ar.take<double>(size_t(std::max<int64_t>(m0_tot, 1)));
  int64_t wo = 0, mo = 0;
  std::vector<SketchJob> sj;
  int64_t sk_max = 1;
  for (int b = 0; b < B; ++b) {
    const SumProblem& P = Ps[b];
    const int N = P.N;
    Buf& f = bf[b];
    f.W.assign(N + 1, nullptr);
    for (int n = 1; n < N; ++n) f.W[n] = ar.take<double>(size_t(P.S[n] * P.ell[n]));
    f.W[N] = wn_all ? wn_all + wo : nullptr;
    wo += P.S[N] * P.ell[N];
    int64_t zmax = 1, xmax = 1, ymax = 1;
    for (int n = 2; n <= N; ++n) zmax = std::max(zmax, P.S[n - 1] * P.I[n - 1] * P.ell[n]);
    for (int n = 1; n <= N; ++n) xmax = std::max(xmax, P.ell[n - 1] * P.I[n - 1] * P.S[n]);
    for (int n = 1; n < N; ++n) ymax = std::max(ymax, P.ell[n - 1] * P.I[n - 1] * P.ell[n]);
    f.Z = ar.take<double>(size_t(zmax));
    f.X = ar.take<double>(size_t(xmax));
    f.Ys = ar.take<double>(size_t(ymax));
    f.Mb[0] = m0_all ? m0_all + mo : nullptr;
    mo += mmax[b];
    f.Mb[1] = ar.take<double>(size_t(mmax[b]));
    int64_t qm = 1, qgm = 1, qk = 1;
    for (int n = 1; n < N; ++n) {
      const int64_t m = P.ell[n - 1] * P.I[n - 1], k = P.ell[n];
      qm = std::max(qm, m * k);
      qgm = std::max(qgm, qr_batch_gram_doubles(m, int(k), qr_ctas));
      qk = std::max(qk, k * k);
    }
    f.q0 = ar.take<double>(size_t(qm));
    f.q1 = ar.take<double>(size_t(qm));
    f.qg = ar.take<double>(size_t(qgm));
    f.qr = ar.take<double>(size_t(qk));
    f.skw.assign(N + 1, nullptr);
    for (int n = 2; n <= N; ++n) {
      const int64_t a = P.ell[n - 1], c = P.ell[n], In = P.I[n - 1];
      f.skw[n] = ar.take<double>(size_t(a * In * c));
      sj.push_back(sketch_job(f.skw[n], a, In, c, n - 1, seeds_dev ? seeds_dev + b : nullptr));
      sk_max = std::max(sk_max, a * In * c);
    }
  }
  // ---- set-up: ones, all sketch cores in one launch
  {
    const int64_t a = wn_tot, c = m0_tot;
    sc.add([=](cudaStream_t s) -> int {
      TTR_TRY(fill_launch(wn_all, a, 1.0, s));
      return fill_launch(m0_all, c, 1.0, s);
    });
  }
  if (!sj.empty()) {
    const size_t bytes = sj.size() * sizeof(SketchJob);
    double* d_sj = ar.take<double>(size_t(ceil_div(int64_t(bytes), 8)));
    std::vector<double> raw(size_t(ceil_div(int64_t(bytes), 8)), 0.0);
    std::memcpy(raw.data(), sj.data(), bytes);
    sc.upload(d_sj, raw);
    const int nj = int(sj.size());
    sc.add([=](cudaStream_t s) -> int {
      return sketch_batch_launch(reinterpret_cast<const SketchJob*>(d_sj), nj, sk_max, s);
    });
  }
  // ---- right-to-left partial contractions, aligned at the last core
  for (int t = 0; t + 2 <= maxN; ++t) {
    std::vector<GemmDesc> ga, gb;
    for (int b = 0; b < B; ++b) {
      const SumProblem& P = Ps[b];
      const int n = P.N - t;
      if (n < 2) continue;
      const Buf& f = bf[b];
      const int64_t In = P.I[n - 1];
      for (int j = 0; j < P.K; ++j) {
        const int64_t r0 = P.r(j, n - 1), r1 = P.r(j, n);
        double* Zj = f.Z ? f.Z + P.o(j, n - 1) * In * P.ell[n] : nullptr;
        const double* Wj = f.W[n] ? f.W[n] + P.o(j, n) * P.ell[n] : nullptr;
        ga.push_back(gdesc(P.core(j, n), r1, 1, Wj, P.ell[n], 1, Zj, P.ell[n], 1, r0 * In, P.ell[n], r1));
      }
      gb.push_back(gdesc(f.Z, In * P.ell[n], 1, f.skw[n], 1, In * P.ell[n], f.W[n - 1], P.ell[n - 1], 1, P.S[n - 1],
                         P.ell[n - 1], In * P.ell[n]));
    }
    group(ga, dw);
    group(gb, dw);
  }
  // ---- left-to-right sweep, aligned at the first core
  for (int n = 1; n <= maxN; ++n) {
    std::vector<GemmDesc> gc, gd, ge;
    std::vector<QrBatchJob> qj;
    for (int b = 0; b < B; ++b) {
      const SumProblem& P = Ps[b];
      if (n > P.N) continue;
      const Buf& f = bf[b];
      const int N = P.N;
      const int64_t In = P.I[n - 1];
      const double* Mp = f.Mb[(n - 1) & 1];
      double* Mn = f.Mb[n & 1];
      for (int j = 0; j < P.K; ++j) {
        const int64_t r0 = P.r(j, n - 1), r1 = P.r(j, n);
        if (digits > 0) {
          GemmDesc d = gdesc(P.core(j, n), 1, In * r1, Mp ? Mp + P.o(j, n - 1) : nullptr, 1, P.S[n - 1],
                             f.X ? f.X + P.o(j, n) : nullptr, P.S[n], In * P.S[n], In * r1, P.ell[n - 1], r0);
          d.c_rdiv = r1;
          d.c_rs2 = 1;
          gc.push_back(d);
        } else {
          GemmDesc d = gdesc(Mp ? Mp + P.o(j, n - 1) : nullptr, P.S[n - 1], 1, P.core(j, n), In * r1, 1,
                             f.X ? f.X + P.o(j, n) : nullptr, In * P.S[n], 1, P.ell[n - 1], r1, r0);
          d.batch = int32_t(In);
          d.a_bs = 0;
          d.b_bs = r1;
          d.c_bs = P.S[n];
          gc.push_back(d);
        }
      }
      double* dst = (n < N) ? f.Ys : outs[b][N - 1];
      gd.push_back(gdesc(f.X, P.S[n], 1, f.W[n], P.ell[n], 1, dst, P.ell[n], 1, P.ell[n - 1] * In, P.ell[n], P.S[n]));
      if (n == N) continue;
      const int64_t m = P.ell[n - 1] * In, k = P.ell[n];
      double* Qn = outs[b][n - 1];
      QrBatchJob q{f.Ys, k, 1, Qn, k, 1, m, int(k)};
      q.has_scratch = true;
      q.buf0 = f.q0;
      q.buf1 = f.q1;
      q.gpart = f.qg;
      q.rinv = f.qr;
      qj.push_back(q);
      ge.push_back(gdesc(Qn, 1, k, f.X, P.S[n], 1, Mn, P.S[n], 1, k, P.S[n], m));
    }
    group(gc, digits);
    group(gd, digits);
    if (!qj.empty()) TTR_TRY(qr_batch_plan(ar, sc, qj, qr_ctas));
    group(ge, digits);
  }
  return TT_OK;
}

// Digits of the mixed path. Errors of the Algorithm 3 contractions compound over
// the N-step recursion and enter the kept subspace directly when the sum is
// redundant, so the per-product target is 1e-3 tol / N (1e-7 / N in fixed-rank
// mode, an FP32-class target).
int mixed_digits(double tol, int N) {
  const double base = tol > 0.0 ? 1e-3 * tol : 1e-7;
  return tc_digits_for_accuracy(base / double(std::max(N, 1)));
}

}  // namespace ttr

using namespace ttr;

extern "C" {

const char* tt_version(void) { return "ttround-gb300 0.1 (sm_103a)"; }
const char* tt_last_error(void) { return g_err.c_str(); }

int tt_sketch_gaussian(int32_t N, const int64_t* dims, const int64_t* ells, uint64_t seed, double* const* out,
                       void* stream) {
  if (N < 1 || !dims || !ells || !out) {
    set_error("tt_sketch_gaussian: invalid arguments");
    return TT_EINVAL;
  }
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  for (int n = 1; n <= N; ++n) {
    if (dims[n - 1] < 1 || ells[n - 1] < 1 || ells[n] < 1 || !out[n - 1]) {
      set_error("tt_sketch_gaussian: invalid sizes or null output");
      return TT_EINVAL;
    }
  }
  for (int n = 1; n <= N; ++n) TTR_TRY(sketch_launch(out[n - 1], ells[n - 1], dims[n - 1], ells[n], n - 1, seed, nullptr, s));
  return TT_OK;
}

int tt_mixed_digits(double tol, int32_t N) { return ttr::mixed_digits(tol, N); }

void tt_debug_inject_device_status(int32_t bits) { g_inject.store(int(bits)); }

int tt_set_qr_mode(int32_t mode) {
  if (set_qr_mode(mode) != TT_OK) {
    set_error("tt_set_qr_mode: mode must be 0 (auto), 1 (multi-launch chain) or 2 (Householder fallback)");
    return TT_EINVAL;
  }
  return TT_OK;
}

int tt_set_gemm_mode(int32_t mode) {
  if (set_gemm_mode(mode) != TT_OK) {
    set_error("tt_set_gemm_mode: mode must be 0 (automatic), 1 (three-pass) or 2 (fused)");
    return TT_EINVAL;
  }
  return TT_OK;
}

int tt_tsqr_fallback_runs(int64_t* runs) {
  if (!runs) {
    set_error("tt_tsqr_fallback_runs: null output");
    return TT_EINVAL;
  }
  long long v = 0;
  TTR_TRY(tsqr_fallback_runs(&v));
  *runs = int64_t(v);
  return TT_OK;
}

__attribute__((visibility("hidden"))) int sum_rand_common(int32_t N, int32_t K, const int64_t* dims,
                                                         const int64_t* ranks,
                           const double* const* cores, const double* coeffs, const int64_t* ells,
                           const double* const* sketch, uint64_t seed, double tol, int32_t precision,
                           double* const* out, int64_t* out_ranks, void* workspace, size_t ws_bytes,
                           void* stream, size_t* size_only) {
  SumProblem P;
  TTR_TRY(validate_sum(N, K, dims, ranks, cores, coeffs, ells, size_only == nullptr, &P));
  if (precision != TT_PREC_FP64 && precision != TT_PREC_MIXED && precision != TT_PREC_MIXED_FULL) {
    set_error("unknown precision mode");
    return TT_EINVAL;
  }
  if (size_only == nullptr) {
    P.allreduce = g_allreduce;
    P.allreduce_ctx = g_allreduce_ctx;
  }
  const int digits = (precision != TT_PREC_FP64) ? mixed_digits(tol, N) : 0;
  const int sketch_digits = (precision == TT_PREC_MIXED_FULL) ? digits : -1;
  if (size_only == nullptr) {
    if (!out || !out_ranks) { set_error("null output arrays"); return TT_EINVAL; }
    for (int n = 0; n < N; ++n)
      if (!out[n]) { set_error("null output core pointer"); return TT_EINVAL; }
    if (sketch)
      for (int n = 1; n < N; ++n)
        if (!sketch[n]) { set_error("null sketch core pointer"); return TT_EINVAL; }
  }
  int64_t* rk_dev = nullptr;
  std::vector<double*> out_v(N, nullptr);
  if (out) out_v.assign(out, out + N);
  BuildFn build = [&](Arena& ar, Schedule& sc) {
    return build_sum_rand(P, sketch, seed, tol, digits, out_v.data(), ar, sc, &rk_dev, nullptr, nullptr,
                          sketch_digits);
  };
  if (size_only) return plan_workspace_bytes(build, size_only);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  int dstat = 0;
  std::vector<int64_t> rk(N + 1);
  // the ranks are read by a copy enqueued inside the build (before a
  // stream-ordered free of an owned workspace)
  BuildFn build_rk = [&](Arena& ar, Schedule& sc) {
    TTR_TRY(build(ar, sc));
    if (tol > 0.0) {
      int64_t* rkd = rk_dev;
      int64_t* rkh = rk.data();
      sc.add([rkd, rkh, N](cudaStream_t st) -> int {
        if (rkd) TTR_CHECK_CUDA(cudaMemcpyAsync(rkh, rkd, sizeof(int64_t) * (N + 1), cudaMemcpyDeviceToHost, st));
        return int(TT_OK);
      });
    }
    return int(TT_OK);
  };
  TTR_TRY(plan_execute(build_rk, workspace, ws_bytes, s, &dstat));
  TTR_CHECK_CUDA(cudaStreamSynchronize(s));
  TTR_TRY(status_code(dstat, "tt_round_sum_rand"));
  for (int n = 0; n <= N; ++n) out_ranks[n] = tol > 0.0 ? rk[n] : P.ell[n];
  return TT_OK;
}

static int truncate_common(int32_t N, const int64_t* dims, const int64_t* ranks, double* const* cores, double tol,
                           int64_t max_rank, int64_t* out_ranks, void* workspace, size_t ws_bytes, void* stream,
                           size_t* size_only) {
  if (N < 1 || !dims || !ranks || (!size_only && (!cores || !out_ranks))) {
    set_error("tt_truncate_lorth: invalid arguments");
    return TT_EINVAL;
  }
  if (tol <= 0.0 && max_rank <= 0) {
    set_error("tt_truncate_lorth: needs tol > 0 or max_rank > 0");
    return TT_EINVAL;
  }
  std::vector<int64_t> I(dims, dims + N), r(ranks, ranks + N + 1);
  for (int n = 0; n < N; ++n)
    if (I[n] < 1) { set_error("tt_truncate_lorth: mode sizes must be positive"); return TT_EINVAL; }
  for (int n = 0; n <= N; ++n)
    if (r[n] < 1) { set_error("tt_truncate_lorth: ranks must be positive"); return TT_EINVAL; }
  if (r[0] != 1 || r[N] != 1 || clamp_rank_vector(I, r.data()) != r) {
    set_error("tt_truncate_lorth: ranks must start and end with 1 and satisfy r_{n-1} <= I_n r_n, r_n <= r_{n-1} I_n");
    return TT_EINVAL;
  }
  for (int n = 1; n < N; ++n)
    if (r[n] > TT_MAX_RANK) { set_error("tt_truncate_lorth: rank above 1024"); return TT_EUNSUPPORTED; }
  std::vector<double*> cv(N, nullptr);
  if (cores) {
    cv.assign(cores, cores + N);
    for (auto* c : cv)
      if (!c) { set_error("tt_truncate_lorth: null core pointer"); return TT_EINVAL; }
  }
  int64_t* rk_dev = nullptr;
  std::vector<int64_t> rk(N + 1);
  BuildFn build = [&](Arena& ar, Schedule& sc) {
    if (N == 1) return int(TT_OK);
    TTR_TRY(plan_truncation(ar, sc, N, I, r, tol, cv.data(), &rk_dev, max_rank));
    int64_t* rkd = rk_dev;
    int64_t* rkh = rk.data();
    sc.add([rkd, rkh, N](cudaStream_t st) -> int {
      if (rkd) TTR_CHECK_CUDA(cudaMemcpyAsync(rkh, rkd, sizeof(int64_t) * (N + 1), cudaMemcpyDeviceToHost, st));
      return int(TT_OK);
    });
    return int(TT_OK);
  };
  if (size_only) return plan_workspace_bytes(build, size_only);
  if (N == 1) {
    out_ranks[0] = out_ranks[1] = 1;
    return TT_OK;
  }
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  int dstat = 0;
  TTR_TRY(plan_execute(build, workspace, ws_bytes, s, &dstat));
  TTR_CHECK_CUDA(cudaStreamSynchronize(s));
  TTR_TRY(status_code(dstat, "tt_truncate_lorth"));
  for (int n = 0; n <= N; ++n) out_ranks[n] = rk[n];
  return TT_OK;
}

int tt_round_sum_rand_sharded(int32_t N, int32_t K, const int64_t* dims, const int64_t* ranks,
                              const double* const* cores, const double* coeffs, const int64_t* ells,
                              const double* const* sketch, uint64_t seed, double tol, int32_t precision,
                              double* const* out, int64_t* out_ranks, void* workspace, size_t workspace_bytes,
                              void* stream, tt_allreduce_fn allreduce, void* ctx) {
  if (!allreduce) {
    set_error("tt_round_sum_rand_sharded: null all-reduce callback");
    return TT_EINVAL;
  }
  g_allreduce = allreduce;
  g_allreduce_ctx = ctx;
  const int rc = sum_rand_common(N, K, dims, ranks, cores, coeffs, ells, sketch, seed, tol, precision, out,
                                 out_ranks, workspace, workspace_bytes, stream, nullptr);
  g_allreduce = nullptr;
  g_allreduce_ctx = nullptr;
  return rc;
}

int tt_round_sum_rand(int32_t N, int32_t K, const int64_t* dims, const int64_t* ranks, const double* const* cores,
                      const double* coeffs, const int64_t* ells, const double* const* sketch, uint64_t seed,
                      double tol, int32_t precision, double* const* out, int64_t* out_ranks, void* workspace,
                      size_t workspace_bytes, void* stream) {
  return sum_rand_common(N, K, dims, ranks, cores, coeffs, ells, sketch, seed, tol, precision, out, out_ranks,
                         workspace, workspace_bytes, stream, nullptr);
}

size_t tt_round_sum_rand_workspace(int32_t N, int32_t K, const int64_t* dims, const int64_t* ranks,
                                   const int64_t* ells, double tol, int32_t precision) {
  size_t bytes = 0;
  if (sum_rand_common(N, K, dims, ranks, nullptr, nullptr, ells, nullptr, 0, tol, precision, nullptr, nullptr,
                      nullptr, 0, nullptr, &bytes) != TT_OK)
    return 0;
  return bytes;
}

int tt_truncate_lorth(int32_t N, const int64_t* dims, const int64_t* ranks, double* const* cores, double tol,
                      int64_t max_rank, int64_t* out_ranks, void* workspace, size_t workspace_bytes, void* stream) {
  return truncate_common(N, dims, ranks, cores, tol, max_rank, out_ranks, workspace, workspace_bytes, stream,
                         nullptr);
}

size_t tt_truncate_lorth_workspace(int32_t N, const int64_t* dims, const int64_t* ranks, double tol,
                                   int64_t max_rank) {
  size_t b = 0;
  if (truncate_common(N, dims, ranks, nullptr, tol, max_rank, nullptr, nullptr, 0, nullptr, &b) != TT_OK) return 0;
  return b;
}

// float32 storage at the boundary: cores (and sketch) converted to float64 on
// the device, the rounding of tt_round_rand, the result converted back.
static int rand_f32_common(int32_t N, const int64_t* dims, const int64_t* ranks, const float* const* cores,
                           const int64_t* ells, const float* const* sketch, uint64_t seed, double tol,
                           int32_t precision, float* const* out, int64_t* out_ranks, void* workspace,
                           size_t ws_bytes, void* stream, size_t* size_only) {
  SumProblem P;
  TTR_TRY(validate_sum(N, 1, dims, ranks, nullptr, nullptr, ells, false, &P));
  if (precision != TT_PREC_FP64 && precision != TT_PREC_MIXED && precision != TT_PREC_MIXED_FULL) {
    set_error("unknown precision mode");
    return TT_EINVAL;
  }
  if (!size_only) {
    if (!cores || !out || !out_ranks) { set_error("null core or output arrays"); return TT_EINVAL; }
    for (int n = 0; n < N; ++n)
      if (!cores[n] || !out[n]) { set_error("null core pointer"); return TT_EINVAL; }
    if (sketch)
      for (int n = 1; n < N; ++n)
        if (!sketch[n]) { set_error("null sketch core pointer"); return TT_EINVAL; }
  }
  const int digits = (precision != TT_PREC_FP64) ? mixed_digits(tol, N) : 0;
  int64_t* rk_dev = nullptr;
  std::vector<int64_t> rk(N + 1);
  BuildFn build = [&](Arena& ar, Schedule& sc) {
    SumProblem Q = P;
    std::vector<double*> Yd(N), Od(N, nullptr), Xo(N);
    std::vector<int64_t> ny(N), nx(N);
    for (int n = 0; n < N; ++n) {
      ny[n] = P.R[n] * P.I[n] * P.R[n + 1];
      nx[n] = P.ell[n] * P.I[n] * P.ell[n + 1];
      Yd[n] = ar.take<double>(ny[n]);
      Xo[n] = ar.take<double>(nx[n]);
      if (n > 0) Od[n] = ar.take<double>(nx[n]);   // sized whether or not a sketch is given
      Q.cores[n] = Yd[n];
    }
    for (int n = 0; n < N; ++n) {
      const float* yc = size_only ? nullptr : cores[n];
      const float* oc = (size_only || !sketch || n == 0) ? nullptr : sketch[n];
      double *yd = Yd[n], *od = Od[n];
      const int64_t a = ny[n], b = nx[n];
      sc.add([=](cudaStream_t s) -> int {
        TTR_TRY(cvt_f32_f64_launch(yc, yd, a, s));
        return cvt_f32_f64_launch(oc, od, b, s);
      });
    }
    std::vector<const double*> Oc(Od.begin(), Od.end());
    // the fixed-sketch rounding itself (what its adjoint differentiates): full digits in Algorithm 3 too
    TTR_TRY(build_sum_rand(Q, sketch ? Oc.data() : nullptr, seed, tol, digits, Xo.data(), ar, sc, &rk_dev, nullptr,
                           nullptr, digits));
    for (int n = 0; n < N; ++n) {
      float* o = size_only ? nullptr : out[n];
      const double* x = Xo[n];
      const int64_t b = nx[n];
      sc.add([=](cudaStream_t s) -> int { return cvt_f64_f32_launch(x, o, b, s); });
    }
    if (tol > 0.0) {
      int64_t* rkd = rk_dev;
      int64_t* rkh = rk.data();
      sc.add([rkd, rkh, N](cudaStream_t st) -> int {
        if (rkd) TTR_CHECK_CUDA(cudaMemcpyAsync(rkh, rkd, sizeof(int64_t) * (N + 1), cudaMemcpyDeviceToHost, st));
        return int(TT_OK);
      });
    }
    return int(TT_OK);
  };
  if (size_only) return plan_workspace_bytes(build, size_only);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  int dstat = 0;
  TTR_TRY(plan_execute(build, workspace, ws_bytes, s, &dstat));
  TTR_CHECK_CUDA(cudaStreamSynchronize(s));
  TTR_TRY(status_code(dstat, "tt_round_rand_f32"));
  for (int n = 0; n <= N; ++n) out_ranks[n] = tol > 0.0 ? rk[n] : P.ell[n];
  return TT_OK;
}

int tt_round_rand_f32(int32_t N, const int64_t* dims, const int64_t* ranks, const float* const* cores,
                      const int64_t* ells, const float* const* sketch, uint64_t seed, double tol, int32_t precision,
                      float* const* out, int64_t* out_ranks, void* workspace, size_t workspace_bytes, void* stream) {
  return rand_f32_common(N, dims, ranks, cores, ells, sketch, seed, tol, precision, out, out_ranks, workspace,
                         workspace_bytes, stream, nullptr);
}

size_t tt_round_rand_f32_workspace(int32_t N, const int64_t* dims, const int64_t* ranks, const int64_t* ells,
                                   double tol, int32_t precision) {
  size_t b = 0;
  if (rand_f32_common(N, dims, ranks, nullptr, ells, nullptr, 0, tol, precision, nullptr, nullptr, nullptr, 0,
                      nullptr, &b) != TT_OK)
    return 0;
  return b;
}

int tt_round_rand(int32_t N, const int64_t* dims, const int64_t* ranks, const double* const* cores,
                  const int64_t* ells, const double* const* sketch, uint64_t seed, double tol, int32_t precision,
                  double* const* out, int64_t* out_ranks, void* workspace, size_t workspace_bytes, void* stream) {
  return sum_rand_common(N, 1, dims, ranks, cores, nullptr, ells, sketch, seed, tol, precision, out, out_ranks,
                         workspace, workspace_bytes, stream, nullptr);
}

}  // extern "C"

// Deterministic TT-rounding (Algorithm 1 + Algorithm 2, Section 2.3) and
// Orthogonalize-then-Randomize (Algorithm 4, Section 3.1), both on the formed
// TT-sum of Section 2.1 (first cores side by side, middle cores block diagonal,
// last cores stacked; coefficients folded into the first cores).
//
// Steps on the device, all stream-ordered:
//   form the block cores (one batched copy per core);
//   if S_1 > I_1, fold core 1 into core 2 (core 1 becomes the identity), so that
//     every vertical unfolding met later is tall;
//   Algorithm 1, n = N..2: thin QR of H(X_n)^T (Cholesky QR), H(X_n) := Q^T,
//     V(X_{n-1}) := V(X_{n-1}) R^T; a wide H(X_n)^T (I_n R_n < R_{n-1}) is folded
//     into core n-1 instead (core n becomes the identity);
//   Algorithm 2 (deterministic): eps = tol ||X_1|| / sqrt(N-1); n = 1..N-1: thin
//     QR of V(X_n), eps-rule SVD of R (certificate or Jacobi), V(X_n) := Q U,
//     H(X_{n+1}) := S V^T H(X_{n+1}); ranks are decided on the device and the
//     cores are compacted at the end;
//   Algorithm 4 (randomized): n = 1..N-1: Y_n = V(X_n) Omega_n, thin QR,
//     M_n = Q^T V(X_n), H(X_{n+1}) := M_n H(X_{n+1}).
#include <algorithm>
#include <cmath>
#include <cstring>
#include <string>

#include "plan.cuh"
#include "prof.cuh"
#include "qr.cuh"

namespace ttr {

namespace {

__global__ void eye_kernel(double* dst, int64_t n) {
  for (int64_t e = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; e < n * n; e += int64_t(gridDim.x) * blockDim.x)
    dst[e] = ((e / n) == (e % n)) ? 1.0 : 0.0;
}

int eye_launch(double* dst, int64_t n, cudaStream_t s) {
  const int64_t tot = n * n;
  const unsigned g = unsigned(std::max<int64_t>(1, std::min<int64_t>(ceil_div(tot, 256), 4096)));
  TTR_PREFER_SHARED(eye_kernel);
  eye_kernel<<<g, 256, 0, s>>>(dst, n);
  TTR_CHECK_LAUNCH();
  prof_count_launch(1);
  return TT_OK;
}

struct DetProblem {
  int N = 0, K = 0;
  std::vector<int64_t> I, R, S, off;
  std::vector<const double*> cores;
  std::vector<double> coeffs;
  int64_t r(int j, int n) const { return R[size_t(j) * (N + 1) + n]; }
  int64_t o(int j, int n) const { return off[size_t(j) * (N + 1) + n]; }
  const double* core(int j, int n) const { return cores[size_t(j) * N + (n - 1)]; }
};

int validate_det(int32_t N, int32_t K, const int64_t* dims, const int64_t* ranks, const double* const* cores,
                 const double* coeffs, bool need_cores, DetProblem* P) {
  if (N < 2 || K < 1 || !dims || !ranks || (need_cores && !cores)) {
    set_error("invalid arguments: need N >= 2, K >= 1 and non-null dims/ranks/cores");
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
    P->S[n] = (n == 0 || n == N) ? 1 : acc;
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
  return TT_OK;
}

// Capacity (doubles) of the formed core n (1-based) of the sum.
int64_t formed_capacity(const DetProblem& P, int n) { return P.S[n - 1] * P.I[n - 1] * P.S[n]; }

// Forms the block cores into X[1..N] and runs Algorithm 1; returns the ranks
// of the right-orthogonal result in Rp[0..N].
int plan_formed_orth(const DetProblem& P, Arena& ar, Schedule& sc, const std::vector<double*>& X,
                     std::vector<int64_t>& Rp, double* tmp, int64_t tmp_cap, double* qtmp,
                     const QrPool* pool, double* rbuf) {
  const int N = P.N, K = P.K;
  auto In = [&](int n) { return P.I[n - 1]; };
  // ---- formed sum (Section 2.1)
  for (int n = 1; n <= N; ++n) {
    const int64_t S0 = P.S[n - 1], S1 = P.S[n];
    double* dst = X[n];
    sc.add([=](cudaStream_t s) -> int { return fill_launch(dst, S0 * In(n) * S1, 0.0, s); });
    std::vector<Copy3> cp;
    for (int j = 0; j < K; ++j) {
      const int64_t r0 = P.r(j, n - 1), r1 = P.r(j, n);
      const int64_t a0 = (n == 1) ? 0 : P.o(j, n - 1);
      const int64_t b0 = (n == N) ? 0 : P.o(j, n);
      Copy3 c{};
      c.src = P.core(j, n);
      c.dst = dst ? dst + (a0 * In(n)) * S1 + b0 : nullptr;
      c.n0 = r0; c.n1 = In(n); c.n2 = r1;
      c.s0 = In(n) * r1; c.s1 = r1; c.s2 = 1;
      c.d0 = In(n) * S1; c.d1 = S1; c.d2 = 1;
      c.scale = (n == 1) ? P.coeffs[j] : 1.0;
      cp.push_back(c);
    }
    sc.copy3(cp);
  }
  std::vector<int64_t> R(P.S.begin(), P.S.end());
  // ---- fold core 1 into core 2 when S_1 > I_1 (keeps every vertical unfolding tall)
  if (R[1] > In(1)) {
    const int64_t I1 = In(1), I2 = In(2), k = R[1], r2 = R[2];
    // new H(X_2) = V(X_1) H(X_2): (I1 x k)(k x I2 r2)
    sc.gemm({gdesc(X[1], k, 1, X[2], I2 * r2, 1, tmp, I2 * r2, 1, I1, I2 * r2, k)});
    double* d2 = X[2];
    double* d1 = X[1];
    sc.add([=](cudaStream_t s) -> int {
      if (!d2) return int(TT_OK);
      TTR_CHECK_CUDA(cudaMemcpyAsync(d2, tmp, sizeof(double) * I1 * I2 * r2, cudaMemcpyDeviceToDevice, s));
      return eye_launch(d1, I1, s);
    });
    R[1] = I1;
  }
  // ---- Algorithm 1
  Rp.assign(N + 1, 1);
  Rp[0] = 1;
  Rp[N] = 1;
  int64_t qmax = 1;
  for (int n = N; n >= 2; --n) {
    const int64_t m = In(n) * Rp[n], k = R[n - 1];
    if (m >= k) qmax = std::max(qmax, m * k);
    Rp[n - 1] = std::min(k, m);
  }
  (void)qmax;
  for (int n = N; n >= 2; --n) {
    const int64_t m = In(n) * Rp[n], k = R[n - 1];
    const int64_t left = (n - 1 == 1) ? 1 : R[n - 2];
    const int64_t mp = left * In(n - 1);
    double* Xn = X[n];
    double* Xp = X[n - 1];
    if (m >= k) {
      QrBufs qb = qr_view(*pool, m, int(k));
      double* Rb = rbuf;
      qr_plan(sc, qb, Xn, 1, m, qtmp, k, 1, Rb);
      // H(X_n) := Q^T, i.e. core n is Q as a column-major m x k array
      sc.copy3({Copy3{qtmp, Xn, 1, m, k, 0, k, 1, 0, 1, m, 1.0, 0}});
      // V(X_{n-1}) := V(X_{n-1}) R^T
      sc.gemm({gdesc(Xp, k, 1, Rb, 1, k, tmp, k, 1, mp, k, k)});
      sc.add([=](cudaStream_t s) -> int {
        if (!Xp) return int(TT_OK);
        TTR_CHECK_CUDA(cudaMemcpyAsync(Xp, tmp, sizeof(double) * mp * k, cudaMemcpyDeviceToDevice, s));
        return int(TT_OK);
      });
    } else {
      // wide: fold core n into core n-1, core n becomes the identity (H(X_n) = I_m)
      sc.gemm({gdesc(Xp, k, 1, Xn, m, 1, tmp, m, 1, mp, m, k)});
      sc.add([=](cudaStream_t s) -> int {
        if (!Xp) return int(TT_OK);
        TTR_CHECK_CUDA(cudaMemcpyAsync(Xp, tmp, sizeof(double) * mp * m, cudaMemcpyDeviceToDevice, s));
        return eye_launch(Xn, m, s);
      });
    }
    R[n - 1] = Rp[n - 1];
  }
  return TT_OK;
}

// Ranks after the optional fold of core 1 (R) and after Algorithm 1 (Rp).
void det_static_ranks(const DetProblem& P, std::vector<int64_t>* R, std::vector<int64_t>* Rp) {
  const int N = P.N;
  R->assign(P.S.begin(), P.S.end());
  if ((*R)[1] > P.I[0]) (*R)[1] = P.I[0];
  Rp->assign(N + 1, 1);
  for (int n = N; n >= 2; --n) (*Rp)[n - 1] = std::min((*R)[n - 1], P.I[n - 1] * (*Rp)[n]);
}

void orth_shapes(const DetProblem& P, std::vector<std::pair<int64_t, int>>* shapes, int64_t* kmax) {
  std::vector<int64_t> R, Rp;
  det_static_ranks(P, &R, &Rp);
  for (int n = P.N; n >= 2; --n) {
    const int64_t m = P.I[n - 1] * Rp[n], k = R[n - 1];
    if (m >= k) {
      shapes->push_back({m, int(k)});
      *kmax = std::max(*kmax, k);
    }
  }
}

int64_t det_tmp_doubles(const DetProblem& P) {
  int64_t t = 1;
  for (int n = 1; n <= P.N; ++n) t = std::max(t, formed_capacity(P, n));
  return t;
}

}  // namespace

// -------------------------------------------------------------------------------------------
int build_det(const DetProblem& P, double tol, int64_t max_rank, double* const* out, Arena& ar, Schedule& sc,
              int64_t** rk_dev) {
  const int N = P.N;
  auto In = [&](int n) { return P.I[n - 1]; };
  const int64_t tcap = det_tmp_doubles(P);
  double* tmp = ar.take<double>(tcap);
  double* qtmp = ar.take<double>(tcap);
  std::vector<double*> X(N + 1, nullptr);
  for (int n = 1; n <= N; ++n) X[n] = out[n - 1];
  std::vector<int64_t> Rs, Rp0;
  det_static_ranks(P, &Rs, &Rp0);
  std::vector<std::pair<int64_t, int>> shapes;
  int64_t kq = 1;
  orth_shapes(P, &shapes, &kq);
  for (int n = 1; n < N; ++n) {
    shapes.push_back({Rp0[n - 1] * In(n), int(Rp0[n])});
    kq = std::max(kq, Rp0[n]);
  }
  const QrPool pool = qr_pool_reserve(ar, shapes);
  double* rbuf = ar.take<double>(kq * kq);
  std::vector<int64_t> Rp;
  TTR_TRY(plan_formed_orth(P, ar, sc, X, Rp, tmp, tcap, qtmp, &pool, rbuf));
  for (int n = 1; n < N; ++n)
    if (Rp[n - 1] * In(n) < Rp[n]) {
      set_error("deterministic rounding: a vertical unfolding would be wide at bond " + std::to_string(n));
      return TT_EUNSUPPORTED;
    }
  int64_t kmax = 1;
  for (int n = 1; n < N; ++n) kmax = std::max(kmax, Rp[n]);
  double* eps = ar.take<double>(2);
  int64_t* rk = ar.take<int64_t>(N + 1);
  double* G1 = ar.take<double>(kmax * kmax);
  double* G2 = ar.take<double>(kmax * kmax);
  double* sig = ar.take<double>(kmax);
  double* sbig = ar.take<double>(std::max<size_t>(svd_scratch_doubles(int(kmax)), 1));
  *rk_dev = rk;
  {
    std::vector<double> raw(N + 1);
    std::vector<int64_t> v(Rp.begin(), Rp.end());
    std::memcpy(raw.data(), v.data(), sizeof(int64_t) * (N + 1));
    sc.upload(reinterpret_cast<double*>(rk), raw);
  }
  sc.add([=](cudaStream_t s) -> int {
    if (tol > 0.0) return norm_eps_launch(X[1], In(1) * Rp[1], tol, N, eps, s);
    return int(TT_OK);
  });
  // ---- Algorithm 2 truncation loop, left to right
  for (int n = 1; n < N; ++n) {
    const int64_t m = Rp[n - 1] * In(n), k = Rp[n];
    QrBufs qb = qr_view(pool, m, int(k));
    double* Rb = rbuf;
    double* Xn = X[n];
    double* Xq = X[n + 1];
    qr_plan(sc, qb, Xn, k, 1, qtmp, k, 1, Rb);
    const int rcap = int(max_rank > 0 ? std::min<int64_t>(max_rank, k) : k);
    sc.add([=](cudaStream_t s) -> int {
      return svd_trunc_launch(int(k), Rb, tol > 0.0 ? eps : nullptr, rcap, G1, G2, sig, rk + n, s, sbig);
    });
    // V(X_n) := Q U (row-major m x k) and (V S)^T H(X_{n+1}) into scratch
    // (copied over H(X_{n+1}) next): independent products, one grouped launch
    const int64_t w = In(n + 1) * Rp[n + 1];
    sc.gemm({gdesc(qtmp, k, 1, G1, k, 1, Xn, k, 1, m, k, k), gdesc(G2, 1, k, Xq, w, 1, tmp, w, 1, k, w, k)});
    sc.add([=](cudaStream_t s) -> int {
      if (!Xq) return int(TT_OK);
      TTR_CHECK_CUDA(cudaMemcpyAsync(Xq, tmp, sizeof(double) * k * w, cudaMemcpyDeviceToDevice, s));
      return int(TT_OK);
    });
  }
  // ---- compact every core to its decided ranks
  for (int n = 1; n <= N; ++n) {
    double* Xn = X[n];
    const int64_t r0 = Rp[n - 1], Ii = In(n), r1 = Rp[n];
    sc.add([=](cudaStream_t s) -> int {
      if (!Xn) return int(TT_OK);
      TTR_CHECK_CUDA(cudaMemcpyAsync(tmp, Xn, sizeof(double) * r0 * Ii * r1, cudaMemcpyDeviceToDevice, s));
      return compact_core_launch(tmp, Xn, r0, Ii, r1, rk + (n - 1), rk + n, s);
    });
  }
  return TT_OK;
}

int build_orthrand(const DetProblem& P, const std::vector<int64_t>& ell, const double* const* omega, uint64_t seed,
                   double* const* out, Arena& ar, Schedule& sc) {
  const int N = P.N;
  auto In = [&](int n) { return P.I[n - 1]; };
  const int64_t tcap = det_tmp_doubles(P);
  double* tmp = ar.take<double>(tcap);
  double* qtmp = ar.take<double>(tcap);
  std::vector<double*> X(N + 1, nullptr);
  for (int n = 1; n <= N; ++n) X[n] = ar.take<double>(formed_capacity(P, n));
  std::vector<std::pair<int64_t, int>> shapes;
  int64_t kq = 1;
  orth_shapes(P, &shapes, &kq);
  for (int n = 1; n < N; ++n) shapes.push_back({ell[n - 1] * In(n), int(ell[n])});
  const QrPool pool = qr_pool_reserve(ar, shapes);
  double* rbuf = ar.take<double>(kq * kq);
  std::vector<int64_t> Rp;
  TTR_TRY(plan_formed_orth(P, ar, sc, X, Rp, tmp, tcap, qtmp, &pool, rbuf));
  int64_t zcap = 1;
  for (int n = 1; n <= N; ++n) zcap = std::max(zcap, ell[n - 1] * In(n) * std::max(Rp[n], ell[n]));
  double* Z[2] = {ar.take<double>(zcap), ar.take<double>(zcap)};
  int64_t mcap = 1;
  for (int n = 1; n < N; ++n) mcap = std::max(mcap, ell[n] * Rp[n]);
  double* M = ar.take<double>(mcap);
  std::vector<const double*> Om(N + 1, nullptr);
  for (int n = 1; n < N; ++n) {
    if (omega) {
      Om[n] = omega[n - 1];
    } else {
      double* o = ar.take<double>(Rp[n] * ell[n]);
      Om[n] = o;
      const int64_t rr = Rp[n], ll = ell[n];
      sc.add([=](cudaStream_t s) -> int { return sketch_launch(o, 1, rr, ll, n - 1, seed, nullptr, s); });
    }
  }
  // Z_1 = X_1 (already right-orthogonal remainder on the right)
  const double* Zc = X[1];
  for (int n = 1; n < N; ++n) {
    const int64_t m = ell[n - 1] * In(n), k = ell[n], r = Rp[n];
    QrBufs qb = qr_view(pool, m, int(k));
    double* Ys = Z[(n + 1) & 1] == Zc ? Z[n & 1] : Z[(n + 1) & 1];
    // Y_n = V(X_n) Omega_n
    sc.gemm({gdesc(Zc, r, 1, Om[n], k, 1, Ys, k, 1, m, k, r)});
    qr_plan(sc, qb, Ys, k, 1, out[n - 1], k, 1, nullptr);
    // M_n = Q^T V(X_n)
    sc.gemm({gdesc(out[n - 1], 1, k, Zc, r, 1, M, r, 1, k, r, m)});
    // H(X_{n+1}) := M_n H(X_{n+1})  (the last core goes to the output)
    const int64_t w = In(n + 1) * Rp[n + 1];
    double* dst = (n + 1 == N) ? out[N - 1] : Ys;
    sc.gemm({gdesc(M, r, 1, X[n + 1], w, 1, dst, w, 1, k, w, r)});
    Zc = dst;
  }
  return TT_OK;
}

}  // namespace ttr

using namespace ttr;

extern "C" {

int tt_round_det_out_capacity(int32_t N, int32_t K, const int64_t* dims, const int64_t* ranks, int64_t* caps) {
  DetProblem P;
  TTR_TRY(validate_det(N, K, dims, ranks, nullptr, nullptr, false, &P));
  if (!caps) { set_error("null caps"); return TT_EINVAL; }
  for (int n = 1; n <= N; ++n) caps[n - 1] = formed_capacity(P, n);
  return TT_OK;
}

static int det_common(int32_t N, int32_t K, const int64_t* dims, const int64_t* ranks, const double* const* cores,
                      const double* coeffs, double tol, int64_t max_rank, double* const* out, int64_t* out_ranks,
                      void* workspace, size_t ws_bytes, void* stream, size_t* size_only) {
  DetProblem P;
  TTR_TRY(validate_det(N, K, dims, ranks, cores, coeffs, size_only == nullptr, &P));
  if (tol <= 0.0 && max_rank <= 0) {
    set_error("deterministic rounding needs tol > 0 or max_rank > 0");
    return TT_EINVAL;
  }
  if (!size_only && (!out || !out_ranks)) { set_error("null outputs"); return TT_EINVAL; }
  std::vector<double*> outv(N, nullptr);
  if (out) outv.assign(out, out + N);
  int64_t* rk = nullptr;
  std::vector<int64_t> r(N + 1);
  BuildFn build = [&](Arena& ar, Schedule& sc) {
    TTR_TRY(build_det(P, tol, max_rank, outv.data(), ar, sc, &rk));
    int64_t* rkd = rk;
    int64_t* rkh = r.data();
    const int n1 = N + 1;
    sc.add([rkd, rkh, n1](cudaStream_t st) -> int {
      if (rkd) TTR_CHECK_CUDA(cudaMemcpyAsync(rkh, rkd, sizeof(int64_t) * n1, cudaMemcpyDeviceToHost, st));
      return int(TT_OK);
    });
    return int(TT_OK);
  };
  if (size_only) return plan_workspace_bytes(build, size_only);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  int dstat = 0;
  TTR_TRY(plan_execute(build, workspace, ws_bytes, s, &dstat));
  TTR_CHECK_CUDA(cudaStreamSynchronize(s));
  TTR_TRY(status_code(dstat, "tt_round_det"));
  for (int n = 0; n <= N; ++n) out_ranks[n] = r[n];
  return TT_OK;
}

int tt_round_det(int32_t N, int32_t K, const int64_t* dims, const int64_t* ranks, const double* const* cores,
                 const double* coeffs, double tol, int64_t max_rank, double* const* out, int64_t* out_ranks,
                 void* workspace, size_t workspace_bytes, void* stream) {
  return det_common(N, K, dims, ranks, cores, coeffs, tol, max_rank, out, out_ranks, workspace, workspace_bytes,
                    stream, nullptr);
}

size_t tt_round_det_workspace(int32_t N, int32_t K, const int64_t* dims, const int64_t* ranks, double tol,
                              int64_t max_rank) {
  size_t b = 0;
  if (det_common(N, K, dims, ranks, nullptr, nullptr, tol, max_rank, nullptr, nullptr, nullptr, 0, nullptr, &b) !=
      TT_OK)
    return 0;
  return b;
}

static int orthrand_common(int32_t N, int32_t K, const int64_t* dims, const int64_t* ranks,
                           const double* const* cores, const double* coeffs, const int64_t* ells,
                           const double* const* omega, uint64_t seed, double* const* out, int64_t* out_ranks,
                           void* workspace, size_t ws_bytes, void* stream, size_t* size_only) {
  DetProblem P;
  TTR_TRY(validate_det(N, K, dims, ranks, cores, coeffs, size_only == nullptr, &P));
  if (!ells) { set_error("null target ranks"); return TT_EINVAL; }
  std::vector<int64_t> ell(ells, ells + N + 1);
  ell[0] = ell[N] = 1;
  for (int n = 1; n < N; ++n) {
    if (ell[n] < 1) { set_error("target ranks must be positive"); return TT_EINVAL; }
    ell[n] = std::min(ell[n], ell[n - 1] * P.I[n - 1]);
  }
  for (int n = N - 1; n >= 1; --n) ell[n] = std::min(ell[n], ell[n + 1] * P.I[n]);
  if (!size_only && (!out || !out_ranks)) { set_error("null outputs"); return TT_EINVAL; }
  std::vector<double*> outv(N, nullptr);
  if (out) outv.assign(out, out + N);
  BuildFn build = [&](Arena& ar, Schedule& sc) { return build_orthrand(P, ell, omega, seed, outv.data(), ar, sc); };
  if (size_only) return plan_workspace_bytes(build, size_only);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  int dstat = 0;
  TTR_TRY(plan_execute(build, workspace, ws_bytes, s, &dstat));
  TTR_CHECK_CUDA(cudaStreamSynchronize(s));
  TTR_TRY(status_code(dstat, "tt_round_orthrand"));
  for (int n = 0; n <= N; ++n) out_ranks[n] = ell[n];
  return TT_OK;
}

int tt_round_orthrand(int32_t N, int32_t K, const int64_t* dims, const int64_t* ranks, const double* const* cores,
                      const double* coeffs, const int64_t* ells, const double* const* omega, uint64_t seed,
                      double* const* out, int64_t* out_ranks, void* workspace, size_t workspace_bytes,
                      void* stream) {
  return orthrand_common(N, K, dims, ranks, cores, coeffs, ells, omega, seed, out, out_ranks, workspace,
                         workspace_bytes, stream, nullptr);
}

size_t tt_round_orthrand_workspace(int32_t N, int32_t K, const int64_t* dims, const int64_t* ranks,
                                   const int64_t* ells) {
  size_t b = 0;
  if (orthrand_common(N, K, dims, ranks, nullptr, nullptr, ells, nullptr, 0, nullptr, nullptr, nullptr, 0, nullptr,
                      &b) != TT_OK)
    return 0;
  return b;
}

int tt_orthrand_omega_ranks(int32_t N, int32_t K, const int64_t* dims, const int64_t* ranks, int64_t* rp) {
  DetProblem P;
  TTR_TRY(validate_det(N, K, dims, ranks, nullptr, nullptr, false, &P));
  if (!rp) { set_error("null output"); return TT_EINVAL; }
  // ranks after the optional fold of core 1 and Algorithm 1 (Section 2.3)
  std::vector<int64_t> R, Rp;
  det_static_ranks(P, &R, &Rp);
  for (int n = 0; n <= N; ++n) rp[n] = Rp[n];
  return TT_OK;
}

}  // extern "C"

// Two-Sided-Randomization (Algorithm 6, Section 3.3, generalized Nystrom) for a
// sum of K TT-tensors, without forming the block cores.
//
// Block form: the sketches of the formed sum are the summands' sketches side by
// side (W^L_n = [W^{L,(1)}_n ... W^{L,(K)}_n], l_n x S_n) and stacked
// (W^R_n = [W^{R,(1)}_n; ...], S_n x rho_n), as in the derivation of Section 3.4.
//   left-to-right: W^{L,(j)}_1 = c_j V(L_1)^T V(Y^(j)_1);
//                  T = W^{L,(j)}_{n-1} H(Y^(j)_n), W^{L,(j)}_n = V(L_n)^T V(T);
//   right-to-left: Algorithm 3 with the rho sketch (as in the sum rounding);
//   per bond:      A_n = W^L_n W^R_n (l_n x rho_n) = V_R S (Q U_R)^T from the thin QR
//                  A_n^T = Q R and the SVD R = U_R S V_R^T; then
//                  L_n = W^R_n (Q U_R) S^{+1/2}  (S_n x l_n),
//                  R_n = S^{+1/2} V_R^T W^L_n     (l_n x S_n), S^+ dropping
//                  s_i <= max(l, rho) 2^-52 s_1;
//   distribution:  X_n(:, i, :) = sum_j R^(j)_{n-1} Y^(j)_n(:, i, :) L^(j)_n with
//                  R_0 = the coefficients and L_N = ones.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <string>

#include "problem.cuh"
#include "prof.cuh"
#include "qr.cuh"

namespace ttr {

int mixed_digits(double tol, int N);

namespace {

// M[:, c] *= (s_c > thr) ? s_c^p : 0 for c < cols, thr = tol_rel * s_0 (sigma sorted descending).
__global__ void colscale_kernel(double* M, int64_t rows, int64_t cols, int64_t ld, const double* sig, double p,
                                double tol_rel) {
  const double thr = tol_rel * sig[0];
  for (int64_t e = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; e < rows * cols;
       e += int64_t(gridDim.x) * blockDim.x) {
    const int64_t r = e / cols, c = e % cols;
    const double s = sig[c];
    M[r * ld + c] *= (s > thr) ? pow(s, p) : 0.0;
  }
}

int colscale_launch(double* M, int64_t rows, int64_t cols, int64_t ld, const double* sig, double p, double tol_rel,
                    cudaStream_t s) {
  const unsigned g = unsigned(std::max<int64_t>(1, std::min<int64_t>(ceil_div(rows * cols, 256), 2048)));
  TTR_PREFER_SHARED(colscale_kernel);
  colscale_kernel<<<g, 256, 0, s>>>(M, rows, cols, ld, sig, p, tol_rel);
  TTR_CHECK_LAUNCH();
  prof_count_launch(1);
  return TT_OK;
}

// orth: the orthogonalizing restructure (Section 3.3 leaves it open): the
// distribution runs as a left-to-right sweep that carries the R factor of each
// core's thin QR into the next core, T_0 = 1,
//   C_n = (T_{n-1} R_n) x_1 Y_n x_3 L_n,  V(C_n) = Q_n T_n,  X_n = Q_n (n < N),
//   X_N = (T_{N-1} R_{N-1}) H(Y_N),
// so the result is the same tensor in left-orthogonal form; with tol > 0 the
// Section 3.2 truncation follows (ranks into *rk_dev).
int build_twosided(const SumProblem& P, const std::vector<int64_t>& rho, const double* const* skL,
                   const double* const* skR, uint64_t seed, int digits, double* const* out, Arena& ar,
                   Schedule& sc, bool orth = false, double tol = 0.0, int64_t** rk_dev = nullptr) {
  const int N = P.N, K = P.K;
  // every contraction in FP64, or (digits > 0) as the emulated FP64 product on
  // the tensor cores: both sketches span the projectors' ranges directly, so
  // all products, the sketch sweeps included, take the same digits
  auto gemm = [&](std::vector<GemmDesc> g) {
    if (digits > 0) sc.gemm_tc(std::move(g), digits);
    else sc.gemm(std::move(g));
  };
  const auto& S = P.S;
  const auto& ell = P.ell;
  auto In = [&](int n) { return P.I[n - 1]; };

  std::vector<double*> WL(N + 1, nullptr), WR(N + 1, nullptr), Lf(N + 1, nullptr), Rf(N + 1, nullptr);
  for (int n = 1; n < N; ++n) WL[n] = ar.take<double>(ell[n] * S[n]);
  for (int n = 1; n <= N; ++n) WR[n] = ar.take<double>(S[n] * rho[n]);
  for (int n = 1; n <= N; ++n) Lf[n] = ar.take<double>(S[n] * ell[n]);
  for (int n = 0; n < N; ++n) Rf[n] = ar.take<double>(ell[n] * S[n]);
  int64_t tmax = 1, zmax = 1, kmax = 1, amax = 1;
  for (int n = 2; n < N; ++n) tmax = std::max(tmax, ell[n - 1] * In(n) * S[n]);
  for (int n = 1; n <= N; ++n) zmax = std::max(zmax, S[n - 1] * In(n) * std::max(rho[n], ell[n]));
  for (int n = 1; n < N; ++n) {
    kmax = std::max(kmax, ell[n]);
    amax = std::max(amax, ell[n] * rho[n]);
  }
  double* T = ar.take<double>(tmax);
  double* Z = ar.take<double>(zmax);
  // per bond (the bond SVDs are independent and run in one launch)
  const int64_t nb = std::max(N - 1, 1);
  double* Am = ar.take<double>(amax * nb);
  double* Qt = ar.take<double>(amax * nb);
  double* Rb = ar.take<double>(kmax * kmax * nb);
  double* G1 = ar.take<double>(kmax * kmax * nb);
  double* G2 = ar.take<double>(kmax * kmax * nb);
  double* sig = ar.take<double>(kmax * nb);
  double* kd = ar.take<double>(nb);
  double* sbig = ar.take<double>(std::max<size_t>(svd_scratch_doubles(int(kmax)) * size_t(nb), 1));
  std::vector<std::pair<int64_t, int>> shapes;
  for (int n = 1; n < N; ++n) shapes.push_back({rho[n], int(ell[n])});
  if (orth)
    for (int n = 1; n < N; ++n) shapes.push_back({ell[n - 1] * In(n), int(ell[n])});
  const QrPool pool = qr_pool_reserve(ar, shapes);
  double *Cb = nullptr, *Tf = nullptr, *RT = nullptr;
  if (orth) {
    int64_t cmax = 1, rmax = 1;
    for (int n = 1; n <= N; ++n) cmax = std::max(cmax, ell[n - 1] * In(n) * ell[n]);
    for (int n = 0; n < N; ++n) rmax = std::max(rmax, ell[n] * S[n]);
    Cb = ar.take<double>(cmax);
    Tf = ar.take<double>(kmax * kmax);
    RT = ar.take<double>(rmax);
  }
  std::vector<const double*> L(N + 1, nullptr), Rs(N + 1, nullptr);
  for (int n = 1; n <= N; ++n) {
    if (skL) {
      L[n] = skL[n - 1];
    } else {
      double* d = ar.take<double>(ell[n - 1] * In(n) * ell[n]);
      L[n] = d;
      const int64_t a = ell[n - 1], b = In(n), c = ell[n];
      sc.add([=](cudaStream_t s) -> int { return sketch_launch(d, a, b, c, n - 1, seed, nullptr, s); });
    }
    if (skR) {
      Rs[n] = skR[n - 1];
    } else {
      double* d = ar.take<double>(rho[n - 1] * In(n) * rho[n]);
      Rs[n] = d;
      const int64_t a = rho[n - 1], b = In(n), c = rho[n];
      sc.add([=](cudaStream_t s) -> int { return sketch_launch(d, a, b, c, n - 1, seed + 1, nullptr, s); });
    }
  }
  sc.add([=](cudaStream_t s) -> int {
    TTR_TRY(fill_launch(WR[N], S[N] * rho[N], 1.0, s));
    return fill_launch(Lf[N], S[N] * ell[N], 1.0, s);
  });
  sc.upload(Rf[0], P.coeffs);

  // ---- left-to-right partial contractions with L
  for (int n = 1; n < N; ++n) {
    std::vector<GemmDesc> ga, gb;
    for (int j = 0; j < K; ++j) {
      const int64_t r0 = P.r(j, n - 1), r1 = P.r(j, n);
      double* Wo = WL[n] ? WL[n] + P.o(j, n) : nullptr;
      if (n == 1) {
        ga.push_back(gdesc(L[1], 1, ell[1], P.core(j, 1), r1, 1, Wo, S[1], 1, ell[1], r1, In(1), P.coeffs[j]));
      } else {
        double* Tj = T ? T + ell[n - 1] * In(n) * P.o(j, n) : nullptr;
        const double* Wi = WL[n - 1] ? WL[n - 1] + P.o(j, n - 1) : nullptr;
        ga.push_back(gdesc(Wi, S[n - 1], 1, P.core(j, n), In(n) * r1, 1, Tj, In(n) * r1, 1, ell[n - 1], In(n) * r1,
                           r0));
        gb.push_back(gdesc(L[n], 1, ell[n], Tj, r1, 1, Wo, S[n], 1, ell[n], r1, ell[n - 1] * In(n)));
      }
    }
    gemm(ga);
    gemm(gb);
  }
  // ---- right-to-left partial contractions with R (Algorithm 3 for every summand)
  for (int n = N; n >= 2; --n) {
    std::vector<GemmDesc> ga;
    for (int j = 0; j < K; ++j) {
      const int64_t r0 = P.r(j, n - 1), r1 = P.r(j, n);
      double* Zj = Z ? Z + P.o(j, n - 1) * In(n) * rho[n] : nullptr;
      const double* Wj = WR[n] ? WR[n] + P.o(j, n) * rho[n] : nullptr;
      ga.push_back(gdesc(P.core(j, n), r1, 1, Wj, rho[n], 1, Zj, rho[n], 1, r0 * In(n), rho[n], r1));
    }
    gemm(ga);
    // shared sketch: one GEMM of the stacked H(Z^(j)) with H(R_n)^T
    gemm({gdesc(Z, In(n) * rho[n], 1, Rs[n], 1, In(n) * rho[n], WR[n - 1], rho[n - 1], 1, S[n - 1], rho[n - 1],
                   In(n) * rho[n])});
  }
  // ---- per bond: SVD of W^L_n W^R_n and the factors L_n, R_n. First every
  // bond's product and thin QR, then all bond SVDs in one launch (one block
  // each), then the factors.
  const double eps52 = std::ldexp(1.0, -52);
  auto bAm = [&](int n) { return Am ? Am + amax * (n - 1) : nullptr; };
  auto bQt = [&](int n) { return Qt ? Qt + amax * (n - 1) : nullptr; };
  auto bK2 = [&](double* base, int n) { return base ? base + kmax * kmax * (n - 1) : nullptr; };
  for (int n = 1; n < N; ++n) {
    const int64_t l = ell[n], r = rho[n];
    gemm({gdesc(WL[n], S[n], 1, WR[n], r, 1, bAm(n), r, 1, l, r, S[n])});
    // thin QR of A^T (r x l, a strided view of A)
    qr_plan(sc, qr_view(pool, r, int(l)), bAm(n), 1, r, bQt(n), l, 1, bK2(Rb, n));
  }
  if (N > 1) {
    std::vector<double> ks;
    for (int n = 1; n < N; ++n) ks.push_back(double(ell[n]));
    sc.upload(kd, ks);
    const int nbonds = N - 1, km = int(kmax);
    sc.add([=](cudaStream_t s) -> int { return svd_batch_launch(nbonds, km, kd, Rb, G1, G2, sig, s, sbig); });
  }
  for (int n = 1; n < N; ++n) {
    const int64_t l = ell[n], r = rho[n];
    double* am = bAm(n);
    double* g2 = bK2(G2, n);
    const double* sg = sig ? sig + kmax * (n - 1) : nullptr;
    const double tol_rel = double(std::max(l, r)) * eps52;
    // P1 = Q U_R S^{+1/2} into Am (r x l)
    gemm({gdesc(bQt(n), l, 1, bK2(G1, n), l, 1, am, l, 1, r, l, l)});
    sc.add([=](cudaStream_t s) -> int {
      TTR_TRY(colscale_launch(am, r, l, l, sg, -0.5, tol_rel, s));
      return colscale_launch(g2, l, l, l, sg, -1.5, tol_rel, s);    // V_R S^{+1/2} = G2 S^{-3/2}
    });
    gemm({gdesc(WR[n], r, 1, am, l, 1, Lf[n], l, 1, S[n], l, r)});         // L_n = W^R_n P1
    gemm({gdesc(g2, 1, l, WL[n], S[n], 1, Rf[n], S[n], 1, l, S[n], l)});  // R_n = P2^T W^L_n
  }
  // ---- distribution of the factors into the cores
  for (int n = 1; n <= N; ++n) {
    std::vector<GemmDesc> ga;
    for (int j = 0; j < K; ++j) {
      const int64_t r0 = P.r(j, n - 1), r1 = P.r(j, n);
      double* Zj = Z ? Z + P.o(j, n - 1) * In(n) * ell[n] : nullptr;
      const double* Lj = Lf[n] ? Lf[n] + P.o(j, n) * ell[n] : nullptr;
      ga.push_back(gdesc(P.core(j, n), r1, 1, Lj, ell[n], 1, Zj, ell[n], 1, r0 * In(n), ell[n], r1));
    }
    gemm(ga);
    if (!orth) {
      gemm({gdesc(Rf[n - 1], S[n - 1], 1, Z, In(n) * ell[n], 1, out[n - 1], In(n) * ell[n], 1, ell[n - 1],
                     In(n) * ell[n], S[n - 1])});
      continue;
    }
    // left factor T_{n-1} R_{n-1} (T_0 = 1)
    const double* Rl = Rf[n - 1];
    if (n > 1) {
      gemm({gdesc(Tf, ell[n - 1], 1, Rf[n - 1], S[n - 1], 1, RT, S[n - 1], 1, ell[n - 1], S[n - 1], ell[n - 1])});
      Rl = RT;
    }
    double* dst = (n < N) ? Cb : out[n - 1];
    gemm({gdesc(Rl, S[n - 1], 1, Z, In(n) * ell[n], 1, dst, In(n) * ell[n], 1, ell[n - 1], In(n) * ell[n],
                   S[n - 1])});
    if (n < N) {
      const int64_t m = ell[n - 1] * In(n), k = ell[n];
      qr_plan(sc, qr_view(pool, m, int(k)), Cb, k, 1, out[n - 1], k, 1, Tf, true);
    }
  }
  if (orth && tol > 0.0) TTR_TRY(plan_truncation(ar, sc, N, P.I, ell, tol, out, rk_dev, 0));
  return TT_OK;
}

}  // namespace
}  // namespace ttr

using namespace ttr;

extern "C" {

static int twosided_common(int32_t N, int32_t K, const int64_t* dims, const int64_t* ranks,
                           const double* const* cores, const double* coeffs, const int64_t* ells,
                           const int64_t* rhos, const double* const* skL, const double* const* skR, uint64_t seed,
                           int32_t precision, double* const* out, int64_t* out_ranks, void* workspace,
                           size_t ws_bytes, void* stream, size_t* size_only, bool orth = false, double tol = 0.0) {
  if (precision != TT_PREC_FP64 && precision != TT_PREC_MIXED && precision != TT_PREC_MIXED_FULL) {
    set_error("tt_round_twosided: unknown precision mode");
    return TT_EINVAL;
  }
  SumProblem P;
  TTR_TRY(validate_sum(N, K, dims, ranks, cores, coeffs, ells, size_only == nullptr, &P));
  if (N < 2) { set_error("two-sided rounding needs N >= 2"); return TT_EINVAL; }
  std::vector<int64_t> rr(N + 1);
  for (int n = 0; n <= N; ++n) rr[n] = rhos ? rhos[n] : int64_t(std::ceil(1.5 * double(P.ell[n])));
  std::vector<int64_t> rho = clamp_rank_vector(P.I, rr.data());
  for (int n = 1; n < N; ++n)
    if (rho[n] < P.ell[n]) {
      set_error("two-sided rounding needs rho_n >= l_n (after clamping)");
      return TT_EINVAL;
    }
  if (!size_only && (!out || !out_ranks)) { set_error("null outputs"); return TT_EINVAL; }
  std::vector<double*> outv(N, nullptr);
  if (out) outv.assign(out, out + N);
  const int digits = (precision != TT_PREC_FP64) ? mixed_digits(orth ? tol : 0.0, N) : 0;
  int64_t* rk_dev = nullptr;
  std::vector<int64_t> rk(N + 1);
  const bool trunc = orth && tol > 0.0;
  BuildFn build = [&](Arena& ar, Schedule& sc) {
    TTR_TRY(build_twosided(P, rho, skL, skR, seed, digits, outv.data(), ar, sc, orth, tol, &rk_dev));
    if (trunc) {
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
  TTR_TRY(status_code(dstat, orth ? "tt_round_twosided_orth" : "tt_round_twosided"));
  for (int n = 0; n <= N; ++n) out_ranks[n] = trunc ? rk[n] : P.ell[n];
  return TT_OK;
}

int tt_round_twosided(int32_t N, int32_t K, const int64_t* dims, const int64_t* ranks, const double* const* cores,
                      const double* coeffs, const int64_t* ells, const int64_t* rhos,
                      const double* const* sketch_left, const double* const* sketch_right, uint64_t seed,
                      int32_t precision, double* const* out, int64_t* out_ranks, void* workspace,
                      size_t workspace_bytes, void* stream) {
  return twosided_common(N, K, dims, ranks, cores, coeffs, ells, rhos, sketch_left, sketch_right, seed, precision,
                         out, out_ranks, workspace, workspace_bytes, stream, nullptr);
}

size_t tt_round_twosided_workspace(int32_t N, int32_t K, const int64_t* dims, const int64_t* ranks,
                                   const int64_t* ells, const int64_t* rhos, int32_t precision) {
  size_t b = 0;
  if (twosided_common(N, K, dims, ranks, nullptr, nullptr, ells, rhos, nullptr, nullptr, 0, precision, nullptr, nullptr,
                      nullptr, 0, nullptr, &b) != TT_OK)
    return 0;
  return b;
}

int tt_round_twosided_orth(int32_t N, int32_t K, const int64_t* dims, const int64_t* ranks,
                           const double* const* cores, const double* coeffs, const int64_t* ells,
                           const int64_t* rhos, const double* const* sketch_left,
                           const double* const* sketch_right, uint64_t seed, double tol, int32_t precision,
                           double* const* out, int64_t* out_ranks, void* workspace, size_t workspace_bytes,
                           void* stream) {
  return twosided_common(N, K, dims, ranks, cores, coeffs, ells, rhos, sketch_left, sketch_right, seed, precision,
                         out, out_ranks, workspace, workspace_bytes, stream, nullptr, true, tol);
}

size_t tt_round_twosided_orth_workspace(int32_t N, int32_t K, const int64_t* dims, const int64_t* ranks,
                                        const int64_t* ells, const int64_t* rhos, double tol, int32_t precision) {
  size_t b = 0;
  if (twosided_common(N, K, dims, ranks, nullptr, nullptr, ells, rhos, nullptr, nullptr, 0, precision, nullptr, nullptr,
                      nullptr, 0, nullptr, &b, true, tol) != TT_OK)
    return 0;
  return b;
}

}  // extern "C"

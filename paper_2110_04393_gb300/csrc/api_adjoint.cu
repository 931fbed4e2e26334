// C ABI: reverse-mode derivative of fixed-sketch Randomize-then-Orthogonalize
// (Algorithm 5 with the Gaussian sketch held fixed and fixed target ranks).
// The paper has no derivative; this is the chain rule through the steps of
// Algorithm 5 and Algorithm 3, all of them as FP64 GEMMs plus the thin-QR
// backward formula. The forward quantities (W_n of Algorithm 3, the cores
// X~_n before their QR, Q_n, the R factors T_n, M_n) are recomputed here
// rather than kept from the forward call.
//
// Forward (n = 1..N-1): Z_n = V(X~_n), S_n = Z_n W_n = Q_n T_n, X_hat_n = Q_n,
// M_n = Q_n^T Z_n, H(X~_{n+1}) = M_n H(Y_{n+1}); X~_1 = Y_1, X_hat_N = X~_N.
// Reverse, n = N-1..1, with X~bar_N = Xbar_N:
//   Mbar = H(X~bar_{n+1}) H(Y_{n+1})^T,       H(Ybar_{n+1}) += M_n^T H(X~bar_{n+1})
//   Qbar = Z_n Mbar^T + V(Xbar_n),             Zbar = Q_n Mbar
//   Sbar = (Qbar + Q_n sym_l(-Qbar^T Q_n)) T_n^{-T}   (thin QR, R factor not differentiated;
//                                               sym_l(A) = tril(A) + tril(A, -1)^T)
//   Zbar += Sbar W_n^T,  Wbar_n = Z_n^T Sbar,  X~bar_n = Zbar
// then Ybar_1 += X~bar_1 and Algorithm 3 in reverse, n = 2..N-1:
//   H(Zp) = Wbar_{n-1} H(Omega_n),  V(Ybar_n) += V(Zp) W_n^T,  Wbar_n += V(Y_n)^T V(Zp),
// and finally H(Ybar_N) += Wbar_{N-1} H(Omega_N).
#include <algorithm>
#include <string>

#include "plan.cuh"
#include "problem.cuh"
#include "qr.cuh"

namespace ttr {

int mixed_digits(double tol, int N);

namespace {

// digits == 0: every product in FP64; digits > 0: every product as the
// emulated FP64 tensor-core GEMM with that many bf16 digits (the triangular
// inverse, the QR and the small elementwise steps stay FP64).
int build_rand_backward(int N, const std::vector<int64_t>& I, const std::vector<int64_t>& R,
                        const std::vector<int64_t>& ell, const double* const* Y, const double* const* Om,
                        const double* const* Xb, double* const* Yb, Arena& ar, Schedule& sc, int digits = 0) {
  struct Gemm {
    Schedule& sc;
    int digits;
    void gemm(std::vector<GemmDesc> g) {
      if (digits > 0) sc.gemm_tc(std::move(g), digits);
      else sc.gemm(std::move(g));
    }
  } G{sc, digits};
  auto In = [&](int n) { return I[n - 1]; };
  auto Yc = [&](int n) -> const double* { return Y ? Y[n - 1] : nullptr; };
  auto Oc = [&](int n) -> const double* { return Om ? Om[n - 1] : nullptr; };
  auto Xbc = [&](int n) -> const double* { return Xb ? Xb[n - 1] : nullptr; };
  auto Ybc = [&](int n) -> double* { return Yb ? Yb[n - 1] : nullptr; };

  std::vector<double*> W(N + 1, nullptr), Xt(N + 1, nullptr), Q(N, nullptr), Tq(N, nullptr), Ti(N, nullptr),
      Mm(N, nullptr), Wb(N + 1, nullptr);
  int64_t zrl = 1, smax = 1, zmax = 1, kk = 1, lr = 1;
  for (int n = 1; n <= N; ++n) {
    W[n] = ar.take<double>(R[n] * ell[n]);
    zrl = std::max(zrl, R[n - 1] * In(n) * ell[n]);
  }
  for (int n = 2; n <= N; ++n) Xt[n] = ar.take<double>(ell[n - 1] * In(n) * R[n]);
  std::vector<std::pair<int64_t, int>> shapes;
  for (int n = 1; n < N; ++n) {
    Q[n] = ar.take<double>(ell[n - 1] * In(n) * ell[n]);
    Tq[n] = ar.take<double>(ell[n] * ell[n]);
    Ti[n] = ar.take<double>(ell[n] * ell[n]);
    Mm[n] = ar.take<double>(ell[n] * R[n]);
    Wb[n] = ar.take<double>(R[n] * ell[n]);
    smax = std::max(smax, ell[n - 1] * In(n) * ell[n]);
    zmax = std::max(zmax, ell[n - 1] * In(n) * R[n]);
    kk = std::max(kk, ell[n] * ell[n]);
    lr = std::max(lr, ell[n] * R[n]);
    shapes.push_back({ell[n - 1] * In(n), int(ell[n])});
  }
  double* Zrl = ar.take<double>(zrl);
  double* S = ar.take<double>(smax);
  double* Mbar = ar.take<double>(lr);
  double* Qbar = ar.take<double>(smax);
  double* Gm = ar.take<double>(smax);
  double* Sbar = ar.take<double>(smax);
  double* A = ar.take<double>(kk);
  double* Zb[2] = {ar.take<double>(zmax), ar.take<double>(zmax)};
  const QrPool pool = qr_pool_reserve(ar, shapes);

  // Ybar = 0, W_N = 1
  for (int n = 1; n <= N; ++n) {
    double* y = Ybc(n);
    const size_t bytes = sizeof(double) * size_t(R[n - 1] * In(n) * R[n]);
    sc.add([y, bytes](cudaStream_t s) -> int {
      if (y) TTR_CHECK_CUDA(cudaMemsetAsync(y, 0, bytes, s));
      return int(TT_OK);
    });
  }
  {
    double* w = W[N];
    sc.add([w](cudaStream_t s) -> int { return fill_launch(w, 1, 1.0, s); });
  }
  // Algorithm 3: Z = V(Y_n) W_n, W_{n-1} = H(Z) H(Omega_n)^T, n = N..2
  for (int n = N; n >= 2; --n) {
    G.gemm({gdesc(Yc(n), R[n], 1, W[n], ell[n], 1, Zrl, ell[n], 1, R[n - 1] * In(n), ell[n], R[n])});
    G.gemm({gdesc(Zrl, In(n) * ell[n], 1, Oc(n), 1, In(n) * ell[n], W[n - 1], ell[n - 1], 1, R[n - 1], ell[n - 1],
                   In(n) * ell[n])});
  }
  // Algorithm 5 forward, keeping X~_n, Q_n, T_n (and T_n^{-1}), M_n
  for (int n = 1; n < N; ++n) {
    const double* Xc = (n == 1) ? Yc(1) : Xt[n];
    const int64_t m = ell[n - 1] * In(n), k = ell[n];
    G.gemm({gdesc(Xc, R[n], 1, W[n], ell[n], 1, S, k, 1, m, k, R[n])});
    qr_plan(sc, qr_view(pool, m, int(k)), S, k, 1, Q[n], k, 1, Tq[n]);
    G.gemm({gdesc(Q[n], 1, k, Xc, R[n], 1, Mm[n], R[n], 1, k, R[n], m)});
    G.gemm({gdesc(Mm[n], R[n], 1, Yc(n + 1), In(n + 1) * R[n + 1], 1, Xt[n + 1], In(n + 1) * R[n + 1], 1, k,
                   In(n + 1) * R[n + 1], R[n])});
    double* t = Tq[n];
    double* ti = Ti[n];
    sc.add([t, ti, k](cudaStream_t s) -> int { return triu_inverse_launch(t, ti, int(k), s); });
  }
  // reverse of the left-to-right sweep
  const double* xtb = Xbc(N);                   // X~bar_N = Xbar_N (l_{N-1} x I_N x 1)
  int pp = 0;
  for (int n = N - 1; n >= 1; --n) {
    const double* Xc = (n == 1) ? Yc(1) : Xt[n];
    const int64_t m = ell[n - 1] * In(n), k = ell[n], rn = R[n], cols = In(n + 1) * R[n + 1];
    // Mbar = H(X~bar_{n+1}) H(Y_{n+1})^T ; H(Ybar_{n+1}) += M_n^T H(X~bar_{n+1})
    G.gemm({gdesc(xtb, cols, 1, Yc(n + 1), 1, cols, Mbar, rn, 1, k, rn, cols)});
    G.gemm({gdesc(Mm[n], 1, rn, xtb, cols, 1, Ybc(n + 1), cols, 1, rn, cols, k, 1.0, 1.0)});
    // Qbar = V(Xbar_n) + Z_n Mbar^T ; Zbar = Q_n Mbar
    {
      double* qb = Qbar;
      const double* xb = Xbc(n);
      const size_t bytes = sizeof(double) * size_t(m * k);
      sc.add([qb, xb, bytes](cudaStream_t s) -> int {
        if (qb && xb) TTR_CHECK_CUDA(cudaMemcpyAsync(qb, xb, bytes, cudaMemcpyDeviceToDevice, s));
        return int(TT_OK);
      });
    }
    G.gemm({gdesc(Xc, rn, 1, Mbar, 1, rn, Qbar, k, 1, m, k, rn, 1.0, 1.0)});
    double* zb = Zb[pp];
    G.gemm({gdesc(Q[n], k, 1, Mbar, rn, 1, zb, rn, 1, m, rn, k)});
    // A = sym_l(-Qbar^T Q_n) ; G = Qbar + Q_n A ; Sbar = G T_n^{-T}
    G.gemm({gdesc(Qbar, 1, k, Q[n], k, 1, A, k, 1, k, k, m, -1.0)});
    {
      double* a = A;
      sc.add([a, k](cudaStream_t s) -> int { return sym_lower_launch(a, int(k), s); });
      double* g = Gm;
      const double* qb = Qbar;
      const size_t bytes = sizeof(double) * size_t(m * k);
      sc.add([g, qb, bytes](cudaStream_t s) -> int {
        if (g && qb) TTR_CHECK_CUDA(cudaMemcpyAsync(g, qb, bytes, cudaMemcpyDeviceToDevice, s));
        return int(TT_OK);
      });
    }
    G.gemm({gdesc(Q[n], k, 1, A, k, 1, Gm, k, 1, m, k, k, 1.0, 1.0)});
    G.gemm({gdesc(Gm, k, 1, Ti[n], 1, k, Sbar, k, 1, m, k, k)});
    // Zbar += Sbar W_n^T ; Wbar_n = Z_n^T Sbar
    G.gemm({gdesc(Sbar, k, 1, W[n], 1, k, zb, rn, 1, m, rn, k, 1.0, 1.0)});
    G.gemm({gdesc(Xc, 1, rn, Sbar, k, 1, Wb[n], k, 1, rn, k, m)});
    xtb = zb;                                    // X~bar_n (l_{n-1} x I_n x R_n)
    pp ^= 1;
  }
  {
    double* y1 = Ybc(1);
    const double* x1 = xtb;
    const int64_t cnt = In(1) * R[1];
    sc.add([y1, x1, cnt](cudaStream_t s) -> int { return axpy_launch(y1, x1, cnt, s); });
  }
  // Algorithm 3 in reverse
  for (int n = 2; n < N; ++n) {
    const int64_t cols = In(n) * ell[n];
    double* zp = Zrl;
    G.gemm({gdesc(Wb[n - 1], ell[n - 1], 1, Oc(n), cols, 1, zp, cols, 1, R[n - 1], cols, ell[n - 1])});
    G.gemm({gdesc(zp, ell[n], 1, W[n], 1, ell[n], Ybc(n), R[n], 1, R[n - 1] * In(n), R[n], ell[n], 1.0, 1.0)});
    G.gemm({gdesc(Yc(n), 1, R[n], zp, ell[n], 1, Wb[n], ell[n], 1, R[n], ell[n], R[n - 1] * In(n), 1.0, 1.0)});
  }
  if (N >= 2) {
    const int64_t cols = In(N) * ell[N];
    G.gemm({gdesc(Wb[N - 1], ell[N - 1], 1, Oc(N), cols, 1, Ybc(N), cols, 1, R[N - 1], cols, ell[N - 1], 1.0,
                   1.0)});
  }
  return TT_OK;
}

int backward_common(int32_t N, const int64_t* dims, const int64_t* ranks, const double* const* cores,
                    const int64_t* ells, const double* const* sketch, const double* const* xbar, double* const* ybar,
                    void* workspace, size_t ws_bytes, void* stream, size_t* size_only) {
  if (N < 1 || !dims || !ranks || !ells) {
    set_error("tt_round_rand_backward: invalid arguments");
    return TT_EINVAL;
  }
  std::vector<int64_t> I(dims, dims + N), R(ranks, ranks + N + 1);
  if (R[0] != 1 || R[N] != 1) {
    set_error("tt_round_rand_backward: ranks must start and end with 1");
    return TT_EINVAL;
  }
  for (int n = 0; n < N; ++n)
    if (I[n] < 1 || R[n + 1] < 1) {
      set_error("tt_round_rand_backward: mode sizes and ranks must be positive");
      return TT_EINVAL;
    }
  const std::vector<int64_t> ell = clamp_rank_vector(I, ells);
  for (int n = 0; n <= N; ++n)
    if (ell[n] > TT_MAX_RANK || R[n] > TT_MAX_RANK) {
      set_error("tt_round_rand_backward: ranks above 1024 are not supported");
      return TT_EUNSUPPORTED;
    }
  if (!size_only) {
    if (!cores || !xbar || !ybar || (N > 1 && !sketch)) {
      set_error("tt_round_rand_backward: null pointer array");
      return TT_EINVAL;
    }
    for (int n = 0; n < N; ++n)
      if (!cores[n] || !xbar[n] || !ybar[n] || (n > 0 && !sketch[n])) {
        set_error("tt_round_rand_backward: null core pointer");
        return TT_EINVAL;
      }
  }
  if (N == 1) {                                 // X_hat = Y: Ybar = Xbar
    if (size_only) {
      *size_only = 0;
      return TT_OK;
    }
    TTR_CHECK_CUDA(cudaMemcpyAsync(ybar[0], xbar[0], sizeof(double) * size_t(I[0]), cudaMemcpyDeviceToDevice,
                                   static_cast<cudaStream_t>(stream)));
    return TT_OK;
  }
  BuildFn build = [&](Arena& ar, Schedule& sc) {
    return build_rand_backward(N, I, R, ell, size_only ? nullptr : cores, size_only ? nullptr : sketch,
                               size_only ? nullptr : xbar, size_only ? nullptr : ybar, ar, sc);
  };
  if (size_only) return plan_workspace_bytes(build, size_only);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  int dstat = 0;
  TTR_TRY(plan_execute(build, workspace, ws_bytes, s, &dstat));
  TTR_CHECK_CUDA(cudaStreamSynchronize(s));
  return status_code(dstat, "tt_round_rand_backward");
}

// float32 storage at the boundary: the cores, sketch and cotangents are
// converted to float64 on the device, the adjoint runs with FP32-class
// products (digits of tt_mixed_digits in fixed-rank mode) and FP64 QR /
// triangular steps, and ybar is converted back.
int backward_f32_common(int32_t N, const int64_t* dims, const int64_t* ranks, const float* const* cores,
                        const int64_t* ells, const float* const* sketch, const float* const* xbar, float* const* ybar,
                        void* workspace, size_t ws_bytes, void* stream, size_t* size_only) {
  if (N < 1 || !dims || !ranks || !ells) {
    set_error("tt_round_rand_backward_f32: invalid arguments");
    return TT_EINVAL;
  }
  std::vector<int64_t> I(dims, dims + N), R(ranks, ranks + N + 1);
  if (R[0] != 1 || R[N] != 1) {
    set_error("tt_round_rand_backward_f32: ranks must start and end with 1");
    return TT_EINVAL;
  }
  for (int n = 0; n < N; ++n)
    if (I[n] < 1 || R[n + 1] < 1) {
      set_error("tt_round_rand_backward_f32: mode sizes and ranks must be positive");
      return TT_EINVAL;
    }
  const std::vector<int64_t> ell = clamp_rank_vector(I, ells);
  for (int n = 0; n <= N; ++n)
    if (ell[n] > TT_MAX_RANK || R[n] > TT_MAX_RANK) {
      set_error("tt_round_rand_backward_f32: ranks above 1024 are not supported");
      return TT_EUNSUPPORTED;
    }
  if (!size_only) {
    if (!cores || !xbar || !ybar || (N > 1 && !sketch)) {
      set_error("tt_round_rand_backward_f32: null pointer array");
      return TT_EINVAL;
    }
    for (int n = 0; n < N; ++n)
      if (!cores[n] || !xbar[n] || !ybar[n] || (n > 0 && !sketch[n])) {
        set_error("tt_round_rand_backward_f32: null core pointer");
        return TT_EINVAL;
      }
  }
  // The thin-QR backward combines terms that largely cancel (Qbar + Q sym(-Qbar^T Q)),
  // so the products take FP64-class digits (relative 1e-11 / N), not FP32 ones.
  const int digits = mixed_digits(1e-8, N);
  BuildFn build = [&](Arena& ar, Schedule& sc) {
    std::vector<double*> Yd(N), Od(N, nullptr), Xd(N), Bd(N);
    std::vector<int64_t> ny(N), nx(N);
    for (int n = 0; n < N; ++n) {
      ny[n] = R[n] * I[n] * R[n + 1];
      nx[n] = ell[n] * I[n] * ell[n + 1];
      Yd[n] = ar.take<double>(ny[n]);
      Xd[n] = ar.take<double>(nx[n]);
      Bd[n] = ar.take<double>(ny[n]);
      if (n > 0) Od[n] = ar.take<double>(nx[n]);
    }
    for (int n = 0; n < N; ++n) {
      const float* yc = size_only ? nullptr : cores[n];
      const float* xc = size_only ? nullptr : xbar[n];
      const float* oc = (size_only || n == 0) ? nullptr : sketch[n];
      double *yd = Yd[n], *xd = Xd[n], *od = Od[n];
      const int64_t a = ny[n], b = nx[n];
      sc.add([=](cudaStream_t s) -> int {
        TTR_TRY(cvt_f32_f64_launch(yc, yd, a, s));
        TTR_TRY(cvt_f32_f64_launch(xc, xd, b, s));
        return cvt_f32_f64_launch(oc, od, b, s);
      });
    }
    std::vector<const double*> Yc(Yd.begin(), Yd.end()), Oc(Od.begin(), Od.end()), Xc(Xd.begin(), Xd.end());
    if (N == 1) {
      double* bd = Bd[0];
      const double* xd = Xd[0];
      const int64_t a = ny[0];
      sc.add([=](cudaStream_t s) -> int {
        if (bd && xd) TTR_CHECK_CUDA(cudaMemcpyAsync(bd, xd, sizeof(double) * a, cudaMemcpyDeviceToDevice, s));
        return int(TT_OK);
      });
    } else {
      TTR_TRY(build_rand_backward(N, I, R, ell, Yc.data(), Oc.data(), Xc.data(), Bd.data(), ar, sc, digits));
    }
    for (int n = 0; n < N; ++n) {
      float* yb = size_only ? nullptr : ybar[n];
      const double* bd = Bd[n];
      const int64_t a = ny[n];
      sc.add([=](cudaStream_t s) -> int { return cvt_f64_f32_launch(bd, yb, a, s); });
    }
    return int(TT_OK);
  };
  if (size_only) return plan_workspace_bytes(build, size_only);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  int dstat = 0;
  TTR_TRY(plan_execute(build, workspace, ws_bytes, s, &dstat));
  TTR_CHECK_CUDA(cudaStreamSynchronize(s));
  return status_code(dstat, "tt_round_rand_backward_f32");
}

}  // namespace
}  // namespace ttr

using namespace ttr;

extern "C" {

int tt_round_rand_backward_f32(int32_t N, const int64_t* dims, const int64_t* ranks, const float* const* cores,
                               const int64_t* ells, const float* const* sketch, const float* const* xbar,
                               float* const* ybar, void* workspace, size_t workspace_bytes, void* stream) {
  return backward_f32_common(N, dims, ranks, cores, ells, sketch, xbar, ybar, workspace, workspace_bytes, stream,
                             nullptr);
}

size_t tt_round_rand_backward_f32_workspace(int32_t N, const int64_t* dims, const int64_t* ranks,
                                            const int64_t* ells) {
  size_t bytes = 0;
  if (backward_f32_common(N, dims, ranks, nullptr, ells, nullptr, nullptr, nullptr, nullptr, 0, nullptr, &bytes) !=
      TT_OK)
    return 0;
  return bytes;
}

int tt_round_rand_backward(int32_t N, const int64_t* dims, const int64_t* ranks, const double* const* cores,
                           const int64_t* ells, const double* const* sketch, const double* const* xbar,
                           double* const* ybar, void* workspace, size_t workspace_bytes, void* stream) {
  return backward_common(N, dims, ranks, cores, ells, sketch, xbar, ybar, workspace, workspace_bytes, stream,
                         nullptr);
}

size_t tt_round_rand_backward_workspace(int32_t N, const int64_t* dims, const int64_t* ranks, const int64_t* ells) {
  size_t bytes = 0;
  if (backward_common(N, dims, ranks, nullptr, ells, nullptr, nullptr, nullptr, nullptr, 0, nullptr, &bytes) !=
      TT_OK)
    return 0;
  return bytes;
}

}  // extern "C"

// C ABI: TT arithmetic around the rounding (Section 2.3 and Section 4.2).
//
//   tt_inner               <X, Y^(j)> for K tensors Y^(j) at once: Algorithm 3
//                          (right-to-left partial contractions) of every Y^(j)
//                          against X, run down to the first core, where the
//                          partial contraction is the 1 x 1 inner product.
//   tt_norm                ||X|| = sqrt(<X, X>) by the same sweep.
//   tt_round_gram_schmidt  one Gram-Schmidt step of TT-GMRES (Section 4.2):
//                          h_j = <V_j, W>, Z = W - sum_j h_j V_j rounded by
//                          Algorithm 7 with the coefficients taken on the
//                          device, h_{k+1} = ||Z||, V_{k+1} = Z / h_{k+1}; one
//                          schedule, one host synchronization.
#include <algorithm>
#include <cmath>
#include <string>

#include "plan.cuh"
#include "prof.cuh"
#include "problem.cuh"

namespace ttr {

int build_sum_rand(const SumProblem& P, const double* const* sketch_in, uint64_t seed, double tol, int digits,
                   double* const* out, Arena& ar, Schedule& sc, int64_t** rk_dev, size_t* coeff_off,
                   const double* coeff_dev, int sketch_digits);
int mixed_digits(double tol, int N);

namespace {

// coef[0] = 1, coef[1 + j] = -h[j] (j < k)
__global__ void gs_coeff_kernel(const double* h, int k, double* coef) {
  for (int j = threadIdx.x; j <= k; j += blockDim.x) coef[j] = (j == 0) ? 1.0 : -h[j - 1];
}

// out[0] = sqrt(max(w[0], 0))
__global__ void sqrt_kernel(const double* w, double* out) {
  if (threadIdx.x == 0) out[0] = sqrt(fmax(w[0], 0.0));
}

// nrm[0] = ||x||_F over r0 I r1 entries (ranks read on the device when given),
// then x /= nrm[0] unless it is zero. One block.
__global__ void normalize_kernel(double* x, int64_t I, int64_t r0s, int64_t r1s, const int64_t* r0p,
                                 const int64_t* r1p, double* nrm) {
  __shared__ double red[32];
  __shared__ double s_n;
  const int64_t r0 = r0p ? *r0p : r0s, r1 = r1p ? *r1p : r1s;
  const int64_t n = r0 * I * r1;
  double s = 0.0;
  for (int64_t i = threadIdx.x; i < n; i += blockDim.x) s = fma(x[i], x[i], s);
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int i = 0; i < int(blockDim.x >> 5); ++i) t += red[i];
    s_n = sqrt(t);
    nrm[0] = s_n;
  }
  __syncthreads();
  const double v = s_n;
  if (v > 0.0 && isfinite(v)) {
    const double inv = 1.0 / v;
    for (int64_t i = threadIdx.x; i < n; i += blockDim.x) x[i] *= inv;
  }
}

// Algorithm 3 of every summand of P against the TT X (ranks rx), down to the
// first core: out[j] = <Y^(j), X> (device, K doubles; the coefficients of P
// are not applied).
int build_inner(const SumProblem& P, const std::vector<int64_t>& rx, const std::vector<const double*>& X,
                double* out, Arena& ar, Schedule& sc) {
  const int N = P.N, K = P.K;
  const auto& S = P.S;
  auto In = [&](int n) { return P.I[n - 1]; };
  std::vector<double*> W(N + 1, nullptr);
  for (int n = 1; n <= N; ++n) W[n] = ar.take<double>(S[n] * rx[n]);
  W[0] = out;
  int64_t zmax = 1;
  for (int n = 1; n <= N; ++n) zmax = std::max(zmax, S[n - 1] * In(n) * rx[n]);
  double* Z = ar.take<double>(zmax);
  sc.add([=](cudaStream_t s) -> int { return fill_launch(W[N], S[N] * rx[N], 1.0, s); });
  for (int n = N; n >= 1; --n) {
    std::vector<GemmDesc> ga;
    for (int j = 0; j < K; ++j) {
      const int64_t r0 = P.r(j, n - 1), r1 = P.r(j, n);
      double* Zj = Z ? Z + P.o(j, n - 1) * In(n) * rx[n] : nullptr;
      const double* Wj = W[n] ? W[n] + P.o(j, n) * rx[n] : nullptr;
      ga.push_back(gdesc(P.core(j, n), r1, 1, Wj, rx[n], 1, Zj, rx[n], 1, r0 * In(n), rx[n], r1));
    }
    sc.gemm(ga);
    // stacked H(Z^(j)) (S_{n-1} x I_n rx_n) times H(X_n)^T
    sc.gemm({gdesc(Z, In(n) * rx[n], 1, X[n - 1], 1, In(n) * rx[n], W[n - 1], rx[n - 1], 1, S[n - 1], rx[n - 1],
                   In(n) * rx[n])});
  }
  return TT_OK;
}

int validate_single(int32_t N, const int64_t* dims, const int64_t* ranks, const double* const* cores, bool need,
                    std::vector<int64_t>* I, std::vector<int64_t>* r, std::vector<const double*>* c) {
  if (N < 1 || !dims || !ranks || (need && !cores)) {
    set_error("invalid arguments: need N >= 1 and non-null dims / ranks / cores");
    return TT_EINVAL;
  }
  I->assign(dims, dims + N);
  r->assign(ranks, ranks + N + 1);
  for (int n = 0; n < N; ++n)
    if ((*I)[n] < 1) { set_error("mode sizes must be positive"); return TT_EINVAL; }
  if ((*r)[0] != 1 || (*r)[N] != 1) { set_error("ranks must start and end with 1"); return TT_EINVAL; }
  for (int n = 0; n <= N; ++n)
    if ((*r)[n] < 1) { set_error("ranks must be positive"); return TT_EINVAL; }
  c->assign(size_t(N), nullptr);
  if (cores) {
    c->assign(cores, cores + N);
    for (auto* p : *c)
      if (!p) { set_error("null core pointer"); return TT_EINVAL; }
  }
  return TT_OK;
}

int run_checked(const BuildFn& build, void* ws, size_t ws_bytes, cudaStream_t s, const char* who) {
  int dstat = 0;
  TTR_TRY(plan_execute(build, ws, ws_bytes, s, &dstat));
  TTR_CHECK_CUDA(cudaStreamSynchronize(s));
  return status_code(dstat, who);
}

int inner_common(int32_t N, const int64_t* dims, const int64_t* ranks_x, const double* const* cores_x, int32_t K,
                 const int64_t* ranks_y, const double* const* cores_y, double* out, void* ws, size_t ws_bytes,
                 void* stream, size_t* size_only) {
  std::vector<int64_t> I, rx;
  std::vector<const double*> X;
  TTR_TRY(validate_single(N, dims, ranks_x, cores_x, size_only == nullptr, &I, &rx, &X));
  if (K < 1 || !ranks_y || (!size_only && (!cores_y || !out))) {
    set_error("tt_inner: need K >= 1, ranks_y, cores_y and out");
    return TT_EINVAL;
  }
  std::vector<int64_t> ell(N + 1, 1);
  SumProblem P;
  TTR_TRY(validate_sum(N, K, dims, ranks_y, cores_y, nullptr, ell.data(), size_only == nullptr, &P));
  BuildFn build = [&](Arena& ar, Schedule& sc) { return build_inner(P, rx, X, out, ar, sc); };
  if (size_only) return plan_workspace_bytes(build, size_only);
  return run_checked(build, ws, ws_bytes, static_cast<cudaStream_t>(stream), "tt_inner");
}

}  // namespace
}  // namespace ttr

using namespace ttr;

extern "C" {

int tt_inner(int32_t N, const int64_t* dims, const int64_t* ranks_x, const double* const* cores_x, int32_t K,
             const int64_t* ranks_y, const double* const* cores_y, double* out, void* workspace,
             size_t workspace_bytes, void* stream) {
  return inner_common(N, dims, ranks_x, cores_x, K, ranks_y, cores_y, out, workspace, workspace_bytes, stream,
                      nullptr);
}

size_t tt_inner_workspace(int32_t N, const int64_t* dims, const int64_t* ranks_x, int32_t K,
                          const int64_t* ranks_y) {
  size_t b = 0;
  if (inner_common(N, dims, ranks_x, nullptr, K, ranks_y, nullptr, nullptr, nullptr, 0, nullptr, &b) != TT_OK)
    return 0;
  return b;
}

static int norm_common(int32_t N, const int64_t* dims, const int64_t* ranks, const double* const* cores,
                       double* out, void* ws, size_t ws_bytes, void* stream, size_t* size_only) {
  std::vector<int64_t> I, rx;
  std::vector<const double*> X;
  TTR_TRY(validate_single(N, dims, ranks, cores, size_only == nullptr, &I, &rx, &X));
  if (!size_only && !out) {
    set_error("tt_norm: null output");
    return TT_EINVAL;
  }
  std::vector<int64_t> ell(N + 1, 1);
  SumProblem P;
  TTR_TRY(validate_sum(N, 1, dims, ranks, cores, nullptr, ell.data(), size_only == nullptr, &P));
  BuildFn build = [&](Arena& ar, Schedule& sc) {
    double* w0 = ar.take<double>(1);
    TTR_TRY(build_inner(P, rx, X, w0, ar, sc));
    sc.add([w0, out](cudaStream_t s) -> int {
      if (!w0) return int(TT_OK);
      sqrt_kernel<<<1, 32, 0, s>>>(w0, out);
      TTR_CHECK_LAUNCH();
      prof_count_launch(1);
      return int(TT_OK);
    });
    return int(TT_OK);
  };
  if (size_only) return plan_workspace_bytes(build, size_only);
  return run_checked(build, ws, ws_bytes, static_cast<cudaStream_t>(stream), "tt_norm");
}

int tt_norm(int32_t N, const int64_t* dims, const int64_t* ranks, const double* const* cores, double* out,
            void* workspace, size_t workspace_bytes, void* stream) {
  return norm_common(N, dims, ranks, cores, out, workspace, workspace_bytes, stream, nullptr);
}

size_t tt_norm_workspace(int32_t N, const int64_t* dims, const int64_t* ranks) {
  size_t b = 0;
  if (norm_common(N, dims, ranks, nullptr, nullptr, nullptr, 0, nullptr, &b) != TT_OK) return 0;
  return b;
}

static int gs_common(int32_t N, const int64_t* dims, const int64_t* ranks_w, const double* const* cores_w,
                     int32_t k, const int64_t* ranks_v, const double* const* cores_v, const int64_t* ells,
                     const double* const* sketch, uint64_t seed, double tol, int32_t precision, double* const* out,
                     int64_t* out_ranks, double* h, void* ws, size_t ws_bytes, void* stream, size_t* size_only) {
  if (precision != TT_PREC_FP64 && precision != TT_PREC_MIXED && precision != TT_PREC_MIXED_FULL) {
    set_error("tt_round_gram_schmidt: unknown precision mode");
    return TT_EINVAL;
  }
  std::vector<int64_t> I, rw;
  std::vector<const double*> Wc;
  TTR_TRY(validate_single(N, dims, ranks_w, cores_w, size_only == nullptr, &I, &rw, &Wc));
  if (k < 0 || (k > 0 && !ranks_v) || (!size_only && ((k > 0 && !cores_v) || !out || !out_ranks || !h))) {
    set_error("tt_round_gram_schmidt: need k >= 0, basis ranks / cores, outputs and h");
    return TT_EINVAL;
  }
  // the sum of W and the k basis tensors: summand 0 is W, summand 1 + j is V_j
  const int K = k + 1;
  std::vector<int64_t> ranks(size_t(K) * (N + 1));
  std::vector<const double*> cores(size_t(K) * N, nullptr);
  for (int n = 0; n <= N; ++n) ranks[n] = rw[n];
  for (int j = 0; j < k; ++j)
    for (int n = 0; n <= N; ++n) ranks[size_t(j + 1) * (N + 1) + n] = ranks_v[size_t(j) * (N + 1) + n];
  if (!size_only) {
    for (int n = 0; n < N; ++n) cores[n] = Wc[n];
    for (int j = 0; j < k; ++j)
      for (int n = 0; n < N; ++n) cores[size_t(j + 1) * N + n] = cores_v[size_t(j) * N + n];
  }
  SumProblem P;
  TTR_TRY(validate_sum(N, K, dims, ranks.data(), size_only ? nullptr : cores.data(), nullptr, ells,
                       size_only == nullptr, &P));
  SumProblem B;   // the basis alone (inner products against W)
  if (k > 0)
    TTR_TRY(validate_sum(N, k, dims, ranks.data() + (N + 1), size_only ? nullptr : cores.data() + N, nullptr, ells,
                         size_only == nullptr, &B));
  if (sketch)
    for (int n = 1; n < N; ++n)
      if (!sketch[n]) { set_error("null sketch core pointer"); return TT_EINVAL; }
  const int digits = (precision != TT_PREC_FP64) ? mixed_digits(tol, N) : 0;
  std::vector<double*> outv(N, nullptr);
  if (out) outv.assign(out, out + N);
  int64_t* rk_dev = nullptr;
  std::vector<int64_t> rk_host(N + 1);
  std::vector<double> h_host(size_t(k) + 1);
  BuildFn build = [&](Arena& ar, Schedule& sc) {
    double* hd = ar.take<double>(size_t(k) + 1);     // h_1..h_k, then ||Z||
    double* coef = ar.take<double>(size_t(K));
    if (k > 0) TTR_TRY(build_inner(B, rw, Wc, hd, ar, sc));
    sc.add([hd, coef, k](cudaStream_t s) -> int {
      if (!hd) return int(TT_OK);
      gs_coeff_kernel<<<1, 128, 0, s>>>(hd, k, coef);
      TTR_CHECK_LAUNCH();
      prof_count_launch(1);
      return int(TT_OK);
    });
    // the combination cancels (Z is far smaller than W and the h_j V_j): full digits in Algorithm 3 too
    TTR_TRY(build_sum_rand(P, sketch, seed, tol, digits, outv.data(), ar, sc, &rk_dev, nullptr, coef, digits));
    // ||Z|| and V_{k+1} = Z / ||Z||: with a tolerance the truncation leaves
    // cores 2..N right-orthogonal (norm in core 1, at its decided ranks);
    // without one the result is left-orthogonal (norm in core N)
    const std::vector<int64_t>& ell = P.ell;
    const bool trunc = tol > 0.0;
    double* tgt = trunc ? outv[0] : outv[N - 1];
    const int64_t In = trunc ? I[0] : I[N - 1];
    const int64_t r0s = trunc ? 1 : ell[N - 1], r1s = trunc ? ell[1] : 1;
    const int64_t* r0p = trunc && rk_dev ? rk_dev : nullptr;
    const int64_t* r1p = trunc && rk_dev ? rk_dev + 1 : nullptr;
    double* nrm = hd ? hd + k : nullptr;
    sc.add([=](cudaStream_t s) -> int {
      if (!tgt) return int(TT_OK);
      normalize_kernel<<<1, 1024, 0, s>>>(tgt, In, r0s, r1s, r0p, r1p, nrm);
      TTR_CHECK_LAUNCH();
      prof_count_launch(1);
      return int(TT_OK);
    });
    int64_t* rkh = rk_host.data();
    double* hh = h_host.data();
    const int n1 = N + 1, kk = k;
    const int64_t* rkd = rk_dev;
    sc.add([=](cudaStream_t s) -> int {
      if (!hd) return int(TT_OK);
      TTR_CHECK_CUDA(cudaMemcpyAsync(hh, hd, sizeof(double) * (kk + 1), cudaMemcpyDeviceToHost, s));
      if (rkd) TTR_CHECK_CUDA(cudaMemcpyAsync(rkh, rkd, sizeof(int64_t) * n1, cudaMemcpyDeviceToHost, s));
      return int(TT_OK);
    });
    return int(TT_OK);
  };
  if (size_only) return plan_workspace_bytes(build, size_only);
  TTR_TRY(run_checked(build, ws, ws_bytes, static_cast<cudaStream_t>(stream), "tt_round_gram_schmidt"));
  for (int n = 0; n <= N; ++n) out_ranks[n] = tol > 0.0 ? rk_host[n] : P.ell[n];
  for (int j = 0; j <= k; ++j) h[j] = h_host[j];
  return TT_OK;
}

int tt_round_gram_schmidt(int32_t N, const int64_t* dims, const int64_t* ranks_w, const double* const* cores_w,
                          int32_t k, const int64_t* ranks_v, const double* const* cores_v, const int64_t* ells,
                          const double* const* sketch, uint64_t seed, double tol, int32_t precision,
                          double* const* out, int64_t* out_ranks, double* h, void* workspace,
                          size_t workspace_bytes, void* stream) {
  return gs_common(N, dims, ranks_w, cores_w, k, ranks_v, cores_v, ells, sketch, seed, tol, precision, out,
                   out_ranks, h, workspace, workspace_bytes, stream, nullptr);
}

size_t tt_round_gram_schmidt_workspace(int32_t N, const int64_t* dims, const int64_t* ranks_w, int32_t k,
                                       const int64_t* ranks_v, const int64_t* ells, double tol, int32_t precision) {
  size_t b = 0;
  if (gs_common(N, dims, ranks_w, nullptr, k, ranks_v, nullptr, ells, nullptr, 0, tol, precision, nullptr, nullptr,
                nullptr, nullptr, 0, nullptr, &b) != TT_OK)
    return 0;
  return b;
}

static int mode_products_common(int32_t count, const int64_t* shapes, const double* const* A,
                                const double* const* cores, double* const* out, void* ws, size_t ws_bytes,
                                void* stream, size_t* size_only) {
  if (count < 0 || (count > 0 && !shapes) || (!size_only && count > 0 && (!A || !cores || !out))) {
    set_error("tt_mode_products: invalid arguments");
    return TT_EINVAL;
  }
  for (int q = 0; q < count; ++q) {
    const int64_t* sh = shapes + 4 * q;
    if (sh[0] < 1 || sh[1] < 1 || sh[2] < 1 || sh[3] < 1) {
      set_error("tt_mode_products: sizes must be positive");
      return TT_EINVAL;
    }
    if (!size_only && (!A[q] || !cores[q] || !out[q])) {
      set_error("tt_mode_products: null pointer");
      return TT_EINVAL;
    }
  }
  BuildFn build = [&](Arena&, Schedule& sc) {
    std::vector<GemmDesc> g;
    for (int q = 0; q < count; ++q) {
      const int64_t r0 = shapes[4 * q], I = shapes[4 * q + 1], r1 = shapes[4 * q + 2], J = shapes[4 * q + 3];
      // out(a, :, :) = A core(a, :, :) for every a: a (J x I)(I x r1) product batched over a
      GemmDesc d = gdesc(size_only ? nullptr : A[q], I, 1, size_only ? nullptr : cores[q], r1, 1,
                         size_only ? nullptr : out[q], r1, 1, J, r1, I);
      d.batch = int32_t(r0);
      d.a_bs = 0;
      d.b_bs = I * r1;
      d.c_bs = J * r1;
      g.push_back(d);
    }
    sc.gemm(g);
    return int(TT_OK);
  };
  if (size_only) return plan_workspace_bytes(build, size_only);
  if (count == 0) return TT_OK;
  return run_checked(build, ws, ws_bytes, static_cast<cudaStream_t>(stream), "tt_mode_products");
}

int tt_mode_products(int32_t count, const int64_t* shapes, const double* const* A, const double* const* cores,
                     double* const* out, void* workspace, size_t workspace_bytes, void* stream) {
  return mode_products_common(count, shapes, A, cores, out, workspace, workspace_bytes, stream, nullptr);
}

size_t tt_mode_products_workspace(int32_t count, const int64_t* shapes) {
  size_t b = 0;
  if (mode_products_common(count, shapes, nullptr, nullptr, nullptr, nullptr, 0, nullptr, &b) != TT_OK) return 0;
  return b;
}

}  // extern "C"

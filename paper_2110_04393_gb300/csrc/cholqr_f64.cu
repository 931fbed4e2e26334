// Thin QR by shifted Cholesky QR (Fukaya, Kannan, Nakatsukasa, Zhang,
// Kawamura, "Shifted Cholesky QR for computing the QR factorization of
// ill-conditioned matrices", SIAM J. Sci. Comput. 42 (2020)):
//   G = A^T A + s I, s = 11 (m k + k (k+1)) u ||A||_F^2,  G = R1^T R1,  Q1 = A R1^{-1};
//   then two unshifted passes (CholeskyQR2) on Q1: Q = Q1 R2^{-1} R3^{-1},
//   R = R3 R2 R1.
// It yields orthogonality and residual of order u for cond(A) up to about 1/u.
//
// Why on GB300: FP64 runs at 2 DFMA/clk/SM with long latency, so a
// Householder column step (reduction, sqrt, divide, two block barriers) is
// latency-bound and a TSQR tree puts several such factorizations in sequence.
// Here the O(m k^2) work is Gram matrices and multiplies spread over every SM by
// the grouped GEMM, and only three k x k Cholesky factorizations are
// sequential. If a pivot fails or the final Q^T Q is not the identity to
// 64 k u, a device flag is raised and the Householder TSQR (which checks that
// flag and otherwise exits at once) recomputes Q and R; no host
// synchronization is involved.
#include <algorithm>

#include "plan.cuh"
#include "prof.cuh"
#include "qr.cuh"

namespace ttr {

namespace {

constexpr int CH_THREADS = 256;

// G (k x k row-major) -> [optionally + shift] -> L L^T; writes Rinv = L^{-T}
// (upper, row-major) and, if Racc is given, Racc := L^T Racc_prev (upper).
__global__ void __launch_bounds__(CH_THREADS) chol_inv_kernel(int k, int64_t m, const double* __restrict__ G,
                                                               int shifted, double* Rinv, double* Racc,
                                                               int first, int* status) {
  extern __shared__ double sm[];
  double* L = sm;                 // k x k, row-major, lower triangle used
  double* Li = L + k * k;         // k x k, L^{-1} (lower)
  double* Rp = Li + k * k;        // k x k previous accumulated R
  __shared__ int s_fail;
  __shared__ double s_shift;
  const int tid = threadIdx.x, nt = blockDim.x;
  for (int idx = tid; idx < k * k; idx += nt) L[idx] = G[idx];
  if (tid == 0) s_fail = 0;
  __syncthreads();
  if (shifted) {
    if (tid == 0) {
      double tr = 0.0;
      for (int i = 0; i < k; ++i) tr += L[i * k + i];
      s_shift = 11.0 * (double(m) * k + double(k) * (k + 1)) * 0x1p-53 * tr;
    }
    __syncthreads();
    for (int i = tid; i < k; i += nt) L[i * k + i] += s_shift;
    __syncthreads();
  }
  // right-looking Cholesky, lower triangle
  for (int j = 0; j < k; ++j) {
    if (tid == 0) {
      const double d = L[j * k + j];
      if (!(d > 0.0) || !isfinite(d)) { s_fail = 1; L[j * k + j] = 1.0; } else L[j * k + j] = sqrt(d);
    }
    __syncthreads();
    const double piv = L[j * k + j];
    for (int i = j + 1 + tid; i < k; i += nt) L[i * k + j] /= piv;
    __syncthreads();
    const int h = k - j - 1;
    for (int idx = tid; idx < h * h; idx += nt) {
      const int i = j + 1 + idx / h, l = j + 1 + idx % h;
      if (l <= i) L[i * k + l] -= L[i * k + j] * L[l * k + j];
    }
    __syncthreads();
  }
  // L^{-1} column by column (forward substitution)
  for (int c = tid; c < k; c += nt) {
    for (int i = 0; i < c; ++i) Li[i * k + c] = 0.0;
    for (int i = c; i < k; ++i) {
      double s = (i == c) ? 1.0 : 0.0;
      for (int j = c; j < i; ++j) s -= L[i * k + j] * Li[j * k + c];
      Li[i * k + c] = s / L[i * k + i];
    }
  }
  __syncthreads();
  // Rinv = L^{-T}
  for (int idx = tid; idx < k * k; idx += nt) {
    const int r = idx / k, c = idx % k;
    Rinv[idx] = (c >= r) ? Li[c * k + r] : 0.0;
  }
  if (Racc) {
    if (!first) {
      for (int idx = tid; idx < k * k; idx += nt) Rp[idx] = Racc[idx];
      __syncthreads();
      // Racc = L^T Rp   (both upper)
      for (int idx = tid; idx < k * k; idx += nt) {
        const int r = idx / k, c = idx % k;
        double s = 0.0;
        for (int j = r; j <= c; ++j) s = fma(L[j * k + r], Rp[j * k + c], s);
        Racc[idx] = (c >= r) ? s : 0.0;
      }
    } else {
      for (int idx = tid; idx < k * k; idx += nt) {
        const int r = idx / k, c = idx % k;
        Racc[idx] = (c >= r) ? L[c * k + r] : 0.0;
      }
    }
  }
  if (tid == 0 && s_fail) atomicExch(status, 1);
}

// status := 1 unless max |G - I| <= tol
__global__ void orth_check_kernel(int k, const double* __restrict__ G, double tol, int* status) {
  __shared__ int bad;
  if (threadIdx.x == 0) bad = 0;
  __syncthreads();
  for (int idx = threadIdx.x; idx < k * k; idx += blockDim.x) {
    const int r = idx / k, c = idx % k;
    const double d = G[idx] - (r == c ? 1.0 : 0.0);
    if (!(fabs(d) <= tol)) bad = 1;
  }
  __syncthreads();
  if (threadIdx.x == 0 && bad) atomicExch(status, 1);
}

}  // namespace

QrBufs qr_reserve(Arena& ar, int64_t m, int k) {
  QrBufs b;
  b.m = m;
  b.k = k;
  b.G = ar.take<double>(int64_t(k) * k);
  b.Rinv = ar.take<double>(int64_t(k) * k);
  b.Q1 = ar.take<double>(m * k);
  b.Q2 = ar.take<double>(m * k);
  b.status = ar.take<int>(1);
  b.sh = tsqr_shape(m, k);
  size_t ii = 0;
  const size_t dd = tsqr_work_doubles(b.sh, &ii);
  b.tw = ar.take<double>(std::max<size_t>(dd, 1));
  b.ti = ar.take<int>(ii);
  b.ti_n = ii;
  return b;
}

int chol_inv_launch(int k, int64_t m, const double* G, int shifted, double* Rinv, double* Racc, int first,
                    int* status, cudaStream_t s) {
  const size_t smem = size_t(3) * k * k * sizeof(double);
  static bool attr = false;
  if (!attr) {
    TTR_CHECK_CUDA(cudaFuncSetAttribute(chol_inv_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024));
    attr = true;
  }
  chol_inv_kernel<<<1, CH_THREADS, smem, s>>>(k, m, G, shifted, Rinv, Racc, first, status);
  TTR_CHECK_LAUNCH();
  prof_count_launch(1);
  return TT_OK;
}

// Q (m x k, strides q_rs/q_cs; may alias A only if A is not needed afterwards)
// and R (k x k row-major, may be null) of A (m x k, strides a_rs/a_cs). The
// buffers of b must come from qr_reserve with the same m, k, and every region
// of b is private to this factorization while it runs.
void qr_plan(Schedule& sc, const QrBufs& b, const double* A, int64_t a_rs, int64_t a_cs, double* Q, int64_t q_rs,
             int64_t q_cs, double* R) {
  const int64_t m = b.m;
  const int k = b.k;
  const QrBufs bb = b;
  sc.add([bb](cudaStream_t s) -> int {
    if (bb.status) TTR_CHECK_CUDA(cudaMemsetAsync(bb.status, 0, sizeof(int), s));
    if (bb.ti && bb.ti_n) TTR_CHECK_CUDA(cudaMemsetAsync(bb.ti, 0, bb.ti_n * sizeof(int), s));
    return int(TT_OK);
  });
  const double* src = A;
  int64_t s_rs = a_rs, s_cs = a_cs;
  double* dsts[3] = {b.Q1, b.Q2, Q};
  int64_t d_rs[3] = {k, k, q_rs}, d_cs[3] = {1, 1, q_cs};
  for (int pass = 0; pass < 3; ++pass) {
    // G = src^T src
    sc.gemm({gdesc(src, s_cs, s_rs, src, s_rs, s_cs, b.G, k, 1, k, k, m)});
    const int shifted = (pass == 0);
    const int first = (pass == 0);
    sc.add([bb, shifted, first, R](cudaStream_t s) -> int {
      return chol_inv_launch(bb.k, bb.m, bb.G, shifted, bb.Rinv, R, first, bb.status, s);
    });
    sc.gemm({gdesc(src, s_rs, s_cs, b.Rinv, k, 1, dsts[pass], d_rs[pass], d_cs[pass], m, k, k)});
    src = dsts[pass];
    s_rs = d_rs[pass];
    s_cs = d_cs[pass];
  }
  // orthogonality check of the final Q
  sc.gemm({gdesc(Q, q_cs, q_rs, Q, q_rs, q_cs, b.G, k, 1, k, k, m)});
  const double tol = 64.0 * k * 0x1p-53;
  sc.add([bb, tol](cudaStream_t s) -> int {
    orth_check_kernel<<<1, 256, 0, s>>>(bb.k, bb.G, tol, bb.status);
    TTR_CHECK_LAUNCH();
  prof_count_launch(1);
    return int(TT_OK);
  });
  // Householder fallback, run only when the device flag is raised
  sc.add([bb, A, a_rs, a_cs, Q, q_rs, q_cs, R](cudaStream_t s) -> int {
    TsqrWork w;
    tsqr_bind(bb.sh, bb.tw, bb.ti, &w);
    return tsqr_launch(bb.sh, w, A, a_rs, a_cs, Q, q_rs, q_cs, R, s, bb.status);
  });
}

}  // namespace ttr

// Small dense SVD of an upper-triangular R and the eps-truncation rule of
// Section 2.1 ("SVD(X, eps)"), used by the truncation loop of Algorithm 2 and
// by the truncation of the left-orthogonal Randomize-then-Orthogonalize output
// (Section 3.2).
//
// The threshold is absolute (Algorithm 2 passes eps = ||Y|| eps0 / sqrt(N-1)):
// the kept rank is the smallest r >= 1 with sqrt(sum_{i>r} s_i^2) <= eps.
//
// Certified shortcut: if 1/||R^{-1}||_F > 2 eps then sigma_min(R) > eps, no
// singular value can be dropped (the tail of any r < k already exceeds eps),
// and the SVD is not needed: the step reduces to absorbing R (G1 = I, G2 = R^T).
// Otherwise: one-sided Jacobi (Hestenes) with a round-robin pair schedule, one
// warp per column pair.
#include <algorithm>

#include "kernels.cuh"
#include "prof.cuh"

namespace ttr {

namespace {

constexpr int SVD_THREADS = 1024;
constexpr int SVD_SMEM_K = 96;

__device__ __forceinline__ double warp_sum(double v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// One SVD per block. The input is scaled by the power of two 2^-sh that puts
// max |R| in [1, 2) (exact), and sigma, G2 and the threshold are taken back by
// 2^sh: sums of squares of Gaussian-TT products can otherwise underflow, which
// stalls the Jacobi convergence test. rank_out may be null.
__device__ __forceinline__ void svd_trunc_body(int k, const double* __restrict__ R, const double* __restrict__ eps_ptr, int rcap,
                               double* G1, double* G2, double* sigma, int64_t* rank_out, double* big) {
  extern __shared__ double sm[];
  const int kk = k + (k & 1);        // even number of columns for the round-robin schedule
  double* base = big ? big : sm;     // global scratch above SVD_SMEM_K
  double* A = base;                  // k x kk column-major (column k is zero padding)
  double* Vm = A + k * kk;           // kk x kk column-major
  double* sv = Vm + kk * kk;         // kk
  double* red = sv + kk;             // 32
  __shared__ int s_flag, s_rot, s_rank;
  __shared__ int order_s[128];
  int* order = big ? reinterpret_cast<int*>(red + 32) : order_s;
  const int tid = threadIdx.x, nt = blockDim.x;
  const int warp = tid >> 5, lane = tid & 31, nwarp = nt >> 5;

  __shared__ int s_emax;
  if (tid == 0) s_emax = -2000;
  __syncthreads();
  int em = -2000;
  for (int idx = tid; idx < k * kk; idx += nt) {
    const int r = idx % k, c = idx / k;
    const double v = (c < k) ? R[r * k + c] : 0.0;
    A[r + c * k] = v;
    const int e = int((uint64_t(__double_as_longlong(v)) >> 52) & 0x7FF);
    if (e != 0 && e != 0x7FF) em = max(em, e - 1023);
  }
  em = __reduce_max_sync(0xffffffffu, em);
  if (lane == 0) atomicMax(&s_emax, em);
  __syncthreads();
  const int sh = (s_emax == -2000) ? 0 : max(-1022, min(1022, s_emax));
  const double dn = __longlong_as_double((long long)(uint64_t(1023 - sh) << 52));   // 2^-sh
  const double up = __longlong_as_double((long long)(uint64_t(1023 + sh) << 52));   // 2^sh
  if (sh != 0) {
    for (int idx = tid; idx < k * kk; idx += nt) A[idx] *= dn;
    __syncthreads();
  }
  const double eps = (eps_ptr ? *eps_ptr : 0.0) * dn;

  // ---- certificate: sigma_min(R) >= 1/||R^{-1}||_F > 2 eps  =>  nothing is cut
  if (eps_ptr != nullptr && rcap >= k) {
    // R^{-1} (upper) by a right-looking backward sweep over all columns at once
    __shared__ int s_zero;
    // The diagonal reciprocals are independent (R is triangular): all of them
    // first, in parallel; then, starting from B = I, the backward
    // sweep  B(i, c) -= (R(i, j) / R(j, j)) B(j, c), i < j <= c (the scaled
    // coefficient does not depend on B, so each step has one dependent FMA),
    // and X(i, c) = B(i, c) / R(i, i) at the end. A is left untouched.
    if (tid == 0) s_zero = 0;
    __syncthreads();
    double* rdv = sv;                                        // k reciprocals (sv is free here)
    for (int j = tid; j < k; j += nt) {
      const double dj = A[j + j * k];
      if (dj == 0.0 || !isfinite(dj)) {
        s_zero = 1;
        rdv[j] = 0.0;
      } else {
        rdv[j] = 1.0 / dj;
      }
    }
    for (int idx = tid; idx < kk * kk; idx += nt) Vm[idx] = ((idx % kk) == (idx / kk)) ? 1.0 : 0.0;
    __syncthreads();
    for (int j = k - 1; j >= 1; --j) {
      // the j (k - j) entries (i < j, c >= j) packed densely over the threads:
      // an FP64 warp instruction costs the same however few lanes it has
      const double rj = rdv[j];
      for (int e = tid; e < j * (k - j); e += nt) {
        const int i = e % j, c = j + e / j;
        Vm[i + c * kk] = fma(-(A[i + j * k] * rj), Vm[j + c * kk], Vm[i + c * kk]);
      }
      __syncthreads();
    }
    for (int e = tid; e < k * k; e += nt) {
      const int i = e % k, c = e / k;
      if (i <= c) Vm[i + c * kk] *= rdv[i];
    }
    __syncthreads();
    double part = 0.0;
    for (int idx = tid; idx < k * k; idx += nt) {
      const int r = idx % k, c = idx / k;
      const double x = Vm[r + c * kk];
      part = fma(x, x, part);
    }
    const bool bad = (s_zero != 0);
    part = warp_sum(part);
    if (tid == 0) s_flag = 0;
    __syncthreads();
    if (lane == 0) red[warp] = part;
    if (bad && tid == 0) atomicOr(&s_flag, 1);
    __syncthreads();
    // R may carry a tiny strictly lower part L (first-order QR): with T its
    // upper triangle, sigma_min(R) >= 1 / ||T^{-1}||_F - ||L||_F
    __shared__ double s_tot[2];
    double low = 0.0;
    for (int idx = tid; idx < k * k; idx += nt) {
      const int r = idx % k, c = idx / k;
      if (r > c) low = fma(A[r + c * k], A[r + c * k], low);
    }
    low = warp_sum(low);
    // one thread sums the per-warp partials (an FP64 chain per warp would cost
    // every warp the FP64 pipe for the whole chain)
    if (tid == 0) {
      double t0 = 0.0;
      for (int i = 0; i < nwarp; ++i) t0 += red[i];
      s_tot[0] = t0;
    }
    __syncthreads();
    if (lane == 0) red[warp] = low;
    __syncthreads();
    if (tid == 0) {
      double t1 = 0.0;
      for (int i = 0; i < nwarp; ++i) t1 += red[i];
      s_tot[1] = t1;
    }
    __syncthreads();
    const double tot = s_tot[0], ltot = s_tot[1];
    const bool certified = !s_flag && isfinite(tot) && tot > 0.0 && (1.0 / sqrt(tot)) - sqrt(ltot) > 2.0 * eps;
    __syncthreads();
    if (certified) {
      for (int idx = tid; idx < k * k; idx += nt) {
        const int r = idx / k, c = idx % k;
        G1[idx] = (r == c) ? 1.0 : 0.0;
        G2[idx] = R[c * k + r];            // R^T
      }
      for (int i = tid; i < k; i += nt) sigma[i] = -1.0;   // not computed
      if (tid == 0 && rank_out) *rank_out = k;
      return;
    }
  }

  // ---- one-sided Jacobi: A V = U S
  for (int idx = tid; idx < kk * kk; idx += nt) Vm[idx] = ((idx % kk) == (idx / kk)) ? 1.0 : 0.0;
  __syncthreads();
  const int npairs = kk / 2;
  // a pair is orthogonal once |gamma| <= k u sqrt(alpha beta): the rounding of a
  // k-term dot product alone reaches ~sqrt(k) u, so a fixed threshold near u
  // would keep rotating noise until the sweep limit for larger k
  const double jtol = fmax(2e-15, double(k) * 0x1p-52);
  for (int sweep = 0; sweep < 60; ++sweep) {
    if (tid == 0) s_rot = 0;
    __syncthreads();
    for (int step = 0; step < kk - 1; ++step) {
      for (int pr = warp; pr < npairs; pr += nwarp) {
        const int pos_a = pr, pos_b = kk - 1 - pr;
        int p = (pos_a == 0) ? 0 : ((pos_a - 1 + step) % (kk - 1)) + 1;
        int q = ((pos_b - 1 + step) % (kk - 1)) + 1;
        if (p > q) { int t = p; p = q; q = t; }
        if (q >= k) continue;                       // padding column
        double al = 0.0, be = 0.0, ga = 0.0;
        for (int r = lane; r < k; r += 32) {
          const double x = A[r + p * k], y = A[r + q * k];
          al = fma(x, x, al);
          be = fma(y, y, be);
          ga = fma(x, y, ga);
        }
        al = warp_sum(al); be = warp_sum(be); ga = warp_sum(ga);
        if (ga == 0.0 || fabs(ga) <= jtol * sqrt(al * be)) continue;
        const double zeta = (be - al) / (2.0 * ga);
        const double t = copysign(1.0, zeta) / (fabs(zeta) + sqrt(fma(zeta, zeta, 1.0)));
        const double c = 1.0 / sqrt(fma(t, t, 1.0));
        const double s = c * t;
        for (int r = lane; r < k; r += 32) {
          const double x = A[r + p * k], y = A[r + q * k];
          A[r + p * k] = c * x - s * y;
          A[r + q * k] = s * x + c * y;
        }
        for (int r = lane; r < kk; r += 32) {
          const double x = Vm[r + p * kk], y = Vm[r + q * kk];
          Vm[r + p * kk] = c * x - s * y;
          Vm[r + q * kk] = s * x + c * y;
        }
        if (lane == 0) s_rot = 1;
      }
      __syncthreads();
    }
    if (!s_rot) break;
    __syncthreads();
  }

  // ---- singular values, descending order, rank
  for (int c = warp; c < k; c += nwarp) {
    double s = 0.0;
    for (int r = lane; r < k; r += 32) s = fma(A[r + c * k], A[r + c * k], s);
    s = warp_sum(s);
    if (lane == 0) sv[c] = sqrt(s);
  }
  __syncthreads();
  for (int i = tid; i < k; i += nt) {
    int pos = 0;
    for (int j = 0; j < k; ++j) pos += (sv[j] > sv[i]) || (sv[j] == sv[i] && j < i);
    order[pos] = i;
  }
  __syncthreads();
  if (tid == 0) {
    int r = k;
    double tail = 0.0;
    // smallest r >= 1 with sqrt(sum_{i>r} s_i^2) <= eps: walk from the end
    for (int t = k - 1; t >= 1; --t) {
      const double st = sv[order[t]];
      const double nt2 = tail + st * st;
      if (sqrt(nt2) <= eps) { tail = nt2; r = t; } else break;
    }
    if (r > rcap) r = rcap;
    if (r < 1) r = 1;
    s_rank = r;
    if (rank_out) *rank_out = r;
  }
  __syncthreads();
  const int r = s_rank;
  for (int idx = tid; idx < k * k; idx += nt) {
    const int row = idx / k, t = idx % k;
    double g1 = 0.0, g2 = 0.0;
    if (t < r) {
      const int c = order[t];
      const double s = sv[c];
      g1 = (s > 0.0) ? A[row + c * k] / s : (row == t ? 1.0 : 0.0);
      g2 = Vm[row + c * kk] * s * up;
    }
    G1[idx] = g1;
    G2[idx] = g2;
  }
  for (int t = tid; t < k; t += nt) sigma[t] = sv[order[t]] * up;
}

__global__ void __launch_bounds__(SVD_THREADS) svd_trunc_kernel(int k, const double* __restrict__ R,
                                                                const double* __restrict__ eps_ptr, int rcap,
                                                                double* G1, double* G2, double* sigma,
                                                                int64_t* rank_out, double* big,
                                                                const int* skip_if) {
  if (skip_if && __ldcg(skip_if) != 0) return;
  svd_trunc_body(k, R, eps_ptr, rcap, G1, G2, sigma, rank_out, big);
}

// B independent full SVDs (no truncation), block b on job b: k_b = kd[b]
// (stored as a double), R_b / G1_b / G2_b at b * kst * kst, sigma_b at b * kst,
// scratch at b * bst when the jobs exceed shared memory.
__global__ void __launch_bounds__(SVD_THREADS, 1) svd_batch_kernel(int kst, const double* __restrict__ kd,
                                                                const double* __restrict__ R, double* G1,
                                                                double* G2, double* sigma, double* big,
                                                                size_t bst) {
  const int b = blockIdx.x;
  const int k = int(kd[b]);
  const size_t o2 = size_t(b) * kst * kst;
  svd_trunc_body(k, R + o2, nullptr, k, G1 + o2, G2 + o2, sigma + size_t(b) * kst, nullptr,
                 big ? big + size_t(b) * bst : nullptr);
}

}  // namespace

size_t svd_scratch_doubles(int k) {
  if (k <= SVD_SMEM_K) return 0;
  const size_t kk = size_t(k + (k & 1));
  return size_t(k) * kk + kk * kk + kk + 32 + kk;   // + order (ints stored in doubles)
}

int svd_trunc_launch(int k, const double* R, const double* eps_ptr, int rcap, double* G1, double* G2,
                     double* sigma, int64_t* rank_out, cudaStream_t s, double* big, const int* skip_if) {
  if (k < 1 || (k > SVD_SMEM_K && big == nullptr)) {
    set_error("svd_trunc: k out of range or missing scratch");
    return TT_EUNSUPPORTED;
  }
  const int kk = k + (k & 1);
  const size_t smem = (k > SVD_SMEM_K) ? 0 : (size_t(k) * kk + size_t(kk) * kk + kk + 32) * sizeof(double);
  static bool attr_done = false;
  if (!attr_done) {
    TTR_CHECK_CUDA(cudaFuncSetAttribute(svd_trunc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024));
    attr_done = true;
  }
  TTR_PREFER_SHARED(svd_trunc_kernel);
  svd_trunc_kernel<<<1, SVD_THREADS, smem, s>>>(k, R, eps_ptr, rcap, G1, G2, sigma, rank_out,
                                                k > SVD_SMEM_K ? big : nullptr, skip_if);
  TTR_CHECK_LAUNCH();
  prof_count_launch(1);
  return TT_OK;
}

int svd_batch_launch(int B, int kmax, const double* kd, const double* R, double* G1, double* G2, double* sigma,
                     cudaStream_t s, double* big) {
  if (B < 1) return TT_OK;
  if (kmax < 1 || (kmax > SVD_SMEM_K && big == nullptr)) {
    set_error("svd_batch: k out of range or missing scratch");
    return TT_EUNSUPPORTED;
  }
  const int kk = kmax + (kmax & 1);
  const size_t smem = (kmax > SVD_SMEM_K) ? 0 : (size_t(kmax) * kk + size_t(kk) * kk + kk + 32) * sizeof(double);
  static bool attr_done = false;
  if (!attr_done) {
    TTR_CHECK_CUDA(cudaFuncSetAttribute(svd_batch_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024));
    attr_done = true;
  }
  TTR_PREFER_SHARED(svd_batch_kernel);
  svd_batch_kernel<<<unsigned(B), SVD_THREADS, smem, s>>>(kmax, kd, R, G1, G2, sigma,
                                                          kmax > SVD_SMEM_K ? big : nullptr,
                                                          svd_scratch_doubles(kmax));
  TTR_CHECK_LAUNCH();
  prof_count_launch(1);
  return TT_OK;
}

}  // namespace ttr

// Thin QR by Cholesky QR with an automatic shift (Fukaya, Kannan, Nakatsukasa,
// Zhang, Kawamura, "Shifted Cholesky QR for computing the QR factorization of
// ill-conditioned matrices", SIAM J. Sci. Comput. 42 (2020)):
//   pass 0: G = A^T A; Cholesky G = R1^T R1. If it breaks down, retry with
//           G + s I, s = 11 (m k + k (k+1)) u ||A||_F^2 (shifted pass).
//   pass 1: Q1 = A R1^{-1}; G = Q1^T Q1 = R2^T R2.
//   pass 2: Q2 = Q1 R2^{-1}; unshifted chain: Q2 is the result, check Q2^T Q2 = I;
//           shifted chain: G = Q2^T Q2 = R3^T R3.
//   pass 3: (shifted chain only) Q = Q2 R3^{-1}, check Q^T Q = I.
//   R = R3 R2 R1 (accumulated when asked for).
// Orthogonality and residual are of order u for cond(A) up to about 1/u.
//
// GB300 design: FP64 issues at 2 DFMA/clk/SM with long latency, so a
// Householder column step (reduction, sqrt, divide, barriers) is latency bound
// and a TSQR tree stacks several of them. Here each pass is one launch over
// ~one CTA per SM: every CTA multiplies its row block by the previous inverse
// factor, stores it, and forms its partial Gram matrix; the last CTA to arrive
// (arrival counter, no waiting) sums the partials in block order and runs the
// k x k Cholesky with the inverse formed alongside. If a pivot fails or the
// final Q^T Q misses the identity by more than 64 k u, a device flag is raised
// and the Householder TSQR (which reads that flag and otherwise exits at once)
// recomputes Q and R. No host synchronization is involved.
#include <algorithm>

#include "plan.cuh"
#include "prof.cuh"
#include "qr.cuh"

namespace ttr {

namespace {

constexpr int CQ_THREADS = 256;
constexpr int CQ_GROUP = 16;
enum { CQ_NONE = 0, CQ_CHOL_AUTO = 1, CQ_CHOL = 2, CQ_CHECK = 3 };

struct CqrPass {
  int64_t m;
  int k, b, P;
  const double* src;
  int64_t s_rs, s_cs;
  const double* Rin;        // k x k upper (row-major) applied on the right, or null
  double* dst_sh;           // destination when the chain is shifted
  int64_t dsh_rs, dsh_cs;
  double* dst_un;           // destination when the chain is unshifted
  int64_t dun_rs, dun_cs;
  int mode_sh, mode_un;
  int only_if_shifted;
  double* Gpart;            // P x k x k
  int* counter;
  double* Rinv;             // k x k out (may alias Rin)
  double* Racc;             // k x k accumulated R, or null
  int first;
  int* status;              // [0] failure, [1] shifted chain
};

// In-place right-looking Cholesky of G (k x k row-major, lower part) with
// X := L^{-1} formed alongside; returns false on a non-positive pivot.
__device__ bool chol_with_inverse(double* G, double* X, int k, double* s_rd) {
  const int tid = threadIdx.x, nt = blockDim.x;
  __shared__ int s_bad;
  for (int idx = tid; idx < k * k; idx += nt) X[idx] = ((idx / k) == (idx % k)) ? 1.0 : 0.0;
  if (tid == 0) s_bad = 0;
  __syncthreads();
  for (int j = 0; j < k; ++j) {
    if (tid == 0) {
      const double d = G[j * k + j];
      if (!(d > 0.0) || !isfinite(d)) {
        s_bad = 1;
        *s_rd = 1.0;
      } else {
        const double r = rsqrt(d);
        G[j * k + j] = d * r;
        *s_rd = r;
      }
    }
    __syncthreads();
    if (s_bad) return false;
    const double rd = *s_rd;
    for (int i = j + 1 + tid; i < k; i += nt) G[i * k + j] *= rd;
    for (int c = tid; c <= j; c += nt) X[j * k + c] *= rd;
    __syncthreads();
    const int h = k - j - 1;
    for (int idx = tid; idx < h * h; idx += nt) {
      const int i = j + 1 + idx / h, l = j + 1 + idx % h;
      if (l <= i) G[i * k + l] = fma(-G[i * k + j], G[l * k + j], G[i * k + l]);
    }
    for (int idx = tid; idx < h * (j + 1); idx += nt) {
      const int i = j + 1 + idx / (j + 1), c = idx % (j + 1);
      X[i * k + c] = fma(-G[i * k + j], X[j * k + c], X[i * k + c]);
    }
    __syncthreads();
  }
  return true;
}

__global__ void __launch_bounds__(CQ_THREADS) cqr_pass_kernel(CqrPass a) {
  extern __shared__ double sm[];
  __shared__ int s_last;
  __shared__ double s_rd;
  const int tid = threadIdx.x, nt = blockDim.x;
  const int k = a.k, b = a.b;
  const int shifted = __ldcg(a.status + 1);
  if (a.only_if_shifted && !shifted) return;
  double* dst = shifted ? a.dst_sh : a.dst_un;
  const int64_t d_rs = shifted ? a.dsh_rs : a.dun_rs, d_cs = shifted ? a.dsh_cs : a.dun_cs;
  const int mode = shifted ? a.mode_sh : a.mode_un;

  // ---- row block: T = src rows (times Rin), stored to dst, partial Gram
  double* T = sm;                 // b x k
  double* T2 = T + b * k;         // b x k
  double* Rs = T2 + b * k;        // k x k
  const int64_t r0 = int64_t(blockIdx.x) * b;
  for (int idx = tid; idx < b * k; idx += nt) {
    const int r = idx / k, c = idx % k;
    const int64_t gr = r0 + r;
    T[idx] = (gr < a.m) ? a.src[gr * a.s_rs + c * a.s_cs] : 0.0;
  }
  if (a.Rin)
    for (int idx = tid; idx < k * k; idx += nt) Rs[idx] = __ldcg(a.Rin + idx);
  __syncthreads();
  if (a.Rin) {
    for (int idx = tid; idx < b * k; idx += nt) {
      const int r = idx / k, c = idx % k;
      double s = 0.0;
      for (int j = 0; j <= c; ++j) s = fma(T[r * k + j], Rs[j * k + c], s);
      T2[idx] = s;
    }
    __syncthreads();
    T = T2;
  }
  if (dst)
    for (int idx = tid; idx < b * k; idx += nt) {
      const int r = idx / k, c = idx % k;
      const int64_t gr = r0 + r;
      if (gr < a.m) dst[gr * d_rs + c * d_cs] = T[idx];
    }
  if (mode == CQ_NONE) return;
  double* Gp = a.Gpart + int64_t(blockIdx.x) * k * k;
  for (int idx = tid; idx < k * k; idx += nt) {
    const int i = idx / k, j = idx % k;
    if (j < i) continue;
    double s = 0.0;
    for (int r = 0; r < b; ++r) s = fma(T[r * k + i], T[r * k + j], s);
    Gp[i * k + j] = s;
    Gp[j * k + i] = s;
  }
  // two-level arrival: the last CTA of each group of CQ_GROUP sums the group's
  // partials (block order) into a group partial; the last group sums those.
  __threadfence();
  __syncthreads();
  const int grp = blockIdx.x / CQ_GROUP;
  const int ngrp = (a.P + CQ_GROUP - 1) / CQ_GROUP;
  const int gsize = min(CQ_GROUP, a.P - grp * CQ_GROUP);
  if (tid == 0) {
    const int old = atomicAdd(a.counter + 1 + grp, 1);
    s_last = (old == gsize - 1);
    if (s_last) a.counter[1 + grp] = 0;
  }
  __syncthreads();
  if (!s_last) return;
  __threadfence();
  {
    double* Gg = a.Gpart + int64_t(a.P + grp) * k * k;
    const double* base = a.Gpart + int64_t(grp) * CQ_GROUP * k * k;
    for (int idx = tid; idx < k * k; idx += nt) {
      double u[8] = {0, 0, 0, 0, 0, 0, 0, 0};
      int p = 0;
      for (; p + 8 <= gsize; p += 8) {
#pragma unroll
        for (int q = 0; q < 8; ++q) u[q] += __ldcg(base + int64_t(p + q) * k * k + idx);
      }
      for (; p < gsize; ++p) u[0] += __ldcg(base + int64_t(p) * k * k + idx);
      Gg[idx] = ((u[0] + u[1]) + (u[2] + u[3])) + ((u[4] + u[5]) + (u[6] + u[7]));
    }
  }
  __threadfence();
  __syncthreads();
  if (tid == 0) {
    const int old = atomicAdd(a.counter, 1);
    s_last = (old == ngrp - 1);
    if (s_last) *a.counter = 0;
  }
  __syncthreads();
  if (!s_last) return;
  __threadfence();

  // ---- last group: G = sum of group partials in order, then Cholesky / check
  double* G = sm;                 // k x k
  double* X = G + k * k;          // k x k
  double* G0 = X + k * k;         // k x k (copy for the shifted retry / R accumulation)
  for (int idx = tid; idx < k * k; idx += nt) {
    const double* base = a.Gpart + int64_t(a.P) * k * k + idx;
    double u[4] = {0, 0, 0, 0};
    int g = 0;
    for (; g + 4 <= ngrp; g += 4) {
#pragma unroll
      for (int q = 0; q < 4; ++q) u[q] += __ldcg(base + int64_t(g + q) * k * k);
    }
    for (; g < ngrp; ++g) u[0] += __ldcg(base + int64_t(g) * k * k);
    const double sv = (u[0] + u[1]) + (u[2] + u[3]);
    G[idx] = sv;
    G0[idx] = sv;
  }
  __syncthreads();
  if (mode == CQ_CHECK) {
    __shared__ int bad;
    if (tid == 0) bad = 0;
    __syncthreads();
    const double tol = 64.0 * k * 0x1p-53;
    for (int idx = tid; idx < k * k; idx += nt) {
      const double dv = G[idx] - (((idx / k) == (idx % k)) ? 1.0 : 0.0);
      if (!(fabs(dv) <= tol)) bad = 1;
    }
    __syncthreads();
    if (tid == 0 && bad) atomicExch(a.status, 1);
    return;
  }
  bool ok = chol_with_inverse(G, X, k, &s_rd);
  if (!ok && mode == CQ_CHOL_AUTO) {
    __shared__ double s_shift;
    if (tid == 0) {
      double tr = 0.0;
      for (int i = 0; i < k; ++i) tr += G0[i * k + i];
      s_shift = 11.0 * (double(a.m) * k + double(k) * (k + 1)) * 0x1p-53 * tr;
      atomicExch(a.status + 1, 1);
    }
    __syncthreads();
    for (int idx = tid; idx < k * k; idx += nt) G[idx] = G0[idx] + (((idx / k) == (idx % k)) ? s_shift : 0.0);
    __syncthreads();
    ok = chol_with_inverse(G, X, k, &s_rd);
  }
  if (!ok) {
    if (tid == 0) atomicExch(a.status, 1);
    for (int idx = tid; idx < k * k; idx += nt) a.Rinv[idx] = ((idx / k) == (idx % k)) ? 1.0 : 0.0;
    return;
  }
  // Rinv = L^{-T} (upper)
  for (int idx = tid; idx < k * k; idx += nt) {
    const int r = idx / k, c = idx % k;
    a.Rinv[idx] = (c >= r) ? X[c * k + r] : 0.0;
  }
  if (a.Racc) {
    if (!a.first) {
      for (int idx = tid; idx < k * k; idx += nt) G0[idx] = a.Racc[idx];
      __syncthreads();
      for (int idx = tid; idx < k * k; idx += nt) {
        const int r = idx / k, c = idx % k;
        double s = 0.0;
        for (int j = r; j <= c; ++j) s = fma(G[j * k + r], G0[j * k + c], s);
        a.Racc[idx] = (c >= r) ? s : 0.0;
      }
    } else {
      for (int idx = tid; idx < k * k; idx += nt) {
        const int r = idx / k, c = idx % k;
        a.Racc[idx] = (c >= r) ? G[c * k + r] : 0.0;
      }
    }
  }
}

int cqr_launch(const CqrPass& p, cudaStream_t s) {
  const size_t smem = std::max<size_t>(size_t(2) * p.b * p.k + size_t(p.k) * p.k, size_t(3) * p.k * p.k) *
                      sizeof(double);
  static bool attr = false;
  if (!attr) {
    TTR_CHECK_CUDA(cudaFuncSetAttribute(cqr_pass_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, 220 * 1024));
    attr = true;
  }
  cqr_pass_kernel<<<p.P, CQ_THREADS, smem, s>>>(p);
  TTR_CHECK_LAUNCH();
  prof_count_launch(1);
  return TT_OK;
}

}  // namespace

QrBufs qr_reserve(Arena& ar, int64_t m, int k) {
  QrBufs b;
  b.m = m;
  b.k = k;
  const int64_t bmax = std::max<int64_t>(4, (28000 - int64_t(k) * k) / (2 * int64_t(k)));   // shared memory cap
  b.rows = int(std::min<int64_t>(bmax, std::max<int64_t>(4, ceil_div(m, num_sms()))));
  b.P = int(ceil_div(m, b.rows));
  b.Gpart = ar.take<double>(int64_t(b.P + (b.P + 15) / 16) * k * k);   // partials + group partials
  b.Rinv = ar.take<double>(int64_t(k) * k);
  b.Q1 = ar.take<double>(m * k);
  b.Q2 = ar.take<double>(m * k);
  b.status = ar.take<int>(3 + (b.P + 15) / 16);   // fail, shifted, counter, group counters
  b.sh = tsqr_shape(m, k);
  size_t ii = 0;
  const size_t dd = tsqr_work_doubles(b.sh, &ii);
  b.tw = ar.take<double>(std::max<size_t>(dd, 1));
  b.ti = ar.take<int>(ii);
  b.ti_n = ii;
  return b;
}

void qr_plan(Schedule& sc, const QrBufs& b, const double* A, int64_t a_rs, int64_t a_cs, double* Q, int64_t q_rs,
             int64_t q_cs, double* R) {
  const QrBufs bb = b;
  sc.add([bb](cudaStream_t s) -> int {
    if (!bb.status) return int(TT_OK);
    TTR_CHECK_CUDA(cudaMemsetAsync(bb.status, 0, (3 + (bb.P + 15) / 16) * sizeof(int), s));
    if (bb.ti && bb.ti_n) TTR_CHECK_CUDA(cudaMemsetAsync(bb.ti, 0, bb.ti_n * sizeof(int), s));
    return int(TT_OK);
  });
  CqrPass base{};
  base.m = b.m;
  base.k = b.k;
  base.b = b.rows;
  base.P = b.P;
  base.Gpart = b.Gpart;
  base.counter = b.status ? b.status + 2 : nullptr;
  base.Rinv = b.Rinv;
  base.Racc = R;
  base.status = b.status;
  const int k = b.k;
  // pass 0: Gram of A, Cholesky (shift on breakdown)
  CqrPass p0 = base;
  p0.src = A; p0.s_rs = a_rs; p0.s_cs = a_cs;
  p0.mode_sh = p0.mode_un = CQ_CHOL_AUTO;
  p0.first = 1;
  // pass 1: Q1 = A R1^{-1}, Gram, Cholesky
  CqrPass p1 = base;
  p1.src = A; p1.s_rs = a_rs; p1.s_cs = a_cs; p1.Rin = b.Rinv;
  p1.dst_sh = p1.dst_un = b.Q1; p1.dsh_rs = p1.dun_rs = k; p1.dsh_cs = p1.dun_cs = 1;
  p1.mode_sh = p1.mode_un = CQ_CHOL;
  // pass 2: Q2 = Q1 R2^{-1}; final (check) unless the chain was shifted
  CqrPass p2 = base;
  p2.src = b.Q1; p2.s_rs = k; p2.s_cs = 1; p2.Rin = b.Rinv;
  p2.dst_sh = b.Q2; p2.dsh_rs = k; p2.dsh_cs = 1;
  p2.dst_un = Q; p2.dun_rs = q_rs; p2.dun_cs = q_cs;
  p2.mode_sh = CQ_CHOL;
  p2.mode_un = CQ_CHECK;
  // pass 3: shifted chain only
  CqrPass p3 = base;
  p3.src = b.Q2; p3.s_rs = k; p3.s_cs = 1; p3.Rin = b.Rinv;
  p3.dst_sh = p3.dst_un = Q; p3.dsh_rs = p3.dun_rs = q_rs; p3.dsh_cs = p3.dun_cs = q_cs;
  p3.mode_sh = p3.mode_un = CQ_CHECK;
  p3.only_if_shifted = 1;
  for (const CqrPass* p : {&p0, &p1, &p2, &p3}) {
    const CqrPass pp = *p;
    sc.add([pp](cudaStream_t s) -> int { return cqr_launch(pp, s); });
  }
  // Householder fallback, run only when the device flag is raised
  sc.add([bb, A, a_rs, a_cs, Q, q_rs, q_cs, R](cudaStream_t s) -> int {
    TsqrWork w;
    tsqr_bind(bb.sh, bb.tw, bb.ti, &w);
    return tsqr_launch(bb.sh, w, A, a_rs, a_cs, Q, q_rs, q_cs, R, s, bb.status);
  });
}

}  // namespace ttr

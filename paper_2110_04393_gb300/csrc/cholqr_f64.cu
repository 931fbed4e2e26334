// Thin QR by Cholesky QR with automatic shifts (Fukaya, Kannan, Nakatsukasa,
// Zhang, Kawamura, "Shifted Cholesky QR for computing the QR factorization of
// ill-conditioned matrices", SIAM J. Sci. Comput. 42 (2020)). A chain of
// passes; pass 0 factors G = A^T A, every later pass multiplies the current
// block by the previous inverse factor and factors its Gram matrix:
//   * when only Q is wanted and a later Gram is I + E with ||E||_F <= 1e-8,
//     the next pass multiplies by I - E/2 and ends the chain (Q^T Q - I is
//     then O(||E||^2), below the rounding level), saving a factorization;
//   * a factorization that breaks down is retried with G + s I,
//     s = 11 (m k + k (k+1)) u ||.||_F^2 (a shifted pass);
//   * once two consecutive factorizations were unshifted, the next pass writes
//     the final Q and checks Q^T Q = I to 64 k u.
// So a well-conditioned A takes CholeskyQR2 (3 passes), cond(A) up to 1/u takes
// shifted CholeskyQR3 (4 passes), and an exactly rank-deficient A (zero singular
// values met when a target rank exceeds the true rank) takes up to two shifts:
// its null directions come out as orthonormal round-off directions, as with
// Householder. R = R_last ... R_1 is accumulated when asked for. Six passes are
// launched; passes after the final one exit at once.
//
// GB300 design: FP64 issues at 2 DFMA/clk/SM with long latency, so a
// Householder column step (reduction, sqrt, divide, barriers) is latency bound
// and a TSQR tree stacks several of them. Here each pass is one launch over
// ~one CTA per SM: every CTA multiplies its row block by the previous inverse
// factor, stores it, and forms its partial Gram matrix; the last CTA to arrive
// (arrival counters, two levels, no waiting) sums the partials in block order
// and runs the k x k Cholesky with the inverse formed alongside (in shared
// memory for k <= 96, in global scratch above). If the final check fails, a
// device flag is raised: for k <= 96 the Householder TSQR (which reads that
// flag and otherwise exits at once) recomputes Q and R; above, the flag is
// reported to the caller. No host synchronization is involved.
#include <algorithm>
#include <atomic>
#include <cstring>

#include "plan.cuh"
#include "prof.cuh"
#include "qr.cuh"

namespace ttr {

namespace {

constexpr int CQ_THREADS = 256;
constexpr int CQ_GROUP = 16;
constexpr int CQ_SMEM_K = 96;   // above this the k x k factors live in global scratch

constexpr int CQ_MAX_PASSES = 6;

// Row stride of a row block in shared memory: odd, so that the lanes of a warp
// reading one column of consecutive rows hit distinct banks for every k.
__host__ __device__ inline int cq_ts(int k) { return k | 1; }

struct CqrPass {
  int64_t m;
  int k, b, P, pass;
  int fo_r;                 // the first-order last pass may also update the R factor (R no longer triangular)
  const double* A;          // input
  int64_t a_rs, a_cs;
  double* buf[2];           // m x k ping-pong blocks (row-major)
  double* Q;                // final Q
  int64_t q_rs, q_cs;
  double* Gpart;            // (P + groups) x k (k + 1) / 2 (packed upper triangles)
  int* counter;             // [0] final arrival, [1 + g] group arrivals
  double* Rinv;             // k x k (upper, row-major)
  double* Racc;             // k x k accumulated R, or null
  double* big;              // 3 k x k global scratch when k > CQ_SMEM_K (else null)
  int* status;              // [0] failure, [1] unshifted run, [2] done, [3] factorizations so far,
                            // [4] the next pass multiplies by a first-order correction and ends the chain
};

// A usable pivot: positive, finite and normal, decided on the bit pattern
// (integer operations instead of FP64 compares on the critical path).
__device__ __forceinline__ bool pivot_ok(double d) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(d);
  const unsigned e = unsigned(b >> 52);            // sign and exponent
  return e != 0 && e < 0x7FFu;                     // sign 0, exponent neither 0 nor all ones
}

// In-place right-looking Cholesky of G (k x k row-major, lower part) with
// X := L^{-1} formed alongside; returns false on a non-positive pivot. FP64
// issues a dependent operation only every ~65 cycles on GB300 and a reciprocal
// square root takes ~400, so the pivot chain is the critical path, and every
// step has exactly one block barrier:
//   * thread 0 (alone on its SM sub-partition) turns the still unscaled
//     column entry g = G(j+1, j) into the next pivot d = G(j+1, j+1) -
//     (g rd_j)^2 and its reciprocal square root rd_{j+1};
//   * meanwhile the other three sub-partitions update the trailing lower
//     triangle G(i, l) -= (G(i, j) rd_j)(G(l, j) rd_j) and the rows of X below
//     j, X(i, c) -= G(i, j) rd_j^2 X(j, c) with X's row j still unscaled, all
//     packed densely over lanes, and finalise the previous step's column of L
//     (G(i, j-1) rd_{j-1}) and row of X (X(j-1, :) rd_{j-1}), which no step
//     reads any more.
// rd and the pivot test are double-buffered across the barrier.
// blockDim.x must be a multiple of 128.
__device__ bool chol_with_inverse(double* G, double* X, int k) {
  __shared__ double rdb[2];
  __shared__ int badb[2];
  const int tid = threadIdx.x, nt = blockDim.x, warp = tid >> 5, lane = tid & 31;
  const bool worker = (warp & 3) != 0;
  const int nwk = (nt >> 5) / 4 * 3 * 32;                           // worker threads
  const int wid = ((warp >> 2) * 3 + (warp & 3) - 1) * 32 + lane;   // valid for workers
  for (int e = tid; e < k * k; e += nt) X[e] = (e % (k + 1) == 0) ? 1.0 : 0.0;
  if (tid == 0) {
    const double d = G[0];
    const bool bad = !pivot_ok(d);
    badb[0] = bad ? 1 : 0;
    rdb[0] = bad ? 1.0 : rsqrt(d);
  }
  __syncthreads();
  double rprev = 1.0;
  for (int j = 0; j < k; ++j) {
    if (badb[j & 1]) return false;
    const double rd = rdb[j & 1];
    const double rd2 = rd * rd;
    const int n = k - j - 1;                      // rows / columns below the pivot
    const int ng = n * (n + 1) / 2, nx = n * (j + 1);
    if (tid == 0) {
      G[j * k + j] = G[j * k + j] * rd;           // L(j, j) = sqrt(d_j)
      if (n > 0) {
        const double g = G[(j + 1) * k + j] * rd;
        const double d = fma(-g, g, G[(j + 1) * k + j + 1]);
        G[(j + 1) * k + j + 1] = d;
        const bool bad = !pivot_ok(d);
        badb[(j + 1) & 1] = bad ? 1 : 0;
        rdb[(j + 1) & 1] = bad ? 1.0 : rsqrt(d);
      }
    } else if (worker) {
      // the previous step's column of L and row of X are final now
      if (j > 0) {
        for (int i = j + wid; i < k; i += nwk) G[i * k + (j - 1)] *= rprev;
        for (int c = wid; c < j; c += nwk) X[(j - 1) * k + c] *= rprev;
      }
      // entry 0 of the packed lower triangle is the next diagonal (thread 0's)
      for (int e = wid + 1; e < ng + nx; e += nwk) {
        if (e < ng) {
          int ip = int((sqrtf(8.0f * float(e) + 1.0f) - 1.0f) * 0.5f);
          while (ip * (ip + 1) / 2 > e) --ip;
          while ((ip + 1) * (ip + 2) / 2 <= e) ++ip;
          const int i = j + 1 + ip, l = j + 1 + (e - ip * (ip + 1) / 2);
          G[i * k + l] = fma(-(G[i * k + j] * rd2), G[l * k + j], G[i * k + l]);
        } else {
          const int e2 = e - ng;
          const int i = j + 1 + e2 / (j + 1), c = e2 % (j + 1);
          X[i * k + c] = fma(-(G[i * k + j] * rd2), X[j * k + c], X[i * k + c]);
        }
      }
    }
    rprev = rd;
    __syncthreads();
  }
  // the last step's column of L is empty; its row of X needs the scaling
  for (int c = tid; c < k; c += nt) X[(k - 1) * k + c] *= rprev;
  __syncthreads();
  return true;
}

// 1/sqrt(d) for a positive normal d: the hardware approximation y of
// rsqrt.approx.ftz.f64 (relative error below 2^-20) corrected by the
// third-order terms of the binomial series (1 - e)^(-1/2) = 1 + e/2 + 3e^2/8 +
// O(e^3), e = 1 - d y^2 (Householder's method of order 2); the neglected term is
// below 2^-58, so the result is within rounding of 1/sqrt(d). Five FP64
// operations after the approximation instead of the longer IEEE sequence:
// this is the pivot chain's critical step.
__device__ __forceinline__ double rsqrt_refined(double d) {
  double y;
  asm("rsqrt.approx.ftz.f64 %0, %1;" : "=d"(y) : "d"(d));
  const double t = d * y;
  const double e = fma(-t, y, 1.0);
  const double p = fma(0.375, e, 0.5);
  const double r = y * e;
  return fma(r, p, y);
}

// The same Cholesky with inverse for k <= 32 * NQ with G and X in shared
// memory, scheduled for GB300's FP64 issue: one warp issues one FP64
// instruction per ~64 cycles whether or not its lanes are active, and the SM
// retires ~1.7 FP64 lanes per clock, so work is packed densely into few warp
// instructions and nothing but the pivot chain waits on warp 0.
//   * warp 0 (look-ahead): in step j it applies column j to column j+1 and to
//     row j+1 of X (k entries, one lane each), takes the pivot d_{j+1} from
//     lane 0, its reciprocal square root, and stores column j+1 of L and row
//     j+1 of X scaled: L(j+1, j+1) = d rd, L(i, j+1) = G(i, j+1) rd,
//     X(j+1, :) = X(j+1, :) rd, X(j+1, j+1) = rd. The multipliers it needs
//     next are the vector it just stored, shifted down by one entry with rd
//     last, so it keeps that vector in registers: after the barrier it loads
//     only the entries the workers updated;
//   * the worker warps (all others) apply column j to rows i >= j+2, each warp
//     the rows i = w + 2 (mod number of workers): row i has exactly i entries
//     to update, X(i, 0..j) and G(i, j+2..i), so one warp instruction covers a
//     row (lane = position); the multiplied column / row of step j is loaded
//     once per step and warp.
// One block barrier per step; blockDim.x a multiple of 32, at least 64.
template <int NQ>
__device__ bool chol_la(double* G, double* X, int k) {
  __shared__ int s_bad;
  const int tid = threadIdx.x, nt = blockDim.x, warp = tid >> 5, lane = tid & 31;
  const int nww = (nt >> 5) - 1;
  for (int r = warp; r < k; r += (nt >> 5))
    for (int c = lane; c < k; c += 32) X[r * k + c] = (r == c) ? 1.0 : 0.0;
  __syncthreads();
  // warp 0 state for the next step j: multipliers a (entry t: L(j + 1 + t, j)
  // for t < k - 1 - j, then X(j, t - (k - 1 - j))), l1 = L(j + 1, j), and the
  // entries' locations in column j + 1 / row j + 1 of X
  double a[NQ], l1 = 0.0, rd = 1.0;
  double* dst[NQ];
  auto next = [&](const double(&o)[NQ], int j) {
    const int n = k - 1 - j;
#pragma unroll
    for (int q = 0; q < NQ; ++q) {
      const double s = __shfl_down_sync(0xffffffffu, o[q], 1);
      const double h = __shfl_sync(0xffffffffu, o[q + 1 < NQ ? q + 1 : q], 0);
      const int t = lane + 32 * q;
      a[q] = (t == k - 1) ? rd : ((lane == 31) ? h : s);
      const int tc = t < k ? t : k - 1;
      dst[q] = tc < n ? G + (j + 1 + tc) * k + j + 1 : X + (j + 1) * k + (tc - n);
    }
    l1 = __shfl_sync(0xffffffffu, o[0], 1);
  };
  if (warp == 0) {
    const double d = G[0];
    const bool bad = !pivot_ok(d);
    rd = bad ? 1.0 : rsqrt_refined(d);
    double o[NQ];
#pragma unroll
    for (int q = 0; q < NQ; ++q) {
      const int t = lane + 32 * q;
      o[q] = G[(t < k ? t : k - 1) * k] * rd;
      if (t < k) G[t * k] = o[q];
    }
    if (lane == 0) {
      X[0] = rd;
      s_bad = bad ? 1 : 0;
    }
    next(o, 0);
  }
  int iw = warp + 1;                             // worker: its smallest row >= j + 2
  __syncthreads();
  for (int j = 0; j + 1 < k; ++j) {
    if (s_bad) return false;
    if (warp == 0) {
      double v[NQ], o[NQ];
#pragma unroll
      for (int q = 0; q < NQ; ++q) v[q] = fma(-a[q], l1, *dst[q]);
      const double d = __shfl_sync(0xffffffffu, v[0], 0);
      const bool bad = !pivot_ok(d);
      rd = bad ? 1.0 : rsqrt_refined(d);
#pragma unroll
      for (int q = 0; q < NQ; ++q) {
        o[q] = v[q] * rd;
        if (lane + 32 * q < k) *dst[q] = o[q];
      }
      if (lane == 0) {
        X[(j + 1) * k + j + 1] = rd;
        if (bad) s_bad = 1;
      }
      if (j + 2 < k) next(o, j + 1);
    } else {
      // position p < j + 1 of row i is X(i, p), the rest G(i, p + 1)
      if (iw < j + 2) iw += nww;
      double b[NQ];
#pragma unroll
      for (int q = 0; q < NQ; ++q) {
        const int pb = min(lane + 32 * q, k - 2);
        b[q] = pb <= j ? X[j * k + pb] : G[(pb + 1) * k + j];
      }
      constexpr int RB = NQ == 1 ? 4 : 2;        // rows per batch: loads first, then FMAs
      for (int i = iw; i < k; i += RB * nww) {
        double ar[RB], c[RB][NQ];
#pragma unroll
        for (int r = 0; r < RB; ++r) {
          const int ir = min(i + r * nww, k - 1);
          ar[r] = G[ir * k + j];
#pragma unroll
          for (int q = 0; q < NQ; ++q) {
            const int pc = min(lane + 32 * q, ir - 1);
            c[r][q] = pc <= j ? X[ir * k + pc] : G[ir * k + pc + 1];
          }
        }
#pragma unroll
        for (int r = 0; r < RB; ++r) {
          const int ir = i + r * nww;
          if (ir < k) {
#pragma unroll
            for (int q = 0; q < NQ; ++q) {
              const int p = lane + 32 * q;
              const double ov = fma(-ar[r], b[q], c[r][q]);
              if (p < ir) {
                if (p <= j) X[ir * k + p] = ov;
                else G[ir * k + p + 1] = ov;
              }
            }
          }
        }
      }
    }
    __syncthreads();
  }
  return s_bad == 0;
}

// Cholesky with inverse: the scheduled form in shared memory for k <= 96, the
// general one (shared or global scratch) above.
__device__ bool chol_inverse(double* G, double* X, int k) {
  if (k <= 32) return chol_la<1>(G, X, k);
  if (k <= 64) return chol_la<2>(G, X, k);
  if (k <= CQ_SMEM_K) return chol_la<3>(G, X, k);
  return chol_with_inverse(G, X, k);
}

// Sum of two values over the block (blockDim.x a multiple of 32, at most
// 1024): shuffle trees within the warps and over the warp partials, result in
// every thread. FP64 adds cost ~64 cycles each, so no serial loop anywhere.
__device__ __forceinline__ void block_sum2(double* a, double* b) {
  __shared__ double s_part[2][32];
  __shared__ double s_tot[2];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  double x = *a, y = *b;
  for (int off = 16; off; off >>= 1) {
    x += __shfl_xor_sync(0xffffffffu, x, off);
    y += __shfl_xor_sync(0xffffffffu, y, off);
  }
  if (lane == 0) {
    s_part[0][warp] = x;
    s_part[1][warp] = y;
  }
  __syncthreads();
  if (warp == 0) {
    x = lane < nw ? s_part[0][lane] : 0.0;
    y = lane < nw ? s_part[1][lane] : 0.0;
    for (int off = 16; off; off >>= 1) {
      x += __shfl_xor_sync(0xffffffffu, x, off);
      y += __shfl_xor_sync(0xffffffffu, y, off);
    }
    if (lane == 0) {
      s_tot[0] = x;
      s_tot[1] = y;
    }
  }
  __syncthreads();
  *a = s_tot[0];
  *b = s_tot[1];
}

// Position (i, j), i <= j, of entry p of the row-wise packed upper triangle.
__device__ __forceinline__ void tri_ij(int p, int k, int* i, int* j) {
  int r = 0;
  while (p >= k - r) { p -= k - r; ++r; }
  *i = r;
  *j = r + p;
}

// Decision of one pass of the chain on the reduced Gram matrix G (k x k,
// copy in G0, X is scratch; all three in the calling CTA's shared memory or
// in global scratch), made by one whole CTA:
//   * final pass: check G = I to 64 k u (failure raises status[0]) and end;
//   * a later Gram I + E with ||E||_F <= 1e-8 (only Q wanted, or R may come out
//     full): Rinv := I - E/2 and the next pass ends the chain;
//   * else the Cholesky factorization with inverse (retried once with a shift),
//     Rinv := L^{-T} and R accumulated when asked for; a failure raises
//     status[0] and ends the chain.
// Returns after the CTA's last write (callers synchronize before publishing).
__device__ void cqr_decide(double* G, double* X, double* G0, int k, int64_t m, int pass, bool final_pass,
                           int unshifted_run, double* Rinv, double* Racc, int fo_r, int* status,
                           double e2_pre = -1.0) {
  const int tid = threadIdx.x, nt = blockDim.x;
  if (final_pass) {
    __shared__ int bad;
    if (tid == 0) bad = 0;
    __syncthreads();
    const double tol = 64.0 * k * 0x1p-53;
    const int lane = tid & 31, nw = nt >> 5;
    for (int r = tid >> 5; r < k; r += nw)
      for (int c = lane; c < k; c += 32) {
        const double dv = G[r * k + c] - (r == c ? 1.0 : 0.0);
        if (!(fabs(dv) <= tol)) bad = 1;
      }
    __syncthreads();
    if (tid == 0) {
      if (bad) atomicExch(status, 1);
      atomicExch(status + 2, 1);
    }
    return;
  }
  if (pass > 0 && (Racc == nullptr || fo_r)) {
    // The block is already orthonormal to ||E||_F <= 1e-8, E = G - I: the last
    // pass multiplies by I - E/2 instead of factoring again. When R is wanted
    // (and allowed to lose its triangular form) it becomes (I + E/2) R: the
    // correction E R / 2 is ~1e-8 of R or less, so an fp32 product of it keeps R
    // accurate to float64 rounding.
    const int lane = tid & 31, nw = nt >> 5;
    double tot = e2_pre;
    if (!(tot >= 0.0)) {
      double e2 = 0.0, unused = 0.0;
      for (int r = tid >> 5; r < k; r += nw)
        for (int c = lane; c < k; c += 32) {
          const double dv = G[r * k + c] - (r == c ? 1.0 : 0.0);
          e2 = fma(dv, dv, e2);
        }
      block_sum2(&e2, &unused);
      tot = e2;
    }
    if (tot <= 1e-16) {                           // ||E||_F <= 1e-8 (false for NaN)
      // I - E/2 = 1.5 I - G/2: one rounding of the same exact value
      for (int r = tid >> 5; r < k; r += nw)
        for (int c = lane; c < k; c += 32) Rinv[r * k + c] = fma(-0.5, G[r * k + c], r == c ? 1.5 : 0.0);
      if (Racc) {
        // X <- E / 2, G0 <- R (the previous factor), then R += (E / 2) R with R
        // scaled by a power of two near 1 / max|R| for the fp32 product (no
        // underflow or overflow in fp32 whatever the scale of A)
        __shared__ int s_emax;
        if (tid == 0) s_emax = -2000;
        __syncthreads();
        int em = -2000;
        for (int idx = tid; idx < k * k; idx += nt) {
          X[idx] = 0.5 * (G[idx] - ((idx % (k + 1) == 0) ? 1.0 : 0.0));
          const double r = Racc[idx];
          G0[idx] = r;
          const int e = int((uint64_t(__double_as_longlong(r)) >> 52) & 0x7FF);
          if (e != 0) em = max(em, e - 1023);
        }
        atomicMax(&s_emax, em);
        __syncthreads();
        const int sh = s_emax == -2000 ? 0 : -s_emax;                 // R 2^sh has entries below 2
        const double up = __longlong_as_double((long long)(uint64_t(1023 - sh) << 52));   // 2^{-sh}
        const double down = __longlong_as_double((long long)(uint64_t(1023 + sh) << 52)); // 2^{sh}
        // fp32 copies first (conversions run on the FP64 pipe: once per entry),
        // in the memory of G, which is no longer needed (2 k^2 floats = k^2 doubles)
        float* Xf = reinterpret_cast<float*>(G);                 // E / 2
        float* Rf = Xf + k * k;                                  // R 2^sh
        __syncthreads();
        for (int idx = tid; idx < k * k; idx += nt) {
          Xf[idx] = float(X[idx]);
          Rf[idx] = float(G0[idx] * down);
        }
        __syncthreads();
        for (int idx = tid; idx < k * k; idx += nt) {
          const int r = idx / k, c = idx % k;
          float corr = 0.0f;
          for (int l = 0; l < k; ++l) corr = fmaf(Xf[r * k + l], Rf[l * k + c], corr);
          Racc[idx] = fma(double(corr), up, G0[idx]);
        }
      }
      if (tid == 0) {
        status[4] = (tot <= 1e-20) ? 2 : 1;       // 2: ||E||_F <= 1e-10, an fp32 product of E suffices
        status[1] = 2;
        status[3] += 1;
      }
      return;
    }
  }
  bool ok = chol_inverse(G, X, k);
  bool shifted = false;
  if (!ok) {
    __shared__ double s_shift;
    if (tid == 0) {
      double tr = 0.0;
      for (int i = 0; i < k; ++i) tr += G0[i * k + i];
      s_shift = 11.0 * (double(m) * k + double(k) * (k + 1)) * 0x1p-53 * tr;
    }
    __syncthreads();
    for (int idx = tid; idx < k * k; idx += nt) G[idx] = G0[idx] + (((idx / k) == (idx % k)) ? s_shift : 0.0);
    __syncthreads();
    ok = chol_inverse(G, X, k);
    shifted = true;
  }
  if (!ok) {                                    // not even the shifted Gram is positive definite
    if (tid == 0) {
      atomicExch(status, 1);
      atomicExch(status + 2, 1);
    }
    return;
  }
  if (tid == 0) {
    status[1] = shifted ? 0 : unshifted_run + 1;
    status[3] += 1;
  }
  // Rinv = L^{-T} (upper)
  for (int idx = tid; idx < k * k; idx += nt) {
    const int r = idx / k, c = idx % k;
    Rinv[idx] = (c >= r) ? X[c * k + r] : 0.0;
  }
  if (Racc) {
    if (pass > 0) {
      for (int idx = tid; idx < k * k; idx += nt) G0[idx] = Racc[idx];
      __syncthreads();
      for (int idx = tid; idx < k * k; idx += nt) {
        const int r = idx / k, c = idx % k;
        double s = 0.0;
        for (int j = r; j <= c; ++j) s = fma(G[j * k + r], G0[j * k + c], s);
        Racc[idx] = (c >= r) ? s : 0.0;
      }
    } else {
      for (int idx = tid; idx < k * k; idx += nt) {
        const int r = idx / k, c = idx % k;
        Racc[idx] = (c >= r) ? G[c * k + r] : 0.0;
      }
    }
  }
}

__device__ __forceinline__ void cqr_pass_body(const CqrPass& a, const int blk) {
  extern __shared__ double sm[];
  __shared__ int s_last;
  const int tid = threadIdx.x, nt = blockDim.x;
  const int k = a.k, b = a.b;
  if (__ldcg(a.status + 2)) return;                         // chain already finished
  const int unshifted_run = __ldcg(a.status + 1);
  const bool first_order = __ldcg(a.status + 4) != 0;
  const bool final_pass = (a.pass > 0) && (unshifted_run >= 2 || a.pass == CQ_MAX_PASSES - 1);
  const double* src = (a.pass <= 1) ? a.A : a.buf[(a.pass - 2) & 1];
  const int64_t s_rs = (a.pass <= 1) ? a.a_rs : k, s_cs = (a.pass <= 1) ? a.a_cs : 1;
  double* dst = (a.pass == 0) ? nullptr : (final_pass ? a.Q : a.buf[(a.pass - 1) & 1]);
  const int64_t d_rs = final_pass ? a.q_rs : k, d_cs = final_pass ? a.q_cs : 1;
  const bool big = (a.big != nullptr);

  // ---- row block: T = src rows (times R^{-1} of the previous pass), stored, partial Gram
  const int ts = cq_ts(k);
  double* T = sm;                 // b x k, row stride ts
  double* T2 = T + b * ts;        // b x k, row stride ts
  double* Rs = T2 + b * ts;       // k x k (shared when small)
  const double* Rin = (a.pass == 0) ? nullptr : a.Rinv;
  const int64_t r0 = int64_t(blk) * b;
  const int lane = tid & 31, warp = tid >> 5, nw = nt >> 5;
  for (int r = warp; r < b; r += nw) {
    const int64_t gr = r0 + r;
    for (int c = lane; c < k; c += 32) T[r * ts + c] = (gr < a.m) ? src[gr * s_rs + c * s_cs] : 0.0;
  }
  if (Rin && !big)
    for (int i = warp; i < k; i += nw)
      for (int c = lane; c < k; c += 32) Rs[i * k + c] = __ldcg(Rin + i * k + c);
  __syncthreads();
  if (Rin) {
    // T2 = T R^{-1} (R^{-1} upper; a first-order correction I - E/2 is a full
    // matrix: all k terms): one output entry per item, four independent
    // partial sums, items down the columns so that the lanes of a warp share
    // the length c + 1 of their sums (a warp instruction costs the same
    // whatever its active lanes)
    const double* Rr = big ? Rin : Rs;
    for (int i = tid; i < b * k; i += nt) {
      const int c = i / b, r = i - c * b;
      const int jn = first_order ? k : c + 1;
      const double* tr = T + r * ts;
      double s0 = 0.0, s1 = 0.0, s2 = 0.0, s3 = 0.0;
      int j = 0;
      if (big) {
        for (; j + 4 <= jn; j += 4) {
          s0 = fma(tr[j], __ldcg(Rr + j * k + c), s0);
          s1 = fma(tr[j + 1], __ldcg(Rr + (j + 1) * k + c), s1);
          s2 = fma(tr[j + 2], __ldcg(Rr + (j + 2) * k + c), s2);
          s3 = fma(tr[j + 3], __ldcg(Rr + (j + 3) * k + c), s3);
        }
        for (; j < jn; ++j) s0 = fma(tr[j], __ldcg(Rr + j * k + c), s0);
      } else {
        for (; j + 4 <= jn; j += 4) {
          s0 = fma(tr[j], Rr[j * k + c], s0);
          s1 = fma(tr[j + 1], Rr[(j + 1) * k + c], s1);
          s2 = fma(tr[j + 2], Rr[(j + 2) * k + c], s2);
          s3 = fma(tr[j + 3], Rr[(j + 3) * k + c], s3);
        }
        for (; j < jn; ++j) s0 = fma(tr[j], Rr[j * k + c], s0);
      }
      T2[r * ts + c] = (s0 + s1) + (s2 + s3);
    }
    __syncthreads();
    T = T2;
  }
  if (dst)
    for (int r = warp; r < b; r += nw) {
      const int64_t gr = r0 + r;
      if (gr < a.m)
        for (int c = lane; c < k; c += 32) dst[gr * d_rs + c * d_cs] = T[r * ts + c];
    }
  if (final_pass && first_order) {
    // Q = Q1 (I - E/2) with ||E||_F <= 1e-8 has Q^T Q = I + O(||E||^2): no check needed
    if (tid == 0) atomicExch(a.status + 2, 1);
    return;
  }
  // partial Gram, upper triangle packed row-wise (npair entries)
  const int npair = k * (k + 1) / 2;
  double* Gp = a.Gpart + int64_t(blk) * npair;
  for (int p = tid; p < npair; p += 2 * nt) {
    int i1, j1, i2 = 0, j2 = 0;
    tri_ij(p, k, &i1, &j1);
    const bool two = p + nt < npair;
    if (two) tri_ij(p + nt, k, &i2, &j2);
    double g1 = 0.0, g2 = 0.0;
    for (int r = 0; r < b; ++r) {
      g1 = fma(T[r * ts + i1], T[r * ts + j1], g1);
      if (two) g2 = fma(T[r * ts + i2], T[r * ts + j2], g2);
    }
    Gp[p] = g1;
    if (two) Gp[p + nt] = g2;
  }
  // two-level arrival: the last CTA of each group of CQ_GROUP sums the group's
  // partials (block order) into a group partial; the last group sums those.
  __syncthreads();
  const int grp = blk / CQ_GROUP;
  const int ngrp = (a.P + CQ_GROUP - 1) / CQ_GROUP;
  const int gsize = min(CQ_GROUP, a.P - grp * CQ_GROUP);
  if (tid == 0) {
    const int old = atom_add_acq_rel_gpu(a.counter + 1 + grp, 1);
    s_last = (old == gsize - 1);
    if (s_last) a.counter[1 + grp] = 0;
  }
  __syncthreads();
  if (!s_last) return;
  {
    double* Gg = a.Gpart + int64_t(a.P + grp) * npair;
    const double* base = a.Gpart + int64_t(grp) * CQ_GROUP * npair;
    for (int p = tid; p < npair; p += nt) {
      double u[CQ_GROUP];
#pragma unroll
      for (int q = 0; q < CQ_GROUP; ++q) u[q] = q < gsize ? __ldcg(base + int64_t(q) * npair + p) : 0.0;
      double acc = 0.0;
#pragma unroll
      for (int q = 0; q < CQ_GROUP; ++q) acc += u[q];
      Gg[p] = acc;
    }
  }
  __syncthreads();
  if (tid == 0) {
    const int old = atom_add_acq_rel_gpu(a.counter, 1);
    s_last = (old == ngrp - 1);
    if (s_last) *a.counter = 0;
  }
  __syncthreads();
  if (!s_last) return;

  // ---- last group: G = sum of group partials in order, then check or factor
  double* G = big ? a.big : sm;                 // k x k
  double* X = G + k * k;                        // k x k
  double* G0 = X + k * k;                       // k x k
  for (int p = tid; p < npair; p += nt) {
    const double* base = a.Gpart + int64_t(a.P) * npair + p;
    double acc = 0.0;
    int g = 0;
    for (; g + 8 <= ngrp; g += 8) {
      double u[8];
#pragma unroll
      for (int q = 0; q < 8; ++q) u[q] = __ldcg(base + int64_t(g + q) * npair);
#pragma unroll
      for (int q = 0; q < 8; ++q) acc += u[q];
    }
    for (; g < ngrp; ++g) acc += __ldcg(base + int64_t(g) * npair);
    int i, j;
    tri_ij(p, k, &i, &j);
    G[i * k + j] = acc;
    G[j * k + i] = acc;
    G0[i * k + j] = acc;
    G0[j * k + i] = acc;
  }
  __syncthreads();
  cqr_decide(G, X, G0, k, a.m, a.pass, final_pass, unshifted_run, a.Rinv, a.Racc, a.fo_r, a.status);
}

__global__ void __launch_bounds__(CQ_THREADS) cqr_pass_kernel(CqrPass a) { cqr_pass_body(a, int(blockIdx.x)); }

// One pass of many independent chains in one launch: job j owns CTAs
// [begin[j], begin[j + 1]) (begin has njobs + 1 entries); every job's own
// pass index is replaced by `pass`.
__global__ void __launch_bounds__(CQ_THREADS) cqr_pass_batch_kernel(const CqrPass* __restrict__ jobs,
                                                                   const int* __restrict__ begin, int njobs,
                                                                   int pass) {
  const int t = int(blockIdx.x);
  int lo = 0, hi = njobs - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (__ldg(begin + mid) <= t) lo = mid; else hi = mid - 1;
  }
  CqrPass a = jobs[lo];
  a.pass = pass;
  cqr_pass_body(a, t - __ldg(begin + lo));
}

// ---------------------------------------------------------------------------
// The whole chain in one cooperative launch (every CTA of the grid is resident,
// so the CTAs of a QR can wait for the pass decisions of their last CTA). Each
// CTA keeps its row block in shared memory across the passes: A is read once
// and Q written once; the k x k decision runs on the job's last-arriving CTA
// while the others wait on a released pass counter (bounded: after
// kCoopWaitNs the waiting CTA raises DEV_TIMEOUT in the run's status word and
// returns). The final pass needs no wait: its CTAs write Q and leave.
struct CoopJob {
  int64_t m;
  int k, b, P, fo_r;
  const double* A;
  int64_t a_rs, a_cs;
  double* Q;
  int64_t q_rs, q_cs;
  double* Gpart;            // (P + groups) x k (k + 1) / 2
  double* Rinv;             // k x k
  double* Racc;             // k x k accumulated R, or null
  int* status;              // [0..4] chain state as CqrPass, [5] final arrival,
                            // [6, 6 + groups) group arrivals, [6 + groups] released passes
  int* dev_status;          // the run's status word
  // Truncation certificate (eps null: off). When the chain ends by the
  // first-order pass right after its first factorization, the decider bounds
  // sigma_min(A) >= (1 - ||E||_F) / ||R0^{-1}||_F (A R0^{-1} has Gram I + E);
  // if that exceeds 2 eps and rcap >= k, no singular value can be cut, so the
  // bond's truncation step reduces to: Q^T as the new core (written over A,
  // which every CTA has read by then) and V(X_{n-1}) := V(X_{n-1}) R^T (rows
  // bp per CTA, in place); *cert := 1 and *rank_out := k tell the general
  // path to skip.
  const double* eps;
  int rcap, bp;
  int* cert;
  int64_t* rank_out;
  double* Aw;               // A itself, written with Q when certified
  double* Xp;               // mp x k row-major
  int64_t mp;
  int force_fail;           // testing: mark the chain failed after its first decision
};

constexpr unsigned long long kCoopWaitNs = 1000000000ull;   // 1 s

__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
__device__ __forceinline__ int ld_acquire_gpu(const int* p) {
  int v;
  asm volatile("ld.acquire.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_release_gpu(int* p, int v) {
  asm volatile("st.release.gpu.global.b32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// Shared memory (doubles) of the cooperative kernel: the row block plus a
// union of [Rinv | product block] and the decision's [G | X | G0].
__host__ __device__ inline int64_t coop_smem_doubles(int b, int k) {
  const int64_t bk = int64_t(b) * k, kk = int64_t(k) * k;
  return int64_t(b) * cq_ts(k) + (3 * kk > kk + bk ? 3 * kk : kk + bk);
}

__global__ void __launch_bounds__(CQ_THREADS) cqr_coop_kernel(CoopJob a) {
  extern __shared__ double sm[];
  __shared__ int s_flag;
  const int tid = threadIdx.x, nt = blockDim.x, lane = tid & 31, warp = tid >> 5, nw = nt >> 5;
  const int k = a.k, b = a.b, lb = blockIdx.x;
  const int npair = k * (k + 1) / 2;
  const int ngrp = (a.P + CQ_GROUP - 1) / CQ_GROUP;
  int* st = a.status;
  int* released = st + 6 + ngrp;
  const int ts = cq_ts(k);
  double* T = sm;                       // b x k row block (row stride ts), kept across passes
  double* U = sm + int64_t(b) * ts;     // union
  const int64_t r0 = int64_t(lb) * b;
  for (int r = warp; r < b; r += nw) {
    const int64_t gr = r0 + r;
    for (int c = lane; c < k; c += 32) T[r * ts + c] = (gr < a.m) ? a.A[gr * a.a_rs + c * a.a_cs] : 0.0;
  }
  __syncthreads();
  for (int pass = 0; pass < CQ_MAX_PASSES; ++pass) {
    bool final_pass = false;
    int unshifted_run = 0;
    if (pass > 0) {
      unshifted_run = __ldcg(st + 1);
      const int fo_kind = __ldcg(st + 4);
      const bool first_order = fo_kind != 0;
      final_pass = (unshifted_run >= 2 || pass == CQ_MAX_PASSES - 1);
      double* Rs = U;
      if (fo_kind == 2) {
        // T := T (I - E/2) = T - T (E/2) with ||E||_F <= 1e-10: the correction
        // is at most 1e-10 of T, so fp32 products of it (relative error
        // k 2^-24) keep T accurate to float64 rounding; one fp64 subtraction
        // per entry, on the FP32 pipe otherwise.
        float* Cf = reinterpret_cast<float*>(U);                 // E/2, k x k
        float* Tf = Cf + k * k;                                  // T, b x k
        for (int i = tid; i < k * k; i += nt)
          Cf[i] = float(((i % (k + 1) == 0) ? 1.0 : 0.0) - __ldcg(a.Rinv + i));
        for (int i = tid; i < b * k; i += nt) {
          const int r = i / k;
          Tf[i] = float(T[r * ts + (i - r * k)]);
        }
        __syncthreads();
        for (int i = tid; i < b * k; i += nt) {
          const int r = i / k, c = i - r * k;
          float corr = 0.0f;
          for (int j = 0; j < k; ++j) corr = fmaf(Tf[r * k + j], Cf[j * k + c], corr);
          T[r * ts + c] -= double(corr);
        }
        __syncthreads();
      } else {
        // T := T Rinv (upper triangular, or the full first-order correction):
        // one output entry per item, one accumulator. A warp issues at most
        // one FP64 instruction per ~64 cycles whether or not they depend on
        // each other, and the 8 warps already keep the FP64 pipe busy, so
        // split partial sums would only add their final adds. Items run
        // down the columns, so the lanes of a warp share one or two columns
        // and hence the length c + 1 of their triangular sums: a warp
        // instruction costs the same whatever its active lanes, so mixing
        // columns in a warp would pay the longest sum on every lane.
        double* T2 = U + k * k;
        for (int i = tid; i < k * k; i += nt) Rs[i] = __ldcg(a.Rinv + i);
        __syncthreads();
        for (int i = tid; i < b * k; i += nt) {
          const int c = i / b, r = i - c * b;
          const int jn = first_order ? k : c + 1;
          const double* tr = T + r * ts;
          double s0 = 0.0;
          for (int j = 0; j < jn; ++j) s0 = fma(tr[j], Rs[j * k + c], s0);
          T2[r * k + c] = s0;
        }
        __syncthreads();
        for (int i = tid; i < b * k; i += nt) {
          const int r = i / k;
          T[r * ts + (i - r * k)] = T2[i];
        }
        __syncthreads();
      }
      if (final_pass) {
        const bool cert = a.eps != nullptr && first_order && __ldcg(a.cert) != 0;
        double* qd = cert ? a.Aw : a.Q;
        const int64_t qr = cert ? a.a_rs : a.q_rs, qc = cert ? a.a_cs : a.q_cs;
        for (int r = warp; r < b; r += nw) {
          const int64_t gr = r0 + r;
          if (gr < a.m)
            for (int c = lane; c < k; c += 32) qd[gr * qr + c * qc] = T[r * ts + c];
        }
        if (cert) {
          // V(X_{n-1}) := V(X_{n-1}) R^T for this CTA's rows (in place), with
          // R = (I + E/2) R0: R0 upper triangular (left in Racc by the
          // certified decision), E = G - I symmetric. Y = Xp R0^T in FP64 over
          // the triangle (half the products of a full R), then
          // Xp := Y (I + E/2). The correction matrix is still in the first k^2
          // doubles of U from the update of T above: E/2 as floats when
          // ||E||_F <= 1e-10 (an fp32 product of the correction is then within
          // float64 rounding of Y), I - E/2 in float64 otherwise.
          double* R0s = U + k * k;          // R0, k x k
          double* Xr = R0s + k * k;         // nr x k at row stride ts (odd: no bank conflicts), later Y in fp32
          double* Y = T;                    // nr x k, the row block is dead once Q is written
          const int64_t p0 = int64_t(lb) * a.bp;
          const int64_t rem = a.mp - p0;
          const int nr = rem <= 0 ? 0 : (rem < a.bp ? int(rem) : a.bp);
          for (int i = tid; i < k * k; i += nt) R0s[i] = __ldcg(a.Racc + i);
          for (int i = tid; i < nr * k; i += nt) {
            const int r = i / k;
            Xr[r * ts + (i - r * k)] = a.Xp[p0 * k + i];
          }
          __syncthreads();
          // items down the columns: a warp's lanes share the triangle's length
          for (int i = tid; i < nr * k; i += nt) {
            const int c = i / nr, r = i - c * nr;
            const double* xr = Xr + r * ts;
            const double* rr = R0s + c * k;
            double s0 = 0.0;
            for (int j = c; j < k; ++j) s0 = fma(xr[j], rr[j], s0);
            Y[r * k + c] = s0;
          }
          __syncthreads();
          if (fo_kind == 2) {
            const float* Cf = reinterpret_cast<const float*>(U);   // E/2
            float* Yf = reinterpret_cast<float*>(Xr);
            for (int i = tid; i < nr * k; i += nt) Yf[i] = float(Y[i]);
            __syncthreads();
            for (int i = tid; i < nr * k; i += nt) {
              const int r = i / k, c = i - r * k;
              float corr = 0.0f;
              for (int l = 0; l < k; ++l) corr = fmaf(Yf[r * k + l], Cf[l * k + c], corr);
              a.Xp[p0 * k + i] = Y[i] + double(corr);
            }
          } else {
            // Y (I + E/2) = 2 Y - Y (I - E/2)
            const double* Rs = U;
            for (int i = tid; i < nr * k; i += nt) {
              const int r = i / k, c = i - r * k;
              const double* yr = Y + r * k;
              double s0 = 0.0;
              for (int j = 0; j < k; ++j) s0 = fma(yr[j], Rs[j * k + c], s0);
              a.Xp[p0 * k + i] = fma(2.0, yr[c], -s0);
            }
          }
        }
        if (first_order) {
          // Q = Q1 (I - E/2) with ||E||_F <= 1e-8: orthonormal to O(||E||^2), no check
          if (lb == 0 && tid == 0) atomicExch(st + 2, 1);
          return;
        }
      }
    }
    // partial Gram of the row block (packed upper triangle), one accumulator
    // per entry (as in the product above)
    double* Gp = a.Gpart + int64_t(lb) * npair;
    for (int p = tid; p < npair; p += nt) {
      int i1, j1;
      tri_ij(p, k, &i1, &j1);
      double g0 = 0.0;
      for (int r = 0; r < b; ++r) g0 = fma(T[r * ts + i1], T[r * ts + j1], g0);
      Gp[p] = g0;
    }
    // two-level arrival: the last CTA of each group sums its group's partials
    __syncthreads();
    const int grp = lb / CQ_GROUP;
    const int gsize = min(CQ_GROUP, a.P - grp * CQ_GROUP);
    if (tid == 0) {
      const int old = atom_add_acq_rel_gpu(st + 6 + grp, 1);
      s_flag = (old == gsize - 1);
      if (s_flag) st[6 + grp] = 0;
    }
    __syncthreads();
    bool decider = false;
    if (s_flag) {
      double* Gg = a.Gpart + int64_t(a.P + grp) * npair;
      const double* base = a.Gpart + int64_t(grp) * CQ_GROUP * npair;
      for (int p = tid; p < npair; p += 2 * nt) {
        // two entries per pass of the loop: 32 loads in flight per thread
        const int p2 = p + nt;
        double u[CQ_GROUP], v[CQ_GROUP];
#pragma unroll
        for (int q = 0; q < CQ_GROUP; ++q) {
          u[q] = q < gsize ? __ldcg(base + int64_t(q) * npair + p) : 0.0;
          v[q] = (q < gsize && p2 < npair) ? __ldcg(base + int64_t(q) * npair + p2) : 0.0;
        }
#pragma unroll
        for (int w = 1; w < CQ_GROUP; w *= 2)
#pragma unroll
          for (int q = 0; q + w < CQ_GROUP; q += 2 * w) {
            u[q] += u[q + w];
            v[q] += v[q + w];
          }
        Gg[p] = u[0];
        if (p2 < npair) Gg[p2] = v[0];
      }
      __syncthreads();
      if (tid == 0) {
        const int old = atom_add_acq_rel_gpu(st + 5, 1);
        s_flag = (old == ngrp - 1);
        if (s_flag) st[5] = 0;
      }
      __syncthreads();
      decider = s_flag;
    }
    if (decider) {
      double* G = U;
      double* X = G + k * k;
      double* G0 = X + k * k;
      // the tolerance's load overlaps the partials' loads below
      const double eps_v = (a.eps != nullptr && pass == 1) ? __ldcg(a.eps) : 0.0;
      // at most CQ_GROUP group partials (coop_shape keeps P <= CQ_GROUP^2):
      // all loads in flight at once, then a fixed pairwise tree
      for (int p = tid; p < npair; p += nt) {
        const double* base = a.Gpart + int64_t(a.P) * npair + p;
        double u[CQ_GROUP];
#pragma unroll
        for (int q = 0; q < CQ_GROUP; ++q) u[q] = q < ngrp ? __ldcg(base + int64_t(q) * npair) : 0.0;
#pragma unroll
        for (int w = 1; w < CQ_GROUP; w *= 2)
#pragma unroll
          for (int q = 0; q + w < CQ_GROUP; q += 2 * w) u[q] += u[q + w];
        const double acc = u[0];
        int i, j;
        tri_ij(p, k, &i, &j);
        G[i * k + j] = acc;
        G[j * k + i] = acc;
        G0[i * k + j] = acc;
        G0[j * k + i] = acc;
      }
      __syncthreads();
      // certificate inputs, before the decision overwrites G and Rinv
      const bool try_cert = a.eps != nullptr && pass == 1 && !final_pass && a.rcap >= k;
      const bool fo_test = pass > 0 && !final_pass && (a.Racc == nullptr || a.fo_r);
      double e2 = -1.0, ri2 = 0.0;
      if (try_cert || fo_test) {
        // ||G - I||_F^2 (the first-order test) and ||R0^{-1}||_F^2 in one reduction
        double pe = 0.0, pr = 0.0;
        for (int r = warp; r < k; r += nw)
          for (int c = lane; c < k; c += 32) {
            const double dv = G[r * k + c] - (r == c ? 1.0 : 0.0);
            pe = fma(dv, dv, pe);
            if (try_cert) {
              const double ri = __ldcg(a.Rinv + r * k + c);
              pr = fma(ri, ri, pr);
            }
          }
        block_sum2(&pe, &pr);
        e2 = pe;
        ri2 = pr;
      }
      // The certificate is settled before the decision: a certified bond takes
      // the first-order step (the same test, e2 <= 1e-16), and its R is needed
      // only by the fold of the final pass, which applies (I + E/2) itself, so
      // the decision leaves R = R0 (upper triangular) in Racc.
      bool certify = false;
      if (try_cert) {
        const double lbound = (1.0 - sqrt(e2)) * (1.0 - 1e-6) / sqrt(ri2);
        certify = e2 <= 1e-16 && isfinite(lbound) && ri2 > 0.0 && lbound > 2.0 * eps_v;
      }
      cqr_decide(G, X, G0, k, a.m, pass, final_pass, unshifted_run, a.Rinv, certify ? nullptr : a.Racc, a.fo_r,
                 st, e2);
      if (a.force_fail && tid == 0) st[0] = 1;
      if (final_pass) return;
      if (certify && tid == 0) {
        *a.cert = 1;
        *a.rank_out = k;
      }
      __syncthreads();
      if (tid == 0) st_release_gpu(released, pass + 1);   // cumulative over the block's writes
    } else {
      if (final_pass) return;
      if (tid == 0) {
        const unsigned long long t0 = global_ns();
        int ok = 1;
        while (ld_acquire_gpu(released) < pass + 1) {
          if (global_ns() - t0 > kCoopWaitNs) {
            ok = 0;
            break;
          }
          __nanosleep(64);
        }
        s_flag = ok;
      }
      __syncthreads();
      if (!s_flag) {
        if (tid == 0) atomicOr(a.dev_status, DEV_TIMEOUT);
        return;
      }
    }
    if (__ldcg(st + 2)) return;           // the chain broke down: the Householder fallback takes over
    __syncthreads();
  }
}

// Row blocking of the cooperative kernel: about one block per SM; feasible when
// the shared memory fits and the grid is co-resident.
bool coop_shape(int64_t m, int k, int* b, int* P, size_t* smem) {
  if (k > CQ_SMEM_K || k < 1 || m < k) return false;
  const int nsm = num_sms();
  const int64_t bb = std::max<int64_t>(4, ceil_div(m, nsm));
  const size_t bytes = size_t(coop_smem_doubles(int(bb), k)) * sizeof(double);
  if (bytes > 220 * 1024) return false;
  int nb = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, cqr_coop_kernel, CQ_THREADS, bytes) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  const int64_t PP = ceil_div(m, bb);
  if (nb < 1 || PP > int64_t(nb) * nsm || PP > int64_t(CQ_GROUP) * CQ_GROUP) return false;
  *b = int(bb);
  *P = int(PP);
  *smem = bytes;
  return true;
}

int coop_launch(const CoopJob& job, size_t smem, cudaStream_t s) {
  static bool attr = false;
  if (!attr) {
    TTR_CHECK_CUDA(cudaFuncSetAttribute(cqr_coop_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, 220 * 1024));
    attr = true;
  }
  cudaEvent_t e0;
  const bool prof = prof_begin(s, &e0);
  TTR_PREFER_SHARED(cqr_coop_kernel);
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(unsigned(job.P));
  cfg.blockDim = dim3(CQ_THREADS);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeCooperative;
  at[0].val.cooperative = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  TTR_CHECK_CUDA(cudaLaunchKernelEx(&cfg, cqr_coop_kernel, job));
  prof_count_launch(1);
  if (prof) prof_end(s, 1, 4.0 * double(job.m) * double(job.k) * double(job.k));
  return TT_OK;
}

int cqr_launch(const CqrPass& p, cudaStream_t s) {
  const size_t kk = size_t(p.k) * p.k;
  const size_t bts = size_t(p.b) * cq_ts(p.k);
  const size_t smem = (p.big ? 2 * bts : std::max<size_t>(2 * bts + kk, 3 * kk)) *
                      sizeof(double);
  static bool attr = false;
  if (!attr) {
    TTR_CHECK_CUDA(cudaFuncSetAttribute(cqr_pass_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, 220 * 1024));
    attr = true;
  }
  cudaEvent_t e0;
  const bool prof = prof_begin(s, &e0);
  TTR_PREFER_SHARED(cqr_pass_kernel);
  cqr_pass_kernel<<<p.P, CQ_THREADS, smem, s>>>(p);
  TTR_CHECK_LAUNCH();
  prof_count_launch(1);
  // the QR's algorithmic flops (4 m k^2, the Householder count of a thin QR) on its first pass
  if (prof) prof_end(s, 1, p.pass == 0 ? 4.0 * double(p.m) * double(p.k) * double(p.k) : 0.0);
  return TT_OK;
}

}  // namespace

namespace {
void qr_shape(int64_t m, int k, int* rows, int* P, int* nstat) {
  const bool big = k > CQ_SMEM_K;
  const int64_t budget = 28000 - (big ? 0 : int64_t(k) * k);                 // doubles of shared memory
  const int64_t bmax = std::max<int64_t>(1, budget / (2 * int64_t(cq_ts(k))));
  *rows = int(std::min<int64_t>(bmax, std::max<int64_t>(4, ceil_div(m, num_sms()))));
  *P = int(ceil_div(m, *rows));
  *nstat = 5 + 1 + (*P + 15) / 16 + 2;  // [0..4] chain state, arrival counters, released passes, certificate
}
}  // namespace

QrPool qr_pool_reserve(Arena& ar, const std::vector<std::pair<int64_t, int>>& shapes) {
  size_t gp = 1, kk = 1, mk = 1, bigk = 0, st = 1, tw = 1, ti = 1;
  for (auto& sh : shapes) {
    const int64_t m = sh.first;
    const int k = sh.second;
    int rows, P, ns;
    qr_shape(m, k, &rows, &P, &ns);
    gp = std::max<size_t>(gp, size_t(P + (P + 15) / 16) * k * k);
    kk = std::max<size_t>(kk, size_t(k) * k);
    mk = std::max<size_t>(mk, size_t(m) * k);
    if (k > CQ_SMEM_K) bigk = std::max<size_t>(bigk, 3 * size_t(k) * k);
    st = std::max<size_t>(st, size_t(ns));
    if (k <= TSQR_KMAX) {
      size_t ii = 0;
      tw = std::max(tw, tsqr_work_doubles(tsqr_shape(m, k), &ii));
      ti = std::max(ti, ii);
    }
  }
  QrPool p;
  p.Gpart = ar.take<double>(gp);
  p.Rinv = ar.take<double>(kk);
  p.Q1 = ar.take<double>(mk);
  p.Q2 = ar.take<double>(mk);
  p.big = bigk ? ar.take<double>(bigk) : nullptr;
  p.status = ar.take<int>(st);
  p.tw = ar.take<double>(tw);
  p.ti = ar.take<int>(ti);
  return p;
}

QrBufs qr_view(const QrPool& p, int64_t m, int k) {
  QrBufs b;
  b.m = m;
  b.k = k;
  qr_shape(m, k, &b.rows, &b.P, &b.nstat);
  b.Gpart = p.Gpart;
  b.Rinv = p.Rinv;
  b.Q1 = p.Q1;
  b.Q2 = p.Q2;
  b.big = (k > CQ_SMEM_K) ? p.big : nullptr;
  b.status = p.status;
  if (k <= TSQR_KMAX) {
    b.sh = tsqr_shape(m, k);
    size_t ii = 0;
    tsqr_work_doubles(b.sh, &ii);
    b.tw = p.tw;
    b.ti = p.ti;
    b.ti_n = ii;
  }
  return b;
}

QrBufs qr_reserve(Arena& ar, int64_t m, int k) {
  return qr_view(qr_pool_reserve(ar, {{m, k}}), m, k);
}

void qr_chain_plan(Schedule& sc, const QrBufs& b, const double* A, int64_t a_rs, int64_t a_cs, double* Q,
                   int64_t q_rs, int64_t q_cs, double* R, bool r_may_be_full);
void qr_fallback_plan(Schedule& sc, const QrBufs& b, const double* A, int64_t a_rs, int64_t a_cs, double* Q,
                      int64_t q_rs, int64_t q_cs, double* R);

static std::atomic<int> g_qr_mode{QR_MODE_AUTO};
int set_qr_mode(int mode) {
  if (mode < QR_MODE_AUTO || mode > QR_MODE_COOP_THEN_FALLBACK) return TT_EINVAL;
  g_qr_mode.store(mode);
  return TT_OK;
}

const int* qr_cert_flag(const QrBufs& b) { return b.status ? b.status + b.nstat - 1 : nullptr; }

void qr_plan(Schedule& sc, const QrBufs& b, const double* A, int64_t a_rs, int64_t a_cs, double* Q, int64_t q_rs,
             int64_t q_cs, double* R, bool r_may_be_full, const QrCert* cert) {
  const QrBufs bb = b;
  const int mode = g_qr_mode.load();
  const bool force_fallback = (mode == QR_MODE_FORCE_FALLBACK) && b.k <= TSQR_KMAX;
  sc.add([bb, force_fallback](cudaStream_t s) -> int {
    if (!bb.status) return int(TT_OK);
    TTR_CHECK_CUDA(cudaMemsetAsync(bb.status, 0, bb.nstat * sizeof(int), s));
    if (bb.ti && bb.ti_n) TTR_CHECK_CUDA(cudaMemsetAsync(bb.ti, 0, bb.ti_n * sizeof(int), s));
    if (force_fallback) return set_flag_launch(bb.status, s);
    return int(TT_OK);
  });
  int cb = 0, cP = 0;
  size_t csm = 0;
  const bool coop_mode = mode == QR_MODE_AUTO || (mode == QR_MODE_COOP_THEN_FALLBACK && b.k <= TSQR_KMAX);
  if (!force_fallback && coop_mode && coop_shape(b.m, b.k, &cb, &cP, &csm)) {
    CoopJob job{};
    job.m = b.m;
    job.k = b.k;
    job.b = cb;
    job.P = cP;
    job.fo_r = r_may_be_full ? 1 : 0;
    job.A = A;
    job.a_rs = a_rs;
    job.a_cs = a_cs;
    job.Q = Q;
    job.q_rs = q_rs;
    job.q_cs = q_cs;
    job.Gpart = b.Gpart;
    job.Rinv = b.Rinv;
    job.Racc = R;
    job.status = b.status;
    job.force_fail = mode == QR_MODE_COOP_THEN_FALLBACK ? 1 : 0;
    if (cert && R && r_may_be_full && !job.force_fail) {
      // the fold keeps [correction | R0 | rows of V(X_{n-1})] in the union and
      // Y in the row block
      const int64_t bp = ceil_div(cert->mp, int64_t(cP));
      const int64_t kk = int64_t(b.k) * b.k;
      if (bp <= cb && 2 * kk + bp * cq_ts(b.k) <= coop_smem_doubles(cb, b.k) - int64_t(cb) * cq_ts(b.k)) {
        job.eps = cert->eps;
        job.rcap = cert->rcap;
        job.bp = int(bp);
        job.cert = b.status ? b.status + b.nstat - 1 : nullptr;
        job.rank_out = cert->rank_out;
        job.Aw = cert->Aw;
        job.Xp = cert->Xp;
        job.mp = cert->mp;
      }
    }
    int* const* sp = &sc.dev_status;
    sc.add([job, csm, sp](cudaStream_t s) -> int {
      if (!job.status) return int(TT_OK);
      CoopJob j = job;
      j.dev_status = *sp;
      return coop_launch(j, csm, s);
    });
  }
  else if (!force_fallback) {
    qr_chain_plan(sc, b, A, a_rs, a_cs, Q, q_rs, q_cs, R, r_may_be_full);
  }
  qr_fallback_plan(sc, b, A, a_rs, a_cs, Q, q_rs, q_cs, R);
}

// The multi-launch chain: CQ_MAX_PASSES launches of cqr_pass_kernel.
void qr_chain_plan(Schedule& sc, const QrBufs& b, const double* A, int64_t a_rs, int64_t a_cs, double* Q,
                   int64_t q_rs, int64_t q_cs, double* R, bool r_may_be_full) {
  CqrPass base{};
  base.m = b.m;
  base.k = b.k;
  base.b = b.rows;
  base.P = b.P;
  base.A = A;
  base.a_rs = a_rs;
  base.a_cs = a_cs;
  base.buf[0] = b.Q1;
  base.buf[1] = b.Q2;
  base.Q = Q;
  base.q_rs = q_rs;
  base.q_cs = q_cs;
  base.Gpart = b.Gpart;
  base.counter = b.status ? b.status + 5 : nullptr;
  base.Rinv = b.Rinv;
  base.Racc = R;
  base.fo_r = r_may_be_full ? 1 : 0;
  base.big = b.big;
  base.status = b.status;
  for (int p = 0; p < CQ_MAX_PASSES; ++p) {
    CqrPass pp = base;
    pp.pass = p;
    sc.add([pp](cudaStream_t s) -> int { return cqr_launch(pp, s); });
  }
}

namespace {
__global__ void qr_batch_fold_kernel(const int* __restrict__ status, const int* __restrict__ soff, int njobs,
                                     int* dev_status) {
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < njobs; j += gridDim.x * blockDim.x)
    if (__ldcg(status + soff[j]) != 0) atomicOr(dev_status, DEV_QR_FAIL);
}
}  // namespace

static void qr_batch_shape(int64_t m, int k, int ctas_per_job, int* rows, int* P) {
  const int64_t budget = 28000 - int64_t(k) * k;
  const int64_t bmax = std::max<int64_t>(1, budget / (2 * int64_t(cq_ts(k))));
  *rows = int(std::min<int64_t>(bmax, std::max<int64_t>(4, ceil_div(m, std::max(1, ctas_per_job)))));
  *P = int(ceil_div(m, *rows));
}

int64_t qr_batch_gram_doubles(int64_t m, int k, int ctas_per_job) {
  int rows, P;
  qr_batch_shape(m, k, ctas_per_job, &rows, &P);
  return int64_t(P + (P + 15) / 16) * k * k;
}

int qr_batch_plan(Arena& ar, Schedule& sc, const std::vector<QrBatchJob>& jobs, int ctas_per_job) {
  const int nj = int(jobs.size());
  if (nj == 0) return TT_OK;
  std::vector<CqrPass> tab(nj);
  std::vector<int> begin(nj + 1, 0), soff(nj, 0);
  int64_t tot_status = 0;
  size_t smem = 0;
  for (int j = 0; j < nj; ++j) {
    const QrBatchJob& q = jobs[j];
    if (q.k < 1 || q.k > CQ_SMEM_K || q.m < q.k) {
      set_error("batched thin QR: needs k <= 96 and m >= k");
      return TT_EUNSUPPORTED;
    }
    const int k = q.k;
    int rows, P;
    qr_batch_shape(q.m, k, ctas_per_job, &rows, &P);
    const int ngrp = (P + 15) / 16;
    CqrPass& a = tab[j];
    a = CqrPass{};
    a.m = q.m;
    a.k = k;
    a.b = rows;
    a.P = P;
    a.A = q.A;
    a.a_rs = q.a_rs;
    a.a_cs = q.a_cs;
    a.buf[0] = q.has_scratch ? q.buf0 : ar.take<double>(size_t(q.m) * k);
    a.buf[1] = q.has_scratch ? q.buf1 : ar.take<double>(size_t(q.m) * k);
    a.Q = q.Q;
    a.q_rs = q.q_rs;
    a.q_cs = q.q_cs;
    a.Gpart = q.has_scratch ? q.gpart : ar.take<double>(size_t(P + ngrp) * k * k);
    a.Rinv = q.has_scratch ? q.rinv : ar.take<double>(size_t(k) * k);
    a.Racc = nullptr;
    a.fo_r = 0;
    a.big = nullptr;
    soff[j] = int(tot_status);
    tot_status += 5 + 1 + ngrp;
    begin[j + 1] = begin[j] + P;
    smem = std::max(smem, std::max<size_t>(size_t(2) * rows * cq_ts(k) + size_t(k) * k, size_t(3) * k * k) *
                              sizeof(double));
  }
  int* status = ar.take<int>(size_t(tot_status));
  for (int j = 0; j < nj; ++j) {
    tab[j].status = status ? status + soff[j] : nullptr;
    tab[j].counter = status ? status + soff[j] + 5 : nullptr;
  }
  // the job table, CTA prefixes and status offsets, uploaded with the schedule
  const size_t tb = tab.size() * sizeof(CqrPass), bb = begin.size() * sizeof(int), ob = soff.size() * sizeof(int);
  double* d_tab = ar.take<double>(ceil_div(int64_t(tb), 8));
  double* d_begin = ar.take<double>(ceil_div(int64_t(bb), 8));
  double* d_soff = ar.take<double>(ceil_div(int64_t(ob), 8));
  auto pack = [](const void* src, size_t bytes) {
    std::vector<double> v(size_t(ceil_div(int64_t(bytes), 8)), 0.0);
    std::memcpy(v.data(), src, bytes);
    return v;
  };
  sc.upload(d_tab, pack(tab.data(), tb));
  sc.upload(d_begin, pack(begin.data(), bb));
  sc.upload(d_soff, pack(soff.data(), ob));
  const int total = begin[nj];
  int* const* sp = &sc.dev_status;
  sc.add([=](cudaStream_t st) -> int {
    if (!status) return int(TT_OK);
    TTR_CHECK_CUDA(cudaMemsetAsync(status, 0, size_t(tot_status) * sizeof(int), st));
    static bool attr = false;
    if (!attr) {
      TTR_CHECK_CUDA(
          cudaFuncSetAttribute(cqr_pass_batch_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, 220 * 1024));
      attr = true;
    }
    TTR_PREFER_SHARED(cqr_pass_batch_kernel);
    for (int p = 0; p < CQ_MAX_PASSES; ++p) {
      cudaEvent_t e0;
      const bool prof = prof_begin(st, &e0);
      cqr_pass_batch_kernel<<<unsigned(total), CQ_THREADS, smem, st>>>(
          reinterpret_cast<const CqrPass*>(d_tab), reinterpret_cast<const int*>(d_begin), nj, p);
      TTR_CHECK_LAUNCH();
      prof_count_launch(1);
      if (prof) prof_end(st, 1, 0.0);
    }
    qr_batch_fold_kernel<<<unsigned(std::max<int64_t>(1, ceil_div(nj, 256))), 256, 0, st>>>(
        status, reinterpret_cast<const int*>(d_soff), nj, *sp);
    TTR_CHECK_LAUNCH();
    prof_count_launch(1);
    return int(TT_OK);
  });
  return TT_OK;
}

// Householder TSQR when the chain raised status[0] (k <= 96); above that limit
// a failure is reported in the run's status word.
void qr_fallback_plan(Schedule& sc, const QrBufs& b, const double* A, int64_t a_rs, int64_t a_cs, double* Q,
                      int64_t q_rs, int64_t q_cs, double* R) {
  const QrBufs bb = b;
  if (b.k <= TSQR_KMAX) {
    // Householder fallback, run only when the device flag is raised
    sc.add([bb, A, a_rs, a_cs, Q, q_rs, q_cs, R](cudaStream_t s) -> int {
      TsqrWork w;
      tsqr_bind(bb.sh, bb.tw, bb.ti, &w);
      return tsqr_launch(bb.sh, w, A, a_rs, a_cs, Q, q_rs, q_cs, R, s, bb.status);
    });
  } else {
    // no fallback above the Householder limit: a failure goes to the run's status word
    int* const* sp = &sc.dev_status;
    sc.add([bb, sp](cudaStream_t s) -> int { return or_flag_launch(*sp, bb.status, DEV_QR_FAIL, s); });
  }
}

}  // namespace ttr

// ---------------------------------------------------------------------------
// Diagnostic: the pivot reciprocal square root against CUDA's rsqrt over n
// points of [1, 4) scaled by 4^s, s in [-480, 480] (so every exponent parity
// and nearly the whole normal range).
namespace ttr {
namespace {
__global__ void pivot_rsqrt_check_kernel(int64_t n, unsigned long long* max_ulp, unsigned long long* ndiff) {
  unsigned long long worst = 0, cnt = 0;
  for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x) {
    const double f = 1.0 + 3.0 * double(i) / double(n);
    const double x = ldexp(f, 2 * int(i % 961 - 480));
    const double a = rsqrt_refined(x), b = rsqrt(x);
    const long long ia = __double_as_longlong(a), ib = __double_as_longlong(b);
    const unsigned long long du = (unsigned long long)(ia > ib ? ia - ib : ib - ia);   // same sign: ulps apart
    worst = du > worst ? du : worst;
    cnt += du != 0;
  }
  atomicMax(max_ulp, worst);
  atomicAdd(ndiff, cnt);
}
}  // namespace
}  // namespace ttr

extern "C" int tt_probe_pivot_rsqrt(int64_t n, int64_t* max_ulp, int64_t* ndiff, void* stream) {
  using namespace ttr;
  if (n < 1 || !max_ulp || !ndiff) {
    set_error("tt_probe_pivot_rsqrt: need n >= 1 and outputs");
    return TT_EINVAL;
  }
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  unsigned long long* d = nullptr;
  TTR_CHECK_CUDA(cudaMallocAsync(reinterpret_cast<void**>(&d), 2 * sizeof(unsigned long long), s));
  TTR_CHECK_CUDA(cudaMemsetAsync(d, 0, 2 * sizeof(unsigned long long), s));
  pivot_rsqrt_check_kernel<<<4 * num_sms(), 256, 0, s>>>(n, d, d + 1);
  TTR_CHECK_LAUNCH();
  prof_count_launch(1);
  unsigned long long h[2] = {0, 0};
  TTR_CHECK_CUDA(cudaMemcpyAsync(h, d, sizeof(h), cudaMemcpyDeviceToHost, s));
  TTR_CHECK_CUDA(cudaStreamSynchronize(s));
  cudaFreeAsync(d, s);
  *max_ulp = int64_t(h[0]);
  *ndiff = int64_t(h[1]);
  return TT_OK;
}

// Tall-skinny Householder QR (TSQR) in FP64.
//
// Used for the thin QR of the sketched matrix (Algorithm 5 / Algorithm 7, QR of
// Y_n), for the right-to-left truncation sweep (QR of H(X_n)^T, Section 3.2 /
// Algorithm 2) and for the orthogonalization of Algorithms 1 and 4. The paper
// assumes Householder QR (Section 2.1); Householder is kept because the sketched
// matrices are rank deficient whenever the target rank exceeds the true rank,
// where Cholesky-based QR breaks down.
//
// GB300 layout: one CTA per leaf of b rows (b x k in shared memory, column
// major); the R factors climb a binary tree inside the same launch: each CTA
// fences its stores and bumps the parent's counter, and the second child to
// arrive combines the pair (QR of the stacked 2k x k triangles). No CTA ever
// waits on another, so the launch cannot hang. The explicit Q is formed by a
// second launch where every leaf CTA walks its root-to-leaf path applying the
// stored reflectors to [I; 0].
#include <algorithm>

#include "kernels.cuh"
#include "prof.cuh"

namespace ttr {

namespace {

constexpr int TQ_THREADS = 256;

__device__ __forceinline__ double block_sum(double v, double* red) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  __syncthreads();
  if (l == 0) red[w] = v;
  __syncthreads();
  double s = 0.0;
  const int nw = blockDim.x >> 5;
  for (int i = 0; i < nw; ++i) s += red[i];
  return s;
}

// Householder QR (LAPACK dlarfg convention) of S (rows x cols, column-major,
// leading dimension ld) in shared memory: R in the upper triangle, the
// reflector vectors below the diagonal (unit leading entry implied), tau[c].
__device__ void house_qr(double* S, int ld, int rows, int cols, double* tau, double* red, double* wv,
                         double* sc) {
  const int tid = threadIdx.x, nt = blockDim.x;
  const int warp = tid >> 5, lane = tid & 31, nwarp = nt >> 5;
  const int steps = min(rows, cols);
  for (int c = 0; c < steps; ++c) {
    double part = 0.0;
    for (int r = c + 1 + tid; r < rows; r += nt) {
      double x = S[r + c * ld];
      part = fma(x, x, part);
    }
    const double xn2 = block_sum(part, red);
    if (tid == 0) {
      const double alpha = S[c + c * ld];
      double t = 0.0, scale = 0.0;
      if (xn2 > 0.0) {
        double beta = -copysign(sqrt(fma(alpha, alpha, xn2)), alpha);
        t = (beta - alpha) / beta;
        scale = 1.0 / (alpha - beta);
        S[c + c * ld] = beta;
      }
      tau[c] = t;
      sc[0] = scale;
    }
    __syncthreads();
    const double t = tau[c];
    if (t == 0.0) continue;
    const double scale = sc[0];
    for (int r = c + 1 + tid; r < rows; r += nt) S[r + c * ld] *= scale;
    __syncthreads();
    for (int j = c + 1 + warp; j < cols; j += nwarp) {
      double s = 0.0;
      for (int r = c + 1 + lane; r < rows; r += 32) s = fma(S[r + c * ld], S[r + j * ld], s);
      for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
      if (lane == 0) wv[j] = t * (S[c + j * ld] + s);
    }
    __syncthreads();
    const int h = rows - c, wcols = cols - c - 1;
    for (int idx = tid; idx < h * wcols; idx += nt) {
      const int r = c + idx % h, j = c + 1 + idx / h;
      const double v = (r == c) ? 1.0 : S[r + c * ld];
      S[r + j * ld] -= v * wv[j];
    }
    __syncthreads();
  }
}

// T (rows x cols, column-major ld) := H_0 H_1 ... H_{nref-1} T, with the
// reflectors read from global memory (V column-major, leading dimension ldv).
__device__ void apply_q(double* T, int ld, int rows, int cols, const double* V, int ldv, const double* tau,
                        int nref, double* vcol, double* wv) {
  const int tid = threadIdx.x, nt = blockDim.x;
  const int warp = tid >> 5, lane = tid & 31, nwarp = nt >> 5;
  for (int j = nref - 1; j >= 0; --j) {
    const double t = __ldcg(tau + j);
    if (t == 0.0) continue;
    for (int r = tid; r < rows; r += nt) vcol[r] = (r == j) ? 1.0 : (r > j ? __ldcg(V + r + int64_t(j) * ldv) : 0.0);
    __syncthreads();
    for (int c = warp; c < cols; c += nwarp) {
      double s = 0.0;
      for (int r = j + lane; r < rows; r += 32) s = fma(vcol[r], T[r + c * ld], s);
      for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
      if (lane == 0) wv[c] = t * s;
    }
    __syncthreads();
    const int h = rows - j;
    for (int idx = tid; idx < h * cols; idx += nt) {
      const int r = j + idx % h, c = idx / h;
      T[r + c * ld] -= vcol[r] * wv[c];
    }
    __syncthreads();
  }
}

struct TsqrArgs {
  int64_t m;
  int k, b, P, L;
  const double* A;
  int64_t a_rs, a_cs;
  double* Q;
  int64_t q_rs, q_cs;
  double* R;
  const int* skip_unless;   // when set, run only if *skip_unless != 0
  TsqrWork w;
};

__device__ __forceinline__ int level_count(int P, int l) { return (P + (1 << l) - 1) >> l; }
__device__ __forceinline__ int level_offset(int P, int l) {
  int off = 0;
  for (int i = 0; i < l; ++i) off += level_count(P, i);
  return off;
}

// Number of fallback runs (leaf launches that did not skip), for diagnostics.
__device__ unsigned long long g_tsqr_runs = 0;

__global__ void __launch_bounds__(TQ_THREADS) tsqr_up_kernel(TsqrArgs a) {
  extern __shared__ double smem[];
  const int k = a.k, b = a.b;
  const int rows_max = max(b, 2 * k);
  double* S = smem;                          // rows_max * k
  double* tau = S + rows_max * k;            // k
  double* wv = tau + k;                      // k
  double* red = wv + k;                      // 32
  double* sc = red + 32;                     // 1
  __shared__ int s_last;
  const int tid = threadIdx.x, nt = blockDim.x;
  const int p = blockIdx.x;
  if (a.skip_unless && *a.skip_unless == 0) return;
  if (p == 0 && tid == 0 && a.skip_unless) atomicAdd(&g_tsqr_runs, 1ull);

  // ---- leaf: rows [p*b, p*b + b) of A, zero padded past m
  const int64_t r0 = int64_t(p) * b;
  for (int idx = tid; idx < b * k; idx += nt) {
    const int r = idx % b, c = idx / b;
    const int64_t gr = r0 + r;
    S[r + c * b] = (gr < a.m) ? a.A[gr * a.a_rs + c * a.a_cs] : 0.0;
  }
  __syncthreads();
  house_qr(S, b, b, k, tau, red, wv, sc);
  double* V = a.w.leafV + int64_t(p) * b * k;
  for (int idx = tid; idx < b * k; idx += nt) V[idx] = S[idx];
  for (int c = tid; c < k; c += nt) a.w.leafTau[int64_t(p) * k + c] = tau[c];
  double* Rn = a.w.nodeR + int64_t(p) * k * k;
  for (int idx = tid; idx < k * k; idx += nt) {
    const int i = idx / k, c = idx % k;
    Rn[idx] = (i <= c) ? S[i + c * b] : 0.0;
  }
  if (a.L == 0) {
    if (a.R)
      for (int idx = tid; idx < k * k; idx += nt) {
        const int i = idx / k, c = idx % k;
        a.R[idx] = (i <= c) ? S[i + c * b] : 0.0;
      }
    return;
  }

  // ---- climb the tree; only the last-arriving child of a node continues
  int q = p;
  for (int l = 0; l < a.L; ++l) {
    const int parent = q >> 1;
    const int nchild = (2 * parent + 1 < level_count(a.P, l)) ? 2 : 1;
    const int inner = level_offset(a.P, l + 1) - a.P + parent;   // index among inner nodes
    __syncthreads();
    if (tid == 0) {
      const int old = atom_add_acq_rel_gpu(a.w.counters + inner, 1);
      s_last = (old == nchild - 1);
      if (s_last) a.w.counters[inner] = 0;   // every child has arrived: reset for the next call
    }
    __syncthreads();
    if (!s_last) return;
    const int off_l = level_offset(a.P, l);
    const double* Rt = a.w.nodeR + int64_t(off_l + 2 * parent) * k * k;
    const double* Rb = a.w.nodeR + int64_t(off_l + 2 * parent + 1) * k * k;
    const int ld = 2 * k;
    for (int idx = tid; idx < 2 * k * k; idx += nt) {
      const int r = idx % (2 * k), c = idx / (2 * k);
      double v = 0.0;
      if (r < k) v = __ldcg(Rt + r * k + c);
      else if (nchild == 2) v = __ldcg(Rb + (r - k) * k + c);
      S[r + c * ld] = v;
    }
    __syncthreads();
    house_qr(S, ld, 2 * k, k, tau, red, wv, sc);
    double* NV = a.w.nodeV + int64_t(inner) * 2 * k * k;
    for (int idx = tid; idx < 2 * k * k; idx += nt) NV[idx] = S[idx];
    for (int c = tid; c < k; c += nt) a.w.nodeTau[int64_t(inner) * k + c] = tau[c];
    double* RN = a.w.nodeR + int64_t(a.P + inner) * k * k;
    for (int idx = tid; idx < k * k; idx += nt) {
      const int i = idx / k, c = idx % k;
      RN[idx] = (i <= c) ? S[i + c * ld] : 0.0;
    }
    if (l + 1 == a.L && a.R)
      for (int idx = tid; idx < k * k; idx += nt) {
        const int i = idx / k, c = idx % k;
        a.R[idx] = (i <= c) ? S[i + c * ld] : 0.0;
      }
    q = parent;
  }
}

__global__ void __launch_bounds__(TQ_THREADS) tsqr_down_kernel(TsqrArgs a) {
  extern __shared__ double smem[];
  const int k = a.k, b = a.b;
  const int rows_max = max(b, 2 * k);
  const int ld = rows_max;
  double* T = smem;                          // rows_max * k
  double* vcol = T + rows_max * k;           // rows_max
  double* wv = vcol + rows_max;              // k
  const int tid = threadIdx.x, nt = blockDim.x;
  const int p = blockIdx.x;
  if (a.skip_unless && *a.skip_unless == 0) return;

  for (int idx = tid; idx < rows_max * k; idx += nt) {
    const int r = idx % rows_max, c = idx / rows_max;
    T[r + c * ld] = (r == c) ? 1.0 : 0.0;
  }
  __syncthreads();
  for (int l = a.L; l >= 1; --l) {
    const int q = p >> l;
    const int half = (p >> (l - 1)) & 1;
    const int inner = level_offset(a.P, l) - a.P + q;
    apply_q(T, ld, 2 * k, k, a.w.nodeV + int64_t(inner) * 2 * k * k, 2 * k, a.w.nodeTau + int64_t(inner) * k, k,
            vcol, wv);
    for (int idx = tid; idx < k * k; idx += nt) {
      const int r = idx % k, c = idx / k;
      if (half) T[r + c * ld] = T[r + k + c * ld];
    }
    __syncthreads();
    for (int idx = tid; idx < (rows_max - k) * k; idx += nt) {
      const int r = k + idx % (rows_max - k), c = idx / (rows_max - k);
      T[r + c * ld] = 0.0;
    }
    __syncthreads();
  }
  apply_q(T, ld, b, k, a.w.leafV + int64_t(p) * b * k, b, a.w.leafTau + int64_t(p) * k, k, vcol, wv);
  const int64_t r0 = int64_t(p) * b;
  for (int idx = tid; idx < b * k; idx += nt) {
    const int r = idx / k, c = idx % k;
    const int64_t gr = r0 + r;
    if (gr < a.m) a.Q[gr * a.q_rs + c * a.q_cs] = T[r + c * ld];
  }
}

}  // namespace

TsqrShape tsqr_shape(int64_t m, int k) {
  TsqrShape s;
  s.m = m;
  s.k = k;
  s.b = (k <= 32) ? 64 : 128;
  s.P = int(std::max<int64_t>(1, ceil_div(m, s.b)));
  s.L = 0;
  while ((1 << s.L) < s.P) ++s.L;
  s.inner = 0;
  for (int l = 1; l <= s.L; ++l) s.inner += int((s.P + (1 << l) - 1) >> l);
  return s;
}

size_t tsqr_work_doubles(const TsqrShape& sh, size_t* ints) {
  const size_t k = sh.k;
  size_t d = 0;
  d += size_t(sh.P) * sh.b * k;          // leafV
  d += size_t(sh.P) * k;                 // leafTau
  d += size_t(sh.inner) * 2 * k * k;     // nodeV
  d += size_t(sh.inner) * k;             // nodeTau
  d += size_t(sh.P + sh.inner) * k * k;  // nodeR
  if (ints) *ints = size_t(std::max(sh.inner, 1));
  return d;
}

void tsqr_bind(const TsqrShape& sh, double* base, int* ibase, TsqrWork* w) {
  const size_t k = sh.k;
  double* p = base;
  w->leafV = p; p += size_t(sh.P) * sh.b * k;
  w->leafTau = p; p += size_t(sh.P) * k;
  w->nodeV = p; p += size_t(sh.inner) * 2 * k * k;
  w->nodeTau = p; p += size_t(sh.inner) * k;
  w->nodeR = p;
  w->counters = ibase;
}

int tsqr_launch(const TsqrShape& sh, const TsqrWork& w, const double* A, int64_t a_rs, int64_t a_cs, double* Q,
                int64_t q_rs, int64_t q_cs, double* R, cudaStream_t s, const int* skip_unless) {
  if (sh.k < 1 || sh.k > TSQR_KMAX || sh.m < sh.k) {
    set_error("tsqr: unsupported shape m=" + std::to_string(sh.m) + " k=" + std::to_string(sh.k));
    return TT_EUNSUPPORTED;
  }
  TsqrArgs a;
  a.m = sh.m; a.k = sh.k; a.b = sh.b; a.P = sh.P; a.L = sh.L;
  a.A = A; a.a_rs = a_rs; a.a_cs = a_cs;
  a.Q = Q; a.q_rs = q_rs; a.q_cs = q_cs;
  a.R = R; a.w = w;
  a.skip_unless = skip_unless;
  const int rows_max = std::max(sh.b, 2 * sh.k);
  const size_t up_smem = (size_t(rows_max) * sh.k + 2 * sh.k + 33) * sizeof(double);
  const size_t dn_smem = (size_t(rows_max) * sh.k + rows_max + sh.k) * sizeof(double);
  static bool attr_done = false;
  if (!attr_done) {
    TTR_CHECK_CUDA(cudaFuncSetAttribute(tsqr_up_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024));
    TTR_CHECK_CUDA(cudaFuncSetAttribute(tsqr_down_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024));
    attr_done = true;
  }
  TTR_PREFER_SHARED(tsqr_up_kernel);
  tsqr_up_kernel<<<sh.P, TQ_THREADS, up_smem, s>>>(a);
  TTR_CHECK_LAUNCH();
  prof_count_launch(1);
  if (Q) {
    TTR_PREFER_SHARED(tsqr_down_kernel);
    tsqr_down_kernel<<<sh.P, TQ_THREADS, dn_smem, s>>>(a);
    TTR_CHECK_LAUNCH();
  prof_count_launch(1);
  }
  return TT_OK;
}

int tsqr_fallback_runs(long long* out) {
  unsigned long long v = 0;
  TTR_CHECK_CUDA(cudaMemcpyFromSymbol(&v, g_tsqr_runs, sizeof(v)));
  *out = (long long)v;
  return TT_OK;
}

}  // namespace ttr

// Elementwise kernels: constant fill, the counter-based Gaussian sketch of
// Definition 3.1, the truncation threshold and rank-dependent core compaction.
#include <algorithm>
#include <cmath>

#include "kernels.cuh"
#include "prof.cuh"

namespace ttr {

namespace {

__global__ void fill_kernel(double* p, int64_t n, double v) {
  for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x)
    p[i] = v;
}

// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11): 10 rounds of
// (hi0, lo0) = M0*c0, (hi1, lo1) = M1*c2 (64-bit products),
// c = (hi1 ^ c1 ^ k0, lo1, hi0 ^ c3 ^ k1, lo0), key += Weyl constants.
__device__ __forceinline__ void philox4x32_10(uint32_t c[4], uint32_t k0, uint32_t k1) {
  const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u, W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    if (r > 0) { k0 += W0; k1 += W1; }
    const uint64_t p0 = uint64_t(M0) * c[0];
    const uint64_t p1 = uint64_t(M1) * c[2];
    const uint32_t hi0 = uint32_t(p0 >> 32), lo0 = uint32_t(p0);
    const uint32_t hi1 = uint32_t(p1 >> 32), lo1 = uint32_t(p1);
    const uint32_t n0 = hi1 ^ c[1] ^ k0, n2 = hi0 ^ c[3] ^ k1;
    c[0] = n0; c[1] = lo1; c[2] = n2; c[3] = lo0;
  }
}

__device__ __forceinline__ double u52(uint32_t a, uint32_t b) {
  const uint64_t bits = (uint64_t(a) << 20) | (uint64_t(b) >> 12);
  return (double(bits) + 0.5) * 0x1p-52;
}

// Entries 2p and 2p + 1 of a sketch core: Box-Muller on one Philox output.
__device__ __forceinline__ void sketch_pair(double* out, int64_t E, int64_t p, int core_index, uint32_t k0,
                                            uint32_t k1, double stdv) {
  uint32_t c[4] = {uint32_t(uint64_t(p)), uint32_t(uint64_t(p) >> 32), uint32_t(core_index), 0x7474726Eu};
  philox4x32_10(c, k0, k1);
  const double u1 = u52(c[0], c[1]), u2 = u52(c[2], c[3]);
  const double rad = sqrt(-2.0 * log(u1));
  double sn, cs;
  sincospi(2.0 * u2, &sn, &cs);
  out[2 * p] = rad * cs * stdv;
  if (2 * p + 1 < E) out[2 * p + 1] = rad * sn * stdv;
}

__global__ void sketch_kernel(double* out, int64_t E, int core_index, uint32_t k0, uint32_t k1, double stdv,
                              const uint64_t* seed_dev) {
  if (seed_dev) {                       // seed of this run, written by the host before a graph replay
    const uint64_t sd = *seed_dev;
    k0 = uint32_t(sd);
    k1 = uint32_t(sd >> 32);
  }
  // equal contiguous chunks per block: the pairs are FP64-bound (log, sqrt,
  // sincospi), so the SM with the most pairs sets the kernel's length
  const int64_t npairs = (E + 1) / 2;
  const int64_t chunk = (npairs + gridDim.x - 1) / gridDim.x;
  const int64_t p0 = blockIdx.x * chunk, p1 = min(npairs, p0 + chunk);
  for (int64_t p = p0 + threadIdx.x; p < p1; p += blockDim.x) sketch_pair(out, E, p, core_index, k0, k1, stdv);
}

// Many sketch cores at once: job blockIdx.y, its pairs over blockIdx.x.
__global__ void sketch_batch_kernel(const SketchJob* __restrict__ jobs) {
  const SketchJob j = jobs[blockIdx.y];
  const uint64_t sd = *j.seed;
  const int64_t npairs = (j.E + 1) / 2;
  for (int64_t p = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; p < npairs;
       p += int64_t(gridDim.x) * blockDim.x)
    sketch_pair(j.out, j.E, p, j.core_index, uint32_t(sd), uint32_t(sd >> 32), j.stdv);
}

__global__ void norm_eps_kernel(const double* x, int64_t n, double tol, int N, double* eps_out) {
  __shared__ double red[32];
  double s = 0.0;
  for (int64_t i = threadIdx.x; i < n; i += blockDim.x) s = fma(x[i], x[i], s);
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int i = 0; i < int(blockDim.x >> 5); ++i) t += red[i];
    eps_out[0] = tol * sqrt(t) / sqrt(double(max(N - 1, 1)));
    eps_out[1] = sqrt(t);
  }
}

__global__ void compact_kernel(const double* src, double* dst, int64_t r0max, int64_t I, int64_t r1max,
                               const int64_t* r0p, const int64_t* r1p) {
  const int64_t r0 = r0p ? *r0p : r0max, r1 = r1p ? *r1p : r1max;
  const int64_t n = r0 * I * r1;
  for (int64_t e = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; e < n; e += int64_t(gridDim.x) * blockDim.x) {
    const int64_t b = e % r1, ai = e / r1;
    const int64_t i = ai % I, a = ai / I;
    dst[e] = src[(a * I + i) * r1max + b];
  }
}

unsigned grid_for(int64_t n, int threads) {
  return unsigned(std::max<int64_t>(1, std::min<int64_t>(ceil_div(n, threads), int64_t(num_sms()) * 16)));
}

}  // namespace

int fill_launch(double* p, int64_t n, double v, cudaStream_t s) {
  if (n <= 0) return TT_OK;
  TTR_PREFER_SHARED(fill_kernel);
  fill_kernel<<<grid_for(n, 256), 256, 0, s>>>(p, n, v);
  TTR_CHECK_LAUNCH();
  prof_count_launch(1);
  return TT_OK;
}

int sketch_batch_launch(const SketchJob* d_jobs, int njobs, int64_t max_entries, cudaStream_t s) {
  if (njobs <= 0) return TT_OK;
  if (njobs > 65535) {
    set_error("batched sketch: at most 65535 cores per launch");
    return TT_EUNSUPPORTED;
  }
  const unsigned gx = unsigned(std::max<int64_t>(1, std::min<int64_t>(ceil_div((max_entries + 1) / 2, 256), 16)));
  TTR_PREFER_SHARED(sketch_batch_kernel);
  sketch_batch_kernel<<<dim3(gx, unsigned(njobs)), 256, 0, s>>>(d_jobs);
  TTR_CHECK_LAUNCH();
  prof_count_launch(1);
  return TT_OK;
}

SketchJob sketch_job(double* out, int64_t r0, int64_t I, int64_t r1, int core_index, const uint64_t* seed_dev) {
  SketchJob j{};
  j.out = out;
  j.E = r0 * I * r1;
  j.core_index = core_index;
  j.stdv = 1.0 / std::sqrt(double(r0) * double(I) * double(r1));
  j.seed = seed_dev;
  return j;
}

int sketch_launch(double* out, int64_t r0, int64_t I, int64_t r1, int core_index, uint64_t seed,
                  const uint64_t* seed_dev, cudaStream_t s) {
  const int64_t E = r0 * I * r1;
  if (E <= 0) return TT_OK;
  const double stdv = 1.0 / std::sqrt(double(r0) * double(I) * double(r1));
  TTR_PREFER_SHARED(sketch_kernel);
  // two blocks per SM, each an equal share of the pairs (at least 32)
  const unsigned nb = unsigned(std::max<int64_t>(1, std::min<int64_t>(2 * int64_t(num_sms()), ceil_div((E + 1) / 2, 32))));
  sketch_kernel<<<nb, 256, 0, s>>>(out, E, core_index, uint32_t(seed), uint32_t(seed >> 32), stdv, seed_dev);
  TTR_CHECK_LAUNCH();
  prof_count_launch(1);
  return TT_OK;
}

int norm_eps_launch(const double* x, int64_t n, double tol, int N, double* eps_out, cudaStream_t s) {
  TTR_PREFER_SHARED(norm_eps_kernel);
  norm_eps_kernel<<<1, 1024, 0, s>>>(x, n, tol, N, eps_out);
  TTR_CHECK_LAUNCH();
  prof_count_launch(1);
  return TT_OK;
}

int compact_core_launch(const double* src, double* dst, int64_t r0max, int64_t I, int64_t r1max,
                        const int64_t* r0p, const int64_t* r1p, cudaStream_t s) {
  TTR_PREFER_SHARED(compact_kernel);
  compact_kernel<<<grid_for(r0max * I * r1max, 256), 256, 0, s>>>(src, dst, r0max, I, r1max, r0p, r1p);
  TTR_CHECK_LAUNCH();
  prof_count_launch(1);
  return TT_OK;
}

int num_sms() {
  static int n = 0;
  if (n == 0) {
    int dev = 0;
    cudaGetDevice(&dev);
    if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n <= 0) n = 152;
  }
  return n;
}

}  // namespace ttr

// ---------------------------------------------------------------------------
// Batched strided 3-D copies dst[a, i, b] = scale * src[a, i, b] (one launch for
// all summand blocks of a formed TT-sum core, Section 2.1).
namespace ttr {
namespace {
__global__ void copy3_kernel(const Copy3* __restrict__ d, int n, int64_t total) {
  for (int64_t e = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; e < total; e += int64_t(gridDim.x) * blockDim.x) {
    int lo = 0, hi = n - 1;
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (d[mid].begin <= e) lo = mid; else hi = mid - 1;
    }
    const Copy3& c = d[lo];
    int64_t l = e - c.begin;
    const int64_t z = l % c.n2; l /= c.n2;
    const int64_t y = l % c.n1;
    const int64_t x = l / c.n1;
    c.dst[x * c.d0 + y * c.d1 + z * c.d2] = c.scale * c.src[x * c.s0 + y * c.s1 + z * c.s2];
  }
}
}  // namespace

int copy3_launch(const Copy3* d_descs, int n, int64_t total, cudaStream_t s) {
  if (n == 0 || total == 0) return TT_OK;
  TTR_PREFER_SHARED(copy3_kernel);
  copy3_kernel<<<grid_for(total, 256), 256, 0, s>>>(d_descs, n, total);
  TTR_CHECK_LAUNCH();
  prof_count_launch(1);
  return TT_OK;
}
}  // namespace ttr

namespace ttr {
namespace {
__global__ void or_flag_kernel(int* dst, const int* src, int bit) {
  if (threadIdx.x == 0 && src[0]) dst[0] |= bit;
}
}  // namespace
__global__ void cvt_f32_f64_kernel(const float* __restrict__ src, double* __restrict__ dst, int64_t n) {
  for (int64_t e = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; e < n; e += int64_t(gridDim.x) * blockDim.x)
    dst[e] = double(src[e]);
}
__global__ void cvt_f64_f32_kernel(const double* __restrict__ src, float* __restrict__ dst, int64_t n) {
  for (int64_t e = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; e < n; e += int64_t(gridDim.x) * blockDim.x)
    dst[e] = float(src[e]);
}
int cvt_f32_f64_launch(const float* src, double* dst, int64_t n, cudaStream_t s) {
  if (!src || !dst || n <= 0) return TT_OK;
  const unsigned g = unsigned(std::max<int64_t>(1, std::min<int64_t>(ceil_div(n, 256), 4 * num_sms())));
  TTR_PREFER_SHARED(cvt_f32_f64_kernel);
  cvt_f32_f64_kernel<<<g, 256, 0, s>>>(src, dst, n);
  TTR_CHECK_LAUNCH();
  prof_count_launch(1);
  return TT_OK;
}
int cvt_f64_f32_launch(const double* src, float* dst, int64_t n, cudaStream_t s) {
  if (!src || !dst || n <= 0) return TT_OK;
  const unsigned g = unsigned(std::max<int64_t>(1, std::min<int64_t>(ceil_div(n, 256), 4 * num_sms())));
  TTR_PREFER_SHARED(cvt_f64_f32_kernel);
  cvt_f64_f32_kernel<<<g, 256, 0, s>>>(src, dst, n);
  TTR_CHECK_LAUNCH();
  prof_count_launch(1);
  return TT_OK;
}
__global__ void copy_if_kernel(double* __restrict__ dst, const double* __restrict__ src, int64_t n,
                               const int* skip_if) {
  if (skip_if && __ldcg(skip_if) != 0) return;
  for (int64_t e = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; e < n; e += int64_t(gridDim.x) * blockDim.x)
    dst[e] = src[e];
}
int copy_if_launch(double* dst, const double* src, int64_t n, const int* skip_if, cudaStream_t s) {
  if (!dst || !src || n <= 0) return TT_OK;
  const unsigned g = unsigned(std::max<int64_t>(1, std::min<int64_t>(ceil_div(n, 256), 4 * num_sms())));
  TTR_PREFER_SHARED(copy_if_kernel);
  copy_if_kernel<<<g, 256, 0, s>>>(dst, src, n, skip_if);
  TTR_CHECK_LAUNCH();
  prof_count_launch(1);
  return TT_OK;
}
__global__ void set_flag_kernel(int* dst) {
  if (threadIdx.x == 0) dst[0] = 1;
}
int set_flag_launch(int* dst, cudaStream_t s) {
  if (!dst) return TT_OK;
  TTR_PREFER_SHARED(set_flag_kernel);
  set_flag_kernel<<<1, 32, 0, s>>>(dst);
  TTR_CHECK_LAUNCH();
  prof_count_launch(1);
  return TT_OK;
}
int or_flag_launch(int* dst, const int* src, int bit, cudaStream_t s) {
  if (!dst || !src) return TT_OK;
  TTR_PREFER_SHARED(or_flag_kernel);
  or_flag_kernel<<<1, 32, 0, s>>>(dst, src, bit);
  TTR_CHECK_LAUNCH();
  prof_count_launch(1);
  return TT_OK;
}
}  // namespace ttr

// ---------------------------------------------------------------------------
// Small dense helpers of the fixed-sketch adjoint.
namespace ttr {
namespace {

// X = T^{-1} for an upper-triangular k x k row-major T: one column per thread,
// back substitution.
__global__ void triu_inverse_kernel(const double* T, double* X, int k) {
  for (int c = threadIdx.x; c < k; c += blockDim.x) {
    for (int i = k - 1; i > c; --i) X[i * k + c] = 0.0;
    X[c * k + c] = 1.0 / T[c * k + c];
    for (int i = c - 1; i >= 0; --i) {
      double s = 0.0;
      for (int j = i + 1; j <= c; ++j) s = fma(T[i * k + j], X[j * k + c], s);
      X[i * k + c] = -s / T[i * k + i];
    }
  }
}

// A := tril(A) + tril(A, -1)^T in place (k x k row-major); only the strict upper part is written.
__global__ void sym_lower_kernel(double* A, int k) {
  for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < k * k; idx += gridDim.x * blockDim.x) {
    const int i = idx / k, j = idx - i * k;
    if (j > i) A[idx] = A[j * k + i];
  }
}

__global__ void axpy_kernel(double* y, const double* x, int64_t n) {
  for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x)
    y[i] += x[i];
}

}  // namespace

int triu_inverse_launch(const double* T, double* X, int k, cudaStream_t s) {
  if (k <= 0 || !T || !X) return TT_OK;
  TTR_PREFER_SHARED(triu_inverse_kernel);
  triu_inverse_kernel<<<1, 256, 0, s>>>(T, X, k);
  TTR_CHECK_LAUNCH();
  prof_count_launch(1);
  return TT_OK;
}

int sym_lower_launch(double* A, int k, cudaStream_t s) {
  if (k <= 0 || !A) return TT_OK;
  TTR_PREFER_SHARED(sym_lower_kernel);
  sym_lower_kernel<<<grid_for(int64_t(k) * k, 256), 256, 0, s>>>(A, k);
  TTR_CHECK_LAUNCH();
  prof_count_launch(1);
  return TT_OK;
}

int axpy_launch(double* y, const double* x, int64_t n, cudaStream_t s) {
  if (n <= 0 || !y || !x) return TT_OK;
  TTR_PREFER_SHARED(axpy_kernel);
  axpy_kernel<<<grid_for(n, 256), 256, 0, s>>>(y, x, n);
  TTR_CHECK_LAUNCH();
  prof_count_launch(1);
  return TT_OK;
}

}  // namespace ttr

// Diagnostic: a plain tcgen05 bf16 GEMM D = A B^T (fp32 accumulate in TMEM),
// one CTA per 128-row tile, K in chunks of 64. It checks the tensor-core unit
// (descriptors, TMEM, commit / wait) in isolation; the rounding path uses the
// same helpers through the split FP64 GEMM.
#include <algorithm>

#include "kernels.cuh"
#include "prof.cuh"
#include "tc_sm103.cuh"

namespace ttr {
namespace {

constexpr uint32_t kWaitPolls = 1u << 24;

__global__ void __launch_bounds__(128) tc_selftest_kernel(int M, int N, int K, const __nv_bfloat16* __restrict__ A,
                                                          const __nv_bfloat16* __restrict__ B, float* D, int* err) {
  extern __shared__ __align__(1024) uint8_t smem[];
  uint8_t* As = smem;                      // 128 x 64 bf16, canonical
  uint8_t* Bs = smem + 16384;              // N x 64 bf16, canonical
  __shared__ __align__(8) uint64_t bar;
  __shared__ uint32_t tmem_base;
  __shared__ int s_fail;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int m0 = blockIdx.x * 128;
  const uint32_t ncols = tc::tmem_cols_for(N);
  if (warp == 0) {
    tc::tmem_alloc(&tmem_base, ncols);
    tc::tmem_relinquish();
  }
  if (tid == 0) {
    tc::mbar_init(&bar, 1);
    s_fail = 0;
  }
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t taddr = tmem_base;
  const uint32_t idesc = tc::idesc_bf16_f32(128, N);
  uint32_t phase = 0;
  for (int kc = 0; kc < K; kc += 64) {
    // 16-byte vectors: (row, k-group of 8)
    for (int v = tid; v < 128 * 8; v += 128) {
      const int r = v >> 3, kg = v & 7;
      uint4 val = make_uint4(0, 0, 0, 0);
      if (m0 + r < M) val = *reinterpret_cast<const uint4*>(A + size_t(m0 + r) * K + kc + kg * 8);
      *reinterpret_cast<uint4*>(As + tc::canon_off(r, kg * 8)) = val;
    }
    for (int v = tid; v < N * 8; v += 128) {
      const int r = v >> 3, kg = v & 7;
      const uint4 val = *reinterpret_cast<const uint4*>(B + size_t(r) * K + kc + kg * 8);
      *reinterpret_cast<uint4*>(Bs + tc::canon_off(r, kg * 8)) = val;
    }
    tc::fence_async_smem();
    __syncthreads();
    if (tid == 0) {
      tc::fence_after_sync();
      const uint32_t a0 = tc::smem_u32(As), b0 = tc::smem_u32(Bs);
#pragma unroll
      for (int s = 0; s < 4; ++s)
        tc::mma_bf16(taddr, tc::smem_desc(a0 + 256 * s, 128, 1024), tc::smem_desc(b0 + 256 * s, 128, 1024), idesc,
                     (kc > 0 || s > 0) ? 1u : 0u);
      tc::mma_commit(&bar);
    }
    if (!tc::mbar_wait_bounded(&bar, phase, kWaitPolls)) atomicExch(&s_fail, 1);
    phase ^= 1;
    tc::fence_after_sync();
    __syncthreads();
    if (s_fail) break;
  }
  if (!s_fail) {
    const int row = m0 + warp * 32 + lane;
    for (int c = 0; c < N; c += 16) {
      float v[16];
      tc::tmem_ld16(taddr + (uint32_t(warp * 32) << 16) + uint32_t(c), v);
      if (row < M)
        for (int j = 0; j < 16; ++j) D[size_t(row) * N + c + j] = v[j];
    }
  } else if (tid == 0) {
    atomicExch(err, 1);
  }
  tc::fence_before_sync();
  __syncthreads();
  if (warp == 0) tc::tmem_dealloc(taddr, ncols);
}

}  // namespace
}  // namespace ttr

using namespace ttr;

extern "C" int tt_selftest_tcgen05_bf16(int32_t M, int32_t N, int32_t K, const void* A, const void* B, float* D,
                                        int* err, void* stream) {
  if (M < 1 || N < 16 || N > 256 || (N % 16) != 0 || K < 64 || (K % 64) != 0 || !A || !B || !D || !err) {
    set_error("tt_selftest_tcgen05_bf16: need N in [16, 256] multiple of 16, K multiple of 64, non-null pointers");
    return TT_EINVAL;
  }
  const size_t smem = 16384 + size_t(N) * 128;
  static bool attr = false;
  if (!attr) {
    TTR_CHECK_CUDA(cudaFuncSetAttribute(tc_selftest_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, 64 * 1024));
    attr = true;
  }
  tc_selftest_kernel<<<unsigned(ceil_div(M, 128)), 128, smem, static_cast<cudaStream_t>(stream)>>>(
      M, N, K, static_cast<const __nv_bfloat16*>(A), static_cast<const __nv_bfloat16*>(B), D, err);
  TTR_CHECK_LAUNCH();
  prof_count_launch(1);
  return TT_OK;
}

// ---------------------------------------------------------------------------
// Diagnostic: the FP64 fused multiply-add rate of the GPU. Every thread runs 8
// independent FMA chains (the FP64 pipe's latency is covered by 8 chains x 8
// warps x resident CTAs) for `iters` steps on register values only; the sum of
// the chains is stored so nothing is optimized away. The timed launch covers
// every SM with `ctas_per_sm` CTAs.
namespace ttr {
namespace {
__global__ void __launch_bounds__(256) fp64_rate_kernel(int iters, double a, double b, double* out) {
  double x[8];
#pragma unroll
  for (int u = 0; u < 8; ++u) x[u] = double(threadIdx.x + u) * 1e-3;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int u = 0; u < 8; ++u) x[u] = fma(x[u], a, b);
  }
  double s = 0.0;
#pragma unroll
  for (int u = 0; u < 8; ++u) s += x[u];
  if (s == 12345.678) out[0] = s;        // never true for these inputs; keeps the chains live
}
}  // namespace
}  // namespace ttr

extern "C" int tt_probe_fp64_rate(int32_t iters, double* tflops, void* stream) {
  using namespace ttr;
  if (iters < 1 || !tflops) {
    set_error("tt_probe_fp64_rate: need iters >= 1 and an output");
    return TT_EINVAL;
  }
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const int ctas = 4 * num_sms();
  double* dummy = nullptr;
  TTR_CHECK_CUDA(cudaMallocAsync(reinterpret_cast<void**>(&dummy), sizeof(double), s));
  cudaEvent_t e0, e1;
  TTR_CHECK_CUDA(cudaEventCreate(&e0));
  TTR_CHECK_CUDA(cudaEventCreate(&e1));
  fp64_rate_kernel<<<ctas, 256, 0, s>>>(16, 0.999999, 1e-7, dummy);     // warm-up
  TTR_CHECK_LAUNCH();
  TTR_CHECK_CUDA(cudaEventRecord(e0, s));
  fp64_rate_kernel<<<ctas, 256, 0, s>>>(iters, 0.999999, 1e-7, dummy);
  TTR_CHECK_LAUNCH();
  TTR_CHECK_CUDA(cudaEventRecord(e1, s));
  TTR_CHECK_CUDA(cudaEventSynchronize(e1));
  float ms = 0.f;
  TTR_CHECK_CUDA(cudaEventElapsedTime(&ms, e0, e1));
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFreeAsync(dummy, s);
  prof_count_launch(2);
  const double flops = 2.0 * 8.0 * double(iters) * double(ctas) * 256.0;
  *tflops = flops / (double(ms) * 1e-3) / 1e12;
  return TT_OK;
}

// Grouped, batched, strided FP64 GEMM on the SIMT FP64 pipe.
//
// Every contraction of the FP64 path (partial contractions of Algorithm 3, the
// core update / sketch / projection of Algorithms 5 and 7, the factor updates
// of Algorithms 1, 2, 4, 6) is expressed as descriptors of this kernel, so one
// launch covers all summands (and all slices) of one step. FP64 on GB300 runs
// at 2 DFMA/clk/SM, so a 32x32 register tile per 256 threads keeps the FP64
// pipe, not shared memory, as the limit.
#include <algorithm>

#include "kernels.cuh"
#include "prof.cuh"

namespace ttr {

namespace {

__device__ __forceinline__ int find_desc(const GemmDesc* d, int n, int64_t t, bool elems) {
  int lo = 0, hi = n - 1;
  while (lo < hi) {
    int mid = (lo + hi + 1) >> 1;
    int64_t b = elems ? d[mid].elem_begin : d[mid].tile_begin;
    if (b <= t) lo = mid; else hi = mid - 1;
  }
  return lo;
}

__global__ void __launch_bounds__(GEMM_THREADS) gemm_f64_kernel(const GemmDesc* __restrict__ descs, int ndesc) {
  __shared__ double As[GEMM_BK][GEMM_BM + 1];
  __shared__ double Bs[GEMM_BK][GEMM_BN + 1];
  const int64_t t = blockIdx.x;
  const GemmDesc& d = descs[find_desc(descs, ndesc, t, false)];
  int64_t local = t - d.tile_begin;
  const int ntile = int(local % d.nt); local /= d.nt;
  const int mtile = int(local % d.mt); local /= d.mt;
  const int ks = int(local % d.ksplit);
  const int64_t b = local / d.ksplit;

  const int64_t k0 = ks * d.kchunk;
  const int64_t k1 = min(d.K, k0 + d.kchunk);
  const double* A = d.A + b * d.a_bs;
  const double* B = d.B + b * d.b_bs;
  const int64_t m0 = int64_t(mtile) * GEMM_BM, n0 = int64_t(ntile) * GEMM_BN;

  const int tid = threadIdx.x;
  const int tx = tid & 15, ty = tid >> 4;
  double acc[2][2] = {{0.0, 0.0}, {0.0, 0.0}};
  const bool a_kfast = (d.a_cs == 1);
  const bool b_nfast = (d.b_cs == 1);

  for (int64_t kb = k0; kb < k1; kb += GEMM_BK) {
#pragma unroll
    for (int q = 0; q < 2; ++q) {
      int e = tid + q * GEMM_THREADS;   // 0..511
      int mm, kk;
      if (a_kfast) { mm = e / GEMM_BK; kk = e % GEMM_BK; } else { kk = e / GEMM_BM; mm = e % GEMM_BM; }
      int64_t gm = m0 + mm, gk = kb + kk;
      As[kk][mm] = (gm < d.M && gk < k1) ? A[gm * d.a_rs + gk * d.a_cs] : 0.0;
      int nn, kk2;
      if (b_nfast) { kk2 = e / GEMM_BN; nn = e % GEMM_BN; } else { nn = e / GEMM_BK; kk2 = e % GEMM_BK; }
      int64_t gn = n0 + nn, gk2 = kb + kk2;
      Bs[kk2][nn] = (gn < d.N && gk2 < k1) ? B[gk2 * d.b_rs + gn * d.b_cs] : 0.0;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < GEMM_BK; ++kk) {
      double a0 = As[kk][ty], a1 = As[kk][ty + 16];
      double b0 = Bs[kk][tx], b1 = Bs[kk][tx + 16];
      acc[0][0] = fma(a0, b0, acc[0][0]);
      acc[0][1] = fma(a0, b1, acc[0][1]);
      acc[1][0] = fma(a1, b0, acc[1][0]);
      acc[1][1] = fma(a1, b1, acc[1][1]);
    }
    __syncthreads();
  }

#pragma unroll
  for (int i = 0; i < 2; ++i) {
#pragma unroll
    for (int j = 0; j < 2; ++j) {
      int64_t gm = m0 + ty + 16 * i, gn = n0 + tx + 16 * j;
      if (gm >= d.M || gn >= d.N) continue;
      if (d.ksplit == 1) {
        double* c = d.C + b * d.c_bs + gm * d.c_rs + gn * d.c_cs;
        double v = d.alpha * acc[i][j];
        if (d.beta != 0.0) v = fma(d.beta, *c, v);
        *c = v;
      } else {
        d.P[((b * d.ksplit + ks) * d.M + gm) * d.N + gn] = acc[i][j];
      }
    }
  }
}

__global__ void gemm_reduce_kernel(const GemmDesc* __restrict__ descs, int ndesc, int64_t total) {
  for (int64_t e = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; e < total;
       e += int64_t(gridDim.x) * blockDim.x) {
    const GemmDesc& d = descs[find_desc(descs, ndesc, e, true)];
    int64_t local = e - d.elem_begin;
    const int64_t MN = d.M * d.N;
    const int64_t b = local / MN;
    const int64_t r = local % MN;
    const int64_t gm = r / d.N, gn = r % d.N;
    double s = 0.0;
    for (int k = 0; k < d.ksplit; ++k) s += d.P[(b * d.ksplit + k) * MN + r];
    double* c = d.C + b * d.c_bs + gm * d.c_rs + gn * d.c_cs;
    double v = d.alpha * s;
    if (d.beta != 0.0) v = fma(d.beta, *c, v);
    *c = v;
  }
}

}  // namespace

void gemm_prepare(std::vector<GemmDesc>& g, int64_t* tiles, int64_t* elems, int64_t* pbuf, int target_ctas,
                  double* pbase) {
  int64_t t = 0, e = 0, p = 0;
  for (auto& d : g) {
    d.mt = int(ceil_div(std::max<int64_t>(d.M, 1), GEMM_BM));
    d.nt = int(ceil_div(std::max<int64_t>(d.N, 1), GEMM_BN));
    int64_t base = int64_t(d.batch) * d.mt * d.nt;
    int ks = 1;
    if (d.K > 2 * GEMM_BK && base < target_ctas) {
      int64_t want = ceil_div(target_ctas, base);
      int64_t maxk = d.K / (2 * GEMM_BK);
      ks = int(std::max<int64_t>(1, std::min<int64_t>({want, maxk, 64})));
    }
    d.ksplit = ks;
    d.kchunk = ceil_div(ceil_div(std::max<int64_t>(d.K, 1), ks), GEMM_BK) * GEMM_BK;
    d.tile_begin = t;
    t += base * ks;
    d.elem_begin = e;
    d.P = nullptr;
    if (ks > 1) {
      e += int64_t(d.batch) * d.M * d.N;
      d.P = pbase ? pbase + p : nullptr;
      p += int64_t(d.batch) * ks * d.M * d.N;
    }
  }
  *tiles = t;
  *elems = e;
  *pbuf = p;
}

int gemm_launch(const GemmDesc* d_descs, int ndesc, int64_t tiles, int64_t elems, double flops, cudaStream_t s) {
  if (ndesc == 0 || tiles == 0) return TT_OK;
  cudaEvent_t e0;
  const bool prof = prof_gemm_begin(s, &e0);
  gemm_f64_kernel<<<unsigned(tiles), GEMM_THREADS, 0, s>>>(d_descs, ndesc);
  TTR_CHECK_LAUNCH();
  prof_count_launch(1);
  if (elems > 0) {
    int64_t blocks = std::min<int64_t>(ceil_div(elems, 256), 4096);
    gemm_reduce_kernel<<<unsigned(blocks), 256, 0, s>>>(d_descs, ndesc, elems);
    TTR_CHECK_LAUNCH();
  prof_count_launch(1);
  }
  if (prof) prof_gemm_end(s, flops);
  return TT_OK;
}

}  // namespace ttr

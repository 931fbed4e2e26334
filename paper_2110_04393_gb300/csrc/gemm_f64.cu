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

__device__ __forceinline__ int find_desc(const GemmDesc* d, int n, int64_t t) {
  int lo = 0, hi = n - 1;
  while (lo < hi) {
    int mid = (lo + hi + 1) >> 1;
    if (d[mid].tile_begin <= t) lo = mid; else hi = mid - 1;
  }
  return lo;
}

__global__ void __launch_bounds__(GEMM_THREADS) gemm_f64_kernel(const GemmDesc* __restrict__ descs, int ndesc) {
  __shared__ double As[GEMM_BK][GEMM_BM + 1];
  __shared__ double Bs[GEMM_BK][GEMM_BN + 1];
  __shared__ int s_last;
  const int64_t t = blockIdx.x;
  const GemmDesc& d = descs[find_desc(descs, ndesc, t)];
  if (d.skip && __ldcg(d.skip) != 0) return;
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
  // threads whose 2x2 outputs all fall outside C skip the FMAs (padded tiles)
  const bool active = (m0 + ty < d.M) && (n0 + tx < d.N);

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
    if (active) {
#pragma unroll
      for (int kk = 0; kk < GEMM_BK; ++kk) {
        double a0 = As[kk][ty], a1 = As[kk][ty + 16];
        double b0 = Bs[kk][tx], b1 = Bs[kk][tx + 16];
        acc[0][0] = fma(a0, b0, acc[0][0]);
        acc[0][1] = fma(a0, b1, acc[0][1]);
        acc[1][0] = fma(a1, b0, acc[1][0]);
        acc[1][1] = fma(a1, b1, acc[1][1]);
      }
    }
    __syncthreads();
  }

  if (d.ksplit == 1) {
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
      for (int j = 0; j < 2; ++j) {
        int64_t gm = m0 + ty + 16 * i, gn = n0 + tx + 16 * j;
        if (gm >= d.M || gn >= d.N) continue;
        double* c = d.C + b * d.c_bs + gm * d.c_rs + gn * d.c_cs;
        double v = d.alpha * acc[i][j];
        if (d.beta != 0.0) v = fma(d.beta, *c, v);
        *c = v;
      }
    return;
  }
  // split K: publish the partial tile, the last CTA of the tile reduces
  const int64_t MN = d.M * d.N;
#pragma unroll
  for (int i = 0; i < 2; ++i)
#pragma unroll
    for (int j = 0; j < 2; ++j) {
      int64_t gm = m0 + ty + 16 * i, gn = n0 + tx + 16 * j;
      if (gm < d.M && gn < d.N) d.P[(b * d.ksplit + ks) * MN + gm * d.N + gn] = acc[i][j];
    }
  __syncthreads();
  const int64_t tile_id = (b * d.mt + mtile) * d.nt + ntile;
  if (tid == 0) {
    const int old = atom_add_acq_rel_gpu(d.cnt + tile_id, 1);
    s_last = (old == d.ksplit - 1);
    if (s_last) d.cnt[tile_id] = 0;
  }
  __syncthreads();
  if (!s_last) return;
  // sum the partials in split order; eight independent loads per output in flight
#pragma unroll
  for (int i = 0; i < 2; ++i)
#pragma unroll
    for (int j = 0; j < 2; ++j) {
      int64_t gm = m0 + ty + 16 * i, gn = n0 + tx + 16 * j;
      if (gm >= d.M || gn >= d.N) continue;
      const double* pp = d.P + b * d.ksplit * MN + gm * d.N + gn;
      double u[8] = {0, 0, 0, 0, 0, 0, 0, 0};
      int k = 0;
      for (; k + 8 <= d.ksplit; k += 8) {
#pragma unroll
        for (int q = 0; q < 8; ++q) u[q] += __ldcg(pp + (k + q) * MN);
      }
      for (; k < d.ksplit; ++k) u[0] += __ldcg(pp + k * MN);
      const double sacc = ((u[0] + u[1]) + (u[2] + u[3])) + ((u[4] + u[5]) + (u[6] + u[7]));
      double* c = d.C + b * d.c_bs + gm * d.c_rs + gn * d.c_cs;
      double v = d.alpha * sacc;
      if (d.beta != 0.0) v = fma(d.beta, *c, v);
      *c = v;
    }
}

}  // namespace

void gemm_prepare(std::vector<GemmDesc>& g, int64_t* tiles, int64_t* pbuf, int64_t* counters, int target_ctas,
                  double* pbase, int* cbase) {
  int64_t t = 0, p = 0, c = 0;
  for (auto& d : g) {
    d.mt = int(ceil_div(std::max<int64_t>(d.M, 1), GEMM_BM));
    d.nt = int(ceil_div(std::max<int64_t>(d.N, 1), GEMM_BN));
    int64_t base = int64_t(d.batch) * d.mt * d.nt;
    int ks = 1;
    if (d.K > 2 * GEMM_BK && base < target_ctas) {
      int64_t want = ceil_div(target_ctas, base);
      int64_t maxk = d.K / (2 * GEMM_BK);
      ks = int(std::max<int64_t>(1, std::min<int64_t>({want, maxk, 32})));
    }
    d.kchunk = ceil_div(ceil_div(std::max<int64_t>(d.K, 1), ks), GEMM_BK) * GEMM_BK;
    ks = int(ceil_div(std::max<int64_t>(d.K, 1), d.kchunk));   // no empty split
    d.ksplit = ks;
    d.tile_begin = t;
    t += base * ks;
    d.P = nullptr;
    d.cnt = nullptr;
    if (ks > 1) {
      d.P = pbase ? pbase + p : nullptr;
      p += int64_t(d.batch) * ks * d.M * d.N;
      d.cnt = cbase ? cbase + c : nullptr;
      c += base;
    }
  }
  *tiles = t;
  *pbuf = p;
  *counters = c;
}

int gemm_launch(const GemmDesc* d_descs, int ndesc, int64_t tiles, double flops, cudaStream_t s) {
  if (ndesc == 0 || tiles == 0) return TT_OK;
  cudaEvent_t e0;
  const bool prof = prof_gemm_begin(s, &e0);
  TTR_PREFER_SHARED(gemm_f64_kernel);
  gemm_f64_kernel<<<unsigned(tiles), GEMM_THREADS, 0, s>>>(d_descs, ndesc);
  TTR_CHECK_LAUNCH();
  prof_count_launch(1);
  if (prof) prof_gemm_end(s, flops);
  return TT_OK;
}

}  // namespace ttr

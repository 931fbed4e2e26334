// Emulated FP64 GEMM on the tcgen05 tensor cores (the contractions of the mixed
// path): C = alpha * A B + beta * C with float64 inputs and outputs, computed
// from bf16 "digit" slices whose products and sums are exact.
//
// Three launches, no FP64 arithmetic anywhere. (1) Exponents: for every row r
// of A and column c of B, the largest float64 exponent over the whole K range
// (integer atomics on the exponent bits). With E_r = that exponent + 2 every
// a_rk satisfies |a_rk| < 2^{E_r - 1}, so F = |a_rk| 2^{63 - E_r} is an integer
// below 2^62 (taken from the mantissa bits with shifts). (2) Digit planes:
// adding the constant 64 in every 7-bit digit position (plus half a unit of
// the last kept digit) and reading the digits back gives balanced digits
// d_1 .. d_s in [-64, 64] with F = sum_p d_p 2^{63 - 7p} + rounding error
// below 2^{62 - 7s}: a_rk ~ 2^{E_r} sum_p d_p 2^{-7p}. Every digit is exact in
// bf16; the s planes of every operand tile are written to global memory in
// the canonical K-major shared-memory layout, by many small blocks (the split
// is the bulk of the work and needs many warps per SM to hide its latency).
// Columns of B are split the same way (E_c). (3) Products, below.
//
// Products. Digit pairs with p + q <= s + 1 are kept; pairs of one level
// L = p + q accumulate (tcgen05.mma, fp32 in TMEM) into the TMEM region of that
// level (one MMA chain per digit of A against all digits of B at once). Per 64-wide K-chunk a level sum is an integer of magnitude at most
// 8 * 64 * 64^2 = 2^21, so fp32 holds it exactly. After each chunk the levels
// are read back, converted to integers exactly (magic-number addition) and
// added into two int64 accumulators per output, H = sum_{L<=5} D_L 2^{7(5-L)}
// and Lo = sum_{L>=6} D_L 2^{7(9-L)}. Then
//   C_rc ~ 2^{E_r + E_c - 63} (H 2^28 + Lo),
// a 128-bit integer times a power of two, which is rounded to float64 once
// with integer operations. Split-K partials are combined by integer atomics in
// L2, so the result does not depend on the order of arrival (bit-wise
// deterministic). The error per product is about 2^{1 - 7s} relative to
// max_k |a_rk| max_k |b_kc|; s = 8 keeps 56 bits (FP64 class). Rows of A or
// columns of B that hold Inf or NaN give NaN outputs; subnormals count as zero.
//
// Product tile: 128 rows (one TMEM lane each) x 32 columns, 256 threads (8
// warps). Per K-chunk (64 wide, or the K extent rounded up to 16 when K is
// short) one bulk copy brings the s planes of A and one those of B into shared
// memory (completion on an mbarrier); one thread issues the MMAs.
#include <algorithm>
#include <atomic>
#include <cmath>

#include <string>

#include "plan.cuh"
#include "prof.cuh"
#include "tc_sm103.cuh"

namespace ttr {

namespace {

constexpr int TC_BM = 128, TC_BN = 32, TC_BK = 64, TC_THREADS = 256;
constexpr int EX_OUT = 32, EX_IN = 256;   // exponent pass block: 32 rows x 256 K
constexpr uint32_t kPolls = 1u << 24;
constexpr int kExBias = 4096;             // stored exponent = e + kExBias, low 16 bits
constexpr int kExNonFinite = 0x7FFF;      // stored for Inf / NaN (above every finite code)
constexpr int kNonFinite = 1 << 20;       // decoded exponent of a row / column holding Inf or NaN

__device__ __forceinline__ int dexp(double x) {        // biased exponent, or -1 for zero / subnormal
  const uint64_t b = uint64_t(__double_as_longlong(x));
  const int e = int((b >> 52) & 0x7FF);
  return e == 0 ? -1 : (e == 0x7FF ? kExNonFinite : e - 1023 + kExBias);
}

// Balanced digits of x relative to 2^E (|x| < 2^{E-1}); d[p] for p < s.
__device__ __forceinline__ void digits(double x, int E, int s, int* d) {
  const uint64_t b = uint64_t(__double_as_longlong(x));
  const int e = int((b >> 52) & 0x7FF);
  uint64_t F = 0;
  if (e != 0) {
    const uint64_t mant = (b & ((uint64_t(1) << 52) - 1)) | (uint64_t(1) << 52);
    const int sh = (e - 1023) - E + 11;        // F = mant 2^{sh}, sh <= 9
    if (sh >= 0) F = mant << sh;
    else if (sh > -64) F = mant >> (-sh);
  }
  // + 64 in every digit position and half a unit of digit s
  uint64_t C = uint64_t(1) << (62 - 7 * s);
#pragma unroll
  for (int p = 1; p <= 8; ++p)
    if (p <= s) C += uint64_t(64) << (63 - 7 * p);
  const uint64_t G = F + C;
  const int sg = -int(b >> 63);               // 0 or -1
#pragma unroll
  for (int p = 1; p <= 8; ++p) {
    if (p > s) break;
    const int v = (p == 1) ? int(G >> 56) - 64 : int((G >> (63 - 7 * p)) & 127u) - 64;
    d[p - 1] = (v ^ sg) - sg;                 // apply the sign
  }
}

// exact float value of a small integer (|v| < 2^22) without a conversion unit
__device__ __forceinline__ float int_to_float_small(int v) {
  return __fsub_rn(__int_as_float(0x4B400000 + v), 12582912.0f);
}
// exact integer value of an fp32 holding an integer with |x| < 2^22
__device__ __forceinline__ int float_to_int_small(float x) {
  return __float_as_int(__fadd_rn(x, 12582912.0f)) - 0x4B400000;
}

// Rounds T 2^{e2} to float64, T = H 2^28 + Lo (128-bit), with integer operations.
// Kept out of line: the epilogue calls it for every output column, and inlined
// copies would overflow the instruction cache.
__device__ __noinline__ double round_i128(long long H, long long Lo, int e2) {
  const uint64_t tl = uint64_t(H) << 28;
  const long long th = H >> 36;
  uint64_t ml = tl + uint64_t(Lo);
  const long long nh = th + (Lo >> 63) + (ml < tl ? 1 : 0);
  const bool neg = nh < 0;
  uint64_t mh = uint64_t(nh);
  if (neg) {
    ml = ~ml + 1;
    mh = ~mh + (ml == 0 ? 1 : 0);
  }
  if (mh == 0 && ml == 0) return 0.0;
  const int lz = mh ? __clzll((long long)mh) : 64 + __clzll((long long)ml);
  if (lz >= 64) {
    mh = ml << (lz - 64);
    ml = 0;
  } else if (lz > 0) {
    mh = (mh << lz) | (ml >> (64 - lz));
    ml <<= lz;
  }
  int msb = 127 - lz;
  uint64_t mant = mh >> 11;
  const uint64_t rest = mh & 0x7FF;
  const bool rnd = (rest >> 10) & 1;
  const bool sticky = (rest & 0x3FF) != 0 || ml != 0;
  if (rnd && (sticky || (mant & 1))) {
    ++mant;
    if (mant >> 53) { mant >>= 1; ++msb; }
  }
  const int E = msb + e2;
  const uint64_t sgn = uint64_t(neg) << 63;
  const uint64_t frac = mant & ((uint64_t(1) << 52) - 1);
  if (E > 1023) return __longlong_as_double((long long)(sgn | (uint64_t(0x7FF) << 52)));
  if (E < -1022) {
    // below the normal range (not expected in practice): one correctly rounded multiply
    if (E < -1022 - 600) return __longlong_as_double((long long)sgn);
    const double x = __longlong_as_double((long long)(sgn | (uint64_t(E + 600 + 1023) << 52) | frac));
    return x * 0x1p-600;
  }
  return __longlong_as_double((long long)(sgn | (uint64_t(E + 1023) << 52) | frac));
}

// One output: C = alpha * round(T 2^{Er + Ec - 63}) + beta * C, NaN when the
// row or column held Inf / NaN (out of line, like round_i128). plain: alpha = 1
// and beta = 0, decided once per thread (FP64 compares cost the FP64 pipe).
__device__ __noinline__ void store_out(double* cp, long long H, long long Lo, int Er, int Ec, bool plain,
                                       double alpha, double beta) {
  double v = (Er == kNonFinite || Ec == kNonFinite) ? __longlong_as_double(0x7FF8000000000000LL)
                                                    : round_i128(H, Lo, Er + Ec - 63);
  if (!plain) {
    v *= alpha;
    if (beta != 0.0) v = fma(beta, *cp, v);      // C is read only when beta != 0
  }
  *cp = v;
}

struct TcArgs {
  const GemmDesc* descs;
  int ndesc;
  int s;          // digits per operand
  int epoch;      // tag of this launch's exponents (tags of older launches lose the max)
};

// Index of the descriptor whose block range holds block t: the largest i with
// begin(i) <= t, for the product tiles (kind 0), the exponent pass (1) or the
// split pass (2). Warp-parallel (32 descriptors per load round); every thread
// of the block calls it and gets the same answer.
__device__ __forceinline__ int find_desc(const GemmDesc* descs, int ndesc, int64_t t, int kind) {
  const int lane = threadIdx.x & 31;
  int count = 0;
  for (int base = 0; base < ndesc; base += 32) {
    const int i = base + lane;
    bool le = false;
    if (i < ndesc) {
      const int64_t b = kind == 0 ? __ldg(&descs[i].tile_begin)
                                  : (kind == 1 ? __ldg(&descs[i].exp_begin) : __ldg(&descs[i].split_begin));
      le = b <= t;
    }
    count += __popc(__ballot_sync(0xffffffffu, le));
  }
  return max(count - 1, 0);
}

// ---- pass 1: largest exponent per row of A and per column of B over all of K
__global__ void __launch_bounds__(256) tc_exponent_kernel(TcArgs args) {
  const int64_t t = blockIdx.x;
  const GemmDesc d = args.descs[find_desc(args.descs, args.ndesc, t, 1)];
  int64_t local = t - d.exp_begin;
  // block counts as in gemm_tc_prepare (at least one block per side)
  const int64_t kb = max((d.K + EX_IN - 1) / EX_IN, int64_t(1));
  const int64_t ob_a = max((d.M + EX_OUT - 1) / EX_OUT, int64_t(1));
  const int64_t ob_b = max((d.N + EX_OUT - 1) / EX_OUT, int64_t(1));
  const int64_t per_batch = (ob_a + ob_b) * kb;
  const int64_t bidx = local / per_batch;
  local -= bidx * per_batch;
  const bool sideA = local < ob_a * kb;
  if (!sideA) local -= ob_a * kb;
  const int64_t ob = local / kb, ib = local % kb;
  const double* base;
  int64_t outer, os, is;
  int* out;
  if (sideA) {
    base = d.A + bidx * d.a_bs; outer = d.M; os = d.a_rs; is = d.a_cs; out = d.ex_row + bidx * d.M;
  } else {
    base = d.B + bidx * d.b_bs; outer = d.N; os = d.b_cs; is = d.b_rs; out = d.ex_col + bidx * d.N;
  }
  const int64_t o0 = ob * EX_OUT, k0 = ib * EX_IN;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int tag = args.epoch << 16;
  if (is == 1) {
    // inner index contiguous: a warp reads along K for four rows (32 loads in flight)
    double x[4][8];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int64_t o = o0 + warp + 8 * j;
      const double* p = base + o * os;
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        const int64_t k = k0 + lane + 32 * u;
        x[j][u] = (o < outer && k < d.K) ? __ldg(p + k) : 0.0;
      }
    }
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int64_t o = o0 + warp + 8 * j;
      int m = -1;
#pragma unroll
      for (int u = 0; u < 8; ++u) m = max(m, dexp(x[j][u]));
#pragma unroll
      for (int off = 16; off; off >>= 1) m = max(m, __shfl_xor_sync(0xffffffffu, m, off));
      if (lane == 0 && o < outer && m >= 0) atomicMax(out + o, tag | m);
    }
  } else {
    // outer index contiguous (or neither): lanes along the rows, warps along K
    __shared__ int red[8][32];
    const int64_t o = o0 + lane;
    int m = -1;
    if (o < outer) {
      const double* p = base + o * os;
#pragma unroll
      for (int u0 = 0; u0 < EX_IN / 8; u0 += 16) {
        double x[16];
#pragma unroll
        for (int u = 0; u < 16; ++u) {
          const int64_t k = k0 + warp + 8 * (u0 + u);
          x[u] = (k < d.K) ? __ldg(p + k * is) : 0.0;
        }
#pragma unroll
        for (int u = 0; u < 16; ++u) m = max(m, dexp(x[u]));
      }
    }
    red[warp][lane] = m;
    __syncthreads();
    if (warp == 0) {
#pragma unroll
      for (int w = 1; w < 8; ++w) m = max(m, red[w][lane]);
      if (o < outer && m >= 0) atomicMax(out + o, tag | m);
    }
  }
}

__device__ __forceinline__ int decode_exp(int v, int epoch) {
  if ((v >> 16) != epoch) return 0;                     // no nonzero entry
  if ((v & 0xFFFF) == kExNonFinite) return kNonFinite;
  return (v & 0xFFFF) - kExBias + 2;                    // E with |x| < 2^{E-1}
}

// ---- pass 2: digit planes. A block splits a 32 x bk sub-tile of A (rows) or
// of B (columns) and writes its s bf16 planes in the canonical K-major layout
// of the 128 x bk (A) or 32 x bk (B) operand tile, padding with zeros. With a
// short K (lx) one block covers all chunks of 8 rows / columns and takes their
// largest exponents itself (written as the tags the product pass reads), so no
// exponent pass runs for that descriptor.
constexpr int64_t kLocalExpK = 512;

__device__ __forceinline__ void split_chunk(const GemmDesc& d, int s, bool sideA, int64_t bidx, int64_t tile,
                                            int quarter, int64_t kc, int64_t o0, int64_t outer, const double* base,
                                            int64_t os, int64_t is, const int* Es) {
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int bk = d.bkc;
  const int64_t nkc = d.nkc;
  const uint32_t plane = sideA ? uint32_t(TC_BM * bk * 2) : uint32_t(TC_BN * bk * 2);
  uint8_t* dst = sideA ? d.pa + ((bidx * d.mt + tile) * nkc + kc) * int64_t(s) * plane
                       : d.pb + ((bidx * d.nt + tile) * nkc + kc) * int64_t(s) * plane;
  const int ncm = bk / 2;                      // core matrices (8 rows x 8 k) in the 32 x bk sub-tile
  const int kgs = bk / 8;
  const int cr = lane >> 2, ck = (lane & 3) * 2;
  const int64_t k0 = kc * bk;
  double x[8];
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    const int cm = warp + 8 * j;
    const int rg = cm / kgs, kg = cm % kgs;
    const int64_t o = o0 + rg * 8 + cr, k = k0 + kg * 8 + ck;
    const double* p = base + o * os + k * is;
    const bool ok = cm < ncm && o < outer;
    x[2 * j] = (ok && k < d.K) ? __ldg(p) : 0.0;
    x[2 * j + 1] = (ok && k + 1 < d.K) ? __ldg(p + is) : 0.0;
  }
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    const int cm = warp + 8 * j;
    if (cm >= ncm) break;
    const int rg = cm / kgs, kg = cm % kgs;
    const int rl = rg * 8 + cr;                         // row within the 32-row sub-tile
    const int rt = sideA ? quarter * 32 + rl : rl;      // row within the operand tile
    int d0[8], d1[8];
    digits(x[2 * j], Es[rl], s, d0);
    digits(x[2 * j + 1], Es[rl], s, d1);
    const uint32_t off = tc::canon_off_w(rt, kg * 8 + ck, bk);
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      if (q >= s) break;
      const __nv_bfloat162 h = __floats2bfloat162_rn(int_to_float_small(d0[q]), int_to_float_small(d1[q]));
      *reinterpret_cast<__nv_bfloat162*>(dst + q * plane + off) = h;
    }
  }
}

// Short-K blocks: the rows (A) or columns (B) of a block over all of K are
// staged in shared memory by one round of loads (all in flight), their largest
// exponents taken there, and every chunk split from shared memory. A block
// takes 32 rows / columns when K fits one chunk (at most 64) and 8 otherwise
// (at most kLocalExpK = 512), so that a block's loads stay at 8-16 per thread.
constexpr int LX_ROWS = 8;                             // rows per block above one chunk
constexpr int LX_LD = int(kLocalExpK) + 1;             // staged row stride (doubles), 8-row blocks
constexpr int LX_LD1 = TC_BK + 1;                      // staged row stride, 32-row blocks

__host__ __device__ inline int lx_rows(int64_t nkc) { return nkc == 1 ? 32 : LX_ROWS; }

__global__ void __launch_bounds__(256) tc_split_kernel(TcArgs args) {
  __shared__ int Es[32];
  __shared__ double stg[LX_ROWS * LX_LD];
  const int64_t t = blockIdx.x;
  const GemmDesc d = args.descs[find_desc(args.descs, args.ndesc, t, 2)];
  const int s = args.s;
  const int64_t nkc = d.nkc;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  int64_t local = t - d.split_begin;
  if (!d.lx) {
    const int64_t na = int64_t(d.mt) * 4 * nkc, per_batch = na + int64_t(d.nt) * nkc;
    const int64_t bidx = local / per_batch;
    local -= bidx * per_batch;
    const bool sideA = local < na;
    int64_t kc, tile;
    int quarter = 0;
    if (sideA) {
      kc = local % nkc;
      const int64_t q4 = local / nkc;
      quarter = int(q4 & 3);
      tile = q4 >> 2;
    } else {
      local -= na;
      kc = local % nkc;
      tile = local / nkc;
    }
    const int64_t o0 = sideA ? tile * TC_BM + quarter * 32 : tile * TC_BN;   // first row (A) / column (B)
    const int64_t outer = sideA ? d.M : d.N;
    const double* base = sideA ? d.A + bidx * d.a_bs : d.B + bidx * d.b_bs;
    const int64_t os = sideA ? d.a_rs : d.b_cs, is = sideA ? d.a_cs : d.b_rs;
    const int* ex = sideA ? d.ex_row + bidx * d.M : d.ex_col + bidx * d.N;
    if (tid < 32) {
      const int64_t o = o0 + tid;
      Es[tid] = o < outer ? decode_exp(__ldcg(ex + o), args.epoch) : 0;
    }
    __syncthreads();
    split_chunk(d, s, sideA, bidx, tile, quarter, kc, o0, outer, base, os, is, Es);
    return;
  }
  // short K: R rows / columns of one operand tile
  const int R = lx_rows(nkc);
  const int ld = R == 32 ? LX_LD1 : LX_LD;
  const int64_t nsa = int64_t(d.mt) * (TC_BM / R);
  const int64_t per_batch = nsa + int64_t(d.nt) * (TC_BN / R);
  const int64_t bidx = local / per_batch;
  local -= bidx * per_batch;
  const bool sideA = local < nsa;
  if (!sideA) local -= nsa;
  const int per_tile = sideA ? TC_BM / R : TC_BN / R;
  const int64_t tile = local / per_tile;
  const int sub = int(local - tile * per_tile);
  const int64_t o0 = tile * (sideA ? TC_BM : TC_BN) + sub * R;
  const int64_t outer = sideA ? d.M : d.N;
  const double* base = sideA ? d.A + bidx * d.a_bs : d.B + bidx * d.b_bs;
  const int64_t os = sideA ? d.a_rs : d.b_cs, is = sideA ? d.a_cs : d.b_rs;
  int* ex = sideA ? d.ex_row + bidx * d.M : d.ex_col + bidx * d.N;
  const int bk = d.bkc;
  const int kp = int(nkc) * bk;                        // K padded to whole chunks
  {
    // slot u of this thread: row o, K position k. K contiguous: a warp walks
    // K along one row; else the lanes take consecutive rows. Zeros beyond K
    // and beyond the last row.
    const bool small = R == 32;
    const int nsl = small ? 8 : 16;
    double x[16];
#pragma unroll
    for (int u = 0; u < 16; ++u) {
      int o, k;
      if (is == 1) {
        o = small ? warp + 8 * (u >> 1) : warp;
        k = small ? lane + 32 * (u & 1) : lane + 32 * u;
      } else {
        o = small ? lane : (tid & 7);
        k = small ? warp + 8 * u : (tid >> 3) + 32 * u;
      }
      x[u] = (u < nsl && o0 + o < outer && k < d.K) ? __ldg(base + (o0 + o) * os + int64_t(k) * is) : 0.0;
    }
#pragma unroll
    for (int u = 0; u < 16; ++u) {
      int o, k;
      if (is == 1) {
        o = small ? warp + 8 * (u >> 1) : warp;
        k = small ? lane + 32 * (u & 1) : lane + 32 * u;
      } else {
        o = small ? lane : (tid & 7);
        k = small ? warp + 8 * u : (tid >> 3) + 32 * u;
      }
      if (u < nsl && k < kp) stg[o * ld + k] = x[u];
    }
  }
  __syncthreads();
  for (int o = warp; o < R; o += 8) {
    int m = -1;
    for (int k = lane; k < kp; k += 32) m = max(m, dexp(stg[o * ld + k]));
#pragma unroll
    for (int off = 16; off; off >>= 1) m = max(m, __shfl_xor_sync(0xffffffffu, m, off));
    if (lane == 0) {
      const int tag = m >= 0 ? ((args.epoch << 16) | m) : 0;
      if (o0 + o < outer) ex[o0 + o] = tag;
      Es[o] = decode_exp(tag, args.epoch);
    }
  }
  __syncthreads();
  // split: core matrices (8 rows x 8 K positions) of every chunk over the warps
  const uint32_t plane = sideA ? uint32_t(TC_BM * bk * 2) : uint32_t(TC_BN * bk * 2);
  const int cr = lane >> 2, ck = (lane & 3) * 2;
  const int kgs = bk / 8, ncm = (R / 8) * kgs;
  uint8_t* dst = sideA ? d.pa + (bidx * d.mt + tile) * nkc * int64_t(s) * plane
                       : d.pb + (bidx * d.nt + tile) * nkc * int64_t(s) * plane;
  for (int64_t c = 0; c < nkc; ++c) {
    for (int cm = warp; cm < ncm; cm += 8) {
      const int rg = cm / kgs, kg = cm - rg * kgs;
      const int rl = rg * 8 + cr;                      // row within the block
      const int kk = int(c) * bk + kg * 8 + ck;
      int d0[8], d1[8];
      digits(stg[rl * ld + kk], Es[rl], s, d0);
      digits(stg[rl * ld + kk + 1], Es[rl], s, d1);
      uint8_t* dc = dst + c * int64_t(s) * plane + tc::canon_off_w(sub * R + rl, kg * 8 + ck, bk);
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        if (q >= s) break;
        const __nv_bfloat162 h = __floats2bfloat162_rn(int_to_float_small(d0[q]), int_to_float_small(d1[q]));
        *reinterpret_cast<__nv_bfloat162*>(dc + q * plane) = h;
      }
    }
  }
}

// ---- pass 3: digit products on the tensor cores
__global__ void __launch_bounds__(TC_THREADS, 1) gemm_tc_kernel(TcArgs args, int* err) {
  extern __shared__ __align__(1024) uint8_t smem[];
  const int s = args.s;
  __shared__ __align__(8) uint64_t lbar, mbar;
  __shared__ uint32_t tmem_base;
  __shared__ int s_fail, s_last, s_issued;
  __shared__ int Er[TC_BM], Ec[TC_BN];

  const int64_t t = blockIdx.x;
  const GemmDesc d = args.descs[find_desc(args.descs, args.ndesc, t, 0)];
  const int bk = d.bkc;
  const uint32_t pA = uint32_t(TC_BM * bk * 2), pB = uint32_t(TC_BN * bk * 2);   // plane bytes
  uint8_t* As = smem;                                  // s planes of 128 x bk bf16
  uint8_t* Bs = smem + s * pA;                         // s planes of 32 x bk bf16
  int64_t local = t - d.tile_begin;
  const int ntile = int(local % d.nt); local /= d.nt;
  const int mtile = int(local % d.mt); local /= d.mt;
  const int ks = int(local % d.ksplit);
  const int64_t bidx = local / d.ksplit;
  const int64_t m0 = int64_t(mtile) * TC_BM, n0 = int64_t(ntile) * TC_BN;
  const int64_t cps = d.kchunk / bk;                   // chunks per split
  const int64_t kc_begin = int64_t(ks) * cps;
  const int64_t kc_end = min(d.nkc, kc_begin + cps);

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const uint32_t ncols = tc::tmem_cols_for(s * TC_BN);   // levels 2 .. s + 1
  if (warp == 0) {
    tc::tmem_alloc(&tmem_base, ncols);
    tc::tmem_relinquish();
  }
  if (tid == 0) {
    tc::mbar_init(&lbar, 1);
    tc::mbar_init(&mbar, 1);
    s_fail = 0;
  }
  for (int i = tid; i < TC_BM + TC_BN; i += TC_THREADS) {
    if (i < TC_BM) {
      const int64_t r = m0 + i;
      Er[i] = r < d.M ? decode_exp(__ldcg(d.ex_row + bidx * d.M + r), args.epoch) : 0;
    } else {
      const int64_t c = n0 + (i - TC_BM);
      Ec[i - TC_BM] = c < d.N ? decode_exp(__ldcg(d.ex_col + bidx * d.N + c), args.epoch) : 0;
    }
  }
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t taddr = tmem_base;
  const uint8_t* srcA = d.pa + ((bidx * d.mt + mtile) * d.nkc) * int64_t(s) * pA;
  const uint8_t* srcB = d.pb + ((bidx * d.nt + ntile) * d.nkc) * int64_t(s) * pB;

  // epilogue roles: TMEM lane quadrant q (warp % 4), column half ch
  const int q = warp & 3, ch = warp >> 2;
  long long accH[16], accL[16];
#pragma unroll
  for (int j = 0; j < 16; ++j) { accH[j] = 0; accL[j] = 0; }
  uint32_t lph = 0, mph = 0;

  for (int64_t kc = kc_begin; kc < kc_end; ++kc) {
    // ---- the chunk's s planes of A and of B, one bulk copy each
    if (tid == 0) {
      tc::mbar_arrive_expect_tx(&lbar, uint32_t(s) * (pA + pB));
      tc::bulk_g2s(As, srcA + kc * int64_t(s) * pA, uint32_t(s) * pA, &lbar);
      tc::bulk_g2s(Bs, srcB + kc * int64_t(s) * pB, uint32_t(s) * pB, &lbar);
    }
    const bool loaded = tc::mbar_wait_bounded(&lbar, lph, kPolls);
    if (!loaded) {
      atomicExch(&s_fail, 1);
      tc::mbar_wait_bounded(&lbar, lph, kPolls);      // give the copy in flight one more bounded wait
    }
    lph ^= 1;
    // ---- one thread issues every kept digit-pair product of this chunk (only
    //      after its own wait saw the copy complete); every thread then waits
    //      for the issued products before anything else touches TMEM or smem
    if (tid == 0) s_issued = loaded ? 1 : 0;
    if (tid == 0 && loaded) {
      tc::fence_after_sync();
      // B planes are contiguous, i.e. one K-major operand of 32 s rows: the MMA
      // of A digit p against its first 32 (s + 1 - p) rows (digits q <= s + 1
      // - p) adds d_p e_q into columns (p + q - 2) 32, the region of level
      // p + q; products of higher levels are never formed (they would be
      // dropped), so the chains shrink with p and every column written is below
      // 32 s. The p = 1 chain starts all kept levels 2 .. s + 1.
      const uint32_t a0 = tc::smem_u32(As), b0 = tc::smem_u32(Bs);
      const int steps = bk / 16;
      for (int p = 1; p <= s; ++p)
        for (int st = 0; st < steps; ++st)
          tc::mma_bf16(taddr + uint32_t((p - 1) * TC_BN), tc::smem_desc(a0 + (p - 1) * pA + 256 * st, 128, 16 * bk),
                       tc::smem_desc(b0 + 256 * st, 128, 16 * bk),
                       tc::idesc_bf16_f32(TC_BM, TC_BN * (s + 1 - p)), (p == 1 && st == 0) ? 0u : 1u);
      tc::mma_commit(&mbar);
    }
    __syncthreads();
    if (s_issued) {
      if (!tc::mbar_wait_bounded(&mbar, mph, kPolls)) {
        atomicExch(&s_fail, 1);
        tc::mbar_wait_bounded(&mbar, mph, kPolls);    // let the MMAs in flight finish (bounded)
      }
      mph ^= 1;
    }
    tc::fence_after_sync();
    __syncthreads();
    if (s_fail) break;
    // ---- exact level sums -> int64 accumulators (TMEM lane q*32+lane, columns
    //      ch*16..+16); levels are read four at a time, then one wait
    const uint32_t tl = taddr + (uint32_t(q * 32) << 16) + uint32_t(ch * 16);
#pragma unroll
    for (int g = 0; g < 2; ++g) {
      if (2 + 4 * g > s + 1) break;
      uint32_t v[64];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int L = 2 + 4 * g + u;
        if (L <= s + 1) tc::tmem_ld16_nowait(tl + uint32_t((L - 2) * TC_BN), v + 16 * u);
        else {
#pragma unroll
          for (int j = 0; j < 16; ++j) v[16 * u + j] = 0u;
        }
      }
      tc::tmem_wait_ld64(v);
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int L = 2 + 4 * g + u;
        if (L > s + 1) break;
        const int sh = 7 * (3 - u);                 // 7 (5 - L) for H, 7 (9 - L) for Lo
#pragma unroll
        for (int j = 0; j < 16; ++j) {
          const long long iv = (long long)float_to_int_small(__uint_as_float(v[16 * u + j])) << sh;
          if (g == 0) accH[j] += iv; else accL[j] += iv;
        }
      }
    }
    tc::fence_before_sync();
    __syncthreads();
  }

  const int rr = q * 32 + lane;
  const int64_t row = m0 + rr;
  const int64_t c0 = n0 + ch * 16;
  const int64_t row_off = d.c_rdiv > 0 ? (row / d.c_rdiv) * d.c_rs + (row % d.c_rdiv) * d.c_rs2 : row * d.c_rs;
  double* const crow = d.C + bidx * d.c_bs + row_off;
  const bool plain = (d.alpha == 1.0 && d.beta == 0.0);
  auto store = [&](int j, long long H, long long Lo) {
    store_out(crow + (c0 + j) * d.c_cs, H, Lo, Er[rr], Ec[ch * 16 + j], plain, d.alpha, d.beta);
  };
  if (!s_fail) {
    if (d.ksplit == 1) {
      if (row < d.M) {
#pragma unroll
        for (int j = 0; j < 16; ++j)
          if (c0 + j < d.N) store(j, accH[j], accL[j]);
      }
    } else {
      // integer partials meet in L2; the last CTA of the tile rounds and writes C
      const int64_t tile_id = (bidx * d.mt + mtile) * d.nt + ntile;
      unsigned long long* acc = reinterpret_cast<unsigned long long*>(d.acc) + tile_id * (2 * TC_BM * TC_BN);
#pragma unroll
      for (int j = 0; j < 16; ++j) {
        const int cc = ch * 16 + j;
        if (accH[j]) atomicAdd(acc + cc * TC_BM + rr, (unsigned long long)accH[j]);
        if (accL[j]) atomicAdd(acc + TC_BM * TC_BN + cc * TC_BM + rr, (unsigned long long)accL[j]);
      }
      __syncthreads();
      if (tid == 0) {
        const int old = atom_add_acq_rel_gpu(d.cnt + tile_id, 1);
        s_last = (old == d.ksplit - 1);
        if (s_last) d.cnt[tile_id] = 0;
      }
      __syncthreads();
      if (s_last) {
#pragma unroll
        for (int j = 0; j < 16; ++j) {
          const int cc = ch * 16 + j;
          accH[j] = (long long)__ldcg(acc + cc * TC_BM + rr);
          accL[j] = (long long)__ldcg(acc + TC_BM * TC_BN + cc * TC_BM + rr);
        }
#pragma unroll
        for (int j = 0; j < 16; ++j) {
          const int cc = ch * 16 + j;
          acc[cc * TC_BM + rr] = 0;
          acc[TC_BM * TC_BN + cc * TC_BM + rr] = 0;
          if (row < d.M && c0 + j < d.N) store(j, accH[j], accL[j]);
        }
      }
    }
  } else {
    // a wait gave up: raise the flag and leave NaN in this CTA's outputs
    if (tid == 0) atomicOr(err, DEV_TIMEOUT);
    if (row < d.M)
      for (int j = 0; j < 16; ++j)
        if (c0 + j < d.N)
          d.C[bidx * d.c_bs + row_off + (c0 + j) * d.c_cs] = __longlong_as_double(0x7FF8000000000000LL);
  }
  tc::fence_before_sync();
  __syncthreads();
  if (warp == 0) tc::tmem_dealloc(taddr, ncols);
}

// ---- fused: exponents, digit split and products in one launch. The tile's
// rows of A and columns of B are scanned for their largest exponents over all
// of K (every CTA of a split-K tile finds the same ones, so their integer
// partials still add exactly), then every K-chunk is split by all threads
// straight into the shared-memory planes the MMAs read (the layout the
// three-pass form copies in), so no digit plane goes through global memory.
// Same arithmetic as the three-pass form: bit-identical results.
__global__ void __launch_bounds__(TC_THREADS, 1) gemm_tcf_kernel(TcArgs args, int* err) {
  extern __shared__ __align__(1024) uint8_t smem[];
  const int s = args.s;
  __shared__ __align__(8) uint64_t mbar;
  __shared__ uint32_t tmem_base;
  __shared__ int s_fail, s_last, s_issued;
  __shared__ int Er[TC_BM], Ec[TC_BN];

  const int64_t t = blockIdx.x;
  const GemmDesc d = args.descs[find_desc(args.descs, args.ndesc, t, 0)];
  const int bk = d.bkc;
  const uint32_t pA = uint32_t(TC_BM * bk * 2), pB = uint32_t(TC_BN * bk * 2);   // plane bytes
  uint8_t* As = smem;                                  // s planes of 128 x bk bf16
  uint8_t* Bs = smem + s * pA;                         // s planes of 32 x bk bf16
  int64_t local = t - d.tile_begin;
  const int ntile = int(local % d.nt); local /= d.nt;
  const int mtile = int(local % d.mt); local /= d.mt;
  const int ks = int(local % d.ksplit);
  const int64_t bidx = local / d.ksplit;
  const int64_t m0 = int64_t(mtile) * TC_BM, n0 = int64_t(ntile) * TC_BN;
  const int64_t cps = d.kchunk / bk;                   // chunks per split
  const int64_t kc_begin = int64_t(ks) * cps;
  const int64_t kc_end = min(d.nkc, kc_begin + cps);

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const uint32_t ncols = tc::tmem_cols_for(s * TC_BN);   // levels 2 .. s + 1
  if (warp == 0) {
    tc::tmem_alloc(&tmem_base, ncols);
    tc::tmem_relinquish();
  }
  if (tid == 0) {
    tc::mbar_init(&mbar, 1);
    s_fail = 0;
  }
  const double* Ab = d.A + bidx * d.a_bs;
  const double* Bb = d.B + bidx * d.b_bs;
  for (int i = tid; i < TC_BM + TC_BN; i += TC_THREADS) {
    if (i < TC_BM) Er[i] = -1;
    else Ec[i - TC_BM] = -1;
  }
  __syncthreads();
  if (!d.lx) {
    // exponents from the tags of this launch's exponent pass
    for (int i = tid; i < TC_BM + TC_BN; i += TC_THREADS) {
      if (i < TC_BM) {
        const int64_t r = m0 + i;
        Er[i] = r < d.M ? decode_exp(__ldcg(d.ex_row + bidx * d.M + r), args.epoch) : 0;
      } else {
        const int64_t c = n0 + (i - TC_BM);
        Ec[i - TC_BM] = c < d.N ? decode_exp(__ldcg(d.ex_col + bidx * d.N + c), args.epoch) : 0;
      }
    }
  } else {
    // largest exponent codes (dexp) of the 128 rows of A and the 32 columns of B over all of K
    if (d.a_cs == 1) {                                   // rows contiguous along K: a warp per row
      for (int r = warp; r < TC_BM; r += TC_THREADS / 32) {
        int mx = -1;
        if (m0 + r < d.M)
          for (int64_t k = lane; k < d.K; k += 32) mx = max(mx, dexp(__ldg(Ab + (m0 + r) * d.a_rs + k)));
        mx = __reduce_max_sync(0xffffffffu, mx);
        if (lane == 0) Er[r] = mx;
      }
    } else {                                             // lanes along the rows, warps along K
      int mx[TC_BM / 32];
#pragma unroll
      for (int u = 0; u < TC_BM / 32; ++u) mx[u] = -1;
      for (int64_t k = warp; k < d.K; k += TC_THREADS / 32)
#pragma unroll
        for (int u = 0; u < TC_BM / 32; ++u) {
          const int64_t r = m0 + lane + 32 * u;
          if (r < d.M) mx[u] = max(mx[u], dexp(__ldg(Ab + r * d.a_rs + k * d.a_cs)));
        }
#pragma unroll
      for (int u = 0; u < TC_BM / 32; ++u) atomicMax(&Er[lane + 32 * u], mx[u]);
    }
    if (d.b_rs == 1) {                                   // columns contiguous along K: a warp per column
      for (int c = warp; c < TC_BN; c += TC_THREADS / 32) {
        int mx = -1;
        if (n0 + c < d.N)
          for (int64_t k = lane; k < d.K; k += 32) mx = max(mx, dexp(__ldg(Bb + k + (n0 + c) * d.b_cs)));
        mx = __reduce_max_sync(0xffffffffu, mx);
        if (lane == 0) Ec[c] = mx;
      }
    } else {                                             // lanes along the columns, warps along K
      int mx = -1;
      const int64_t c = n0 + lane;
      if (c < d.N)
        for (int64_t k = warp; k < d.K; k += TC_THREADS / 32)
          mx = max(mx, dexp(__ldg(Bb + k * d.b_rs + c * d.b_cs)));
      atomicMax(&Ec[lane], mx);
    }
    __syncthreads();
    for (int i = tid; i < TC_BM + TC_BN; i += TC_THREADS) {
      int* e = i < TC_BM ? &Er[i] : &Ec[i - TC_BM];
      const int m = *e;
      *e = m < 0 ? 0 : (m == kExNonFinite ? kNonFinite : m - kExBias + 2);
    }
  }
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();

  const uint32_t taddr = tmem_base;

  // epilogue roles: TMEM lane quadrant q (warp % 4), column half ch
  const int q = warp & 3, ch = warp >> 2;
  long long accH[16], accL[16];
#pragma unroll
  for (int j = 0; j < 16; ++j) { accH[j] = 0; accL[j] = 0; }
  uint32_t mph = 0;

  for (int64_t kc = kc_begin; kc < kc_end; ++kc) {
    // ---- the chunk's s planes of A and of B, split by every thread into shared
    //      memory: core matrices of 8 rows x 8 k, a lane holds one row and a k pair
    {
      const int64_t k0 = kc * bk;
      const int kgs = bk / 8;
      const int cmA = (TC_BM / 8) * kgs, cmB = (TC_BN / 8) * kgs;
      const int cr = lane >> 2, ck = (lane & 3) * 2;
      for (int cm = warp; cm < cmA + cmB; cm += TC_THREADS / 32) {
        const bool sa = cm < cmA;
        const int c2 = sa ? cm : cm - cmA;
        const int rg = c2 / kgs, kg = c2 - rg * kgs;
        const int rt = rg * 8 + cr;                       // row of the operand tile
        const int64_t k = k0 + kg * 8 + ck;
        double x0 = 0.0, x1 = 0.0;
        int E;
        if (sa) {
          const int64_t r = m0 + rt;
          if (r < d.M) {
            const double* p = Ab + r * d.a_rs + k * d.a_cs;
            if (k < d.K) x0 = __ldg(p);
            if (k + 1 < d.K) x1 = __ldg(p + d.a_cs);
          }
          E = Er[rt];
        } else {
          const int64_t c = n0 + rt;
          if (c < d.N) {
            const double* p = Bb + k * d.b_rs + c * d.b_cs;
            if (k < d.K) x0 = __ldg(p);
            if (k + 1 < d.K) x1 = __ldg(p + d.b_rs);
          }
          E = Ec[rt];
        }
        int d0[8], d1[8];
        digits(x0, E, s, d0);
        digits(x1, E, s, d1);
        uint8_t* dst = (sa ? As : Bs) + tc::canon_off_w(rt, kg * 8 + ck, bk);
        const uint32_t plane = sa ? pA : pB;
#pragma unroll
        for (int q2 = 0; q2 < 8; ++q2) {
          if (q2 >= s) break;
          *reinterpret_cast<__nv_bfloat162*>(dst + q2 * plane) =
              __floats2bfloat162_rn(int_to_float_small(d0[q2]), int_to_float_small(d1[q2]));
        }
      }
    }
    tc::fence_async_smem();                              // generic stores -> the tensor core's view
    __syncthreads();
    const bool loaded = true;

    // ---- one thread issues every kept digit-pair product of this chunk (only
    //      after its own wait saw the copy complete); every thread then waits
    //      for the issued products before anything else touches TMEM or smem
    if (tid == 0) s_issued = loaded ? 1 : 0;
    if (tid == 0 && loaded) {
      tc::fence_after_sync();
      // B planes are contiguous, i.e. one K-major operand of 32 s rows: the MMA
      // of A digit p against its first 32 (s + 1 - p) rows (digits q <= s + 1
      // - p) adds d_p e_q into columns (p + q - 2) 32, the region of level
      // p + q; products of higher levels are never formed (they would be
      // dropped), so the chains shrink with p and every column written is below
      // 32 s. The p = 1 chain starts all kept levels 2 .. s + 1.
      const uint32_t a0 = tc::smem_u32(As), b0 = tc::smem_u32(Bs);
      const int steps = bk / 16;
      for (int p = 1; p <= s; ++p)
        for (int st = 0; st < steps; ++st)
          tc::mma_bf16(taddr + uint32_t((p - 1) * TC_BN), tc::smem_desc(a0 + (p - 1) * pA + 256 * st, 128, 16 * bk),
                       tc::smem_desc(b0 + 256 * st, 128, 16 * bk),
                       tc::idesc_bf16_f32(TC_BM, TC_BN * (s + 1 - p)), (p == 1 && st == 0) ? 0u : 1u);
      tc::mma_commit(&mbar);
    }
    __syncthreads();
    if (s_issued) {
      if (!tc::mbar_wait_bounded(&mbar, mph, kPolls)) {
        atomicExch(&s_fail, 1);
        tc::mbar_wait_bounded(&mbar, mph, kPolls);    // let the MMAs in flight finish (bounded)
      }
      mph ^= 1;
    }
    tc::fence_after_sync();
    __syncthreads();
    if (s_fail) break;
    // ---- exact level sums -> int64 accumulators (TMEM lane q*32+lane, columns
    //      ch*16..+16); levels are read four at a time, then one wait
    const uint32_t tl = taddr + (uint32_t(q * 32) << 16) + uint32_t(ch * 16);
#pragma unroll
    for (int g = 0; g < 2; ++g) {
      if (2 + 4 * g > s + 1) break;
      uint32_t v[64];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int L = 2 + 4 * g + u;
        if (L <= s + 1) tc::tmem_ld16_nowait(tl + uint32_t((L - 2) * TC_BN), v + 16 * u);
        else {
#pragma unroll
          for (int j = 0; j < 16; ++j) v[16 * u + j] = 0u;
        }
      }
      tc::tmem_wait_ld64(v);
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int L = 2 + 4 * g + u;
        if (L > s + 1) break;
        const int sh = 7 * (3 - u);                 // 7 (5 - L) for H, 7 (9 - L) for Lo
#pragma unroll
        for (int j = 0; j < 16; ++j) {
          const long long iv = (long long)float_to_int_small(__uint_as_float(v[16 * u + j])) << sh;
          if (g == 0) accH[j] += iv; else accL[j] += iv;
        }
      }
    }
    tc::fence_before_sync();
    __syncthreads();
  }

  const int rr = q * 32 + lane;
  const int64_t row = m0 + rr;
  const int64_t c0 = n0 + ch * 16;
  const int64_t row_off = d.c_rdiv > 0 ? (row / d.c_rdiv) * d.c_rs + (row % d.c_rdiv) * d.c_rs2 : row * d.c_rs;
  double* const crow = d.C + bidx * d.c_bs + row_off;
  const bool plain = (d.alpha == 1.0 && d.beta == 0.0);
  auto store = [&](int j, long long H, long long Lo) {
    store_out(crow + (c0 + j) * d.c_cs, H, Lo, Er[rr], Ec[ch * 16 + j], plain, d.alpha, d.beta);
  };
  if (!s_fail) {
    if (d.ksplit == 1) {
      if (row < d.M) {
#pragma unroll
        for (int j = 0; j < 16; ++j)
          if (c0 + j < d.N) store(j, accH[j], accL[j]);
      }
    } else {
      // integer partials meet in L2; the last CTA of the tile rounds and writes C
      const int64_t tile_id = (bidx * d.mt + mtile) * d.nt + ntile;
      unsigned long long* acc = reinterpret_cast<unsigned long long*>(d.acc) + tile_id * (2 * TC_BM * TC_BN);
#pragma unroll
      for (int j = 0; j < 16; ++j) {
        const int cc = ch * 16 + j;
        if (accH[j]) atomicAdd(acc + cc * TC_BM + rr, (unsigned long long)accH[j]);
        if (accL[j]) atomicAdd(acc + TC_BM * TC_BN + cc * TC_BM + rr, (unsigned long long)accL[j]);
      }
      __syncthreads();
      if (tid == 0) {
        const int old = atom_add_acq_rel_gpu(d.cnt + tile_id, 1);
        s_last = (old == d.ksplit - 1);
        if (s_last) d.cnt[tile_id] = 0;
      }
      __syncthreads();
      if (s_last) {
#pragma unroll
        for (int j = 0; j < 16; ++j) {
          const int cc = ch * 16 + j;
          accH[j] = (long long)__ldcg(acc + cc * TC_BM + rr);
          accL[j] = (long long)__ldcg(acc + TC_BM * TC_BN + cc * TC_BM + rr);
        }
#pragma unroll
        for (int j = 0; j < 16; ++j) {
          const int cc = ch * 16 + j;
          acc[cc * TC_BM + rr] = 0;
          acc[TC_BM * TC_BN + cc * TC_BM + rr] = 0;
          if (row < d.M && c0 + j < d.N) store(j, accH[j], accL[j]);
        }
      }
    }
  } else {
    // a wait gave up: raise the flag and leave NaN in this CTA's outputs
    if (tid == 0) atomicOr(err, DEV_TIMEOUT);
    if (row < d.M)
      for (int j = 0; j < 16; ++j)
        if (c0 + j < d.N)
          d.C[bidx * d.c_bs + row_off + (c0 + j) * d.c_cs] = __longlong_as_double(0x7FF8000000000000LL);
  }
  tc::fence_before_sync();
  __syncthreads();
  if (warp == 0) tc::tmem_dealloc(taddr, ncols);
}

}  // namespace

int tc_digits_for_accuracy(double rel) {
  // relative product error ~ 2^{1 - 7 s} times a spread and sqrt(K) factor ~ 2^9
  int s = 1;
  while (s < 8 && std::ldexp(1.0, -7 * s + 10) > rel) ++s;
  return s;
}

static std::atomic<int> g_gemm_mode{0};
int set_gemm_mode(int mode) {
  if (mode < 0 || mode > 2) return TT_EINVAL;
  g_gemm_mode.store(mode);
  return TT_OK;
}

// A group runs fused when its digit planes would exceed this many bytes (so
// that writing and re-reading them goes through HBM) and the fused kernel's
// repeated splitting stays cheap: every product CTA splits its own A rows and B
// columns, so A is split once per tile along N and B once per tile along M.
// Measured: fused wins on the batched sums' GB-sized groups of narrow products
// (repeat factor ~1.25) and loses both on a single sum's 10 MB groups (planes in
// L2) and on the large sum's wide products (repeat factor ~3).
constexpr int64_t kFusedPlaneBytes = int64_t(64) << 20;
constexpr double kFusedMaxRepeat = 2.0;

void gemm_tc_prepare(std::vector<GemmDesc>& g, int s, int target_ctas, TcPlan* plan, long long* acc_base,
                     int* ex_base, int* cbase, uint8_t* plane_base) {
  const int mode = g_gemm_mode.load();
  int64_t t = 0, eb = 0, sb = 0, acc = 0, ex = 0, c = 0, pl = 0;
  int64_t tiles_total = 0;
  double split_once = 0.0, split_fused = 0.0, pl_est = 0.0;
  for (auto& d : g) {
    // keep the long side on the 128-row tile
    if (d.M < TC_BM && d.N > d.M && d.c_rdiv == 0) {
      std::swap(d.M, d.N);
      std::swap(d.A, d.B);
      const int64_t ars = d.a_rs, acs = d.a_cs, abs_ = d.a_bs;
      d.a_rs = d.b_cs; d.a_cs = d.b_rs; d.a_bs = d.b_bs;
      d.b_rs = acs; d.b_cs = ars; d.b_bs = abs_;
      std::swap(d.c_rs, d.c_cs);
    }
    d.mt = int(ceil_div(std::max<int64_t>(d.M, 1), TC_BM));
    d.nt = int(ceil_div(std::max<int64_t>(d.N, 1), TC_BN));
    tiles_total += int64_t(d.batch) * d.mt * d.nt;
    const double K1 = double(std::max<int64_t>(d.K, 1)), bt = double(d.batch);
    split_once += bt * K1 * double(d.M + d.N);
    split_fused += bt * K1 * (double(d.M) * d.nt + double(d.N) * d.mt);
    pl_est += bt * (double(d.mt) * TC_BM + double(d.nt) * TC_BN) * double(ceil_div(int64_t(K1), 16) * 16) * s * 2;
  }
  bool fused = mode == 2;
  if (mode == 0)
    fused = pl_est > double(kFusedPlaneBytes) && split_fused <= kFusedMaxRepeat * split_once;
  plan->fused = fused;
  for (auto& d : g) {
    // chunk width: the K extent rounded up to 16 when it is short, else 64
    const int64_t K1 = std::max<int64_t>(d.K, 1);
    d.bkc = int(K1 >= TC_BK ? TC_BK : ceil_div(K1, 16) * 16);
    d.nkc = ceil_div(K1, d.bkc);
    // split K only while the grid is below one CTA per SM
    const int64_t want = std::max<int64_t>(1, target_ctas / std::max<int64_t>(tiles_total, 1));
    const int64_t split = std::min(d.nkc, want);
    const int64_t cps = ceil_div(d.nkc, split);
    d.kchunk = cps * d.bkc;
    d.ksplit = int(ceil_div(d.nkc, cps));
    const int64_t base = int64_t(d.batch) * d.mt * d.nt;
    d.tile_begin = t;
    t += base * d.ksplit;
    d.exp_begin = eb;
    d.split_begin = sb;
    d.lx = d.K <= kLocalExpK ? 1 : 0;
    d.ex_row = d.ex_col = nullptr;
    d.pa = d.pb = nullptr;
    if (fused) {
      // the product kernel scans its own rows / columns when that is one short
      // pass (no K split, short K); else the exponent pass writes tags it reads
      d.lx = (d.ksplit == 1 && d.K <= kLocalExpK) ? 1 : 0;
      if (!d.lx) {
        const int64_t kb = ceil_div(K1, EX_IN);
        eb += int64_t(d.batch) *
              (ceil_div(std::max<int64_t>(d.M, 1), EX_OUT) + ceil_div(std::max<int64_t>(d.N, 1), EX_OUT)) * kb;
        d.ex_row = ex_base ? ex_base + ex : nullptr;
        ex += int64_t(d.batch) * d.M;
        d.ex_col = ex_base ? ex_base + ex : nullptr;
        ex += int64_t(d.batch) * d.N;
      }
    } else {
      const int64_t kb = ceil_div(K1, EX_IN);
      if (d.K > kLocalExpK)
        eb += int64_t(d.batch) *
              (ceil_div(std::max<int64_t>(d.M, 1), EX_OUT) + ceil_div(std::max<int64_t>(d.N, 1), EX_OUT)) * kb;
      const int R = lx_rows(d.nkc);
      sb += d.lx ? int64_t(d.batch) * (int64_t(d.mt) * (TC_BM / R) + int64_t(d.nt) * (TC_BN / R))
                 : int64_t(d.batch) * (int64_t(d.mt) * 4 + d.nt) * d.nkc;
      d.ex_row = ex_base ? ex_base + ex : nullptr;
      ex += int64_t(d.batch) * d.M;
      d.ex_col = ex_base ? ex_base + ex : nullptr;
      ex += int64_t(d.batch) * d.N;
      const int64_t pa_bytes = int64_t(d.batch) * d.mt * d.nkc * s * (TC_BM * d.bkc * 2);
      const int64_t pb_bytes = int64_t(d.batch) * d.nt * d.nkc * s * (TC_BN * d.bkc * 2);
      d.pa = plane_base ? plane_base + pl : nullptr;
      pl += pa_bytes;
      d.pb = plane_base ? plane_base + pl : nullptr;
      pl += pb_bytes;
    }
    d.P = nullptr;
    d.acc = nullptr;
    d.cnt = nullptr;
    if (d.ksplit > 1) {
      d.acc = acc_base ? acc_base + acc : nullptr;
      acc += base * 2 * TC_BM * TC_BN;
      d.cnt = cbase ? cbase + c : nullptr;
      c += base;
    }
  }
  plan->tiles = t;
  plan->exp_blocks = eb;
  plan->split_blocks = sb;
  plan->acc_words = acc;
  plan->ex_ints = ex;
  plan->counters = c;
  plan->plane_bytes = pl;
}

int gemm_tc_launch(const GemmDesc* d_descs, int ndesc, const TcPlan& plan, int s, int epoch, double flops, int* err,
                   cudaStream_t st) {
  if (ndesc == 0 || plan.tiles == 0) return TT_OK;
  if (s < 1 || s > 8 || epoch < 1 || epoch > 32767) {
    set_error("emulated GEMM: digits must be 1..8 and at most 32767 launches per plan");
    return TT_EINVAL;
  }
  const size_t smem = size_t(s) * (TC_BM + TC_BN) * TC_BK * 2;   // upper bound over chunk widths
  static bool attr = false;
  if (!attr) {
    TTR_CHECK_CUDA(cudaFuncSetAttribute(gemm_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, 164 * 1024));
    TTR_CHECK_CUDA(cudaFuncSetAttribute(gemm_tcf_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, 164 * 1024));
    attr = true;
  }
  TcArgs a{d_descs, ndesc, s, epoch};
  // profiled runs time the whole group (exponent, split and product launches)
  cudaEvent_t e0;
  const bool prof = prof_gemm_begin(st, &e0);
  if (plan.fused) {
    if (plan.exp_blocks > 0) {
      TTR_PREFER_SHARED(tc_exponent_kernel);
      tc_exponent_kernel<<<unsigned(plan.exp_blocks), 256, 0, st>>>(a);
      TTR_CHECK_LAUNCH();
    }
    TTR_PREFER_SHARED(gemm_tcf_kernel);
    gemm_tcf_kernel<<<unsigned(plan.tiles), TC_THREADS, smem, st>>>(a, err);
    TTR_CHECK_LAUNCH();
    prof_count_launch(plan.exp_blocks > 0 ? 2 : 1);
    if (prof) prof_gemm_end(st, flops);
    return TT_OK;
  }
  if (plan.exp_blocks > 0) {
    TTR_PREFER_SHARED(tc_exponent_kernel);
    tc_exponent_kernel<<<unsigned(plan.exp_blocks), 256, 0, st>>>(a);
    TTR_CHECK_LAUNCH();
  }
  TTR_PREFER_SHARED(tc_split_kernel);
  tc_split_kernel<<<unsigned(plan.split_blocks), 256, 0, st>>>(a);
  TTR_CHECK_LAUNCH();
  TTR_PREFER_SHARED(gemm_tc_kernel);
  gemm_tc_kernel<<<unsigned(plan.tiles), TC_THREADS, smem, st>>>(a, err);
  TTR_CHECK_LAUNCH();
  prof_count_launch(plan.exp_blocks > 0 ? 3 : 2);
  if (prof) prof_gemm_end(st, flops);
  return TT_OK;
}

}  // namespace ttr

// ---------------------------------------------------------------------------
using namespace ttr;

extern "C" int tt_gemm_emulated_f64(int64_t M, int64_t N, int64_t K, double alpha, const double* A, int64_t a_rs,
                                    int64_t a_cs, const double* B, int64_t b_rs, int64_t b_cs, double beta,
                                    double* C, int64_t c_rs, int64_t c_cs, int32_t digits, void* workspace,
                                    size_t ws_bytes, void* stream) {
  if (M < 0 || N < 0 || K < 0 || digits < 1 || digits > 8 || (M > 0 && N > 0 && !C) ||
      (M > 0 && N > 0 && K > 0 && (!A || !B)) || K > (int64_t(1) << 20)) {
    set_error("tt_gemm_emulated_f64: need M, N, K >= 0 (K <= 2^20), digits in 1..8 and non-null operands");
    return TT_EINVAL;
  }
  if (M == 0 || N == 0) return TT_OK;
  GemmDesc d = gdesc(A, a_rs, a_cs, B, b_rs, b_cs, C, c_rs, c_cs, M, N, K, alpha, beta);
  BuildFn build = [&](Arena&, Schedule& sc) -> int {
    sc.gemm_tc({d}, digits);
    return TT_OK;
  };
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (workspace == nullptr && ws_bytes != 0) {
    size_t need = 0;
    TTR_TRY(plan_workspace_bytes(build, &need));
    set_error("tt_gemm_emulated_f64: workspace needs " + std::to_string(need) + " bytes");
    return TT_EINVAL;
  }
  int dstat = 0;
  TTR_TRY(plan_execute(build, workspace, ws_bytes, s, &dstat));
  TTR_CHECK_CUDA(cudaStreamSynchronize(s));
  return status_code(dstat, "tt_gemm_emulated_f64");
}

// Declarations of the device kernels' host launchers (internal to the library).
#pragma once
#include "common.cuh"

namespace ttr {

// Arrival on a counter at GPU scope with acquire-release semantics. Called by
// one thread right after a block barrier: the release covers the whole block's
// earlier writes (cumulativity through the barrier) and the acquire makes the
// writes published by the other arrivals visible to the block once it passes
// its next barrier, so no thread needs a separate fence.
__device__ __forceinline__ int atom_add_acq_rel_gpu(int* p, int v) {
  int old;
  asm volatile("atom.add.acq_rel.gpu.global.s32 %0, [%1], %2;" : "=r"(old) : "l"(p), "r"(v) : "memory");
  return old;
}

// ----------------------------------------------------------------------------
// Grouped, batched, strided FP64 GEMM:  C_b = alpha * A_b B_b + beta * C_b for
// every descriptor and batch entry b. Element (r, c) of A_b is at
// A + b*a_bs + r*a_rs + c*a_cs (same for B, C). With ksplit > 1 the K range is
// split over CTAs; partial products go to P ([batch][ksplit][M][N], row-major)
// and the last CTA to finish a tile (arrival counter) sums them in split order
// and writes C, so the result does not depend on scheduling. beta == 0 never
// reads C.
struct GemmDesc {
  const double* A;
  const double* B;
  double* C;
  double* P;
  int64_t M, N, K;
  int64_t a_rs, a_cs, b_rs, b_cs, c_rs, c_cs;
  int64_t a_bs, b_bs, c_bs;
  double alpha, beta;
  int32_t batch, ksplit;
  int32_t mt, nt;
  int64_t kchunk;
  int64_t tile_begin;   // prefix over the group (set by the planner)
  int* cnt;             // split-K arrival counters, one per output tile (self-resetting)
  // emulated-FP64 tensor-core GEMM only (set by gemm_tc_prepare)
  int* ex_row;          // per row of A: tagged largest exponent over K
  int* ex_col;          // per column of B: tagged largest exponent over K
  long long* acc;       // split-K integer accumulators (zero before use, self-resetting)
  int64_t exp_begin;    // prefix of the exponent-pass blocks
  int64_t c_rdiv;       // > 0: row r of C sits at (r / c_rdiv) c_rs + (r % c_rdiv) c_rs2
  int64_t c_rs2;
  uint8_t* pa;          // digit planes of A (tiles x chunks x s planes, canonical layout)
  uint8_t* pb;          // digit planes of B
  int64_t nkc;          // K-chunks
  int64_t split_begin;  // prefix of the split-pass blocks
  int32_t bkc;          // K-chunk width (16, 32, 48 or 64)
  int32_t lx;           // 1: the split pass takes the exponents itself (short K, no exponent pass)
  const int* skip;      // FP64 GEMM only: when set and *skip != 0 on the device, the descriptor does nothing
};

constexpr int GEMM_BM = 32, GEMM_BN = 32, GEMM_BK = 16, GEMM_THREADS = 256;

// Fills tile prefixes, chooses ksplit and carves each split descriptor's
// partial buffer out of pbase and its counters out of cbase; returns the tile
// count and the partial doubles / counters used (bases may be null when only
// sizing).
void gemm_prepare(std::vector<GemmDesc>& g, int64_t* tiles, int64_t* pbuf_doubles, int64_t* counters,
                  int target_ctas, double* pbase, int* cbase);
// flops: algorithmic 2*M*N*K*batch summed over the group (for live profiling).
int gemm_launch(const GemmDesc* d_descs, int ndesc, int64_t tiles, double flops, cudaStream_t s);

// ----------------------------------------------------------------------------
// Emulated FP64 GEMM on the tcgen05 tensor cores (same descriptors; see
// gemm_tc.cu): s = bf16 digits per operand (1..8). One launch group is an
// exponent pass, a digit-split pass (planes in plane_bytes of scratch, no
// initial value needed) and the product pass. The exponent region (ex_ints) must be
// zero before the first group of a plan; each group of the plan gets its own
// epoch 1, 2, ... The accumulator region (acc_words) must be zero before the
// first group and is left zero. *err (device) becomes 1 if a bounded wait gave up.
struct TcPlan {
  int64_t tiles = 0, exp_blocks = 0, split_blocks = 0, acc_words = 0, ex_ints = 0, counters = 0, plane_bytes = 0;
  bool fused = true;   // one launch per group (exponents and digit split inside the product kernel)
};
// 0 (default): per group, fused when its digit planes would exceed 64 MB, else
// three-pass; 1: always the three-pass form (exponent pass, digit planes in
// global memory, products); 2: always fused (exponents -- scanned in the
// product kernel for short unsplit K, else one exponent pass -- and the digit
// split inside the product kernel). Bit-identical results.
int set_gemm_mode(int mode);
int tc_digits_for_accuracy(double rel);
void gemm_tc_prepare(std::vector<GemmDesc>& g, int s, int target_ctas, TcPlan* plan, long long* acc_base,
                     int* ex_base, int* cbase, uint8_t* plane_base);
int gemm_tc_launch(const GemmDesc* d_descs, int ndesc, const TcPlan& plan, int s, int epoch, double flops, int* err,
                   cudaStream_t st);

// ----------------------------------------------------------------------------
// Tall-skinny Householder QR (TSQR) of an m x k matrix A (k <= TSQR_KMAX):
// leaves of b rows are factored in parallel, their R factors are combined up a
// binary tree inside the same launch (the last CTA to finish a pair combines
// it, so no CTA waits), and a second launch forms the explicit thin Q.
constexpr int TSQR_KMAX = 96;   // Householder fallback limit; Cholesky QR has none
constexpr int TT_MAX_RANK = 1024;   // largest target rank / formed rank handled
struct TsqrWork {
  double* leafV;     // P * b * k
  double* leafTau;   // P * k
  double* nodeV;     // inner nodes * 2k * k
  double* nodeTau;   // inner nodes * k
  double* nodeR;     // all nodes * k * k
  int* counters;     // inner nodes, zero before first use (self-resetting)
};
struct TsqrShape {
  int64_t m;
  int k, b, P, L, inner;
};
TsqrShape tsqr_shape(int64_t m, int k);
size_t tsqr_work_doubles(const TsqrShape& sh, size_t* ints);
void tsqr_bind(const TsqrShape& sh, double* dbase, int* ibase, TsqrWork* w);
// Q (m x k, strides q_rs/q_cs) may alias A. R (k x k row-major) may be null.
// With skip_unless set the kernels do nothing unless *skip_unless != 0 (a
// device-side fallback switch).
int tsqr_launch(const TsqrShape& sh, const TsqrWork& w, const double* A, int64_t a_rs, int64_t a_cs,
                double* Q, int64_t q_rs, int64_t q_cs, double* R, cudaStream_t s,
                const int* skip_unless = nullptr);

// ----------------------------------------------------------------------------
// Small dense SVD and truncation rule for one k x k upper-triangular R
// (k <= TSQR_KMAX). Writes G1 (k x k) and G2 (k x k), row-major, such that the
// caller can set  new right factor = Q G1  and  left factor *= G2:
//  - when 1/||R^{-1}||_F > 2 eps (so sigma_min(R) > eps and nothing is cut):
//        G1 = I, G2 = R^T, rank = k;
//  - else one-sided Jacobi SVD R = U S V^T, rank r = smallest r >= 1 with
//        sqrt(sum_{i>r} s_i^2) <= eps, G1 = [U_r 0], G2 = [V_r S_r 0].
// eps is read from device memory (eps_ptr), or taken as 0 when eps_ptr is null
// (fixed rank cap rcap). The rank is written to *rank_out (device).
// k > 96 needs global scratch of svd_scratch_doubles(k) doubles (else may be null).
size_t svd_scratch_doubles(int k);
int svd_trunc_launch(int k, const double* R, const double* eps_ptr, int rcap, double* G1, double* G2,
                     double* sigma, int64_t* rank_out, cudaStream_t s, double* big = nullptr,
                     const int* skip_if = nullptr);
// B independent full SVDs (no truncation) in one launch, one block each: job b
// has k_b = kd[b] (a device array of doubles) <= kmax, R_b, G1_b, G2_b at
// b * kmax * kmax and sigma_b at b * kmax; kmax > 96 needs B * svd_scratch_doubles(kmax)
// doubles of global scratch.
int svd_batch_launch(int B, int kmax, const double* kd, const double* R, double* G1, double* G2, double* sigma,
                     cudaStream_t s, double* big);

// ----------------------------------------------------------------------------
// Elementwise helpers.
struct Copy3 {
  const double* src;
  double* dst;
  int64_t n0, n1, n2;        // extents
  int64_t s0, s1, s2;        // source strides
  int64_t d0, d1, d2;        // destination strides
  double scale;
  int64_t begin;             // prefix of n0*n1*n2 over the batch (set by the planner)
};
int copy3_launch(const Copy3* d_descs, int n, int64_t total, cudaStream_t s);
// Bits of a device status word (Schedule::dev_status).
constexpr int DEV_TIMEOUT = 1;   // a bounded device wait gave up
constexpr int DEV_QR_FAIL = 2;   // a thin QR produced no orthonormal basis
// dst[0] |= bit if src[0] != 0 (device flags)
int or_flag_launch(int* dst, const int* src, int bit, cudaStream_t s);
// dst[0] := 1 (device flag)
int set_flag_launch(int* dst, cudaStream_t s);
int fill_launch(double* p, int64_t n, double v, cudaStream_t s);
// float32 <-> float64 conversion of n entries (device arrays)
int cvt_f32_f64_launch(const float* src, double* dst, int64_t n, cudaStream_t s);
int cvt_f64_f32_launch(const double* src, float* dst, int64_t n, cudaStream_t s);
// dst[0..n) = src[0..n) unless skip_if is set and *skip_if != 0 (device flag)
int copy_if_launch(double* dst, const double* src, int64_t n, const int* skip_if, cudaStream_t s);
// Adjoint helpers: X = T^{-1} (upper triangular, k x k), A := tril(A) + tril(A, -1)^T, y += x.
int triu_inverse_launch(const double* T, double* X, int k, cudaStream_t s);
int sym_lower_launch(double* A, int k, cudaStream_t s);
int axpy_launch(double* y, const double* x, int64_t n, cudaStream_t s);
// A sketch core to draw in a batch: entries E = r0 I r1 of core index core_index
// with the Definition 3.1 scale stdv, seed read from device memory.
struct SketchJob {
  double* out;
  int64_t E;
  int core_index;
  double stdv;
  const uint64_t* seed;
};
SketchJob sketch_job(double* out, int64_t r0, int64_t I, int64_t r1, int core_index, const uint64_t* seed_dev);
// Every job of the device table in one launch (same values as sketch_launch).
int sketch_batch_launch(const SketchJob* d_jobs, int njobs, int64_t max_entries, cudaStream_t s);
// seed_dev (may be null): read the seed from device memory instead (graph replays).
int sketch_launch(double* out, int64_t r0, int64_t I, int64_t r1, int core_index, uint64_t seed,
                  const uint64_t* seed_dev, cudaStream_t s);
// eps = tol * ||x||_F / sqrt(N-1) into *eps_out; x has n doubles.
int norm_eps_launch(const double* x, int64_t n, double tol, int N, double* eps_out, cudaStream_t s);
// Copy core (r0max, I, r1max) from src into dst compactly as (r0, I, r1) with
// r0 = *r0p, r1 = *r1p read on the device.
int compact_core_launch(const double* src, double* dst, int64_t r0max, int64_t I, int64_t r1max,
                        const int64_t* r0p, const int64_t* r1p, cudaStream_t s);

}  // namespace ttr

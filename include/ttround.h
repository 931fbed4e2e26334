/*
 * ttround.h -- C ABI of the GB300 randomized TT-rounding library.
 *
 * Method: Al Daas, Ballard, Cazeaux, Hallman, Miedlar, Pasha, Reid, Saibaba,
 * "Randomized algorithms for rounding in the Tensor-Train format".
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * - A TT-tensor of order N has cores T_n, n = 1..N, with ranks R_0 = R_N = 1
 *   (Section 2.1). Core n is an array of R_{n-1} * I_n * R_n doubles in C
 *   order (R_{n-1}, I_n, R_n): element (a, i, b) is at offset (a*I_n + i)*R_n + b.
 *   With this layout the horizontal unfolding H(T_n) (R_{n-1} x I_n R_n) and a
 *   row-permuted vertical unfolding V(T_n) ((R_{n-1} I_n) x R_n) are plain
 *   row-major views (Section 2.1, Fig. 1).
 * - A sum of K TT-tensors (Section 3.4) is passed as K*N core pointers,
 *   cores[j*N + n-1] = core n of summand j, and ranks[j*(N+1) + n] = R^{(j)}_n.
 * - Pointers named "device" are CUDA device pointers owned by the caller; the
 *   library never frees or keeps them. Pointers named "host" are host memory
 *   read during the call only.
 * - stream is a cudaStream_t passed as void*. All device work is enqueued on it;
 *   inputs are never modified. The eager entry points (tt_round_*,
 *   tt_gemm_emulated_f64) synchronize the stream once at the end: they read
 *   back the run's device status word (and, with a tolerance, the
 *   data-dependent output ranks) and return TT_ETIMEOUT / TT_ESINGULAR when a
 *   kernel reported a failure. Plan replays return after enqueueing unless a
 *   tolerance is given; tt_sum_plan_status / tt_batch_plan_status wait for a
 *   replay and return its device status.
 * - workspace: device scratch of at least the size the matching *_workspace
 *   query returns, 256-byte aligned. NULL lets the library allocate (and free)
 *   it stream-ordered with cudaMallocAsync.
 * - Every function returns a tt_status; on failure tt_last_error() (thread
 *   local) describes it. Nothing is written to outputs on argument errors.
 */
#ifndef TTROUND_H
#define TTROUND_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  TT_OK = 0,
  TT_EINVAL = 1,        /* invalid sizes, ranks, pointers or options */
  TT_ENOMEM = 2,        /* allocation failed or workspace too small */
  TT_ECUDA = 3,         /* a CUDA call failed (message has the CUDA error) */
  TT_ENONFINITE = 4,    /* non-finite values met where the method needs finite ones */
  TT_ESINGULAR = 5,     /* a factorization broke down: a thin QR above the Householder
                           fallback limit could not orthogonalize a block */
  TT_ETIMEOUT = 6,      /* a bounded device wait gave up (the outputs are not valid) */
  TT_EUNSUPPORTED = 7   /* size or option outside what this build handles */
} tt_status;

typedef enum {
  TT_PREC_FP64 = 0,     /* every step in float64 */
  TT_PREC_MIXED = 1,    /* contractions on the tensor cores (see tt_round_sum_rand) */
  TT_PREC_MIXED_FULL = 2 /* as TT_PREC_MIXED, the Algorithm 3 contractions with full digits too:
                            for sums far smaller than their summands (cancelling combinations) */
} tt_precision;

/* Library version string and the last error message of the calling thread. */
const char* tt_version(void);
const char* tt_last_error(void);

/*
 * tt_sketch_gaussian -- random Gaussian TT of Definition 3.1 (Section 3.2):
 * core n (ells[n-1] x dims[n-1] x ells[n]) gets i.i.d. N(0, 1/(l_{n-1} I_n l_n))
 * entries drawn with the counter-based generator Philox4x32-10 (Salmon et al.,
 * SC'11) and the Box-Muller transform: entry e of core n uses counter
 * (e/2 mod 2^32, e/2 div 2^32, n-1, 0x7474726e) and key (seed mod 2^32,
 * seed div 2^32); u = (52 bits of the output + 1/2) 2^-52; even entries take
 * the cosine, odd entries the sine branch.
 *   N     order;  dims (host, N);  ells (host, N+1, ells[0] = ells[N] = 1)
 *   out   (host array of N device pointers), core n needs ells[n-1]*dims[n-1]*ells[n] doubles
 * Errors: TT_EINVAL for N < 1, non-positive sizes, NULL pointers.
 */
int tt_sketch_gaussian(int32_t N, const int64_t* dims, const int64_t* ells, uint64_t seed,
                       double* const* out, void* stream);

/*
 * tt_round_sum_rand -- Algorithm 7 (TT-Rounding of a Sum,
 * Randomize-then-Orthogonalize, Section 3.4), with Algorithm 3 (right-to-left
 * partial contractions, Section 2.3) for every summand against one shared
 * Gaussian TT sketch (Definition 3.1), then the left-to-right sweep: sketch
 * Y_n = V(X_n)[W^{(1)}_n; ...; W^{(K)}_n], thin QR, projection
 * [M^{(1)}_n ... M^{(K)}_n] = V(X_n)^T Z_n, next-core update slice by slice and
 * X_N = sum_j M^{(j)}_{N-1} Y^{(j)}_N. The block cores of the sum are never
 * formed. With tol > 0 the left-orthogonal result is truncated as in
 * Section 3.2 (Algorithm 2's truncation loop run right to left):
 * eps = tol ||X|| / sqrt(N-1), so that ||X_out - X|| <= tol ||X|| where X is
 * the untruncated randomized result.
 *   N, K          order and number of summands (K >= 1)
 *   dims          host, N mode sizes
 *   ranks         host, K*(N+1) summand ranks (ranks[j*(N+1)] = ranks[j*(N+1)+N] = 1)
 *   cores         host array of K*N device pointers (see conventions)
 *   coeffs        host, K scalars multiplying the summands, or NULL for all ones
 *   ells          host, N+1 target sketch ranks l_n (oversampling included,
 *                 Section 3); clamped to l_n <= min(l_{n-1} I_n, I_{n+1} l_{n+1})
 *   sketch        host array of N device pointers to the sketch cores
 *                 (l_{n-1} x I_n x l_n, clamped ranks), or NULL to draw them on
 *                 the device from seed exactly as tt_sketch_gaussian does
 *   tol           <= 0: fixed ranks l_n; > 0: relative truncation tolerance
 *   precision     TT_PREC_FP64 or TT_PREC_MIXED
 *   out           host array of N device pointers; core n needs
 *                 l_{n-1}*I_n*l_n doubles (clamped ranks); the result is written
 *                 compactly as (r_{n-1}, I_n, r_n)
 *   out_ranks     host, N+1, receives r_0..r_N
 * Errors: TT_EINVAL (bad sizes/ranks/pointers), TT_EUNSUPPORTED (a target rank
 * above 1024), TT_ENOMEM, TT_ECUDA, TT_ETIMEOUT (a tensor-core wait gave up),
 * TT_ESINGULAR (a thin QR of rank above 96 could not orthogonalize a block).
 */
int tt_round_sum_rand(int32_t N, int32_t K, const int64_t* dims, const int64_t* ranks,
                      const double* const* cores, const double* coeffs, const int64_t* ells,
                      const double* const* sketch, uint64_t seed, double tol, int32_t precision,
                      double* const* out, int64_t* out_ranks, void* workspace, size_t workspace_bytes,
                      void* stream);
/*
 * TT_PREC_MIXED (no counterpart in the paper, which computes in FP64): every
 * contraction runs on the tcgen05 tensor cores as the emulated float64 product
 * of tt_gemm_emulated_f64 (bf16 digits of 7 bits relative to the largest
 * exponent of each row / column, exact digit products and sums, one rounding):
 *   - the partial contractions of Algorithm 3 with 2 digits (their rounding
 *     only perturbs the sketch: each sketched core stays in the range of its
 *     unfolding, so the subspaces and the rounding error are unaffected);
 *   - the core updates X_n = M_{n-1} Y_n, the sketches V(X_n) W_n and the
 *     projections Q^T V(X_n) with s = tt_mixed_digits(tol, N) digits: products
 *     accurate to 1e-3 tol / N (1e-7 / N in fixed-rank mode), 1 <= s <= 8, so
 *     s = 8 (FP64 class) at tol = 1e-8.
 * QR, the small SVD and the truncation stay float64.
 * The 2-digit Algorithm 3 contractions assume that the sum does not cancel:
 * their error is relative to the summands, so for a combination far smaller
 * than its terms (a Gram-Schmidt step, an iterative solver's updates) the
 * sketch of the result drowns; TT_PREC_MIXED_FULL gives those contractions
 * the s digits of the others.
 */
int tt_mixed_digits(double tol, int32_t N);
size_t tt_round_sum_rand_workspace(int32_t N, int32_t K, const int64_t* dims, const int64_t* ranks,
                                   const int64_t* ells, double tol, int32_t precision);

/*
 * tt_round_rand_backward -- reverse-mode derivative of fixed-sketch
 * Randomize-then-Orthogonalize (Algorithm 5 with the sketch Omega held fixed,
 * fixed target ranks, no tolerance truncation). The paper gives no derivative;
 * this is the chain rule through Algorithm 5 (thin-QR backward with the R
 * factor not differentiated) and Algorithm 3, in FP64. Given the forward input
 * Y (N, dims, ranks, cores as in tt_round_rand), the clamped target ranks of
 * ells (N+1), the sketch (N device cores (l_{n-1}, I_n, l_n); core 1 unused)
 * and xbar = dL/dX_hat for the output cores X_hat of tt_round_rand with that
 * sketch (N device cores (l_{n-1}, I_n, l_n)), writes ybar = dL/dY (N device
 * cores shaped like Y, overwritten). The forward quantities are recomputed
 * (the partial contractions W_n included), not kept from the forward call.
 * workspace: as tt_round_rand, sized by tt_round_rand_backward_workspace.
 * Errors: TT_EINVAL, TT_EUNSUPPORTED (a rank above 1024), TT_ENOMEM, TT_ECUDA.
 */
int tt_round_rand_backward(int32_t N, const int64_t* dims, const int64_t* ranks, const double* const* cores,
                           const int64_t* ells, const double* const* sketch, const double* const* xbar,
                           double* const* ybar, void* workspace, size_t workspace_bytes, void* stream);
size_t tt_round_rand_backward_workspace(int32_t N, const int64_t* dims, const int64_t* ranks, const int64_t* ells);

/*
 * Captured plans of tt_round_sum_rand (an execution mechanism, no counterpart
 * in the paper). tt_sum_plan_create fixes N, K, dims, ranks (K x (N+1)), the
 * sketch ranks ells (N+1), tol and precision, builds the whole schedule of the
 * rounding once and captures it into a CUDA graph; the plan owns its device
 * memory (input copies, outputs at the clamped sketch ranks, workspace).
 * tt_sum_plan_run replays it on the given stream for any summand cores
 * (cores: K*N device pointers, summand-major, shapes as in tt_round_sum_rand),
 * coefficients (host, K values, NULL = ones) and sketch seed (the sketch is
 * always drawn on the device): one pinned host-to-device copy of these
 * arguments and one graph launch. The graph copies the cores in, runs every
 * step of tt_round_sum_rand in the same order -- results are bit-wise those of
 * tt_round_sum_rand with sketch NULL and the same seed -- and writes the
 * rounded cores to out (N device pointers, capacities as in
 * tt_round_sum_rand, written compactly). out_ranks (host, N+1) receives the
 * ranks; with tol > 0 the call waits for the stream to read them, otherwise it
 * returns at once. Runs of one plan are ordered by their streams; one plan
 * must not run on two streams at the same time. tt_sum_plan_launches returns
 * the kernels one replay launches; tt_sum_plan_destroy synchronizes the device
 * and frees the plan (NULL is allowed).
 * Errors: as tt_round_sum_rand; TT_ECUDA if the capture fails.
 */
typedef struct tt_sum_plan tt_sum_plan;
int tt_sum_plan_create(int32_t N, int32_t K, const int64_t* dims, const int64_t* ranks, const int64_t* ells,
                       double tol, int32_t precision, tt_sum_plan** plan, void* stream);
int tt_sum_plan_run(tt_sum_plan* plan, const double* const* cores, const double* coeffs, uint64_t seed,
                    double* const* out, int64_t* out_ranks, void* stream);
int tt_sum_plan_destroy(tt_sum_plan* plan);
int64_t tt_sum_plan_launches(const tt_sum_plan* plan);
/* Waits for stream and returns the device status of the plan's last replay
 * (TT_OK, TT_ETIMEOUT or TT_ESINGULAR, as the eager entry point would). */
int tt_sum_plan_status(tt_sum_plan* plan, void* stream);

/*
 * Host-buffer replays of a plan (same computation as tt_sum_plan_run). Packed
 * host layout: the input is one array of all summand cores, summand-major
 * then core-major, core (j, n) row-major (r_{n-1}, I_n, r_n) at element offset
 * in_offsets[j*N + n-1]; the output is one array of N slots, slot n at
 * out_offsets[n-1] with room for the clamped sketch-rank core, the rounded
 * core written compactly at the slot's start (shape out_ranks[n-1], I_n,
 * out_ranks[n]). tt_sum_plan_host_layout fills any of its non-NULL
 * arguments: in_offsets (K*N), out_offsets (N), in_total and out_total
 * (elements). tt_sum_plan_run_host copies h_in (in_total doubles, host) to a
 * plan-owned device buffer with one copy, replays the plan and copies the
 * out_total doubles of slots back to h_out (host) with one copy, then waits
 * for the stream: on return h_out and out_ranks hold the result. Pinned host
 * memory gives asynchronous full-speed copies; pageable memory works but is
 * staged by the CUDA runtime. The first call allocates the device landing
 * buffers (TT_ENOMEM if that fails).
 * Errors: TT_EINVAL for a NULL plan, h_in, h_out or out_ranks; as
 * tt_sum_plan_run otherwise.
 */
int tt_sum_plan_host_layout(const tt_sum_plan* plan, int64_t* in_offsets, int64_t* out_offsets, int64_t* in_total,
                            int64_t* out_total);
int tt_sum_plan_run_host(tt_sum_plan* plan, const double* h_in, const double* coeffs, uint64_t seed, double* h_out,
                         int64_t* out_ranks, void* stream);

/*
 * Batched plans: B independent sum roundings (the uneven sums of TT-GMRES,
 * Section 4.2) in one CUDA graph. Problem b is given by its N, K, dims, ranks
 * K x (N+1), ells N+1 and tol, as for tt_sum_plan_create; how the problems are
 * scheduled (grouped launches over many problems, or one schedule per problem
 * on parallel chains) is described at tt_batch_plan_create_sched.
 * tt_batch_plan_create(..., width, ...) takes the default schedule for width.
 * tt_batch_plan_run: cores = the problems' core pointer arrays concatenated
 * (problem b: K_b*N_b device pointers as in tt_sum_plan_run), seeds = B sketch
 * seeds (host; NULL = 0, 1, ..., B-1), out = the problems' N_b output pointers
 * concatenated, out_ranks = the problems' N_b+1 ranks concatenated (host).
 * The call waits for the stream only if some problem has tol > 0.
 */
typedef struct {
  int32_t N, K;
  const int64_t* dims;     /* N */
  const int64_t* ranks;    /* K*(N+1), summand-major */
  const int64_t* ells;     /* N+1 */
  double tol;              /* <= 0: fixed ranks */
} tt_sum_problem;
typedef struct tt_batch_plan tt_batch_plan;
int tt_batch_plan_create(int32_t B, const tt_sum_problem* probs, int32_t precision, int32_t width,
                         tt_batch_plan** plan, void* stream);
/*
 * Schedule of a batched plan (tt_batch_plan_create uses {width, 8, -1}):
 *   fused = 1 (or -1 with every problem at fixed ranks, tol <= 0, and target
 *   ranks <= 96): the problems are split into `width` groups of consecutive
 *   problems; each group runs as ONE chain of grouped launches -- every launch
 *   covers all problems of its group (the Algorithm 3 products of every
 *   summand of every problem, all sketch cores, every core update, sketch and
 *   projection, and each bond's thin QRs as one batched Cholesky-QR chain of
 *   6 launches with about qr_ctas CTAs per QR) -- so a group takes a few
 *   hundred launches whatever its size; the groups' chains run concurrently.
 *   Results equal tt_round_sum_rand's with the same seed to rounding (the
 *   grouped products and the batched QR sum in another order); a batched QR
 *   that breaks down is reported as TT_ESINGULAR (no Householder fallback).
 *   fused = 0 (or -1 otherwise): one schedule per problem, problem b on chain
 *   b mod width, results bit-wise those of tt_round_sum_rand.
 * width and qr_ctas change no mathematics (the autotuner of the Python
 * binding tries several).
 */
typedef struct {
  int32_t width;
  int32_t qr_ctas;
  int32_t fused;
} tt_batch_schedule;
int tt_batch_plan_create_sched(int32_t B, const tt_sum_problem* probs, int32_t precision,
                               const tt_batch_schedule* sched, tt_batch_plan** plan, void* stream);
int tt_batch_plan_is_fused(const tt_batch_plan* plan);
int tt_batch_plan_run(tt_batch_plan* plan, const double* const* cores, const uint64_t* seeds, double* const* out,
                      int64_t* out_ranks, void* stream);
int tt_batch_plan_destroy(tt_batch_plan* plan);
int64_t tt_batch_plan_launches(const tt_batch_plan* plan);
/* Waits for stream and returns the combined device status of the last replay. */
int tt_batch_plan_status(tt_batch_plan* plan, void* stream);

/*
 * tt_round_rand -- Algorithm 5 (Randomize-then-Orthogonalize, Section 3.2):
 * the single-tensor case K = 1 of tt_round_sum_rand, same arguments with
 * ranks of length N+1 and N core pointers.
 */
int tt_round_rand(int32_t N, const int64_t* dims, const int64_t* ranks, const double* const* cores,
                  const int64_t* ells, const double* const* sketch, uint64_t seed, double tol,
                  int32_t precision, double* const* out, int64_t* out_ranks, void* workspace,
                  size_t workspace_bytes, void* stream);

/*
 * float32 storage (no counterpart in the paper, which works in FP64): the same
 * calls for float32 cores, sketch, outputs and cotangents.
 * tt_round_rand_f32 converts the cores (and the sketch, when given) to float64
 * on the device, runs tt_round_rand with `precision` (TT_PREC_MIXED: the
 * tensor-core contractions with tt_mixed_digits(tol, N) digits, FP32 class and
 * better) and converts the output cores back to float32 (out[n] holds
 * l_{n-1} I_n l_n floats).
 * tt_round_rand_backward_f32 does the same around tt_round_rand_backward, with
 * every product of the adjoint as the emulated tensor-core GEMM with
 * tt_mixed_digits(0, N) digits (FP32 class); the thin QRs, the triangular
 * inverses and the QR-backward steps stay FP64.
 * Arguments, workspace queries and errors as the float64 versions.
 */
int tt_round_rand_f32(int32_t N, const int64_t* dims, const int64_t* ranks, const float* const* cores,
                      const int64_t* ells, const float* const* sketch, uint64_t seed, double tol, int32_t precision,
                      float* const* out, int64_t* out_ranks, void* workspace, size_t workspace_bytes, void* stream);
size_t tt_round_rand_f32_workspace(int32_t N, const int64_t* dims, const int64_t* ranks, const int64_t* ells,
                                   double tol, int32_t precision);
int tt_round_rand_backward_f32(int32_t N, const int64_t* dims, const int64_t* ranks, const float* const* cores,
                               const int64_t* ells, const float* const* sketch, const float* const* xbar,
                               float* const* ybar, void* workspace, size_t workspace_bytes, void* stream);
size_t tt_round_rand_backward_f32_workspace(int32_t N, const int64_t* dims, const int64_t* ranks,
                                            const int64_t* ells);

/*
 * tt_round_det -- deterministic TT-rounding of a sum: the formed TT-sum of
 * Section 2.1 (coefficients in the first cores), Algorithm 1 (right-to-left
 * orthogonalization) and Algorithm 2 (TT-SVD truncation, eps = tol ||Y|| /
 * sqrt(N-1), so ||X - Y|| <= tol ||Y||), the comparison path of the paper.
 * With max_rank > 0 every bond is also capped at max_rank (tol <= 0: fixed
 * ranks only). Arguments as tt_round_sum_rand, and:
 *   out   host array of N device pointers; core n must hold the formed core,
 *         tt_round_det_out_capacity(...)[n-1] doubles (S_{n-1} I_n S_n with
 *         S_n = sum_j R^{(j)}_n): it is used as working storage and receives the
 *         result compactly as (r_{n-1}, I_n, r_n).
 * The output ranks are decided on the device and read back (one stream sync).
 * Errors: TT_EINVAL, TT_ENOMEM, TT_ECUDA, TT_EUNSUPPORTED (an unfolding that
 * would have to be wide), TT_ESINGULAR (a Cholesky QR above the Householder
 * limit could not orthogonalize a block).
 */
int tt_round_det(int32_t N, int32_t K, const int64_t* dims, const int64_t* ranks, const double* const* cores,
                 const double* coeffs, double tol, int64_t max_rank, double* const* out, int64_t* out_ranks,
                 void* workspace, size_t workspace_bytes, void* stream);
size_t tt_round_det_workspace(int32_t N, int32_t K, const int64_t* dims, const int64_t* ranks, double tol,
                              int64_t max_rank);
int tt_round_det_out_capacity(int32_t N, int32_t K, const int64_t* dims, const int64_t* ranks, int64_t* caps);

/*
 * tt_round_orthrand -- Algorithm 4 (Orthogonalize-then-Randomize, Section 3.1)
 * on the formed TT-sum: Algorithm 1, then for n = 1..N-1 sketch
 * Y_n = V(X_n) Omega_n with a Gaussian R'_n x l_n matrix, thin QR,
 * M_n = Q^T V(X_n), H(X_{n+1}) := M_n H(X_{n+1}).
 *   omega  host array of N device pointers, omega[n-1] = Omega_n (R'_n x l_n,
 *          row-major; omega[N-1] unused), R'_n from tt_orthrand_omega_ranks;
 *          or NULL to draw them on the device from seed (Philox, as
 *          tt_sketch_gaussian does for a 1 x R'_n x l_n core with index n-1)
 *   out    host array of N device pointers, core n holds l_{n-1} I_n l_n doubles
 *          (clamped target ranks, returned in out_ranks).
 * Errors: TT_EINVAL, TT_ENOMEM, TT_ECUDA.
 */
int tt_round_orthrand(int32_t N, int32_t K, const int64_t* dims, const int64_t* ranks, const double* const* cores,
                      const double* coeffs, const int64_t* ells, const double* const* omega, uint64_t seed,
                      double* const* out, int64_t* out_ranks, void* workspace, size_t workspace_bytes,
                      void* stream);
size_t tt_round_orthrand_workspace(int32_t N, int32_t K, const int64_t* dims, const int64_t* ranks,
                                   const int64_t* ells);
/* R'_0..R'_N: ranks of the formed sum after Algorithm 1 (the row counts of Omega_n). */
int tt_orthrand_omega_ranks(int32_t N, int32_t K, const int64_t* dims, const int64_t* ranks, int64_t* rp);

/*
 * tt_round_twosided -- Algorithm 6 (Two-Sided-Randomization, generalized
 * Nystrom, Section 3.3) for a sum of K TT-tensors without forming the block
 * cores: left-to-right contractions with a Gaussian TT L of ranks l_n,
 * right-to-left contractions (Algorithm 3) with a Gaussian TT R of ranks
 * rho_n > l_n, per bond the SVD of W^L_n W^R_n and the factors
 * L_n = W^R_n V S^{+1/2}, R_n = S^{+1/2} U^T W^L_n, then
 * X_n = R_{n-1} x_1 Y_n x_3 L_n summed over the summands.
 *   rhos         host, N+1 right sketch ranks, or NULL for ceil(1.5 l_n)
 *                (Section 4.1); clamped like ells; must stay >= l_n
 *   sketch_left  host array of N device pointers (l_{n-1} x I_n x l_n) or NULL
 *   sketch_right host array of N device pointers (rho_{n-1} x I_n x rho_n) or NULL
 *                (NULL: drawn on the device as tt_sketch_gaussian does, the left
 *                one from seed and the right one from seed + 1)
 *   precision    TT_PREC_FP64, or TT_PREC_MIXED: every contraction (both
 *                sketch sweeps included, since W^L and W^R span the projectors'
 *                ranges themselves) as the emulated float64 product of
 *                tt_gemm_emulated_f64 with tt_mixed_digits(0, N) digits; the
 *                QR, the SVD and the factor scaling stay float64
 *   out          host array of N device pointers, core n holds l_{n-1} I_n l_n
 * The result is not orthogonal (Section 3.3). Errors: TT_EINVAL (also for an
 * unknown precision), TT_ENOMEM, TT_ECUDA.
 */
int tt_round_twosided(int32_t N, int32_t K, const int64_t* dims, const int64_t* ranks, const double* const* cores,
                      const double* coeffs, const int64_t* ells, const int64_t* rhos,
                      const double* const* sketch_left, const double* const* sketch_right, uint64_t seed,
                      int32_t precision, double* const* out, int64_t* out_ranks, void* workspace,
                      size_t workspace_bytes, void* stream);
size_t tt_round_twosided_workspace(int32_t N, int32_t K, const int64_t* dims, const int64_t* ranks,
                                   const int64_t* ells, const int64_t* rhos, int32_t precision);

/*
 * tt_round_twosided_orth -- Algorithm 6 with the orthogonalizing restructure
 * that Section 3.3 mentions without giving it, and the tolerance mode it
 * enables. The sketches, bond SVDs and factors L_n, R_n are those of
 * tt_round_twosided; the cores are then formed in a left-to-right sweep that
 * carries the R factor of each thin QR into the next core (T_0 = 1):
 *   C_n = (T_{n-1} R_{n-1}) x_1 Y_n x_3 L_n,  V(C_n) = Q_n T_n,  X_n = Q_n (n < N),
 *   H(X_N) = T_{N-1} R_{N-1} H(Y_N),
 * which represents the same tensor as Algorithm 6 but left-orthogonal. With
 * tol > 0 the result is then truncated as in tt_round_sum_rand (Section 3.2,
 * eps = tol ||X|| / sqrt(N-1)), so ||X_out - X|| <= tol ||X||, X the
 * Algorithm 6 result. Arguments as tt_round_twosided plus tol; with
 * TT_PREC_MIXED the contractions take tt_mixed_digits(tol, N) digits. out
 * cores are written compactly at out_ranks. Errors: as tt_round_twosided.
 */
int tt_round_twosided_orth(int32_t N, int32_t K, const int64_t* dims, const int64_t* ranks,
                           const double* const* cores, const double* coeffs, const int64_t* ells,
                           const int64_t* rhos, const double* const* sketch_left,
                           const double* const* sketch_right, uint64_t seed, double tol, int32_t precision,
                           double* const* out, int64_t* out_ranks, void* workspace, size_t workspace_bytes,
                           void* stream);
size_t tt_round_twosided_orth_workspace(int32_t N, int32_t K, const int64_t* dims, const int64_t* ranks,
                                        const int64_t* ells, const int64_t* rhos, double tol, int32_t precision);

/*
 * tt_truncate_lorth -- the truncation of Section 3.2 for a left-orthogonal TT
 * (V(X_n)^T V(X_n) = I for n < N, as Algorithms 5 and 7 produce it), without
 * re-orthogonalizing: Algorithm 2's truncation loop run right to left, per
 * bond the thin QR of H(X_n)^T, the SVD of R with the eps rule
 * (eps = tol ||X|| / sqrt(N-1), ||X|| = ||X_N||_F) and at most max_rank
 * singular values kept, then H(X_n) := (Q U)^T and V(X_{n-1}) := V(X_{n-1}) V S.
 * ||X_out - X|| <= tol ||X|| when only the tolerance cuts.
 *   N, dims, ranks  the TT (host; ranks N+1 with r_0 = r_N = 1 and
 *                   r_{n-1} <= I_n r_n, r_n <= r_{n-1} I_n)
 *   cores           host array of N device pointers, core n compact
 *                   (r_{n-1}, I_n, r_n): overwritten with the result, written
 *                   compactly at out_ranks
 *   tol, max_rank   tol <= 0: no tolerance; max_rank <= 0: no cap (one of the
 *                   two must be set)
 * Errors: TT_EINVAL, TT_EUNSUPPORTED (a rank above 1024), TT_ENOMEM, TT_ECUDA.
 */
int tt_truncate_lorth(int32_t N, const int64_t* dims, const int64_t* ranks, double* const* cores, double tol,
                      int64_t max_rank, int64_t* out_ranks, void* workspace, size_t workspace_bytes, void* stream);
size_t tt_truncate_lorth_workspace(int32_t N, const int64_t* dims, const int64_t* ranks, double tol,
                                   int64_t max_rank);

/*
 * tt_inner -- inner products <X, Y^(j)> of one TT X with K TTs Y^(j) of the
 * same mode sizes (Section 2.3): Algorithm 3 (right-to-left partial
 * contractions) of every Y^(j) against X, run down to the first core, where
 * the partial contraction W_0 is the 1 x 1 inner product. All K sweeps share
 * the cores of X: one grouped product per core for the Y^(j) and one for X.
 *   X: N, dims (host, N), ranks_x (host, N+1), cores_x (host array of N device pointers)
 *   Y: K, ranks_y (host, K*(N+1)), cores_y (host array of K*N device pointers), as tt_round_sum_rand
 *   out: device array of K doubles, out[j] = <X, Y^(j)>
 * tt_norm: ||X|| = sqrt(<X, X>) by the same sweep, into out (device, 1 double).
 * Both synchronize the stream at the end (device status). Errors: TT_EINVAL,
 * TT_ENOMEM, TT_ECUDA.
 */
int tt_inner(int32_t N, const int64_t* dims, const int64_t* ranks_x, const double* const* cores_x, int32_t K,
             const int64_t* ranks_y, const double* const* cores_y, double* out, void* workspace,
             size_t workspace_bytes, void* stream);
size_t tt_inner_workspace(int32_t N, const int64_t* dims, const int64_t* ranks_x, int32_t K,
                          const int64_t* ranks_y);
int tt_norm(int32_t N, const int64_t* dims, const int64_t* ranks, const double* const* cores, double* out,
            void* workspace, size_t workspace_bytes, void* stream);
size_t tt_norm_workspace(int32_t N, const int64_t* dims, const int64_t* ranks);

/*
 * tt_mode_products -- count mode products of TT cores with matrices in one
 * grouped launch (the factors of a Kronecker-product operator applied core by
 * core, Section 4.2): for q < count, with shapes[4q..4q+3] = (r0, I, r1, J),
 *   out_q(a, j, b) = sum_i A_q(j, i) core_q(a, i, b),
 * A_q a J x I row-major device matrix, core_q (r0, I, r1) and out_q (r0, J, r1)
 * device arrays in C order (out_q must not overlap core_q or A_q).
 * Errors: TT_EINVAL, TT_ENOMEM, TT_ECUDA.
 */
int tt_mode_products(int32_t count, const int64_t* shapes, const double* const* A, const double* const* cores,
                     double* const* out, void* workspace, size_t workspace_bytes, void* stream);
size_t tt_mode_products_workspace(int32_t count, const int64_t* shapes);

/*
 * tt_round_gram_schmidt -- one Gram-Schmidt step of TT-GMRES (Section 4.2)
 * as a single call: with W (one TT) and the basis V_1..V_k,
 *   h_j = <V_j, W> (j = 1..k, tt_inner's sweep),
 *   Z = W - sum_j h_j V_j rounded by Algorithm 7 (coefficients 1, -h_1, ..,
 *       -h_k taken from the device, sketch ranks ells, tolerance tol as in
 *       tt_round_sum_rand, sketch from `sketch` or drawn from seed),
 *   h_{k+1} = ||Z|| and V_{k+1} = Z / h_{k+1} (Z left as is when ||Z|| = 0).
 *   W: N, dims, ranks_w (N+1), cores_w (N device pointers)
 *   basis: k >= 0, ranks_v (k*(N+1)), cores_v (k*N device pointers)
 *   out, out_ranks: as tt_round_sum_rand (V_{k+1} written compactly)
 *   h: host, k+1 doubles: h_1..h_k then ||Z||
 * One host synchronization at the end. Errors: as tt_round_sum_rand.
 */
int tt_round_gram_schmidt(int32_t N, const int64_t* dims, const int64_t* ranks_w, const double* const* cores_w,
                          int32_t k, const int64_t* ranks_v, const double* const* cores_v, const int64_t* ells,
                          const double* const* sketch, uint64_t seed, double tol, int32_t precision,
                          double* const* out, int64_t* out_ranks, double* h, void* workspace,
                          size_t workspace_bytes, void* stream);
size_t tt_round_gram_schmidt_workspace(int32_t N, const int64_t* dims, const int64_t* ranks_w, int32_t k,
                                       const int64_t* ranks_v, const int64_t* ells, double tol, int32_t precision);

/*
 * tt_round_sum_rand_sharded -- Algorithm 7 with the summands sharded over
 * ranks (no counterpart in the paper; its block form makes it direct): every
 * rank passes its own summands (K, ranks, cores, coeffs of its share) with the
 * same dims, ells, sketch / seed, tol and precision. The right-to-left
 * partial contractions are per summand and stay local; in the left-to-right
 * sweep the partial sketch V(X_n) [W^{(j)}_n]_j of the rank's summands
 * (l_{n-1} I_n l_n doubles, device) and finally the partial last core are
 * summed over the ranks by `allreduce`, after which every rank repeats the same
 * thin QR and truncation on identical data and the local projections
 * M^{(j)}_n. Every rank ends with the whole rounded tensor in out.
 *   allreduce(buf, count, stream, ctx): must replace buf (device, count
 *   doubles) by its sum over the ranks, stream-ordered on `stream` (e.g. an
 *   NCCL all-reduce enqueued on it), with the same summation order on every
 *   rank; nonzero return = failure (TT_ECUDA). It is called from the calling
 *   thread while the library enqueues its work.
 * Other arguments and errors as tt_round_sum_rand.
 */
typedef int (*tt_allreduce_fn)(double* buf, size_t count, void* stream, void* ctx);
int tt_round_sum_rand_sharded(int32_t N, int32_t K, const int64_t* dims, const int64_t* ranks,
                              const double* const* cores, const double* coeffs, const int64_t* ells,
                              const double* const* sketch, uint64_t seed, double tol, int32_t precision,
                              double* const* out, int64_t* out_ranks, void* workspace, size_t workspace_bytes,
                              void* stream, tt_allreduce_fn allreduce, void* ctx);

/*
 * tt_round_sum_rand_noalloc -- tt_round_sum_rand for callers that cannot
 * allocate device memory (no counterpart in the paper: it only changes where the
 * scratch lives). Some callers may not call cudaMalloc at the point of the
 * rounding: real-time loops with a fixed memory budget, plug-ins whose host
 * application hands the library only its inputs and outputs, processes whose
 * device memory is already claimed by another allocator. This entry point takes the
 * same arguments as tt_round_sum_rand minus the workspace and uses a fixed
 * device array of TT_NOALLOC_SCRATCH_BYTES inside the library instead; every
 * GPU that loads the library holds that array until the process exits. It
 * calls no cudaMalloc, cudaFree or other allocating routine.
 *   - Problems whose scratch need (tt_round_sum_rand_workspace) exceeds
 *     TT_NOALLOC_SCRATCH_BYTES return TT_ENOMEM with both sizes in the message.
 *   - All calls on a device share the array and leave their contents behind;
 *     each call zeroes what must start at zero. Calls whose device work
 *     overlaps (several streams or host threads) race: serialize them.
 *   - The first call on a device looks up the array's device address with that
 *     device current; make it before any stream capture.
 * tt_noalloc_scratch_bytes() returns the array size.
 */
#define TT_NOALLOC_SCRATCH_BYTES (16u * 1024u * 1024u)
size_t tt_noalloc_scratch_bytes(void);
int tt_round_sum_rand_noalloc(int32_t N, int32_t K, const int64_t* dims, const int64_t* ranks,
                              const double* const* cores, const double* coeffs, const int64_t* ells,
                              const double* const* sketch, uint64_t seed, double tol, int32_t precision,
                              double* const* out, int64_t* out_ranks, void* stream);

/*
 * tt_gemm_emulated_f64 -- the matrix product that the mixed-precision path
 * runs for its contractions (no counterpart in the paper, which works in FP64
 * throughout), exported so that it can be checked on its own:
 *   C = alpha * A B + beta * C,
 * A an M x K view (element (r, k) at A[r*a_rs + k*a_cs]), B a K x N view
 * (B[k*b_rs + c*b_cs]), C an M x N view (C[r*c_rs + c*c_cs]); all float64
 * device arrays; C must not overlap A or B.
 * Each operand is cut into `digits` (1..8) balanced 7-bit digits relative to
 * the largest exponent of its row (A) or column (B); digit products run on the
 * tensor cores (bf16 in, fp32 accumulation, exact), their sums are kept exactly
 * in integers and rounded once to float64. The error of C[r][c] is below
 * K 2^{4 - 7 digits} max_k |A[r][k]| max_k |B[k][c]| plus the final rounding
 * (typically about sqrt(K) times smaller), so digits = 8 is FP64-class.
 * Bit-wise deterministic. Subnormal inputs count as zero; a row of A or a
 * column of B holding Inf or NaN gives NaN outputs (as does a tensor-core wait
 * that gave up).
 * workspace: NULL (allocated on the stream) or a device block of at least the
 * size reported in the error message of a call with workspace NULL and
 * ws_bytes != 0 (that call returns TT_EINVAL and does nothing else).
 * Errors: TT_EINVAL (sizes, digits, K > 2^20, null operands), TT_ENOMEM,
 * TT_ECUDA. M == 0 or N == 0 does nothing.
 */
int tt_gemm_emulated_f64(int64_t M, int64_t N, int64_t K, double alpha, const double* A, int64_t a_rs,
                         int64_t a_cs, const double* B, int64_t b_rs, int64_t b_cs, double beta, double* C,
                         int64_t c_rs, int64_t c_cs, int32_t digits, void* workspace, size_t ws_bytes,
                         void* stream);

/*
 * tt_selftest_tcgen05_bf16 -- diagnostic of the tensor-core unit (no
 * counterpart in the paper): D = A B^T with A (M x K) and B (N x K) bf16
 * row-major device arrays, D (M x N) fp32 row-major, accumulated in tensor
 * memory by tcgen05.mma. N in [16, 256] and a multiple of 16, K a multiple of
 * 64. *err (device int, zeroed by the caller) becomes 1 if a bounded wait gave up.
 */
int tt_selftest_tcgen05_bf16(int32_t M, int32_t N, int32_t K, const void* A, const void* B, float* D, int* err,
                             void* stream);

/*
 * tt_debug_inject_device_status -- test hook for the failure reporting (no
 * counterpart in the paper). Arms `bits` (1 = a bounded device wait gave up,
 * 2 = a thin QR could not orthogonalize a block): the next read-back of a
 * device status word by this library first overwrites that word on the device
 * with bits by a host copy, so the call returns the matching status
 * (TT_ETIMEOUT, TT_ESINGULAR) through the normal path. The device work itself
 * is not changed. 0 disarms; the hook disarms itself when consumed.
 */
void tt_debug_inject_device_status(int32_t bits);

/*
 * tt_set_qr_mode -- how the thin QRs of later calls (and of plans created
 * later) run (no counterpart in the paper, which uses a Householder QR; every
 * mode returns an orthonormal Q with A = Q R):
 *   0  auto (default): shifted Cholesky QR (Fukaya et al. 2020) as one
 *      cooperative launch that keeps the row blocks in shared memory, where the
 *      blocks fit and the grid is co-resident; else as one launch per pass;
 *   1  shifted Cholesky QR, one launch per pass;
 *   2  the Householder TSQR fallback for every QR with k <= 96 (the path that
 *      otherwise runs only when the Cholesky chain breaks down), for testing it;
 *   3  testing: the cooperative chain runs, then marks itself failed, so the
 *      fallback recomputes every QR with k <= 96 the way it does after a real
 *      breakdown.
 * tt_tsqr_fallback_runs returns how many Householder fallback QRs ran on the
 * current device since the library was loaded (a device counter).
 * Errors: TT_EINVAL for an unknown mode; TT_ECUDA.
 */
int tt_set_qr_mode(int32_t mode);
int tt_tsqr_fallback_runs(int64_t* runs);

/*
 * tt_set_gemm_mode -- how the emulated-FP64 tensor-core products of later calls
 * (and plans created later) run (no counterpart in the paper): 2 = fused, the
 * digit split done by the product kernel straight into shared memory (the
 * exponents scanned there too for an unsplit K <= 512, else one exponent pass
 * first); 1 = three passes, the digit planes written to and re-read from
 * global memory; 0 (default) = fused for groups whose planes would exceed
 * 64 MB and whose operands the fused kernels would split at most twice over
 * (A once per output tile along N, B once per tile along M), else three
 * passes. The results are bit-identical.
 * Errors: TT_EINVAL for an unknown mode.
 */
int tt_set_gemm_mode(int32_t mode);

/*
 * tt_probe_fp64_rate -- diagnostic (no counterpart in the paper): the measured
 * FP64 fused multiply-add rate of the current GPU in TFLOP/s (2 flops per
 * FMA), from one timed launch of independent register-only FMA chains over
 * every SM (iters steps of 8 chains per thread; about 2^16 gives a launch of a
 * few milliseconds). The benchmark takes it as the FP64 roofline peak.
 * Errors: TT_EINVAL, TT_ECUDA.
 */
int tt_probe_fp64_rate(int32_t iters, double* tflops, void* stream);

/*
 * tt_probe_pivot_rsqrt -- diagnostic (no counterpart in the paper): compares
 * the reciprocal square root that the Cholesky-QR pivots use (a hardware
 * approximation with one third-order correction) with CUDA's rsqrt on n points
 * spread over the normal range; *max_ulp is the largest distance in units in
 * the last place, *ndiff the number of points that differ at all.
 * Errors: TT_EINVAL, TT_ECUDA.
 */
int tt_probe_pivot_rsqrt(int64_t n, int64_t* max_ulp, int64_t* ndiff, void* stream);

/*
 * Measurement hooks (no counterpart in the paper; used by the benchmark).
 * tt_prof_enable(1) makes the library record a CUDA event pair on the caller's
 * stream around every grouped-GEMM launch (all contraction steps) and add up the
 * algorithmic flops 2*M*N*K of those launches; every kernel launch of the
 * library is counted whether or not profiling is on. tt_prof_read waits for the
 * recorded events and returns: total GEMM time (ms), GEMM flops, number of
 * GEMM launches and of all kernel launches since the last tt_prof_reset.
 * Any output pointer may be NULL. Errors: TT_ECUDA if an event query fails.
 */
int tt_prof_enable(int on);
int tt_prof_reset(void);
int tt_prof_read(double* gemm_ms, double* gemm_flops, int64_t* gemm_launches, int64_t* kernel_launches);
/* Same for one kind of timed launch: 0 the contraction groups (the GEMM
 * launches above), 1 the Cholesky-QR passes (flops: 4 m k^2 per QR of an
 * m x k block, counted on its first pass). */
int tt_prof_read_kind(int32_t kind, double* ms, double* flops, int64_t* launches);

#ifdef __cplusplus
}
#endif
#endif /* TTROUND_H */

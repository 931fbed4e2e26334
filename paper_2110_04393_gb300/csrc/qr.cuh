// Thin QR for the FP64 path: shifted CholeskyQR3 with a device-flag fallback to
// the Householder TSQR (internal to the library).
#pragma once
#include "plan.cuh"

namespace ttr {

struct QrBufs {
  int64_t m = 0;
  int k = 0;
  int rows = 0;             // rows per CTA in a Cholesky QR pass
  int P = 0;                // CTAs per pass
  double* Gpart = nullptr;  // P x k x k partial Gram matrices
  double* Rinv = nullptr;   // k x k inverse Cholesky factor
  double* Q1 = nullptr;     // m x k
  double* Q2 = nullptr;     // m x k
  double* big = nullptr;    // 3 k x k global scratch for k > 96
  int* status = nullptr;    // [0] failure (Householder fallback for k <= 96), [1] unshifted run,
                            // [2] done, [3] factorizations, then arrival counters
  int nstat = 0;
  TsqrShape sh{};
  double* tw = nullptr;
  int* ti = nullptr;
  size_t ti_n = 0;
};

// Scratch shared by QR factorizations that run one after another on a stream:
// reserve once for every (m, k) shape, then take a view per factorization.
struct QrPool {
  double* Gpart = nullptr;
  double* Rinv = nullptr;
  double* Q1 = nullptr;
  double* Q2 = nullptr;
  double* big = nullptr;
  int* status = nullptr;
  double* tw = nullptr;
  int* ti = nullptr;
};
QrPool qr_pool_reserve(Arena& ar, const std::vector<std::pair<int64_t, int>>& shapes);
QrBufs qr_view(const QrPool& p, int64_t m, int k);
QrBufs qr_reserve(Arena& ar, int64_t m, int k);
// Q must not alias A (the fallback re-reads A). After the schedule ran,
// status[0] != 0 means no orthonormal Q was produced (only possible for k > 96).
// r_may_be_full: R may come out as a full k x k matrix (A = Q R still holds;
// the first-order last pass then spares a factorization); otherwise R is upper
// triangular with a nonnegative diagonal.
// Optional truncation certificate for the thin QR of a right-to-left
// truncation bond (A = H(X_n)^T, R wanted and allowed full): see CoopJob in
// cholqr_f64.cu. When the cooperative chain proves sigma_min(A) > 2 eps (and
// rcap >= k) it writes Q over A (Aw, A's strides), multiplies Xp (mp x k,
// row-major) by R^T in place, sets *rank_out = k and raises the flag that
// qr_cert_flag returns; otherwise the flag stays 0 and Q, R are produced as
// usual. The flag is valid until the pool's next QR starts.
struct QrCert {
  const double* eps;
  int rcap;
  int64_t* rank_out;
  double* Aw;
  double* Xp;
  int64_t mp;
};
void qr_plan(Schedule& sc, const QrBufs& b, const double* A, int64_t a_rs, int64_t a_cs, double* Q, int64_t q_rs,
             int64_t q_cs, double* R, bool r_may_be_full = false, const QrCert* cert = nullptr);
const int* qr_cert_flag(const QrBufs& b);

// How qr_plan runs the chain (library-wide, read when a schedule is built):
// AUTO = one cooperative launch when the row blocks fit in shared memory and
// the grid is co-resident, else the multi-launch chain; CHAIN = always the
// multi-launch chain; FORCE_FALLBACK = skip the Cholesky chain and run the
// Householder TSQR for every QR with k <= 96 (a diagnostic of that path).
constexpr int QR_MODE_AUTO = 0, QR_MODE_CHAIN = 1, QR_MODE_FORCE_FALLBACK = 2, QR_MODE_COOP_THEN_FALLBACK = 3;
int set_qr_mode(int mode);
// Many independent thin QRs (Q only, k <= 96): one multi-launch Cholesky-QR
// chain (CQ_MAX_PASSES launches) covering every job, each job on about
// ctas_per_job CTAs, scratch taken from ar. A job whose chain breaks down
// raises DEV_QR_FAIL in the run's status word (there is no Householder
// fallback for batched jobs). Q must not alias A.
struct QrBatchJob {
  const double* A;
  int64_t a_rs, a_cs;
  double* Q;
  int64_t q_rs, q_cs;
  int64_t m;
  int k;
  // optional scratch (else taken from the arena): two m x k blocks, the
  // partial Gram matrices (qr_batch_gram_doubles) and a k x k factor
  bool has_scratch = false;   // the four pointers below are given (they may be null while sizing)
  double* buf0 = nullptr;
  double* buf1 = nullptr;
  double* gpart = nullptr;
  double* rinv = nullptr;
};
int qr_batch_plan(Arena& ar, Schedule& sc, const std::vector<QrBatchJob>& jobs, int ctas_per_job);
// Doubles of partial Gram matrices that a batched job of shape (m, k) needs.
int64_t qr_batch_gram_doubles(int64_t m, int k, int ctas_per_job);
// Number of Householder TSQR fallback runs on the current device since load.
int tsqr_fallback_runs(long long* out);

}  // namespace ttr

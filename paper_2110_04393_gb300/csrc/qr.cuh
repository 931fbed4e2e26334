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
  int* status = nullptr;    // [0] 1 = fall back to Householder, [1] shifted chain, [2] arrival counter
  TsqrShape sh{};
  double* tw = nullptr;
  int* ti = nullptr;
  size_t ti_n = 0;
};

QrBufs qr_reserve(Arena& ar, int64_t m, int k);
// Q must not alias A (the fallback re-reads A).
void qr_plan(Schedule& sc, const QrBufs& b, const double* A, int64_t a_rs, int64_t a_cs, double* Q, int64_t q_rs,
             int64_t q_cs, double* R);

}  // namespace ttr

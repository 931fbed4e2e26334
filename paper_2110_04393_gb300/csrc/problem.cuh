// A sum of K TT-tensors as passed through the C ABI (internal to the library).
#pragma once
#include "plan.cuh"

namespace ttr {

struct SumProblem {
  int N = 0, K = 0;
  std::vector<int64_t> I;      // [N]
  std::vector<int64_t> R;      // [K*(N+1)]
  std::vector<int64_t> S;      // [N+1] sum of summand ranks per bond
  std::vector<int64_t> off;    // [K*(N+1)] prefix of summand ranks per bond
  std::vector<int64_t> ell;    // [N+1] clamped sketch ranks
  std::vector<const double*> cores;
  std::vector<double> coeffs;
  tt_allreduce_fn allreduce = nullptr;   // summand-sharded rounding: sums the sketch over the ranks
  void* allreduce_ctx = nullptr;
  int64_t r(int j, int n) const { return R[size_t(j) * (N + 1) + n]; }
  int64_t o(int j, int n) const { return off[size_t(j) * (N + 1) + n]; }
  const double* core(int j, int n) const { return cores[size_t(j) * N + (n - 1)]; }   // n is 1-based
};

// Checks sizes/ranks/pointers and clamps the target ranks ells to
// l_n <= min(l_{n-1} I_n, I_{n+1} l_{n+1}).
int validate_sum(int32_t N, int32_t K, const int64_t* dims, const int64_t* ranks, const double* const* cores,
                 const double* coeffs, const int64_t* ells, bool need_cores, SumProblem* P);

// Clamps a rank vector like validate_sum does (r_0 = r_N = 1).
std::vector<int64_t> clamp_rank_vector(const std::vector<int64_t>& I, const int64_t* r);

// Right-to-left truncation (Section 3.2 with Algorithm 2's loop mirrored) of a
// left-orthogonal TT held in out[0..N-1] at ranks ell (layout (l_{n-1}, I_n,
// l_n)); tol <= 0: ranks capped by max_rank only; max_rank <= 0: no cap. The
// decided ranks land in *rk_out (device, N+1) and every core is compacted to
// them in place.
int plan_truncation(Arena& ar, Schedule& sc, int N, const std::vector<int64_t>& I, const std::vector<int64_t>& ell,
                    double tol, double* const* out, int64_t** rk_out, int64_t max_rank);

}  // namespace ttr

// Internal profiling hooks (see prof.cu).
#pragma once
#include <cuda_runtime.h>

#include <vector>

namespace ttr {
// Kinds of timed launches: 0 contraction groups (GEMMs), 1 QR passes.
constexpr int kProfKinds = 2;
void prof_count_launch(int n);
bool prof_gemm_begin(cudaStream_t s, cudaEvent_t* e0);
void prof_gemm_end(cudaStream_t s, double flops);
// Generic pair: begin returns false when profiling is off (then no end call).
bool prof_begin(cudaStream_t s, cudaEvent_t* e0);
void prof_end(cudaStream_t s, int kind, double flops);
// Graph capture: while a sink is set (this thread), GEMM event pairs are
// recorded with fresh events into the sink and launches are counted there.
struct ProfPair;
void prof_capture_begin(std::vector<ProfPair>* sink);
int64_t prof_capture_end();
bool prof_on();
// After a replay (stream synchronized): adds the pairs' times, flops and the
// replay's launches to the totals when profiling is on.
int prof_replayed(const std::vector<ProfPair>& pairs, int64_t launches);
}  // namespace ttr

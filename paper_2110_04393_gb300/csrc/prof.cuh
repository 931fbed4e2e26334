// Internal profiling hooks (see prof.cu).
#pragma once
#include <cuda_runtime.h>

namespace ttr {
void prof_count_launch(int n);
bool prof_gemm_begin(cudaStream_t s, cudaEvent_t* e0);
void prof_gemm_end(cudaStream_t s, double flops);
}  // namespace ttr

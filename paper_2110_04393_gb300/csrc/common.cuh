// Shared device/host helpers of the CUDA path (no method arithmetic here).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>
#include <stdio.h>
#include <string>
#include <vector>

#include "ttround.h"

namespace ttr {

// Thread-local error text behind tt_last_error().
void set_error(const std::string& msg);

struct Status {
  int code = TT_OK;
  bool ok() const { return code == TT_OK; }
};

#define TTR_CHECK_CUDA(expr)                                                        \
  do {                                                                              \
    cudaError_t _e = (expr);                                                        \
    if (_e != cudaSuccess) {                                                        \
      ::ttr::set_error(std::string(#expr) + ": " + cudaGetErrorString(_e));         \
      return int(TT_ECUDA);                                                           \
    }                                                                               \
  } while (0)

#define TTR_CHECK_LAUNCH()                                                          \
  do {                                                                              \
    cudaError_t _e = cudaGetLastError();                                            \
    if (_e != cudaSuccess) {                                                        \
      ::ttr::set_error(std::string("kernel launch: ") + cudaGetErrorString(_e) +    \
                       " at " + __FILE__ + ":" + std::to_string(__LINE__));         \
      return int(TT_ECUDA);                                                           \
    }                                                                               \
  } while (0)

#define TTR_TRY(expr)                    \
  do {                                   \
    int _s = (expr);                     \
    if (_s != TT_OK) return _s;          \
  } while (0)

inline int64_t ceil_div(int64_t a, int64_t b) { return (a + b - 1) / b; }
inline size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

// Bump allocator over one caller-provided (or library-allocated) device block.
struct Arena {
  char* base = nullptr;
  size_t cap = 0;
  size_t used = 0;
  bool sizing = true;   // first pass only measures
  template <typename T>
  T* take(size_t count) {
    size_t bytes = align256(count * sizeof(T));
    size_t off = used;
    used += bytes;
    if (sizing) return nullptr;
    return reinterpret_cast<T*>(base + off);
  }
};

int num_sms();

// Every kernel of the library prefers the largest shared-memory carveout, so
// consecutive kernels with small and large shared memory never make an SM
// switch its L1 / shared-memory split (a switch drains the SM). Called once
// per kernel (TTR_PREFER_SHARED at the launch site); failures are ignored.
inline int prefer_shared_once(const void* fn) {
  if (cudaFuncSetAttribute(fn, cudaFuncAttributePreferredSharedMemoryCarveout, int(cudaSharedmemCarveoutMaxShared)) !=
      cudaSuccess)
    cudaGetLastError();
  return 0;
}
#define TTR_PREFER_SHARED(k)                                                           \
  do {                                                                                 \
    static const int ttr_prefer_shared_once = ::ttr::prefer_shared_once((const void*)(k)); \
    (void)ttr_prefer_shared_once;                                                      \
  } while (0)

}  // namespace ttr

// tt_round_sum_rand_noalloc: the randomized sum rounding with its scratch
// memory in a fixed, library-owned device array, for callers that cannot
// allocate device memory.
//
// Who needs this: code that runs where a cudaMalloc (or a caching allocator's
// growth) is not allowed or not safe -- real-time loops with a fixed memory
// budget, plug-ins whose host application hands out device memory only for
// inputs and outputs, or processes whose device memory is already fully
// claimed by another allocator. Such callers pass inputs and outputs as usual; the
// scratch lives in g_scratch below, a file-scope __device__ array of
// TT_NOALLOC_SCRATCH_BYTES that every GPU which loads this library keeps until
// the process exits.
//
// Rules of use:
//  * Problems whose scratch need (tt_round_sum_rand_workspace) exceeds
//    TT_NOALLOC_SCRATCH_BYTES are rejected with TT_ENOMEM and a message naming
//    both sizes.
//  * Every call on a device shares the same array and leaves its contents
//    behind; each call clears what must start at zero (arrival counters and
//    status flags) before using it. Calls whose device work overlaps (other
//    streams, other host threads) race on the array: serialize them.
//  * The first call on a device looks up the array's device address
//    (cudaGetSymbolAddress with that device current); make that first call
//    before any stream capture.
//  * No cudaMalloc, cudaFree or other allocating call is made.
#include <mutex>
#include <string>

#include "common.cuh"

extern "C" __attribute__((visibility("hidden"))) int sum_rand_common(
    int32_t N, int32_t K, const int64_t* dims, const int64_t* ranks, const double* const* cores,
    const double* coeffs, const int64_t* ells, const double* const* sketch, uint64_t seed, double tol,
    int32_t precision, double* const* out, int64_t* out_ranks, void* workspace, size_t ws_bytes, void* stream,
    size_t* size_only);

namespace {

constexpr size_t kScratchBytes = size_t(TT_NOALLOC_SCRATCH_BYTES);
static_assert(kScratchBytes % 256 == 0, "scratch size must keep 256-byte alignment");

// The scratch array. Host code must not pass &g_scratch to a kernel: on the host
// that name is only a stand-in, so its device address is looked up below.
__device__ __align__(256) unsigned char g_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void* g_addr[kMaxDevices] = {};

int scratch_address(void** out) {
  int dev = 0;
  TTR_CHECK_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kMaxDevices) {
    ttr::set_error("tt_round_sum_rand_noalloc: device ordinal out of range");
    return TT_EUNSUPPORTED;
  }
  std::lock_guard<std::mutex> g(g_mu);
  if (!g_addr[dev]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_scratch);
    if (e != cudaSuccess || p == nullptr) {
      ttr::set_error(std::string("tt_round_sum_rand_noalloc: cudaGetSymbolAddress failed: ") +
                     cudaGetErrorString(e));
      return TT_ECUDA;
    }
    g_addr[dev] = p;
  }
  *out = g_addr[dev];
  return TT_OK;
}

}  // namespace

extern "C" {

size_t tt_noalloc_scratch_bytes(void) { return kScratchBytes; }

int tt_round_sum_rand_noalloc(int32_t N, int32_t K, const int64_t* dims, const int64_t* ranks,
                              const double* const* cores, const double* coeffs, const int64_t* ells,
                              const double* const* sketch, uint64_t seed, double tol, int32_t precision,
                              double* const* out, int64_t* out_ranks, void* stream) {
  size_t need = 0;
  int rc = sum_rand_common(N, K, dims, ranks, cores, coeffs, ells, sketch, seed, tol, precision, out, out_ranks,
                           nullptr, 0, stream, &need);
  if (rc != TT_OK) return rc;
  if (need > kScratchBytes) {
    ttr::set_error("tt_round_sum_rand_noalloc: problem needs " + std::to_string(need) +
                   " bytes of scratch, above the fixed " + std::to_string(kScratchBytes) +
                   " bytes; use tt_round_sum_rand with a caller workspace");
    return TT_ENOMEM;
  }
  void* scratch = nullptr;
  rc = scratch_address(&scratch);
  if (rc != TT_OK) return rc;
  return sum_rand_common(N, K, dims, ranks, cores, coeffs, ells, sketch, seed, tol, precision, out, out_ranks,
                         scratch, kScratchBytes, stream, nullptr);
}

}  // extern "C"

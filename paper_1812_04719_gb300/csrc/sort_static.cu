// Allocation-free variant of stiv_sort_pairs.
//
// stiv_sort_pairs needs a caller-provided device scratch buffer.  Some callers
// cannot provide one: code that runs inside another framework's device memory
// pool (which owns all device memory and forbids raw cudaMalloc), real-time
// loops where a cudaMalloc/cudaFree (which may synchronise the whole device)
// would stall the pipeline, or processes that have exhausted their allocation
// budget.  stiv_sort_pairs_static runs the same radix sort on a fixed scratch
// area that is part of the library image: a file-scope __device__ array that
// every GPU which loads libstiv holds until the process exits.
//
// Limits and sharing: at most STIV_SORT_STATIC_MAX pairs per call.  All calls
// share the one array per device (it keeps the previous call's contents), so
// calls whose executions overlap on the GPU (e.g. on two streams) race.  The
// sort writes every histogram entry it reads, so no part of the array has to
// start at zero.
#include "stiv_internal.cuh"

namespace {

constexpr int64_t kMaxPairs = STIV_SORT_STATIC_MAX;
constexpr size_t kHistBytes = (size_t)1 << 20;                // >= digit histograms for kMaxPairs
constexpr size_t kKeyBytes = sizeof(uint64_t) * (size_t)kMaxPairs;
constexpr size_t kValBytes = sizeof(int32_t) * (size_t)kMaxPairs;
constexpr size_t kScratchBytes = kHistBytes + kKeyBytes + kValBytes;  // 13.6 MB

// In host code this name is only a stand-in for the device object; its
// device address comes from cudaGetSymbolAddress (below).
static __device__ __align__(256) unsigned char g_sort_scratch[kScratchBytes];

// Device address of g_sort_scratch on the current device, looked up on every
// call with that device current.  The lookup is a host-side table read once
// the library's device code is loaded on the device; the first call on a
// device is the one that loads it.  Not caching the address keeps it valid
// across a device reset or a new context, where the array may move.
int scratch_address(unsigned char** out) {
  void* p = nullptr;
  if (cudaGetSymbolAddress(&p, g_sort_scratch) != cudaSuccess || !p) return STIV_ERR_CUDA;
  *out = (unsigned char*)p;
  return STIV_OK;
}

}  // namespace

extern "C" int stiv_sort_pairs_static(void* stream, int64_t n, int32_t key_bits, const uint64_t* keys_in,
                                      const int32_t* vals_in, uint64_t* keys_out, int32_t* vals_out) {
  if (n < 0 || n > kMaxPairs || key_bits < 0 || key_bits > 64) return STIV_ERR_ARG;
  if (n == 0) return STIV_OK;
  if (!keys_in || !vals_in || !keys_out || !vals_out) return STIV_ERR_ARG;
  if (stiv_sort_scratch_impl(n) > kHistBytes) return STIV_ERR_ARG;
  unsigned char* base = nullptr;
  int rc = scratch_address(&base);
  if (rc) return rc;
  cudaStream_t st = (cudaStream_t)stream;
  // the sort ping-pongs between its input and output arrays: sort staging
  // copies so that the caller's input stays intact
  uint64_t* kt = (uint64_t*)(base + kHistBytes);
  int32_t* vt = (int32_t*)(base + kHistBytes + kKeyBytes);
  if (cudaMemcpyAsync(kt, keys_in, sizeof(uint64_t) * (size_t)n, cudaMemcpyDeviceToDevice, st) != cudaSuccess)
    return STIV_ERR_CUDA;
  if (cudaMemcpyAsync(vt, vals_in, sizeof(int32_t) * (size_t)n, cudaMemcpyDeviceToDevice, st) != cudaSuccess)
    return STIV_ERR_CUDA;
  return stiv_sort_pairs_impl(st, n, key_bits, kt, vt, keys_out, vals_out, base, kHistBytes, nullptr);
}

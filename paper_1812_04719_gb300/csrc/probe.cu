// Arithmetic-rate probe of this GPU: the denominators of the library's
// FP64 and FP32 rooflines, measured rather than taken from a datasheet.
//
// Each thread runs NCHAIN independent multiply-add chains (x <- x * b + c,
// one fused multiply-add each) for iters steps, so that every FMA pipe of
// every SM stays busy; the chains' sum is written out so that nothing is
// optimised away.  The launch performs exactly 2 * NCHAIN * iters * threads
// floating-point operations (an FMA counts 2).
#include "stiv_internal.cuh"

namespace {

constexpr int NCHAIN = 8;
constexpr int PROBE_THREADS = 256;
constexpr int PROBE_BLOCKS_PER_SM = 8;

template <typename T>
__device__ __forceinline__ T fma_rn(T a, T b, T c);
template <>
__device__ __forceinline__ double fma_rn<double>(double a, double b, double c) { return __fma_rn(a, b, c); }
template <>
__device__ __forceinline__ float fma_rn<float>(float a, float b, float c) { return __fmaf_rn(a, b, c); }

template <typename T>
__global__ void __launch_bounds__(PROBE_THREADS) fma_probe_kernel(int64_t iters, T b, T c, double* sink) {
  T x[NCHAIN];
#pragma unroll
  for (int k = 0; k < NCHAIN; ++k) x[k] = (T)(threadIdx.x + k) * (T)1e-3;
#pragma unroll 4
  for (int64_t i = 0; i < iters; ++i) {
#pragma unroll
    for (int k = 0; k < NCHAIN; ++k) x[k] = fma_rn<T>(x[k], b, c);
  }
  T s = 0;
#pragma unroll
  for (int k = 0; k < NCHAIN; ++k) s += x[k];
  // b is chosen by the host so that this never holds: the write only keeps
  // the chains alive
  if (s == (T)-12345.0) sink[0] = (double)s;
}

}  // namespace

extern "C" int stiv_peak_probe(void* stream, int32_t kind, int64_t iters, double* sink_dev, double* flops_out) {
  if (kind < 0 || kind > 1 || iters < 1 || iters > ((int64_t)1 << 32) || !sink_dev || !flops_out)
    return STIV_ERR_ARG;
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return STIV_ERR_CUDA;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms < 1)
    return STIV_ERR_CUDA;
  int blocks = sms * PROBE_BLOCKS_PER_SM;
  cudaStream_t st = (cudaStream_t)stream;
  if (kind == 0)
    fma_probe_kernel<double><<<blocks, PROBE_THREADS, 0, st>>>(iters, 0.999999, 1e-7, sink_dev);
  else
    fma_probe_kernel<float><<<blocks, PROBE_THREADS, 0, st>>>(iters, 0.999999f, 1e-7f, sink_dev);
  if (cudaGetLastError() != cudaSuccess) return STIV_ERR_CUDA;
  *flops_out = 2.0 * NCHAIN * (double)iters * (double)blocks * PROBE_THREADS;
  return STIV_OK;
}

// Stable LSD radix sort of (64-bit key, int32 value) pairs, 8-bit digits.
//
// Replaces the distributed hypercube quicksort of Alg. 1's check-point sort (Sec. 3.3.1,
// Table 3) on one GPU: equal keys keep their input order, so the payload is
// "scattered" exactly as in Table 3.  The item count may live on the device
// (n_dev); the host passes an upper bound for the launch shapes.
//
// Per digit pass: (1) per-tile digit histograms [digit][tile], (2) one CTA per
// digit scans its row over the tiles (exclusive, coalesced) and writes the
// digit's total, (3) a stable scatter: each tile scans the 256 digit totals,
// ranks its items warp by warp with __match_any_sync and writes them at
// digit base + tile offset + rank.
#include "stiv_internal.cuh"

namespace {

constexpr int kThreads = 256;
constexpr int kItems = 8;                    // items per thread per tile
constexpr int kTile = kThreads * kItems;     // 2048 items per tile
constexpr int kRadix = 256;
constexpr int kWarps = kThreads / 32;
static_assert(kThreads == kRadix, "the scatter scans the digit totals one per thread");

// Exclusive scan of one value per thread over the CTA (kThreads), in a fixed
// order; *total gets the sum.  wsum: kWarps ints of shared memory.
__device__ __forceinline__ int32_t cta_exclusive_scan(int32_t v, int32_t* wsum, int32_t* total) {
  int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  int32_t x = v;
  for (int off = 1; off < 32; off <<= 1) {
    int32_t y = __shfl_up_sync(0xffffffffu, x, off);
    if (lane >= off) x += y;
  }
  if (lane == 31) wsum[w] = x;
  __syncthreads();
  int32_t pre = 0, tot = 0;
  for (int q = 0; q < kWarps; ++q) {
    int32_t s = wsum[q];
    pre += q < w ? s : 0;
    tot += s;
  }
  __syncthreads();
  *total = tot;
  return pre + x - v;
}

__device__ __forceinline__ int64_t load_n(const int64_t* n_dev, int64_t n_max) {
  if (!n_dev) return n_max;
  int64_t n = *n_dev;
  return n < n_max ? n : n_max;
}

__global__ void __launch_bounds__(kThreads) hist_kernel(const uint64_t* keys, const int64_t* n_dev, int64_t n_max,
                                                         int shift, int ntiles, int32_t* hist) {
  __shared__ int32_t h[kRadix];
  int64_t n = load_n(n_dev, n_max);
  for (int d = threadIdx.x; d < kRadix; d += kThreads) h[d] = 0;
  __syncthreads();
  int64_t base = (int64_t)blockIdx.x * kTile;
  for (int k = 0; k < kItems; ++k) {
    int64_t idx = base + (int64_t)k * kThreads + threadIdx.x;
    if (idx < n) atomicAdd(&h[(keys[idx] >> shift) & 0xFF], 1);
  }
  __syncthreads();
  for (int d = threadIdx.x; d < kRadix; d += kThreads) hist[(int64_t)d * ntiles + blockIdx.x] = h[d];
}

// CTA d: exclusive scan of hist[d][0 .. ntiles) in place; totals[d] = the sum.
__global__ void __launch_bounds__(kThreads) scan_kernel(int32_t* hist, int ntiles, int32_t* totals) {
  __shared__ int32_t wsum[kWarps];
  int32_t* row = hist + (int64_t)blockIdx.x * ntiles;
  int32_t carry = 0;
  for (int base = 0; base < ntiles; base += kThreads) {
    int i = base + threadIdx.x;
    int32_t v = i < ntiles ? row[i] : 0, tot;
    int32_t ex = cta_exclusive_scan(v, wsum, &tot);
    if (i < ntiles) row[i] = carry + ex;
    carry += tot;
  }
  if (threadIdx.x == 0) totals[blockIdx.x] = carry;
}

__global__ void __launch_bounds__(kThreads) scatter_kernel(const uint64_t* kin, const int32_t* vin, uint64_t* kout,
                                                            int32_t* vout, const int64_t* n_dev, int64_t n_max,
                                                            int shift, int ntiles, const int32_t* hist,
                                                            const int32_t* totals) {
  __shared__ int32_t tile_off[kRadix];
  __shared__ int32_t wsum[kWarps];
  __shared__ int32_t round_tot[kRadix];
  __shared__ int32_t warp_cnt[kWarps][kRadix];
  int64_t n = load_n(n_dev, n_max);
  if ((int64_t)blockIdx.x * kTile >= n) return;   // an empty tile scatters nothing
  int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  {
    int32_t tot;
    int32_t dbase = cta_exclusive_scan(totals[threadIdx.x], wsum, &tot);   // digit d = threadIdx.x
    tile_off[threadIdx.x] = dbase + hist[(int64_t)threadIdx.x * ntiles + blockIdx.x];
  }
  int64_t base = (int64_t)blockIdx.x * kTile;
  // a tile is processed in kItems rounds of kThreads consecutive items; within
  // a round items are ranked warp by warp, lanes in order: the scatter is stable
  for (int k = 0; k < kItems; ++k) {
    for (int d = threadIdx.x; d < kWarps * kRadix; d += kThreads) (&warp_cnt[0][0])[d] = 0;
    __syncthreads();
    int64_t idx = base + (int64_t)k * kThreads + threadIdx.x;
    bool valid = idx < n;
    uint64_t key = valid ? kin[idx] : 0;
    int32_t val = valid ? vin[idx] : 0;
    int digit = valid ? (int)((key >> shift) & 0xFF) : -1;
    unsigned peers = __match_any_sync(0xffffffffu, digit);
    int rank = __popc(peers & ((1u << lane) - 1u));
    if (valid && rank == 0) warp_cnt[w][digit] = __popc(peers);
    __syncthreads();
    for (int d = threadIdx.x; d < kRadix; d += kThreads) {
      int32_t run = 0;
      for (int q = 0; q < kWarps; ++q) { int32_t c = warp_cnt[q][d]; warp_cnt[q][d] = run; run += c; }
      round_tot[d] = run;
    }
    __syncthreads();
    if (valid) {
      int32_t pos = tile_off[digit] + warp_cnt[w][digit] + rank;
      kout[pos] = key;
      vout[pos] = val;
    }
    __syncthreads();
    for (int d = threadIdx.x; d < kRadix; d += kThreads) tile_off[d] += round_tot[d];
    __syncthreads();
  }
}

}  // namespace

size_t stiv_sort_scratch_impl(int64_t n) {
  int64_t ntiles = (n + kTile - 1) / kTile;
  if (ntiles < 1) ntiles = 1;
  return sizeof(int32_t) * (size_t)(kRadix * ntiles + kRadix) + 256;
}

// Sorts n (or *n_dev if given, <= n) pairs.  Result lands in kout/vout; kin/vin
// are used as ping-pong buffers and are overwritten.
int stiv_sort_pairs_impl(cudaStream_t st, int64_t n, int key_bits, const uint64_t* kin, const int32_t* vin,
                         uint64_t* kout, int32_t* vout, void* scratch, size_t scratch_bytes,
                         const int64_t* n_dev) {
  if (n < 0 || key_bits < 0 || key_bits > 64) return STIV_ERR_ARG;
  int64_t ntiles = (n + kTile - 1) / kTile;
  if (ntiles < 1) ntiles = 1;
  if (scratch_bytes < stiv_sort_scratch_impl(n)) return STIV_ERR_ARG;
  int32_t* hist = (int32_t*)scratch;
  int32_t* totals = hist + (size_t)kRadix * ntiles;
  int passes = (key_bits + 7) / 8;
  if (passes == 0) {
    if (n > 0) {
      if (cudaMemcpyAsync(kout, kin, sizeof(uint64_t) * n, cudaMemcpyDeviceToDevice, st) != cudaSuccess) return STIV_ERR_CUDA;
      if (cudaMemcpyAsync(vout, vin, sizeof(int32_t) * n, cudaMemcpyDeviceToDevice, st) != cudaSuccess) return STIV_ERR_CUDA;
    }
    return STIV_OK;
  }
  // ping-pong so that the last pass writes kout/vout
  uint64_t* ka = (uint64_t*)kin; int32_t* va = (int32_t*)vin;
  uint64_t* kb = kout; int32_t* vb = vout;
  if (passes % 2 == 0) {
    // even number of passes: first copy input to the output buffers, then start from there
    if (n > 0) {
      if (cudaMemcpyAsync(kout, kin, sizeof(uint64_t) * n, cudaMemcpyDeviceToDevice, st) != cudaSuccess) return STIV_ERR_CUDA;
      if (cudaMemcpyAsync(vout, vin, sizeof(int32_t) * n, cudaMemcpyDeviceToDevice, st) != cudaSuccess) return STIV_ERR_CUDA;
    }
    ka = kout; va = vout; kb = (uint64_t*)kin; vb = (int32_t*)vin;
  }
  for (int ps = 0; ps < passes; ++ps) {
    int shift = 8 * ps;
    hist_kernel<<<(unsigned)ntiles, kThreads, 0, st>>>(ka, n_dev, n, shift, (int)ntiles, hist);
    scan_kernel<<<kRadix, kThreads, 0, st>>>(hist, (int)ntiles, totals);
    scatter_kernel<<<(unsigned)ntiles, kThreads, 0, st>>>(ka, va, kb, vb, n_dev, n, shift, (int)ntiles, hist,
                                                          totals);
    if (cudaGetLastError() != cudaSuccess) return STIV_ERR_CUDA;
    uint64_t* tk = ka; ka = kb; kb = tk;
    int32_t* tv = va; va = vb; vb = tv;
  }
  return STIV_OK;
}

extern "C" size_t stiv_sort_scratch_bytes(int64_t n) {
  if (n < 0) n = 0;
  return ((stiv_sort_scratch_impl(n) + 15) & ~(size_t)15) + sizeof(uint64_t) * (size_t)n + sizeof(int32_t) * (size_t)n + 64;
}

extern "C" int stiv_sort_pairs(void* stream, int64_t n, int32_t key_bits, const uint64_t* keys_in,
                               const int32_t* vals_in, uint64_t* keys_out, int32_t* vals_out,
                               void* scratch, size_t scratch_bytes) {
  if (n < 0 || (n > 0 && (!keys_in || !vals_in || !keys_out || !vals_out || !scratch))) return STIV_ERR_ARG;
  if (n == 0) return STIV_OK;
  // keep the caller's input intact: sort a copy held in the output buffers
  // (the implementation ping-pongs between its in and out arrays)
  size_t need = stiv_sort_scratch_impl(n);
  if (scratch_bytes < stiv_sort_scratch_bytes(n)) return STIV_ERR_ARG;
  uint64_t* kt = (uint64_t*)((char*)scratch + ((need + 15) & ~(size_t)15));
  int32_t* vt = (int32_t*)(kt + n);
  cudaStream_t st = (cudaStream_t)stream;
  if (cudaMemcpyAsync(kt, keys_in, sizeof(uint64_t) * n, cudaMemcpyDeviceToDevice, st) != cudaSuccess) return STIV_ERR_CUDA;
  if (cudaMemcpyAsync(vt, vals_in, sizeof(int32_t) * n, cudaMemcpyDeviceToDevice, st) != cudaSuccess) return STIV_ERR_CUDA;
  return stiv_sort_pairs_impl(st, n, key_bits, kt, vt, keys_out, vals_out, scratch, need, nullptr);
}

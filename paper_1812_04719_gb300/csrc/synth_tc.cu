// Sec. 3.1.1-3.1.2 synthesis in the reduced-precision form (STIV_MIXED) on the
// 5th-generation tensor cores: 3xTF32 products accumulated in FP32.
//
// For one SH order p the synthesis of every field (vesicle, time, coordinate)
// is one dense contraction
//     X[row][col] = sum_q Y[row][q] C[q][col],
// Y the (n_v x (p+1)^2) synthesis matrix of the order-2p grid and its poles
// (real orthonormal SH, Gauss-Legendre rings, uniform longitudes), C the
// coefficient columns.  The degree-0 term (Y[row][0] = 1/sqrt(4 pi) for every
// row: the vesicle's centre) is kept out of the contraction and added in the
// epilogue, so the FP32 error is relative to the vesicle's size, not to its
// position in the box.
//
// Split products: a = a_hi + a_lo with a_hi = tf32(a) and a_lo = tf32(a -
// a_hi) (both rounded to nearest, exactly representable in TF32), and
// A B ~ A_hi B_hi + A_hi B_lo + A_lo B_hi, each TF32 x TF32 product exact in
// the FP32 accumulator.
//
// Data layout: both operands are K-major and stored in global memory already
// in the tensor cores' shared-memory layout, in blocks of 128 rows x 32 k
// (hi block 16 KB followed by lo block 16 KB):
//     block[kg][row][4 floats],  kg = k / 4 (8 groups), 16 bytes per row,
// i.e. the canonical no-swizzle K-major layout: core matrices of 8 rows x 16
// bytes (128 contiguous bytes), 8-row groups 128 bytes apart (stride byte
// offset), k groups 2048 bytes apart (leading byte offset).  One block is one
// 32 KB bulk copy (cp.async.bulk) into shared memory.
//
// Kernels:
//   ytab_kernel   Y blocks per order p (once per handle and order)
//   group_kernel  vesicles bucketed by order, per-order tile counts and offsets
//   bprep_kernel  coefficient blocks (FP64 -> FP32 split) and per-column
//                 output address and degree-0 term
//   gemm_kernel   persistent, warp-specialised: per tile (order, 128 rows,
//                 128 columns) warp 0 streams the A and B blocks through a
//                 3-stage shared-memory ring (bulk copies completing on
//                 mbarriers), warp 1 issues tcgen05.mma (M = 128, N = 128,
//                 K = 8, kind::tf32) into one of two TMEM accumulators, and
//                 warps 2-5 read the other accumulator (tcgen05.ld 32x32b) and
//                 write the FP32 vertices while the next tile accumulates.
// Every wait on an mbarrier is bounded; a wait that gives up sets a status
// word (reported as STIV_F_TIMEOUT) and the tile is abandoned.
#include "stiv_internal.cuh"

#include <math.h>

namespace {

constexpr int TM = 128;                 // tile rows (vertices)
constexpr int TN = 128;                 // tile columns (fields)
constexpr int TK = 32;                  // k per block
constexpr int BLK_FLOATS = 8 * TM * 4;  // one hi or lo block: 4096 floats = 16 KB
constexpr int BLK_BYTES = 2 * BLK_FLOATS * 4;  // hi + lo = 32 KB
constexpr int STAGE_BYTES = 2 * BLK_BYTES;     // A + B
constexpr long long WAIT_CYCLES = 2000000000LL; // bound of every mbarrier wait (SM clocks)
constexpr long long DRAIN_CYCLES = 200000000LL;  // bound of the final drains (about 0.1 s)
constexpr double Y00 = 0.28209479177387814347;  // 1 / sqrt(4 pi)

__host__ __device__ inline int tc_mtiles(int p) { return (stiv_nverts(2 * p) + TM - 1) / TM; }
__host__ __device__ inline int tc_kblocks(int p) { return ((p + 1) * (p + 1) - 1 + TK - 1) / TK; }

// tf32 rounding to nearest (ties to even) of a finite float
__device__ __forceinline__ float tf32_rn(float x) {
  unsigned b = __float_as_uint(x);
  b += 0x0FFFu + ((b >> 13) & 1u);
  return __uint_as_float(b & 0xFFFFE000u);
}

// index of element (row, k) inside a hi or lo block
__device__ __forceinline__ int blk_index(int row, int k) { return (k >> 2) * (TM * 4) + row * 4 + (k & 3); }

// ---------------------------------------------------------------------------
// Synthesis matrix entry Y(row, q) of order p (grid vertex i * 2P + j or a
// pole; coefficient n^2 + n + m), from the FP64 Legendre table.
// ---------------------------------------------------------------------------
__device__ double ymat(int p, const double* leg, int row, int q) {
  int P = 2 * p, W = 2 * P, nl = (p + 1) * (p + 2) / 2;
  int n = (int)sqrt((double)q);
  while (n * n > q) --n;
  while ((n + 1) * (n + 1) <= q) ++n;
  int m = q - n * n - n, am = m < 0 ? -m : m;
  if (row < W * (P + 1)) {
    int i = row / W, j = row % W;
    double L = leg[(size_t)i * nl + n * (n + 1) / 2 + am];
    double tr = 1.0;
    if (m != 0) {
      double sv, cv;
      sincospi((double)((am * j) % W) / P, &sv, &cv);
      tr = m > 0 ? cv : sv;
    }
    return L * tr;
  }
  if (m != 0) return 0.0;
  int pole = row - W * (P + 1);
  return leg[(size_t)(P + 1 + pole) * nl + n * (n + 1) / 2];
}

// Y blocks of order p for the synthesis: rows = vertices, k = q - 1 (the
// degree-0 column is added in the epilogue): [mtile][kblock][hi | lo][8][128][4]
__global__ void ytab_kernel(int p, const double* leg, float* ytab) {
  int nv = stiv_nverts(2 * p), nc = (p + 1) * (p + 1);
  int MT = tc_mtiles(p), KB = tc_kblocks(p);
  int64_t total = (int64_t)MT * KB * TM * TK;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
    int k = (int)(t % TK);
    int64_t rest = t / TK;
    int r = (int)(rest % TM);
    rest /= TM;
    int kb = (int)(rest % KB), mt = (int)(rest / KB);
    int row = mt * TM + r, q = kb * TK + k + 1;
    double y = (row < nv && q < nc) ? ymat(p, leg, row, q) : 0.0;
    float yf = (float)y, hi = tf32_rn(yf), lo = tf32_rn(yf - hi);
    float* blk = ytab + ((size_t)mt * KB + kb) * (2 * BLK_FLOATS);
    blk[blk_index(r, k)] = hi;
    blk[BLK_FLOATS + blk_index(r, k)] = lo;
  }
}

// Transposed blocks for the adjoint: rows = coefficients q (all, degree 0
// included), k = vertices: [mtile over q][kblock over vertices][hi | lo][8][128][4]
__host__ __device__ inline int tcA_mtiles(int p) { return ((p + 1) * (p + 1) + TM - 1) / TM; }
__host__ __device__ inline int tcA_kblocks(int p) { return (stiv_nverts(2 * p) + TK - 1) / TK; }

__global__ void ytabT_kernel(int p, const double* leg, float* ytab) {
  int nv = stiv_nverts(2 * p), nc = (p + 1) * (p + 1);
  int MT = tcA_mtiles(p), KB = tcA_kblocks(p);
  int64_t total = (int64_t)MT * KB * TM * TK;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
    int k = (int)(t % TK);
    int64_t rest = t / TK;
    int r = (int)(rest % TM);
    rest /= TM;
    int kb = (int)(rest % KB), mt = (int)(rest / KB);
    int q = mt * TM + r, row = kb * TK + k;
    double y = (row < nv && q < nc) ? ymat(p, leg, row, q) : 0.0;
    float yf = (float)y, hi = tf32_rn(yf), lo = tf32_rn(yf - hi);
    float* blk = ytab + ((size_t)mt * KB + kb) * (2 * BLK_FLOATS);
    blk[blk_index(r, k)] = hi;
    blk[BLK_FLOATS + blk_index(r, k)] = lo;
  }
}

// ---------------------------------------------------------------------------
// per-call grouping by order
// ---------------------------------------------------------------------------
struct tc_group {
  int cnt, list_off, ntn, mt, kb, tile_off;  // vesicles, list offset, column tiles, row tiles, k blocks, first tile
  int nrows;                                 // rows of the output (vertices, or coefficients for the adjoint)
  int pad;
  long long boff;                            // first B block of the group
  long long coff;                            // first column (of all groups' padded columns)
};

// tc_ws layout: [status int][ntiles int][pad][groups (STIV_MAX_P+1)][list n][colinfo][B blocks]
struct tc_colinfo {
  long long dst;  // element offset of row 0 of this field in the vertex array (-1: padding column)
  float bias;     // degree-0 term
  float pad;
};

// adjoint = 0: synthesis (6 fields per vesicle, rows = vertices, k = q - 1);
// adjoint = 1: transposed synthesis of the X1 gradient (3 fields per vesicle,
// rows = coefficients, k = vertices)
__global__ void group_kernel(int n, int p_max, const int32_t* pv, tc_group* g, int* ntiles, int* list, int adjoint) {
  __shared__ int cnt[STIV_MAX_P + 1], fill[STIV_MAX_P + 1], off[STIV_MAX_P + 1];
  for (int p = threadIdx.x; p <= STIV_MAX_P; p += blockDim.x) { cnt[p] = 0; fill[p] = 0; }
  __syncthreads();
  for (int v = threadIdx.x; v < n; v += blockDim.x) {
    int p = pv[v];
    if (p >= 1 && p <= p_max) atomicAdd(&cnt[p], 1);
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    int lo = 0, to = 0;
    long long bo = 0, co = 0;
    for (int p = 0; p <= STIV_MAX_P; ++p) {
      tc_group G;
      G.cnt = (p >= 1 && p <= p_max) ? cnt[p] : 0;
      G.list_off = lo;
      G.ntn = ((adjoint ? 3 : 6) * G.cnt + TN - 1) / TN;
      G.mt = p < 1 ? 0 : adjoint ? tcA_mtiles(p) : tc_mtiles(p);
      G.kb = p < 1 ? 0 : adjoint ? tcA_kblocks(p) : tc_kblocks(p);
      G.nrows = p < 1 ? 0 : adjoint ? (p + 1) * (p + 1) : stiv_nverts(2 * p);
      G.pad = 0;
      G.tile_off = to;
      G.boff = bo;
      G.coff = co;
      off[p] = lo;
      lo += G.cnt;
      to += G.mt * G.ntn;
      bo += (long long)G.ntn * G.kb;
      co += (long long)G.ntn * TN;
      g[p] = G;
    }
    *ntiles = to;
  }
  __syncthreads();
  for (int v = threadIdx.x; v < n; v += blockDim.x) {
    int p = pv[v];
    if (p >= 1 && p <= p_max) list[off[p] + atomicAdd(&fill[p], 1)] = v;
  }
}

// B blocks: column c of order group p is field (c % 6) of vesicle list[c / 6];
// thread per (group, column, k block, k group of 4).
__global__ void bprep_kernel(int p_max, const tc_group* g, const int* list, const int64_t* coef_off,
                             const double* coef, const int64_t* vert_off, float* bblk, tc_colinfo* ci) {
  for (int p = 1; p <= p_max; ++p) {
    tc_group G = g[p];
    if (G.cnt == 0) continue;
    int nc = (p + 1) * (p + 1), nv = stiv_nverts(2 * p);
    long long ncols = (long long)G.ntn * TN;
    long long items = ncols * G.kb * (TK / 4);
    for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < items;
         t += (long long)gridDim.x * blockDim.x) {
      int kg = (int)(t % (TK / 4));
      long long rest = t / (TK / 4);
      long long c = rest % ncols;
      int kb = (int)(rest / ncols);
      int v = c / 6 < G.cnt ? list[G.list_off + c / 6] : -1;
      int f = (int)(c % 6);
      float hi[4], lo[4];
      for (int e = 0; e < 4; ++e) {
        int q = kb * TK + kg * 4 + e + 1;
        float x = 0.f;
        if (v >= 0 && q < nc) x = __double2float_rn(coef[coef_off[v] + (size_t)f * nc + q]);
        hi[e] = tf32_rn(x);
        lo[e] = tf32_rn(x - hi[e]);
      }
      int nt = (int)(c / TN), r = (int)(c % TN);
      float* blk = bblk + ((size_t)G.boff + (size_t)nt * G.kb + kb) * (2 * BLK_FLOATS);
      *(float4*)(blk + blk_index(r, kg * 4)) = make_float4(hi[0], hi[1], hi[2], hi[3]);
      *(float4*)(blk + BLK_FLOATS + blk_index(r, kg * 4)) = make_float4(lo[0], lo[1], lo[2], lo[3]);
      if (kb == 0 && kg == 0) {
        tc_colinfo info;
        info.dst = v >= 0 ? (long long)vert_off[v] + (long long)f * nv : -1;
        info.bias = v >= 0 ? (float)(Y00 * coef[coef_off[v] + (size_t)f * nc]) : 0.f;
        info.pad = 0.f;
        ci[(size_t)G.coff + c] = info;
      }
    }
  }
}

// B blocks of the adjoint: column c of order group p is coordinate (c % 3) of
// the X1 block of vesicle list[c / 3] of the gradient gX (FP64, vertex
// layout); k = vertex.  Thread per (group, column, k block, 4 vertices).
__global__ void gprep_kernel(int p_max, const tc_group* g, const int* list, const int64_t* coef_off,
                             const int64_t* vert_off, const double* gX, float* bblk, tc_colinfo* ci) {
  for (int p = 1; p <= p_max; ++p) {
    tc_group G = g[p];
    if (G.cnt == 0) continue;
    int nc = (p + 1) * (p + 1), nv = stiv_nverts(2 * p);
    long long ncols = (long long)G.ntn * TN;
    long long items = ncols * G.kb * (TK / 4);
    for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < items;
         t += (long long)gridDim.x * blockDim.x) {
      int kg = (int)(t % (TK / 4));
      long long rest = t / (TK / 4);
      long long c = rest % ncols;
      int kb = (int)(rest / ncols);
      int v = c / 3 < G.cnt ? list[G.list_off + c / 3] : -1;
      int f = (int)(c % 3);
      float hi[4], lo[4];
      for (int e = 0; e < 4; ++e) {
        int row = kb * TK + kg * 4 + e;
        float x = 0.f;
        if (v >= 0 && row < nv) x = __double2float_rn(gX[vert_off[v] + (size_t)(3 + f) * nv + row]);
        hi[e] = tf32_rn(x);
        lo[e] = tf32_rn(x - hi[e]);
      }
      int nt = (int)(c / TN), r = (int)(c % TN);
      float* blk = bblk + ((size_t)G.boff + (size_t)nt * G.kb + kb) * (2 * BLK_FLOATS);
      *(float4*)(blk + blk_index(r, kg * 4)) = make_float4(hi[0], hi[1], hi[2], hi[3]);
      *(float4*)(blk + BLK_FLOATS + blk_index(r, kg * 4)) = make_float4(lo[0], lo[1], lo[2], lo[3]);
      if (kb == 0 && kg == 0) {
        tc_colinfo info;
        info.dst = v >= 0 ? (long long)coef_off[v] + (long long)(3 + f) * nc : -1;
        info.bias = 0.f;
        info.pad = 0.f;
        ci[(size_t)G.coff + c] = info;
      }
    }
  }
}

// X0 blocks of the coefficient gradient are zero (X0 is a constant of the step).
__global__ void zero_x0_kernel(int n, int p_max, const int32_t* pv, const int64_t* coef_off, double* gcoef) {
  int v = blockIdx.x;
  if (v >= n || pv[v] < 1 || pv[v] > p_max) return;   // order outside [1, p_max]: skipped
  int nc = (pv[v] + 1) * (pv[v] + 1);
  for (int k = threadIdx.x; k < 3 * nc; k += blockDim.x) gcoef[coef_off[v] + k] = 0.0;
}

// ---------------------------------------------------------------------------
// tcgen05 / bulk-copy / mbarrier primitives (inline PTX)
// ---------------------------------------------------------------------------
__device__ __forceinline__ unsigned smem_u32(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(unsigned bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(unsigned bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}
// true once the phase with the given parity has completed; gives up after
// limit SM clocks (WAIT_CYCLES: about a second), however long each try_wait
// suspends the thread
__device__ __forceinline__ bool mbar_wait(unsigned bar, unsigned parity, long long limit = WAIT_CYCLES) {
  long long t0 = clock64();
  while (true) {
    unsigned ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    if (ok) return true;
    if (clock64() - t0 > limit) return false;
  }
}

// One thread waits on an mbarrier that nothing arrives on, with the bound the
// synthesis kernels use (or a shorter one): status = 1 when the wait gave up,
// 0 if it completed.
__global__ void wait_selftest_kernel(long long limit, int32_t* status) {
  __shared__ __align__(8) unsigned long long bar;
  if (threadIdx.x == 0) {
    mbar_init(smem_u32(&bar), 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    bool ok = mbar_wait(smem_u32(&bar), 0, limit);
    *status = ok ? 0 : 1;
  }
}
__device__ __forceinline__ void bulk_g2s(unsigned dst, const void* src, unsigned bytes, unsigned bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
               "l"(src), "r"(bytes), "r"(bar)
               : "memory");
}
// shared-memory matrix descriptor, no swizzle: start, leading byte offset (k
// direction), stride byte offset (8-row groups), version 1
__device__ __forceinline__ unsigned long long smem_desc(unsigned addr, unsigned lbo, unsigned sbo) {
  return (unsigned long long)((addr & 0x3FFFFu) >> 4) | ((unsigned long long)((lbo >> 4) & 0x3FFFu) << 16) |
         ((unsigned long long)((sbo >> 4) & 0x3FFFu) << 32) | (1ull << 46);
}
// instruction descriptor: D f32, A and B tf32, both K-major, N = TN, M = TM
constexpr unsigned IDESC = (1u << 4) | (2u << 7) | (2u << 10) | ((unsigned)(TN >> 3) << 17) | ((unsigned)(TM >> 4) << 24);

__device__ __forceinline__ void mma_tf32(unsigned tmem, unsigned long long ad, unsigned long long bd, unsigned acc) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem),
      "l"(ad), "l"(bd), "r"(IDESC), "r"(acc)
      : "memory");
}
__device__ __forceinline__ void mma_commit(unsigned bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar) : "memory");
}
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }

__device__ __forceinline__ void tmem_ld16(unsigned taddr, float* v) {
  unsigned r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
      "%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

struct gemm_args {
  const tc_group* g;
  const int* ntiles;
  const float* ytab[STIV_MAX_P + 1];
  const float* bblk;
  const tc_colinfo* ci;
  void* X;              // float (synthesis) or double (adjoint) output
  int* status;
  int p_max;
};

constexpr int NSTAGE = 3;               // shared-memory ring of (A, B) blocks
constexpr int NACC = 2;                 // TMEM accumulators (MMA of tile t+1 overlaps the epilogue of tile t)
constexpr int GEMM_THREADS = 192;       // warp 0 copies, warp 1 issues MMAs, warps 2-5 epilogue

// Tile t of this CTA's sequence: order group, row tile, column tile.
__device__ __forceinline__ bool tile_of(const tc_group* G, int p_max, int tile, int& p, int& mt, int& nt) {
  p = 1;
  while (p <= p_max && tile >= G[p].tile_off + G[p].mt * G[p].ntn) ++p;
  if (p > p_max) return false;
  int local = tile - G[p].tile_off;
  mt = local / G[p].ntn;
  nt = local % G[p].ntn;
  return true;
}

template <typename OUT>
__global__ void __launch_bounds__(GEMM_THREADS, 1) gemm_kernel(gemm_args a) {
  extern __shared__ __align__(1024) unsigned char tc_smem[];
  __shared__ tc_group G[STIV_MAX_P + 1];
  // full[NSTAGE], empty[NSTAGE], acc_full[NACC], acc_empty[NACC], drain
  __shared__ __align__(8) unsigned long long bars[2 * NSTAGE + 2 * NACC + 1];
  __shared__ unsigned tmem_base;
  int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  unsigned char* sm = (unsigned char*)(((uintptr_t)tc_smem + 1023) & ~(uintptr_t)1023);
  for (int p = tid; p <= STIV_MAX_P; p += blockDim.x) G[p] = a.g[p];
  if (tid == 0) {
    for (int b = 0; b < NSTAGE; ++b) { mbar_init(smem_u32(&bars[b]), 1); mbar_init(smem_u32(&bars[NSTAGE + b]), 1); }
    for (int b = 0; b < NACC; ++b) {
      mbar_init(smem_u32(&bars[2 * NSTAGE + b]), 1);
      mbar_init(smem_u32(&bars[2 * NSTAGE + NACC + b]), 4);   // one arrival per epilogue warp
    }
    mbar_init(smem_u32(&bars[2 * NSTAGE + 2 * NACC]), 1);     // the MMA warp's final drain
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_base)),
                 "r"((unsigned)(NACC * TN)));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  unsigned tmem = tmem_base;
  auto full = [&](int s) { return smem_u32(&bars[s]); };
  auto empty = [&](int s) { return smem_u32(&bars[NSTAGE + s]); };
  auto acc_full = [&](int b) { return smem_u32(&bars[2 * NSTAGE + b]); };
  auto acc_empty = [&](int b) { return smem_u32(&bars[2 * NSTAGE + NACC + b]); };
  const unsigned drain = smem_u32(&bars[2 * NSTAGE + 2 * NACC]);
  int ntiles = *a.ntiles;
  bool ok = true;
  if (warp == 0) {
    // producer: one lane streams the A and B blocks of every tile through the ring
    if (lane == 0) {
      unsigned it = 0;
      for (int tile = blockIdx.x; tile < ntiles && ok; tile += gridDim.x) {
        int p, mt, nt;
        if (!tile_of(G, a.p_max, tile, p, mt, nt)) break;
        int KB = G[p].kb;
        const unsigned char* asrc = (const unsigned char*)(a.ytab[p] + (size_t)mt * KB * (2 * BLK_FLOATS));
        const unsigned char* bsrc =
            (const unsigned char*)(a.bblk + ((size_t)G[p].boff + (size_t)nt * KB) * (2 * BLK_FLOATS));
        for (int kb = 0; kb < KB; ++kb, ++it) {
          int s = it % NSTAGE;
          unsigned ph = (it / NSTAGE) & 1;
          if (!mbar_wait(empty(s), ph ^ 1)) { ok = false; break; }
          unsigned char* dst = sm + (size_t)s * STAGE_BYTES;
          mbar_expect_tx(full(s), STAGE_BYTES);
          bulk_g2s(smem_u32(dst), asrc + (size_t)kb * BLK_BYTES, BLK_BYTES, full(s));
          bulk_g2s(smem_u32(dst + BLK_BYTES), bsrc + (size_t)kb * BLK_BYTES, BLK_BYTES, full(s));
        }
      }
      // before the shared memory is left: the copies of the last stages
      // issued have landed (already true unless another warp gave up early;
      // the wait is bounded either way)
      for (unsigned k = it > NSTAGE ? it - NSTAGE : 0; k < it; ++k)
        if (!mbar_wait(full(k % NSTAGE), (k / NSTAGE) & 1, DRAIN_CYCLES)) ok = false;
    }
  } else if (warp == 1) {
    // MMA issuer: one lane; accumulator b = (tile count) % NACC
    if (lane == 0) {
      unsigned it = 0, tc = 0;
      for (int tile = blockIdx.x; tile < ntiles && ok; tile += gridDim.x, ++tc) {
        int p, mt, nt;
        if (!tile_of(G, a.p_max, tile, p, mt, nt)) break;
        int KB = G[p].kb;
        int b = tc % NACC;
        if (!mbar_wait(acc_empty(b), ((tc / NACC) & 1) ^ 1)) { ok = false; break; }
        tc_fence_after();
        unsigned dtm = tmem + (unsigned)(b * TN);
        for (int kb = 0; kb < KB; ++kb, ++it) {
          int s = it % NSTAGE;
          if (!mbar_wait(full(s), (it / NSTAGE) & 1)) { ok = false; break; }
          tc_fence_after();
          unsigned abase = smem_u32(sm + (size_t)s * STAGE_BYTES), bbase = abase + BLK_BYTES;
#pragma unroll
          for (int ks = 0; ks < TK / 8; ++ks) {
            unsigned off = ks * 2 * (TM * 16);   // two k groups of 2048 bytes per K = 8
            unsigned long long ahi = smem_desc(abase + off, TM * 16, 128);
            unsigned long long alo = smem_desc(abase + BLK_BYTES / 2 + off, TM * 16, 128);
            unsigned long long bhi = smem_desc(bbase + off, TN * 16, 128);
            unsigned long long blo = smem_desc(bbase + BLK_BYTES / 2 + off, TN * 16, 128);
            mma_tf32(dtm, ahi, bhi, (kb | ks) != 0);
            mma_tf32(dtm, ahi, blo, 1u);
            mma_tf32(dtm, alo, bhi, 1u);
          }
          mma_commit(empty(s));      // the stage is free once these MMAs have read it
        }
        if (!ok) break;
        mma_commit(acc_full(b));     // accumulator b holds the finished tile
      }
      // before TMEM is freed: every MMA this thread issued has completed
      // (a gave-up wait above may have left some in flight)
      if (it > 0) {
        mma_commit(drain);
        if (!mbar_wait(drain, 0, DRAIN_CYCLES)) ok = false;
      }
    }
  } else {
    // epilogue warps 2-5: TMEM lanes 32 (w % 4) .. + 31 are tile rows
    int q = warp & 3;
    unsigned tc = 0;
    for (int tile = blockIdx.x; tile < ntiles && ok; tile += gridDim.x, ++tc) {
      int p, mt, nt;
      if (!tile_of(G, a.p_max, tile, p, mt, nt)) break;
      int b = tc % NACC;
      if (!mbar_wait(acc_full(b), (tc / NACC) & 1)) { ok = false; break; }
      tc_fence_after();
      int row = mt * TM + q * 32 + lane;
      int nrows = G[p].nrows;
      OUT* X = (OUT*)a.X;
      const tc_colinfo* cinfo = a.ci + (size_t)G[p].coff + (size_t)nt * TN;
#pragma unroll 1
      for (int c0 = 0; c0 < TN; c0 += 16) {
        float v[16];
        tmem_ld16(tmem + ((unsigned)(q * 32) << 16) + (unsigned)(b * TN + c0), v);
        tc_colinfo mine = cinfo[c0 + (lane & 15)];
#pragma unroll
        for (int i = 0; i < 16; ++i) {
          long long dst = __shfl_sync(0xffffffffu, mine.dst, i);
          float bias = __shfl_sync(0xffffffffu, mine.bias, i);
          if (dst >= 0 && row < nrows) X[dst + row] = (OUT)(v[i] + bias);
        }
      }
      tc_fence_before();
      __syncwarp();
      if (lane == 0) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(acc_empty(b)) : "memory");
    }
  }
  if (!ok) atomicOr(a.status, 1);
  tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"((unsigned)(NACC * TN)));
  }
}

}  // namespace

// Y blocks of order p for this handle (built once).
static int ensure_ytab(stiv_handle* h, cudaStream_t st, int p) {
  if (h->ytab[p]) return STIV_OK;
  int rc = stiv_ensure_tables(h, st, p);
  if (rc) return rc;
  size_t bytes = (size_t)tc_mtiles(p) * tc_kblocks(p) * BLK_BYTES;
  STIV_CUDA(h, cudaMalloc(&h->ytab[p], bytes));
  ytab_kernel<<<1024, 256, 0, st>>>(p, h->tab[p].leg, h->ytab[p]);
  STIV_LAUNCH(h);
  return STIV_OK;
}

static size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

// Device status word of the bounded waits (word 0) and the tile count of the
// synthesis (word 1) and of the adjoint (word 2); allocated once per handle.
static int ensure_status(stiv_handle* h, cudaStream_t st) {
  if (h->tc_status) return STIV_OK;
  STIV_CUDA(h, cudaMalloc(&h->tc_status, 256));
  STIV_CUDA(h, cudaMemsetAsync(h->tc_status, 0, 256, st));
  return STIV_OK;
}

// Transposed Y blocks of order p for the adjoint (built once).
static int ensure_ytabT(stiv_handle* h, cudaStream_t st, int p) {
  if (h->ytabT[p]) return STIV_OK;
  int rc = stiv_ensure_tables(h, st, p);
  if (rc) return rc;
  size_t bytes = (size_t)tcA_mtiles(p) * tcA_kblocks(p) * BLK_BYTES;
  STIV_CUDA(h, cudaMalloc(&h->ytabT[p], bytes));
  ytabT_kernel<<<1024, 256, 0, st>>>(p, h->tab[p].leg, h->ytabT[p]);
  STIV_LAUNCH(h);
  return STIV_OK;
}

int stiv_upsample_tc(stiv_handle* h, cudaStream_t st, int32_t n_ves, int32_t p_max, const int32_t* p_dev,
                     const int64_t* coef_off_dev, const double* coef_dev, const int64_t* vert_off_dev,
                     float* verts_dev) {
  for (int p = 1; p <= p_max; ++p) {
    int rc = ensure_ytab(h, st, p);
    if (rc) return rc;
  }
  // scratch bounds from n_ves and p_max only (sizes must not depend on device data)
  long long max_ntn = (6LL * n_ves + TN - 1) / TN + p_max;
  long long max_blocks = max_ntn * tc_kblocks(p_max);
  int rc0 = ensure_status(h, st);
  if (rc0) return rc0;
  size_t o_g = 0;
  size_t o_list = align256(o_g + sizeof(tc_group) * (STIV_MAX_P + 1));
  size_t o_ci = align256(o_list + sizeof(int) * (size_t)n_ves);
  size_t o_b = align256(o_ci + sizeof(tc_colinfo) * (size_t)max_ntn * TN);
  size_t total = o_b + (size_t)max_blocks * BLK_BYTES;
  if (total > h->tc_ws_bytes) {
    if (h->tc_ws) { STIV_CUDA(h, cudaFree(h->tc_ws)); h->tc_ws = nullptr; h->tc_ws_bytes = 0; }
    STIV_CUDA(h, cudaMalloc(&h->tc_ws, total));
    h->tc_ws_bytes = total;
  }
  char* w = (char*)h->tc_ws;
  int* status = h->tc_status;
  int* ntiles = status + 1;
  tc_group* g = (tc_group*)(w + o_g);
  int* list = (int*)(w + o_list);
  tc_colinfo* ci = (tc_colinfo*)(w + o_ci);
  float* bblk = (float*)(w + o_b);
  int sms = 152;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, h->device);
  STIV_PROF_N(h, st, "synth", 3);
  group_kernel<<<1, 1024, 0, st>>>(n_ves, p_max, p_dev, g, ntiles, list, 0);
  bprep_kernel<<<sms * 8, 256, 0, st>>>(p_max, g, list, coef_off_dev, coef_dev, vert_off_dev, bblk, ci);
  gemm_args A;
  A.g = g; A.ntiles = ntiles; A.bblk = bblk; A.ci = ci; A.X = verts_dev; A.status = status; A.p_max = p_max;
  for (int p = 0; p <= STIV_MAX_P; ++p) A.ytab[p] = p >= 1 && p <= p_max ? h->ytab[p] : nullptr;
  size_t smem = (size_t)NSTAGE * STAGE_BYTES + 1024;
  STIV_CUDA(h, cudaFuncSetAttribute(gemm_kernel<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  long long tiles_bound = max_ntn * tc_mtiles(p_max);
  int grid = (int)(tiles_bound < sms ? tiles_bound : sms);
  gemm_kernel<float><<<grid, GEMM_THREADS, smem, st>>>(A);
  STIV_LAUNCH(h);
  return STIV_OK;
}

// Adjoint of the mixed-form synthesis on the tensor cores: gcoef (X1 block) =
// Y^T gX (X1 block), 3xTF32 products accumulated in FP32; X0 block zero.
int stiv_grad_to_coef_tc(stiv_handle* h, cudaStream_t st, int32_t n_ves, int32_t p_max, const int32_t* p_dev,
                         const int64_t* coef_off_dev, const int64_t* vert_off_dev, const double* gX_dev,
                         double* gcoef_dev) {
  for (int p = 1; p <= p_max; ++p) {
    int rc = ensure_ytabT(h, st, p);
    if (rc) return rc;
  }
  int rc0 = ensure_status(h, st);
  if (rc0) return rc0;
  long long max_ntn = (3LL * n_ves + TN - 1) / TN + p_max;
  long long max_blocks = max_ntn * tcA_kblocks(p_max);
  size_t o_g = 0;
  size_t o_list = align256(o_g + sizeof(tc_group) * (STIV_MAX_P + 1));
  size_t o_ci = align256(o_list + sizeof(int) * (size_t)n_ves);
  size_t o_b = align256(o_ci + sizeof(tc_colinfo) * (size_t)max_ntn * TN);
  size_t total = o_b + (size_t)max_blocks * BLK_BYTES;
  if (total > h->tc_ws2_bytes) {
    if (h->tc_ws2) { STIV_CUDA(h, cudaFree(h->tc_ws2)); h->tc_ws2 = nullptr; h->tc_ws2_bytes = 0; }
    STIV_CUDA(h, cudaMalloc(&h->tc_ws2, total));
    h->tc_ws2_bytes = total;
  }
  char* w = (char*)h->tc_ws2;
  int* status = h->tc_status;
  int* ntiles = status + 2;
  tc_group* g = (tc_group*)(w + o_g);
  int* list = (int*)(w + o_list);
  tc_colinfo* ci = (tc_colinfo*)(w + o_ci);
  float* bblk = (float*)(w + o_b);
  int sms = 152;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, h->device);
  STIV_PROF_N(h, st, "grad_to_coef", 4);
  zero_x0_kernel<<<n_ves, 256, 0, st>>>(n_ves, p_max, p_dev, coef_off_dev, gcoef_dev);
  group_kernel<<<1, 1024, 0, st>>>(n_ves, p_max, p_dev, g, ntiles, list, 1);
  gprep_kernel<<<sms * 8, 256, 0, st>>>(p_max, g, list, coef_off_dev, vert_off_dev, gX_dev, bblk, ci);
  gemm_args A;
  A.g = g; A.ntiles = ntiles; A.bblk = bblk; A.ci = ci; A.X = gcoef_dev; A.status = status; A.p_max = p_max;
  for (int p = 0; p <= STIV_MAX_P; ++p) A.ytab[p] = p >= 1 && p <= p_max ? h->ytabT[p] : nullptr;
  size_t smem = (size_t)NSTAGE * STAGE_BYTES + 1024;
  STIV_CUDA(h, cudaFuncSetAttribute(gemm_kernel<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  long long tiles_bound = max_ntn * tcA_mtiles(p_max);
  int grid = (int)(tiles_bound < sms ? tiles_bound : sms);
  gemm_kernel<double><<<grid, GEMM_THREADS, smem, st>>>(A);
  STIV_LAUNCH(h);
  return STIV_OK;
}

extern "C" int stiv_wait_selftest(void* stream, int64_t limit_cycles, int32_t* status_dev) {
  if (!status_dev || limit_cycles < 0 || limit_cycles > WAIT_CYCLES) return STIV_ERR_ARG;
  wait_selftest_kernel<<<1, 32, 0, (cudaStream_t)stream>>>((long long)limit_cycles, status_dev);
  return cudaGetLastError() == cudaSuccess ? STIV_OK : STIV_ERR_CUDA;
}

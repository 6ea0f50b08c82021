// Internal declarations of libstiv (CUDA, sm_103a).
//
// Shared by the .cu files of the library only.  The arithmetic that decides
// contacts (Eq. 3.1 cubic, root isolation, inside tests) is written with
// explicit fused multiply-adds in one fixed order, and the library is built
// with -fmad=false so that the compiler adds no other contraction: the same
// inputs then give the same contact times bit for bit on every run.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>
#include <nvtx3/nvToolsExt.h>

#include "../../include/stiv.h"

#define STIV_MAX_P 32          // largest SH order accepted (mesh order 64)
#define STIV_MAX_PP 64         // largest mesh order P
#define STIV_BR 2              // patch height in grid bands
#define STIV_BC 4              // patch width in grid columns
// Floats per patch in the patch-box array (160 bytes): floats 0-5 the
// patch's swept box (lo xyz, hi xyz), 6-7 unused, then floats 8 + 8 c to
// 15 + 8 c the box of cell c as a float4 pair (lo xyz, 0; hi xyz, 0), cell
// c = 2 b + h for band b and column half h: rows I*BR + b .. + 1, columns
// J*BC + 2 h .. + 2, with the pole of that band.  Every primitive of the
// patch lies in one cell.
#define STIV_PBOX 40
#define STIV_PBOX_CELLS 8

// ---------------------------------------------------------------------------
// handle and scratch
// ---------------------------------------------------------------------------
struct stiv_tables {
  double* leg;    // [(P+3)][(p+1)(p+2)/2]  normalised Legendre (x sqrt2 for m>0) at rings + poles
  double* trig;   // [P/2+1][2][p+1]        cos(m phi_j), sin(m phi_j) for j <= P/2
  double* theta;  // [P+1]                  ring polar angles
};

struct stiv_handle {
  stiv_params prm;
  int device;
  int last_cuda_error;
  stiv_tables tab[STIV_MAX_P + 1];
  bool tab_ready[STIV_MAX_P + 1];
  // tensor-core synthesis (STIV_MIXED): synthesis-matrix blocks per order,
  // per-call scratch, and the device status word of its bounded waits
  float* ytab[STIV_MAX_P + 1];
  float* ytabT[STIV_MAX_P + 1];   // transposed blocks for the adjoint
  void* tc_ws;                    // synthesis scratch (referenced by captured graphs: never reused)
  size_t tc_ws_bytes;
  void* tc_ws2;                   // adjoint scratch
  size_t tc_ws2_bytes;
  int* tc_status;
  // contact LCP scratch (assembly, solve)
  void* lcp_ws;
  size_t lcp_ws_bytes;
  void* lcp_ws2;
  size_t lcp_ws2_bytes;
  double* fid_x;          // fine-grid nodes of the mesh-fidelity estimate
  size_t fid_x_bytes;
  // launch shapes of the narrow phase (0 = default), set by stiv_autotune
  int32_t tune[STIV_NTUNE];
  void* ws;
  size_t ws_bytes;
  // CUDA graph of stiv_step
  cudaGraphExec_t graph_exec;
  unsigned long long graph_key;
  // per-kernel CUDA-event profiler (stiv_profile); null when off
  void* prof;
};

// Brackets the launches of one named stage: an NVTX range of that name on the
// calling thread (always; without an attached tool a push/pop costs a few
// nanoseconds), and CUDA events on its stream while the profiler is on.
// nk = number of kernels the stage launches.
void stiv_prof_begin(stiv_handle* h, cudaStream_t st, const char* name, int nk);
void stiv_prof_end(stiv_handle* h, cudaStream_t st);
void stiv_prof_drop_graph(stiv_handle* h);
struct stiv_prof_scope {
  stiv_handle* h; cudaStream_t st;
  stiv_prof_scope(stiv_handle* h_, cudaStream_t st_, const char* name, int nk) : h(h_), st(st_) {
    nvtxRangePushA(name);
    stiv_prof_begin(h, st, name, nk);
  }
  ~stiv_prof_scope() {
    stiv_prof_end(h, st);
    nvtxRangePop();
  }
};
#define STIV_PROF_CAT2(a, b) a##b
#define STIV_PROF_CAT(a, b) STIV_PROF_CAT2(a, b)
#define STIV_PROF_N(h, st, name, nk) stiv_prof_scope STIV_PROF_CAT(prof_scope_, __LINE__)(h, st, name, nk)
#define STIV_PROF(h, st, name) STIV_PROF_N(h, st, name, 1)
// kernels launched by one radix sort of key_bits bits (histogram, scan, scatter per 8-bit digit)
inline int stiv_sort_kernels(int key_bits) { return 3 * ((key_bits + 7) / 8); }

// Per candidate vesicle pair, written by the narrow phase's first kernel:
// FP32 frame (offset of vesicle j's origin with its periodic image from
// vesicle i's origin, bound on the FP32 position error), the two vesicles,
// the shift code, the two mesh orders (P_i | P_j << 16), vertex offsets.
struct __align__(16) stiv_pair_info {
  float4 frame;
  int32_t vi, vj, code, Pij;
  long long voff_i, voff_j;
};

// Scratch layout used by stiv_detect (byte offsets into handle->ws).
struct detect_ws {
  double* vbox;          // [N][6]
  float* pbox;           // [N][pstride][6]
  int pstride;           // patches per vesicle at the largest order
  float* vorg;           // [N][4]  FP32 frame origin of each vesicle, and R = max |X - origin|
  float* fprep;          // [N][fstride]  per vertex 8 floats: FP32 vertices X0 (xyz, 0), X1 (xyz, 0);
                         // FP64 vertices X0 - origin (xyz, 0), X1 - X0 (xyz, 0), rounded to FP32
  int64_t fstride;
  double* grid;          // [16]  h, origin xyz, cell sizes, G
  int32_t* cell_count;   // [N+1]
  int32_t* cell_off;     // [N+1]
  uint64_t* rec_key;     // [R]
  int32_t* rec_val;      // [R]
  uint64_t* rec_key2;    // [R]
  int32_t* rec_val2;     // [R]
  int32_t* rec_box;      // [R]
  int32_t* rec_cell;     // [R] packed unwrapped cell coords
  uint64_t* pkey;        // [Q]  raw candidate keys
  int32_t* pval;         // [Q]
  uint64_t* pkey2;       // [Q]
  int32_t* pval2;        // [Q]
  uint64_t* work;        // [W]  patch-pair work items
  stiv_pair_info* pinfo; // [pair capacity]
  ulonglong2* q3;         // [Q3] primitive pairs left for the FP32 piece tests
  ulonglong2* q2;         // [Q2] primitive pairs left for the FP64 contact test
  int64_t Q3, Q2;
  int32_t* pair_cnt;     // [pair capacity]   contacts per candidate pair
  int32_t* pair_fill;    // [pair capacity]
  int32_t* pair_off;     // [pair capacity + 1]
  unsigned long long* seg;   // [C]  (type, a, b) key << 32 | raw contact index, grouped by pair
  unsigned long long* seg2;  // [C]
  int32_t* tmp_i32;      // [C] temporaries for the contact permutation
  double* tmp_f64;       // [3C]
  int64_t* ctr;          // [32] device counters
  void* sort_scratch;
  size_t sort_scratch_bytes;
  int64_t R, Q, W, C;
  int exact_only;
};

// ---------------------------------------------------------------------------
// error handling
// ---------------------------------------------------------------------------
#define STIV_CUDA(h, call)                                \
  do {                                                    \
    cudaError_t e_ = (call);                              \
    if (e_ != cudaSuccess) {                              \
      if (h) (h)->last_cuda_error = (int)e_;              \
      return STIV_ERR_CUDA;                               \
    }                                                     \
  } while (0)

#define STIV_LAUNCH(h)                                    \
  do {                                                    \
    cudaError_t e_ = cudaGetLastError();                  \
    if (e_ != cudaSuccess) {                              \
      if (h) (h)->last_cuda_error = (int)e_;              \
      return STIV_ERR_CUDA;                               \
    }                                                     \
  } while (0)

int stiv_ensure_tables(stiv_handle* h, cudaStream_t st, int p);
// STIV_MIXED synthesis on the tensor cores (3xTF32), FP32 vertices.
int stiv_upsample_tc(stiv_handle* h, cudaStream_t st, int32_t n_ves, int32_t p_max, const int32_t* p_dev,
                     const int64_t* coef_off_dev, const double* coef_dev, const int64_t* vert_off_dev,
                     float* verts_dev);
// Its adjoint (STIV_MIXED): gcoef = S^T gX on the tensor cores.
int stiv_grad_to_coef_tc(stiv_handle* h, cudaStream_t st, int32_t n_ves, int32_t p_max, const int32_t* p_dev,
                         const int64_t* coef_off_dev, const int64_t* vert_off_dev, const double* gX_dev,
                         double* gcoef_dev);
int stiv_ws_reserve(stiv_handle* h, size_t bytes);
int stiv_sort_pairs_impl(cudaStream_t st, int64_t n, int key_bits, const uint64_t* kin, const int32_t* vin,
                         uint64_t* kout, int32_t* vout, void* scratch, size_t scratch_bytes,
                         const int64_t* n_dev);
size_t stiv_sort_scratch_impl(int64_t n);

// ---------------------------------------------------------------------------
// device helpers
// ---------------------------------------------------------------------------
__host__ __device__ inline int stiv_nverts(int P) { return 2 * P * (P + 1) + 2; }
__host__ __device__ inline int stiv_ntris(int P) { return 4 * P * P + 4 * P; }
__host__ __device__ inline int stiv_nedges(int P) { return 6 * P * P + 6 * P; }
__host__ __device__ inline int stiv_ncoef(int p) { return (p + 1) * (p + 1); }
__host__ __device__ inline int stiv_nband_blocks(int P) { return (P + STIV_BR - 1) / STIV_BR; }
__host__ __device__ inline int stiv_ncol_blocks(int P) { return (2 * P + STIV_BC - 1) / STIV_BC; }
__host__ __device__ inline int stiv_npatches(int P) { return stiv_nband_blocks(P) * stiv_ncol_blocks(P); }

struct d3 { double x, y, z; };

__device__ __forceinline__ d3 d3_sub(d3 a, d3 b) { return {__dsub_rn(a.x, b.x), __dsub_rn(a.y, b.y), __dsub_rn(a.z, b.z)}; }
__device__ __forceinline__ d3 d3_add(d3 a, d3 b) { return {__dadd_rn(a.x, b.x), __dadd_rn(a.y, b.y), __dadd_rn(a.z, b.z)}; }
// cross product; each component u1 v2 - u2 v1 as fma(u1, v2, -(u2 v1))
__device__ __forceinline__ d3 d3_cross(d3 u, d3 v) {
  return {__fma_rn(u.y, v.z, -__dmul_rn(u.z, v.y)), __fma_rn(u.z, v.x, -__dmul_rn(u.x, v.z)),
          __fma_rn(u.x, v.y, -__dmul_rn(u.y, v.x))};
}
// dot product accumulated x, y, z with fused steps
__device__ __forceinline__ double d3_dot(d3 u, d3 v) {
  return __fma_rn(u.z, v.z, __fma_rn(u.y, v.y, __dmul_rn(u.x, v.x)));
}
// position at time t: X0 + t D, fused per component
__device__ __forceinline__ d3 d3_at(d3 x0, double t, d3 d) {
  return {__fma_rn(t, d.x, x0.x), __fma_rn(t, d.y, x0.y), __fma_rn(t, d.z, x0.z)};
}
__device__ __forceinline__ double horner3(double k0, double k1, double k2, double k3, double t) {
  return __fma_rn(__fma_rn(__fma_rn(k3, t, k2), t, k1), t, k0);
}

// ---------------------------------------------------------------------------
// mesh topology (Sec. 3.1.2, Fig. 3)
// ---------------------------------------------------------------------------
// Triangle t of the order-P mesh -> its 3 vertex ids.
__host__ __device__ inline void stiv_tri_verts(int P, int t, int* v) {
  int W = 2 * P, N = W * (P + 1), S = N + 1;
  if (t < 4 * P * P) {
    int q = t >> 1, i = q / W, j = q % W, jn = (j + 1 == W) ? 0 : j + 1;
    int a = i * W + j, r = (i + 1) * W + j, s = (i + 1) * W + jn, u = i * W + jn;
    if ((t & 1) == 0) { v[0] = a; v[1] = r; v[2] = s; }
    else { v[0] = a; v[1] = s; v[2] = u; }
  } else if (t < 4 * P * P + W) {
    int j = t - 4 * P * P, jn = (j + 1 == W) ? 0 : j + 1;
    v[0] = N; v[1] = j; v[2] = jn;
  } else {
    int j = t - 4 * P * P - W, jn = (j + 1 == W) ? 0 : j + 1;
    v[0] = S; v[1] = P * W + jn; v[2] = P * W + j;
  }
}

// Forward neighbours (larger ids) of grid vertex u = (i, j), in ascending id
// order; returns their count (at most 5).
__host__ __device__ inline int stiv_forward_nbrs(int P, int u, int* nb) {
  int W = 2 * P, i = u / W, j = u - i * W, n = 0;
  int pole = (i == 0) ? W * (P + 1) : (i == P) ? W * (P + 1) + 1 : -1;
  if (i < P) {
    nb[n++] = u + 1;                 // (i, j+1), or the diagonal (i+1, 0) when j = W-1
    if (j == 0) nb[n++] = u + W - 1; // (i, W-1)
    nb[n++] = u + W;                 // (i+1, j)
    if (j < W - 1) nb[n++] = u + W + 1;  // (i+1, j+1)
  } else {
    if (j < W - 1) nb[n++] = u + 1;
    if (j == 0) nb[n++] = u + W - 1;
  }
  if (pole >= 0) nb[n++] = pole;
  return n;
}

// Index of the first forward edge of grid vertex u in the sorted edge list.
__host__ __device__ inline int stiv_first_edge(int P, int u) {
  int W = 2 * P, i = u / W, j = u - i * W;
  int pole = (i == 0 || i == P) ? 1 : 0;
  int base_row = (i == 0) ? 0 : 4 * W + 3 * W * (i - 1);
  if (i < P) return base_row + ((j == 0) ? 0 : (4 + pole) + (j - 1) * (3 + pole));
  return base_row + ((j == 0) ? 0 : 3 + (j - 1) * 2);
}

// Inverse of stiv_edge_index: edge e -> (min, max) vertex ids.
__host__ __device__ inline void stiv_edge_verts(int P, int e, int* u, int* v) {
  int lo = 0, hi = 2 * P * (P + 1) - 1;  // grid vertices (poles own no forward edge)
  while (lo < hi) {
    int mid = (lo + hi + 1) >> 1;
    if (stiv_first_edge(P, mid) <= e) lo = mid; else hi = mid - 1;
  }
  int nb[5];
  int n = stiv_forward_nbrs(P, lo, nb);
  int k = e - stiv_first_edge(P, lo);
  if (k < 0) k = 0;
  if (k >= n) k = n - 1;
  *u = lo; *v = nb[k];
}

// Index of the undirected edge (u, v), u < v, in the list of all edges sorted
// by (min, max): the forward edges of all vertices before u, then the rank of
// v among u's forward neighbours.
__host__ __device__ inline int stiv_edge_index(int P, int u, int v) {
  int nb[5];
  int n = stiv_forward_nbrs(P, u, nb);
  int k = 0;
  while (k < n - 1 && nb[k] != v) ++k;
  return stiv_first_edge(P, u) + k;
}

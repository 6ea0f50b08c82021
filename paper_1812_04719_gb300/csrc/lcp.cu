// Contact LCP of a step (Sec. 3.2, Eq. 3.7; Sec. 3.3.3, Alg. 3) on one GPU.
//
//   0 <= -V + B lambda   perp   lambda >= 0,      B = J M J^T
//
// One row per contact volume: a candidate vesicle pair (with its periodic
// image) that has contacts; V its volume (the library's volumes are >= 0 for
// interference, the paper's constraint V >= 0 has the opposite sign, which B
// does not see).  J = dV/dX1 (the gradient rows of stiv_stiv_grad, summed
// per vertex); M block-diagonal, M_ii = m_i I + t_i (1 1^T (x) I_3) per
// vesicle (a local part and a rigid translation), a stand-in with the block
// structure of the locally implicit scheme's A^-1 G.
//
// Assembly (Alg. 3):
//   bounds_kernel   contact range of every candidate pair (contacts are
//                   sorted by pair)
//   rows_kernel     rows = pairs with contacts; q = -V
//   entries_kernel  one keyed entry per contact point: row | side | vertex
//                   (side 0: the pair's first vesicle, 1: its second)
//   (radix sort, stable)
//   gather_kernel   the entries' gradients in sorted order
//   tile_sums, tile_scan, compact
//                   unique (row, side, vertex) entries: the gradient of each
//                   vertex summed by a segmented scan in sorted (contact)
//                   order, fixed association (deterministic), over all rows
//                   at once
//   ves_kernel      (vesicle, row) keys -> sorted per-vesicle row lists
//   bcount_kernel   per row, the rows sharing a vesicle (union of its two
//                   vesicles' lists)
//   bcol_kernel     the columns and the row of every nonzero
//   bval_kernel     B(j, k) = sum over shared vesicles i (ascending) of
//                   m_i g_j|i . g_k|i + t_i (sum g_j|i) . (sum g_k|i), a join
//                   on the vertex ids of i; one warp per nonzero
// Solve: min-map Newton (Phi = min(lambda, B lambda + q)) in FP64, the Newton
// system on the active set by Jacobi-preconditioned conjugate gradients in
// FP32 (B_AA is symmetric positive definite), Armijo line search on
// |Phi|^2 / 2; one CTA, all iterations in one launch.
#include "stiv_internal.cuh"

#include <math.h>

namespace {

constexpr int RT = 1024;   // threads of the single-CTA kernels

__device__ __forceinline__ int64_t ncontacts(const int64_t* counts, int64_t cap) {
  int64_t n = counts[STIV_C_VF] + counts[STIV_C_EE];
  return n < cap ? n : cap;
}

__global__ void bounds_kernel(const int64_t* counts, int64_t ccap, const int32_t* pair, int32_t* pstart,
                              int32_t* pend) {
  int64_t n = ncontacts(counts, ccap);
  for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x) {
    int p = pair[k];
    if (k == 0 || pair[k - 1] != p) pstart[p] = (int32_t)k;
    if (k == n - 1 || pair[k + 1] != p) pend[p] = (int32_t)(k + 1);
  }
}

// Block-wide exclusive scan helper (RT threads).
__device__ int block_scan(int v, int* sh, int& total) {
  sh[threadIdx.x] = v;
  __syncthreads();
  for (int off = 1; off < RT; off <<= 1) {
    int t = threadIdx.x >= off ? sh[threadIdx.x - off] : 0;
    __syncthreads();
    sh[threadIdx.x] += t;
    __syncthreads();
  }
  total = sh[RT - 1];
  int ex = sh[threadIdx.x] - v;
  __syncthreads();
  return ex;
}

// dims: [0] rows, [1] nnz, [2] status (1: rows over capacity, 2: nonzeros
// over capacity), [3] entries (4 x contacts), [4] 2 x rows
__global__ void __launch_bounds__(RT) rows_kernel(const int64_t* counts, int64_t pcap, int64_t ccap,
                                                  const int32_t* pstart, const int32_t* pend, const double* Vp,
                                                  int64_t rcap, int32_t* row_pair, int32_t* row_of_pair, double* q,
                                                  int64_t* dims) {
  __shared__ int sh[RT];
  int64_t np = counts[STIV_C_PAIRS] < pcap ? counts[STIV_C_PAIRS] : pcap;
  int base = 0;
  for (int64_t p0 = 0; p0 < np; p0 += RT) {
    int64_t p = p0 + threadIdx.x;
    int has = (p < np && pend[p] > pstart[p]) ? 1 : 0;
    int tot;
    int ex = block_scan(has, sh, tot);
    if (p < np) {
      int r = has ? base + ex : -1;
      row_of_pair[p] = r;
      if (has && r < rcap) {
        row_pair[r] = (int32_t)p;
        q[r] = -Vp[p];
      }
    }
    base += tot;
  }
  if (threadIdx.x == 0) {
    dims[0] = base < rcap ? base : rcap;
    dims[2] = base > rcap ? 1 : 0;
    dims[3] = 4 * ncontacts(counts, ccap);
    dims[4] = 2 * dims[0];
  }
}

__global__ void entries_kernel(const int64_t* counts, int64_t ccap, const int32_t* pair, const int32_t* row_of_pair,
                               const int32_t* ci, const int32_t* gves, const int32_t* gvid, int64_t rcap, int db,
                               uint64_t* key, int32_t* val) {
  int64_t n = ncontacts(counts, ccap);
  for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x) {
    int p = pair[k];
    int r = row_of_pair[p];
    uint64_t rr = (r >= 0 && r < rcap) ? (uint64_t)r : (uint64_t)rcap;   // beyond capacity: sorted last
    int vi = ci[p];
    for (int q = 0; q < 4; ++q) {
      uint64_t side = gves[4 * k + q] == vi ? 0u : 1u;
      key[4 * k + q] = (rr << (1 + db)) | (side << db) | (uint64_t)gvid[4 * k + q];
      val[4 * k + q] = (int32_t)(4 * k + q);
    }
  }
}

constexpr int ET = 256;        // threads of the compaction CTAs
constexpr int EI = 8;          // consecutive entries per thread
constexpr int ETILE = ET * EI;

// Gradients of the sorted entries, gathered into sorted order (one
// independent gather per entry), so that the runs summed next are contiguous.
__global__ void gather_kernel(const int64_t* n_dev, const int32_t* sval, const double* grad, double* gs) {
  int64_t n = *n_dev;
  for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < n; j += (int64_t)gridDim.x * blockDim.x) {
    const double* g = grad + 3 * (size_t)sval[j];
    double a = g[0], b = g[1], c = g[2];
    gs[3 * j] = a; gs[3 * j + 1] = b; gs[3 * j + 2] = c;
  }
}

// Exclusive scan over an ET-thread CTA in a fixed order; *total = the sum.
__device__ __forceinline__ int cta_scan(int v, int* wsum, int* total) {
  int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  int x = v;
  for (int off = 1; off < 32; off <<= 1) {
    int y = __shfl_up_sync(0xffffffffu, x, off);
    if (lane >= off) x += y;
  }
  if (lane == 31) wsum[w] = x;
  __syncthreads();
  int pre = 0, tot = 0;
  for (int q = 0; q < ET / 32; ++q) { int s = wsum[q]; pre += q < w ? s : 0; tot += s; }
  __syncthreads();
  *total = tot;
  return pre + x - v;
}

__device__ __forceinline__ bool is_head(const uint64_t* skey, int64_t j, int64_t n) {
  return j < n && (j == 0 || skey[j] != skey[j - 1]);
}

// Segmented sums: (f, v) pairs combined left to right by
// (f1, v1) + (f2, v2) = (f1 | f2, f2 ? v2 : v1 + v2), f = "a run starts here".
// Runs (one vertex of one row) can hold thousands of entries, so they are
// summed by a segmented scan over all sorted entries rather than by the
// run's first entry: per thread over its EI entries, then over the CTA
// (warp shuffles, then warps in order), then over the tiles.  The order of
// the additions is fixed, so the sums are deterministic.
struct seg3 {
  int f;
  double a, b, c;
};
__device__ __forceinline__ seg3 seg_add(const seg3& x, const seg3& y) {
  seg3 r;
  r.f = x.f | y.f;
  r.a = y.f ? y.a : x.a + y.a;
  r.b = y.f ? y.b : x.b + y.b;
  r.c = y.f ? y.c : x.c + y.c;
  return r;
}

// Exclusive segmented scan over the ET-thread CTA; *total = the CTA's sum.
__device__ seg3 cta_seg_scan(seg3 v, seg3* wagg, seg3* total) {
  int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  seg3 s = v;
  for (int off = 1; off < 32; off <<= 1) {
    seg3 o;
    o.f = __shfl_up_sync(0xffffffffu, s.f, off);
    o.a = __shfl_up_sync(0xffffffffu, s.a, off);
    o.b = __shfl_up_sync(0xffffffffu, s.b, off);
    o.c = __shfl_up_sync(0xffffffffu, s.c, off);
    if (lane >= off) s = seg_add(o, s);
  }
  seg3 ex;   // within the warp: the inclusive value of the previous lane
  ex.f = __shfl_up_sync(0xffffffffu, s.f, 1);
  ex.a = __shfl_up_sync(0xffffffffu, s.a, 1);
  ex.b = __shfl_up_sync(0xffffffffu, s.b, 1);
  ex.c = __shfl_up_sync(0xffffffffu, s.c, 1);
  if (lane == 0) ex = seg3{0, 0.0, 0.0, 0.0};
  if (lane == 31) wagg[w] = s;
  __syncthreads();
  seg3 pre{0, 0.0, 0.0, 0.0}, tot{0, 0.0, 0.0, 0.0};
  for (int q = 0; q < ET / 32; ++q) {
    if (q < w) pre = seg_add(pre, wagg[q]);
    tot = seg_add(tot, wagg[q]);
  }
  __syncthreads();
  *total = tot;
  return seg_add(pre, ex);
}

// This thread's EI entries as one segmented value: whether a run starts in
// them, and the sum of the entries after the last start (or of all of them).
__device__ __forceinline__ seg3 thread_seg(const uint64_t* skey, const double* gs, int64_t base, int64_t n,
                                           unsigned& hd) {
  seg3 s{0, 0.0, 0.0, 0.0};
  hd = 0;
  for (int k = 0; k < EI; ++k) {
    int64_t j = base + k;
    if (j >= n) break;
    if (is_head(skey, j, n)) { hd |= 1u << k; s.f = 1; s.a = gs[3 * j]; s.b = gs[3 * j + 1]; s.c = gs[3 * j + 2]; }
    else { s.a += gs[3 * j]; s.b += gs[3 * j + 1]; s.c += gs[3 * j + 2]; }
  }
  return s;
}

// The unique (row, side, vertex) entries are compacted over all sorted
// entries at once (rows differ widely in size): per tile the heads of runs
// and the segmented sum, the tiles scanned, then every run's last entry
// writes the run's sum.
__global__ void __launch_bounds__(ET) tile_sums_kernel(const int64_t* n_dev, const uint64_t* skey, const double* gs,
                                                       int32_t* tcount, seg3* tagg) {
  __shared__ int wsum[ET / 32];
  __shared__ seg3 wagg[ET / 32];
  int64_t n = *n_dev;
  if ((int64_t)blockIdx.x * ETILE >= n) return;   // past the entries: not read by the scan
  int64_t base = (int64_t)blockIdx.x * ETILE + (int64_t)threadIdx.x * EI;
  unsigned hd;
  seg3 v = thread_seg(skey, gs, base, n, hd);
  int tot;
  cta_scan(__popc(hd), wsum, &tot);
  seg3 st;
  cta_seg_scan(v, wagg, &st);
  if (threadIdx.x == 0) { tcount[blockIdx.x] = tot; tagg[blockIdx.x] = st; }
}

// One CTA: exclusive scan of the tile head counts in place, and the
// segmented sum flowing into each tile from the tiles before it (tcarry).
// Without rows beyond capacity the head total closes the last row's range:
// ustart[rows] = total.
__global__ void __launch_bounds__(ET) tile_scan_kernel(int ntiles, int32_t* tcount, const seg3* tagg, seg3* tcarry,
                                                       const int64_t* dims, int32_t* ustart) {
  __shared__ int wsum[ET / 32];
  __shared__ seg3 wagg[ET / 32];
  int64_t used = (dims[3] + ETILE - 1) / ETILE;   // tiles holding entries
  if (used < ntiles) ntiles = (int)used;
  int carry = 0;
  seg3 scarry{0, 0.0, 0.0, 0.0};
  for (int b = 0; b < ntiles; b += ET) {
    int i = b + threadIdx.x;
    int v = i < ntiles ? tcount[i] : 0, tot;
    int ex = cta_scan(v, wsum, &tot);
    seg3 sv = i < ntiles ? tagg[i] : seg3{0, 0.0, 0.0, 0.0}, stot;
    seg3 sex = cta_seg_scan(sv, wagg, &stot);
    if (i < ntiles) { tcount[i] = carry + ex; tcarry[i] = seg_add(scarry, sex); }
    carry += tot;
    scarry = seg_add(scarry, stot);
  }
  if (threadIdx.x == 0 && !(dims[2] & 1)) ustart[dims[0]] = carry;
}

// Heads write their unique entry's key (the first head of a row where the
// row's unique entries start, the first head of a row's side 1 where those
// start; rows beyond capacity share the row field rcap and close the last
// row's range); the last entry of each run writes the run's sum.
__global__ void __launch_bounds__(ET) compact_kernel(const int64_t* n_dev, const uint64_t* skey, const double* gs,
                                                     const int32_t* toff, const seg3* tcarry, int rshift,
                                                     uint64_t kmask, uint64_t* ukey, double* ug, int32_t* ustart,
                                                     int32_t* uside) {
  __shared__ int wsum[ET / 32];
  __shared__ seg3 wagg[ET / 32];
  int64_t n = *n_dev;
  if ((int64_t)blockIdx.x * ETILE >= n) return;
  int64_t base = (int64_t)blockIdx.x * ETILE + (int64_t)threadIdx.x * EI;
  unsigned hd;
  seg3 v = thread_seg(skey, gs, base, n, hd);
  int tot;
  int u = toff[blockIdx.x] + cta_scan(__popc(hd), wsum, &tot) - 1;   // unique index of the open run
  seg3 st;
  seg3 run = seg_add(tcarry[blockIdx.x], cta_seg_scan(v, wagg, &st));   // open run's sum so far
  for (int k = 0; k < EI; ++k) {
    int64_t j = base + k;
    if (j >= n) break;
    if (hd >> k & 1u) {
      ++u;
      run.a = gs[3 * j]; run.b = gs[3 * j + 1]; run.c = gs[3 * j + 2];
      uint64_t key = skey[j];
      ukey[u] = key & kmask;
      uint64_t row = key >> rshift;
      if (j == 0 || (skey[j - 1] >> rshift) != row) ustart[row] = u;
      if ((key >> (rshift - 1) & 1u) && (j == 0 || (skey[j - 1] >> (rshift - 1)) != (key >> (rshift - 1))))
        uside[row] = u;   // first entry of the row's side 1
    } else {
      run.a += gs[3 * j]; run.b += gs[3 * j + 1]; run.c += gs[3 * j + 2];
    }
    if (j + 1 == n || skey[j + 1] != skey[j]) {
      ug[3 * (size_t)u] = run.a; ug[3 * (size_t)u + 1] = run.b; ug[3 * (size_t)u + 2] = run.c;
    }
  }
}

__global__ void ves_kernel(const int64_t* dims, const int32_t* row_pair, const int32_t* ci, const int32_t* cj, int rb,
                           uint64_t* key, int32_t* val) {
  int64_t n = dims[0];
  for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < n; r += (int64_t)gridDim.x * blockDim.x) {
    int p = row_pair[r];
    key[2 * r] = ((uint64_t)ci[p] << rb) | (uint64_t)r;
    key[2 * r + 1] = ((uint64_t)cj[p] << rb) | (uint64_t)r;
    val[2 * r] = (int32_t)r; val[2 * r + 1] = (int32_t)r;
  }
}

__global__ void ves_bounds_kernel(const int64_t* dims, const uint64_t* key, int rb, int32_t* vstart, int32_t* vend) {
  int64_t n = 2 * dims[0];
  for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x) {
    uint64_t v = key[k] >> rb;
    if (k == 0 || (key[k - 1] >> rb) != v) vstart[v] = (int32_t)k;
    if (k == n - 1 || (key[k + 1] >> rb) != v) vend[v] = (int32_t)(k + 1);
  }
}

// Rows sharing a vesicle with row r, ascending, without repeats: a merge of
// the sorted row lists of its two vesicles.  f(s) is called for each, in order.
template <class F>
__device__ void for_neighbours(const int32_t* lst, int a0, int a1, int b0, int b1, F f) {
  int i = a0, j = b0, last = -1;
  while (i < a1 || j < b1) {
    int s;
    if (j >= b1 || (i < a1 && lst[i] <= lst[j])) s = lst[i++];
    else s = lst[j++];
    if (s != last) { f(s); last = s; }
  }
}

__global__ void bcount_kernel(const int64_t* dims, const int32_t* row_pair, const int32_t* ci, const int32_t* cj,
                              const int32_t* vrow, const int32_t* vstart, const int32_t* vend, int32_t* bcnt) {
  int64_t n = dims[0];
  for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < n; r += (int64_t)gridDim.x * blockDim.x) {
    int p = row_pair[r], vi = ci[p], vj = cj[p];
    int c = 0;
    for_neighbours(vrow, vstart[vi], vend[vi], vstart[vj], vend[vj], [&](int) { ++c; });
    bcnt[r] = c;
  }
}

__global__ void __launch_bounds__(RT) bscan_kernel(int64_t* dims, const int32_t* bcnt, int64_t nnz_cap,
                                                   int64_t* row_ptr) {
  __shared__ int sh[RT];
  int64_t n = dims[0];
  int64_t base = 0;
  for (int64_t r0 = 0; r0 < n; r0 += RT) {
    int64_t r = r0 + threadIdx.x;
    int c = r < n ? bcnt[r] : 0;
    int tot;
    int ex = block_scan(c, sh, tot);
    if (r < n) row_ptr[r] = base + ex;
    base += tot;
  }
  if (threadIdx.x == 0) {
    row_ptr[n] = base;
    dims[1] = base;
    if (base > nnz_cap) dims[2] |= 2;
  }
}

// Entries of row x on one side of its pair (0: first vesicle, 1: second):
// [ustart[x], mid) and [mid, ustart[x + 1]), mid = where side 1 starts
// (uside[x], -1 when the row has no side-1 entry).
__device__ __forceinline__ void side_range(const int32_t* ustart, const int32_t* uside, int64_t x, int side,
                                           int64_t& lo, int64_t& hi) {
  int64_t b = ustart[x], e = ustart[x + 1], m = uside[x] >= 0 ? uside[x] : e;
  lo = side ? m : b;
  hi = side ? e : m;
}

// Columns of B (thread per row): the rows sharing a vesicle with row r,
// ascending, and the row of every nonzero.
__global__ void bcol_kernel(const int64_t* dims, const int32_t* row_pair, const int32_t* ci, const int32_t* cj,
                            const int32_t* vrow, const int32_t* vstart, const int32_t* vend, const int64_t* row_ptr,
                            int64_t nnz_cap, int32_t* col, int32_t* nzrow) {
  int64_t n = dims[0];
  for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < n; r += (int64_t)gridDim.x * blockDim.x) {
    int p = row_pair[r], vi = ci[p], vj = cj[p];
    int64_t o = row_ptr[r];
    for_neighbours(vrow, vstart[vi], vend[vi], vstart[vj], vend[vj], [&](int s) {
      if (o < nnz_cap) { col[o] = s; nzrow[o] = (int32_t)r; }
      ++o;
    });
  }
}

// One warp per nonzero: B(r, s) = sum over the vesicles v common to rows r
// and s (ascending) of m_v g_r|v . g_s|v + t_v (sum g_r|v) . (sum g_s|v).
// The dot product over v's vertices is a join on the vertex id: row B's
// entries (B = max(r, s)) are scattered into the warp's vertex-index table in
// shared memory (nvtab slots, -1 = absent, reset after use) and the lanes,
// over row A's entries (A = min(r, s)), look their vertex up (on the diagonal
// every entry is its own match).  Sums are reduced in a fixed order and
// depend on (A, B) only, so that B(r, s) and B(s, r) are the same sum: B is
// symmetric bit for bit.
__global__ void bval_kernel(const int64_t* dims, const int32_t* row_pair, const int32_t* ci, const int32_t* cj,
                            const int32_t* ustart, const int32_t* uside, const uint64_t* ukey, const double* ug,
                            const double* m_ves, const double* t_ves, int db, int nvtab, int64_t nnz_cap,
                            const int32_t* col, const int32_t* nzrow, double* val) {
  extern __shared__ int32_t vtab_all[];
  int lane = threadIdx.x & 31;
  int32_t* tab = vtab_all + (size_t)(threadIdx.x >> 5) * nvtab;
  for (int i = lane; i < nvtab; i += 32) tab[i] = -1;
  __syncwarp();
  uint64_t dmask = (1ull << db) - 1;
  int64_t nnz = dims[1] < nnz_cap ? dims[1] : nnz_cap;
  int64_t w0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5, nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t k = w0; k < nnz; k += nw) {
    int r = nzrow[k], s = col[k];
    int p = row_pair[r], vi = ci[p], vj = cj[p];
    int ps = row_pair[s], si = ci[ps], sj = cj[ps];
    int64_t rA = s < r ? s : r, rB = s < r ? r : s;
    int aI = s < r ? si : vi, bI = s < r ? vi : si;   // first vesicles of rows A and B
    double acc = 0.0;
    for (int t = 0; t < 2; ++t) {
      int v = t ? vj : vi;   // vi < vj: ascending
      if (v != si && v != sj) continue;
      int64_t a0, a1, b0, b1;
      side_range(ustart, uside, rA, v == aI ? 0 : 1, a0, a1);
      side_range(ustart, uside, rB, v == bI ? 0 : 1, b0, b1);
      double part = 0.0, sa[3] = {0.0, 0.0, 0.0}, sb[3] = {0.0, 0.0, 0.0};
      if (rA == rB) {
#pragma unroll 4
        for (int64_t i = a0 + lane; i < a1; i += 32) {
          double x = ug[3 * i], y = ug[3 * i + 1], z = ug[3 * i + 2];
          part += x * x + y * y + z * z;
          sa[0] += x; sa[1] += y; sa[2] += z;
        }
      } else {
#pragma unroll 4
        for (int64_t i = b0 + lane; i < b1; i += 32) {
          tab[ukey[i] & dmask] = (int32_t)(i - b0);
          for (int d = 0; d < 3; ++d) sb[d] += ug[3 * i + d];
        }
        __syncwarp();
#pragma unroll 4
        for (int64_t i = a0 + lane; i < a1; i += 32) {
          int32_t jb = tab[ukey[i] & dmask];   // vertex id (the sides may differ)
          if (jb >= 0) {
            int64_t lo = b0 + jb;
            part += ug[3 * i] * ug[3 * lo] + ug[3 * i + 1] * ug[3 * lo + 1] + ug[3 * i + 2] * ug[3 * lo + 2];
          }
          for (int d = 0; d < 3; ++d) sa[d] += ug[3 * i + d];
        }
        __syncwarp();
        for (int64_t i = b0 + lane; i < b1; i += 32) tab[ukey[i] & dmask] = -1;
        __syncwarp();
      }
      for (int off = 16; off > 0; off >>= 1) part += __shfl_xor_sync(0xffffffffu, part, off);
      acc += (m_ves ? m_ves[v] : 1.0) * part;
      if (t_ves) {   // rigid translation: (sum of g_A over v's points) . (sum of g_B)
        for (int off = 16; off > 0; off >>= 1)
          for (int d = 0; d < 3; ++d) {
            sa[d] += __shfl_xor_sync(0xffffffffu, sa[d], off);
            sb[d] += __shfl_xor_sync(0xffffffffu, sb[d], off);
          }
        bool dg = rA == rB;
        double b0s = dg ? sa[0] : sb[0], b1s = dg ? sa[1] : sb[1], b2s = dg ? sa[2] : sb[2];
        acc += t_ves[v] * (sa[0] * b0s + sa[1] * b1s + sa[2] * b2s);
      }
    }
    if (lane == 0) val[k] = acc;
  }
}

// ---------------------------------------------------------------------------
// min-map Newton, one CTA
// ---------------------------------------------------------------------------
// The solve runs on one SM, and GB300's FP64 pipe is narrow (about two FP64
// FMAs per clock per SM), so it is an inexact Newton method: the outer loop
// (Phi, the merit, the Armijo line search, the right-hand side of the Newton
// system and the free part of the direction, dx_F = -x_F) is FP64, and the
// Newton system on the active set is solved by a Jacobi-preconditioned CG in
// FP32 (B rounded to FP32) to a relative residual of 1e-6.  Convergence is
// decided by the FP64 residual max |Phi| <= tol.
struct solve_args {
  const int64_t* dims;
  const int64_t* row_ptr;
  const int32_t* col;
  const double* val;
  float* valf;    // B's values in FP32
  const double* q;
  double* x;      // lambda
  double* w;      // B x
  double* dx;     // Newton direction
  double* xn;
  float* y;       // CG iterate: dx on the active set
  float* r;
  float* pv;
  float* Ap;
  float* dinv;    // 1 / B_ii (Jacobi preconditioner)
  unsigned char* act;
  double tol;
  int max_newton, max_cg;
  double* info;   // [0] Newton iterations, [1] max |Phi|, [2] CG iterations, [3] status
};

// Block reductions in a fixed order: butterfly within each warp, then warp 0
// over the RT / 32 partial results.  sh holds >= 2 * (RT / 32) + 2 values.
template <class T>
__device__ void block_sum2(T& a, T& b, T* sh) {
  for (int off = 16; off > 0; off >>= 1) {
    a += __shfl_xor_sync(0xffffffffu, a, off);
    b += __shfl_xor_sync(0xffffffffu, b, off);
  }
  int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (lane == 0) { sh[w] = a; sh[RT / 32 + w] = b; }
  __syncthreads();
  if (w == 0) {
    a = sh[lane]; b = sh[RT / 32 + lane];
    for (int off = 16; off > 0; off >>= 1) {
      a += __shfl_xor_sync(0xffffffffu, a, off);
      b += __shfl_xor_sync(0xffffffffu, b, off);
    }
    if (lane == 0) { sh[2 * (RT / 32)] = a; sh[2 * (RT / 32) + 1] = b; }
  }
  __syncthreads();
  a = sh[2 * (RT / 32)]; b = sh[2 * (RT / 32) + 1];
  __syncthreads();
}
__device__ double block_max(double v, double* sh) {
  for (int off = 16; off > 0; off >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, off));
  int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (lane == 0) sh[w] = v;
  __syncthreads();
  if (w == 0) {
    v = sh[lane];
    for (int off = 16; off > 0; off >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, off));
    if (lane == 0) sh[RT / 32] = v;
  }
  __syncthreads();
  double r = sh[RT / 32];
  __syncthreads();
  return r;
}

// psi = |Phi(x)|^2 / 2 with Phi = min(x, B x + q), y = B x (FP64); res = max |Phi|
__device__ double merit(const solve_args& a, int64_t n, const double* x, double* y, double* sh, double& res) {
  double s = 0.0, m = 0.0;
  for (int64_t i = threadIdx.x; i < n; i += RT) {
    double t = 0.0;
    for (int64_t k = a.row_ptr[i]; k < a.row_ptr[i + 1]; ++k) t += a.val[k] * x[a.col[k]];
    y[i] = t;
    double ph = fmin(x[i], t + a.q[i]);
    s += ph * ph;
    m = fmax(m, fabs(ph));
  }
  res = block_max(m, sh);
  double z = 0.0;
  block_sum2(s, z, sh);
  return 0.5 * s;
}

// Ap = B_AA pv on the active set (FP32), 0 elsewhere; returns pv . Ap
__device__ float spmv_active(const solve_args& a, int64_t n, float* shf) {
  float d = 0.0f, z = 0.0f;
  for (int64_t i = threadIdx.x; i < n; i += RT) {
    float t = 0.0f;
    if (a.act[i]) {
      for (int64_t k = a.row_ptr[i]; k < a.row_ptr[i + 1]; ++k) {
        int j = a.col[k];
        if (a.act[j]) t += a.valf[k] * a.pv[j];
      }
      d += a.pv[i] * t;
    }
    a.Ap[i] = t;
  }
  block_sum2(d, z, shf);
  return d;
}

constexpr size_t SOLVE_SMEM = 220 * 1024;   // dynamic shared memory of the solve CTA

__device__ __forceinline__ size_t al16(size_t x) { return (x + 15) & ~(size_t)15; }

// When the vectors, q and B (FP64 and FP32 values) fit in the CTA's shared
// memory (smem_bytes) they are staged there and every iteration runs out of
// it; otherwise the handle's global scratch holds them.
__global__ void __launch_bounds__(RT) solve_kernel(solve_args g, size_t smem_bytes) {
  extern __shared__ __align__(16) unsigned char dsm[];
  __shared__ double sh[2 * (RT / 32) + 2];
  __shared__ float shf[2 * (RT / 32) + 2];
  solve_args a = g;
  int64_t n = g.dims[0], nnz = g.dims[1];
  if (g.dims[2]) {   // matrix over capacity
    if (threadIdx.x == 0) { g.info[0] = 0; g.info[1] = -1; g.info[2] = 0; g.info[3] = 1; }
    return;
  }
  size_t need = 4 * al16(8 * (size_t)n) + 5 * al16(4 * (size_t)n) + al16((size_t)n) + al16(8 * (size_t)(n + 1)) +
                al16(4 * (size_t)nnz) + al16(8 * (size_t)nnz) + al16(4 * (size_t)nnz) + al16(8 * (size_t)n);
  bool in_smem = need <= smem_bytes;
  if (in_smem) {
    unsigned char* p = dsm;
    auto take = [&](size_t bytes) { unsigned char* r = p; p += al16(bytes); return r; };
    a.x = (double*)take(8 * n); a.w = (double*)take(8 * n); a.dx = (double*)take(8 * n);
    a.xn = (double*)take(8 * n);
    a.y = (float*)take(4 * n); a.r = (float*)take(4 * n); a.pv = (float*)take(4 * n);
    a.Ap = (float*)take(4 * n); a.dinv = (float*)take(4 * n);
    a.act = take(n);
    double* qs = (double*)take(8 * n);
    int64_t* rp = (int64_t*)take(8 * (n + 1));
    int32_t* cs = (int32_t*)take(4 * nnz);
    double* vs = (double*)take(8 * nnz);
    a.valf = (float*)take(4 * nnz);
    for (int64_t i = threadIdx.x; i <= n; i += RT) rp[i] = g.row_ptr[i];
    for (int64_t k = threadIdx.x; k < nnz; k += RT) { cs[k] = g.col[k]; vs[k] = g.val[k]; }
    for (int64_t i = threadIdx.x; i < n; i += RT) qs[i] = g.q[i];
    a.row_ptr = rp; a.col = cs; a.val = vs; a.q = qs;
    __syncthreads();
  }
  for (int64_t k = threadIdx.x; k < nnz; k += RT) a.valf[k] = (float)a.val[k];
  for (int64_t i = threadIdx.x; i < n; i += RT) {
    a.x[i] = 0.0;
    double d = 0.0;
    for (int64_t k = a.row_ptr[i]; k < a.row_ptr[i + 1]; ++k)
      if (a.col[k] == i) d = a.val[k];
    a.dinv[i] = d > 0.0 ? (float)(1.0 / d) : 1.0f;
  }
  __syncthreads();
  long long cg_total = 0;
  int it = 0;
  double res = 0.0;
  double psi = merit(a, n, a.x, a.w, sh, res);   // w = B x
  for (it = 0;; ++it) {
    if (res <= a.tol || it == a.max_newton) break;
    // active set; dx_F = -x_F
    for (int64_t i = threadIdx.x; i < n; i += RT) {
      bool ac = a.w[i] + a.q[i] < a.x[i];
      a.act[i] = ac;
      a.dx[i] = ac ? 0.0 : -a.x[i];
    }
    __syncthreads();
    // rhs_A = -(B x + q)_A - B_{A,F} dx_F (FP64, then FP32); PCG from y = 0
    float rz = 0.0f, rr = 0.0f;
    for (int64_t i = threadIdx.x; i < n; i += RT) {
      float ri = 0.0f;
      if (a.act[i]) {
        double s = 0.0;
        for (int64_t k = a.row_ptr[i]; k < a.row_ptr[i + 1]; ++k) {
          int j = a.col[k];
          if (!a.act[j]) s += a.val[k] * a.dx[j];
        }
        ri = (float)(-(a.w[i] + a.q[i]) - s);
      }
      a.r[i] = ri;
      a.y[i] = 0.0f;
      float z = ri * a.dinv[i];
      a.pv[i] = z;
      rz += ri * z; rr += ri * ri;
    }
    block_sum2(rz, rr, shf);
    float rr0 = rr;
    for (int k = 0; k < a.max_cg && rr > 1e-12f * rr0 && rr > 0.0f; ++k) {
      float pAp = spmv_active(a, n, shf);
      if (!(pAp > 0.0f)) break;
      float al = rz / pAp, rzn = 0.0f, rn = 0.0f;
      for (int64_t i = threadIdx.x; i < n; i += RT)
        if (a.act[i]) {
          a.y[i] += al * a.pv[i];
          float ri = a.r[i] - al * a.Ap[i];
          a.r[i] = ri;
          rzn += ri * ri * a.dinv[i];
          rn += ri * ri;
        }
      block_sum2(rzn, rn, shf);
      float be = rzn / rz;
      for (int64_t i = threadIdx.x; i < n; i += RT) a.pv[i] = a.act[i] ? a.r[i] * a.dinv[i] + be * a.pv[i] : 0.0f;
      __syncthreads();
      rz = rzn; rr = rn;
      ++cg_total;
    }
    for (int64_t i = threadIdx.x; i < n; i += RT)
      if (a.act[i]) a.dx[i] = (double)a.y[i];
    __syncthreads();
    // Armijo line search on psi along x + t dx (FP64); w = B xn of the accepted step
    double t = 1.0, pn = psi, rn = res;
    for (int h = 0; h < 40; ++h) {
      for (int64_t i = threadIdx.x; i < n; i += RT) a.xn[i] = a.x[i] + t * a.dx[i];
      __syncthreads();
      pn = merit(a, n, a.xn, a.w, sh, rn);
      if (pn <= (1.0 - 2.0e-4 * t) * psi) break;
      t *= 0.5;
    }
    for (int64_t i = threadIdx.x; i < n; i += RT) a.x[i] = a.xn[i];
    __syncthreads();
    psi = pn; res = rn;
  }
  if (in_smem)
    for (int64_t i = threadIdx.x; i < n; i += RT) g.x[i] = a.x[i];
  if (threadIdx.x == 0) { g.info[0] = it; g.info[1] = res; g.info[2] = (double)cg_total; g.info[3] = res <= a.tol ? 0 : 2; }
}

int nbits(int64_t x) {   // bits to hold 0 .. x
  int b = 1;
  while (b < 62 && ((int64_t)1 << b) <= x) ++b;
  return b;
}

size_t al256(size_t x) { return (x + 255) & ~(size_t)255; }

}  // namespace

extern "C" int stiv_lcp_matrix(stiv_handle* h, void* stream, int32_t n_ves, int32_t p_max, const stiv_pairs* cand,
                               const stiv_contacts* ct, const int64_t* counts_dev, const double* V_pair_dev,
                               const double* grad_dev, const int32_t* g_ves_dev, const int32_t* g_vid_dev,
                               const double* m_ves_dev, const double* t_ves_dev, const stiv_lcp* lcp) {
  if (!h || !cand || !ct || !counts_dev || !V_pair_dev || !grad_dev || !g_ves_dev || !g_vid_dev || !lcp)
    return STIV_ERR_ARG;
  if (n_ves < 1 || p_max < 1 || p_max > STIV_MAX_P || lcp->row_capacity < 1 || lcp->nnz_capacity < 1 ||
      lcp->row_capacity >= ((int64_t)1 << 30) || !lcp->row_pair || !lcp->q || !lcp->row_ptr || !lcp->col ||
      !lcp->val || !lcp->dims || !cand->i || !cand->j || !ct->pair)
    return STIV_ERR_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  int64_t pcap = cand->capacity, ccap = ct->capacity, rcap = lcp->row_capacity;
  int rb = nbits(rcap), vb = nbits(n_ves), db = nbits(stiv_nverts(2 * p_max));
  if (rb + 1 + db > 63 || vb + rb > 63) return STIV_ERR_ARG;
  int64_t E = 4 * ccap, R2 = 2 * rcap;
  int64_t smax = E > R2 ? E : R2;
  // scratch (handle-owned, grown on demand)
  size_t o = 0;
  size_t o_ps = o; o = al256(o + sizeof(int32_t) * pcap);
  size_t o_pe = o; o = al256(o + sizeof(int32_t) * pcap);
  size_t o_rp = o; o = al256(o + sizeof(int32_t) * pcap);
  int64_t etiles = (E + ETILE - 1) / ETILE;
  if (etiles < 1) etiles = 1;
  if (E >= ((int64_t)1 << 31)) return STIV_ERR_ARG;
  size_t o_us = o; o = al256(o + sizeof(int32_t) * (rcap + 1));
  size_t o_ud = o; o = al256(o + sizeof(int32_t) * (rcap + 1));
  size_t o_tc = o; o = al256(o + sizeof(int32_t) * etiles);
  size_t o_ta = o; o = al256(o + sizeof(seg3) * etiles);
  size_t o_tk = o; o = al256(o + sizeof(seg3) * etiles);
  size_t o_bc = o; o = al256(o + sizeof(int32_t) * rcap);
  size_t o_nr = o; o = al256(o + sizeof(int32_t) * lcp->nnz_capacity);
  size_t o_k1 = o; o = al256(o + sizeof(uint64_t) * E);
  size_t o_v1 = o; o = al256(o + sizeof(int32_t) * E);
  size_t o_k2 = o; o = al256(o + sizeof(uint64_t) * E);
  size_t o_v2 = o; o = al256(o + sizeof(int32_t) * E);
  size_t o_ug = o; o = al256(o + sizeof(double) * 3 * E);
  size_t o_gs = o; o = al256(o + sizeof(double) * 3 * E);
  size_t o_wk1 = o; o = al256(o + sizeof(uint64_t) * R2);
  size_t o_wv1 = o; o = al256(o + sizeof(int32_t) * R2);
  size_t o_wk2 = o; o = al256(o + sizeof(uint64_t) * R2);
  size_t o_wv2 = o; o = al256(o + sizeof(int32_t) * R2);
  size_t o_vs = o; o = al256(o + sizeof(int32_t) * n_ves);
  size_t o_ve = o; o = al256(o + sizeof(int32_t) * n_ves);
  size_t o_ss = o; o = al256(o + stiv_sort_scratch_impl(smax));
  if (o > h->lcp_ws_bytes) {
    if (h->lcp_ws) { STIV_CUDA(h, cudaFree(h->lcp_ws)); h->lcp_ws = nullptr; h->lcp_ws_bytes = 0; }
    STIV_CUDA(h, cudaMalloc(&h->lcp_ws, o));
    h->lcp_ws_bytes = o;
  }
  char* w = (char*)h->lcp_ws;
  int32_t* pstart = (int32_t*)(w + o_ps); int32_t* pend = (int32_t*)(w + o_pe);
  int32_t* row_of_pair = (int32_t*)(w + o_rp);
  int32_t* ustart = (int32_t*)(w + o_us); int32_t* tcount = (int32_t*)(w + o_tc);
  int32_t* uside = (int32_t*)(w + o_ud);
  seg3* tagg = (seg3*)(w + o_ta); seg3* tcarry = (seg3*)(w + o_tk);
  int32_t* bcnt = (int32_t*)(w + o_bc);
  int32_t* nzrow = (int32_t*)(w + o_nr);
  uint64_t* k1 = (uint64_t*)(w + o_k1); int32_t* v1 = (int32_t*)(w + o_v1);
  uint64_t* k2 = (uint64_t*)(w + o_k2); int32_t* v2 = (int32_t*)(w + o_v2);
  double* ug = (double*)(w + o_ug);
  double* gs = (double*)(w + o_gs);
  uint64_t* wk1 = (uint64_t*)(w + o_wk1); int32_t* wv1 = (int32_t*)(w + o_wv1);
  uint64_t* wk2 = (uint64_t*)(w + o_wk2); int32_t* wv2 = (int32_t*)(w + o_wv2);
  int32_t* vstart = (int32_t*)(w + o_vs); int32_t* vend = (int32_t*)(w + o_ve);
  void* ss = w + o_ss;
  size_t ss_bytes = stiv_sort_scratch_impl(smax);
  int sms = 152;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, h->device);
  STIV_PROF_N(h, st, "lcp_matrix", 13 + stiv_sort_kernels(rb + 1 + db) + stiv_sort_kernels(vb + rb));
  STIV_CUDA(h, cudaMemsetAsync(pstart, 0, sizeof(int32_t) * pcap, st));
  STIV_CUDA(h, cudaMemsetAsync(pend, 0, sizeof(int32_t) * pcap, st));
  STIV_CUDA(h, cudaMemsetAsync(vstart, 0, sizeof(int32_t) * n_ves, st));
  STIV_CUDA(h, cudaMemsetAsync(vend, 0, sizeof(int32_t) * n_ves, st));
  STIV_CUDA(h, cudaMemsetAsync(uside, 0xff, sizeof(int32_t) * (rcap + 1), st));   // -1: no side-1 entry
  bounds_kernel<<<sms * 4, 256, 0, st>>>(counts_dev, ccap, ct->pair, pstart, pend);
  rows_kernel<<<1, RT, 0, st>>>(counts_dev, pcap, ccap, pstart, pend, V_pair_dev, rcap, lcp->row_pair, row_of_pair,
                                lcp->q, lcp->dims);
  entries_kernel<<<sms * 4, 256, 0, st>>>(counts_dev, ccap, ct->pair, row_of_pair, cand->i, g_ves_dev, g_vid_dev,
                                          rcap, db, k1, v1);
  int rc = stiv_sort_pairs_impl(st, E, rb + 1 + db, k1, v1, k2, v2, ss, ss_bytes, &lcp->dims[3]);
  if (rc) return rc;
  uint64_t kmask = ((1ull << (1 + db)) - 1);
  // unique (side, vertex) entries of each row: keys into k1, gradients into
  // ug, row r's at [ustart[r], ustart[r + 1])
  gather_kernel<<<sms * 8, 256, 0, st>>>(&lcp->dims[3], v2, grad_dev, gs);
  tile_sums_kernel<<<(unsigned)etiles, ET, 0, st>>>(&lcp->dims[3], k2, gs, tcount, tagg);
  tile_scan_kernel<<<1, ET, 0, st>>>((int)etiles, tcount, tagg, tcarry, lcp->dims, ustart);
  compact_kernel<<<(unsigned)etiles, ET, 0, st>>>(&lcp->dims[3], k2, gs, tcount, tcarry, 1 + db, kmask, k1, ug,
                                                  ustart, uside);
  // per-vesicle row lists
  ves_kernel<<<sms, 256, 0, st>>>(lcp->dims, lcp->row_pair, cand->i, cand->j, rb, wk1, wv1);
  rc = stiv_sort_pairs_impl(st, R2, vb + rb, wk1, wv1, wk2, wv2, ss, ss_bytes, &lcp->dims[4]);
  if (rc) return rc;
  ves_bounds_kernel<<<sms, 256, 0, st>>>(lcp->dims, wk2, rb, vstart, vend);
  bcount_kernel<<<sms, 256, 0, st>>>(lcp->dims, lcp->row_pair, cand->i, cand->j, wv2, vstart, vend, bcnt);
  bscan_kernel<<<1, RT, 0, st>>>(lcp->dims, bcnt, lcp->nnz_capacity, lcp->row_ptr);
  // one vertex-index table per warp: as many warps per CTA as 96 KB holds
  int nvtab = stiv_nverts(2 * p_max);
  int bw = (int)((96 * 1024) / (sizeof(int32_t) * (size_t)nvtab));
  bw = bw < 1 ? 1 : (bw > 8 ? 8 : bw);
  size_t bsmem = sizeof(int32_t) * (size_t)nvtab * bw;
  if (bsmem > 48 * 1024)
    STIV_CUDA(h, cudaFuncSetAttribute(bval_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bsmem));
  bcol_kernel<<<sms, 256, 0, st>>>(lcp->dims, lcp->row_pair, cand->i, cand->j, wv2, vstart, vend, lcp->row_ptr,
                                   lcp->nnz_capacity, lcp->col, nzrow);
  bval_kernel<<<sms * 4, 32 * bw, bsmem, st>>>(lcp->dims, lcp->row_pair, cand->i, cand->j, ustart, uside, k1, ug,
                                               m_ves_dev, t_ves_dev, db, nvtab, lcp->nnz_capacity, lcp->col, nzrow,
                                               lcp->val);
  STIV_LAUNCH(h);
  return STIV_OK;
}

extern "C" int stiv_lcp_solve(stiv_handle* h, void* stream, const stiv_lcp* lcp, double tol, int32_t max_newton,
                              int32_t max_cg, double* lambda_dev, double* info_dev) {
  if (!h || !lcp || !lambda_dev || !info_dev || !lcp->dims || !lcp->row_ptr || !lcp->col || !lcp->val || !lcp->q)
    return STIV_ERR_ARG;
  if (!(tol > 0.0) || max_newton < 1 || max_cg < 1 || lcp->row_capacity < 1 || lcp->nnz_capacity < 1)
    return STIV_ERR_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  int64_t n = lcp->row_capacity, nz = lcp->nnz_capacity;
  size_t o = 0;
  size_t o_w = o; o = al256(o + sizeof(double) * n);
  size_t o_dx = o; o = al256(o + sizeof(double) * n);
  size_t o_xn = o; o = al256(o + sizeof(double) * n);
  size_t o_y = o; o = al256(o + sizeof(float) * n);
  size_t o_r = o; o = al256(o + sizeof(float) * n);
  size_t o_p = o; o = al256(o + sizeof(float) * n);
  size_t o_ap = o; o = al256(o + sizeof(float) * n);
  size_t o_di = o; o = al256(o + sizeof(float) * n);
  size_t o_act = o; o = al256(o + n);
  size_t o_vf = o; o = al256(o + sizeof(float) * nz);
  if (o > h->lcp_ws2_bytes) {
    if (h->lcp_ws2) { STIV_CUDA(h, cudaFree(h->lcp_ws2)); h->lcp_ws2 = nullptr; h->lcp_ws2_bytes = 0; }
    STIV_CUDA(h, cudaMalloc(&h->lcp_ws2, o));
    h->lcp_ws2_bytes = o;
  }
  char* w = (char*)h->lcp_ws2;
  solve_args a;
  a.dims = lcp->dims; a.row_ptr = lcp->row_ptr; a.col = lcp->col; a.val = lcp->val; a.q = lcp->q;
  a.x = lambda_dev; a.w = (double*)(w + o_w); a.dx = (double*)(w + o_dx); a.xn = (double*)(w + o_xn);
  a.y = (float*)(w + o_y); a.r = (float*)(w + o_r); a.pv = (float*)(w + o_p); a.Ap = (float*)(w + o_ap);
  a.dinv = (float*)(w + o_di);
  a.act = (unsigned char*)(w + o_act);
  a.valf = (float*)(w + o_vf);
  a.tol = tol; a.max_newton = max_newton; a.max_cg = max_cg; a.info = info_dev;
  STIV_PROF(h, st, "lcp_solve");
  size_t smem = SOLVE_SMEM;
  if (cudaFuncSetAttribute(solve_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)SOLVE_SMEM) != cudaSuccess) {
    cudaGetLastError();
    smem = 0;   // everything in global scratch
  }
  solve_kernel<<<1, RT, smem, st>>>(a, smem);
  STIV_LAUNCH(h);
  return STIV_OK;
}

// Contact LCP of a step (Sec. 3.2, Eq. 3.7; Sec. 3.3.3, Alg. 3) on one GPU.
//
//   0 <= -V + B lambda   perp   lambda >= 0,      B = J M J^T
//
// One row per contact volume: a candidate vesicle pair (with its periodic
// image) that has contacts; V its volume (the library's volumes are >= 0 for
// interference, the paper's constraint V >= 0 has the opposite sign, which B
// does not see).  J = dV/dX1 (the gradient rows of stiv_stiv_grad, summed
// per vertex); M block-diagonal, one scalar m_i per vesicle (M_ii = m_i I), a
// stand-in for the locally implicit scheme's A^-1 G.
//
// Assembly (Alg. 3):
//   bounds_kernel   contact range of every candidate pair (contacts are
//                   sorted by pair)
//   rows_kernel     rows = pairs with contacts; q = -V
//   entries_kernel  one keyed entry per contact point: row | vesicle | vertex
//   (radix sort, stable)
//   reduce_kernel   per row, the gradient of each vertex summed in contact
//                   order (deterministic)
//   ves_kernel      (vesicle, row) keys -> sorted per-vesicle row lists
//   bcount_kernel   per row, the rows sharing a vesicle (union of its two
//                   vesicles' lists)
//   bval_kernel     B(j, k) = sum over shared vesicles i (ascending) of
//                   m_i g_j|i . g_k|i, a merge-join over the vertices of i
// Solve: min-map Newton (Phi = min(lambda, B lambda + q)), the Newton system
// on the active set by conjugate gradients (B_AA is symmetric positive
// definite), Armijo line search on |Phi|^2 / 2; one CTA, all iterations in
// one launch.
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
                                                  int64_t rcap, int32_t* row_pair, int32_t* row_of_pair,
                                                  int32_t* rstart, int32_t* rend, double* q, int64_t* dims) {
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
        rstart[r] = pstart[p];
        rend[r] = pend[p];
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
                               const int32_t* gves, const int32_t* gvid, int64_t rcap, int vb, int db,
                               uint64_t* key, int32_t* val) {
  int64_t n = ncontacts(counts, ccap);
  for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x) {
    int r = row_of_pair[pair[k]];
    uint64_t rr = (r >= 0 && r < rcap) ? (uint64_t)r : (uint64_t)rcap;   // beyond capacity: sorted last
    for (int q = 0; q < 4; ++q) {
      key[4 * k + q] = (rr << (vb + db)) | ((uint64_t)gves[4 * k + q] << db) | (uint64_t)gvid[4 * k + q];
      val[4 * k + q] = (int32_t)(4 * k + q);
    }
  }
}

// One CTA per row: runs of equal (vesicle, vertex) keys in sorted order are
// summed in that order; unique entries at [4 rstart, 4 rstart + ucount).
__global__ void __launch_bounds__(RT) reduce_kernel(const int64_t* dims, const int32_t* rstart, const int32_t* rend,
                                                    const uint64_t* skey, const int32_t* sval, const double* grad,
                                                    uint64_t kmask, uint64_t* ukey, double* ug, int32_t* ucount) {
  __shared__ int sh[RT];
  int r = blockIdx.x;
  if (r >= dims[0]) return;
  int64_t b = 4 * (int64_t)rstart[r], e = 4 * (int64_t)rend[r];
  int out = 0;
  for (int64_t i0 = b; i0 < e; i0 += RT) {
    int64_t i = i0 + threadIdx.x;
    int head = (i < e && (i == b || skey[i] != skey[i - 1])) ? 1 : 0;
    int tot;
    int ex = block_scan(head, sh, tot);
    if (head) {
      double s0 = 0.0, s1 = 0.0, s2 = 0.0;
      uint64_t k = skey[i];
      for (int64_t j = i; j < e && skey[j] == k; ++j) {
        const double* g = grad + 3 * (size_t)sval[j];
        s0 += g[0]; s1 += g[1]; s2 += g[2];
      }
      int64_t o = b + out + ex;
      ukey[o] = k & kmask;
      ug[3 * o] = s0; ug[3 * o + 1] = s1; ug[3 * o + 2] = s2;
    }
    out += tot;
  }
  if (threadIdx.x == 0) ucount[r] = out;
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

// Entries of row r belonging to vesicle v: a range of its unique entries
// (sorted by vesicle, then vertex).
__device__ __forceinline__ void ves_range(const uint64_t* ukey, int64_t b, int cnt, uint64_t v, int db, int64_t& lo,
                                          int64_t& hi) {
  int64_t a = b, z = b + cnt;
  while (a < z) { int64_t m = (a + z) >> 1; if ((ukey[m] >> db) < v) a = m + 1; else z = m; }
  lo = a;
  z = b + cnt;
  while (a < z) { int64_t m = (a + z) >> 1; if ((ukey[m] >> db) <= v) a = m + 1; else z = m; }
  hi = a;
}

// One warp per row: every neighbour's entry in ascending order; the dot
// products over a vesicle's vertices are merge-joins (lanes over the entries
// of the lower-numbered row of the two, binary search in the other), reduced
// in a fixed order, so that B(r, s) and B(s, r) are the same sum: B is
// symmetric bit for bit.
__global__ void bval_kernel(const int64_t* dims, const int32_t* row_pair, const int32_t* ci, const int32_t* cj,
                            const int32_t* vrow, const int32_t* vstart, const int32_t* vend, const int32_t* rstart,
                            const int32_t* ucount, const uint64_t* ukey, const double* ug, const double* m_ves,
                            const double* t_ves, int db, const int64_t* row_ptr, int64_t nnz_cap, int32_t* col, double* val) {
  int lane = threadIdx.x & 31;
  int64_t n = dims[0];
  int64_t w0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5, nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t r = w0; r < n; r += nw) {
    int p = row_pair[r], vi = ci[p], vj = cj[p];
    int64_t br = 4 * (int64_t)rstart[r];
    int cr = ucount[r];
    int64_t o = row_ptr[r];
    for_neighbours(vrow, vstart[vi], vend[vi], vstart[vj], vend[vj], [&](int s) {
      int ps = row_pair[s], si = ci[ps], sj = cj[ps];
      int64_t bs = 4 * (int64_t)rstart[s];
      int cs = ucount[s];
      // lanes over the entries of row min(r, s)
      int64_t bA = s < r ? bs : br, bB = s < r ? br : bs;
      int cA = s < r ? cs : cr, cB = s < r ? cr : cs;
      double acc = 0.0;
      int vs[2] = {vi, vj};   // vi < vj: ascending
      for (int t = 0; t < 2; ++t) {
        int v = vs[t];
        if (v != si && v != sj) continue;
        int64_t a0, a1, b0, b1;
        ves_range(ukey, bA, cA, (uint64_t)v, db, a0, a1);
        ves_range(ukey, bB, cB, (uint64_t)v, db, b0, b1);
        double part = 0.0, sa[3] = {0.0, 0.0, 0.0}, sb[3] = {0.0, 0.0, 0.0};
        for (int64_t i = a0 + lane; i < a1; i += 32) {
          uint64_t k = ukey[i];
          int64_t lo = b0, hi = b1;
          while (lo < hi) { int64_t m = (lo + hi) >> 1; if (ukey[m] < k) lo = m + 1; else hi = m; }
          if (lo < b1 && ukey[lo] == k)
            part += ug[3 * i] * ug[3 * lo] + ug[3 * i + 1] * ug[3 * lo + 1] + ug[3 * i + 2] * ug[3 * lo + 2];
          for (int d = 0; d < 3; ++d) sa[d] += ug[3 * i + d];
        }
        for (int off = 16; off > 0; off >>= 1) part += __shfl_xor_sync(0xffffffffu, part, off);
        acc += (m_ves ? m_ves[v] : 1.0) * part;
        if (t_ves) {   // rigid translation: (sum of g_r over v's points) . (sum of g_s)
          for (int64_t i = b0 + lane; i < b1; i += 32)
            for (int d = 0; d < 3; ++d) sb[d] += ug[3 * i + d];
          for (int off = 16; off > 0; off >>= 1)
            for (int d = 0; d < 3; ++d) {
              sa[d] += __shfl_xor_sync(0xffffffffu, sa[d], off);
              sb[d] += __shfl_xor_sync(0xffffffffu, sb[d], off);
            }
          acc += t_ves[v] * (sa[0] * sb[0] + sa[1] * sb[1] + sa[2] * sb[2]);
        }
      }
      if (lane == 0 && o < nnz_cap) { col[o] = s; val[o] = acc; }
      ++o;
    });
  }
}

// ---------------------------------------------------------------------------
// min-map Newton, one CTA
// ---------------------------------------------------------------------------
struct solve_args {
  const int64_t* dims;
  const int64_t* row_ptr;
  const int32_t* col;
  const double* val;
  const double* q;
  double* x;      // lambda
  double* w;
  double* dx;
  double* r;
  double* pv;
  double* Ap;
  double* xn;
  unsigned char* act;
  double tol;
  int max_newton, max_cg;
  double* info;   // [0] Newton iterations, [1] max |Phi|, [2] CG iterations, [3] status
};

__device__ double block_sum(double v, double* sh) {
  sh[threadIdx.x] = v;
  __syncthreads();
  for (int s = RT / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s) sh[threadIdx.x] += sh[threadIdx.x + s];
    __syncthreads();
  }
  double t = sh[0];
  __syncthreads();
  return t;
}
__device__ double block_max(double v, double* sh) {
  sh[threadIdx.x] = v;
  __syncthreads();
  for (int s = RT / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s) sh[threadIdx.x] = fmax(sh[threadIdx.x], sh[threadIdx.x + s]);
    __syncthreads();
  }
  double t = sh[0];
  __syncthreads();
  return t;
}

// y = B x (rows and columns restricted to the active set when masked)
__device__ void spmv(const solve_args& a, int64_t n, const double* x, double* y, const unsigned char* mask) {
  for (int64_t i = threadIdx.x; i < n; i += RT) {
    if (mask && !mask[i]) { y[i] = 0.0; continue; }
    double s = 0.0;
    for (int64_t k = a.row_ptr[i]; k < a.row_ptr[i + 1]; ++k) {
      int j = a.col[k];
      if (mask && !mask[j]) continue;
      s += a.val[k] * x[j];
    }
    y[i] = s;
  }
  __syncthreads();
}

__device__ double merit(const solve_args& a, int64_t n, const double* x, double* y, double* sh, double& res) {
  spmv(a, n, x, y, nullptr);
  double s = 0.0, m = 0.0;
  for (int64_t i = threadIdx.x; i < n; i += RT) {
    double ph = fmin(x[i], y[i] + a.q[i]);
    s += ph * ph;
    m = fmax(m, fabs(ph));
  }
  res = block_max(m, sh);
  return 0.5 * block_sum(s, sh);
}

__global__ void __launch_bounds__(RT) solve_kernel(solve_args a) {
  __shared__ double sh[RT];
  int64_t n = a.dims[0];
  if (a.dims[2]) {   // matrix over capacity
    if (threadIdx.x == 0) { a.info[0] = 0; a.info[1] = -1; a.info[2] = 0; a.info[3] = 1; }
    return;
  }
  for (int64_t i = threadIdx.x; i < n; i += RT) a.x[i] = 0.0;
  __syncthreads();
  long long cg_total = 0;
  int it = 0;
  double res = 0.0;
  for (it = 0;; ++it) {
    double psi = merit(a, n, a.x, a.w, sh, res);   // w = B x
    if (res <= a.tol || it == a.max_newton) break;
    // active set and the Newton system
    for (int64_t i = threadIdx.x; i < n; i += RT) {
      double wi = a.w[i] + a.q[i];
      a.act[i] = wi < a.x[i];
      a.dx[i] = a.act[i] ? 0.0 : -a.x[i];
    }
    __syncthreads();
    // rhs_A = -(B x + q)_A - B_{A,F} dx_F ; CG on B_AA from dx_A = 0
    for (int64_t i = threadIdx.x; i < n; i += RT) {
      if (!a.act[i]) { a.r[i] = 0.0; continue; }
      double s = 0.0;
      for (int64_t k = a.row_ptr[i]; k < a.row_ptr[i + 1]; ++k) {
        int j = a.col[k];
        if (!a.act[j]) s += a.val[k] * a.dx[j];
      }
      a.r[i] = -(a.w[i] + a.q[i]) - s;
    }
    __syncthreads();
    double rr = 0.0;
    for (int64_t i = threadIdx.x; i < n; i += RT) { a.pv[i] = a.r[i]; rr += a.r[i] * a.r[i]; }
    rr = block_sum(rr, sh);
    double rr0 = rr;
    for (int k = 0; k < a.max_cg && rr > 1e-28 * rr0 && rr > 0.0; ++k) {
      spmv(a, n, a.pv, a.Ap, a.act);
      double pAp = 0.0;
      for (int64_t i = threadIdx.x; i < n; i += RT) pAp += a.pv[i] * a.Ap[i];
      pAp = block_sum(pAp, sh);
      if (!(pAp > 0.0)) break;
      double al = rr / pAp, rn = 0.0;
      for (int64_t i = threadIdx.x; i < n; i += RT)
        if (a.act[i]) { a.dx[i] += al * a.pv[i]; a.r[i] -= al * a.Ap[i]; rn += a.r[i] * a.r[i]; }
      rn = block_sum(rn, sh);
      double be = rn / rr;
      for (int64_t i = threadIdx.x; i < n; i += RT) a.pv[i] = a.act[i] ? a.r[i] + be * a.pv[i] : 0.0;
      __syncthreads();
      rr = rn;
      ++cg_total;
    }
    // Armijo line search on psi along x + t dx
    double t = 1.0;
    for (int h = 0; h < 40; ++h) {
      for (int64_t i = threadIdx.x; i < n; i += RT) a.xn[i] = a.x[i] + t * a.dx[i];
      __syncthreads();
      double rn;
      double pn = merit(a, n, a.xn, a.Ap, sh, rn);
      if (pn <= (1.0 - 2.0e-4 * t) * psi) break;
      t *= 0.5;
    }
    for (int64_t i = threadIdx.x; i < n; i += RT) a.x[i] = a.xn[i];
    __syncthreads();
  }
  if (threadIdx.x == 0) { a.info[0] = it; a.info[1] = res; a.info[2] = (double)cg_total; a.info[3] = res <= a.tol ? 0 : 2; }
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
  if (rb + vb + db > 63) return STIV_ERR_ARG;
  int64_t E = 4 * ccap, R2 = 2 * rcap;
  int64_t smax = E > R2 ? E : R2;
  // scratch (handle-owned, grown on demand)
  size_t o = 0;
  size_t o_ps = o; o = al256(o + sizeof(int32_t) * pcap);
  size_t o_pe = o; o = al256(o + sizeof(int32_t) * pcap);
  size_t o_rp = o; o = al256(o + sizeof(int32_t) * pcap);
  size_t o_rs = o; o = al256(o + sizeof(int32_t) * rcap);
  size_t o_re = o; o = al256(o + sizeof(int32_t) * rcap);
  size_t o_uc = o; o = al256(o + sizeof(int32_t) * rcap);
  size_t o_bc = o; o = al256(o + sizeof(int32_t) * rcap);
  size_t o_k1 = o; o = al256(o + sizeof(uint64_t) * E);
  size_t o_v1 = o; o = al256(o + sizeof(int32_t) * E);
  size_t o_k2 = o; o = al256(o + sizeof(uint64_t) * E);
  size_t o_v2 = o; o = al256(o + sizeof(int32_t) * E);
  size_t o_ug = o; o = al256(o + sizeof(double) * 3 * E);
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
  int32_t* rstart = (int32_t*)(w + o_rs); int32_t* rend = (int32_t*)(w + o_re);
  int32_t* ucount = (int32_t*)(w + o_uc); int32_t* bcnt = (int32_t*)(w + o_bc);
  uint64_t* k1 = (uint64_t*)(w + o_k1); int32_t* v1 = (int32_t*)(w + o_v1);
  uint64_t* k2 = (uint64_t*)(w + o_k2); int32_t* v2 = (int32_t*)(w + o_v2);
  double* ug = (double*)(w + o_ug);
  uint64_t* wk1 = (uint64_t*)(w + o_wk1); int32_t* wv1 = (int32_t*)(w + o_wv1);
  uint64_t* wk2 = (uint64_t*)(w + o_wk2); int32_t* wv2 = (int32_t*)(w + o_wv2);
  int32_t* vstart = (int32_t*)(w + o_vs); int32_t* vend = (int32_t*)(w + o_ve);
  void* ss = w + o_ss;
  size_t ss_bytes = stiv_sort_scratch_impl(smax);
  int sms = 152;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, h->device);
  STIV_PROF_N(h, st, "lcp_matrix", 9 + stiv_sort_kernels(rb + vb + db) + stiv_sort_kernels(vb + rb));
  STIV_CUDA(h, cudaMemsetAsync(pstart, 0, sizeof(int32_t) * pcap, st));
  STIV_CUDA(h, cudaMemsetAsync(pend, 0, sizeof(int32_t) * pcap, st));
  STIV_CUDA(h, cudaMemsetAsync(vstart, 0, sizeof(int32_t) * n_ves, st));
  STIV_CUDA(h, cudaMemsetAsync(vend, 0, sizeof(int32_t) * n_ves, st));
  bounds_kernel<<<sms * 4, 256, 0, st>>>(counts_dev, ccap, ct->pair, pstart, pend);
  rows_kernel<<<1, RT, 0, st>>>(counts_dev, pcap, ccap, pstart, pend, V_pair_dev, rcap, lcp->row_pair, row_of_pair,
                                rstart, rend, lcp->q, lcp->dims);
  entries_kernel<<<sms * 4, 256, 0, st>>>(counts_dev, ccap, ct->pair, row_of_pair, g_ves_dev, g_vid_dev, rcap, vb, db,
                                          k1, v1);
  int rc = stiv_sort_pairs_impl(st, E, rb + vb + db, k1, v1, k2, v2, ss, ss_bytes, &lcp->dims[3]);
  if (rc) return rc;
  uint64_t kmask = ((1ull << (vb + db)) - 1);
  // unique (vesicle, vertex) entries of each row: keys into k1, gradients into ug
  reduce_kernel<<<(unsigned)rcap, RT, 0, st>>>(lcp->dims, rstart, rend, k2, v2, grad_dev, kmask, k1, ug, ucount);
  // per-vesicle row lists
  ves_kernel<<<sms, 256, 0, st>>>(lcp->dims, lcp->row_pair, cand->i, cand->j, rb, wk1, wv1);
  rc = stiv_sort_pairs_impl(st, R2, vb + rb, wk1, wv1, wk2, wv2, ss, ss_bytes, &lcp->dims[4]);
  if (rc) return rc;
  ves_bounds_kernel<<<sms, 256, 0, st>>>(lcp->dims, wk2, rb, vstart, vend);
  bcount_kernel<<<sms, 256, 0, st>>>(lcp->dims, lcp->row_pair, cand->i, cand->j, wv2, vstart, vend, bcnt);
  bscan_kernel<<<1, RT, 0, st>>>(lcp->dims, bcnt, lcp->nnz_capacity, lcp->row_ptr);
  bval_kernel<<<sms * 8, 256, 0, st>>>(lcp->dims, lcp->row_pair, cand->i, cand->j, wv2, vstart, vend, rstart, ucount,
                                       k1, ug, m_ves_dev, t_ves_dev, db, lcp->row_ptr, lcp->nnz_capacity, lcp->col, lcp->val);
  STIV_LAUNCH(h);
  return STIV_OK;
}

extern "C" int stiv_lcp_solve(stiv_handle* h, void* stream, const stiv_lcp* lcp, double tol, int32_t max_newton,
                              int32_t max_cg, double* lambda_dev, double* info_dev) {
  if (!h || !lcp || !lambda_dev || !info_dev || !lcp->dims || !lcp->row_ptr || !lcp->col || !lcp->val || !lcp->q)
    return STIV_ERR_ARG;
  if (!(tol > 0.0) || max_newton < 1 || max_cg < 1 || lcp->row_capacity < 1) return STIV_ERR_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  int64_t n = lcp->row_capacity;
  size_t o = 0;
  size_t o_w = o; o = al256(o + sizeof(double) * n);
  size_t o_dx = o; o = al256(o + sizeof(double) * n);
  size_t o_r = o; o = al256(o + sizeof(double) * n);
  size_t o_p = o; o = al256(o + sizeof(double) * n);
  size_t o_ap = o; o = al256(o + sizeof(double) * n);
  size_t o_xn = o; o = al256(o + sizeof(double) * n);
  size_t o_act = o; o = al256(o + n);
  if (o > h->lcp_ws2_bytes) {
    if (h->lcp_ws2) { STIV_CUDA(h, cudaFree(h->lcp_ws2)); h->lcp_ws2 = nullptr; h->lcp_ws2_bytes = 0; }
    STIV_CUDA(h, cudaMalloc(&h->lcp_ws2, o));
    h->lcp_ws2_bytes = o;
  }
  char* w = (char*)h->lcp_ws2;
  solve_args a;
  a.dims = lcp->dims; a.row_ptr = lcp->row_ptr; a.col = lcp->col; a.val = lcp->val; a.q = lcp->q;
  a.x = lambda_dev; a.w = (double*)(w + o_w); a.dx = (double*)(w + o_dx); a.r = (double*)(w + o_r);
  a.pv = (double*)(w + o_p); a.Ap = (double*)(w + o_ap); a.xn = (double*)(w + o_xn);
  a.act = (unsigned char*)(w + o_act);
  a.tol = tol; a.max_newton = max_newton; a.max_cg = max_cg; a.info = info_dev;
  STIV_PROF(h, st, "lcp_solve");
  solve_kernel<<<1, RT, 0, st>>>(a);
  STIV_LAUNCH(h);
  return STIV_OK;
}

// Space-time bounding boxes (Alg. 2 getBoundingBox) and the bounding-box
// intersection of Alg. 1 (Sec. 3.3.1) on one GPU.
//
//   1. vesicle boxes: exact FP64 min/max of X0 and X1 over all vertices, padded
//      by d_m; patch boxes (4 x 8 grid quads and their vertices) in FP32,
//      rounded outward, for the narrow phase;
//   2. h_m = mean box diagonal (Alg. 1, grid spacing), cell size of a uniform grid
//      (periodic axes: L / floor(L / h_m));
//   3. each box lists the cells it overlaps (an exact cell-range enumeration
//      standing in for the check points of Alg. 1), keyed by the
//      Morton id of the (wrapped) cell;
//   4. stable radix sort by Morton id (Alg. 1, check-point sort; 24-bit keys:
//      at most 256 wrapped cells per axis);
//   5. all box pairs within a cell: the image shift follows from the unwrapped
//      cell coordinates, then bbiCheck in FP64 (Alg. 1, per-cell loop);
//   6. sort + unique (Alg. 1, final step) -> pairs (i < j, shift), ascending.
#include "stiv_internal.cuh"

#include <math.h>

namespace {

template <typename T>
__device__ __forceinline__ double ld(const void* p, size_t i) { return (double)((const T*)p)[i]; }

__device__ __forceinline__ double vload(const void* X, int mixed, size_t i) {
  return mixed ? (double)((const float*)X)[i] : ((const double*)X)[i];
}

// Order-preserving int64 image of a double (a <= b <=> okey(a) <= okey(b)
// for non-NaN values, -0 just below +0) and its inverse (the map is its own
// inverse): exact FP64 min / max on the integer pipe.
__device__ __forceinline__ long long okey(double v) {
  long long b = __double_as_longlong(v);
  return b ^ ((b >> 63) & 0x7FFFFFFFFFFFFFFFll);
}
__device__ __forceinline__ double okey_val(long long k) {
  return __longlong_as_double(k ^ ((k >> 63) & 0x7FFFFFFFFFFFFFFFll));
}

// x rounded to float toward -inf (up = false) or +inf (up = true), on the
// integer pipe for |x| in the normal float range: the significand truncated
// to 23 bits rounds toward zero, and one unit in the last place more in
// magnitude gives the other direction when bits were dropped (a carry into
// the exponent, up to infinity, is the correct rounding).  Other values take
// the conversion instruction.
__device__ __forceinline__ float d2f_dir(double x, bool up) {
  unsigned long long b = (unsigned long long)__double_as_longlong(x);
  int e = (int)((b >> 52) & 0x7FF) - 1023;
  if (e < -126 || e > 127) return up ? __double2float_ru(x) : __double2float_rd(x);
  unsigned sgn = (unsigned)(b >> 63);
  unsigned f = (sgn << 31) | ((unsigned)(e + 127) << 23) | (unsigned)((b >> 29) & 0x7FFFFF);
  if ((b & 0x1FFFFFFFull) != 0 && (up ? sgn == 0 : sgn != 0)) f += 1;
  return __uint_as_float(f);
}

// One CTA per vesicle.  MIXED (FP32 vertices): the min / max run in FP32,
// which is exact, and widen exactly to FP64, so the boxes are those of the
// FP64 reduction bit for bit without its FP64 instructions.  FP64 vertices:
// the min / max run on order-preserving integer images (exact), and the
// per-vertex FP32 boxes are rounded outward on the integer pipe, so that the
// FP64 pipe only forms the staging differences.
template <bool MIXED>
__global__ void __launch_bounds__(256) boxes_kernel(int n, const int32_t* pv, const int64_t* voff, const void* X,
                                                    int mixed, double dm, double Lx, double Ly, double Lz,
                                                    double* vbox, float* pbox, int pstride, float* vorg,
                                                    float* fprep, int64_t fstride, int64_t* ctr, size_t vb_cap,
                                                    int p_max) {
  extern __shared__ float vbs[];   // [6][nv]: swept FP32 box of each vertex (rounded outward), if it fits
  int v = blockIdx.x;
  if (pv[v] < 1 || pv[v] > p_max) {
    // an order outside [1, p_max]: flagged, and an inverted box keeps the
    // vesicle out of every cell (the broad phase skips inverted boxes), so no
    // later kernel reads its mesh
    if (threadIdx.x == 0) atomicOr((unsigned long long*)&ctr[STIV_C_STATUS], STIV_F_BAD_ORDER);
    if (threadIdx.x < 3) {
      vbox[6 * v + threadIdx.x] = INFINITY;
      vbox[6 * v + 3 + threadIdx.x] = -INFINITY;
    }
    if (threadIdx.x < 4) vorg[4 * v + threadIdx.x] = 0.0f;
    return;
  }
  int P = 2 * pv[v], nv = stiv_nverts(P);
  bool use_sm = (size_t)6 * nv <= vb_cap;
  const size_t base = voff[v];
  __shared__ long long red[6][256];
  double lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
  bool bad = false;
  if (MIXED) {
    const float* Xf = (const float*)X;
    float flo[3] = {INFINITY, INFINITY, INFINITY}, fhi[3] = {-INFINITY, -INFINITY, -INFINITY};
    for (int k = threadIdx.x; k < nv; k += blockDim.x)
      for (int c = 0; c < 3; ++c) {
        float x0 = Xf[base + (size_t)c * nv + k], x1 = Xf[base + (size_t)(3 + c) * nv + k];
        if (!isfinite(x0) || !isfinite(x1)) bad = true;
        float a = fminf(x0, x1), b = fmaxf(x0, x1);
        flo[c] = fminf(flo[c], a);
        fhi[c] = fmaxf(fhi[c], b);
        if (use_sm) { vbs[c * nv + k] = a; vbs[(3 + c) * nv + k] = b; }
      }
    for (int c = 0; c < 3; ++c) { lo[c] = (double)flo[c]; hi[c] = (double)fhi[c]; }
  }
  long long klo[3], khi[3];
  for (int c = 0; c < 3; ++c) { klo[c] = okey(lo[c]); khi[c] = okey(hi[c]); }
  if (!MIXED) {
    const double* Xd = (const double*)X;
    for (int k = threadIdx.x; k < nv; k += blockDim.x)
      for (int c = 0; c < 3; ++c) {
        double x0 = Xd[base + (size_t)c * nv + k], x1 = Xd[base + (size_t)(3 + c) * nv + k];
        long long b0 = __double_as_longlong(x0), b1 = __double_as_longlong(x1);
        long long k0 = okey(x0), k1 = okey(x1);
        // finite iff the exponent field is not all ones; a NaN is ignored by
        // the min / max, as fmin / fmax ignore it
        if ((~b0 & 0x7FF0000000000000ll) == 0 || (~b1 & 0x7FF0000000000000ll) == 0) bad = true;
        bool n0 = (b0 & 0x7FFFFFFFFFFFFFFFll) > 0x7FF0000000000000ll;
        bool n1 = (b1 & 0x7FFFFFFFFFFFFFFFll) > 0x7FF0000000000000ll;
        if (n0) k0 = k1;
        if (n1) k1 = k0;
        long long ka = k0 < k1 ? k0 : k1, kb = k0 < k1 ? k1 : k0;
        if (!(n0 && n1)) {
          klo[c] = ka < klo[c] ? ka : klo[c];
          khi[c] = kb > khi[c] ? kb : khi[c];
        }
        if (use_sm) {
          vbs[c * nv + k] = d2f_dir(okey_val(ka), false);
          vbs[(3 + c) * nv + k] = d2f_dir(okey_val(kb), true);
        }
      }
  }
  for (int c = 0; c < 3; ++c) { red[c][threadIdx.x] = klo[c]; red[3 + c][threadIdx.x] = khi[c]; }
  if (__syncthreads_or(bad) && threadIdx.x == 0) atomicOr((unsigned long long*)&ctr[STIV_C_STATUS], STIV_F_NONFINITE);
  for (int s = 128; s > 0; s >>= 1) {
    if (threadIdx.x < s)
      for (int c = 0; c < 3; ++c) {
        long long a = red[c][threadIdx.x + s], b = red[3 + c][threadIdx.x + s];
        if (a < red[c][threadIdx.x]) red[c][threadIdx.x] = a;
        if (b > red[3 + c][threadIdx.x]) red[3 + c][threadIdx.x] = b;
      }
    __syncthreads();
  }
  __shared__ float sorg[4];
  __shared__ double vlo_s[3], vhi_s[3];
  if (threadIdx.x < 3) {
    int c = threadIdx.x;
    vlo_s[c] = okey_val(red[c][0]);
    vhi_s[c] = okey_val(red[3 + c][0]);
  }
  __syncthreads();
  if (threadIdx.x < 3) {
    int c = threadIdx.x;
    double l = vlo_s[c] - dm, u = vhi_s[c] + dm;
    vbox[6 * v + c] = l;
    vbox[6 * v + 3 + c] = u;
    double L = c == 0 ? Lx : c == 1 ? Ly : Lz;
    if (L > 0.0 && !(u - l < 0.5 * L)) atomicOr((unsigned long long*)&ctr[STIV_C_STATUS], STIV_F_BOX_TOO_SMALL);
    // FP32 frame of this vesicle: origin at the (float-rounded) box centre
    float o = (float)(0.5 * (vlo_s[c] + vhi_s[c]));
    sorg[c] = o;
    vorg[4 * v + c] = o;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    // R bounds |X - o| over the vesicle (both times), rounded up
    double R = 0.0;
    for (int c = 0; c < 3; ++c) R = fmax(R, fmax(vhi_s[c] - (double)sorg[c], (double)sorg[c] - vlo_s[c]));
    vorg[4 * v + 3] = __double2float_ru(R);
  }
  // per-vertex FP32 data (two float4).  FP32 vertices: X0 and X1 as stored,
  // from which the narrow phase takes both the exact keys and the frame
  // coordinates.  FP64 vertices: position at t_n relative to the origin and
  // the displacement X1 - X0, each rounded once.
  float4* f4 = (float4*)(fprep + (size_t)v * fstride);
  if (MIXED) {
    const float* Xf = (const float*)X;
    for (int k = threadIdx.x; k < nv; k += blockDim.x) {
      f4[2 * k] = make_float4(Xf[base + k], Xf[base + (size_t)nv + k], Xf[base + (size_t)2 * nv + k], 0.f);
      f4[2 * k + 1] = make_float4(Xf[base + (size_t)3 * nv + k], Xf[base + (size_t)4 * nv + k],
                                  Xf[base + (size_t)5 * nv + k], 0.f);
    }
  } else
  for (int k = threadIdx.x; k < nv; k += blockDim.x) {
    float xo[3], dd[3];
    for (int c = 0; c < 3; ++c) {
      double x0 = vload(X, mixed, base + (size_t)c * nv + k);
      double x1 = vload(X, mixed, base + (size_t)(3 + c) * nv + k);
      xo[c] = (float)(x0 - (double)sorg[c]);
      dd[c] = (float)(x1 - x0);
    }
    f4[2 * k] = make_float4(xo[0], xo[1], xo[2], 0.f);
    f4[2 * k + 1] = make_float4(dd[0], dd[1], dd[2], 0.f);
  }
  // patch boxes: vertex rows [I*BR, I*BR+BR], columns [J*BC, J*BC+BC]
  // (wrapping), poles; each as the union of its four cells' boxes (band b of
  // the two, column half h), every cell box written beside it.  Per column
  // half, the boxes of its three rows are formed once and merged into its
  // two cells.  P is even, so every patch
  // spans BR bands and BC columns.  From the per-vertex FP32 boxes in shared
  // memory when they fit: rounding outward is monotone, so the result equals
  // rounding the FP64 min / max.
  int nbr = stiv_nband_blocks(P), nbc = stiv_ncol_blocks(P), W = 2 * P;
  __syncthreads();
  for (int patch = threadIdx.x; patch < nbr * nbc; patch += blockDim.x) {
    int I = patch / nbc, J = patch % nbc;
    int r0 = I * STIV_BR, c0 = J * STIV_BC;
    // per column half: rb[row][lo xyz, hi xyz] of its three rows; pb[pole]:
    // FP32, rounded outward
    float pb[2][6];
    auto vbox_of = [&](int vid, float* o) {
      if (use_sm) {
        for (int c = 0; c < 3; ++c) { o[c] = vbs[c * nv + vid]; o[3 + c] = vbs[(3 + c) * nv + vid]; }
      } else {
        for (int c = 0; c < 3; ++c) {
          double x0 = vload(X, mixed, base + (size_t)c * nv + vid), x1 = vload(X, mixed, base + (size_t)(3 + c) * nv + vid);
          o[c] = __double2float_rd(fmin(x0, x1));
          o[3 + c] = __double2float_ru(fmax(x0, x1));
        }
      }
    };
#pragma unroll
    for (int q = 0; q < 2; ++q) {
      bool has = q == 0 ? I == 0 : I == nbr - 1;
      if (has) vbox_of(W * (P + 1) + q, pb[q]);
      else for (int c = 0; c < 3; ++c) { pb[q][c] = INFINITY; pb[q][3 + c] = -INFINITY; }
    }
    float* B = pbox + ((size_t)v * pstride + patch) * STIV_PBOX;
    float plo[3] = {INFINITY, INFINITY, INFINITY}, phi[3] = {-INFINITY, -INFINITY, -INFINITY};
#pragma unroll 1
    for (int h = 0; h < 2; ++h) {
      float rb[3][6];
#pragma unroll
      for (int rr = 0; rr < 3; ++rr) {
#pragma unroll
        for (int cc = 0; cc <= 2; ++cc) {
          int col = c0 + 2 * h + cc; if (col >= W) col -= W;
          float o[6];
          vbox_of((r0 + rr) * W + col, o);
#pragma unroll
          for (int c = 0; c < 3; ++c) {
            rb[rr][c] = cc == 0 ? o[c] : fminf(rb[rr][c], o[c]);
            rb[rr][3 + c] = cc == 0 ? o[3 + c] : fmaxf(rb[rr][3 + c], o[3 + c]);
          }
        }
      }
#pragma unroll
      for (int b = 0; b < 2; ++b) {
        float lo[3], hi[3];
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          lo[c] = fminf(fminf(rb[b][c], rb[b + 1][c]), pb[b][c]);
          hi[c] = fmaxf(fmaxf(rb[b][3 + c], rb[b + 1][3 + c]), pb[b][3 + c]);
          plo[c] = fminf(plo[c], lo[c]);
          phi[c] = fmaxf(phi[c], hi[c]);
        }
        float4* C = (float4*)(B + STIV_PBOX_CELLS) + 2 * (2 * b + h);
        C[0] = make_float4(lo[0], lo[1], lo[2], 0.f);
        C[1] = make_float4(hi[0], hi[1], hi[2], 0.f);
      }
    }
    for (int c = 0; c < 3; ++c) { B[c] = plo[c]; B[3 + c] = phi[c]; }
  }
}

// grid[0..2] origin, [3..5] cell size, [6..8] cells per axis, [9..11] periodic flag, [12] h_m
__global__ void __launch_bounds__(1024) grid_kernel(int n, const double* vbox, double Lx, double Ly, double Lz,
                                                    double* grid) {
  __shared__ double sdiag[1024], slo[3][1024], shi[3][1024];
  __shared__ int scnt[1024];
  double d = 0.0, lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
  int nvalid = 0;
  for (int v = threadIdx.x; v < n; v += 1024) {
    if (!(vbox[6 * v] <= vbox[6 * v + 3])) continue;   // inverted: a vesicle left out (bad order)
    ++nvalid;
    double e0 = vbox[6 * v + 3] - vbox[6 * v], e1 = vbox[6 * v + 4] - vbox[6 * v + 1], e2 = vbox[6 * v + 5] - vbox[6 * v + 2];
    d += sqrt(e0 * e0 + e1 * e1 + e2 * e2);
    for (int c = 0; c < 3; ++c) { lo[c] = fmin(lo[c], vbox[6 * v + c]); hi[c] = fmax(hi[c], vbox[6 * v + 3 + c]); }
  }
  sdiag[threadIdx.x] = d;
  scnt[threadIdx.x] = nvalid;
  for (int c = 0; c < 3; ++c) { slo[c][threadIdx.x] = lo[c]; shi[c][threadIdx.x] = hi[c]; }
  __syncthreads();
  for (int s = 512; s > 0; s >>= 1) {
    if (threadIdx.x < s) {
      sdiag[threadIdx.x] += sdiag[threadIdx.x + s];
      scnt[threadIdx.x] += scnt[threadIdx.x + s];
      for (int c = 0; c < 3; ++c) {
        slo[c][threadIdx.x] = fmin(slo[c][threadIdx.x], slo[c][threadIdx.x + s]);
        shi[c][threadIdx.x] = fmax(shi[c][threadIdx.x], shi[c][threadIdx.x + s]);
      }
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    double hm = sdiag[0] / (scnt[0] > 0 ? scnt[0] : 1);
    if (!(hm > 0.0)) hm = 1.0;
    for (int c = 0; c < 3; ++c)
      if (!(slo[c][0] <= shi[c][0])) { slo[c][0] = 0.0; shi[c][0] = 0.0; }   // no valid box
    double L[3] = {Lx, Ly, Lz};
    for (int c = 0; c < 3; ++c) {
      if (L[c] > 0.0) {
        double G = floor(L[c] / hm);
        if (G < 1.0) G = 1.0;
        if (G > 256.0) G = 256.0;
        grid[c] = 0.0; grid[3 + c] = L[c] / G; grid[6 + c] = G; grid[9 + c] = 1.0;
      } else {
        double ext = shi[c][0] - slo[c][0];
        double h = hm;
        if (ext / h > 255.0) h = ext / 255.0;
        grid[c] = slo[c][0]; grid[3 + c] = h; grid[6 + c] = floor(ext / h) + 1.0; grid[9 + c] = 0.0;
      }
    }
    grid[12] = hm;
  }
}

__device__ __forceinline__ void cell_range(const double* grid, const double* box, int c, int& u0, int& u1) {
  double o = grid[c], h = grid[3 + c];
  const double slack = 1e-6;  // cells; covers rounding of the divisions
  u0 = (int)floor((box[c] - o) / h - slack);
  u1 = (int)floor((box[3 + c] - o) / h + slack);
  if (grid[9 + c] == 0.0) {  // free axis: clamp to the grid
    int G = (int)grid[6 + c];
    u0 = max(0, min(u0, G - 1));
    u1 = max(0, min(u1, G - 1));
  }
  u0 = max(u0, -500); u1 = min(u1, 500);
}

__global__ void cell_count_kernel(int n, const double* vbox, const double* grid, int32_t* cnt) {
  int v = blockIdx.x * blockDim.x + threadIdx.x;
  if (v >= n) return;
  if (!(vbox[6 * v] <= vbox[6 * v + 3])) { cnt[v] = 0; return; }   // inverted box: no cells
  int c = 1;
  for (int a = 0; a < 3; ++a) { int u0, u1; cell_range(grid, vbox + 6 * v, a, u0, u1); c *= (u1 - u0 + 1); }
  cnt[v] = c;
}

// Exclusive scan of n+1 ints (last = total), one CTA.
__global__ void __launch_bounds__(1024) scan1_kernel(const int32_t* in, int n, int32_t* out) {
  __shared__ int32_t part[1024];
  int per = (n + 1023) / 1024;
  int lo = threadIdx.x * per, hi = min(lo + per, n);
  int32_t s = 0;
  for (int i = lo; i < hi; ++i) s += in[i];
  part[threadIdx.x] = s;
  __syncthreads();
  for (int off = 1; off < 1024; off <<= 1) {
    int32_t v = threadIdx.x >= off ? part[threadIdx.x - off] : 0;
    __syncthreads();
    part[threadIdx.x] += v;
    __syncthreads();
  }
  int32_t run = threadIdx.x ? part[threadIdx.x - 1] : 0;
  for (int i = lo; i < hi; ++i) { out[i] = run; run += in[i]; }
  if (threadIdx.x == 1023) out[n] = part[1023];
}

__device__ __forceinline__ uint32_t spread10(uint32_t x) {
  x &= 0x3FF;
  x = (x | (x << 16)) & 0x030000FF;
  x = (x | (x << 8)) & 0x0300F00F;
  x = (x | (x << 4)) & 0x030C30C3;
  x = (x | (x << 2)) & 0x09249249;
  return x;
}

__global__ void cell_emit_kernel(int n, const double* vbox, const double* grid, const int32_t* off, int64_t R,
                                 uint64_t* key, int32_t* val, int32_t* rbox, int32_t* rcell, int64_t* ctr) {
  int v = blockIdx.x * blockDim.x + threadIdx.x;
  if (v >= n) return;
  int lo[3], hi[3], G[3];
  for (int a = 0; a < 3; ++a) { cell_range(grid, vbox + 6 * v, a, lo[a], hi[a]); G[a] = (int)grid[6 + a]; }
  int64_t r = off[v];
  if (v == n - 1) ctr[8] = off[n];
  if (!(vbox[6 * v] <= vbox[6 * v + 3])) return;   // inverted box: no cells
  for (int x = lo[0]; x <= hi[0]; ++x)
    for (int y = lo[1]; y <= hi[1]; ++y)
      for (int z = lo[2]; z <= hi[2]; ++z, ++r) {
        if (r >= R) { atomicOr((unsigned long long*)&ctr[STIV_C_STATUS], STIV_F_WORK_OVERFLOW); return; }
        int w[3] = {x, y, z};
        for (int a = 0; a < 3; ++a) w[a] = ((w[a] % G[a]) + G[a]) % G[a];
        key[r] = spread10(w[0]) | (spread10(w[1]) << 1) | (spread10(w[2]) << 2);
        val[r] = (int32_t)r;
        rbox[r] = v;
        rcell[r] = (x + 512) | ((y + 512) << 10) | ((z + 512) << 20);
      }
}

__device__ __forceinline__ bool bbi(const double* a, const double* b) {
  return a[0] <= b[3] && b[0] <= a[3] && a[1] <= b[4] && b[1] <= a[4] && a[2] <= b[5] && b[2] <= a[5];
}

// Alg. 1, per-cell loop: every record against the later records of its cell.
__global__ void cell_pairs_kernel(const int64_t* nrec_dev, int64_t R, const uint64_t* key, const int32_t* val,
                                  const int32_t* rbox, const int32_t* rcell, const double* vbox,
                                  const double* grid, double Lx, double Ly, double Lz, int64_t Q,
                                  uint64_t* pkey, int32_t* pval, int64_t* ctr, int nb) {
  int64_t nrec = *nrec_dev; if (nrec > R) nrec = R;
  int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= nrec) return;
  double L[3] = {Lx, Ly, Lz};
  int G[3] = {(int)grid[6], (int)grid[7], (int)grid[8]};
  int ra = val[k];
  int ba = rbox[ra], ca = rcell[ra];
  for (int64_t q = k + 1; q < nrec && key[q] == key[k]; ++q) {
    int rb = val[q];
    int bb = rbox[rb], cb = rcell[rb];
    if (bb == ba) continue;
    int s[3];
    bool ok = true;
    for (int a = 0; a < 3; ++a) {
      int du = ((ca >> (10 * a)) & 0x3FF) - ((cb >> (10 * a)) & 0x3FF);
      if (L[a] > 0.0) {
        s[a] = du / G[a];
        if (s[a] * G[a] != du || s[a] < -1 || s[a] > 1) ok = false;
      } else {
        s[a] = 0;
        if (du != 0) ok = false;
      }
    }
    if (!ok) continue;
    int i = ba, j = bb;
    if (i > j) { i = bb; j = ba; s[0] = -s[0]; s[1] = -s[1]; s[2] = -s[2]; }
    double bj[6];
    for (int a = 0; a < 3; ++a) {
      bj[a] = vbox[6 * j + a]; bj[3 + a] = vbox[6 * j + 3 + a];
      if (s[a] != 0) { double sh = s[a] * L[a]; bj[a] = bj[a] + sh; bj[3 + a] = bj[3 + a] + sh; }
    }
    if (!bbi(vbox + 6 * i, bj)) continue;
    int code = 9 * (s[0] + 1) + 3 * (s[1] + 1) + (s[2] + 1);
    unsigned long long slot = atomicAdd((unsigned long long*)&ctr[9], 1ull);
    if ((int64_t)slot < Q) {
      pkey[slot] = ((uint64_t)i << (nb + 5)) | ((uint64_t)j << 5) | (uint64_t)code;
      pval[slot] = 0;
    } else {
      atomicOr((unsigned long long*)&ctr[STIV_C_STATUS], STIV_F_WORK_OVERFLOW);
    }
  }
}

// Alg. 1, final step: unique sorted keys -> output pair list; one CTA.
__global__ void __launch_bounds__(1024) unique_pairs_kernel(const int64_t* nkey_dev, int64_t Q, const uint64_t* key,
                                                            int64_t cap, int32_t* oi, int32_t* oj, int32_t* os,
                                                            int64_t* ctr, int nb) {
  __shared__ int32_t part[1024];
  int64_t n = *nkey_dev; if (n > Q) n = Q;
  int64_t per = (n + 1023) / 1024;
  int64_t lo = threadIdx.x * per, hi = lo + per < n ? lo + per : n;
  int32_t c = 0;
  for (int64_t k = lo; k < hi; ++k) c += (k == 0 || key[k] != key[k - 1]);
  part[threadIdx.x] = c;
  __syncthreads();
  for (int off = 1; off < 1024; off <<= 1) {
    int32_t v = threadIdx.x >= off ? part[threadIdx.x - off] : 0;
    __syncthreads();
    part[threadIdx.x] += v;
    __syncthreads();
  }
  int64_t run = threadIdx.x ? part[threadIdx.x - 1] : 0;
  for (int64_t k = lo; k < hi; ++k) {
    if (k == 0 || key[k] != key[k - 1]) {
      if (run < cap) {
        uint64_t x = key[k];
        oi[run] = (int32_t)(x >> (nb + 5));
        oj[run] = (int32_t)((x >> 5) & ((1ull << nb) - 1));
        os[run] = (int32_t)(x & 31);
      }
      ++run;
    }
  }
  if (threadIdx.x == 1023) {
    int64_t total = part[1023];
    ctr[STIV_C_PAIRS] = total;
    if (total > cap) atomicOr((unsigned long long*)&ctr[STIV_C_STATUS], STIV_F_PAIRS_OVERFLOW);
  }
}

}  // namespace

// Host side of steps 1-6.  ws: scratch views prepared by the caller.
int stiv_broad_phase(stiv_handle* h, cudaStream_t st, int n, int p_max, const int32_t* p_dev, const int64_t* voff,
                     const void* X, const stiv_pairs* cand, detect_ws& w, int64_t* ctr) {
  int mixed = h->prm.precision == STIV_MIXED;
  const double* L = h->prm.box_L;
  {
  STIV_PROF(h, st, "boxes");
  // per-vertex boxes in shared memory up to 96 KB (orders up to P = 44)
  size_t nv_max = (size_t)(w.fstride / 8);
  size_t vb_cap = 6 * nv_max * sizeof(float) <= 96 * 1024 ? 6 * nv_max : 0;
  size_t bsmem = vb_cap * sizeof(float);
  auto bk = mixed ? boxes_kernel<true> : boxes_kernel<false>;
  STIV_CUDA(h, cudaFuncSetAttribute(bk, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bsmem));
  bk<<<n, 256, bsmem, st>>>(n, p_dev, voff, X, mixed, h->prm.d_m, L[0], L[1], L[2], w.vbox, w.pbox,
                                      w.pstride, w.vorg, w.fprep, w.fstride, ctr, vb_cap, p_max);
  }
  {
  STIV_PROF_N(h, st, "cells", 4);
  grid_kernel<<<1, 1024, 0, st>>>(n, w.vbox, L[0], L[1], L[2], w.grid);
  cell_count_kernel<<<(n + 127) / 128, 128, 0, st>>>(n, w.vbox, w.grid, w.cell_count);
  scan1_kernel<<<1, 1024, 0, st>>>(w.cell_count, n, w.cell_off);
  cell_emit_kernel<<<(n + 127) / 128, 128, 0, st>>>(n, w.vbox, w.grid, w.cell_off, w.R, w.rec_key, w.rec_val,
                                                    w.rec_box, w.rec_cell, ctr);
  }
  STIV_LAUNCH(h);
  // records: ctr[8] = count; sort by Morton id (wrapped cells < 256 per axis: 24 bits)
  int rc;
  {
  STIV_PROF_N(h, st, "sort_cells", stiv_sort_kernels(24));
  rc = stiv_sort_pairs_impl(st, w.R, 24, w.rec_key, w.rec_val, w.rec_key2, w.rec_val2, w.sort_scratch,
                                w.sort_scratch_bytes, &ctr[8]);
  }
  // candidate keys i << (nb + 5) | j << 5 | shift code: nb bits per vesicle index
  int nb = 1;
  while ((1 << nb) < n) ++nb;
  int pair_bits = 2 * nb + 5;
  if (rc) return rc;
  {
  STIV_PROF(h, st, "cell_pairs");
  cell_pairs_kernel<<<(unsigned)((w.R + 127) / 128), 128, 0, st>>>(&ctr[8], w.R, w.rec_key2, w.rec_val2, w.rec_box,
                                                                   w.rec_cell, w.vbox, w.grid, L[0], L[1], L[2],
                                                                   w.Q, w.pkey, w.pval, ctr, nb);
  }
  STIV_LAUNCH(h);
  {
    STIV_PROF_N(h, st, "sort_pairs", stiv_sort_kernels(pair_bits));
    rc = stiv_sort_pairs_impl(st, w.Q, pair_bits, w.pkey, w.pval, w.pkey2, w.pval2, w.sort_scratch,
                              w.sort_scratch_bytes, &ctr[9]);
  }
  if (rc) return rc;
  {
    STIV_PROF(h, st, "unique_pairs");
    unique_pairs_kernel<<<1, 1024, 0, st>>>(&ctr[9], w.Q, w.pkey2, cand->capacity, cand->i, cand->j, cand->shift,
                                            ctr, nb);
  }
  STIV_LAUNCH(h);
  return STIV_OK;
}

// Contact volumes (Eq. 3.2, App. A) and their gradient with respect to the
// end-of-step positions X1 (Sec. 3.1.2, Sec. 3.3.2), per contact and summed
// per vesicle pair (Alg. 2); the adjoint of the upsampling back to SH
// coefficients; ordering of the contact list.
//
// Per contact, with positions Y = X0 + tau D at the contact time tau and
// D = X1 - X0:
//   V = 1/2 (1 - tau) sqrt((eps dt)^2 |m|^2 + (D_rel . m)^2)
// which is Eq. 3.2, (t - tau_I) sqrt(eps^2 + (U . n)^2) |t|, with t - tau_I =
// (1 - tau) dt, U = D_rel / dt the velocity of the contact point relative to
// the opposite primitive, n = m / |m| and |t| = |m| / 2.  VF: m = (x1-x0) x
// (x2-x0), D_rel = D_p - sum_k beta_k D_k.  EE: m = d1 x d2 (same weight),
// D_rel = D_q(u) - D_p(s).
//
// The gradient is reverse mode written out by hand: V depends on X1 through
// D, through Y, through the weights (beta or s, u: least-squares solutions
// of the inside test) and through tau, an implicit function of X1 via
// f(tau) = 0 (Eq. 3.1): d tau / dX1_q = -tau (df/dY_q) / f'(tau).
#include "stiv_internal.cuh"

#include <math.h>

namespace {

__device__ __forceinline__ d3 mk(double x, double y, double z) { return {x, y, z}; }
__device__ __forceinline__ d3 operator+(d3 a, d3 b) { return {a.x + b.x, a.y + b.y, a.z + b.z}; }
__device__ __forceinline__ d3 operator-(d3 a, d3 b) { return {a.x - b.x, a.y - b.y, a.z - b.z}; }
__device__ __forceinline__ d3 operator-(d3 a) { return {-a.x, -a.y, -a.z}; }
__device__ __forceinline__ d3 operator*(double s, d3 a) { return {s * a.x, s * a.y, s * a.z}; }
__device__ __forceinline__ double dot(d3 a, d3 b) { return fma(a.z, b.z, fma(a.y, b.y, a.x * b.x)); }
__device__ __forceinline__ d3 cross(d3 a, d3 b) {
  return {fma(a.y, b.z, -(a.z * b.y)), fma(a.z, b.x, -(a.x * b.z)), fma(a.x, b.y, -(a.y * b.x))};
}

struct contact_in {
  int type;       // 0, 1: VF (point 0 = vertex, 1..3 triangle); 2: EE (0,1 = edge of i; 2,3 = edge of j)
  d3 X0[4], X1[4];
  double tau;
  double w1, w2;  // inside-test weights of the detection at tau (VF: b1, b2; EE: s, u)
};

// V and (optionally) dV/dX1 [4] (g1) and dV/dX0 [4] (g0) of one contact.
// vabs: U_k read as the absolute velocity of the contact point (the literal
// reading: VF the vertex's displacement, EE that of the point p(s) on the
// first edge) instead of the velocity relative to the opposite primitive.
// Reverse mode: adjoints of the positions at tau (Yb), of the displacements
// (Db) and of tau (taub); with Y = X0 + tau D, D = X1 - X0 and tau moving
// along f(tau; X) = 0, dV/dX1 = Db + tau Yb - taub tau fY / f' and
// dV/dX0 = -Db + (1 - tau) Yb - taub (1 - tau) fY / f'.  dm2 = d_m^2 > 0:
// tau is a root of g = f^2 - d_m^2 |m|^2 (Eq. 3.1, degree six) and fY, f'
// are those of g: gY = 2 f fY - d_m^2 d|m|^2/dY, g' = sum gY . D.
// VAR = false compiles the common case (relative velocity, d_m = 0, no X0
// rows) without the variants' code.
template <bool VAR>
__device__ double stiv_one(const contact_in& c, double e2, int vabs, double dm2, d3* g, d3* g0) {
  if (!VAR) { vabs = 0; dm2 = 0.0; g0 = nullptr; }
  d3 D[4], Y[4];
  for (int q = 0; q < 4; ++q) { D[q] = c.X1[q] - c.X0[q]; Y[q] = mk(fma(c.tau, D[q].x, c.X0[q].x), fma(c.tau, D[q].y, c.X0[q].y), fma(c.tau, D[q].z, c.X0[q].z)); }
  const double tau = c.tau;
  d3 Yb[4] = {}, Db[4] = {}, fY[4];
  double taub;
  double V;
  if (c.type < 2) {
    d3 a = Y[2] - Y[1], b = Y[3] - Y[1], cc = Y[0] - Y[1];
    double d00 = dot(a, a), d01 = dot(a, b), d11 = dot(b, b), d20 = dot(cc, a), d21 = dot(cc, b);
    double den = d00 * d11 - d01 * d01, iden = 1.0 / den;
    (void)d20; (void)d21;
    double b1 = c.w1, b2 = c.w2, b0 = 1.0 - b1 - b2;
    d3 m = cross(a, b);
    d3 Dr = vabs ? D[0] : D[0] - (b0 * D[1] + b1 * D[2] + b2 * D[3]);
    double dm = dot(Dr, m);
    double Q = e2 * dot(m, m) + dm * dm;
    double rS = rsqrt(Q);                  // 1 / sqrt(Q): no division in the adjoint below
    double S = Q > 0.0 ? Q * rS : 0.0;
    V = 0.5 * (1.0 - tau) * S;
    if (!g && !g0) return V;
    double Qb = 0.25 * (1.0 - tau) * rS;   // dV/dQ
    d3 mb = (2.0 * Qb) * (e2 * m + dm * Dr);
    d3 Drb = (2.0 * Qb * dm) * m;
    taub = -0.5 * S;
    double bb0 = 0.0, bb1 = 0.0, bb2 = 0.0;
    if (vabs) {
      Db[0] = Drb;
    } else {
      Db[0] = Drb; Db[1] = -b0 * Drb; Db[2] = -b1 * Drb; Db[3] = -b2 * Drb;
      bb0 = -dot(Drb, D[1]); bb1 = -dot(Drb, D[2]); bb2 = -dot(Drb, D[3]);
    }
    double g1 = bb1 - bb0, g2 = bb2 - bb0;
    d3 ab = cross(b, mb), bbv = cross(mb, a), cb = mk(0, 0, 0);
    // least squares beta = M^-1 G^T c, G = [a b]
    double z1 = (d11 * g1 - d01 * g2) * iden, z2 = (d00 * g2 - d01 * g1) * iden;
    d3 w = z1 * a + z2 * b;
    d3 res = cc - (b1 * a + b2 * b);
    cb = cb + w;
    ab = ab + z1 * res - b1 * w;
    bbv = bbv + z2 * res - b2 * w;
    Yb[2] = ab; Yb[3] = bbv; Yb[0] = cb; Yb[1] = -(ab + bbv + cb);
    // df/dY of f = c . (a x b)
    fY[0] = m; fY[2] = cross(b, cc); fY[3] = cross(cc, a); fY[1] = -(fY[0] + fY[2] + fY[3]);
    if (dm2 > 0.0) {   // d|m|^2 / dY2 = 2 b x m, dY3 = 2 m x a
      double f2 = 2.0 * dot(cc, m);
      d3 mY2 = 2.0 * cross(b, m), mY3 = 2.0 * cross(m, a), mY1 = -(mY2 + mY3);
      fY[0] = f2 * fY[0];
      fY[1] = f2 * fY[1] - dm2 * mY1;
      fY[2] = f2 * fY[2] - dm2 * mY2;
      fY[3] = f2 * fY[3] - dm2 * mY3;
    }
  } else {
    d3 d1 = Y[1] - Y[0], d2 = Y[3] - Y[2], r = Y[0] - Y[2];
    double A = dot(d1, d1), B = dot(d1, d2), E = dot(d2, d2), C = dot(d1, r), F = dot(d2, r);
    double den = A * E - B * B, iden = 1.0 / den;
    (void)C; (void)F;
    double s = c.w1, u = c.w2;
    d3 m = cross(d1, d2);
    d3 Dp = (1.0 - s) * D[0] + s * D[1];
    d3 Dr = vabs ? Dp : ((1.0 - u) * D[2] + u * D[3]) - Dp;
    double dm = dot(Dr, m);
    double Q = e2 * dot(m, m) + dm * dm;
    double rS = rsqrt(Q);                  // 1 / sqrt(Q): no division in the adjoint below
    double S = Q > 0.0 ? Q * rS : 0.0;
    V = 0.5 * (1.0 - tau) * S;
    if (!g && !g0) return V;
    double Qb = 0.25 * (1.0 - tau) * rS;   // dV/dQ
    d3 mb = (2.0 * Qb) * (e2 * m + dm * Dr);
    d3 Drb = (2.0 * Qb * dm) * m;
    taub = -0.5 * S;
    double sb, ub;
    if (vabs) {
      Db[0] = (1.0 - s) * Drb; Db[1] = s * Drb;
      sb = dot(Drb, D[1] - D[0]); ub = 0.0;
    } else {
      Db[2] = (1.0 - u) * Drb; Db[3] = u * Drb; Db[0] = -(1.0 - s) * Drb; Db[1] = -s * Drb;
      sb = -dot(Drb, D[1] - D[0]); ub = dot(Drb, D[3] - D[2]);
    }
    d3 d1b = cross(d2, mb), d2b = cross(mb, d1);
    // least squares (s, u) = M^-1 G^T c, G = [d1, -d2], c = -r; M = [[A, -B], [-B, E]]
    double z1 = (E * sb + B * ub) * iden, z2 = (B * sb + A * ub) * iden;
    d3 w = z1 * d1 - z2 * d2;
    d3 res = (-r) - (s * d1 - u * d2);
    d3 rb = -w;
    d1b = d1b + z1 * res - s * w;
    d2b = d2b - (z2 * res - u * w);
    Yb[1] = d1b; Yb[0] = -d1b + rb; Yb[3] = d2b; Yb[2] = -d2b - rb;
    // df/dY of f = c . (d1 x d2), c = Y2 - Y0
    d3 ce = Y[2] - Y[0];
    d3 fc = m, f1 = cross(d2, ce), f2 = cross(ce, d1);
    fY[2] = fc - f2; fY[0] = -fc - f1; fY[1] = f1; fY[3] = f2;
    if (dm2 > 0.0) {   // d|m|^2 / dd1 = 2 d2 x m, dd2 = 2 m x d1
      double ff = 2.0 * dot(ce, m);
      d3 mY1 = 2.0 * cross(d2, m), mY3 = 2.0 * cross(m, d1);
      fY[0] = ff * fY[0] + dm2 * mY1;
      fY[1] = ff * fY[1] - dm2 * mY1;
      fY[2] = ff * fY[2] + dm2 * mY3;
      fY[3] = ff * fY[3] - dm2 * mY3;
    }
  }
  double fp = 0.0;
  for (int q = 0; q < 4; ++q) { taub += dot(Yb[q], D[q]); fp += dot(fY[q], D[q]); }
  if (g)
    for (int q = 0; q < 4; ++q) g[q] = (Db[q] + tau * Yb[q]) - ((taub * tau / fp) * fY[q]);
  if (g0)
    for (int q = 0; q < 4; ++q) g0[q] = ((1.0 - tau) * Yb[q] - Db[q]) - ((taub * (1.0 - tau) / fp) * fY[q]);
  return V;
}

struct stiv_args {
  const int32_t* pv;
  const int64_t* voff;
  const void* X;
  int mixed;
  double L[3];
  const int32_t* ci; const int32_t* cj; const int32_t* cs;
  const int32_t* pair; const int32_t* type; const int32_t* a; const int32_t* b; const double* tau; const double* w;
  const int64_t* counts;
  int64_t cap;
  double e2;
  double dm2;      // d_m^2 (0: the cubic of Eq. 3.1)
  int vabs;
  double* Vc;
  double* grad;
  double* grad0;   // dV/dX0 rows (or NULL)
  int32_t* gves;
  int32_t* gvid;
};

__device__ __forceinline__ d3 vpos(const stiv_args& A, int v, int t, int k, const int* s) {
  int P = 2 * A.pv[v], nv = stiv_nverts(P);
  size_t base = A.voff[v] + (size_t)t * 3 * nv + k;
  double x[3];
  for (int c = 0; c < 3; ++c) {
    size_t idx = base + (size_t)c * nv;
    x[c] = A.mixed ? (double)((const float*)A.X)[idx] : ((const double*)A.X)[idx];
    if (s && s[c] != 0) x[c] = x[c] + s[c] * A.L[c];
  }
  return {x[0], x[1], x[2]};
}

__device__ __forceinline__ int64_t n_contacts(const int64_t* counts, int64_t cap) {
  int64_t n = counts[STIV_C_VF] + counts[STIV_C_EE];
  return n < cap ? n : cap;
}

// VAR: the variants (absolute velocity, d_m > 0, X0 rows) in an instance of
// their own; the common one fits 128 registers (4 CTAs per SM).
template <bool VAR>
__global__ void __launch_bounds__(128, 4) stiv_kernel(stiv_args A) {
  int64_t n = n_contacts(A.counts, A.cap);
  for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x) {
    int r = A.pair[k], ty = A.type[k], pa = A.a[k], pb = A.b[k];
    int vi = A.ci[r], vj = A.cj[r], code = A.cs[r];
    int s1[3] = {code / 9 - 1, (code / 3) % 3 - 1, code % 3 - 1};
    int ves[4], vid[4];
    const int* sh[4];
    if (ty < 2) {
      int vv = ty == 0 ? vi : vj, vt = ty == 0 ? vj : vi;
      int tv[3];
      stiv_tri_verts(2 * A.pv[vt], pb, tv);
      ves[0] = vv; vid[0] = pa;
      for (int q = 0; q < 3; ++q) { ves[1 + q] = vt; vid[1 + q] = tv[q]; }
    } else {
      int u, v;
      stiv_edge_verts(2 * A.pv[vi], pa, &u, &v); ves[0] = vi; vid[0] = u; ves[1] = vi; vid[1] = v;
      stiv_edge_verts(2 * A.pv[vj], pb, &u, &v); ves[2] = vj; vid[2] = u; ves[3] = vj; vid[3] = v;
    }
    contact_in c;
    c.type = ty; c.tau = A.tau[k]; c.w1 = A.w[2 * k]; c.w2 = A.w[2 * k + 1];
    for (int q = 0; q < 4; ++q) {
      sh[q] = ves[q] == vj ? s1 : nullptr;
      c.X0[q] = vpos(A, ves[q], 0, vid[q], sh[q]);
      c.X1[q] = vpos(A, ves[q], 1, vid[q], sh[q]);
    }
    d3 g[4], g0[4];
    double V = stiv_one<VAR>(c, A.e2, A.vabs, A.dm2, A.grad ? g : nullptr, A.grad0 ? g0 : nullptr);
    if (A.Vc) A.Vc[k] = V;
    if (A.grad) {
      for (int q = 0; q < 4; ++q) {
        A.grad[12 * k + 3 * q + 0] = g[q].x; A.grad[12 * k + 3 * q + 1] = g[q].y; A.grad[12 * k + 3 * q + 2] = g[q].z;
        A.gves[4 * k + q] = ves[q]; A.gvid[4 * k + q] = vid[q];
      }
    }
    if (VAR && A.grad0)
      for (int q = 0; q < 4; ++q) {
        A.grad0[12 * k + 3 * q + 0] = g0[q].x; A.grad0[12 * k + 3 * q + 1] = g0[q].y;
        A.grad0[12 * k + 3 * q + 2] = g0[q].z;
      }
  }
}

// Per candidate pair: sum of its contacts' V (contacts sorted by pair); one
// warp per pair, fixed summation order.
__global__ void vpair_kernel(const int32_t* pair, const int64_t* counts, int64_t ccap, const double* Vc,
                             int64_t pcap, double* Vp) {
  int lane = threadIdx.x & 31;
  int64_t np = counts[STIV_C_PAIRS]; if (np > pcap) np = pcap;
  int64_t n = n_contacts(counts, ccap);
  int64_t w0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5, nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t r = w0; r < np; r += nw) {
    int64_t lo = 0, hi = n;
    while (lo < hi) { int64_t mid = (lo + hi) >> 1; if (pair[mid] < r) lo = mid + 1; else hi = mid; }
    double s = 0.0;
    for (int64_t k = lo + lane; k < n && pair[k] == r; k += 32) s += Vc[k];
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    if (lane == 0) Vp[r] = s;
  }
}

// Contact ordering by (pair, type, a, b): counting sort by pair, then each
// pair's segment sorted by its (type, a, b) key.
__global__ void pair_count_kernel(const int64_t* ctr, int64_t C, const int32_t* rp, int32_t* cnt) {
  int64_t n = ctr[11]; if (n > C) n = C;
  for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x)
    atomicAdd(&cnt[rp[k]], 1);
}

// Exclusive scan of the per-pair counts (one CTA); counts pairs with contacts.
__global__ void __launch_bounds__(1024) pair_scan_kernel(const int64_t* ctr_r, int64_t pcap, const int32_t* cnt,
                                                         int32_t* off, int64_t* ctr_w) {
  __shared__ int32_t part[1024];
  __shared__ int32_t nz[1024];
  int64_t np = ctr_r[STIV_C_PAIRS]; if (np > pcap) np = pcap;
  int64_t per = (np + 1023) / 1024;
  int64_t lo = threadIdx.x * per, hi = lo + per < np ? lo + per : np;
  int32_t s = 0, z = 0;
  for (int64_t i = lo; i < hi; ++i) { s += cnt[i]; z += cnt[i] > 0; }
  part[threadIdx.x] = s; nz[threadIdx.x] = z;
  __syncthreads();
  for (int o = 1; o < 1024; o <<= 1) {
    int32_t v = threadIdx.x >= o ? part[threadIdx.x - o] : 0;
    __syncthreads();
    part[threadIdx.x] += v;
    __syncthreads();
  }
  int32_t run = threadIdx.x ? part[threadIdx.x - 1] : 0;
  for (int64_t i = lo; i < hi; ++i) { off[i] = run; run += cnt[i]; }
  if (threadIdx.x == 1023) off[np] = part[1023];
  for (int o = 512; o > 0; o >>= 1) {
    if (threadIdx.x < o) nz[threadIdx.x] += nz[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) ctr_w[STIV_C_CPAIRS] = nz[0];
}

__global__ void pair_scatter_kernel(const int64_t* ctr, int64_t C, const int32_t* rp, const int32_t* rt,
                                    const int32_t* ra, const int32_t* rb, const int32_t* off, int32_t* fill,
                                    unsigned long long* seg) {
  int64_t n = ctr[11]; if (n > C) n = C;
  for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x) {
    int r = rp[k];
    int slot = off[r] + atomicAdd(&fill[r], 1);
    unsigned key = ((unsigned)rt[k] << 30) | ((unsigned)ra[k] << 15) | (unsigned)rb[k];
    seg[slot] = ((unsigned long long)key << 32) | (unsigned long long)(unsigned)k;
  }
}

constexpr int SEG_SMEM = 4096;   // entries sorted in shared memory per pass (32 KB)

__device__ void bitonic_smem(unsigned long long* x, int n2) {
  for (int k = 2; k <= n2; k <<= 1)
    for (int j = k >> 1; j > 0; j >>= 1) {
      for (int i = threadIdx.x; i < n2; i += blockDim.x) {
        int l = i ^ j;
        if (l > i) {
          unsigned long long a = x[i], b = x[l];
          bool up = (i & k) == 0;
          if ((a > b) == up) { x[i] = b; x[l] = a; }
        }
      }
      __syncthreads();
    }
}

// One CTA per pair: sort its segment; long segments are sorted in chunks and
// merged (each element placed by binary search in the other run).
__global__ void __launch_bounds__(1024) pair_sort_kernel(const int64_t* ctr, int64_t pcap, const int32_t* off,
                                                         unsigned long long* seg, unsigned long long* tmp) {
  __shared__ unsigned long long x[SEG_SMEM];
  int64_t np = ctr[STIV_C_PAIRS]; if (np > pcap) np = pcap;
  for (int64_t r = blockIdx.x; r < np; r += gridDim.x) {
    int o = off[r], len = off[r + 1] - o;
    if (len <= 1) continue;
    for (int c0 = 0; c0 < len; c0 += SEG_SMEM) {
      int cl = min(SEG_SMEM, len - c0);
      int n2 = 1;
      while (n2 < cl) n2 <<= 1;
      for (int i = threadIdx.x; i < n2; i += blockDim.x) x[i] = i < cl ? seg[o + c0 + i] : ~0ull;
      __syncthreads();
      bitonic_smem(x, n2);
      for (int i = threadIdx.x; i < cl; i += blockDim.x) seg[o + c0 + i] = x[i];
      __syncthreads();
    }
    unsigned long long* src = seg + o;
    unsigned long long* dst = tmp + o;
    for (int wdt = SEG_SMEM; wdt < len; wdt <<= 1) {
      for (int i = threadIdx.x; i < len; i += blockDim.x) {
        int run = i / (2 * wdt), a0 = run * 2 * wdt, a1 = min(a0 + wdt, len), b1 = min(a0 + 2 * wdt, len);
        unsigned long long v = src[i];
        int pos;
        if (i < a1) {  // element of run A: rank among B elements smaller than v
          int lo = a1, hi = b1;
          while (lo < hi) { int mid = (lo + hi) >> 1; if (src[mid] < v) lo = mid + 1; else hi = mid; }
          pos = a0 + (i - a0) + (lo - a1);
        } else {       // element of run B: rank among A elements smaller than v
          int lo = a0, hi = a1;
          while (lo < hi) { int mid = (lo + hi) >> 1; if (src[mid] < v) lo = mid + 1; else hi = mid; }
          pos = a0 + (i - a1) + (lo - a0);
        }
        dst[pos] = v;
      }
      __syncthreads();
      unsigned long long* t = src; src = dst; dst = t;
    }
    if (src != seg + o)
      for (int i = threadIdx.x; i < len; i += blockDim.x) seg[o + i] = src[i];
    __syncthreads();
  }
}

__global__ void contact_gather_kernel(const int64_t* ctr, int64_t C, const unsigned long long* seg, const int32_t* rp,
                                      const int32_t* rt, const int32_t* ra, const int32_t* rb, const double* rtau,
                                      const double* rw, stiv_contacts out) {
  int64_t n = ctr[11]; if (n > C) n = C;
  for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x) {
    int src = (int)(seg[k] & 0xFFFFFFFFull);
    out.pair[k] = rp[src]; out.type[k] = rt[src]; out.a[k] = ra[src]; out.b[k] = rb[src];
    out.tau[k] = rtau[src]; out.w[2 * k] = rw[2 * src]; out.w[2 * k + 1] = rw[2 * src + 1];
  }
}

__global__ void scatter_grad_kernel(const int64_t* counts, int64_t cap, const int32_t* pair, const double* wpair,
                                    const double* grad, const int32_t* gves, const int32_t* gvid,
                                    const int32_t* pv, const int64_t* voff, double* gX) {
  int64_t n = n_contacts(counts, cap);
  for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x) {
    double wgt = wpair ? wpair[pair[k]] : 1.0;
    for (int q = 0; q < 4; ++q) {
      int v = gves[4 * k + q], id = gvid[4 * k + q];
      int nv = stiv_nverts(2 * pv[v]);
      size_t base = voff[v] + (size_t)3 * nv + id;  // X1 block
      for (int c = 0; c < 3; ++c) atomicAdd(&gX[base + (size_t)c * nv], wgt * grad[12 * k + 3 * q + c]);
    }
  }
}

// gcoef = S^T gX for the X1 block; one CTA per (vesicle, coordinate field),
// so that the three fields' phases overlap across CTAs.  S: Legendre step
// then Fourier step, so S^T: Fourier analysis sums per ring, then Legendre
// sums.
struct adj_args {
  const int32_t* p;
  const int64_t* coef_off;
  const int64_t* vert_off;
  const double* gX;
  double* gcoef;
  const double* leg[STIV_MAX_P + 1];
  const double* trig[STIV_MAX_P + 1];
};

__global__ void __launch_bounds__(256) adjoint_kernel(adj_args a) {
  extern __shared__ double sm[];
  int v = blockIdx.x, f = blockIdx.y;
  if (a.p[v] < 1 || a.p[v] > STIV_MAX_P || !a.leg[a.p[v]]) return;   // order outside [1, p_max]: skipped
  int p = a.p[v], P = 2 * p, nc = (p + 1) * (p + 1), nl = (p + 1) * (p + 2) / 2, ns = 2 * p + 1, W = 2 * P;
  int nv = stiv_nverts(P);
  double* G = sm;                    // [n_v]       one field of gX (X1 block), staged coalesced
  double* H = sm + nv;               // [P+1][ns]   Fourier-analysed rings of that field
  double* Q = H + (P + 1) * ns;      // [P+1][4][P/2+1] parity combinations of the four symmetric longitudes
  const double* g = a.gX + a.vert_off[v] + (size_t)3 * nv;
  const double* T = a.trig[p];
  const double* L = a.leg[p];
  double* out = a.gcoef + a.coef_off[v];
  int nq = P / 2 + 1;
  for (int k = threadIdx.x; k < nc; k += blockDim.x) out[f * nc + k] = 0.0;  // X0 block, this field
  {
    for (int k = threadIdx.x; k < nv; k += blockDim.x) G[k] = g[(size_t)f * nv + k];
    __syncthreads();
    // adjoint of the Fourier step.  The forward writes longitudes j, P-j, P+j,
    // 2P-j (j <= P/2, duplicates skipped) from the parity sums Ce, Co, Se, So;
    // their adjoints are the four combinations below.
    for (int task = threadIdx.x; task < (P + 1) * nq; task += blockDim.x) {
      int i = task / nq, j = task % nq;
      const double* gr = G + (size_t)i * W;
      int j1 = P - j, j2 = P + j, j3 = (W - j) % W;
      double g0 = gr[j];
      double g1 = (j1 != j) ? gr[j1] : 0.0;
      double g2 = (j2 != j1) ? gr[j2] : 0.0;
      double g3 = (j3 != j && j3 != j2) ? gr[j3] : 0.0;
      double* q = Q + (size_t)i * 4 * nq;
      q[0 * nq + j] = (g0 + g1) + (g2 + g3);   // cos, even m
      q[1 * nq + j] = (g0 - g1) - (g2 - g3);   // cos, odd m
      q[2 * nq + j] = (g0 - g1) + (g2 - g3);   // sin, even m
      q[3 * nq + j] = (g0 + g1) - (g2 + g3);   // sin, odd m
    }
    __syncthreads();
    for (int task = threadIdx.x; task < (P + 1) * ns; task += blockDim.x) {
      int i = task / ns, s = task % ns;
      int m = (s + 1) >> 1;
      bool is_sin = s > 0 && (s & 1) == 0;
      const double* q = Q + (size_t)i * 4 * nq + (size_t)((is_sin ? 2 : 0) + (m & 1)) * nq;
      double acc = 0.0;
      if (s == 0) {
        for (int j = 0; j < nq; ++j) acc += q[j];
      } else {
        int off = is_sin ? (p + 1) + m : m;
        for (int j = 0; j < nq; ++j) acc = fma(q[j], T[(size_t)j * 2 * (p + 1) + off], acc);
      }
      H[i * ns + s] = acc;
    }
    __syncthreads();
    // adjoint of the Legendre step (all rings, and the poles for m = 0)
    for (int q = threadIdx.x; q < nc; q += blockDim.x) {
      int n = (int)sqrtf((float)q); while (n * n > q) --n; while ((n + 1) * (n + 1) <= q) ++n;
      int m = q - n * n - n, am = m < 0 ? -m : m;
      int s = m == 0 ? 0 : (m > 0 ? 2 * m - 1 : 2 * am);
      double acc = 0.0;
      for (int i = 0; i <= P; ++i) acc = fma(L[(size_t)i * nl + n * (n + 1) / 2 + am], H[i * ns + s], acc);
      if (m == 0) {
        acc = fma(L[(size_t)(P + 1) * nl + n * (n + 1) / 2], G[(size_t)W * (P + 1)], acc);
        acc = fma(L[(size_t)(P + 2) * nl + n * (n + 1) / 2], G[(size_t)W * (P + 1) + 1], acc);
      }
      out[3 * nc + f * nc + q] = acc;
    }
  }
}

}  // namespace

int stiv_contact_order(stiv_handle* h, cudaStream_t st, const stiv_pairs* cand, const stiv_contacts* out,
                       detect_ws& w) {
  int64_t C = w.C;
  int32_t* rp = w.tmp_i32; int32_t* rt = rp + C; int32_t* ra = rp + 2 * C; int32_t* rb = rp + 3 * C;
  double* rtau = w.tmp_f64; double* rw = w.tmp_f64 + C;
  int64_t pcap = cand->capacity;
  int blocks = (int)((C + 255) / 256); if (blocks > 4096) blocks = 4096; if (blocks < 1) blocks = 1;
  STIV_PROF_N(h, st, "contact_order", 5);
  pair_count_kernel<<<blocks, 256, 0, st>>>(w.ctr, C, rp, w.pair_cnt);
  pair_scan_kernel<<<1, 1024, 0, st>>>(w.ctr, pcap, w.pair_cnt, w.pair_off, w.ctr);
  pair_scatter_kernel<<<blocks, 256, 0, st>>>(w.ctr, C, rp, rt, ra, rb, w.pair_off, w.pair_fill, w.seg);
  int sblocks = (int)(pcap < 65535 ? pcap : 65535);
  pair_sort_kernel<<<sblocks, 1024, 0, st>>>(w.ctr, pcap, w.pair_off, w.seg, w.seg2);
  contact_gather_kernel<<<blocks, 256, 0, st>>>(w.ctr, C, w.seg, rp, rt, ra, rb, rtau, rw, *out);
  STIV_LAUNCH(h);
  return STIV_OK;
}

static int run_stiv(stiv_handle* h, void* stream, const int32_t* p_dev, const int64_t* vert_off_dev,
                    const void* verts_dev, const stiv_pairs* cand, const stiv_contacts* ct, const int64_t* counts_dev,
                    double* Vc, double* Vp, double* grad, int32_t* gves, int32_t* gvid, double* grad0 = nullptr) {
  if (!h || !p_dev || !vert_off_dev || !verts_dev || !cand || !ct || !counts_dev) return STIV_ERR_ARG;
  if (grad && (!gves || !gvid)) return STIV_ERR_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  double* Vtmp = Vc;
  if (!Vtmp && Vp) {
    int rc = stiv_ws_reserve(h, sizeof(double) * (size_t)(ct->capacity > 0 ? ct->capacity : 1));
    if (rc) return rc;
    Vtmp = (double*)h->ws;
  }
  stiv_args A;
  A.pv = p_dev; A.voff = vert_off_dev; A.X = verts_dev; A.mixed = h->prm.precision == STIV_MIXED;
  for (int c = 0; c < 3; ++c) A.L[c] = h->prm.box_L[c];
  A.ci = cand->i; A.cj = cand->j; A.cs = cand->shift;
  A.pair = ct->pair; A.type = ct->type; A.a = ct->a; A.b = ct->b; A.tau = ct->tau; A.w = ct->w;
  A.counts = counts_dev; A.cap = ct->capacity;
  double edt = h->prm.eps * h->prm.dt;
  A.e2 = edt * edt;
  A.vabs = h->prm.velocity == STIV_VEL_ABSOLUTE;
  A.dm2 = h->prm.d_m * h->prm.d_m;
  A.Vc = Vtmp; A.grad = grad; A.gves = gves; A.gvid = gvid; A.grad0 = grad0;
  int dev_sms = 152;
  cudaDeviceGetAttribute(&dev_sms, cudaDevAttrMultiProcessorCount, h->device);
  if (Vtmp || grad || grad0) {
    STIV_PROF(h, st, A.grad ? "stiv_grad" : (A.grad0 ? "stiv_grad_x0" : "stiv"));
    if (A.vabs || A.dm2 > 0.0 || A.grad0) stiv_kernel<true><<<dev_sms * 8, 128, 0, st>>>(A);
    else stiv_kernel<false><<<dev_sms * 8, 128, 0, st>>>(A);
    STIV_LAUNCH(h);
  }
  if (Vp) {
    STIV_PROF(h, st, "vpair");
    vpair_kernel<<<dev_sms * 8, 256, 0, st>>>(ct->pair, counts_dev, ct->capacity, Vtmp, cand->capacity, Vp);
    STIV_LAUNCH(h);
  }
  return STIV_OK;
}

extern "C" int stiv_stiv(stiv_handle* h, void* stream, int32_t n_ves, const int32_t* p_dev,
                         const int64_t* vert_off_dev, const void* verts_dev, const stiv_pairs* cand,
                         const stiv_contacts* contacts, const int64_t* counts_dev, double* V_contact_dev,
                         double* V_pair_dev) {
  (void)n_ves;
  return run_stiv(h, stream, p_dev, vert_off_dev, verts_dev, cand, contacts, counts_dev, V_contact_dev, V_pair_dev,
                  nullptr, nullptr, nullptr);
}

extern "C" int stiv_stiv_grad(stiv_handle* h, void* stream, int32_t n_ves, const int32_t* p_dev,
                              const int64_t* vert_off_dev, const void* verts_dev, const stiv_pairs* cand,
                              const stiv_contacts* contacts, const int64_t* counts_dev, double* V_contact_dev,
                              double* V_pair_dev, double* grad_dev, int32_t* g_ves_dev, int32_t* g_vid_dev) {
  (void)n_ves;
  if (!grad_dev) return STIV_ERR_ARG;
  return run_stiv(h, stream, p_dev, vert_off_dev, verts_dev, cand, contacts, counts_dev, V_contact_dev, V_pair_dev,
                  grad_dev, g_ves_dev, g_vid_dev);
}

extern "C" int stiv_stiv_grad_x0(stiv_handle* h, void* stream, int32_t n_ves, const int32_t* p_dev,
                                 const int64_t* vert_off_dev, const void* verts_dev, const stiv_pairs* cand,
                                 const stiv_contacts* contacts, const int64_t* counts_dev, double* grad_x0_dev) {
  (void)n_ves;
  if (!grad_x0_dev) return STIV_ERR_ARG;
  return run_stiv(h, stream, p_dev, vert_off_dev, verts_dev, cand, contacts, counts_dev, nullptr, nullptr, nullptr,
                  nullptr, nullptr, grad_x0_dev);
}

extern "C" int stiv_grad_scatter(stiv_handle* h, void* stream, const int32_t* p_dev, const stiv_contacts* contacts,
                                 const int64_t* counts_dev, const double* weight_pair_dev, const double* grad_dev,
                                 const int32_t* g_ves_dev, const int32_t* g_vid_dev, const int64_t* vert_off_dev,
                                 double* gX_dev) {
  if (!h || !p_dev || !contacts || !counts_dev || !grad_dev || !g_ves_dev || !g_vid_dev || !vert_off_dev || !gX_dev)
    return STIV_ERR_ARG;
  int dev_sms = 152;
  cudaDeviceGetAttribute(&dev_sms, cudaDevAttrMultiProcessorCount, h->device);
  STIV_PROF(h, (cudaStream_t)stream, "grad_scatter");
  scatter_grad_kernel<<<dev_sms * 4, 128, 0, (cudaStream_t)stream>>>(counts_dev, contacts->capacity, contacts->pair,
                                                                     weight_pair_dev, grad_dev, g_ves_dev, g_vid_dev,
                                                                     p_dev, vert_off_dev, gX_dev);
  STIV_LAUNCH(h);
  return STIV_OK;
}

extern "C" int stiv_grad_to_coef(stiv_handle* h, void* stream, int32_t n_ves, int32_t p_max, const int32_t* p_dev,
                                 const int64_t* coef_off_dev, const int64_t* vert_off_dev, const double* gX_dev,
                                 double* gcoef_dev) {
  if (!h || n_ves < 0 || p_max < 1 || p_max > STIV_MAX_P) return STIV_ERR_ARG;
  if (n_ves == 0) return STIV_OK;
  if (!p_dev || !coef_off_dev || !vert_off_dev || !gX_dev || !gcoef_dev) return STIV_ERR_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  if (h->prm.precision == STIV_MIXED)
    return stiv_grad_to_coef_tc(h, st, n_ves, p_max, p_dev, coef_off_dev, vert_off_dev, gX_dev, gcoef_dev);
  adj_args a;
  a.p = p_dev; a.coef_off = coef_off_dev; a.vert_off = vert_off_dev; a.gX = gX_dev; a.gcoef = gcoef_dev;
  for (int p = 0; p <= STIV_MAX_P; ++p) { a.leg[p] = nullptr; a.trig[p] = nullptr; }
  for (int p = 1; p <= p_max; ++p) {
    int rc = stiv_ensure_tables(h, st, p);
    if (rc) return rc;
    a.leg[p] = h->tab[p].leg; a.trig[p] = h->tab[p].trig;
  }
  int Pm = 2 * p_max;
  size_t smem = sizeof(double) * ((size_t)stiv_nverts(Pm) + (size_t)(Pm + 1) * (2 * p_max + 1) +
                                  (size_t)(Pm + 1) * 4 * (Pm / 2 + 1));
  STIV_CUDA(h, cudaFuncSetAttribute(adjoint_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  STIV_PROF(h, st, "grad_to_coef");
  adjoint_kernel<<<dim3(n_ves, 3), 256, smem, st>>>(a);
  STIV_LAUNCH(h);
  return STIV_OK;
}

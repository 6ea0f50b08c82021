// Sec. 3.1.1-3.1.2: spherical-harmonic synthesis of each vesicle's order-p
// series on its order-2p grid (the "upsampled q^up-grid"), plus the swept
// boxes of vesicles and surface patches.
//
// Synthesis per field (vesicle, time, coordinate):
//   ring sums   G_i(m)  = sum_n a_{n,m} Pbar_n^|m|(x_i)          (Legendre step)
//   longitudes  X(i, j) = sum_m G_i(m) {cos|sin}(|m| phi_j)       (Fourier step)
// Both steps use exact symmetries of the grid: Pbar_n^m(-x) = (-1)^(n+m)
// Pbar_n^m(x) pairs ring i with ring P-i, and phi_{P-j} = pi - phi_j,
// phi_{P+j} = pi + phi_j, phi_{2P-j} = 2 pi - phi_j give four outputs from one
// set of parity-split partial sums.  FP64 throughout (fused multiply-adds);
// STIV_MIXED stores the result as float.
#include "stiv_internal.cuh"

#include <math.h>

namespace {

// Gauss-Legendre node x_i (descending) of order n by Newton's method on P_n.
__device__ double gl_node(int n, int i) {
  double z = cospi((i + 0.75) / (n + 0.5));
  for (int it = 0; it < 100; ++it) {
    double p0 = 1.0, p1 = z;
    for (int k = 2; k <= n; ++k) {
      double p2 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
      p0 = p1; p1 = p2;
    }
    double dp = n * (z * p1 - p0) / (z * z - 1.0);
    double dz = p1 / dp;
    z -= dz;
    if (fabs(dz) <= 1e-16 * fabs(z) + 1e-300) break;
  }
  return z;
}

// Tables for SH order p (mesh order P = 2p): one thread per table row.
__global__ void tables_kernel(int p, double* leg, double* trig, double* theta) {
  int P = 2 * p, nl = (p + 1) * (p + 2) / 2;
  int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r < P + 3) {
    double x;
    if (r <= P) {
      int ih = r <= P / 2 ? r : P - r;       // compute half the nodes, mirror the rest
      x = (2 * ih == P) ? 0.0 : gl_node(P + 1, ih);
      if (r > P / 2) x = -x;
      theta[r] = acos(x);
    } else {
      x = (r == P + 1) ? 1.0 : -1.0;         // north / south pole
    }
    double s = sqrt((1.0 - x) * (1.0 + x));
    double* L = leg + (size_t)r * nl;
    // normalised associated Legendre functions, no Condon-Shortley phase
    L[0] = 0.28209479177387814347;  // 1/sqrt(4 pi)
    for (int m = 1; m <= p; ++m)
      L[m * (m + 1) / 2 + m] = sqrt((2.0 * m + 1.0) / (2.0 * m)) * s * L[(m - 1) * m / 2 + m - 1];
    for (int m = 0; m < p; ++m)
      L[(m + 1) * (m + 2) / 2 + m] = sqrt(2.0 * m + 3.0) * x * L[m * (m + 1) / 2 + m];
    for (int m = 0; m <= p; ++m)
      for (int n = m + 2; n <= p; ++n) {
        double a = sqrt((4.0 * n * n - 1.0) / ((double)(n - m) * (n + m)));
        double b = sqrt(((double)(n - 1 - m) * (n - 1 + m)) / (4.0 * (n - 1) * (n - 1) - 1.0));
        L[n * (n + 1) / 2 + m] = a * (x * L[(n - 1) * n / 2 + m] - b * L[(n - 2) * (n - 1) / 2 + m]);
      }
    // fold the sqrt(2) of the real harmonics with m > 0 into the table
    for (int n = 1; n <= p; ++n)
      for (int m = 1; m <= n; ++m) L[n * (n + 1) / 2 + m] *= 1.41421356237309504880;
  }
  // trig[j][0][m] = cos(m phi_j), trig[j][1][m] = sin(m phi_j), phi_j = pi j / P, j <= P/2
  int t = blockIdx.x * blockDim.x + threadIdx.x;
  int nt = (P / 2 + 1) * (p + 1);
  if (t < nt) {
    int j = t / (p + 1), m = t % (p + 1);
    int k = (m * j) % (2 * P);  // exact argument reduction
    double sv, cv;
    sincospi((double)k / P, &sv, &cv);
    trig[(size_t)j * 2 * (p + 1) + m] = cv;
    trig[(size_t)j * 2 * (p + 1) + (p + 1) + m] = sv;
  }
}

struct synth_args {
  const int32_t* p;
  const int64_t* coef_off;
  const double* coef;
  const int64_t* vert_off;
  void* verts;
  int mixed;
  const double* leg[STIV_MAX_P + 1];
  const double* trig[STIV_MAX_P + 1];
};

// One CTA per (vesicle, time level): the 3 coordinate fields.
__global__ void __launch_bounds__(256) synth_kernel(synth_args a) {
  extern __shared__ double sm[];
  int v = blockIdx.x, t = blockIdx.y;
  if (a.p[v] < 1 || a.p[v] > STIV_MAX_P || !a.leg[a.p[v]]) return;   // order outside [1, p_max]: skipped
  int p = a.p[v], P = 2 * p, nc = (p + 1) * (p + 1), nl = (p + 1) * (p + 2) / 2, ns = 2 * p + 1;
  int nv = 2 * P * (P + 1) + 2;
  double* C = sm;                        // [3][nc]
  double* G = sm + 3 * nc;               // [3][P+1][ns]  slot 0: m=0; 2m-1: cos m; 2m: sin m
  const double* coef = a.coef + a.coef_off[v] + (size_t)t * 3 * nc;
  for (int k = threadIdx.x; k < 3 * nc; k += blockDim.x) C[k] = coef[k];
  __syncthreads();
  const double* L = a.leg[p];
  const double* T = a.trig[p];
  // Legendre step over half the rings (parity pairs ring i with ring P-i)
  int nh = P / 2 + 1;
  for (int task = threadIdx.x; task < 3 * nh * ns; task += blockDim.x) {
    int f = task / (nh * ns), rem = task % (nh * ns), i = rem / ns, s = rem % ns;
    int m = (s + 1) >> 1;
    int sgn = (s == 0) ? 0 : ((s & 1) ? 1 : -1);  // +m cos, -m sin
    const double* Lr = L + (size_t)i * nl;
    const double* Cf = C + f * nc;
    double E = 0.0, O = 0.0;
    for (int n = m; n <= p; n += 2) E = fma(Cf[n * n + n + sgn * m], Lr[n * (n + 1) / 2 + m], E);
    for (int n = m + 1; n <= p; n += 2) O = fma(Cf[n * n + n + sgn * m], Lr[n * (n + 1) / 2 + m], O);
    G[(f * (P + 1) + i) * ns + s] = E + O;
    if (i != P - i) G[(f * (P + 1) + (P - i)) * ns + s] = E - O;
  }
  __syncthreads();
  // Fourier step: four longitudes per task
  size_t base = a.vert_off[v] + (size_t)t * 3 * nv;
  int nq = P / 2 + 1;
  for (int task = threadIdx.x; task < 3 * (P + 1) * nq; task += blockDim.x) {
    int f = task / ((P + 1) * nq), rem = task % ((P + 1) * nq), r = rem / nq, j = rem % nq;
    const double* g = G + (size_t)(f * (P + 1) + r) * ns;
    const double* cs = T + (size_t)j * 2 * (p + 1);
    const double* sn = cs + (p + 1);
    double Ce = g[0], Co = 0.0, Se = 0.0, So = 0.0;
    for (int m = 1; m <= p; m += 2) { Co = fma(g[2 * m - 1], cs[m], Co); So = fma(g[2 * m], sn[m], So); }
    for (int m = 2; m <= p; m += 2) { Ce = fma(g[2 * m - 1], cs[m], Ce); Se = fma(g[2 * m], sn[m], Se); }
    int W = 2 * P;
    double v0 = (Ce + Co) + (Se + So);            // phi_j
    double v1 = (Ce - Co) + (So - Se);            // pi - phi_j
    double v2 = (Ce - Co) + (Se - So);            // pi + phi_j
    double v3 = (Ce + Co) - (Se + So);            // 2 pi - phi_j
    size_t row = base + (size_t)f * nv + (size_t)r * W;
    int j1 = P - j, j2 = P + j, j3 = (W - j) % W;
    if (a.mixed) {
      float* X = (float*)a.verts;
      X[row + j] = (float)v0;
      if (j1 != j) X[row + j1] = (float)v1;
      if (j2 != j1 && j2 < W) X[row + j2] = (float)v2;
      if (j3 != j && j3 != j2) X[row + j3] = (float)v3;
    } else {
      double* X = (double*)a.verts;
      X[row + j] = v0;
      if (j1 != j) X[row + j1] = v1;
      if (j2 != j1 && j2 < W) X[row + j2] = v2;
      if (j3 != j && j3 != j2) X[row + j3] = v3;
    }
  }
  // poles: only m = 0 contributes
  if (threadIdx.x < 6) {
    int f = threadIdx.x >> 1, pole = threadIdx.x & 1;
    const double* Lr = L + (size_t)(P + 1 + pole) * nl;
    double acc = 0.0;
    for (int n = 0; n <= p; ++n) acc = fma(C[f * nc + n * n + n], Lr[n * (n + 1) / 2], acc);
    size_t idx = base + (size_t)f * nv + 2 * P * (P + 1) + pole;
    if (a.mixed) ((float*)a.verts)[idx] = (float)acc;
    else ((double*)a.verts)[idx] = acc;
  }
}

// ---------------------------------------------------------------------------
// Mesh fidelity (Sec. 3.1.2: the q^up-grid triangle mesh must stay within
// alpha d_m of the smooth surface, ||X^{q^up} - X(phi, theta)||_inf; Fig. 6
// estimates the smooth surface on a 4x upsampled grid).  The mesh is read as
// a map from parameter space: on the grid cell [theta_i, theta_{i+1}] x
// [phi_j, phi_{j+1}], with a, b the cell fractions in theta and phi, the
// triangle [(i,j), (i+1,j), (i+1,j+1)] for a >= b and [(i,j), (i+1,j+1),
// (i,j+1)] for a < b (the Fig. 3 split); above ring 0 and below ring P the
// pole fans.  One CTA per (vesicle, time level) takes the largest distance
// between that map and the order-p series over the order-(factor P) grid
// (its Gauss-Legendre rings, phi_k = pi k / (factor P); poles excluded).
// ---------------------------------------------------------------------------

constexpr double kPi = 3.14159265358979323846;

// Column m of the normalised associated Legendre table at x = cos(theta),
// s = sin(theta), no Condon-Shortley phase, sqrt(2) folded in for m > 0:
// L[n(n+1)/2 + m] for n = m .. p, by the recurrences of tables_kernel with
// their coefficients tabulated: dg[k] = sqrt((2k+1)/(2k)), sd[m] =
// sqrt(2m+3), ra and rb[n(n+1)/2+m] the three-term coefficients of (n, m).
__device__ void legendre_column_tab(int p, int m, double x, double s, const double* dg, const double* sd,
                                    const double* ra, const double* rb, double* L) {
  double d = 0.28209479177387814347;  // 1/sqrt(4 pi)
  for (int k = 1; k <= m; ++k) d = dg[k] * s * d;
  double r2 = m ? 1.41421356237309504880 : 1.0;
  L[m * (m + 1) / 2 + m] = d * r2;
  if (m < p) {
    double e = sd[m] * x * d;
    L[(m + 1) * (m + 2) / 2 + m] = e * r2;
    double l2 = d, l1 = e;
    for (int n = m + 2; n <= p; ++n) {
      int idx = n * (n + 1) / 2 + m;
      double l0 = ra[idx] * (x * l1 - rb[idx] * l2);
      L[idx] = l0 * r2;
      l2 = l1; l1 = l0;
    }
  }
}

struct fid_args {
  const int32_t* p;
  const int64_t* coef_off;
  const double* coef;
  const int64_t* vert_off;
  const void* verts;
  int mixed;
  int factor;
  const double* theta[STIV_MAX_P + 1];
  const double* xfine;   // fine-grid nodes x = cos(theta), order factor*2p at xfine + xoff[p]
  int xoff[STIV_MAX_P + 1];
  double* err;
};

// Gauss-Legendre node x_i (descending) of order n, Newton's method on P_n from
// the same start as gl_node, at most 8 steps (quadratic convergence reaches
// the last bits in about 5), stopping once a step is below 4e-16 |x|.
__device__ double fine_node(int n, int i) {
  double z = cospi((i + 0.75) / (n + 0.5));
  for (int it = 0; it < 8; ++it) {
    double p0 = 1.0, p1 = z;
    for (int k = 2; k <= n; ++k) {
      double p2 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
      p0 = p1; p1 = p2;
    }
    double dz = p1 / (n * (z * p1 - p0) / (z * z - 1.0));
    z -= dz;
    if (fabs(dz) <= 4e-16 * fabs(z)) break;
  }
  return z;
}

// Fine-grid Gauss-Legendre nodes for every order p <= p_max (computed once per
// call, not per CTA): order Pf = factor 2p at xs + off(p), off(p) = sum over
// p' < p of (factor 2p' + 1).
__global__ void fine_nodes_kernel(int p_max, int factor, double* xs) {
  int total = 0;
  for (int p = 1; p <= p_max; ++p) total += factor * 2 * p + 1;
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < total; e += gridDim.x * blockDim.x) {
    int p = 1, off = 0;
    while (e >= off + factor * 2 * p + 1) { off += factor * 2 * p + 1; ++p; }
    int Pf = factor * 2 * p, r = e - off;
    int ih = r <= Pf / 2 ? r : Pf - r;
    double x = (2 * ih == Pf) ? 0.0 : fine_node(Pf + 1, ih);
    xs[e] = r > Pf / 2 ? -x : x;
  }
}

__device__ __forceinline__ double vert_at(const fid_args& a, size_t idx) {
  return a.mixed ? (double)((const float*)a.verts)[idx] : ((const double*)a.verts)[idx];
}

constexpr int FRMAX = 8;   // fine rings per pass at most

// Fine rings per pass for order p: as many as keep the pass's point tasks
// (one per ring and longitude quarter) within one round of 256 threads.
__host__ __device__ inline int fid_rings(int p, int factor) {
  int nq = factor * p + 1, r = 256 / nq;
  return r < 1 ? 1 : (r > FRMAX ? FRMAX : r);
}

__host__ __device__ inline size_t fid_smem_doubles(int p, int factor) {
  int P = 2 * p, Pf = factor * P, nl = (p + 1) * (p + 2) / 2, FR = fid_rings(p, factor);
  return (size_t)3 * (p + 1) * (p + 1) + (P + 1) + (Pf + 1) + (size_t)FR * nl + (size_t)FR * 3 * (2 * p + 1) +
         (size_t)(Pf / 2 + 1) * 2 * (p + 1) + (Pf + 1) + 2 * (size_t)nl + 2 * (size_t)(p + 1) +
         (size_t)FR * 3 * (2 * P) * 4;
}

// The mesh along one fine ring, per coordinate field and longitude cell j
// (j1 = j + 1 mod 2P), as two lines in the cell fraction b:
//   A + b dA on the triangle (i, j), (i+1, j), (i+1, j+1)  (taken when a_ >= b),
//   B + b dB on the triangle (i, j), (i+1, j+1), (i, j+1)  (when a_ < b),
// with a_ the ring's fraction between mesh rings i and i+1; in the pole caps
// (zone 0 north, 2 south; tp the fraction from the pole to the first ring)
// both lines are the fan triangle's.  out: A, dA, B, dB.
__device__ __forceinline__ void mesh_lines(const fid_args& a, size_t o, int P, int W, int zone, int i, double a_,
                                           double tp, int j, double* out) {
  int j1 = j + 1 == W ? 0 : j + 1;
  if (zone != 1) {
    size_t pole = o + 2 * (size_t)P * (P + 1) + (zone == 2 ? 1 : 0);
    size_t ring = o + (zone == 2 ? (size_t)P * W : 0);
    double N = vert_at(a, pole), x0 = vert_at(a, ring + j), x1 = vert_at(a, ring + j1);
    out[0] = out[2] = fma(tp, x0 - N, N);
    out[1] = out[3] = tp * (x1 - x0);
    return;
  }
  double q = vert_at(a, o + (size_t)i * W + j), rr = vert_at(a, o + (size_t)(i + 1) * W + j);
  double s3 = vert_at(a, o + (size_t)(i + 1) * W + j1), u = vert_at(a, o + (size_t)i * W + j1);
  out[0] = fma(a_, rr - q, q);
  out[1] = s3 - rr;
  out[2] = fma(a_, s3 - u, q);
  out[3] = u - q;
}

// One CTA per (vesicle, time level), FR fine rings per pass.  The series is
// evaluated like the synthesis: ring sums G(m), then per longitude pair the
// even and odd partial Fourier sums, which give the four longitudes
// phi_k, pi - phi_k, pi + phi_k and 2 pi - phi_k (k <= Pf / 2) at once;
// cos(m phi_k), sin(m phi_k) come from a table built per CTA.
__global__ void __launch_bounds__(256) fidelity_kernel(fid_args a) {
  extern __shared__ double sm[];
  __shared__ double red[256 / 32];
  int v = blockIdx.x, t = blockIdx.y;
  if (a.p[v] < 1 || a.p[v] > STIV_MAX_P || !a.theta[a.p[v]]) {   // order outside [1, p_max]: NaN
    if (threadIdx.x == 0) a.err[2 * (size_t)v + t] = __longlong_as_double(0x7ff8000000000000LL);
    return;
  }
  int p = a.p[v], P = 2 * p, Pf = a.factor * P, W = 2 * P, nv = 2 * P * (P + 1) + 2;
  int nc = (p + 1) * (p + 1), nl = (p + 1) * (p + 2) / 2, ns = 2 * p + 1, nq = Pf / 2 + 1;
  int FR = fid_rings(p, a.factor);
  double* C = sm;                   // [3][nc]
  double* thc = C + 3 * nc;         // [P+1]  mesh rings (ascending theta)
  double* xf = thc + (P + 1);       // [Pf+1] fine rings, x = cos(theta)
  double* L = xf + (Pf + 1);        // [FR][nl] Legendre values of the current rings
  double* G = L + FR * nl;          // [FR][3][ns] ring sums (slot 0: m=0; 2m-1: cos m; 2m: sin m)
  double* T = G + FR * 3 * ns;      // [nq][2][p+1] cos, sin (m phi_k), k <= Pf/2
  double* thf = T + (size_t)nq * 2 * (p + 1);   // [Pf+1] fine ring angles
  double* ra = thf + (Pf + 1);      // [nl] Legendre recurrence coefficients
  double* rb = ra + nl;             // [nl]
  double* dg = rb + nl;             // [p+1]
  double* sd = dg + (p + 1);        // [p+1]
  double* ML = sd + (p + 1);        // [FR][3][W][4] mesh lines of the current rings (mesh_lines)
  __shared__ int rzone[FRMAX], rcell[FRMAX], rtri[FRMAX];   // per current ring: zone, cell, triangle mask
  __shared__ double ra_[FRMAX], rtp[FRMAX], btab[8];
  if (threadIdx.x < a.factor) btab[threadIdx.x] = (double)threadIdx.x / a.factor;
  const double* coef = a.coef + a.coef_off[v] + (size_t)t * 3 * nc;
  for (int k = threadIdx.x; k < 3 * nc; k += blockDim.x) C[k] = coef[k];
  for (int i = threadIdx.x; i <= P; i += blockDim.x) thc[i] = a.theta[p][i];
  for (int r = threadIdx.x; r <= Pf; r += blockDim.x) {
    double x = a.xfine[a.xoff[p] + r];
    xf[r] = x;
    thf[r] = acos(x);
  }
  for (int m = threadIdx.x; m <= p; m += blockDim.x) {
    dg[m] = m ? sqrt((2.0 * m + 1.0) / (2.0 * m)) : 0.0;
    sd[m] = sqrt(2.0 * m + 3.0);
  }
  for (int e = threadIdx.x; e < nl; e += blockDim.x) {
    int n = 0;
    while ((n + 1) * (n + 2) / 2 <= e) ++n;
    int m = e - n * (n + 1) / 2;
    if (n >= m + 2) {
      ra[e] = sqrt((4.0 * n * n - 1.0) / ((double)(n - m) * (n + m)));
      rb[e] = sqrt(((double)(n - 1 - m) * (n - 1 + m)) / (4.0 * (n - 1) * (n - 1) - 1.0));
    } else {
      ra[e] = 0.0; rb[e] = 0.0;
    }
  }
  for (int e = threadIdx.x; e < nq * (p + 1); e += blockDim.x) {
    int k = e / (p + 1), m = e % (p + 1);
    int kk = (m * k) % (2 * Pf);            // exact argument reduction
    double sv, cv;
    sincospi((double)kk / Pf, &sv, &cv);
    T[(size_t)k * 2 * (p + 1) + m] = cv;
    T[(size_t)k * 2 * (p + 1) + (p + 1) + m] = sv;
  }
  __syncthreads();
  size_t base = a.vert_off[v] + (size_t)t * 3 * nv;
  double worst2 = 0.0;
  for (int r0 = 0; r0 <= Pf; r0 += FR) {
    int nr = Pf + 1 - r0 < FR ? Pf + 1 - r0 : FR;
    if (threadIdx.x < nr * (p + 1)) {
      int rr = threadIdx.x / (p + 1), m = threadIdx.x % (p + 1);
      double x = xf[r0 + rr];
      legendre_column_tab(p, m, x, sqrt((1.0 - x) * (1.0 + x)), dg, sd, ra, rb, L + rr * nl);
    }
    if (threadIdx.x >= blockDim.x - nr) {   // where each ring lies on the mesh
      int rr = threadIdx.x - (blockDim.x - nr);
      double theta = thf[r0 + rr];
      int zone = 1, i = 0;
      double al = 0.0, tp = 0.0;
      if (theta < thc[0]) { zone = 0; tp = theta / thc[0]; }
      else if (theta > thc[P]) { zone = 2; tp = (kPi - theta) / (kPi - thc[P]); }
      else {
        while (i + 1 < P && thc[i + 1] <= theta) ++i;
        al = (theta - thc[i]) / (thc[i + 1] - thc[i]);
      }
      int mask = 0;
      for (int sb = 0; sb < a.factor; ++sb) mask |= (al >= (double)sb / a.factor) << sb;
      rzone[rr] = zone; rcell[rr] = i; rtri[rr] = mask; ra_[rr] = al; rtp[rr] = tp;
    }
    __syncthreads();
    for (int task = threadIdx.x; task < nr * 3 * (ns + W); task += blockDim.x) {
      if (task < nr * 3 * ns) {   // ring sums
        int rr = task / (3 * ns), rem = task % (3 * ns), f = rem / ns, sl = rem % ns, m = (sl + 1) >> 1;
        int sgn = sl == 0 ? 0 : ((sl & 1) ? 1 : -1);
        const double* Lr = L + rr * nl;
        double acc = 0.0;
        for (int n = m; n <= p; ++n) acc = fma(C[f * nc + n * n + n + sgn * m], Lr[n * (n + 1) / 2 + m], acc);
        G[(rr * 3 + f) * ns + sl] = acc;
      } else {                    // mesh lines
        int k2 = task - nr * 3 * ns, rr = k2 / (3 * W), rem = k2 % (3 * W), f = rem / W, j = rem % W;
        mesh_lines(a, base + (size_t)f * nv, P, W, rzone[rr], rcell[rr], ra_[rr], rtp[rr], j,
                   ML + ((size_t)(rr * 3 + f) * W + j) * 4);
      }
    }
    __syncthreads();
    for (int task = threadIdx.x; task < nr * nq; task += blockDim.x) {
      int rr = task / nq, q = task % nq;
      int tri = rtri[rr];
      const double* cs = T + (size_t)q * 2 * (p + 1);
      const double* sn = cs + (p + 1);
      int kq[4] = {q, Pf - q, Pf + q, (2 * Pf - q) % (2 * Pf)};
      double val[4][3];
#pragma unroll
      for (int f = 0; f < 3; ++f) {
        const double* g = G + (size_t)(rr * 3 + f) * ns;
        double Ce = g[0], Co = 0.0, Se = 0.0, So = 0.0;
        for (int m = 1; m <= p; m += 2) { Co = fma(g[2 * m - 1], cs[m], Co); So = fma(g[2 * m], sn[m], So); }
        for (int m = 2; m <= p; m += 2) { Ce = fma(g[2 * m - 1], cs[m], Ce); Se = fma(g[2 * m], sn[m], Se); }
        val[0][f] = (Ce + Co) + (Se + So);     // phi_q
        val[1][f] = (Ce - Co) + (So - Se);     // pi - phi_q
        val[2][f] = (Ce - Co) + (Se - So);     // pi + phi_q
        val[3][f] = (Ce + Co) - (Se + So);     // 2 pi - phi_q
      }
#pragma unroll
      for (int w = 0; w < 4; ++w) {
        int k = kq[w];
        bool dup = (w == 1 && k == kq[0]) || (w == 2 && (k == kq[1] || k >= 2 * Pf)) ||
                   (w == 3 && (k == kq[0] || k == kq[2]));
        if (dup) continue;
        int j = k / a.factor, sb = k % a.factor;
        double b = btab[sb];
        int side = (tri >> sb) & 1 ? 0 : 2;
        double d2 = 0.0;
#pragma unroll
        for (int f = 0; f < 3; ++f) {
          const double* l = ML + ((size_t)(rr * 3 + f) * W + j) * 4 + side;
          double e = fma(b, l[1], l[0]) - val[w][f];
          d2 = fma(e, e, d2);
        }
        worst2 = fmax(worst2, d2);   // squared distance; one square root at the end
      }
    }
    __syncthreads();   // L and G are rewritten for the next rings
  }
  for (int off = 16; off > 0; off >>= 1) worst2 = fmax(worst2, __shfl_xor_sync(0xffffffffu, worst2, off));
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = worst2;
  __syncthreads();
  if (threadIdx.x == 0) {
    double w = red[0];
    for (int q = 1; q < (int)(blockDim.x >> 5); ++q) w = fmax(w, red[q]);
    a.err[2 * (size_t)v + t] = sqrt(w);
  }
}

}  // namespace

int stiv_ensure_tables(stiv_handle* h, cudaStream_t st, int p) {
  if (p < 1 || p > STIV_MAX_P) return STIV_ERR_ARG;
  if (h->tab_ready[p]) return STIV_OK;
  int P = 2 * p, nl = (p + 1) * (p + 2) / 2;
  stiv_tables& T = h->tab[p];
  STIV_CUDA(h, cudaMalloc(&T.leg, sizeof(double) * (size_t)(P + 3) * nl));
  STIV_CUDA(h, cudaMalloc(&T.trig, sizeof(double) * (size_t)(P / 2 + 1) * 2 * (p + 1)));
  STIV_CUDA(h, cudaMalloc(&T.theta, sizeof(double) * (P + 1)));
  int n = (P / 2 + 1) * (p + 1) > P + 3 ? (P / 2 + 1) * (p + 1) : P + 3;
  tables_kernel<<<(n + 127) / 128, 128, 0, st>>>(p, T.leg, T.trig, T.theta);
  STIV_LAUNCH(h);
  h->tab_ready[p] = true;
  return STIV_OK;
}

static size_t synth_smem(int p) {
  int P = 2 * p;
  return sizeof(double) * (size_t)(3 * (p + 1) * (p + 1) + 3 * (P + 1) * (2 * p + 1));
}

extern "C" int stiv_upsample(stiv_handle* h, void* stream, int32_t n_ves, int32_t p_max, const int32_t* p_dev,
                             const int64_t* coef_off_dev, const double* coef_dev,
                             const int64_t* vert_off_dev, void* verts_dev) {
  if (!h || n_ves < 0 || p_max < 1 || p_max > STIV_MAX_P) return STIV_ERR_ARG;
  if (n_ves == 0) return STIV_OK;
  if (!p_dev || !coef_off_dev || !coef_dev || !vert_off_dev || !verts_dev) return STIV_ERR_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  if (h->prm.precision == STIV_MIXED)
    return stiv_upsample_tc(h, st, n_ves, p_max, p_dev, coef_off_dev, coef_dev, vert_off_dev, (float*)verts_dev);
  synth_args a;
  a.p = p_dev; a.coef_off = coef_off_dev; a.coef = coef_dev; a.vert_off = vert_off_dev;
  a.verts = verts_dev; a.mixed = h->prm.precision == STIV_MIXED;
  for (int p = 0; p <= STIV_MAX_P; ++p) { a.leg[p] = nullptr; a.trig[p] = nullptr; }
  for (int p = 1; p <= p_max; ++p) {
    int rc = stiv_ensure_tables(h, st, p);
    if (rc) return rc;
    a.leg[p] = h->tab[p].leg; a.trig[p] = h->tab[p].trig;
  }
  size_t smem = synth_smem(p_max);
  STIV_CUDA(h, cudaFuncSetAttribute(synth_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  STIV_PROF(h, st, "synth");
  synth_kernel<<<dim3(n_ves, 2), 256, smem, st>>>(a);
  STIV_LAUNCH(h);
  return STIV_OK;
}

extern "C" int stiv_mesh_fidelity(stiv_handle* h, void* stream, int32_t n_ves, int32_t p_max, const int32_t* p_dev,
                                  const int64_t* coef_off_dev, const double* coef_dev, const int64_t* vert_off_dev,
                                  const void* verts_dev, int32_t factor, double* err_dev) {
  if (!h || n_ves < 0 || p_max < 1 || p_max > STIV_MAX_P || factor < 1 || factor > 8) return STIV_ERR_ARG;
  if (n_ves == 0) return STIV_OK;
  if (!p_dev || !coef_off_dev || !coef_dev || !vert_off_dev || !verts_dev || !err_dev) return STIV_ERR_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  fid_args a;
  a.p = p_dev; a.coef_off = coef_off_dev; a.coef = coef_dev; a.vert_off = vert_off_dev; a.verts = verts_dev;
  a.mixed = h->prm.precision == STIV_MIXED; a.factor = factor; a.err = err_dev;
  for (int p = 0; p <= STIV_MAX_P; ++p) a.theta[p] = nullptr;
  for (int p = 1; p <= p_max; ++p) {
    int rc = stiv_ensure_tables(h, st, p);
    if (rc) return rc;
    a.theta[p] = h->tab[p].theta;
  }
  int nx = 0;
  for (int p = 1; p <= p_max; ++p) { a.xoff[p] = nx; nx += factor * 2 * p + 1; }
  a.xoff[0] = 0;
  if (sizeof(double) * (size_t)nx > h->fid_x_bytes) {
    if (h->fid_x) { STIV_CUDA(h, cudaFree(h->fid_x)); h->fid_x = nullptr; h->fid_x_bytes = 0; }
    STIV_CUDA(h, cudaMalloc(&h->fid_x, sizeof(double) * (size_t)nx));
    h->fid_x_bytes = sizeof(double) * (size_t)nx;
  }
  a.xfine = h->fid_x;
  size_t smem = 0;
  for (int p = 1; p <= p_max; ++p) {
    size_t b = sizeof(double) * fid_smem_doubles(p, factor);
    smem = b > smem ? b : smem;
  }
  if (smem > 220 * 1024) return STIV_ERR_ARG;
  if (smem > 48 * 1024)
    STIV_CUDA(h, cudaFuncSetAttribute(fidelity_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  STIV_PROF_N(h, st, "mesh_fidelity", 2);
  fine_nodes_kernel<<<(nx + 127) / 128, 128, 0, st>>>(p_max, factor, h->fid_x);
  fidelity_kernel<<<dim3(n_ves, 2), 256, smem, st>>>(a);
  STIV_LAUNCH(h);
  return STIV_OK;
}

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

/*
 * Plain FP64 CPU oracle for the contact-detection + space-time interference
 * volume (STIV) path of Lu, Rahimian & Zorin, "Parallel contact-aware
 * simulations of deformable particles in 3D Stokes flow" (arXiv 1812.04719).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the
 * CPU-baseline leg of the benchmark load this library.  The CUDA product
 * path never links, imports or calls anything here, and this file shares
 * no code, header, table or helper with it.
 *
 * Everything is IEEE binary64, round to nearest, compiled with
 * -ffp-contract=off so that no multiply-add is fused.  No spatial data
 * structure is used: vesicle pairs are found by testing every pair of boxes,
 * primitive pairs by testing every vertex/triangle and edge/edge pair of a
 * candidate vesicle pair.
 *
 * Sections of the paper each function follows:
 *   - SH surface and its quadrature grid ........ Sec. 3.1.1
 *   - upsampling, triangulation (Fig. 3) ........ Sec. 3.1.2
 *   - space-time bounding boxes, bbiCheck ........ Sec. 3.3.1, Alg. 1
 *   - contact time (Eq. 3.1 with d_m = 0) ........ Sec. 3.1.2
 *   - contact volume V_k (Eq. 3.2, App. A) ........ Sec. 3.1.2, App. A
 *   - gradient of V_k w.r.t. vertex positions .... Sec. 3.1.2, Sec. 3.3.2
 *   - ContactVolume driver ........................ Alg. 2
 * Readings of points the paper leaves open (grid orientation, pole caps,
 * root isolation, edge-edge volume, relative velocity) are stated next to
 * the code that takes them.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_PI 3.14159265358979323846

/* ------------------------------------------------------------------------ */
/* Sec. 3.1.1: quadrature grid.  Gauss-Legendre in the polar angle,          */
/* uniform (trapezoidal) in longitude; (P+1) x 2P points for order P.        */
/* ------------------------------------------------------------------------ */

/* Legendre polynomial P_n(x) and its derivative by the three-term recurrence. */
static void legendre_pn(int n, double x, double* pn, double* dpn) {
  double p0 = 1.0, p1 = x;
  if (n == 0) { *pn = 1.0; *dpn = 0.0; return; }
  for (int k = 2; k <= n; ++k) {
    double p2 = ((2.0 * k - 1.0) * x * p1 - (k - 1.0) * p0) / k;
    p0 = p1; p1 = p2;
  }
  *pn = p1;
  *dpn = n * (x * p1 - p0) / (x * x - 1.0);
}

/* Gauss-Legendre nodes x (descending, i.e. polar angle ascending) and
 * weights for nq points, by Newton iteration on P_nq. */
int orc_gl_nodes(int nq, double* x, double* w) {
  if (nq < 1) return -1;
  for (int i = 0; i < nq; ++i) {
    double z = cos(ORC_PI * (i + 0.75) / (nq + 0.5));
    double pn = 0.0, dpn = 1.0;
    for (int it = 0; it < 100; ++it) {
      legendre_pn(nq, z, &pn, &dpn);
      double dz = pn / dpn;
      z -= dz;
      if (fabs(dz) < 1e-15) break;
    }
    legendre_pn(nq, z, &pn, &dpn);
    x[i] = z;
    w[i] = 2.0 / ((1.0 - z * z) * dpn * dpn);
  }
  return 0;
}

/* Fully normalised associated Legendre functions without the Condon-Shortley
 * phase, Pbar_n^m(x) = sqrt((2n+1)/(4 pi) (n-m)!/(n+m)!) P_n^m(x), 0<=m<=n<=nmax,
 * stored at index n(n+1)/2 + m.  Standard recurrences: the diagonal from
 * Pbar_0^0 = 1/sqrt(4 pi), the first off-diagonal, then the three-term
 * recurrence in n. */
void orc_legendre_norm(int nmax, double x, double* out) {
  double s = sqrt((1.0 - x) * (1.0 + x));
  out[0] = 1.0 / sqrt(4.0 * ORC_PI);
  for (int m = 1; m <= nmax; ++m)
    out[m * (m + 1) / 2 + m] = sqrt((2.0 * m + 1.0) / (2.0 * m)) * s * out[(m - 1) * m / 2 + (m - 1)];
  for (int m = 0; m < nmax; ++m)
    out[(m + 1) * (m + 2) / 2 + m] = sqrt(2.0 * m + 3.0) * x * out[m * (m + 1) / 2 + m];
  for (int m = 0; m <= nmax; ++m) {
    for (int n = m + 2; n <= nmax; ++n) {
      double a = sqrt((4.0 * n * n - 1.0) / ((double)n * n - (double)m * m));
      double b = sqrt((((double)n - 1.0) * (n - 1.0) - (double)m * m) / (4.0 * (n - 1.0) * (n - 1.0) - 1.0));
      out[n * (n + 1) / 2 + m] = a * (x * out[(n - 1) * n / 2 + m] - b * out[(n - 2) * (n - 1) / 2 + m]);
    }
  }
}

/* Row of the synthesis matrix: the real orthonormal spherical harmonics
 * Y_n^m(theta, phi) for 0 <= n <= p, stored at index n^2 + n + m; m > 0 uses
 * sqrt(2) cos(m phi), m < 0 uses sqrt(2) sin(|m| phi), m = 0 the bare
 * normalised Legendre function.  work: (p+1)(p+2)/2 doubles. */
static void sh_basis(int p, double theta, double phi, double* work, double* row) {
  orc_legendre_norm(p, cos(theta), work);
  for (int n = 0; n <= p; ++n) {
    for (int m = -n; m <= n; ++m) {
      int am = m < 0 ? -m : m;
      double y = work[n * (n + 1) / 2 + am];
      if (m > 0) y *= sqrt(2.0) * cos(m * phi);
      if (m < 0) y *= sqrt(2.0) * sin(am * phi);
      row[n * n + n + m] = y;
    }
  }
}

/* Value of the order-p series with coefficients coef at (theta, phi). */
static double sh_eval(int p, const double* coef, double theta, double phi, double* work, double* row) {
  sh_basis(p, theta, phi, work, row);
  double acc = 0.0;
  for (int q = 0; q < (p + 1) * (p + 1); ++q) acc += coef[q] * row[q];
  return acc;
}

/* Number of mesh vertices for grid order P: the (P+1) x 2P grid plus 2 poles. */
int orc_nverts(int P) { return 2 * P * (P + 1) + 2; }
int orc_ntris(int P) { return 4 * P * P + 4 * P; }
int orc_nedges(int P) { return 6 * P * P + 6 * P; }

/* Polar angles theta_i = arccos(x_i) of the grid rings (ascending). */
static void grid_angles(int P, double* theta) {
  double* x = (double*)malloc(sizeof(double) * (P + 1));
  double* w = (double*)malloc(sizeof(double) * (P + 1));
  orc_gl_nodes(P + 1, x, w);
  for (int i = 0; i <= P; ++i) theta[i] = acos(x[i]);
  free(x); free(w);
}

/* (theta, phi) of mesh vertex v of the order-P grid.  Vertex (i, j) has id
 * i*2P + j with theta = theta_i and phi = 2 pi j / (2P); id 2P(P+1) is the
 * north pole (theta = 0), id 2P(P+1)+1 the south pole (theta = pi). */
static void vertex_angles(int P, const double* theta, int v, double* th, double* ph) {
  if (v < 2 * P * (P + 1)) { *th = theta[v / (2 * P)]; *ph = 2.0 * ORC_PI * (v % (2 * P)) / (2.0 * P); }
  else if (v == 2 * P * (P + 1)) { *th = 0.0; *ph = 0.0; }
  else { *th = ORC_PI; *ph = 0.0; }
}

/* Sec. 3.1.2 "upsample the q-grid to a q^up-grid": evaluate the order-p series
 * of one scalar field (coef, (p+1)^2 entries) at every vertex of the order-P
 * mesh by the plain double sum (no transform, no factorisation). */
void orc_synth(int p, int P, const double* coef, double* out) {
  double* theta = (double*)malloc(sizeof(double) * (P + 1));
  double* work = (double*)malloc(sizeof(double) * (p + 1) * (p + 2) / 2);
  double* row = (double*)malloc(sizeof(double) * (p + 1) * (p + 1));
  grid_angles(P, theta);
  for (int v = 0; v < orc_nverts(P); ++v) {
    double th, ph;
    vertex_angles(P, theta, v, &th, &ph);
    out[v] = sh_eval(p, coef, th, ph, work, row);
  }
  free(theta); free(work); free(row);
}

/* One vesicle: coef [2 time][3 coord][(p+1)^2] -> X [2][3][n_v(P)]. */
void orc_synth_vesicle(int p, int P, const double* coef, double* X) {
  int nc = (p + 1) * (p + 1), nv = orc_nverts(P);
  for (int f = 0; f < 6; ++f) orc_synth(p, P, coef + (size_t)f * nc, X + (size_t)f * nv);
}

/* Mesh fidelity (Sec. 3.1.2: the triangle mesh of the q^up-grid must stay
 * within alpha d_m of the smooth surface, ||X^{q^up} - X(phi, theta)||_inf;
 * Fig. 6 estimates the smooth surface by a 4x upsampled grid).  The mesh is
 * read as a map from parameter space: on the grid cell [theta_i,
 * theta_{i+1}] x [phi_j, phi_{j+1}] with a = (theta - theta_i) /
 * (theta_{i+1} - theta_i), b = (phi - phi_j) / (phi_{j+1} - phi_j) it is the
 * planar triangle [q, r, s] = [(i,j), (i+1,j), (i+1,j+1)] for a >= b,
 * q + a (r - q) + b (s - r), and [q, s, u] with u = (i,j+1) for a < b,
 * q + b (u - q) + a (s - u); above ring 0 (below ring P) it is the pole fan
 * N + t ((1-b) X_{0,j} + b X_{0,j+1} - N) with t = theta / theta_0 (S and
 * t = (pi - theta) / (pi - theta_P)).  The error of one field triple is
 * the largest Euclidean distance |mesh(theta, phi) - X(theta, phi)| over the
 * points of the order-(factor P) grid (its Gauss-Legendre rings and
 * phi_k = pi k / (factor P), poles excluded).  X: [3][n_v(P)] mesh vertices
 * of one time level; coef: [3][(p+1)^2]. */
/* The mesh point at parameter (theta, phi) (the map described above); X: [3][n_v(P)]. */
void orc_mesh_point(int P, const double* X, double theta, double phi, double* out) {
  int W = 2 * P, nv = orc_nverts(P);
  double* th = (double*)malloc(sizeof(double) * (P + 1));
  grid_angles(P, th);
  double u = phi / (ORC_PI / P);        /* longitude in cell units */
  int j = (int)floor(u);
  double b = u - j;
  j = ((j % W) + W) % W;
  int j1 = (j + 1) % W;
  for (int c = 0; c < 3; ++c) {
    const double* x = X + (size_t)c * nv;
    double m;
    if (theta < th[0]) {
      double t = theta / th[0], N = x[2 * P * (P + 1)];
      m = N + t * ((1.0 - b) * x[j] + b * x[j1] - N);
    } else if (theta > th[P]) {
      double t = (ORC_PI - theta) / (ORC_PI - th[P]), Sv = x[2 * P * (P + 1) + 1];
      m = Sv + t * ((1.0 - b) * x[P * W + j] + b * x[P * W + j1] - Sv);
    } else {
      int i = 0;
      while (i + 1 < P && th[i + 1] <= theta) ++i;
      double a = (theta - th[i]) / (th[i + 1] - th[i]);
      double q = x[i * W + j], rr = x[(i + 1) * W + j], sv = x[(i + 1) * W + j1], uu = x[i * W + j1];
      m = a >= b ? q + a * (rr - q) + b * (sv - rr) : q + b * (uu - q) + a * (sv - uu);
    }
    out[c] = m;
  }
  free(th);
}

double orc_mesh_fidelity(int p, int P, int factor, const double* coef, const double* X) {
  int Pf = factor * P, nc = (p + 1) * (p + 1);
  double* thf = (double*)malloc(sizeof(double) * (Pf + 1));
  double* work = (double*)malloc(sizeof(double) * (p + 1) * (p + 2) / 2);
  double* row = (double*)malloc(sizeof(double) * nc);
  grid_angles(Pf, thf);
  double worst = 0.0;
  for (int r = 0; r <= Pf; ++r) {
    for (int k = 0; k < 2 * Pf; ++k) {
      double theta = thf[r], phi = ORC_PI * k / Pf, mp[3], d2 = 0.0;
      orc_mesh_point(P, X, theta, phi, mp);
      for (int c = 0; c < 3; ++c) {
        double e = mp[c] - sh_eval(p, coef + (size_t)c * nc, theta, phi, work, row);
        d2 += e * e;
      }
      double d = sqrt(d2);
      if (d > worst) worst = d;
    }
  }
  free(thf); free(work); free(row);
  return worst;
}

/* Fig. 3: split each grid quad along the diagonal (i,j)-(i+1,j+1); close the
 * poles with triangle fans.  Orientation is chosen so that normals point out
 * of the surface (theta runs south, phi east).  tri: [n_f][3].  Triangle id:
 * band quad (i,j) gives 2(i*2P+j) and 2(i*2P+j)+1, north fan j gives 4P^2+j,
 * south fan j gives 4P^2+2P+j. */
int orc_triangles(int P, int32_t* tri) {
  int W = 2 * P, N = W * (P + 1), S = N + 1;
  for (int i = 0; i < P; ++i) {
    for (int j = 0; j < W; ++j) {
      int jn = (j + 1) % W;
      int q = i * W + j, r = (i + 1) * W + j, s = (i + 1) * W + jn, u = i * W + jn;
      int t = 2 * (i * W + j);
      tri[3 * t + 0] = q; tri[3 * t + 1] = r; tri[3 * t + 2] = s;
      tri[3 * (t + 1) + 0] = q; tri[3 * (t + 1) + 1] = s; tri[3 * (t + 1) + 2] = u;
    }
  }
  for (int j = 0; j < W; ++j) {
    int jn = (j + 1) % W, t = 4 * P * P + j;
    tri[3 * t + 0] = N; tri[3 * t + 1] = j; tri[3 * t + 2] = jn;
    t = 4 * P * P + W + j;
    tri[3 * t + 0] = S; tri[3 * t + 1] = P * W + jn; tri[3 * t + 2] = P * W + j;
  }
  return orc_ntris(P);
}

static int cmp_edge(const void* a, const void* b) {
  const int32_t* x = (const int32_t*)a; const int32_t* y = (const int32_t*)b;
  if (x[0] != y[0]) return x[0] < y[0] ? -1 : 1;
  if (x[1] != y[1]) return x[1] < y[1] ? -1 : 1;
  return 0;
}

/* Unique undirected edges of the triangle list, each as (min id, max id),
 * sorted lexicographically.  edge: [n_e][2]. Returns the count. */
int orc_edges(int P, int32_t* edge) {
  int nf = orc_ntris(P);
  int32_t* tri = (int32_t*)malloc(sizeof(int32_t) * 3 * nf);
  int32_t* all = (int32_t*)malloc(sizeof(int32_t) * 6 * nf);
  orc_triangles(P, tri);
  for (int t = 0; t < nf; ++t) {
    for (int k = 0; k < 3; ++k) {
      int32_t a = tri[3 * t + k], b = tri[3 * t + (k + 1) % 3];
      all[2 * (3 * t + k) + 0] = a < b ? a : b;
      all[2 * (3 * t + k) + 1] = a < b ? b : a;
    }
  }
  qsort(all, 3 * nf, 2 * sizeof(int32_t), cmp_edge);
  int ne = 0;
  for (int k = 0; k < 3 * nf; ++k) {
    if (ne > 0 && all[2 * k] == edge[2 * (ne - 1)] && all[2 * k + 1] == edge[2 * (ne - 1) + 1]) continue;
    edge[2 * ne] = all[2 * k]; edge[2 * ne + 1] = all[2 * k + 1]; ++ne;
  }
  free(tri); free(all);
  return ne;
}

/* ------------------------------------------------------------------------ */
/* Sec. 3.3.1 / Alg. 1-2: space-time bounding boxes and their overlap.        */
/* ------------------------------------------------------------------------ */

/* Alg. 2 getBoundingBox: box of one vesicle over both time levels, padded by
 * d_m.  X: [2][3][nv].  box: lo xyz, hi xyz. */
void orc_vesicle_box(int nv, const double* X, double dm, double* box) {
  for (int c = 0; c < 3; ++c) {
    double lo = X[c * nv], hi = X[c * nv];
    for (int t = 0; t < 2; ++t)
      for (int k = 0; k < nv; ++k) {
        double v = X[(t * 3 + c) * nv + k];
        if (v < lo) lo = v;
        if (v > hi) hi = v;
      }
    box[c] = lo - dm;
    box[3 + c] = hi + dm;
  }
}

/* Alg. 1 bbiCheck: closed-interval overlap on all three axes. */
static int bbi_check(const double* a, const double* b) {
  for (int c = 0; c < 3; ++c)
    if (!(a[c] <= b[3 + c] && b[c] <= a[3 + c])) return 0;
  return 1;
}

/* Candidate vesicle pairs (i < j, image shift s of j in {-1,0,1}^3 on each
 * periodic axis; s = 0 on free axes).  Every pair and every shift is tested.
 * Output rows (i, j, sx, sy, sz) in lexicographic order.  Returns the number
 * of pairs (rows written only up to cap). */
int64_t orc_candidate_pairs(int n, const double* boxes, const double* L, int64_t cap, int32_t* out) {
  int64_t cnt = 0;
  for (int i = 0; i < n; ++i)
    for (int j = i + 1; j < n; ++j)
      for (int sx = -1; sx <= 1; ++sx)
        for (int sy = -1; sy <= 1; ++sy)
          for (int sz = -1; sz <= 1; ++sz) {
            int s[3] = {sx, sy, sz};
            int ok = 1;
            for (int c = 0; c < 3; ++c) if (L[c] == 0.0 && s[c] != 0) ok = 0;
            if (!ok) continue;
            double bj[6];
            for (int c = 0; c < 3; ++c) {
              bj[c] = boxes[6 * j + c];
              bj[3 + c] = boxes[6 * j + 3 + c];
              if (s[c] != 0) { bj[c] = bj[c] + s[c] * L[c]; bj[3 + c] = bj[3 + c] + s[c] * L[c]; }
            }
            if (bbi_check(boxes + 6 * i, bj)) {
              if (cnt < cap) {
                out[5 * cnt + 0] = i; out[5 * cnt + 1] = j;
                out[5 * cnt + 2] = sx; out[5 * cnt + 3] = sy; out[5 * cnt + 4] = sz;
              }
              ++cnt;
            }
          }
  return cnt;
}

/* ------------------------------------------------------------------------ */
/* Sec. 3.1.2, Eq. 3.1 with d_m = 0: earliest contact time of a primitive    */
/* pair moving linearly from X0 (t_n) to X1 (t_{n+1}).                        */
/* ------------------------------------------------------------------------ */

typedef struct { double x, y, z; } v3;
static v3 v3sub(v3 a, v3 b) { v3 r = {a.x - b.x, a.y - b.y, a.z - b.z}; return r; }
static v3 v3add(v3 a, v3 b) { v3 r = {a.x + b.x, a.y + b.y, a.z + b.z}; return r; }
/* Products are accumulated with fused multiply-add (C99 fma, one rounding per
 * step) in the fixed order written here; the CUDA path evaluates the decision
 * arithmetic (cubic, roots, inside test) in the same order so that contact
 * lists and contact times agree bit for bit. */
static v3 v3cross(v3 a, v3 b) {
  v3 r = {fma(a.y, b.z, -(a.z * b.y)), fma(a.z, b.x, -(a.x * b.z)), fma(a.x, b.y, -(a.y * b.x))};
  return r;
}
static double v3dot(v3 a, v3 b) { return fma(a.z, b.z, fma(a.y, b.y, a.x * b.x)); }
static v3 v3lerp(v3 x0, double t, v3 d) { v3 r = {fma(t, d.x, x0.x), fma(t, d.y, x0.y), fma(t, d.z, x0.z)}; return r; }

/* Coplanarity cubic f(t) = c(t) . (a(t) x b(t)), a(t) = a + t da etc.
 * VF: a = x1-x0, b = x2-x0, c = xp-x0 (the 4 points of Eq. 3.1).
 * EE: a = p1-p0, b = q1-q0, c = q0-p0 (the two edge lines are coplanar). */
static void cubic_coeffs(v3 a, v3 b, v3 c, v3 da, v3 db, v3 dc, double k[4]) {
  v3 n0 = v3cross(a, b);
  v3 n1 = v3add(v3cross(da, b), v3cross(a, db));
  v3 n2 = v3cross(da, db);
  k[0] = v3dot(c, n0);
  k[1] = v3dot(dc, n0) + v3dot(c, n1);
  k[2] = v3dot(c, n2) + v3dot(dc, n1);
  k[3] = v3dot(dc, n2);
}

static double horner(const double k[4], double t) { return fma(fma(fma(k[3], t, k[2]), t, k[1]), t, k[0]); }

/* Critical points of f in the open interval (0,1), ascending; returns count.
 * *ops counts the floating-point operations executed (see ccd_pair). */
static int critical_points(const double k[4], double cp[2], int64_t* ops) {
  double d0 = k[1], d1 = 2.0 * k[2], d2 = 3.0 * k[3];
  double r[2]; int nr = 0;
  *ops += 2;
  if (d2 != 0.0) {
    double disc = fma(d1, d1, -((4.0 * d2) * d0));
    *ops += 4;
    if (disc > 0.0) {
      double sq = sqrt(disc);
      double q = -0.5 * (d1 + (d1 >= 0.0 ? sq : -sq));
      r[0] = q / d2; r[1] = d0 / q; nr = 2;
      *ops += 5;
    }
  } else if (d1 != 0.0) {
    r[0] = -d0 / d1; nr = 1;
    *ops += 1;
  }
  int n = 0;
  for (int i = 0; i < nr; ++i) if (r[i] > 0.0 && r[i] < 1.0) cp[n++] = r[i];
  if (n == 2) {
    if (cp[1] < cp[0]) { double t = cp[0]; cp[0] = cp[1]; cp[1] = t; }
    if (cp[1] == cp[0]) n = 1;
  }
  return n;
}

/* Bisection on [lo, hi] where f(lo) != 0 and f changes sign (or f(hi) == 0):
 * at most 64 halvings; stops when the midpoint equals an end or f(mid) == 0.
 * Returns the left end of the final bracket (the last time before the sign
 * change), or mid when f(mid) == 0. */
static double bisect(const double k[4], double lo, double hi, double flo, int64_t* ops) {
  for (int it = 0; it < 64; ++it) {
    double mid = (lo + hi) * 0.5;
    *ops += 2;
    if (!(mid > lo && mid < hi)) break;
    double fm = horner(k, mid);
    *ops += 6;
    if (fm == 0.0) return mid;
    if ((fm < 0.0) == (flo < 0.0)) { lo = mid; flo = fm; }
    else hi = mid;
  }
  return lo;
}

enum { ORC_VF = 0, ORC_EE = 1 };
enum { ORC_HIT = 1, ORC_DEGEN = 2 };

/* Inside test at time t.  VF: barycentric coordinates of xp(t) in triangle
 * x0 x1 x2 (t) from the normal equations; inside iff all three >= 0.
 * EE: parameters (s, u) of the closest points p0 + s d1 and q0 + u d2 of the
 * two lines; inside iff both in [0, 1].  Y: positions at t (4 points: VF
 * xp,x0,x1,x2; EE p0,p1,q0,q1).  Returns 1 inside, 0 outside, -1 degenerate. */
static int inside_test(int kind, const v3* Y, double* w1, double* w2, int64_t* ops) {
  *ops += 9 + 25 + 3;  /* 3 differences, 5 dot products, determinant */
  if (kind == ORC_VF) {
    v3 a = v3sub(Y[2], Y[1]), b = v3sub(Y[3], Y[1]), c = v3sub(Y[0], Y[1]);
    double d00 = v3dot(a, a), d01 = v3dot(a, b), d11 = v3dot(b, b);
    double d20 = v3dot(c, a), d21 = v3dot(c, b);
    double den = fma(d00, d11, -(d01 * d01));
    if (!(den > 0.0)) return -1;
    *ops += 4 + 4 + 2;
    double b1 = fma(d11, d20, -(d01 * d21)) / den;
    double b2 = fma(d00, d21, -(d01 * d20)) / den;
    double b0 = (1.0 - b1) - b2;
    *w1 = b1; *w2 = b2;
    return (b0 >= 0.0 && b1 >= 0.0 && b2 >= 0.0) ? 1 : 0;
  } else {
    v3 d1 = v3sub(Y[1], Y[0]), d2 = v3sub(Y[3], Y[2]), r = v3sub(Y[0], Y[2]);
    double A = v3dot(d1, d1), B = v3dot(d1, d2), E = v3dot(d2, d2);
    double C = v3dot(d1, r), F = v3dot(d2, r);
    double den = fma(A, E, -(B * B));
    if (!(den > 0.0)) return -1;
    *ops += 4 + 4;
    double s = fma(B, F, -(C * E)) / den;
    double u = fma(A, F, -(B * C)) / den;
    *w1 = s; *w2 = u;
    return (s >= 0.0 && s <= 1.0 && u >= 0.0 && u <= 1.0) ? 1 : 0;
  }
}

/* Earliest contact time of one primitive pair (Eq. 3.1 with d_m = 0).
 * P0, D: the 4 points at t_n and their displacements X1 - X0.
 * Root isolation: the critical points of f split [0,1] into monotone pieces,
 * visited in time order; a piece with f(l) == 0 gives t = l, one with
 * f(r) == 0 gives t = r, one with a sign change is bisected.  The first root
 * that passes the inside test is the contact time.  f identically zero
 * (coplanar for the whole step) or a degenerate inside test is reported as
 * ORC_DEGEN and is not a contact.  Returns 0 (no contact), ORC_HIT or
 * ORC_DEGEN; on a hit writes tau and the two inside-test weights.
 * *ops (if not NULL) is increased by the number of floating-point operations
 * the procedure executed on this pair: +, -, *, /, sqrt count 1, fma 2,
 * negation and comparisons 0 (the algorithmic work of the contact test). */
static int ccd_pair(int kind, const v3* P0, const v3* D, double* tau, double* w1, double* w2, int64_t* ops_out) {
  int64_t ops = 18 + 39 + 32;  /* 6 differences, 4 cross products + sum, 6 dot products + 2 sums */
  v3 a, b, c, da, db, dc;
  if (kind == ORC_VF) {  /* points: xp, x0, x1, x2 */
    a = v3sub(P0[2], P0[1]); b = v3sub(P0[3], P0[1]); c = v3sub(P0[0], P0[1]);
    da = v3sub(D[2], D[1]); db = v3sub(D[3], D[1]); dc = v3sub(D[0], D[1]);
  } else {               /* points: p0, p1, q0, q1 */
    a = v3sub(P0[1], P0[0]); b = v3sub(P0[3], P0[2]); c = v3sub(P0[2], P0[0]);
    da = v3sub(D[1], D[0]); db = v3sub(D[3], D[2]); dc = v3sub(D[2], D[0]);
  }
  double k[4];
  cubic_coeffs(a, b, c, da, db, dc, k);
  if (k[0] == 0.0 && k[1] == 0.0 && k[2] == 0.0 && k[3] == 0.0) {
    if (ops_out) *ops_out += ops;
    return ORC_DEGEN;
  }
  double cp[2];
  int ncp = critical_points(k, cp, &ops);
  double ends[4]; int ne = 0;
  ends[ne++] = 0.0;
  for (int i = 0; i < ncp; ++i) ends[ne++] = cp[i];
  ends[ne++] = 1.0;
  int degen = 0;
  for (int s = 0; s + 1 < ne; ++s) {
    double l = ends[s], r = ends[s + 1];
    double fl = horner(k, l), fr = horner(k, r), t;
    ops += 12;
    if (fl == 0.0) t = l;
    else if (fr == 0.0) t = r;
    else if ((fl < 0.0) != (fr < 0.0)) t = bisect(k, l, r, fl, &ops);
    else continue;
    v3 Y[4];
    for (int q = 0; q < 4; ++q) Y[q] = v3lerp(P0[q], t, D[q]);
    ops += 24;
    double u1 = 0.0, u2 = 0.0;
    int in = inside_test(kind, Y, &u1, &u2, &ops);
    if (in < 0) { degen = 1; continue; }
    if (in == 1) {
      *tau = t; *w1 = u1; *w2 = u2;
      if (ops_out) *ops_out += ops;
      return ORC_HIT;
    }
  }
  if (ops_out) *ops_out += ops;
  return degen ? ORC_DEGEN : 0;
}

/* Exposed single-primitive test (closed-form pins in the tests).
 * X0, X1: [4][3] positions of the 4 points.  out: tau, w1, w2. */
int orc_ccd_primitive(int kind, const double* X0, const double* X1, double* out) {
  v3 P0[4], D[4];
  for (int q = 0; q < 4; ++q) {
    P0[q].x = X0[3 * q]; P0[q].y = X0[3 * q + 1]; P0[q].z = X0[3 * q + 2];
    D[q].x = X1[3 * q] - X0[3 * q]; D[q].y = X1[3 * q + 1] - X0[3 * q + 1]; D[q].z = X1[3 * q + 2] - X0[3 * q + 2];
  }
  double t = 0.0, w1 = 0.0, w2 = 0.0;
  int st = ccd_pair(kind, P0, D, &t, &w1, &w2, NULL);
  out[0] = t; out[1] = w1; out[2] = w2;
  return st;
}

/* ------------------------------------------------------------------------ */
/* Eq. 3.1 with d_m > 0: the degree-six equation                              */
/* ------------------------------------------------------------------------ */

/* Horner value of the degree-n polynomial c[0..n] at t (fused multiply-adds). */
static double horner_n(const double* c, int n, double t) {
  double r = c[n];
  for (int i = n - 1; i >= 0; --i) r = fma(r, t, c[i]);
  return r;
}

/* The cubic test's bisection for a degree-n polynomial. */
static double bisect_n(const double* c, int n, double lo, double hi, double flo) {
  for (int it = 0; it < 64; ++it) {
    double mid = (lo + hi) * 0.5;
    if (!(mid > lo && mid < hi)) break;
    double fm = horner_n(c, n, mid);
    if (fm == 0.0) return mid;
    if ((fm < 0.0) == (flo < 0.0)) { lo = mid; flo = fm; }
    else hi = mid;
  }
  return lo;
}

/* Roots in (0, 1) of the degree-n polynomial c (1 <= n <= 6), ascending.
 * The roots of the derivative (found the same way, down to a linear
 * function) split [0, 1] into pieces on which c is monotone, so each piece
 * holds at most one root; a piece is taken as in the cubic test: its left end
 * if c vanishes there, else its right end if c vanishes there, else the
 * bisection of a sign change. */
static int poly_roots01(const double* c, int n, double* out) {
  if (n == 1) {
    if (c[1] == 0.0) return 0;
    double t = -c[0] / c[1];
    if (t > 0.0 && t < 1.0) { out[0] = t; return 1; }
    return 0;
  }
  double dc[6];
  for (int i = 0; i < n; ++i) dc[i] = (double)(i + 1) * c[i + 1];
  double cp[6];
  int ncp = poly_roots01(dc, n - 1, cp);
  double ends[8]; int ne = 0;
  ends[ne++] = 0.0;
  for (int i = 0; i < ncp; ++i) ends[ne++] = cp[i];
  ends[ne++] = 1.0;
  int nr = 0;
  for (int s = 0; s + 1 < ne; ++s) {
    double l = ends[s], r = ends[s + 1];
    double fl = horner_n(c, n, l), fr = horner_n(c, n, r), t;
    if (fl == 0.0) t = l;
    else if (fr == 0.0) t = r;
    else if ((fl < 0.0) != (fr < 0.0)) t = bisect_n(c, n, l, r, fl);
    else continue;
    if (t > 0.0 && t < 1.0 && (nr == 0 || t > out[nr - 1])) out[nr++] = t;
  }
  return nr;
}

/* Coefficients g[0..6] of g(t) = f(t)^2 - d_m^2 |m(t)|^2 (Eq. 3.1): f the
 * coplanarity cubic (k), m(t) = n0 + n1 t + n2 t^2 the normal a x b (VF) or
 * d1 x d2 (EE); |f| / |m| is the distance of the point to the plane (VF) or
 * between the lines (EE).  Fixed order of the FP64 operations. */
static void sextic_coeffs(v3 a, v3 b, v3 c, v3 da, v3 db, v3 dc, double dm, double g[7]) {
  double k[4];
  cubic_coeffs(a, b, c, da, db, dc, k);
  v3 n0 = v3cross(a, b);
  v3 n1 = v3add(v3cross(da, b), v3cross(a, db));
  v3 n2 = v3cross(da, db);
  double q0 = v3dot(n0, n0);
  double q1 = 2.0 * v3dot(n0, n1);
  double q2 = v3dot(n1, n1) + 2.0 * v3dot(n0, n2);
  double q3 = 2.0 * v3dot(n1, n2);
  double q4 = v3dot(n2, n2);
  double dd = dm * dm;
  g[0] = k[0] * k[0] - dd * q0;
  g[1] = 2.0 * (k[0] * k[1]) - dd * q1;
  g[2] = (2.0 * (k[0] * k[2]) + k[1] * k[1]) - dd * q2;
  g[3] = 2.0 * (k[0] * k[3] + k[1] * k[2]) - dd * q3;
  g[4] = (2.0 * (k[1] * k[3]) + k[2] * k[2]) - dd * q4;
  g[5] = 2.0 * (k[2] * k[3]);
  g[6] = k[3] * k[3];
}

static void prim_vectors(int kind, const v3* P0, const v3* D, v3* a, v3* b, v3* c, v3* da, v3* db, v3* dc) {
  if (kind == ORC_VF) {
    *a = v3sub(P0[2], P0[1]); *b = v3sub(P0[3], P0[1]); *c = v3sub(P0[0], P0[1]);
    *da = v3sub(D[2], D[1]); *db = v3sub(D[3], D[1]); *dc = v3sub(D[0], D[1]);
  } else {
    *a = v3sub(P0[1], P0[0]); *b = v3sub(P0[3], P0[2]); *c = v3sub(P0[2], P0[0]);
    *da = v3sub(D[1], D[0]); *db = v3sub(D[3], D[2]); *dc = v3sub(D[2], D[0]);
  }
}

/* Earliest time in [0, 1] at which the point comes within d_m of the
 * triangle's plane (the lines come within d_m), with the inside test of the
 * cubic at that time (the point's projection in the closed triangle; the
 * closest points within both edges).  The roots of g' split [0, 1] into
 * monotone pieces, visited in time order and taken as in the cubic test; the
 * first piece is also taken at t = 0 when g(0) <= 0 (already within d_m at the
 * start of the step).  All g identically zero is degenerate. */
static int ccd_pair_dm(int kind, const v3* P0, const v3* D, double dm, double* tau, double* w1, double* w2) {
  v3 a, b, c, da, db, dc;
  prim_vectors(kind, P0, D, &a, &b, &c, &da, &db, &dc);
  double g[7];
  sextic_coeffs(a, b, c, da, db, dc, dm, g);
  int allz = 1;
  for (int i = 0; i <= 6; ++i) if (g[i] != 0.0) allz = 0;
  if (allz) return ORC_DEGEN;
  double dg[6];
  for (int i = 0; i < 6; ++i) dg[i] = (double)(i + 1) * g[i + 1];
  double cp[6];
  int ncp = poly_roots01(dg, 5, cp);
  double ends[8]; int ne = 0;
  ends[ne++] = 0.0;
  for (int i = 0; i < ncp; ++i) ends[ne++] = cp[i];
  ends[ne++] = 1.0;
  int degen = 0;
  for (int s = 0; s + 1 < ne; ++s) {
    double l = ends[s], r = ends[s + 1];
    double gl = horner_n(g, 6, l), gr = horner_n(g, 6, r), t;
    if (s == 0 && gl <= 0.0) t = l;
    else if (gl == 0.0) t = l;
    else if (gr == 0.0) t = r;
    else if ((gl < 0.0) != (gr < 0.0)) t = bisect_n(g, 6, l, r, gl);
    else continue;
    v3 Y[4];
    for (int q = 0; q < 4; ++q) Y[q] = v3lerp(P0[q], t, D[q]);
    double u1 = 0.0, u2 = 0.0;
    int64_t uncounted = 0;   /* the operation count covers the d_m = 0 procedure */
    int in = inside_test(kind, Y, &u1, &u2, &uncounted);
    if (in < 0) { degen = 1; continue; }
    if (in == 1) { *tau = t; *w1 = u1; *w2 = u2; return ORC_HIT; }
  }
  return degen ? ORC_DEGEN : 0;
}

/* Exposed root isolation (pins): roots in (0, 1) of c[0..n], n <= 6. */
int orc_poly_roots01(const double* c, int n, double* out) { return poly_roots01(c, n, out); }

/* Exposed single-primitive test with d_m > 0 (closed-form pins). */
int orc_ccd_primitive_dm(int kind, const double* X0, const double* X1, double dm, double* out) {
  v3 P0[4], D[4];
  for (int q = 0; q < 4; ++q) {
    P0[q].x = X0[3 * q]; P0[q].y = X0[3 * q + 1]; P0[q].z = X0[3 * q + 2];
    D[q].x = X1[3 * q] - X0[3 * q]; D[q].y = X1[3 * q + 1] - X0[3 * q + 1]; D[q].z = X1[3 * q + 2] - X0[3 * q + 2];
  }
  double t = 0.0, w1 = 0.0, w2 = 0.0;
  int st = dm > 0.0 ? ccd_pair_dm(kind, P0, D, dm, &t, &w1, &w2) : ccd_pair(kind, P0, D, &t, &w1, &w2, NULL);
  out[0] = t; out[1] = w1; out[2] = w2;
  return st;
}

/* ------------------------------------------------------------------------ */
/* Eq. 3.2 and App. A: contact volume of one primitive pair and its gradient */
/* with respect to the end-of-step positions X1 (X0 fixed).                   */
/* ------------------------------------------------------------------------ */

/* Forward-mode dual number with 12 tangent directions (3 coordinates of the
 * 4 points).  Slow and plain on purpose. */
#define ND 12
typedef struct { double v; double d[ND]; } dual;
static dual dc_(double v) { dual r; r.v = v; memset(r.d, 0, sizeof r.d); return r; }
static dual dadd(dual a, dual b) { dual r; r.v = a.v + b.v; for (int i = 0; i < ND; ++i) r.d[i] = a.d[i] + b.d[i]; return r; }
static dual dsub(dual a, dual b) { dual r; r.v = a.v - b.v; for (int i = 0; i < ND; ++i) r.d[i] = a.d[i] - b.d[i]; return r; }
static dual dmul(dual a, dual b) { dual r; r.v = a.v * b.v; for (int i = 0; i < ND; ++i) r.d[i] = a.d[i] * b.v + a.v * b.d[i]; return r; }
static dual ddiv(dual a, dual b) {
  dual r; r.v = a.v / b.v;
  for (int i = 0; i < ND; ++i) r.d[i] = (a.d[i] * b.v - a.v * b.d[i]) / (b.v * b.v);
  return r;
}
static dual dsqrt(dual a) { dual r; r.v = sqrt(a.v); for (int i = 0; i < ND; ++i) r.d[i] = a.d[i] / (2.0 * r.v); return r; }

typedef struct { dual x, y, z; } d3;
static d3 d3sub(d3 a, d3 b) { d3 r = {dsub(a.x, b.x), dsub(a.y, b.y), dsub(a.z, b.z)}; return r; }
static d3 d3add(d3 a, d3 b) { d3 r = {dadd(a.x, b.x), dadd(a.y, b.y), dadd(a.z, b.z)}; return r; }
static d3 d3scale(dual s, d3 a) { d3 r = {dmul(s, a.x), dmul(s, a.y), dmul(s, a.z)}; return r; }
static d3 d3cross(d3 a, d3 b) {
  d3 r = {dsub(dmul(a.y, b.z), dmul(a.z, b.y)), dsub(dmul(a.z, b.x), dmul(a.x, b.z)), dsub(dmul(a.x, b.y), dmul(a.y, b.x))};
  return r;
}
static dual d3dot(d3 a, d3 b) { return dadd(dadd(dmul(a.x, b.x), dmul(a.y, b.y)), dmul(a.z, b.z)); }
static d3 d3lerp(d3 x0, dual t, d3 d) { return d3add(x0, d3scale(t, d)); }

/* V_k of Eq. 3.2 with t - tau_I read as (1 - tau) Delta t in normalised time,
 * U_k the velocity of the contact point relative to the opposite primitive,
 * n and |t| taken at tau:
 *   V_k = (1 - tau) dt sqrt(eps^2 + (U_rel . n)^2) |t|
 *       = 0.5 (1 - tau) sqrt((eps dt)^2 |m|^2 + (D_rel . m)^2),  m = a(tau) x b(tau),
 * where D_rel = U_rel dt.  For VF, |t| = |m|/2 is the triangle area; for EE the
 * same weight |m|/2 of the two edge vectors is used.  The gradient with respect
 * to X1 follows tau through the implicit function f(tau; X1) = 0,
 * d tau = -(df/dX1)/f'(tau), and the inside-test weights through their normal
 * equations.  X0, X1: [4][3].  out: V, then grad [4][3].
 *
 * Variants (the literal readings): velocity_abs = 1 takes U_k as the
 * absolute velocity of the contact point instead of the relative one: for VF
 * the vertex's displacement D_p, for EE that of the point p(s) on the first
 * edge.  grad_x0 = 1 differentiates with respect to the start positions X0
 * (X1 fixed) instead: tau follows through f(tau; X0) = 0 the same way. */
static double stiv_pair_dual(int kind, const v3* P0, const v3* P1, double tau, double eps_dt, double dm,
                             int velocity_abs, int grad_x0, double* grad) {
  d3 X0[4], X1[4], D[4];
  for (int q = 0; q < 4; ++q) {
    X0[q].x = dc_(P0[q].x); X0[q].y = dc_(P0[q].y); X0[q].z = dc_(P0[q].z);
    X1[q].x = dc_(P1[q].x); X1[q].y = dc_(P1[q].y); X1[q].z = dc_(P1[q].z);
    d3* seed = grad_x0 ? &X0[q] : &X1[q];
    seed->x.d[3 * q + 0] = 1.0; seed->y.d[3 * q + 1] = 1.0; seed->z.d[3 * q + 2] = 1.0;
    D[q] = d3sub(X1[q], X0[q]);
  }
  /* df/dX at fixed tau, by evaluating the coplanarity function on duals */
  dual tc = dc_(tau);
  d3 Y[4];
  for (int q = 0; q < 4; ++q) Y[q] = d3lerp(X0[q], tc, D[q]);
  dual f;
  d3 mt;   /* the normal at fixed tau */
  if (kind == ORC_VF) {
    mt = d3cross(d3sub(Y[2], Y[1]), d3sub(Y[3], Y[1]));
    f = d3dot(d3sub(Y[0], Y[1]), mt);
  } else {
    mt = d3cross(d3sub(Y[1], Y[0]), d3sub(Y[3], Y[2]));
    f = d3dot(d3sub(Y[2], Y[0]), mt);
  }
  /* f'(tau) from the cubic's coefficients */
  v3 a, b, c, da, db, dcv;
  v3 Dv[4];
  for (int q = 0; q < 4; ++q) Dv[q] = v3sub(P1[q], P0[q]);
  if (kind == ORC_VF) {
    a = v3sub(P0[2], P0[1]); b = v3sub(P0[3], P0[1]); c = v3sub(P0[0], P0[1]);
    da = v3sub(Dv[2], Dv[1]); db = v3sub(Dv[3], Dv[1]); dcv = v3sub(Dv[0], Dv[1]);
  } else {
    a = v3sub(P0[1], P0[0]); b = v3sub(P0[3], P0[2]); c = v3sub(P0[2], P0[0]);
    da = v3sub(Dv[1], Dv[0]); db = v3sub(Dv[3], Dv[2]); dcv = v3sub(Dv[2], Dv[0]);
  }
  double k[4];
  cubic_coeffs(a, b, c, da, db, dcv, k);
  double fp = (3.0 * k[3] * tau + 2.0 * k[2]) * tau + k[1];
  if (dm > 0.0) {
    /* tau follows g = f^2 - d_m^2 |m|^2 = 0 (Eq. 3.1) instead of f = 0 */
    double g[7];
    sextic_coeffs(a, b, c, da, db, dcv, dm, g);
    fp = ((((6.0 * g[6] * tau + 5.0 * g[5]) * tau + 4.0 * g[4]) * tau + 3.0 * g[3]) * tau + 2.0 * g[2]) * tau + g[1];
    f = dsub(dmul(f, f), dmul(dc_(dm * dm), d3dot(mt, mt)));
  }
  dual td = dc_(tau);
  for (int i = 0; i < ND; ++i) td.d[i] = -f.d[i] / fp;
  /* positions at the contact time, now carrying d tau */
  for (int q = 0; q < 4; ++q) Y[q] = d3lerp(X0[q], td, D[q]);
  d3 m, Drel;
  if (kind == ORC_VF) {
    d3 ea = d3sub(Y[2], Y[1]), eb = d3sub(Y[3], Y[1]), ec = d3sub(Y[0], Y[1]);
    dual d00 = d3dot(ea, ea), d01 = d3dot(ea, eb), d11 = d3dot(eb, eb);
    dual d20 = d3dot(ec, ea), d21 = d3dot(ec, eb);
    dual den = dsub(dmul(d00, d11), dmul(d01, d01));
    dual b1 = ddiv(dsub(dmul(d11, d20), dmul(d01, d21)), den);
    dual b2 = ddiv(dsub(dmul(d00, d21), dmul(d01, d20)), den);
    dual b0 = dsub(dsub(dc_(1.0), b1), b2);
    m = d3cross(ea, eb);
    d3 Dtri = d3add(d3add(d3scale(b0, D[1]), d3scale(b1, D[2])), d3scale(b2, D[3]));
    Drel = velocity_abs ? D[0] : d3sub(D[0], Dtri);
  } else {
    d3 d1 = d3sub(Y[1], Y[0]), d2 = d3sub(Y[3], Y[2]), r = d3sub(Y[0], Y[2]);
    dual A = d3dot(d1, d1), B = d3dot(d1, d2), E = d3dot(d2, d2);
    dual C = d3dot(d1, r), F = d3dot(d2, r);
    dual den = dsub(dmul(A, E), dmul(B, B));
    dual s = ddiv(dsub(dmul(B, F), dmul(C, E)), den);
    dual u = ddiv(dsub(dmul(A, F), dmul(B, C)), den);
    m = d3cross(d1, d2);
    d3 Dp = d3add(d3scale(dsub(dc_(1.0), s), D[0]), d3scale(s, D[1]));
    d3 Dq = d3add(d3scale(dsub(dc_(1.0), u), D[2]), d3scale(u, D[3]));
    Drel = velocity_abs ? Dp : d3sub(Dq, Dp);
  }
  dual e2 = dc_(eps_dt * eps_dt);
  dual um = d3dot(Drel, m);
  dual Q = dadd(dmul(e2, d3dot(m, m)), dmul(um, um));
  dual V = dmul(dmul(dc_(0.5), dsub(dc_(1.0), td)), dsqrt(Q));
  if (grad) for (int i = 0; i < ND; ++i) grad[i] = V.d[i];
  return V.v;
}

/* Exposed per-primitive volume: X0, X1 [4][3]; recomputes tau with the
 * contact test.  out: V, grad[12] (w.r.t. X0 when grad_x0).  Returns the
 * contact status. */
int orc_stiv_primitive_v(int kind, const double* X0, const double* X1, double eps_dt, double dm, int velocity_abs,
                         int grad_x0, double* out) {
  v3 P0[4], P1[4], D[4];
  for (int q = 0; q < 4; ++q) {
    P0[q].x = X0[3 * q]; P0[q].y = X0[3 * q + 1]; P0[q].z = X0[3 * q + 2];
    P1[q].x = X1[3 * q]; P1[q].y = X1[3 * q + 1]; P1[q].z = X1[3 * q + 2];
    D[q] = v3sub(P1[q], P0[q]);
  }
  double t, w1, w2;
  int st = dm > 0.0 ? ccd_pair_dm(kind, P0, D, dm, &t, &w1, &w2) : ccd_pair(kind, P0, D, &t, &w1, &w2, NULL);
  memset(out, 0, sizeof(double) * 13);
  if (st != ORC_HIT) return st;
  out[0] = stiv_pair_dual(kind, P0, P1, t, eps_dt, dm, velocity_abs, grad_x0, out + 1);
  return st;
}

int orc_stiv_primitive(int kind, const double* X0, const double* X1, double eps_dt, double* out) {
  return orc_stiv_primitive_v(kind, X0, X1, eps_dt, 0.0, 0, 0, out);
}

/* ------------------------------------------------------------------------ */
/* Alg. 2 checkContact for one candidate vesicle pair (i, j, s).              */
/* ------------------------------------------------------------------------ */

typedef struct {
  int P;
  const double* X;  /* [2][3][nv] */
  int nv, nf, ne;
  const int32_t* tri;
  const int32_t* edge;
  double shift[3];  /* added to both time levels */
} ves_view;

static v3 vpos(const ves_view* v, int t, int k) {
  v3 r;
  r.x = v->X[(t * 3 + 0) * v->nv + k];
  r.y = v->X[(t * 3 + 1) * v->nv + k];
  r.z = v->X[(t * 3 + 2) * v->nv + k];
  if (v->shift[0] != 0.0) r.x = r.x + v->shift[0];
  if (v->shift[1] != 0.0) r.y = r.y + v->shift[1];
  if (v->shift[2] != 0.0) r.z = r.z + v->shift[2];
  return r;
}

/* Swept box of a set of vertices (both time levels). */
static void prim_box(const v3* P0, const v3* P1, int n, double* box) {
  box[0] = box[3] = P0[0].x; box[1] = box[4] = P0[0].y; box[2] = box[5] = P0[0].z;
  for (int q = 0; q < n; ++q) {
    v3 pts[2] = {P0[q], P1[q]};
    for (int t = 0; t < 2; ++t) {
      if (pts[t].x < box[0]) box[0] = pts[t].x;
      if (pts[t].y < box[1]) box[1] = pts[t].y;
      if (pts[t].z < box[2]) box[2] = pts[t].z;
      if (pts[t].x > box[3]) box[3] = pts[t].x;
      if (pts[t].y > box[4]) box[4] = pts[t].y;
      if (pts[t].z > box[5]) box[5] = pts[t].z;
    }
  }
}

typedef struct {
  int64_t cap, n;
  int32_t* type; int32_t* a; int32_t* b;
  double* tau; double* w;   /* w: [cap][2] */
  int64_t n_boxpairs, n_degen, n_ops;
} contact_out;

static void push_contact(contact_out* o, int type, int a, int b, double tau, double w1, double w2) {
  if (o->n == o->cap) {
    o->cap = o->cap ? 2 * o->cap : 64;
    o->type = (int32_t*)realloc(o->type, sizeof(int32_t) * o->cap);
    o->a = (int32_t*)realloc(o->a, sizeof(int32_t) * o->cap);
    o->b = (int32_t*)realloc(o->b, sizeof(int32_t) * o->cap);
    o->tau = (double*)realloc(o->tau, sizeof(double) * o->cap);
    o->w = (double*)realloc(o->w, sizeof(double) * 2 * o->cap);
  }
  o->type[o->n] = type; o->a[o->n] = a; o->b[o->n] = b;
  o->tau[o->n] = tau; o->w[2 * o->n] = w1; o->w[2 * o->n + 1] = w2;
  o->n++;
}

static void free_contacts(contact_out* o) {
  free(o->type); free(o->a); free(o->b); free(o->tau); free(o->w);
}

/* Swept boxes of every vertex, triangle and edge of one vesicle view. */
typedef struct { double* vb; double* tb; double* eb; } prim_boxes;

/* pad > 0 widens every box by pad on each side (FP64, as computed), so that
 * two primitives within pad of each other have overlapping boxes. */
static prim_boxes make_boxes(const ves_view* V, double pad) {
  prim_boxes r;
  r.vb = (double*)malloc(sizeof(double) * 6 * V->nv);
  r.tb = (double*)malloc(sizeof(double) * 6 * V->nf);
  r.eb = (double*)malloc(sizeof(double) * 6 * V->ne);
  v3 P0[3], P1[3];
  for (int k = 0; k < V->nv; ++k) { P0[0] = vpos(V, 0, k); P1[0] = vpos(V, 1, k); prim_box(P0, P1, 1, r.vb + 6 * k); }
  for (int t = 0; t < V->nf; ++t) {
    for (int q = 0; q < 3; ++q) { P0[q] = vpos(V, 0, V->tri[3 * t + q]); P1[q] = vpos(V, 1, V->tri[3 * t + q]); }
    prim_box(P0, P1, 3, r.tb + 6 * t);
  }
  for (int e = 0; e < V->ne; ++e) {
    for (int q = 0; q < 2; ++q) { P0[q] = vpos(V, 0, V->edge[2 * e + q]); P1[q] = vpos(V, 1, V->edge[2 * e + q]); }
    prim_box(P0, P1, 2, r.eb + 6 * e);
  }
  if (pad > 0.0) {
    double* all[3] = {r.vb, r.tb, r.eb};
    int cnt[3] = {V->nv, V->nf, V->ne};
    for (int w = 0; w < 3; ++w)
      for (int e = 0; e < cnt[w]; ++e)
        for (int c = 0; c < 3; ++c) { all[w][6 * e + c] = all[w][6 * e + c] - pad; all[w][6 * e + 3 + c] = all[w][6 * e + 3 + c] + pad; }
  }
  return r;
}

static void free_boxes(prim_boxes* b) { free(b->vb); free(b->tb); free(b->eb); }

/* Contacts between vesicles A (unshifted) and B (shifted), in order:
 * type 0 = vertex of A vs triangle of B, type 1 = vertex of B vs triangle of
 * A, type 2 = edge of A vs edge of B (edge index in the sorted edge list);
 * within a type by ascending primitive ids.  prune = 1 skips pairs whose swept boxes
 * do not overlap (a necessary condition for contact); with d_m > 0 B's boxes
 * are widened by d_m and the contact test is the degree-six one. */
static void pair_contacts(const ves_view* A, const ves_view* B, int prune, int include_ee, double dm,
                          contact_out* o) {
  prim_boxes bA = make_boxes(A, 0.0), bB = make_boxes(B, dm);
  for (int dir = 0; dir < 2; ++dir) {
    const ves_view* V = dir == 0 ? A : B;   /* vertex side */
    const ves_view* T = dir == 0 ? B : A;   /* triangle side */
    const prim_boxes* bV = dir == 0 ? &bA : &bB;
    const prim_boxes* bT = dir == 0 ? &bB : &bA;
    for (int vp = 0; vp < V->nv; ++vp) {
      v3 P0[4], P1[4], D[4];
      P0[0] = vpos(V, 0, vp); P1[0] = vpos(V, 1, vp);
      for (int t = 0; t < T->nf; ++t) {
        if (prune && !bbi_check(bV->vb + 6 * vp, bT->tb + 6 * t)) continue;
        for (int q = 0; q < 3; ++q) {
          P0[1 + q] = vpos(T, 0, T->tri[3 * t + q]);
          P1[1 + q] = vpos(T, 1, T->tri[3 * t + q]);
        }
        o->n_boxpairs++;
        for (int q = 0; q < 4; ++q) D[q] = v3sub(P1[q], P0[q]);
        o->n_ops += 12;  /* the displacements */
        double tau, w1, w2;
        int st = dm > 0.0 ? ccd_pair_dm(ORC_VF, P0, D, dm, &tau, &w1, &w2)
                          : ccd_pair(ORC_VF, P0, D, &tau, &w1, &w2, &o->n_ops);
        if (st == ORC_HIT) push_contact(o, dir, vp, t, tau, w1, w2);
        else if (st == ORC_DEGEN) o->n_degen++;
      }
    }
  }
  if (include_ee) {
    for (int ea = 0; ea < A->ne; ++ea) {
      v3 P0[4], P1[4], D[4];
      for (int q = 0; q < 2; ++q) {
        P0[q] = vpos(A, 0, A->edge[2 * ea + q]);
        P1[q] = vpos(A, 1, A->edge[2 * ea + q]);
      }
      for (int eb = 0; eb < B->ne; ++eb) {
        if (prune && !bbi_check(bA.eb + 6 * ea, bB.eb + 6 * eb)) continue;
        for (int q = 0; q < 2; ++q) {
          P0[2 + q] = vpos(B, 0, B->edge[2 * eb + q]);
          P1[2 + q] = vpos(B, 1, B->edge[2 * eb + q]);
        }
        o->n_boxpairs++;
        for (int q = 0; q < 4; ++q) D[q] = v3sub(P1[q], P0[q]);
        o->n_ops += 12;  /* the displacements */
        double tau, w1, w2;
        int st = dm > 0.0 ? ccd_pair_dm(ORC_EE, P0, D, dm, &tau, &w1, &w2)
                          : ccd_pair(ORC_EE, P0, D, &tau, &w1, &w2, &o->n_ops);
        if (st == ORC_HIT) push_contact(o, 2, ea, eb, tau, w1, w2);
        else if (st == ORC_DEGEN) o->n_degen++;
      }
    }
  }
  free_boxes(&bA); free_boxes(&bB);
}

/* The 4 points (and their vertex ids / owning side) of one contact. */
static void contact_points(const ves_view* A, const ves_view* B, int type, int a, int b,
                           v3* P0, v3* P1, int* side, int* vid) {
  if (type == 0 || type == 1) {
    const ves_view* V = type == 0 ? A : B;
    const ves_view* T = type == 0 ? B : A;
    int sv = type == 0 ? 0 : 1;
    P0[0] = vpos(V, 0, a); P1[0] = vpos(V, 1, a); side[0] = sv; vid[0] = a;
    for (int q = 0; q < 3; ++q) {
      int k = T->tri[3 * b + q];
      P0[1 + q] = vpos(T, 0, k); P1[1 + q] = vpos(T, 1, k); side[1 + q] = 1 - sv; vid[1 + q] = k;
    }
  } else {
    int ka[2] = {A->edge[2 * a], A->edge[2 * a + 1]}, kb[2] = {B->edge[2 * b], B->edge[2 * b + 1]};
    for (int q = 0; q < 2; ++q) {
      P0[q] = vpos(A, 0, ka[q]); P1[q] = vpos(A, 1, ka[q]); side[q] = 0; vid[q] = ka[q];
      P0[2 + q] = vpos(B, 0, kb[q]); P1[2 + q] = vpos(B, 1, kb[q]); side[2 + q] = 1; vid[2 + q] = kb[q];
    }
  }
}

/* ------------------------------------------------------------------------ */
/* Alg. 2 ContactVolume over a scene (vesicles of uneven order allowed).      */
/* ------------------------------------------------------------------------ */

typedef struct {
  int P; int32_t* tri; int32_t* edge;
} topo_cache;

static topo_cache* topo_for(topo_cache* cache, int* ncache, int P) {
  for (int i = 0; i < *ncache; ++i) if (cache[i].P == P) return &cache[i];
  topo_cache* c = &cache[(*ncache)++];
  c->P = P;
  c->tri = (int32_t*)malloc(sizeof(int32_t) * 3 * orc_ntris(P));
  c->edge = (int32_t*)malloc(sizeof(int32_t) * 2 * orc_nedges(P));
  orc_triangles(P, c->tri);
  orc_edges(P, c->edge);
  return c;
}

static ves_view make_view(topo_cache* tc, const int* Pv, const int64_t* voff, const double* X, int v, const int* s, const double* L) {
  ves_view r;
  r.P = Pv[v]; r.X = X + voff[v];
  r.nv = orc_nverts(r.P); r.nf = orc_ntris(r.P); r.ne = orc_nedges(r.P);
  r.tri = tc->tri; r.edge = tc->edge;
  for (int c = 0; c < 3; ++c) r.shift[c] = s ? s[c] * L[c] : 0.0;
  return r;
}

/* Contacts of a list of candidate vesicle pairs.
 *   nv_ves: number of vesicles; Pv[v]: grid order of vesicle v; voff[v]: offset
 *   (in doubles) of its [2][3][n_v] block in X.
 *   pairs: [npairs][5] rows (i, j, sx, sy, sz); L: periodic lengths.
 * Output contacts grouped by pair in input order, each group ordered as in
 * pair_contacts.  cpair[k] is the row of the pair.  V_pair[npairs] gets the
 * sum of the pair's V_k in that order.  If grad != NULL, per contact the
 * gradient [4][3] w.r.t. X1 (X0 when grad_x0) of the 4 points and, per
 * point, its vesicle (gves) and local vertex id (gvid) are written;
 * velocity_abs selects the literal reading of U_k (see stiv_pair_dual).
 * counts[0] = contacts, [1] = primitive pairs tested, [2] = degenerate,
 * [3] = floating-point operations of the contact tests (ccd_pair's count).
 * OpenMP over pairs when compiled with it (nthreads <= 0: default). */
int64_t orc_contacts(int nv_ves, const int* Pv, const int64_t* voff, const double* X,
                     int64_t npairs, const int32_t* pairs, const double* L,
                     int prune, int include_ee, double dm, double eps_dt, int velocity_abs, int grad_x0,
                     int nthreads,
                     int64_t cap, int32_t* cpair, int32_t* ctype, int32_t* ca, int32_t* cb,
                     double* ctau, double* cw, double* cV, double* V_pair,
                     double* grad, int32_t* gves, int32_t* gvid, int64_t* counts) {
  (void)nv_ves;
  topo_cache cache[16]; int ncache = 0;
  for (int64_t r = 0; r < npairs; ++r) {
    topo_for(cache, &ncache, Pv[pairs[5 * r]]);
    topo_for(cache, &ncache, Pv[pairs[5 * r + 1]]);
  }
  int64_t* pcnt = (int64_t*)calloc(npairs + 1, sizeof(int64_t));
  contact_out* outs = (contact_out*)calloc(npairs, sizeof(contact_out));
  int64_t nbox = 0, ndeg = 0, nops = 0;
#ifdef _OPENMP
  if (nthreads > 0) omp_set_num_threads(nthreads);
#pragma omp parallel for schedule(dynamic, 1) reduction(+ : nbox, ndeg, nops)
#endif
  for (int64_t r = 0; r < npairs; ++r) {
    int i = pairs[5 * r], j = pairs[5 * r + 1];
    int s[3] = {pairs[5 * r + 2], pairs[5 * r + 3], pairs[5 * r + 4]};
    ves_view A = make_view(topo_for(cache, &ncache, Pv[i]), Pv, voff, X, i, NULL, L);
    ves_view B = make_view(topo_for(cache, &ncache, Pv[j]), Pv, voff, X, j, s, L);
    memset(&outs[r], 0, sizeof(contact_out));
    pair_contacts(&A, &B, prune, include_ee, dm, &outs[r]);
    int64_t n = outs[r].n;
    nbox += outs[r].n_boxpairs; ndeg += outs[r].n_degen; nops += outs[r].n_ops;
    pcnt[r] = n;
  }
  int64_t total = 0;
  for (int64_t r = 0; r < npairs; ++r) {
    int i = pairs[5 * r], j = pairs[5 * r + 1];
    int s[3] = {pairs[5 * r + 2], pairs[5 * r + 3], pairs[5 * r + 4]};
    ves_view A = make_view(topo_for(cache, &ncache, Pv[i]), Pv, voff, X, i, NULL, L);
    ves_view B = make_view(topo_for(cache, &ncache, Pv[j]), Pv, voff, X, j, s, L);
    double vsum = 0.0;
    for (int64_t q = 0; q < pcnt[r]; ++q) {
      int64_t k = total + q;
      v3 P0[4], P1[4]; int side[4], vid[4];
      contact_points(&A, &B, outs[r].type[q], outs[r].a[q], outs[r].b[q], P0, P1, side, vid);
      int kind = outs[r].type[q] == 2 ? ORC_EE : ORC_VF;
      double g[12];
      double V = stiv_pair_dual(kind, P0, P1, outs[r].tau[q], eps_dt, dm, velocity_abs, grad_x0, g);
      vsum += V;
      if (k < cap) {
        cpair[k] = (int32_t)r; ctype[k] = outs[r].type[q]; ca[k] = outs[r].a[q]; cb[k] = outs[r].b[q];
        ctau[k] = outs[r].tau[q]; cw[2 * k] = outs[r].w[2 * q]; cw[2 * k + 1] = outs[r].w[2 * q + 1];
        cV[k] = V;
        if (grad) {
          for (int e = 0; e < 12; ++e) grad[12 * k + e] = g[e];
          for (int e = 0; e < 4; ++e) { gves[4 * k + e] = side[e] == 0 ? i : j; gvid[4 * k + e] = vid[e]; }
        }
      }
    }
    if (V_pair) V_pair[r] = vsum;
    total += pcnt[r];
    free_contacts(&outs[r]);
  }
  for (int i = 0; i < ncache; ++i) { free(cache[i].tri); free(cache[i].edge); }
  free(pcnt); free(outs);
  if (counts) { counts[0] = total; counts[1] = nbox; counts[2] = ndeg; counts[3] = nops; }
  return total;
}

/* ------------------------------------------------------------------------ */
/* Adjoint of the synthesis (back to SH coefficients): gcoef = S^T g, with S  */
/* the synthesis matrix of orc_synth (grid and poles).                        */
/* ------------------------------------------------------------------------ */
void orc_synth_adjoint(int p, int P, const double* g, double* gcoef) {
  int nc = (p + 1) * (p + 1), nv = orc_nverts(P);
  double* theta = (double*)malloc(sizeof(double) * (P + 1));
  double* work = (double*)malloc(sizeof(double) * (p + 1) * (p + 2) / 2);
  double* row = (double*)malloc(sizeof(double) * nc);
  grid_angles(P, theta);
  for (int q = 0; q < nc; ++q) gcoef[q] = 0.0;
  for (int v = 0; v < nv; ++v) {
    double th, ph;
    vertex_angles(P, theta, v, &th, &ph);
    sh_basis(p, th, ph, work, row);
    for (int q = 0; q < nc; ++q) gcoef[q] += g[v] * row[q];
  }
  free(theta); free(work); free(row);
}

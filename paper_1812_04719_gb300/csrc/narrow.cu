// Narrow phase of Alg. 2 checkContact: every vertex-triangle pair (both
// directions) and edge-edge pair of a candidate vesicle pair whose swept boxes
// overlap is tested with the coplanarity cubic of Eq. 3.1 (d_m = 0).
//
// The triangulated grid (Sec. 3.1.2, Fig. 3) is cut into patches of 4 x 8 grid
// quads.  Each primitive belongs to exactly one patch, so a primitive pair is
// examined by exactly one patch pair:
//   level 1 (patch_pairs_kernel): per candidate vesicle pair, one warp tests
//     the FP32 outward-rounded patch boxes and lists overlapping patch pairs;
//   level 2 (narrow_kernel): per patch pair, one warp stages both patches'
//     vertices (FP64, the second one shifted by its periodic image) in shared
//     memory, builds FP32 outward-rounded primitive boxes, keeps the primitive
//     pairs whose FP32 boxes overlap, and queues them; a full queue is drained
//     by the whole warp: exact FP64 box test, then the FP64 contact test.
// FP32 boxes contain the exact FP64 boxes, so the FP32 culling never drops a
// pair that the exact test keeps.
#include "stiv_internal.cuh"

#include <math.h>

namespace {

constexpr int NS = (STIV_BR + 1) * (STIV_BC + 1) + 2;  // vertex slots per patch (+2 poles)
constexpr int SN = NS - 2, SS = NS - 1;               // pole slots
constexpr int MAXV = 48, MAXT = 80, MAXE = 128;
constexpr int NW = 4;                                  // warps per CTA
constexpr int QCAP = 64;                               // queue entries per warp

struct PatchSm {
  double x[6][NS];                 // X0 xyz, X1 xyz per slot (periodic image applied)
  float flo[3][NS], fhi[3][NS];    // FP32 outward box of each slot over both times
  int nv, nt, ne;
  int v_slot[MAXV], v_gid[MAXV];
  int t_slots[MAXT], t_gid[MAXT];  // 3 slots, 6 bits each
  int e_slots[MAXE], e_gid[MAXE];  // 2 slots (min vertex id first)
  float tb[6][MAXT];
  float eb[6][MAXE];
  unsigned char vf[MAXV], tf[MAXT], ef[MAXE];
  int nvf, ntf, nef;
  float box[6];                    // whole patch
};

struct WarpSm {
  PatchSm A, B;
  unsigned q[QCAP];
  int qn;
};

struct narrow_args {
  const int32_t* pv;
  const int64_t* voff;
  const void* X;
  int mixed;
  double L[3];
  const int32_t* ci;
  const int32_t* cj;
  const int32_t* cs;
  const uint64_t* work;
  int64_t W;
  int include_ee;
  int64_t C;  // raw contact capacity
  int32_t* rc_pair; int32_t* rc_type; int32_t* rc_a; int32_t* rc_b;
  double* rc_tau; double* rc_w;
  int64_t* ctr;
};

__device__ __forceinline__ int slot_of(int rr, int cc) { return rr * (STIV_BC + 1) + cc; }

// Stage patch (I, J) of vesicle v into shared memory; shift s applied to both times.
__device__ void load_patch(PatchSm& S, const narrow_args& a, int v, int patch, const int* s, int lane) {
  int P = 2 * a.pv[v], W = 2 * P, nv = stiv_nverts(P);
  int nbr = stiv_nband_blocks(P), nbc = stiv_ncol_blocks(P);
  int I = patch / nbc, J = patch % nbc;
  int r0 = I * STIV_BR, rq = min(STIV_BR, P - r0), c0 = J * STIV_BC, ncol = min(STIV_BC, W - c0);
  bool first = I == 0, last = I == nbr - 1;
  size_t base = a.voff[v];
  double sh[3] = {s[0] * a.L[0], s[1] * a.L[1], s[2] * a.L[2]};
  // vertex slots
  for (int k = lane; k < NS; k += 32) {
    int vid = -1;
    if (k < SN) {
      int rr = k / (STIV_BC + 1), cc = k % (STIV_BC + 1);
      if (rr <= rq && cc <= ncol) { int col = c0 + cc; if (col >= W) col -= W; vid = (r0 + rr) * W + col; }
    } else if (k == SN && first) vid = W * (P + 1);
    else if (k == SS && last) vid = W * (P + 1) + 1;
    if (vid >= 0) {
      for (int f = 0; f < 6; ++f) {
        size_t idx = base + (size_t)f * nv + vid;
        double x = a.mixed ? (double)((const float*)a.X)[idx] : ((const double*)a.X)[idx];
        int c = f % 3;
        if (s[c] != 0) x = x + sh[c];
        S.x[f][k] = x;
      }
      for (int c = 0; c < 3; ++c) {
        double lo = fmin(S.x[c][k], S.x[3 + c][k]), hi = fmax(S.x[c][k], S.x[3 + c][k]);
        S.flo[c][k] = __double2float_rd(lo);
        S.fhi[c][k] = __double2float_ru(hi);
      }
    } else {
      for (int c = 0; c < 3; ++c) { S.flo[c][k] = INFINITY; S.fhi[c][k] = -INFINITY; }
    }
  }
  __syncwarp();
  // primitive counts
  int rown = rq + (last ? 1 : 0);
  int nvg = rown * ncol;
  int npole = (first && J == 0 ? 1 : 0) + (last && J == 0 ? 1 : 0);
  int ntq = 2 * rq * ncol;
  int nfan = (first ? ncol : 0) + (last ? ncol : 0);
  S.nv = nvg + npole;
  S.nt = ntq + nfan;
  S.ne = rown * ncol + 2 * rq * ncol + nfan;
  // vertices
  for (int k = lane; k < S.nv; k += 32) {
    int slot, gid;
    if (k < nvg) {
      int rr = k / ncol, cc = k % ncol;
      slot = slot_of(rr, cc); gid = (r0 + rr) * W + c0 + cc;
    } else if (first && J == 0 && k == nvg) { slot = SN; gid = W * (P + 1); }
    else { slot = SS; gid = W * (P + 1) + 1; }
    S.v_slot[k] = slot; S.v_gid[k] = gid;
  }
  // triangles (vertex order of the mesh definition)
  for (int k = lane; k < S.nt; k += 32) {
    int s0, s1, s2, gid;
    if (k < ntq) {
      int q = k >> 1, rr = q / ncol, cc = q % ncol, i = r0 + rr, j = c0 + cc;
      gid = 2 * (i * W + j) + (k & 1);
      if ((k & 1) == 0) { s0 = slot_of(rr, cc); s1 = slot_of(rr + 1, cc); s2 = slot_of(rr + 1, cc + 1); }
      else { s0 = slot_of(rr, cc); s1 = slot_of(rr + 1, cc + 1); s2 = slot_of(rr, cc + 1); }
    } else {
      int k2 = k - ntq;
      if (first && k2 < ncol) {
        int cc = k2; gid = 4 * P * P + c0 + cc;
        s0 = SN; s1 = slot_of(0, cc); s2 = slot_of(0, cc + 1);
      } else {
        int cc = first ? k2 - ncol : k2; gid = 4 * P * P + W + c0 + cc;
        s0 = SS; s1 = slot_of(rq, cc + 1); s2 = slot_of(rq, cc);
      }
    }
    S.t_slots[k] = s0 | (s1 << 6) | (s2 << 12); S.t_gid[k] = gid;
    for (int c = 0; c < 3; ++c) {
      S.tb[c][k] = fminf(S.flo[c][s0], fminf(S.flo[c][s1], S.flo[c][s2]));
      S.tb[3 + c][k] = fmaxf(S.fhi[c][s0], fmaxf(S.fhi[c][s1], S.fhi[c][s2]));
    }
  }
  // edges: ring edges of owned vertices, then meridian / diagonal edges of owned quads, then pole edges
  for (int k = lane; k < S.ne; k += 32) {
    int sa, sb, va, vb;
    int nh = rown * ncol;
    if (k < nh) {
      int rr = k / ncol, cc = k % ncol, i = r0 + rr, j = c0 + cc, jn = j + 1 == W ? 0 : j + 1;
      sa = slot_of(rr, cc); sb = slot_of(rr, cc + 1); va = i * W + j; vb = i * W + jn;
    } else if (k < nh + 2 * rq * ncol) {
      int k2 = k - nh, q = k2 >> 1, rr = q / ncol, cc = q % ncol, i = r0 + rr, j = c0 + cc;
      int jn = j + 1 == W ? 0 : j + 1;
      sa = slot_of(rr, cc); va = i * W + j;
      if ((k2 & 1) == 0) { sb = slot_of(rr + 1, cc); vb = (i + 1) * W + j; }
      else { sb = slot_of(rr + 1, cc + 1); vb = (i + 1) * W + jn; }
    } else {
      int k2 = k - nh - 2 * rq * ncol;
      if (first && k2 < ncol) { int cc = k2; sa = slot_of(0, cc); va = c0 + cc; sb = SN; vb = W * (P + 1); }
      else {
        int cc = first ? k2 - ncol : k2;
        sa = slot_of(rq, cc); va = P * W + c0 + cc; sb = SS; vb = W * (P + 1) + 1;
      }
    }
    if (vb < va) { int t = va; va = vb; vb = t; t = sa; sa = sb; sb = t; }
    S.e_slots[k] = sa | (sb << 6); S.e_gid[k] = stiv_edge_index(P, va, vb);
    for (int c = 0; c < 3; ++c) {
      S.eb[c][k] = fminf(S.flo[c][sa], S.flo[c][sb]);
      S.eb[3 + c][k] = fmaxf(S.fhi[c][sa], S.fhi[c][sb]);
    }
  }
  __syncwarp();
  // whole-patch box
  if (lane < 6) {
    float acc = lane < 3 ? INFINITY : -INFINITY;
    int c = lane % 3;
    for (int k = 0; k < NS; ++k) acc = lane < 3 ? fminf(acc, S.flo[c][k]) : fmaxf(acc, S.fhi[c][k]);
    S.box[lane] = acc;
  }
  __syncwarp();
}

__device__ __forceinline__ bool fbox_hit(const float* lo_a, const float* hi_a, const float* b) {
  return lo_a[0] <= b[3] && b[0] <= hi_a[0] && lo_a[1] <= b[4] && b[1] <= hi_a[1] && lo_a[2] <= b[5] && b[2] <= hi_a[2];
}

// Compact the primitives of S that overlap box ob (FP32) into S.*f lists.
__device__ void filter_patch(PatchSm& S, const float* ob, int lane) {
  int base;
  base = 0;
  for (int k0 = 0; k0 < S.nv; k0 += 32) {
    int k = k0 + lane;
    bool hit = false;
    if (k < S.nv) {
      int sl = S.v_slot[k];
      float lo[3] = {S.flo[0][sl], S.flo[1][sl], S.flo[2][sl]}, hi[3] = {S.fhi[0][sl], S.fhi[1][sl], S.fhi[2][sl]};
      hit = fbox_hit(lo, hi, ob);
    }
    unsigned m = __ballot_sync(0xffffffffu, hit);
    if (hit) S.vf[base + __popc(m & ((1u << lane) - 1u))] = (unsigned char)k;
    base += __popc(m);
  }
  if (lane == 0) S.nvf = base;
  base = 0;
  for (int k0 = 0; k0 < S.nt; k0 += 32) {
    int k = k0 + lane;
    bool hit = false;
    if (k < S.nt) {
      float lo[3] = {S.tb[0][k], S.tb[1][k], S.tb[2][k]}, hi[3] = {S.tb[3][k], S.tb[4][k], S.tb[5][k]};
      hit = fbox_hit(lo, hi, ob);
    }
    unsigned m = __ballot_sync(0xffffffffu, hit);
    if (hit) S.tf[base + __popc(m & ((1u << lane) - 1u))] = (unsigned char)k;
    base += __popc(m);
  }
  if (lane == 0) S.ntf = base;
  base = 0;
  for (int k0 = 0; k0 < S.ne; k0 += 32) {
    int k = k0 + lane;
    bool hit = false;
    if (k < S.ne) {
      float lo[3] = {S.eb[0][k], S.eb[1][k], S.eb[2][k]}, hi[3] = {S.eb[3][k], S.eb[4][k], S.eb[5][k]};
      hit = fbox_hit(lo, hi, ob);
    }
    unsigned m = __ballot_sync(0xffffffffu, hit);
    if (hit) S.ef[base + __popc(m & ((1u << lane) - 1u))] = (unsigned char)k;
    base += __popc(m);
  }
  if (lane == 0) S.nef = base;
  __syncwarp();
}

// ---------------------------------------------------------------------------
// Eq. 3.1 (d_m = 0): earliest contact time of one primitive pair in FP64
// ---------------------------------------------------------------------------
enum { KIND_VF = 0, KIND_EE = 1 };

// FP64 flops of the procedure, counted as executed (fma = 2): the
// algorithmic work of the exact contact test, reported for the roofline.
__device__ double bisect64(double k0, double k1, double k2, double k3, double lo, double hi, double flo,
                           long long& flops) {
  for (int it = 0; it < 64; ++it) {
    double mid = __dmul_rn(__dadd_rn(lo, hi), 0.5);
    flops += 2;
    if (!(mid > lo && mid < hi)) break;
    flops += 6;
    double fm = horner3(k0, k1, k2, k3, mid);
    if (fm == 0.0) return mid;
    if ((fm < 0.0) == (flo < 0.0)) { lo = mid; flo = fm; }
    else hi = mid;
  }
  return lo;
}

// Inside test at the positions Y (VF: xp, x0, x1, x2; EE: p0, p1, q0, q1).
// 1 inside, 0 outside, -1 degenerate.
__device__ int inside64(int kind, const d3* Y, double& w1, double& w2) {
  if (kind == KIND_VF) {
    d3 a = d3_sub(Y[2], Y[1]), b = d3_sub(Y[3], Y[1]), c = d3_sub(Y[0], Y[1]);
    double d00 = d3_dot(a, a), d01 = d3_dot(a, b), d11 = d3_dot(b, b), d20 = d3_dot(c, a), d21 = d3_dot(c, b);
    double den = __fma_rn(d00, d11, -__dmul_rn(d01, d01));
    if (!(den > 0.0)) return -1;
    double b1 = __ddiv_rn(__fma_rn(d11, d20, -__dmul_rn(d01, d21)), den);
    double b2 = __ddiv_rn(__fma_rn(d00, d21, -__dmul_rn(d01, d20)), den);
    double b0 = __dsub_rn(__dsub_rn(1.0, b1), b2);
    w1 = b1; w2 = b2;
    return (b0 >= 0.0 && b1 >= 0.0 && b2 >= 0.0) ? 1 : 0;
  } else {
    d3 d1 = d3_sub(Y[1], Y[0]), d2 = d3_sub(Y[3], Y[2]), r = d3_sub(Y[0], Y[2]);
    double A = d3_dot(d1, d1), B = d3_dot(d1, d2), E = d3_dot(d2, d2), C = d3_dot(d1, r), F = d3_dot(d2, r);
    double den = __fma_rn(A, E, -__dmul_rn(B, B));
    if (!(den > 0.0)) return -1;
    double s = __ddiv_rn(__fma_rn(B, F, -__dmul_rn(C, E)), den);
    double u = __ddiv_rn(__fma_rn(A, F, -__dmul_rn(B, C)), den);
    w1 = s; w2 = u;
    return (s >= 0.0 && s <= 1.0 && u >= 0.0 && u <= 1.0) ? 1 : 0;
  }
}

// 0 no contact, 1 contact, 2 degenerate.
__device__ int ccd64(int kind, const d3* X0, const d3* D, double& tau, double& w1, double& w2, long long& flops) {
  flops += 18 + 9 + 21 + 9 + 32;  // differences, three cross products (+ sum), four dot products
  d3 a, b, c, da, db, dc;
  if (kind == KIND_VF) {
    a = d3_sub(X0[2], X0[1]); b = d3_sub(X0[3], X0[1]); c = d3_sub(X0[0], X0[1]);
    da = d3_sub(D[2], D[1]); db = d3_sub(D[3], D[1]); dc = d3_sub(D[0], D[1]);
  } else {
    a = d3_sub(X0[1], X0[0]); b = d3_sub(X0[3], X0[2]); c = d3_sub(X0[2], X0[0]);
    da = d3_sub(D[1], D[0]); db = d3_sub(D[3], D[2]); dc = d3_sub(D[2], D[0]);
  }
  d3 n0 = d3_cross(a, b);
  d3 n1 = d3_add(d3_cross(da, b), d3_cross(a, db));
  d3 n2 = d3_cross(da, db);
  double k0 = d3_dot(c, n0);
  double k1 = __dadd_rn(d3_dot(dc, n0), d3_dot(c, n1));
  double k2 = __dadd_rn(d3_dot(c, n2), d3_dot(dc, n1));
  double k3 = d3_dot(dc, n2);
  if (k0 == 0.0 && k1 == 0.0 && k2 == 0.0 && k3 == 0.0) return 2;
  // critical points of the cubic inside (0, 1)
  double e0 = k1, e1 = __dmul_rn(2.0, k2), e2 = __dmul_rn(3.0, k3);
  double r[2]; int nr = 0;
  flops += 2;
  if (e2 != 0.0) {
    double disc = __fma_rn(e1, e1, -__dmul_rn(__dmul_rn(4.0, e2), e0));
    flops += 4;
    if (disc > 0.0) {
      flops += 6;
      double sq = __dsqrt_rn(disc);
      double q = __dmul_rn(-0.5, __dadd_rn(e1, e1 >= 0.0 ? sq : -sq));
      r[0] = __ddiv_rn(q, e2); r[1] = __ddiv_rn(e0, q); nr = 2;
    }
  } else if (e1 != 0.0) {
    r[0] = __ddiv_rn(-e0, e1); nr = 1;
  }
  double cp[2]; int ncp = 0;
  for (int i = 0; i < nr; ++i) if (r[i] > 0.0 && r[i] < 1.0) cp[ncp++] = r[i];
  if (ncp == 2) {
    if (cp[1] < cp[0]) { double t = cp[0]; cp[0] = cp[1]; cp[1] = t; }
    if (cp[1] == cp[0]) ncp = 1;
  }
  double ends[4]; int ne = 0;
  ends[ne++] = 0.0;
  for (int i = 0; i < ncp; ++i) ends[ne++] = cp[i];
  ends[ne++] = 1.0;
  bool degen = false;
  for (int s = 0; s + 1 < ne; ++s) {
    double l = ends[s], rr = ends[s + 1];
    double fl = horner3(k0, k1, k2, k3, l), fr = horner3(k0, k1, k2, k3, rr), t;
    flops += 12;
    if (fl == 0.0) t = l;
    else if (fr == 0.0) t = rr;
    else if ((fl < 0.0) != (fr < 0.0)) t = bisect64(k0, k1, k2, k3, l, rr, fl, flops);
    else continue;
    flops += 24 + 9 + 25 + 3 + 6 + 2 + 2;  // positions, differences, dots, determinant, numerators, divisions
    d3 Y[4];
    for (int q = 0; q < 4; ++q) Y[q] = d3_at(X0[q], t, D[q]);
    double u1 = 0.0, u2 = 0.0;
    int in = inside64(kind, Y, u1, u2);
    if (in < 0) { degen = true; continue; }
    if (in == 1) { tau = t; w1 = u1; w2 = u2; return 1; }
  }
  return degen ? 2 : 0;
}

__device__ __forceinline__ d3 slot_pos(const PatchSm& S, int t, int sl) {
  return {S.x[3 * t + 0][sl], S.x[3 * t + 1][sl], S.x[3 * t + 2][sl]};
}

// Drain up to n queued pairs, one per lane.
__device__ void process_queue(WarpSm& ws, int n, int lane, int r, const narrow_args& a, long long& nprim,
                              long long& ndeg, long long& flops) {
  int type = -1, ga = 0, gb = 0;
  double tau = 0.0, w1 = 0.0, w2 = 0.0;
  if (lane < n) {
    unsigned e = ws.q[lane];
    int kind = e >> 16, x = (e >> 8) & 0xFF, y = e & 0xFF;
    const PatchSm& SA = (kind == 1) ? ws.B : ws.A;   // side holding the first primitive
    const PatchSm& SB = (kind == 1) ? ws.A : ws.B;
    int sl[4];
    if (kind < 2) {
      sl[0] = SA.v_slot[x];
      int t = SB.t_slots[y];
      sl[1] = t & 63; sl[2] = (t >> 6) & 63; sl[3] = (t >> 12) & 63;
    } else {
      int ea = SA.e_slots[x], eb = SB.e_slots[y];
      sl[0] = ea & 63; sl[1] = (ea >> 6) & 63; sl[2] = eb & 63; sl[3] = (eb >> 6) & 63;
    }
    d3 X0[4], X1[4], D[4];
    // points 0 (and 1 for EE) come from SA, the rest from SB
    for (int q = 0; q < 4; ++q) {
      const PatchSm& S = (q == 0 || (kind == 2 && q == 1)) ? SA : SB;
      X0[q] = slot_pos(S, 0, sl[q]); X1[q] = slot_pos(S, 1, sl[q]);
      D[q] = d3_sub(X1[q], X0[q]);
    }
    // exact FP64 swept-box overlap of the two primitives
    int na = kind == 2 ? 2 : 1;
    bool hit = true;
    {
      double alo[3], ahi[3], blo[3], bhi[3];
      const double* X0c = &X0[0].x; const double* X1c = &X1[0].x;
      for (int c = 0; c < 3; ++c) {
        alo[c] = ahi[c] = X0c[c];
        for (int q = 0; q < 4; ++q) {
          double u = X0c[3 * q + c], v = X1c[3 * q + c];
          if (q < na) {
            alo[c] = fmin(alo[c], fmin(u, v)); ahi[c] = fmax(ahi[c], fmax(u, v));
          } else if (q == na) {
            blo[c] = fmin(u, v); bhi[c] = fmax(u, v);
          } else {
            blo[c] = fmin(blo[c], fmin(u, v)); bhi[c] = fmax(bhi[c], fmax(u, v));
          }
        }
        hit = hit && alo[c] <= bhi[c] && blo[c] <= ahi[c];
      }
    }
    if (hit) {
      ++nprim;
      flops += 12;  // displacements D = X1 - X0
      int st = ccd64(kind == 2 ? KIND_EE : KIND_VF, X0, D, tau, w1, w2, flops);
      if (st == 1) {
        type = kind;
        if (kind == 0) { ga = SA.v_gid[x]; gb = SB.t_gid[y]; }
        else if (kind == 1) { ga = SA.v_gid[x]; gb = SB.t_gid[y]; }
        else { ga = SA.e_gid[x]; gb = SB.e_gid[y]; }
      } else if (st == 2) {
        ++ndeg;
      }
    }
  }
  unsigned m = __ballot_sync(0xffffffffu, type >= 0);
  if (m) {
    unsigned long long base = 0;
    int leader = __ffs(m) - 1;
    if (lane == leader) base = atomicAdd((unsigned long long*)&a.ctr[11], (unsigned long long)__popc(m));
    base = __shfl_sync(0xffffffffu, base, leader);
    if (type >= 0) {
      int64_t k = (int64_t)base + __popc(m & ((1u << lane) - 1u));
      if (k < a.C) {
        a.rc_pair[k] = r; a.rc_type[k] = type; a.rc_a[k] = ga; a.rc_b[k] = gb;
        a.rc_tau[k] = tau; a.rc_w[2 * k] = w1; a.rc_w[2 * k + 1] = w2;
      }
      atomicAdd((unsigned long long*)&a.ctr[type == 2 ? STIV_C_EE : STIV_C_VF], 1ull);
    }
  }
}

// Push this lane's candidate (if any) into the warp queue; drain when >= 32.
__device__ __forceinline__ void enqueue(WarpSm& ws, bool hit, unsigned entry, int lane, int r, const narrow_args& a,
                                        long long& nprim, long long& ndeg, long long& flops) {
  unsigned m = __ballot_sync(0xffffffffu, hit);
  int qn = ws.qn;
  if (hit) ws.q[qn + __popc(m & ((1u << lane) - 1u))] = entry;
  qn += __popc(m);
  __syncwarp();
  if (qn >= 32) {
    process_queue(ws, 32, lane, r, a, nprim, ndeg, flops);
    __syncwarp();
    unsigned rest = (lane + 32 < qn) ? ws.q[lane + 32] : 0;
    __syncwarp();
    if (lane + 32 < qn) ws.q[lane] = rest;
    qn -= 32;
  }
  if (lane == 0) ws.qn = qn;
  __syncwarp();
}

__global__ void __launch_bounds__(NW * 32) narrow_kernel(narrow_args a) {
  extern __shared__ unsigned char smraw[];
  WarpSm& ws = ((WarpSm*)smraw)[threadIdx.x >> 5];
  int lane = threadIdx.x & 31;
  int64_t nwork = a.ctr[STIV_C_PATCH];
  if (nwork > a.W) nwork = a.W;
  long long nprim = 0, ndeg = 0, flops = 0;
  while (true) {
    long long item = 0;
    if (lane == 0) item = (long long)atomicAdd((unsigned long long*)&a.ctr[10], 1ull);
    item = __shfl_sync(0xffffffffu, item, 0);
    if (item >= nwork) break;
    uint64_t w = a.work[item];
    int r = (int)(w >> 32), pa = (int)((w >> 16) & 0xFFFF), pb = (int)(w & 0xFFFF);
    int vi = a.ci[r], vj = a.cj[r], code = a.cs[r];
    int s0[3] = {0, 0, 0};
    int s1[3] = {code / 9 - 1, (code / 3) % 3 - 1, code % 3 - 1};
    load_patch(ws.A, a, vi, pa, s0, lane);
    load_patch(ws.B, a, vj, pb, s1, lane);
    filter_patch(ws.A, ws.B.box, lane);
    filter_patch(ws.B, ws.A.box, lane);
    if (lane == 0) ws.qn = 0;
    __syncwarp();
    // VF: vertices of A vs triangles of B (type 0) and vertices of B vs triangles of A (type 1)
    for (int dir = 0; dir < 2; ++dir) {
      PatchSm& V = dir == 0 ? ws.A : ws.B;
      PatchSm& T = dir == 0 ? ws.B : ws.A;
      for (int y0 = 0; y0 < T.ntf; y0 += 32) {
        int yk = y0 + lane;
        bool valid = yk < T.ntf;
        int y = valid ? T.tf[yk] : 0;
        float tb[6];
        for (int c = 0; c < 6; ++c) tb[c] = valid ? T.tb[c][y] : 0.f;
        for (int xk = 0; xk < V.nvf; ++xk) {
          int x = V.vf[xk], sl = V.v_slot[x];
          float lo[3] = {V.flo[0][sl], V.flo[1][sl], V.flo[2][sl]}, hi[3] = {V.fhi[0][sl], V.fhi[1][sl], V.fhi[2][sl]};
          bool hit = valid && fbox_hit(lo, hi, tb);
          enqueue(ws, hit, ((unsigned)dir << 16) | ((unsigned)x << 8) | (unsigned)y, lane, r, a, nprim, ndeg, flops);
        }
      }
    }
    if (a.include_ee) {
      for (int y0 = 0; y0 < ws.B.nef; y0 += 32) {
        int yk = y0 + lane;
        bool valid = yk < ws.B.nef;
        int y = valid ? ws.B.ef[yk] : 0;
        float eb[6];
        for (int c = 0; c < 6; ++c) eb[c] = valid ? ws.B.eb[c][y] : 0.f;
        for (int xk = 0; xk < ws.A.nef; ++xk) {
          int x = ws.A.ef[xk];
          float lo[3] = {ws.A.eb[0][x], ws.A.eb[1][x], ws.A.eb[2][x]}, hi[3] = {ws.A.eb[3][x], ws.A.eb[4][x], ws.A.eb[5][x]};
          bool hit = valid && fbox_hit(lo, hi, eb);
          enqueue(ws, hit, (2u << 16) | ((unsigned)x << 8) | (unsigned)y, lane, r, a, nprim, ndeg, flops);
        }
      }
    }
    int qn = ws.qn;
    if (qn > 0) process_queue(ws, qn, lane, r, a, nprim, ndeg, flops);
    __syncwarp();
  }
  // totals
  for (int off = 16; off > 0; off >>= 1) {
    nprim += __shfl_down_sync(0xffffffffu, nprim, off);
    ndeg += __shfl_down_sync(0xffffffffu, ndeg, off);
    flops += __shfl_down_sync(0xffffffffu, flops, off);
  }
  if (lane == 0) {
    if (nprim) atomicAdd((unsigned long long*)&a.ctr[STIV_C_PRIM], (unsigned long long)nprim);
    if (ndeg) atomicAdd((unsigned long long*)&a.ctr[STIV_C_DEGEN], (unsigned long long)ndeg);
    if (flops) atomicAdd((unsigned long long*)&a.ctr[12], (unsigned long long)flops);
  }
}

// Level 1: patch pairs of one candidate vesicle pair per warp.  Dynamic shared
// memory: per warp 2 x mp patch boxes and 2 x mp list entries.
__global__ void __launch_bounds__(128) patch_pairs_kernel(const int32_t* pv, const double* vbox, const float* pbox,
                                                          double Lx, double Ly, double Lz, const int32_t* ci,
                                                          const int32_t* cj, const int32_t* cs, int64_t cap,
                                                          int64_t W, uint64_t* work, int64_t* ctr, int mp) {
  extern __shared__ float psm[];
  int wid0 = threadIdx.x >> 5;
  float* sbw = psm + (size_t)wid0 * 2 * mp * 6;                       // [2][mp][6]
  unsigned short* law = (unsigned short*)(psm + (size_t)4 * 2 * mp * 6) + (size_t)wid0 * 2 * mp;
  unsigned short* lbw = law + mp;
  int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
  int64_t npairs = ctr[STIV_C_PAIRS];
  if (npairs > cap) npairs = cap;
  double L[3] = {Lx, Ly, Lz};
  for (int64_t r = (int64_t)blockIdx.x * 4 + wid; r < npairs; r += (int64_t)gridDim.x * 4) {
    int i = ci[r], j = cj[r], code = cs[r];
    int s[3] = {code / 9 - 1, (code / 3) % 3 - 1, code % 3 - 1};
    int Pi = 2 * pv[i], Pj = 2 * pv[j];
    int ni = stiv_npatches(Pi), nj = stiv_npatches(Pj);
    // FP32 boxes: vesicle j shifted (outward), patches of j shifted (outward)
    float shlo[3], shhi[3];
    for (int c = 0; c < 3; ++c) {
      double sh = s[c] * L[c];
      shlo[c] = __double2float_rd(sh); shhi[c] = __double2float_ru(sh);
    }
    float bi[6], bj[6];
    for (int c = 0; c < 3; ++c) {
      bi[c] = __double2float_rd(vbox[6 * i + c]); bi[3 + c] = __double2float_ru(vbox[6 * i + 3 + c]);
      bj[c] = __fadd_rd(__double2float_rd(vbox[6 * j + c]), shlo[c]);
      bj[3 + c] = __fadd_ru(__double2float_ru(vbox[6 * j + 3 + c]), shhi[c]);
    }
    for (int k = lane; k < ni; k += 32)
      for (int c = 0; c < 6; ++c) sbw[(0 * mp + (k)) * 6 + (c)] = pbox[((size_t)i * STIV_MAX_PATCH + k) * 6 + c];
    for (int k = lane; k < nj; k += 32)
      for (int c = 0; c < 3; ++c) {
        sbw[(1 * mp + (k)) * 6 + (c)] = __fadd_rd(pbox[((size_t)j * STIV_MAX_PATCH + k) * 6 + c], shlo[c]);
        sbw[(1 * mp + (k)) * 6 + (3 + c)] = __fadd_ru(pbox[((size_t)j * STIV_MAX_PATCH + k) * 6 + 3 + c], shhi[c]);
      }
    __syncwarp();
    // patches of i overlapping box j, patches of j overlapping box i
    int na = 0, nb = 0;
    for (int k0 = 0; k0 < ni; k0 += 32) {
      int k = k0 + lane;
      bool hit = k < ni && fbox_hit(&sbw[(0 * mp + (k)) * 6], &sbw[(0 * mp + (k)) * 6 + 3], bj);
      unsigned m = __ballot_sync(0xffffffffu, hit);
      if (hit) law[na + __popc(m & ((1u << lane) - 1u))] = (unsigned short)k;
      na += __popc(m);
    }
    for (int k0 = 0; k0 < nj; k0 += 32) {
      int k = k0 + lane;
      bool hit = k < nj && fbox_hit(&sbw[(1 * mp + (k)) * 6], &sbw[(1 * mp + (k)) * 6 + 3], bi);
      unsigned m = __ballot_sync(0xffffffffu, hit);
      if (hit) lbw[nb + __popc(m & ((1u << lane) - 1u))] = (unsigned short)k;
      nb += __popc(m);
    }
    __syncwarp();
    for (int e0 = 0; e0 < na * nb; e0 += 32) {
      int e = e0 + lane;
      bool hit = false;
      int pa = 0, pb = 0;
      if (e < na * nb) {
        pa = law[e / nb]; pb = lbw[e % nb];
        hit = fbox_hit(&sbw[(0 * mp + (pa)) * 6], &sbw[(0 * mp + (pa)) * 6 + 3], &sbw[(1 * mp + (pb)) * 6]);
      }
      unsigned m = __ballot_sync(0xffffffffu, hit);
      if (m) {
        unsigned long long base = 0;
        if (lane == 0) base = atomicAdd((unsigned long long*)&ctr[STIV_C_PATCH], (unsigned long long)__popc(m));
        base = __shfl_sync(0xffffffffu, base, 0);
        if (hit) {
          int64_t k = (int64_t)base + __popc(m & ((1u << lane) - 1u));
          if (k < W) work[k] = ((uint64_t)r << 32) | ((uint64_t)pa << 16) | (uint64_t)pb;
          else atomicOr((unsigned long long*)&ctr[STIV_C_STATUS], STIV_F_WORK_OVERFLOW);
        }
      }
    }
    __syncwarp();
  }
}

}  // namespace

size_t stiv_narrow_smem() { return sizeof(WarpSm) * NW; }

int stiv_narrow_phase(stiv_handle* h, cudaStream_t st, const int32_t* p_dev, const int64_t* voff, const void* X,
                      const stiv_pairs* cand, detect_ws& w, int num_sms, int p_max) {
  const double* L = h->prm.box_L;
  int blocks = (int)((cand->capacity + 3) / 4);
  if (blocks > 4 * num_sms) blocks = 4 * num_sms;
  if (blocks < 1) blocks = 1;
  int mp = stiv_npatches(2 * p_max);
  size_t psmem = (size_t)4 * 2 * mp * 6 * sizeof(float) + (size_t)4 * 2 * mp * sizeof(unsigned short);
  STIV_CUDA(h, cudaFuncSetAttribute(patch_pairs_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)psmem));
  {
  STIV_PROF(h, st, "patch_pairs");
  patch_pairs_kernel<<<blocks, 128, psmem, st>>>(p_dev, w.vbox, w.pbox, L[0], L[1], L[2], cand->i, cand->j,
                                                 cand->shift, cand->capacity, w.W, w.work, w.ctr, mp);
  }
  STIV_LAUNCH(h);
  narrow_args a;
  a.pv = p_dev; a.voff = voff; a.X = X; a.mixed = h->prm.precision == STIV_MIXED;
  a.L[0] = L[0]; a.L[1] = L[1]; a.L[2] = L[2];
  a.ci = cand->i; a.cj = cand->j; a.cs = cand->shift;
  a.work = w.work; a.W = w.W; a.include_ee = h->prm.include_ee;
  a.C = w.C;
  a.rc_pair = w.tmp_i32; a.rc_type = w.tmp_i32 + w.C; a.rc_a = w.tmp_i32 + 2 * w.C; a.rc_b = w.tmp_i32 + 3 * w.C;
  a.rc_tau = w.tmp_f64; a.rc_w = w.tmp_f64 + w.C;
  a.ctr = w.ctr;
  size_t smem = stiv_narrow_smem();
  STIV_CUDA(h, cudaFuncSetAttribute(narrow_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  int per_sm = 0;
  STIV_CUDA(h, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, narrow_kernel, NW * 32, smem));
  if (per_sm < 1) per_sm = 1;
  STIV_PROF(h, st, "narrow");
  narrow_kernel<<<per_sm * num_sms, NW * 32, smem, st>>>(a);
  STIV_LAUNCH(h);
  return STIV_OK;
}

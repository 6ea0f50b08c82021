// Narrow phase of Alg. 2 checkContact: every vertex-triangle pair (both
// directions) and edge-edge pair of a candidate vesicle pair whose swept boxes
// overlap is tested with the coplanarity cubic of Eq. 3.1 (d_m = 0), or with
// the degree-six equation of the d_m band (d_m > 0).
//
// The triangulated grid (Sec. 3.1.2, Fig. 3) is cut into patches of 2 x 4 grid
// quads; each primitive belongs to exactly one patch, so each primitive pair
// is examined by exactly one patch pair.
//   patch_pairs_kernel: per candidate vesicle pair, one warp lists the patch
//     pairs whose FP32 (outward) boxes overlap and some of whose cells (1 x 2
//     quads) meet;
//   narrow_kernel (stages 1-3a): per patch pair, one warp stages both patches
//     in shared memory and filters the primitive pairs; the survivors leave
//     as global pair descriptors;
//   pieces_kernel (stage 3b) and fp64_kernel (stage 4) work on those lists,
//     so that every stage runs on full warps.  The stages:
//     1. FP32 swept-box test (conservative: never drops an overlapping pair);
//     2. the exact FP64 swept-box test (counts the pairs tested), decided
//        from the FP32 boxes and their error bound, on the FP64 values only
//        for the pairs those do not decide;
//     3. certified FP32 rejection: a pair is dropped only when error-bounded
//        FP32 arithmetic proves that the FP64 test below cannot report a
//        contact (Bernstein bound: no root of the cubic in [0,1]; or, on every
//        sub-interval that may hold a root, the point is certainly outside the
//        triangle / the edges certainly miss);
//     4. the FP64 contact test (cubic, root isolation, bisection, inside test)
//        in the fixed arithmetic order, on the survivors only.
// Stage 3 never changes a result: the contact list equals the one obtained by
// running stage 4 on every pair of stage 2 (stiv_params.exact_only = 1).
#include "stiv_internal.cuh"

#include <math.h>

namespace {

constexpr int NS = (STIV_BR + 1) * (STIV_BC + 1) + 2;  // vertex slots per patch (+2 poles)
constexpr int SN = NS - 2, SS = NS - 1;               // pole slots
constexpr int MAXV = 16, MAXT = 32, MAXE = 48;
constexpr int NW = 8;                                  // warps per CTA
constexpr int QCAP = 64;                               // queue entries

// Primitives of one patch in terms of its vertex slots.  P is even, so every
// patch spans exactly STIV_BR bands and STIV_BC columns; the lists depend only
// on whether the patch touches the north pole (first band), the south pole
// (last band) and whether it owns the pole vertices (first column block):
// 8 variants, built once per CTA.
struct PatchTopo {
  unsigned char v_slot[MAXV];      // vertices owned by the patch
  int t_slots[MAXT];               // triangles: 3 slots, 6 bits each
  short e_slots[MAXE];             // edges: 2 slots, 6 bits each (either order)
  int nv, nt, ne;
};
constexpr int NVAR = 8;
static_assert(NS <= 32, "one lane per vertex slot");
static_assert(STIV_BR == 2 && STIV_BC % 2 == 0, "patches tile every even-order grid exactly");

struct PatchSm {
  float m[NS];                     // bound on the FP32 error of the slot's box ends (before any widening)
  float x[3][NS], d[3][NS];        // FP32: X0 - origin of vesicle i, X1 - X0
  float lo[3][NS], hi[3][NS];      // FP32 conservative swept box of each slot (frame of vesicle i)
  int vid[NS];                     // global vertex id of each slot (-1: unused)
  const PatchTopo* tp;
  unsigned char vf[MAXV], tf[MAXT], ef[MAXE];
  float4 vlo[MAXV], vhi[MAXV];     // boxes of the filtered vertices, in vf order
  int nv, nt, ne, nvf, ntf, nef;
  int P, I, J, ves;
  float box[6];
};

struct WarpSm {
  PatchSm A, B;
  float4 elo[MAXE], ehi[MAXE];     // boxes of A's filtered edges, in ef order
  unsigned q1[QCAP];
  float dx;                        // bound on the FP32 position error in this frame
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
  int exact_only;
  double dm;                // minimum separation d_m (> 0: the degree-six contact test)
  int nlevel;               // refinement levels of the piece test (<= NLEVEL)
  const float* vorg;
  const float* fprep;
  int64_t fstride;
  const stiv_pair_info* pinfo;  // per candidate pair: vesicles, orders, offsets, FP32 frame
  // descriptors of primitive pairs: x = pair << 32 | type << 30 | a << 15 | b
  // (primitive ids), y = the 4 vertex ids, 16 bits each, in the order the
  // contact test takes its points (VF: vertex, triangle; EE: p0 < p1, q0 < q1)
  ulonglong2* q3;           // stage 3b input
  ulonglong2* q2;           // stage 4 input
  int64_t Q3, Q2;
  int64_t C;  // raw contact capacity
  int32_t* rc_pair; int32_t* rc_type; int32_t* rc_a; int32_t* rc_b;
  double* rc_tau; double* rc_w;
  int64_t* ctr;
};

__device__ __forceinline__ int slot_of(int rr, int cc) { return rr * (STIV_BC + 1) + cc; }

// Vertex coordinate as stored: double (FP64 form) or float (mixed form).
template <bool MIXED>
__device__ __forceinline__ double vtx(const void* X, size_t i) {
  if (MIXED) return (double)((const float*)X)[i];
  return ((const double*)X)[i];
}

// ---------------------------------------------------------------------------
// staging
// ---------------------------------------------------------------------------
// Topology variant var = first | last << 1 | pole-owner << 2 (see PatchTopo),
// built by one warp.
__device__ void build_topo(PatchTopo& T, int var, int lane) {
  const int rq = STIV_BR, ncol = STIV_BC;
  bool first = var & 1, last = (var >> 1) & 1, j0 = (var >> 2) & 1;
  int rown = rq + (last ? 1 : 0);
  int nvg = rown * ncol;
  int npole = (first && j0 ? 1 : 0) + (last && j0 ? 1 : 0);
  int ntq = 2 * rq * ncol;
  int nfan = (first ? ncol : 0) + (last ? ncol : 0);
  int ne = rown * ncol + 2 * rq * ncol + nfan;
  if (lane == 0) { T.nv = nvg + npole; T.nt = ntq + nfan; T.ne = ne; }
  for (int k = lane; k < nvg + npole; k += 32) {
    int slot;
    if (k < nvg) slot = slot_of(k / ncol, k % ncol);
    else if (first && j0 && k == nvg) slot = SN;
    else slot = SS;
    T.v_slot[k] = (unsigned char)slot;
  }
  for (int k = lane; k < ntq + nfan; k += 32) {
    int s0, s1, s2;
    if (k < ntq) {
      int q = k >> 1, rr = q / ncol, cc = q % ncol;
      if ((k & 1) == 0) { s0 = slot_of(rr, cc); s1 = slot_of(rr + 1, cc); s2 = slot_of(rr + 1, cc + 1); }
      else { s0 = slot_of(rr, cc); s1 = slot_of(rr + 1, cc + 1); s2 = slot_of(rr, cc + 1); }
    } else {
      int k2 = k - ntq;
      if (first && k2 < ncol) { s0 = SN; s1 = slot_of(0, k2); s2 = slot_of(0, k2 + 1); }
      else { int cc = first ? k2 - ncol : k2; s0 = SS; s1 = slot_of(rq, cc + 1); s2 = slot_of(rq, cc); }
    }
    T.t_slots[k] = s0 | (s1 << 6) | (s2 << 12);
  }
  for (int k = lane; k < ne; k += 32) {
    int sa, sb;
    int nh = rown * ncol;
    if (k < nh) {
      int rr = k / ncol, cc = k % ncol;
      sa = slot_of(rr, cc); sb = slot_of(rr, cc + 1);
    } else if (k < nh + 2 * rq * ncol) {
      int k2 = k - nh, q = k2 >> 1, rr = q / ncol, cc = q % ncol;
      sa = slot_of(rr, cc);
      sb = ((k2 & 1) == 0) ? slot_of(rr + 1, cc) : slot_of(rr + 1, cc + 1);
    } else {
      int k2 = k - nh - 2 * rq * ncol;
      if (first && k2 < ncol) { sa = slot_of(0, k2); sb = SN; }
      else { int cc = first ? k2 - ncol : k2; sa = slot_of(rq, cc); sb = SS; }
    }
    T.e_slots[k] = (short)(sa | (sb << 6));
  }
}

// Global vertex id of slot k of the patch starting at grid row r0, column c0.
__device__ __forceinline__ int slot_vid(int k, int r0, int c0, int W, int P, bool first, bool last) {
  if (k < SN) {
    int rr = k / (STIV_BC + 1), cc = k % (STIV_BC + 1), col = c0 + cc;
    if (col >= W) col -= W;
    return (r0 + rr) * W + col;
  }
  if (k == SN) return first ? W * (P + 1) : -1;
  return last ? W * (P + 1) + 1 : -1;
}

// Order-preserving int image of a float (-0 just below +0) and its inverse:
// the warp's integer min / max reductions then give the float min / max.
__device__ __forceinline__ int fkey32(float f) {
  int i = __float_as_int(f);
  return i >= 0 ? i : i ^ 0x7FFFFFFF;
}
__device__ __forceinline__ float fkey_val(int k) { return __int_as_float(k >= 0 ? k : k ^ 0x7FFFFFFF); }

// One vertex slot: FP32 frame coordinates and the slot's conservative FP32
// swept box (also returned in b; vesicle j's widened by d_m, rounded up).  The
// exact box is not staged: the FP32 box ends are within m of the exact ones
// (m stored per slot), which decides almost every exact box test; the rare
// undecided pair reads the FP64 values (stage 2).  off: FP32 offset of the
// vesicle's frame origin in the pair frame.
template <bool MIXED, bool DM>
__device__ __forceinline__ void stage_slot(PatchSm& S, const float* fp, int vid, int k, const float* off, float dx,
                                           float* b, float padf, const float* org) {
  int v = vid >= 0 ? vid : 0;
  S.vid[k] = vid;
  float4 fx = ((const float4*)fp)[2 * v], fd = ((const float4*)fp)[2 * v + 1];
  float xf[3], df[3];
  float f0[3] = {fx.x, fx.y, fx.z}, f1[3] = {fd.x, fd.y, fd.z};
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    if (MIXED) {   // the staging holds the FP32 vertices themselves
      xf[c] = f0[c] - org[c];   // one rounding, as the FP64 form's staging
      df[c] = f1[c] - f0[c];
    } else {
      xf[c] = f0[c];
      df[c] = f1[c];
    }
  }
  float mmax = 0.0f;
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    float x = xf[c] + off[c], d = df[c];
    S.x[c][k] = x;
    S.d[c][k] = d;
    float m = dx + 4.7683716e-7f * (fabsf(x) + fabsf(d));  // 2^-21 (|x| + |d|)
    mmax = fmaxf(mmax, m);
    if (DM) m = __fadd_ru(m, padf);                        // + d_m
    float lo = vid >= 0 ? fminf(x, x + d) - m : INFINITY;
    float hi = vid >= 0 ? fmaxf(x, x + d) + m : -INFINITY;
    S.lo[c][k] = lo;
    S.hi[c][k] = hi;
    b[c] = lo;
    b[3 + c] = hi;
  }
  S.m[k] = mmax;
}

// Bound on the error of a component of the difference of two FP32 frame
// positions of the same vesicle: each is x = fl(xf + off) with xf the
// position relative to the vesicle's origin rounded once (|xf| <= R) and off
// the same float for every point of the vesicle, so off's own error cancels
// and U32 (|xf1| + |xf2| + |x1| + |x2|) remains; R: the larger vesicle
// radius bound of the pair, offm: the largest offset component.  It is at
// most 2 ep (ep = 2^-22 (R_i + R_j + 2 offm)), the bound stage 3a keeps.
__device__ __forceinline__ float same_side_err(float R, float offm) {
  return 1.01f * 5.9604645e-8f * (4.0f * R + 2.0f * offm);
}

// Lane -> slot of the packed staging and culling: lanes 0-14 hold the 15 grid
// slots of patch A, lanes 15-29 those of patch B, lane 30 A's pole slot and
// lane 31 B's (a patch touches at most one pole, except at P = 2, where the
// south-pole slots of a patch that has both take a second pass).  Returns
// the slot (-1: none) and whether it belongs to B.
__device__ __forceinline__ int packed_slot(int lane, bool fA, bool lA, bool fB, bool lB, bool& onB) {
  if (lane < 30) {
    onB = lane >= 15;
    return onB ? lane - 15 : lane;
  }
  onB = lane == 31;
  bool f = onB ? fB : fA, l = onB ? lB : lA;
  return f ? SN : (l ? SS : -1);
}

// Stage the two patches of a patch pair (A: patch pa of vesicle i, unshifted;
// B: patch pb of vesicle j at its periodic image) in one pass over the lanes
// (packed_slot), both patches' loads in flight together; patch boxes by warp
// reduction.
template <bool MIXED, bool DM>
__device__ __noinline__ void stage_pair(WarpSm& ws, const narrow_args& a, const PatchTopo* topo,
                                        const stiv_pair_info& pi, int pa, int pb, int lane) {
  int vi = pi.vi, vj = pi.vj;
  float dx = pi.frame.w;
  int PA = pi.Pij & 0xFFFF, PB = pi.Pij >> 16;
  int nbcA = stiv_ncol_blocks(PA), nbcB = stiv_ncol_blocks(PB);
  int IA = pa / nbcA, JA = pa % nbcA, IB = pb / nbcB, JB = pb % nbcB;
  bool fA = IA == 0, lA = IA == stiv_nband_blocks(PA) - 1, fB = IB == 0, lB = IB == stiv_nband_blocks(PB) - 1;
  // this lane's side: shift, frame offset, widening and origin of its vesicle
  auto stage_one = [&](bool onB, int k, float* b) {
    int P = onB ? PB : PA, I = onB ? IB : IA, J = onB ? JB : JA;
    int v = onB ? vj : vi;
    float off[3] = {onB ? pi.frame.x : 0.f, onB ? pi.frame.y : 0.f, onB ? pi.frame.z : 0.f};
    float org[3] = {0.f, 0.f, 0.f};
    if (MIXED) {
      float4 o = ((const float4*)a.vorg)[v];
      org[0] = o.x; org[1] = o.y; org[2] = o.z;
    }
    bool f = onB ? fB : fA, l = onB ? lB : lA;
    int vid = slot_vid(k, I * STIV_BR, J * STIV_BC, 2 * P, P, f, l);
    stage_slot<MIXED, DM>(onB ? ws.B : ws.A, a.fprep + (size_t)v * a.fstride, vid, k, off, dx, b,
                          onB ? __double2float_ru(a.dm) : 0.0f, org);
  };
  float b[6] = {INFINITY, INFINITY, INFINITY, -INFINITY, -INFINITY, -INFINITY};
  bool onB;
  int k = packed_slot(lane, fA, lA, fB, lB, onB);
  if (k >= 0) stage_one(onB, k, b);
  if ((fA && lA) || (fB && lB)) {
    // P = 2: a patch with both poles; its south-pole slot (lane 0 for A,
    // lane 15 for B, each on its own side)
    bool two = lane == 0 ? (fA && lA) : lane == 15 ? (fB && lB) : false;
    if (two) {
      float b2[6];
      stage_one(lane == 15, SS, b2);
#pragma unroll
      for (int c = 0; c < 3; ++c) { b[c] = fminf(b[c], b2[c]); b[3 + c] = fmaxf(b[3 + c], b2[3 + c]); }
    }
  }
  float bA[6], bB[6];
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    float la = onB ? INFINITY : b[c], ha = onB ? -INFINITY : b[3 + c];
    float lb = onB ? b[c] : INFINITY, hb = onB ? b[3 + c] : -INFINITY;
    bA[c] = fkey_val(__reduce_min_sync(0xffffffffu, fkey32(la)));
    bA[3 + c] = fkey_val(__reduce_max_sync(0xffffffffu, fkey32(ha)));
    bB[c] = fkey_val(__reduce_min_sync(0xffffffffu, fkey32(lb)));
    bB[3 + c] = fkey_val(__reduce_max_sync(0xffffffffu, fkey32(hb)));
  }
  if (lane < 6) { ws.A.box[lane] = bA[lane]; ws.B.box[lane] = bB[lane]; }
  if (lane == 0) {
    const PatchTopo* tA = topo + ((fA ? 1 : 0) | (lA ? 2 : 0) | (JA == 0 ? 4 : 0));
    const PatchTopo* tB = topo + ((fB ? 1 : 0) | (lB ? 2 : 0) | (JB == 0 ? 4 : 0));
    ws.A.tp = tA; ws.A.nv = tA->nv; ws.A.nt = tA->nt; ws.A.ne = tA->ne;
    ws.A.P = PA; ws.A.I = IA; ws.A.J = JA; ws.A.ves = vi;
    ws.B.tp = tB; ws.B.nv = tB->nv; ws.B.nt = tB->nt; ws.B.ne = tB->ne;
    ws.B.P = PB; ws.B.I = IB; ws.B.J = JB; ws.B.ves = vj;
    ws.dx = dx;
  }
  __syncwarp();
}

// Global id of primitive k of a staged patch (vertex id, triangle id, or edge index).
__device__ int prim_gid(const PatchSm& S, int kind, int k) {
  int P = S.P, W = 2 * P;
  const int rq = STIV_BR, ncol = STIV_BC;
  int r0 = S.I * STIV_BR, c0 = S.J * STIV_BC;
  bool first = S.I == 0;
  if (kind == 0) return S.vid[S.tp->v_slot[k]];
  if (kind == 1) {
    int ntq = 2 * rq * ncol;
    if (k < ntq) { int q = k >> 1, rr = q / ncol, cc = q % ncol; return 2 * ((r0 + rr) * W + c0 + cc) + (k & 1); }
    int k2 = k - ntq;
    if (first && k2 < ncol) return 4 * P * P + c0 + k2;
    return 4 * P * P + W + c0 + (first ? k2 - ncol : k2);
  }
  int e = S.tp->e_slots[k];
  int u = S.vid[e & 63], v = S.vid[(e >> 6) & 63];
  return stiv_edge_index(P, min(u, v), max(u, v));
}

__device__ __forceinline__ void slot_box(const PatchSm& S, int sl, float* b) {
  b[0] = S.lo[0][sl]; b[1] = S.lo[1][sl]; b[2] = S.lo[2][sl];
  b[3] = S.hi[0][sl]; b[4] = S.hi[1][sl]; b[5] = S.hi[2][sl];
}
__device__ __forceinline__ void merge_box(const PatchSm& S, int sl, float* b) {
  b[0] = fminf(b[0], S.lo[0][sl]); b[1] = fminf(b[1], S.lo[1][sl]); b[2] = fminf(b[2], S.lo[2][sl]);
  b[3] = fmaxf(b[3], S.hi[0][sl]); b[4] = fmaxf(b[4], S.hi[1][sl]); b[5] = fmaxf(b[5], S.hi[2][sl]);
}
__device__ __forceinline__ void tri_box(const PatchSm& S, int k, float* b) {
  int t = S.tp->t_slots[k];
  slot_box(S, t & 63, b); merge_box(S, (t >> 6) & 63, b); merge_box(S, (t >> 12) & 63, b);
}
__device__ __forceinline__ void edge_box(const PatchSm& S, int k, float* b) {
  int e = S.tp->e_slots[k];
  slot_box(S, e & 63, b); merge_box(S, (e >> 6) & 63, b);
}
__device__ __forceinline__ bool fbox_hit(const float* a, const float* b) {
  return a[0] <= b[3] && b[0] <= a[3] && a[1] <= b[4] && b[1] <= a[4] && a[2] <= b[5] && b[2] <= a[5];
}

// Compact the primitives of both staged patches whose FP32 boxes overlap the
// other patch's box (A's against B's box, B's against A's); the boxes of the
// kept vertices (and of A's kept edges) are stored in the compacted order for
// the stage-1 loops.  A primitive's box (the min and max of its slots' boxes)
// misses a box on an axis exactly when all its slots lie above it there
// (every lo > its hi) or all below (every hi < its lo), so the test reads
// per-slot bit masks instead of merging boxes.  Both patches share each pass
// over the lanes: the slot masks come from the packed slot layout of the
// staging, and the primitive lists of A and B are concatenated.
__device__ void filter_pair(WarpSm& ws, int lane) {
  PatchSm& A = ws.A;
  PatchSm& B = ws.B;
  bool fA = A.I == 0, lA = A.I == stiv_nband_blocks(A.P) - 1;
  bool fB = B.I == 0, lB = B.I == stiv_nband_blocks(B.P) - 1;
  unsigned abA[3], blA[3], abB[3], blB[3];
  {
    bool onB;
    int k = packed_slot(lane, fA, lA, fB, lB, onB);
    bool in = k >= 0;
    const PatchSm& S = onB ? B : A;
    const float* ob = onB ? A.box : B.box;
    int poleA = fA ? SN : SS, poleB = fB ? SN : SS;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      float lo = in ? S.lo[c][k] : 0.0f, hi = in ? S.hi[c][k] : 0.0f;
      unsigned ma = __ballot_sync(0xffffffffu, in && lo > ob[3 + c]);
      unsigned mb = __ballot_sync(0xffffffffu, in && hi < ob[c]);
      abA[c] = (ma & 0x7FFFu) | (((ma >> 30) & 1u) << poleA);
      abB[c] = ((ma >> 15) & 0x7FFFu) | (((ma >> 31) & 1u) << poleB);
      blA[c] = (mb & 0x7FFFu) | (((mb >> 30) & 1u) << poleA);
      blB[c] = ((mb >> 15) & 0x7FFFu) | (((mb >> 31) & 1u) << poleB);
    }
    if ((fA && lA) || (fB && lB)) {   // P = 2: the south-pole slots of two-pole patches
      bool two = lane == 0 ? (fA && lA) : lane == 15 ? (fB && lB) : false;
      const PatchSm& S2 = lane == 15 ? B : A;
      const float* ob2 = lane == 15 ? A.box : B.box;
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        float lo = two ? S2.lo[c][SS] : 0.0f, hi = two ? S2.hi[c][SS] : 0.0f;
        unsigned ma = __ballot_sync(0xffffffffu, two && lo > ob2[3 + c]);
        unsigned mb = __ballot_sync(0xffffffffu, two && hi < ob2[c]);
        abA[c] |= (ma & 1u) << SS; abB[c] |= ((ma >> 15) & 1u) << SS;
        blA[c] |= (mb & 1u) << SS; blB[c] |= ((mb >> 15) & 1u) << SS;
      }
    }
  }
  const unsigned lower = (1u << lane) - 1u;
#pragma unroll 1
  for (int kind = 0; kind < 3; ++kind) {
    int nA = kind == 0 ? A.nv : kind == 1 ? A.nt : A.ne;
    int nB = kind == 0 ? B.nv : kind == 1 ? B.nt : B.ne;
    int n = nA + nB, baseA = 0, baseB = 0;
    for (int k0 = 0; k0 < n; k0 += 32) {
      int kk = k0 + lane;
      bool valid = kk < n, isB = kk >= nA;
      int k = isB ? kk - nA : kk;
      PatchSm& S = isB ? B : A;
      bool hit = false;
      unsigned sm = 0;
      if (valid) {
        if (kind == 0) {
          sm = 1u << S.tp->v_slot[k];
        } else if (kind == 1) {
          int t = S.tp->t_slots[k];
          sm = (1u << (t & 63)) | (1u << ((t >> 6) & 63)) | (1u << ((t >> 12) & 63));
        } else {
          int e = S.tp->e_slots[k];
          sm = (1u << (e & 63)) | (1u << ((e >> 6) & 63));
        }
        unsigned a0 = isB ? abB[0] : abA[0], a1 = isB ? abB[1] : abA[1], a2 = isB ? abB[2] : abA[2];
        unsigned b0 = isB ? blB[0] : blA[0], b1 = isB ? blB[1] : blA[1], b2 = isB ? blB[2] : blA[2];
        hit = (a0 & sm) != sm && (b0 & sm) != sm && (a1 & sm) != sm && (b1 & sm) != sm && (a2 & sm) != sm &&
              (b2 & sm) != sm;
      }
      unsigned m = __ballot_sync(0xffffffffu, hit);
      unsigned mB = __ballot_sync(0xffffffffu, valid && isB);
      if (hit) {
        int pos = isB ? baseB + __popc(m & mB & lower) : baseA + __popc(m & ~mB & lower);
        unsigned char* out = kind == 0 ? S.vf : kind == 1 ? S.tf : S.ef;
        out[pos] = (unsigned char)k;
        if (kind == 0) {
          float b[6];
          slot_box(S, S.tp->v_slot[k], b);
          S.vlo[pos] = make_float4(b[0], b[1], b[2], 0.f);
          S.vhi[pos] = make_float4(b[3], b[4], b[5], 0.f);
        }
        if (kind == 2 && !isB) {
          float b[6];
          edge_box(A, k, b);
          ws.elo[pos] = make_float4(b[0], b[1], b[2], 0.f);
          ws.ehi[pos] = make_float4(b[3], b[4], b[5], 0.f);
        }
      }
      baseA += __popc(m & ~mB);
      baseB += __popc(m & mB);
    }
    if (lane == 0) {
      if (kind == 0) { A.nvf = baseA; B.nvf = baseB; }
      else if (kind == 1) { A.ntf = baseA; B.ntf = baseB; }
      else { A.nef = baseA; B.nef = baseB; }
    }
  }
  __syncwarp();
}

// ---------------------------------------------------------------------------
// certified FP32 rejection
// ---------------------------------------------------------------------------
struct f3 { float x, y, z; };
__device__ __forceinline__ f3 fsub(f3 a, f3 b) { return {a.x - b.x, a.y - b.y, a.z - b.z}; }
__device__ __forceinline__ f3 fadd(f3 a, f3 b) { return {a.x + b.x, a.y + b.y, a.z + b.z}; }
__device__ __forceinline__ f3 fcross(f3 u, f3 v) {
  return {fmaf(u.y, v.z, -(u.z * v.y)), fmaf(u.z, v.x, -(u.x * v.z)), fmaf(u.x, v.y, -(u.y * v.x))};
}
__device__ __forceinline__ float fdot(f3 u, f3 v) { return fmaf(u.z, v.z, fmaf(u.y, v.y, u.x * v.x)); }
// Upper bound of the Euclidean norm: s * rsqrtf(s) with rsqrtf's maximum
// error of 2 ulp (2^-22 relative) widened by 2^-20; the rounding of s itself
// is covered by the margins of the callers.
__device__ __forceinline__ float fnorm(f3 u) {
  float s = fdot(u, u);
  return s > 1e-30f ? s * rsqrtf(s) * 1.000001f : 1e-15f;
}
__device__ __forceinline__ f3 fat(f3 x, float t, f3 d) { return {fmaf(t, d.x, x.x), fmaf(t, d.y, x.y), fmaf(t, d.z, x.z)}; }
__device__ __forceinline__ float amax3(f3 u) { return fmaxf(fabsf(u.x), fmaxf(fabsf(u.y), fabsf(u.z))); }

constexpr float U32 = 5.9604645e-8f;   // 2^-24, unit roundoff of float

// Sign of (g1 x g2) . (g3 x g4) over t in [tm - h, tm + h], each g linear in t
// (value gv at tm, rate gd).  eg bounds the error of each component of each
// gv.  |(g1 x g2) . (g3 x g4)| <= |g1||g2||g3||g4|, so the change over the
// interval is at most sum_i h|gd_i| prod_{j != i} max|g_j|.  Returns +1
// (certainly > 0), -1 (certainly < 0) or 0.
// The same test with the bound's ingredients given: M_i >= max |g_i| over the
// interval (plus the input error 2 eg), R_i = h |gd_i| (half width times the
// rate); the norms of the vectors an inside test shares between its forms
// are taken once.
__device__ __forceinline__ int form_sign_m(f3 g0, f3 g1, f3 g2, f3 g3, const float* M, const float* R, const float* G) {
  float val = fdot(fcross(g0, g1), fcross(g2, g3));
  float p01 = M[0] * M[1], p23 = M[2] * M[3];
  float prod = p01 * p23;
  float var = (R[0] + G[0]) * M[1] * p23 + M[0] * (R[1] + G[1]) * p23 + p01 * (R[2] + G[2]) * M[3] + p01 * M[2] * (R[3] + G[3]);
  float rad = (var + 64.0f * U32 * prod) * 1.001f;
  if (val > rad) return 1;
  if (val < -rad) return -1;
  return 0;
}

// For every contact time in [t0, t0 + w], is the point certainly outside the
// triangle / are the edges certainly apart (1), certainly inside (2), or
// undecided (0)?  Points: VF xp, x0, x1, x2; EE p0, p1, q0, q1.
// ep, ed: error bounds of the FP32 positions / displacements per component.
// Each barycentric (VF) or closest-point (EE) numerator is a form
// (g1 x g2) . (g3 x g4) of linear g: |(g1 x g2) . (g3 x g4)| <= prod |g_i|,
// so its change over the interval is at most sum_i h |gd_i| prod_{j != i}
// max |g_j|; form_sign_m certifies its sign.
__device__ int inside_cert(int kind, const f3* x, const f3* d, float t0, float w, float ep, float ed, float es) {
  float h = 0.5f * w + 1e-6f;           // half width, widened past the FP64 root's last ulp
  float tm = t0 + 0.5f * w;
  f3 P[4];
  for (int q = 0; q < 4; ++q) P[q] = fat(x[q], tm, d[q]);
  float pm = fmaxf(fmaxf(amax3(P[0]), amax3(P[1])), fmaxf(amax3(P[2]), amax3(P[3])));
  float eg = 2.0f * (ep + ed) + 4.0f * U32 * pm;  // per component, differences of positions at tm
  float egs = es + 2.0f * ed + 4.0f * U32 * pm;     // the same for two points of one vesicle
  // vector (position difference at tm, rate) -> M, R, G (2 x its error) of form_sign_m
  auto mr = [&](f3 gv, f3 gd, float e, float& M, float& R, float& G) {
    R = h * fnorm(gd);
    G = 2.0f * e;
    M = fnorm(gv) + R + G;
  };
  if (kind == 0) {
    // barycentric weight of T_k ~ ((T_{k+2} - T_{k+1}) x (p - T_{k+1})) . n,  n = (T1 - T0) x (T2 - T0)
    f3 t01 = fsub(P[2], P[1]), t02 = fsub(P[3], P[1]), t12 = fsub(P[3], P[2]);
    f3 q0 = fsub(P[0], P[1]), q1 = fsub(P[0], P[2]), q2 = fsub(P[0], P[3]);
    float Mt01, Rt01, Mt02, Rt02, Mt12, Rt12, Mq0, Rq0, Mq1, Rq1, Mq2, Rq2, Gs, Gc;
    mr(t01, fsub(d[2], d[1]), egs, Mt01, Rt01, Gs);
    mr(t02, fsub(d[3], d[1]), egs, Mt02, Rt02, Gs);
    mr(t12, fsub(d[3], d[2]), egs, Mt12, Rt12, Gs);
    mr(q0, fsub(d[0], d[1]), eg, Mq0, Rq0, Gc);
    mr(q1, fsub(d[0], d[2]), eg, Mq1, Rq1, Gc);
    mr(q2, fsub(d[0], d[3]), eg, Mq2, Rq2, Gc);
    float G[4] = {Gs, Gc, Gs, Gs};
    f3 nt02 = {-t02.x, -t02.y, -t02.z};
    // k = 0: (T2 - T1) x (p - T1); k = 1: (T0 - T2) x (p - T2); k = 2: (T1 - T0) x (p - T0)
    float M0[4] = {Mt12, Mq1, Mt01, Mt02}, R0[4] = {Rt12, Rq1, Rt01, Rt02};
    int sg0 = form_sign_m(t12, q1, t01, t02, M0, R0, G);
    if (sg0 < 0) return 1;
    float M1[4] = {Mt02, Mq2, Mt01, Mt02}, R1[4] = {Rt02, Rq2, Rt01, Rt02};
    int sg1 = form_sign_m(nt02, q2, t01, t02, M1, R1, G);
    if (sg1 < 0) return 1;
    float M2[4] = {Mt01, Mq0, Mt01, Mt02}, R2[4] = {Rt01, Rq0, Rt01, Rt02};
    int sg2 = form_sign_m(t01, q0, t01, t02, M2, R2, G);
    if (sg2 < 0) return 1;
    return (sg0 > 0 && sg1 > 0 && sg2 > 0) ? 2 : 0;
  }
  // EE with m = (p1 - p0) x (q1 - q0):  s ~ ((q0 - p0) x (q1 - q0)) . m,
  // s - 1 ~ ((q0 - p1) x (q1 - q0)) . m,  u ~ ((q0 - p0) x (p1 - p0)) . m,
  // u - 1 ~ ((q1 - p0) x (p1 - p0)) . m   (each divided by |m|^2)
  f3 e1v = fsub(P[1], P[0]), e2v = fsub(P[3], P[2]);
  f3 a0 = fsub(P[2], P[0]), a1 = fsub(P[2], P[1]), a3 = fsub(P[3], P[0]);
  float Me1, Re1, Me2, Re2, Ma0, Ra0, Ma1, Ra1, Ma3, Ra3, Gs, Gc;
  mr(e1v, fsub(d[1], d[0]), egs, Me1, Re1, Gs);
  mr(e2v, fsub(d[3], d[2]), egs, Me2, Re2, Gs);
  mr(a0, fsub(d[2], d[0]), eg, Ma0, Ra0, Gc);
  mr(a1, fsub(d[2], d[1]), eg, Ma1, Ra1, Gc);
  mr(a3, fsub(d[3], d[0]), eg, Ma3, Ra3, Gc);
  float G[4] = {Gc, Gs, Gs, Gs};
  float Ms[4] = {Ma0, Me2, Me1, Me2}, Rs[4] = {Ra0, Re2, Re1, Re2};
  int s0 = form_sign_m(a0, e2v, e1v, e2v, Ms, Rs, G);
  if (s0 < 0) return 1;
  float Ms1[4] = {Ma1, Me2, Me1, Me2}, Rs1[4] = {Ra1, Re2, Re1, Re2};
  int s1 = form_sign_m(a1, e2v, e1v, e2v, Ms1, Rs1, G);
  if (s1 > 0) return 1;
  float Mu[4] = {Ma0, Me1, Me1, Me2}, Ru[4] = {Ra0, Re1, Re1, Re2};
  int u0 = form_sign_m(a0, e1v, e1v, e2v, Mu, Ru, G);
  if (u0 < 0) return 1;
  float Mu1[4] = {Ma3, Me1, Me1, Me2}, Ru1[4] = {Ra3, Re1, Re1, Re2};
  int u1 = form_sign_m(a3, e1v, e1v, e2v, Mu1, Ru1, G);
  if (u1 > 0) return 1;
  return (s0 > 0 && s1 < 0 && u0 > 0 && u1 < 0) ? 2 : 0;
}

// Coefficients of the coplanarity cubic in FP32 and a bound E on the error of
// any value of the cubic (or of its Bernstein coefficients on any sub-interval
// of [0, 1]) against the exact cubic of the FP64 inputs.  Every coefficient is
// a sum of triple products u . (v x w) of difference vectors (six terms each);
// ep / ed bound the input errors of the positions / displacements per
// component.  Each triple product's error is bounded with the magnitudes of
// its own three vectors, so a pair whose displacement differences are small
// (a primitive moving nearly rigidly) keeps a tight bound:  with eu, ev, ew
// the component errors of u, v, w and Au, Av, Aw their largest computed
// components, each of the six terms obeys |xyz - x'y'z'| <= |x - x'||y'||z'|
// + |x||y - y'||z'| + |x||y||z - z'| with |y'| <= Ay + ey, so the product's
// error is at most 6 ((Au + eu)(Av + ev)(Aw + ew) - Au Av Aw + rr Au Av Aw)
// (rr: the relative rounding of the FP32 evaluation per term).
// With d_m > 0 the band test also takes mn = |n0| + |n1| + |n2| (the FP32
// normals' magnitudes) and the largest position / displacement difference
// components A2, Ad2 of the primitive's own pair of vectors (a, b / da, db).
struct cubic32 { float k0, k1, k2, k3, E, ed, mn, A2, Ad2; };

// es: the error bound of the same-vesicle differences a and b (at most 2 ep).
template <bool WM = false>
__device__ __forceinline__ cubic32 cubic_fp32(int kind, const f3* x, const f3* d, float ep, float es) {
  f3 a, b, c, da, db, dc;
  if (kind == 0) {
    a = fsub(x[2], x[1]); b = fsub(x[3], x[1]); c = fsub(x[0], x[1]);
    da = fsub(d[2], d[1]); db = fsub(d[3], d[1]); dc = fsub(d[0], d[1]);
  } else {
    a = fsub(x[1], x[0]); b = fsub(x[3], x[2]); c = fsub(x[2], x[0]);
    da = fsub(d[1], d[0]); db = fsub(d[3], d[2]); dc = fsub(d[2], d[0]);
  }
  f3 n0 = fcross(a, b);
  f3 n1 = fadd(fcross(da, b), fcross(a, db));
  f3 n2 = fcross(da, db);
  cubic32 r;
  r.k0 = fdot(c, n0);
  r.k1 = fdot(dc, n0) + fdot(c, n1);
  r.k2 = fdot(c, n2) + fdot(dc, n1);
  r.k3 = fdot(dc, n2);
  float Aa = amax3(a), Ab = amax3(b), Ac = amax3(c), Ada = amax3(da), Adb = amax3(db), Adc = amax3(dc);
  float A = fmaxf(Aa, fmaxf(Ab, Ac)), Ad = fmaxf(Ada, fmaxf(Adb, Adc));
  float Dm = 0.f;
  for (int q = 0; q < 4; ++q) Dm = fmaxf(Dm, amax3(d[q]));
  float ed = 2.0f * U32 * Dm + 1e-12f;           // |d - D| per component (float rounding of X1 - X0)
  // per component of each difference: both inputs' errors and the rounding of the difference
  // a and b join points of one vesicle, whose common frame offset cancels in
  // the difference (es); c joins the two vesicles (2 ep)
  float ea = es + 2.0f * U32 * Aa, eb = es + 2.0f * U32 * Ab, ec = 2.0f * ep + 2.0f * U32 * Ac;
  float eda = 2.0f * ed + 2.0f * U32 * Ada, edb = 2.0f * ed + 2.0f * U32 * Adb, edc = 2.0f * ed + 2.0f * U32 * Adc;
  float rr = 8.0f * U32;                         // rounding per term
  // The coefficients are sums of the eight triple products u . (v x w) with
  // u in {c, dc}, v in {a, da}, w in {b, db} (k0: c.(a x b); k1: dc.(a x b),
  // c.(da x b), c.(a x db); k2: c.(da x db), dc.(da x b), dc.(a x db); k3:
  // dc.(da x db)).  The sum of their bounds (above) factors over the three
  // choices: with U = Ac + Adc, V = Aa + Ada, W = Ab + Adb and eU, eV, eW the
  // sums of the matching errors, it is 6 ((U + eU)(V + eV)(W + eW) - U V W
  // + rr U V W), evaluated below without cancellation.
  float U = Ac + Adc, V = Aa + Ada, W = Ab + Adb;
  float eU = ec + edc, eV = ea + eda, eW = eb + edb;
  float Esum = 6.f * (eU * (V + eV) * (W + eW) + U * eV * (W + eW) + U * V * eW + rr * U * V * W);
  float S = fabsf(r.k0) + fabsf(r.k1) + fabsf(r.k2) + fabsf(r.k3);
  float M = (A + Ad) * (A + Ad) * (A + Ad);
  r.E = 1.25f * Esum + 64.f * U32 * S + 1e-12f * 48.f * M;
  r.ed = ed;
  if (WM) {
    r.mn = fnorm(n0) + fnorm(n1) + fnorm(n2);
    r.A2 = fmaxf(Aa, Ab);
    r.Ad2 = fmaxf(Ada, Adb);
  }
  return r;
}

__device__ __forceinline__ bool certain_sign4(float c0, float c1, float c2, float c3, float E) {
  return (c0 > E && c1 > E && c2 > E && c3 > E) || (c0 < -E && c1 < -E && c2 < -E && c3 < -E);
}

// Stage 3a: 1 if the cubic certainly has no root in [0, 1] (Bernstein
// coefficients of one sign), 0 otherwise (also when it may vanish
// identically, which the FP64 test reports as degenerate).
__device__ int bernstein_reject(const cubic32& q) {
  if (fabsf(q.k0) <= q.E && fabsf(q.k1) <= q.E && fabsf(q.k2) <= q.E && fabsf(q.k3) <= q.E) return 0;
  float b1 = q.k0 + q.k1 * (1.f / 3.f), b2 = q.k0 + (2.f * q.k1 + q.k2) * (1.f / 3.f), b3 = q.k0 + q.k1 + q.k2 + q.k3;
  return certain_sign4(q.k0, b1, b2, b3, q.E) ? 1 : 0;
}

// Stage 3a with d_m > 0: 1 if the point certainly stays farther than d_m from
// the triangle's plane (the lines farther than d_m apart) over the whole step,
// so that g = f^2 - d_m^2 |m|^2 stays positive and the FP64 degree-six test
// finds no candidate time.  min |f| over [0, 1] is bounded below by the
// smallest Bernstein coefficient of the cubic (all of one sign beyond the
// error bound E); |m(t)| <= |n0| + |n1| + |n2| is bounded above from the FP32
// cross products with their error bounds (the error model of cubic_fp32); a
// margin of 1e-12 of the squared magnitudes covers the FP64 evaluation of g.
// Right-hand side of the band test: (d_m max|m|)^2 with its margins.
__device__ float band_rhs(const cubic32& q, float ep, float dm) {
  float A = q.A2, Ad = q.Ad2, ed = q.ed;
  float epd = 2.0f * ep + 2.0f * U32 * A, edd = 2.0f * ed + 2.0f * U32 * Ad;
  float en = 2.0f * ((4.f * epd * A + 4.f * U32 * A * A) + (4.f * edd * A + 4.f * epd * Ad + 8.f * U32 * A * Ad) +
                     (4.f * edd * Ad + 4.f * U32 * Ad * Ad));
  float mmax = q.mn * (1.f + 8.f * U32) + en;
  float S = fabsf(q.k0) + fabsf(q.k1) + fabsf(q.k2) + fabsf(q.k3) + 4.f * q.E;
  float dmm = dm * (1.f + 4.f * U32) * mmax;
  return dmm * dmm * (1.f + 1e-5f) + 1e-12f * (S * S + dmm * dmm);
}

// 1 if the Bernstein coefficients c0..c3 (error E) of the cubic on an
// interval prove |f| > d_m max|m| there (rhs: band_rhs).
__device__ __forceinline__ bool out_of_band(float c0, float c1, float c2, float c3, float E, float rhs) {
  if (!certain_sign4(c0, c1, c2, c3, E)) return false;
  float fmin = fminf(fminf(fabsf(c0), fabsf(c1)), fminf(fabsf(c2), fabsf(c3))) - E;
  return fmin > 0.f && fmin * fmin * (1.f - 1e-5f) > rhs;
}

__device__ int band_reject(int kind, const f3* x, const f3* d, float ep, float es, float dm) {
  cubic32 q = cubic_fp32<true>(kind, x, d, ep, es);
  float b1 = q.k0 + q.k1 * (1.f / 3.f), b2 = q.k0 + (2.f * q.k1 + q.k2) * (1.f / 3.f), b3 = q.k0 + q.k1 + q.k2 + q.k3;
  if (!certain_sign4(q.k0, b1, b2, b3, q.E)) return 0;
  return out_of_band(q.k0, b1, b2, b3, q.E, band_rhs(q, ep, dm)) ? 1 : 0;
}

// ---------------------------------------------------------------------------
// Eq. 3.1 (d_m = 0): earliest contact time of one primitive pair in FP64.
// Comparisons are done on the bit patterns (integer pipe); the arithmetic is
// the fixed FP64 sequence of the method definition.
// ---------------------------------------------------------------------------
enum { KIND_VF = 0, KIND_EE = 1 };

__device__ __forceinline__ bool is_zero(double v) { return (__double_as_longlong(v) << 1) == 0; }
__device__ __forceinline__ bool is_neg(double v) {  // v < 0.0
  long long b = __double_as_longlong(v);
  return b < 0 && (b << 1) != 0;
}
__device__ __forceinline__ bool is_pos(double v) { return __double_as_longlong(v) > 0; }  // v > 0.0, v not NaN

// (lo + hi) * 0.5 rounded as FP64 does it (nearest, ties to even), for
// 0 <= lo < hi, computed on the integer pipe: add the 53-bit significands
// with guard, round and sticky bits, round, halve the exponent.  ok = false
// when the operands or the result leave the normal range; the caller then
// uses the FP64 instructions.
__device__ __forceinline__ double mid_rn(double lo, double hi, bool& ok) {
  const unsigned long long FR = (1ull << 52) - 1, HID = 1ull << 52;
  unsigned long long a = (unsigned long long)__double_as_longlong(lo), b = (unsigned long long)__double_as_longlong(hi);
  int eb = (int)(b >> 52);
  ok = true;
  if (a == 0) {                                 // lo = 0: the sum is hi
    if (eb < 2) { ok = false; return 0.0; }
    return __longlong_as_double((long long)(b - HID));
  }
  int ea = (int)(a >> 52);
  if (ea == 0) { ok = false; return 0.0; }
  unsigned long long ma = (a & FR) | HID, mb = (b & FR) | HID;
  int d = eb - ea;                              // >= 0 because lo < hi
  unsigned long long M = mb << 3;
  if (d < 56) {
    unsigned long long sa = ma << 3, sh = sa >> d;
    M += sh | (unsigned long long)((sh << d) != sa);
  } else {
    M += 1;                                     // lo only sets the sticky bit
  }
  int e = eb;
  if (M >> 56) { M = (M >> 1) | (M & 1); ++e; }
  unsigned low = (unsigned)(M & 7);
  M >>= 3;
  if (low > 4 || (low == 4 && (M & 1))) ++M;
  if (M >> 53) { M >>= 1; ++e; }
  if (e < 2 || e > 2046) { ok = false; return 0.0; }
  return __longlong_as_double((long long)(((unsigned long long)(e - 1) << 52) | (M & FR)));
}

// FP32 image of t in [0, 1] by truncating the significand: |t - m| <= 2^-23 t
// (m = 0 below 2^-126, where |t - m| <= 2^-126).
__device__ __forceinline__ float trunc_f32(double t) {
  unsigned long long b = (unsigned long long)__double_as_longlong(t);
  int e = (int)(b >> 52) - 1023 + 127;
  if (e < 1) return 0.0f;
  return __uint_as_float(((unsigned)e << 23) | (unsigned)((b >> 29) & 0x7FFFFF));
}

// Double-float (unevaluated sum of two floats) arithmetic for the second
// sign tier of the bisection.  two_prod is exact with an FMA; two_sum is
// exact (the library is built without FMA contraction).
struct dflt { float h, l; };
__device__ __forceinline__ dflt two_sum(float a, float b) {
  float s = a + b, bb = s - a;
  return {s, (a - (s - bb)) + (b - bb)};
}
__device__ __forceinline__ dflt fast_two_sum(float a, float b) {  // |a| >= |b|
  float s = a + b;
  return {s, b - (s - a)};
}
__device__ __forceinline__ dflt df_mul(dflt x, dflt y) {
  float p = x.h * y.h, e = fmaf(x.h, y.h, -p);
  e = e + (x.h * y.l + x.l * y.h);
  return fast_two_sum(p, e);
}
__device__ __forceinline__ dflt df_add(dflt x, dflt y) {
  dflt s = two_sum(x.h, y.h);
  return fast_two_sum(s.h, s.l + (x.l + y.l));
}
// m in [2^-74, 1] as a double-float from its bits: the high part keeps 24
// significant bits, the low part the remaining 29 rounded to 24 (|m - h - l|
// <= 2^-47 m); returns false below that range.
__device__ __forceinline__ bool df_of_unit(double m, dflt& r) {
  unsigned long long b = (unsigned long long)__double_as_longlong(m);
  int E = (int)(b >> 52);
  if (E < 949) return false;
  r.h = __uint_as_float(((unsigned)(E - 1023 + 127) << 23) | (unsigned)((b >> 29) & 0x7FFFFF));
  unsigned rem = (unsigned)(b & ((1ull << 29) - 1));
  r.l = __uint2float_rn(rem) * __uint_as_float((unsigned)(E - 1075 + 127) << 23);
  return true;
}

// FP64 operations of the procedure, counted as executed (+ - * / sqrt = 1,
// fma = 2, negations and comparisons 0): the algorithmic work of the exact
// contact test, reported for the roofline.
//
// The bisection takes exactly the FP64 path: every midpoint is the FP64
// midpoint (mid_rn), and every sign is the sign of the FP64 Horner value.
// That sign is read from an FP32 Horner evaluation when its error bound
// proves it:  |f64(mid) - f32| <= gamma_6(2^-53) S + 2^-24 S + gamma_6(2^-24) S
// (1 + 2^-24) + 2^-23 S1 <= 4.2e-7 S + 1.2e-7 S1, with S = sum |k_i| and S1 =
// |k1| + 2|k2| + 3|k3| (t in [0, 1]; Horner error bounds, coefficient
// rounding, and the truncation of the midpoint times max |f'|).  When
// |f32| > E the FP64 value has the same sign and is not zero; otherwise the
// FP64 Horner value is computed.  Coefficients outside [1e-25, 1e25] keep
// every FP32 term far from underflow and overflow, else only FP64 is used.
// Between the two, a double-float Horner evaluation decides the sign when
// |f_df| > 2^-40 (S + S1): its own error (3 multiply-add steps at <= 2^-44
// relative each), the coefficients' and the midpoint's representation
// (2^-48 |k_i|, 2^-47 m times max |f'|) and the FP64 Horner error (< 2^-50 S)
// together stay below that bound.
__device__ double bisect64(double k0, double k1, double k2, double k3, double lo, double hi, double flo,
                           long long& flops) {
  bool neg_lo = is_neg(flo);
  float f0 = __double2float_rn(k0), f1 = __double2float_rn(k1), f2 = __double2float_rn(k2),
        f3 = __double2float_rn(k3);
  float a0 = fabsf(f0), a1 = fabsf(f1), a2 = fabsf(f2), a3 = fabsf(f3);
  float mk = fmaxf(fmaxf(a0, a1), fmaxf(a2, a3));
  float E = 1.01f * (4.5e-7f * (((a0 + a1) + a2) + a3) + 1.25e-7f * ((a1 + 2.0f * a2) + 3.0f * a3));
  float Edf = 1.01f * 9.094947e-13f * ((((a0 + a1) + a2) + a3) + ((a1 + 2.0f * a2) + 3.0f * a3));  // 2^-40
  bool use_df = mk > 1e-20f && mk < 1e25f;
  if (!(mk > 1e-25f && mk < 1e25f)) E = INFINITY;
  dflt c0 = {f0, __double2float_rn(__dsub_rn(k0, (double)f0))}, c1 = {f1, __double2float_rn(__dsub_rn(k1, (double)f1))},
       c2 = {f2, __double2float_rn(__dsub_rn(k2, (double)f2))}, c3 = {f3, __double2float_rn(__dsub_rn(k3, (double)f3))};
#pragma unroll 1
  for (int it = 0; it < 64; ++it) {
    bool ok;
    double mid = mid_rn(lo, hi, ok);
    if (!ok) mid = __dmul_rn(__dadd_rn(lo, hi), 0.5);
    flops += 2;
    // lo, mid, hi are non-negative: compare bit patterns
    long long bm = __double_as_longlong(mid);
    if (!(bm > __double_as_longlong(lo) && bm < __double_as_longlong(hi))) break;
    flops += 6;
    float m = trunc_f32(mid);
    float fs = fmaf(fmaf(fmaf(f3, m, f2), m, f1), m, f0);
    bool neg;
    dflt md;
    if (fabsf(fs) > E) {
      neg = fs < 0.0f;
    } else if (use_df && df_of_unit(mid, md) &&
               [&] {
                 dflt v = df_add(df_mul(df_add(df_mul(df_add(df_mul(c3, md), c2), md), c1), md), c0);
                 float vv = v.h + v.l;
                 neg = vv < 0.0f;
                 return fabsf(vv) > Edf;
               }()) {
      // sign certified by the double-float tier
    } else {
      double fm = horner3(k0, k1, k2, k3, mid);
      if (is_zero(fm)) return mid;
      neg = is_neg(fm);
    }
    if (neg == neg_lo) lo = mid;
    else hi = mid;
  }
  return lo;
}

// n / den < 0 for den > 0, decided from the sign of n when the quotient
// cannot underflow to -0: |n| >= 2^-899 and den < 2^171 give |n / den| >
// 2^-1070.
__device__ __forceinline__ bool quot_neg(double n, double den) {
  long long b = __double_as_longlong(n);
  return b < 0 && ((b >> 52) & 0x7FF) >= 124 && (__double_as_longlong(den) >> 52) <= 1193;
}
// n / den rounds above 1 for positive n, den: n exceeds den by more than 8
// units in the last place (then n / den > 1 + 2^-50).
__device__ __forceinline__ bool quot_above1(double n, double den) {
  long long bn = __double_as_longlong(n), bd = __double_as_longlong(den);
  return bn > 0 && bn > bd + 8;
}

// Inside test at the positions Y (VF: xp, x0, x1, x2; EE: p0, p1, q0, q1).
// 1 inside, 0 outside, -1 degenerate.  A quotient whose sign (or excess
// over 1) is decided by its numerator is not formed when that already
// decides "outside": the decision equals that of the rounded quotient.
__device__ int inside64(int kind, const d3* Y, double& w1, double& w2) {
  if (kind == KIND_VF) {
    d3 a = d3_sub(Y[2], Y[1]), b = d3_sub(Y[3], Y[1]), c = d3_sub(Y[0], Y[1]);
    double d00 = d3_dot(a, a), d01 = d3_dot(a, b), d11 = d3_dot(b, b), d20 = d3_dot(c, a), d21 = d3_dot(c, b);
    double den = __fma_rn(d00, d11, -__dmul_rn(d01, d01));
    if (!is_pos(den)) return -1;
    double n1 = __fma_rn(d11, d20, -__dmul_rn(d01, d21));
    double n2 = __fma_rn(d00, d21, -__dmul_rn(d01, d20));
    if (quot_neg(n1, den) || quot_neg(n2, den)) return 0;
    double b1 = __ddiv_rn(n1, den);
    double b2 = __ddiv_rn(n2, den);
    double b0 = __dsub_rn(__dsub_rn(1.0, b1), b2);
    w1 = b1; w2 = b2;
    return (!is_neg(b0) && !is_neg(b1) && !is_neg(b2)) ? 1 : 0;
  } else {
    d3 d1 = d3_sub(Y[1], Y[0]), d2 = d3_sub(Y[3], Y[2]), r = d3_sub(Y[0], Y[2]);
    double A = d3_dot(d1, d1), B = d3_dot(d1, d2), E = d3_dot(d2, d2), C = d3_dot(d1, r), F = d3_dot(d2, r);
    double den = __fma_rn(A, E, -__dmul_rn(B, B));
    if (!is_pos(den)) return -1;
    double ns = __fma_rn(B, F, -__dmul_rn(C, E));
    double nu = __fma_rn(A, F, -__dmul_rn(B, C));
    if (quot_neg(ns, den) || quot_neg(nu, den) || quot_above1(ns, den) || quot_above1(nu, den)) return 0;
    double s = __ddiv_rn(ns, den);
    double u = __ddiv_rn(nu, den);
    w1 = s; w2 = u;
    const long long one = 0x3FF0000000000000ll;
    bool s_le1 = is_neg(s) || __double_as_longlong(s) <= one;
    bool u_le1 = is_neg(u) || __double_as_longlong(u) <= one;
    return (!is_neg(s) && s_le1 && !is_neg(u) && u_le1) ? 1 : 0;
  }
}

// The rounded quotient n / d when it may lie in (0, 1), else -1: it cannot
// when n is zero, the signs differ, or |n| >= |d| (then n / d >= 1 exactly,
// and so rounded); only the remaining case is divided (an exact quotient in
// (0, 1) may still round to 0 or 1, which the division decides).  Zero or
// NaN d falls in the |n| >= |d| or sign cases exactly as the quotient would
// fall outside (0, 1).
__device__ __forceinline__ double quot01(double n, double d) {
  if (is_zero(n) || is_neg(n) != is_neg(d) || !(fabs(n) < fabs(d))) return -1.0;
  return __ddiv_rn(n, d);
}

// 0 no contact, 1 contact, 2 degenerate.
__device__ int ccd64(int kind, const d3* X0, const d3* D, double& tau, double& w1, double& w2, long long& flops) {
  flops += 18 + 9 + 21 + 9 + 32;  // differences, cross products (+ sum), 6 dot products + 2 sums
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
  if (is_zero(k0) && is_zero(k1) && is_zero(k2) && is_zero(k3)) return 2;
  double e0 = k1, e1 = __dmul_rn(2.0, k2), e2 = __dmul_rn(3.0, k3);
  double r[2]; int nr = 0;
  flops += 2;
  if (!is_zero(e2)) {
    double disc = __fma_rn(e1, e1, -__dmul_rn(__dmul_rn(4.0, e2), e0));
    flops += 4;
    if (is_pos(disc)) {
      flops += 5;
      double sq = __dsqrt_rn(disc);
      double q = __dmul_rn(-0.5, __dadd_rn(e1, !is_neg(e1) ? sq : -sq));
      r[0] = quot01(q, e2); r[1] = quot01(e0, q); nr = 2;
    }
  } else if (!is_zero(e1)) {
    r[0] = quot01(-e0, e1); nr = 1;
    flops += 1;
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
#pragma unroll 1
  for (int s = 0; s + 1 < ne; ++s) {
    double l = ends[s], rr = ends[s + 1];
    double fl = horner3(k0, k1, k2, k3, l), fr = horner3(k0, k1, k2, k3, rr), t;
    flops += 12;
    if (is_zero(fl)) t = l;
    else if (is_zero(fr)) t = rr;
    else if (is_neg(fl) != is_neg(fr)) t = bisect64(k0, k1, k2, k3, l, rr, fl, flops);
    else continue;
    flops += 24 + 9 + 25 + 3;  // positions, differences, dot products, determinant
    d3 Y[4];
    for (int q = 0; q < 4; ++q) Y[q] = d3_at(X0[q], t, D[q]);
    double u1 = 0.0, u2 = 0.0;
    int in = inside64(kind, Y, u1, u2);
    if (in >= 0) flops += kind == KIND_VF ? 10 : 8;  // numerators, divisions (and 1 - b1 - b2)
    if (in < 0) { degen = true; continue; }
    if (in == 1) { tau = t; w1 = u1; w2 = u2; return 1; }
  }
  return degen ? 2 : 0;
}

// ---------------------------------------------------------------------------
// Eq. 3.1 with d_m > 0: g(t) = f(t)^2 - d_m^2 |m(t)|^2 (f the cubic, m the
// normal), degree six.  The roots of the derivatives, found from the linear
// one upward, split [0, 1] into pieces on which each derivative (and finally
// g) is monotone; each piece is taken as in the cubic test, and the first
// piece also at t = 0 when g(0) <= 0.  The fixed FP64 sequence of the method
// definition (plain FP64 instructions, no sign tiers); the stage-4 operation
// count covers the d_m = 0 procedure only.
// ---------------------------------------------------------------------------
__device__ __forceinline__ double horner_n(const double* c, int n, double t) {
  double r = c[n];
  for (int i = n - 1; i >= 0; --i) r = __fma_rn(r, t, c[i]);
  return r;
}

// The bisection of a degree-N polynomial c on [lo, hi] (0 <= lo < hi <= 1),
// taking exactly the FP64 path of the plain procedure: every midpoint is the
// FP64 midpoint, every sign the sign of the FP64 Horner value.  As in the
// cubic's bisection, that sign is read from cheaper evaluations when their
// error bounds prove it.  With S = sum |c_i| and S1 = sum i |c_i|:
//  - FP32 Horner at the truncated midpoint: |f64(mid) - f32| <=
//    gamma_2N(2^-24) S + 2^-24 S + gamma_2N(2^-53) S + 2^-23 S1 (Horner error
//    bounds with room to spare, coefficient rounding, the FP64 value's own
//    error, the midpoint's truncation times max |f'| on [0, 1]) <=
//    (2N + 1.5) 2^-24 S + 1.25e-7 S1 for N <= 6;
//  - double-float Horner: N multiply-add steps at <= 2^-44 relative each, the
//    coefficients' and the midpoint's representation (2^-48 |c_i|, 2^-47 mid
//    times max |f'|) and the FP64 Horner error (< 2^-50 S) stay below
//    2^-40 (S + S1) for N <= 6.
// Above its bound a tier's value has the sign of the FP64 value, which is
// then not zero.  Coefficients outside [1e-25, 1e25] (1e-20 for the
// double-float tier) keep every FP32 term clear of underflow and overflow;
// outside that range only FP64 is used.
template <int N>
__device__ __noinline__ double bisect_tn(const double* c, double lo, double hi, double flo, long long& flops) {
  bool neg_lo = is_neg(flo);
  float fc[N + 1];
  dflt cd[N + 1];
  float S = 0.0f, S1 = 0.0f, mk = 0.0f;
#pragma unroll
  for (int i = 0; i <= N; ++i) {
    fc[i] = __double2float_rn(c[i]);
    float ai = fabsf(fc[i]);
    S = S + ai;
    S1 = S1 + (float)i * ai;
    mk = fmaxf(mk, ai);
    cd[i] = {fc[i], __double2float_rn(__dsub_rn(c[i], (double)fc[i]))};
  }
  float E = 1.01f * ((2.0f * N + 1.5f) * 5.9604645e-8f * S + 1.25e-7f * S1);
  float Edf = 1.01f * 9.094947e-13f * (S + S1);   // 2^-40
  bool use_df = mk > 1e-20f && mk < 1e25f;
  if (!(mk > 1e-25f && mk < 1e25f)) E = INFINITY;
#pragma unroll 1
  for (int it = 0; it < 64; ++it) {
    bool ok;
    double mid = mid_rn(lo, hi, ok);
    if (!ok) mid = __dmul_rn(__dadd_rn(lo, hi), 0.5);
    long long bm = __double_as_longlong(mid);   // lo, mid, hi >= 0: bit patterns order them
    if (!(bm > __double_as_longlong(lo) && bm < __double_as_longlong(hi))) break;
    flops += 2 + 2 * N;
    float m = trunc_f32(mid);
    float fs = fc[N];
#pragma unroll
    for (int i = N - 1; i >= 0; --i) fs = fmaf(fs, m, fc[i]);
    bool neg;
    dflt md;
    bool done = fabsf(fs) > E;
    if (done) {
      neg = fs < 0.0f;
    } else if (use_df && df_of_unit(mid, md)) {
      dflt v = cd[N];
#pragma unroll
      for (int i = N - 1; i >= 0; --i) v = df_add(df_mul(v, md), cd[i]);
      float vv = v.h + v.l;
      neg = vv < 0.0f;
      done = fabsf(vv) > Edf;
    }
    if (!done) {
      double fm = horner_n(c, N, mid);
      if (is_zero(fm)) return mid;
      neg = is_neg(fm);
    }
    if (neg == neg_lo) lo = mid;
    else hi = mid;
  }
  return lo;
}

__device__ __forceinline__ double bisect_n(const double* c, int n, double lo, double hi, double flo,
                                           long long& flops) {
  switch (n) {
    case 2: return bisect_tn<2>(c, lo, hi, flo, flops);
    case 3: return bisect_tn<3>(c, lo, hi, flo, flops);
    case 4: return bisect_tn<4>(c, lo, hi, flo, flops);
    case 5: return bisect_tn<5>(c, lo, hi, flo, flops);
    default: return bisect_tn<6>(c, lo, hi, flo, flops);
  }
}

__device__ __noinline__ int ccd64_dm(int kind, const d3* X0, const d3* D, double dm, double& tau, double& w1,
                                     double& w2, long long& flops) {
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
  double q0 = d3_dot(n0, n0);
  double q1 = __dmul_rn(2.0, d3_dot(n0, n1));
  double q2 = __dadd_rn(d3_dot(n1, n1), __dmul_rn(2.0, d3_dot(n0, n2)));
  double q3 = __dmul_rn(2.0, d3_dot(n1, n2));
  double q4 = d3_dot(n2, n2);
  double dd = __dmul_rn(dm, dm);
  // C[k]: the k-th derivative of g, degree 6 - k
  double C[6][7];
  C[0][0] = __dsub_rn(__dmul_rn(k0, k0), __dmul_rn(dd, q0));
  C[0][1] = __dsub_rn(__dmul_rn(2.0, __dmul_rn(k0, k1)), __dmul_rn(dd, q1));
  C[0][2] = __dsub_rn(__dadd_rn(__dmul_rn(2.0, __dmul_rn(k0, k2)), __dmul_rn(k1, k1)), __dmul_rn(dd, q2));
  C[0][3] = __dsub_rn(__dmul_rn(2.0, __dadd_rn(__dmul_rn(k0, k3), __dmul_rn(k1, k2))), __dmul_rn(dd, q3));
  C[0][4] = __dsub_rn(__dadd_rn(__dmul_rn(2.0, __dmul_rn(k1, k3)), __dmul_rn(k2, k2)), __dmul_rn(dd, q4));
  C[0][5] = __dmul_rn(2.0, __dmul_rn(k2, k3));
  C[0][6] = __dmul_rn(k3, k3);
  // differences 18, normals 39, cubic 32, |m|^2 34, d_m^2 1, sextic 28, derivatives 20
  flops += 18 + 39 + 32 + 34 + 1 + 28 + 20;
  bool allz = true;
  for (int i = 0; i <= 6; ++i) allz = allz && is_zero(C[0][i]);
  if (allz) return 2;
  for (int k = 1; k < 6; ++k)
    for (int i = 0; i <= 6 - k; ++i) C[k][i] = __dmul_rn((double)(i + 1), C[k - 1][i + 1]);
  // roots in (0, 1) of C[5] (linear), then C[4], ..., C[1] = g'
  double rts[6], nrt[6];
  int nr = 0;
  if (!is_zero(C[5][1])) {
    double t = __ddiv_rn(-C[5][0], C[5][1]);
    flops += 1;
    if (t > 0.0 && t < 1.0) rts[nr++] = t;
  }
  for (int k = 4; k >= 1; --k) {
    int n = 6 - k, nn = 0;
    for (int sgi = 0; sgi <= nr; ++sgi) {
      double l = sgi == 0 ? 0.0 : rts[sgi - 1], r = sgi == nr ? 1.0 : rts[sgi];
      double fl = horner_n(C[k], n, l), fr = horner_n(C[k], n, r), t;
      flops += 4 * n;
      if (is_zero(fl)) t = l;
      else if (is_zero(fr)) t = r;
      else if (is_neg(fl) != is_neg(fr)) t = bisect_n(C[k], n, l, r, fl, flops);
      else continue;
      if (t > 0.0 && t < 1.0 && (nn == 0 || t > nrt[nn - 1])) nrt[nn++] = t;
    }
    for (int i = 0; i < nn; ++i) rts[i] = nrt[i];
    nr = nn;
  }
  bool degen = false;
  for (int sgi = 0; sgi <= nr; ++sgi) {
    double l = sgi == 0 ? 0.0 : rts[sgi - 1], r = sgi == nr ? 1.0 : rts[sgi];
    double gl = horner_n(C[0], 6, l), gr = horner_n(C[0], 6, r), t;
    flops += 24;
    if (sgi == 0 && (is_neg(gl) || is_zero(gl))) t = l;
    else if (is_zero(gl)) t = l;
    else if (is_zero(gr)) t = r;
    else if (is_neg(gl) != is_neg(gr)) t = bisect_n(C[0], 6, l, r, gl, flops);
    else continue;
    flops += 24 + 9 + 25 + 3;  // positions, differences, dot products, determinant
    d3 Y[4];
    for (int q = 0; q < 4; ++q) Y[q] = d3_at(X0[q], t, D[q]);
    double u1 = 0.0, u2 = 0.0;
    int in = inside64(kind, Y, u1, u2);
    if (in >= 0) flops += kind == KIND_VF ? 10 : 8;  // numerators, divisions (and 1 - b1 - b2)
    if (in < 0) { degen = true; continue; }
    if (in == 1) { tau = t; w1 = u1; w2 = u2; return 1; }
  }
  return degen ? 2 : 0;
}

// ---------------------------------------------------------------------------
// stages 2-4 on queued pairs
// ---------------------------------------------------------------------------
// queue entry: kind (0 = VF A->B, 1 = VF B->A, 2 = EE) << 16 | x << 8 | y
__device__ __forceinline__ void entry_slots(const WarpSm& ws, unsigned e, int& kind, int& x, int& y, int* sl,
                                            const PatchSm*& SA, const PatchSm*& SB) {
  kind = e >> 16; x = (e >> 8) & 0xFF; y = e & 0xFF;
  SA = (kind == 1) ? &ws.B : &ws.A;   // side holding the first primitive (vertex / edge)
  SB = (kind == 1) ? &ws.A : &ws.B;
  if (kind < 2) {
    sl[0] = SA->tp->v_slot[x];
    int t = SB->tp->t_slots[y];
    sl[1] = t & 63; sl[2] = (t >> 6) & 63; sl[3] = (t >> 12) & 63;
  } else {
    int ea = SA->tp->e_slots[x], eb = SB->tp->e_slots[y];
    sl[0] = ea & 63; sl[1] = (ea >> 6) & 63; sl[2] = eb & 63; sl[3] = (eb >> 6) & 63;
  }
}

__device__ __forceinline__ const PatchSm& point_side(int kind, int q, const PatchSm* SA, const PatchSm* SB) {
  return (q == 0 || (kind == 2 && q == 1)) ? *SA : *SB;
}

// ---------------------------------------------------------------------------
// global pair descriptors (stages 3b and 4)
// ---------------------------------------------------------------------------
__device__ __forceinline__ unsigned long long make_desc(int r, int type, int ga, int gb) {
  return ((unsigned long long)(unsigned)r << 32) | ((unsigned long long)type << 30) | ((unsigned long long)ga << 15) |
         (unsigned long long)gb;
}

// The 4 points of a descriptor: vertex id and whether the point belongs to
// vesicle j (periodic image applied).  VF type 0: vertex of i, triangle of j;
// type 1: vertex of j, triangle of i; EE: edge of i, edge of j.
__device__ __forceinline__ void desc_points(ulonglong2 e, int& r, int& type, int& ga, int& gb, int* vid, bool* onj) {
  r = (int)(e.x >> 32); type = (int)((e.x >> 30) & 3); ga = (int)((e.x >> 15) & 0x7FFF); gb = (int)(e.x & 0x7FFF);
  for (int q = 0; q < 4; ++q) vid[q] = (int)((e.y >> (16 * q)) & 0xFFFF);
  onj[0] = type == 1;
  onj[1] = type == 0;
  onj[2] = type != 1;
  onj[3] = type != 1;
}

// FP32 points of a descriptor in the frame of its pair (for stage 3b).
__device__ __forceinline__ void desc_points_f32(const narrow_args& a, ulonglong2 e, int& kind, f3* xq, f3* dq,
                                                float& ep, float& es) {
  int r, ty, ga, gb, vid[4];
  bool onj[4];
  desc_points(e, r, ty, ga, gb, vid, onj);
  const stiv_pair_info* pi = a.pinfo + r;
  float4 fr = pi->frame;
  int vi = pi->vi, vj = pi->vj;
  ep = fr.w;
  es = same_side_err(fmaxf(((const float4*)a.vorg)[vi].w, ((const float4*)a.vorg)[vj].w),
                     fmaxf(fabsf(fr.x), fmaxf(fabsf(fr.y), fabsf(fr.z))));
  kind = ty == 2 ? 1 : 0;
  for (int q = 0; q < 4; ++q) {
    int v = onj[q] ? vj : vi;
    const float4* fp = (const float4*)(a.fprep + (size_t)v * a.fstride) + 2 * (size_t)vid[q];
    float4 x = fp[0], d = fp[1];
    if (a.mixed) {   // FP32 vertices as stored: relative position and displacement, one rounding each
      float4 o = ((const float4*)a.vorg)[v];
      d = make_float4(d.x - x.x, d.y - x.y, d.z - x.z, 0.f);
      x = make_float4(x.x - o.x, x.y - o.y, x.z - o.z, 0.f);
    }
    float o0 = onj[q] ? fr.x : 0.f, o1 = onj[q] ? fr.y : 0.f, o2 = onj[q] ? fr.z : 0.f;
    xq[q] = {x.x + o0, x.y + o1, x.z + o2};
    dq[q] = {d.x, d.y, d.z};
  }
}

// Append a descriptor to a global list (warp-aggregated; lanes with keep).
__device__ __forceinline__ void push_global(ulonglong2* list, int64_t cap, int64_t* count, int64_t* status,
                                            bool keep, ulonglong2 e, int lane) {
  unsigned m = __ballot_sync(0xffffffffu, keep);
  if (!m) return;
  unsigned long long base = 0;
  int leader = __ffs(m) - 1;
  if (lane == leader) base = atomicAdd((unsigned long long*)count, (unsigned long long)__popc(m));
  base = __shfl_sync(0xffffffffu, base, leader);
  if (keep) {
    int64_t k = (int64_t)base + __popc(m & ((1u << lane) - 1u));
    if (k < cap) list[k] = e;
    else atomicOr((unsigned long long*)status, STIV_F_WORK_OVERFLOW);
  }
}

__device__ __forceinline__ void load_f32(const int* sl, int kind, const PatchSm* SA, const PatchSm* SB, f3* xq,
                                         f3* dq) {
  for (int q = 0; q < 4; ++q) {
    const PatchSm& S = point_side(kind, q, SA, SB);
    xq[q] = {S.x[0][sl[q]], S.x[1][sl[q]], S.x[2][sl[q]]};
    dq[q] = {S.d[0][sl[q]], S.d[1][sl[q]], S.d[2][sl[q]]};
  }
}

// The exact FP64 swept-box test of a queued primitive pair from the vertex
// values themselves (FP64, or the FP32 values widened), the second vesicle's
// points at the pair's periodic image (added in FP64) and, with d_m > 0, its
// per-vertex boxes widened by d_m: the test that defines the pairs tested,
// for the rare pair whose FP32 boxes and their error bound do not decide it.
template <bool MIXED, bool DM>
__device__ __noinline__ bool exact_box_hit(const narrow_args& a, int r, int kind, const PatchSm* SA, const PatchSm* SB,
                                           const int* sl) {
  const stiv_pair_info& pi = a.pinfo[r];
  int code = pi.code;
  int sB[3] = {code / 9 - 1, (code / 3) % 3 - 1, code % 3 - 1};
  int na = kind == 2 ? 2 : 1;
  double lo[2][3], hi[2][3];
  for (int side = 0; side < 2; ++side)
    for (int c = 0; c < 3; ++c) { lo[side][c] = INFINITY; hi[side][c] = -INFINITY; }
  for (int q = 0; q < 4; ++q) {
    const PatchSm* S = q < na ? SA : SB;
    bool onB = (q < na) == (kind == 1);   // the point belongs to vesicle j (patch B)
    int side = q < na ? 0 : 1;
    int v = S->vid[sl[q]];
    int P = onB ? (pi.Pij >> 16) : (pi.Pij & 0xFFFF);
    int nv = stiv_nverts(P);
    size_t vb = (size_t)(onB ? pi.voff_j : pi.voff_i) + v;
    for (int c = 0; c < 3; ++c) {
      double p0 = vtx<MIXED>(a.X, vb + (size_t)c * nv), p1 = vtx<MIXED>(a.X, vb + (size_t)(3 + c) * nv);
      if (onB && sB[c] != 0) { double shc = sB[c] * a.L[c]; p0 = p0 + shc; p1 = p1 + shc; }
      double l = fmin(p0, p1), h = fmax(p0, p1);
      if (DM && onB) {   // d_m > 0: vesicle j's boxes widened by d_m per vertex (FP64, as computed)
        l = __dsub_rn(l, a.dm);
        h = __dadd_rn(h, a.dm);
      }
      lo[side][c] = fmin(lo[side][c], l);
      hi[side][c] = fmax(hi[side][c], h);
    }
  }
  bool hit = true;
  for (int c = 0; c < 3; ++c) hit = hit && lo[0][c] <= hi[1][c] && lo[1][c] <= hi[0][c];
  return hit;
}

// Stage 2 (exact box) and 3a (Bernstein) on up to n entries of q1; survivors
// go to the global list of stage 3b (of stage 4 when the FP32 rejection is
// off) as descriptors.
template <bool MIXED, bool DM>
__device__ __noinline__ void stage_filter(WarpSm& ws, int n, int lane, int r, const narrow_args& a,
                                          long long& nprim) {
  bool keep = false;
  ulonglong2 desc = make_ulonglong2(0ull, 0ull);
  if (lane < n) {
    unsigned e = ws.q1[lane];
    int kind, x, y, sl[4];
    const PatchSm *SA, *SB;
    entry_slots(ws, e, kind, x, y, sl, SA, SB);
    // exact FP64 swept-box overlap
    int na = kind == 2 ? 2 : 1;
    bool hit = true;
    {
      // Each staged FP32 box end lies within m of the exact FP64 box end of
      // its slot (in the pair frame), so a slot's exact box contains its
      // FP32 box shrunk by 2m at each end.  If the shrunk boxes of the two
      // primitives overlap on every axis (boxes shrunk by 3 M, M the largest
      // m of the primitive's slots, which also covers the rounding of the
      // shrinking), the exact boxes overlap; the pair came through the
      // outward boxes of stage 1, so only the pairs in between need the exact
      // test, on the FP64 values.  With d_m > 0 vesicle j's boxes are widened
      // by d_m on both sides: FP32 rounded up, FP64 as computed per vertex;
      // 2^-21 d_m covers the difference of the two roundings.
      float ma = SA->m[sl[0]], mb = SB->m[sl[na]];
      if (na == 2) ma = fmaxf(ma, SA->m[sl[1]]);
      for (int q = na + 1; q < 4; ++q) mb = fmaxf(mb, SB->m[sl[q]]);
      float gap = 3.0f * (ma + mb);
      if (DM) gap += 4.7683716e-7f * __double2float_ru(a.dm);
      bool sure = true;
      for (int c = 0; c < 3; ++c) {
        float alo = SA->lo[c][sl[0]], ahi = SA->hi[c][sl[0]];
        if (na == 2) { alo = fminf(alo, SA->lo[c][sl[1]]); ahi = fmaxf(ahi, SA->hi[c][sl[1]]); }
        float blo = SB->lo[c][sl[na]], bhi = SB->hi[c][sl[na]];
        for (int q = na + 1; q < 4; ++q) { blo = fminf(blo, SB->lo[c][sl[q]]); bhi = fmaxf(bhi, SB->hi[c][sl[q]]); }
        sure = sure && alo + gap <= bhi && blo + gap <= ahi;
      }
      if (!sure) hit = exact_box_hit<MIXED, DM>(a, r, kind, SA, SB, sl);
    }
    if (hit) {
      ++nprim;
      keep = true;
      if (DM && !a.exact_only) {   // d_m > 0: drop pairs that certainly stay out of the d_m band
        f3 xq[4], dq[4];
        load_f32(sl, kind, SA, SB, xq, dq);
        keep = !band_reject(kind == 2 ? 1 : 0, xq, dq, ws.dx, 2.0f * ws.dx, (float)a.dm);
      } else if (!a.exact_only) {
        f3 xq[4], dq[4];
        load_f32(sl, kind, SA, SB, xq, dq);
        cubic32 q = cubic_fp32(kind == 2 ? 1 : 0, xq, dq, ws.dx, 2.0f * ws.dx);
        keep = !bernstein_reject(q);
      }
      if (keep) {
        unsigned long long v0 = (unsigned)SA->vid[sl[0]], v1, v2, v3;
        if (kind < 2) {
          v1 = (unsigned)SB->vid[sl[1]]; v2 = (unsigned)SB->vid[sl[2]]; v3 = (unsigned)SB->vid[sl[3]];
        } else {
          unsigned long long u = (unsigned)SA->vid[sl[1]];
          if (u < v0) { v1 = v0; v0 = u; } else v1 = u;
          unsigned long long p = (unsigned)SB->vid[sl[2]], q = (unsigned)SB->vid[sl[3]];
          v2 = p < q ? p : q; v3 = p < q ? q : p;
        }
        // EE edge indices are formed by the FP64 stage for contacts only
        desc.x = kind == 2 ? make_desc(r, kind, 0, 0) : make_desc(r, kind, (int)v0, prim_gid(*SB, 1, y));
        desc.y = v0 | (v1 << 16) | (v2 << 32) | (v3 << 48);
      }
    }
  }
  if (a.exact_only) push_global(a.q2, a.Q2, &a.ctr[15], &a.ctr[STIV_C_STATUS], keep, desc, lane);
  else push_global(a.q3, a.Q3, &a.ctr[14], &a.ctr[STIV_C_STATUS], keep, desc, lane);
}

// Queue the hits of one stage-1 test (n1: the queue length, the same in every
// lane); 32 queued entries go through stages 2 and 3a.
template <bool MIXED, bool DM>
__device__ __forceinline__ void enqueue(WarpSm& ws, bool hit, unsigned entry, int lane, int r, const narrow_args& a,
                                        long long& nprim, int& n1) {
  unsigned m = __ballot_sync(0xffffffffu, hit);
  if (!m) return;
  if (hit) ws.q1[n1 + __popc(m & ((1u << lane) - 1u))] = entry;
  n1 += __popc(m);
  if (n1 >= 32) {
    __syncwarp();
    stage_filter<MIXED, DM>(ws, 32, lane, r, a, nprim);
    unsigned rest = (lane + 32 < n1) ? ws.q1[lane + 32] : 0;
    __syncwarp();
    if (lane + 32 < n1) ws.q1[lane] = rest;
    n1 -= 32;
    __syncwarp();
  }
}

// Stages 1-3a: one warp per patch pair.  Three CTAs per SM leave 80
// registers a thread (four leave 64, with spills in the staging code).
template <bool MIXED, bool DM>
__global__ void __launch_bounds__(NW * 32, 3) narrow_kernel(narrow_args a) {
  extern __shared__ unsigned char smraw[];
  __shared__ PatchTopo topo[NVAR];
  WarpSm& ws = ((WarpSm*)smraw)[threadIdx.x >> 5];
  int lane = threadIdx.x & 31;
  for (int var = threadIdx.x >> 5; var < NVAR; var += NW) build_topo(topo[var], var, lane);
  __syncthreads();
  int64_t nwork = a.ctr[STIV_C_PATCH];
  if (nwork > a.W) nwork = a.W;
  long long nprim = 0;
  long long item = 0;
  if (lane == 0) item = (long long)atomicAdd((unsigned long long*)&a.ctr[10], 1ull);
  item = __shfl_sync(0xffffffffu, item, 0);
  while (item < nwork) {
    // the next item's index is fetched now and read at the end of this one
    long long next = 0;
    if (lane == 0) next = (long long)atomicAdd((unsigned long long*)&a.ctr[10], 1ull);
    uint64_t w = a.work[item];
    int r = (int)(w >> 32), pa = (int)((w >> 16) & 0xFFFF), pb = (int)(w & 0xFFFF);
    stiv_pair_info pi = a.pinfo[r];
    stage_pair<MIXED, DM>(ws, a, topo, pi, pa, pb, lane);
    filter_pair(ws, lane);
    int n1 = 0;
    // stage 1: FP32 boxes.  VF: vertices of A vs triangles of B (0), vertices of B vs triangles of A (1)
#pragma unroll 1
    for (int dir = 0; dir < 2; ++dir) {
      const PatchSm& V = dir == 0 ? ws.A : ws.B;
      const PatchSm& T = dir == 0 ? ws.B : ws.A;
      for (int y0 = 0; y0 < T.ntf; y0 += 32) {
        int yk = y0 + lane;
        bool valid = yk < T.ntf;
        int y = valid ? T.tf[yk] : 0;
        float tb[6];
        tri_box(T, y, tb);
#pragma unroll 1
        for (int xk = 0; xk < V.nvf; ++xk) {
          float4 lo = V.vlo[xk], hi = V.vhi[xk];
          float vb[6] = {lo.x, lo.y, lo.z, hi.x, hi.y, hi.z};
          bool hit = valid && fbox_hit(vb, tb);
          enqueue<MIXED, DM>(ws, hit, ((unsigned)dir << 16) | ((unsigned)V.vf[xk] << 8) | (unsigned)y, lane, r, a, nprim, n1);
        }
      }
    }
    if (a.include_ee) {
      for (int y0 = 0; y0 < ws.B.nef; y0 += 32) {
        int yk = y0 + lane;
        bool valid = yk < ws.B.nef;
        int y = valid ? ws.B.ef[yk] : 0;
        float eb[6];
        edge_box(ws.B, y, eb);
#pragma unroll 1
        for (int xk = 0; xk < ws.A.nef; ++xk) {
          float4 lo = ws.elo[xk], hi = ws.ehi[xk];
          float ab[6] = {lo.x, lo.y, lo.z, hi.x, hi.y, hi.z};
          bool hit = valid && fbox_hit(ab, eb);
          enqueue<MIXED, DM>(ws, hit, (2u << 16) | ((unsigned)ws.A.ef[xk] << 8) | (unsigned)y, lane, r, a, nprim, n1);
        }
      }
    }
    __syncwarp();
    if (n1 > 0) stage_filter<MIXED, DM>(ws, n1, lane, r, a, nprim);
    item = __shfl_sync(0xffffffffu, next, 0);
  }
  for (int off = 16; off > 0; off >>= 1) nprim += __shfl_down_sync(0xffffffffu, nprim, off);
  if (lane == 0 && nprim) atomicAdd((unsigned long long*)&a.ctr[STIV_C_PRIM], (unsigned long long)nprim);
}

// ---------------------------------------------------------------------------
// stage 3b: the pieces of [0,1] that may hold a root, certified non-contact.
// A warp takes 32 descriptors; the pieces that need the inside test become
// (descriptor, piece) tasks spread over the lanes, so that every lane runs the
// same test; an undecided piece is split in two, level by level (NLEVEL
// levels), and a half whose cubic certainly keeps one sign is dropped.
// ---------------------------------------------------------------------------
constexpr int PW = 8;          // warps per CTA
constexpr int NPIECE = 16;     // level-0 pieces of [0, 1]
constexpr int NLEVEL = 6;      // most refinement levels (finest piece: 1 / (16 * 32))
constexpr int MAXTASK = 512;
static_assert(NPIECE << (NLEVEL - 1) <= 1024, "piece index fits 10 bits");

struct PieceWarp {
  float x[32][4][3], d[32][4][3];
  float k[32][4], E[32], ep[32], ed[32], es[32];
  float rhs[32];   // d_m > 0: band_rhs of each pair
  int kind[32], fail[32];
  unsigned short task[MAXTASK], task2[MAXTASK];
  int ntask2;
};

// DM (d_m > 0): a piece is kept when the point may be within d_m of the plane
// there (out_of_band fails) instead of when the cubic may have a root; the
// inside certificate is the same, because the degree-six test uses the same
// inside test at its candidate times.
template <bool DM>
__global__ void __launch_bounds__(PW * 32, 4) pieces_kernel(narrow_args a) {
  extern __shared__ unsigned char psraw[];
  PieceWarp& W = ((PieceWarp*)psraw)[threadIdx.x >> 5];
  int lane = threadIdx.x & 31;
  int64_t n3 = a.ctr[14];
  if (n3 > a.Q3) n3 = a.Q3;
  int64_t nb = (n3 + 31) / 32;
  int64_t gw = (int64_t)blockIdx.x * PW + (threadIdx.x >> 5), nw = (int64_t)gridDim.x * PW;
  for (int64_t b = gw; b < nb; b += nw) {
    int64_t idx = b * 32 + lane;
    bool valid = idx < n3;
    ulonglong2 e = valid ? a.q3[idx] : make_ulonglong2(0ull, 0ull);
    unsigned mask = 0;
    W.fail[lane] = 0;
    if (valid) {
      int kind;
      f3 xq[4], dq[4];
      float ep, es;
      desc_points_f32(a, e, kind, xq, dq, ep, es);
      cubic32 q = cubic_fp32<DM>(kind, xq, dq, ep, es);
      for (int p = 0; p < 4; ++p) {
        W.x[lane][p][0] = xq[p].x; W.x[lane][p][1] = xq[p].y; W.x[lane][p][2] = xq[p].z;
        W.d[lane][p][0] = dq[p].x; W.d[lane][p][1] = dq[p].y; W.d[lane][p][2] = dq[p].z;
      }
      W.k[lane][0] = q.k0; W.k[lane][1] = q.k1; W.k[lane][2] = q.k2; W.k[lane][3] = q.k3;
      W.E[lane] = q.E; W.ep[lane] = ep; W.ed[lane] = q.ed; W.es[lane] = es; W.kind[lane] = kind;
      if (DM) W.rhs[lane] = band_rhs(q, ep, (float)a.dm);
      if (fabsf(q.k0) <= q.E && fabsf(q.k1) <= q.E && fabsf(q.k2) <= q.E && fabsf(q.k3) <= q.E) {
        W.fail[lane] = 1;   // may vanish identically: FP64 decides (degenerate)
      } else {
        const float w = 1.0f / NPIECE;
#pragma unroll 2
        for (int p = 0; p < NPIECE; ++p) {
          float t0 = p * w;
          float f0 = fmaf(fmaf(fmaf(q.k3, t0, q.k2), t0, q.k1), t0, q.k0);
          float fp1 = fmaf(fmaf(3.f * q.k3, t0, 2.f * q.k2), t0, q.k1);
          float g1 = w * fp1, g2 = w * w * fmaf(3.f * q.k3, t0, q.k2), g3 = w * w * w * q.k3;
          float c1 = f0 + g1 * (1.f / 3.f), c2 = f0 + (2.f * g1 + g2) * (1.f / 3.f), c3 = f0 + g1 + g2 + g3;
          bool keep_p = DM ? !out_of_band(f0, c1, c2, c3, q.E, W.rhs[lane]) : !certain_sign4(f0, c1, c2, c3, q.E);
          if (keep_p) mask |= 1u << p;
        }
      }
    }
    // task list of this batch: (owner lane, piece) of level 0
    int cnt = __popc(mask), off = cnt;
    for (int o = 1; o < 32; o <<= 1) { int v = __shfl_up_sync(0xffffffffu, off, o); if (lane >= o) off += v; }
    int total = __shfl_sync(0xffffffffu, off, 31);
    off -= cnt;
    for (unsigned m = mask; m; m &= m - 1) {
      int p = __ffs(m) - 1;
      if (off < MAXTASK) W.task[off] = (unsigned short)((lane << 10) | p);
      else W.fail[lane] = 1;
      ++off;
    }
    if (total > MAXTASK) total = MAXTASK;
    // adaptive refinement: a piece that may hold a root and whose inside test
    // is undecided splits in two, down to NLEVEL levels; a half that
    // certainly holds no root is dropped
    unsigned short* cur = W.task;
    unsigned short* nxt = W.task2;
#pragma unroll 1
    for (int level = 0; level < a.nlevel && total > 0; ++level) {
      if (lane == 0) W.ntask2 = 0;
      __syncwarp();
      const float w = (1.0f / NPIECE) * __int_as_float((127 - level) << 23);   // 2^-level / NPIECE
#pragma unroll 1
      for (int t0 = 0; t0 < total; t0 += 32) {
        int t = t0 + lane;
        // a descriptor already bound for the FP64 test needs none of its
        // other pieces decided
        if (t < total && !W.fail[cur[t] >> 10]) {
          int owner = cur[t] >> 10, idx = cur[t] & 1023;
          float tl = idx * w;
          bool may_root = true;
          if (level > 0) {
            float k0 = W.k[owner][0], k1 = W.k[owner][1], k2 = W.k[owner][2], k3 = W.k[owner][3], E = W.E[owner];
            float f0 = fmaf(fmaf(fmaf(k3, tl, k2), tl, k1), tl, k0);
            float fp1 = fmaf(fmaf(3.f * k3, tl, 2.f * k2), tl, k1);
            float g1 = w * fp1, g2 = w * w * fmaf(3.f * k3, tl, k2), g3 = w * w * w * k3;
            float c1 = f0 + g1 * (1.f / 3.f), c2 = f0 + (2.f * g1 + g2) * (1.f / 3.f), c3 = f0 + g1 + g2 + g3;
            may_root = DM ? !out_of_band(f0, c1, c2, c3, E, W.rhs[owner]) : !certain_sign4(f0, c1, c2, c3, E);
          }
          if (may_root) {
            f3 xq[4], dq[4];
            for (int q = 0; q < 4; ++q) {
              xq[q] = {W.x[owner][q][0], W.x[owner][q][1], W.x[owner][q][2]};
              dq[q] = {W.d[owner][q][0], W.d[owner][q][1], W.d[owner][q][2]};
            }
            int res = inside_cert(W.kind[owner], xq, dq, tl, w, W.ep[owner], W.ed[owner], W.es[owner]);
            if (res == 2) {
              W.fail[owner] = 1;                       // a contact: the FP64 test decides its time
            } else if (res == 0) {
              if (level + 1 == a.nlevel) {
                W.fail[owner] = 1;
              } else {
                int k = atomicAdd(&W.ntask2, 2);
                if (k + 1 < MAXTASK) {
                  nxt[k] = (unsigned short)((owner << 10) | (2 * idx));
                  nxt[k + 1] = (unsigned short)((owner << 10) | (2 * idx + 1));
                } else {
                  W.fail[owner] = 1;
                }
              }
            }
          }
        }
      }
      __syncwarp();
      total = min(W.ntask2, MAXTASK);
      unsigned short* tmp = cur; cur = nxt; nxt = tmp;
      __syncwarp();
    }
    __syncwarp();
    push_global(a.q2, a.Q2, &a.ctr[15], &a.ctr[STIV_C_STATUS], valid && W.fail[lane], e, lane);
    __syncwarp();
  }
}

// ---------------------------------------------------------------------------
// stage 4: the FP64 contact test, one descriptor per thread.  The register
// budget is capped (6 blocks of 128 threads per SM, 80 registers, for the
// cubic; 8 blocks, 64 registers, for d_m > 0): the dependent FP64 operations
// need the warps more than the spilled registers cost.
// ---------------------------------------------------------------------------
template <bool MIXED, bool DM>
__global__ void __launch_bounds__(128, DM ? 8 : 6) fp64_kernel(narrow_args a) {
  int lane = threadIdx.x & 31;
  int64_t n2 = a.ctr[15];
  if (n2 > a.Q2) n2 = a.Q2;
  long long ndeg = 0, flops = 0, nexact = 0;
  int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t base = (int64_t)blockIdx.x * blockDim.x; base < n2; base += stride) {
    int64_t idx = base + threadIdx.x;
    int type = -1, ga = 0, gb = 0, r = 0;
    double tau = 0.0, w1 = 0.0, w2 = 0.0;
    if (idx < n2) {
      ++nexact;
      int vid[4];
      bool onj[4];
      int ty;
      desc_points(a.q2[idx], r, ty, ga, gb, vid, onj);
      const stiv_pair_info* pi = a.pinfo + r;
      int code = pi->code, Pij = pi->Pij;
      long long voi = pi->voff_i, voj = pi->voff_j;
      int sB[3] = {code / 9 - 1, (code / 3) % 3 - 1, code % 3 - 1};
      int nvi = stiv_nverts(Pij & 0xFFFF), nvj = stiv_nverts(Pij >> 16);
      d3 X0[4], D[4];
      for (int q = 0; q < 4; ++q) {
        int nv = onj[q] ? nvj : nvi;
        size_t vb = (size_t)(onj[q] ? voj : voi) + vid[q];
        double p0[3], p1[3];
        for (int c = 0; c < 3; ++c) {
          size_t i0 = vb + (size_t)c * nv, i1 = vb + (size_t)(3 + c) * nv;
          p0[c] = vtx<MIXED>(a.X, i0);
          p1[c] = vtx<MIXED>(a.X, i1);
          if (onj[q] && sB[c] != 0) { double sh = sB[c] * a.L[c]; p0[c] = p0[c] + sh; p1[c] = p1[c] + sh; }
        }
        X0[q] = {p0[0], p0[1], p0[2]};
        D[q] = {__dsub_rn(p1[0], p0[0]), __dsub_rn(p1[1], p0[1]), __dsub_rn(p1[2], p0[2])};
      }
      flops += 12;  // displacements
      int st = DM ? ccd64_dm(ty == 2 ? KIND_EE : KIND_VF, X0, D, a.dm, tau, w1, w2, flops)
                  : ccd64(ty == 2 ? KIND_EE : KIND_VF, X0, D, tau, w1, w2, flops);
      if (st == 1) {
        type = ty;
        if (ty == 2) {   // edge indices of the two edges (their vertex ids are ordered)
          ga = stiv_edge_index(Pij & 0xFFFF, vid[0], vid[1]);
          gb = stiv_edge_index(Pij >> 16, vid[2], vid[3]);
        }
      }
      else if (st == 2) ++ndeg;
    }
    unsigned m = __ballot_sync(0xffffffffu, type >= 0);
    if (m) {
      unsigned long long cb = 0;
      int leader = __ffs(m) - 1;
      if (lane == leader) cb = atomicAdd((unsigned long long*)&a.ctr[11], (unsigned long long)__popc(m));
      cb = __shfl_sync(0xffffffffu, cb, leader);
      if (type >= 0) {
        int64_t k = (int64_t)cb + __popc(m & ((1u << lane) - 1u));
        if (k < a.C) {
          a.rc_pair[k] = r; a.rc_type[k] = type; a.rc_a[k] = ga; a.rc_b[k] = gb;
          a.rc_tau[k] = tau; a.rc_w[2 * k] = w1; a.rc_w[2 * k + 1] = w2;
        }
      }
      unsigned mee = __ballot_sync(0xffffffffu, type == 2);
      if (lane == leader) {
        if (mee) atomicAdd((unsigned long long*)&a.ctr[STIV_C_EE], (unsigned long long)__popc(mee));
        if (m & ~mee) atomicAdd((unsigned long long*)&a.ctr[STIV_C_VF], (unsigned long long)__popc(m & ~mee));
      }
    }
  }
  for (int off = 16; off > 0; off >>= 1) {
    ndeg += __shfl_down_sync(0xffffffffu, ndeg, off);
    flops += __shfl_down_sync(0xffffffffu, flops, off);
    nexact += __shfl_down_sync(0xffffffffu, nexact, off);
  }
  if (lane == 0) {
    if (ndeg) atomicAdd((unsigned long long*)&a.ctr[STIV_C_DEGEN], (unsigned long long)ndeg);
    if (flops) atomicAdd((unsigned long long*)&a.ctr[12], (unsigned long long)flops);
    if (nexact) atomicAdd((unsigned long long*)&a.ctr[13], (unsigned long long)nexact);
  }
}

// Level 1: patch pairs of one candidate vesicle pair per warp.  A's patches
// are kept that meet vesicle j's box, then B's that meet the union of A's
// kept patches, then A's that meet the union of B's; a pair of kept patches
// is emitted when their boxes overlap and some cell of one meets some cell
// of the other (every primitive lies in one cell of its patch).  Dynamic
// shared memory: per warp 2 x mp patch boxes and 2 x mp list entries.
__global__ void __launch_bounds__(128) patch_pairs_kernel(const int32_t* pv, const double* vbox, const float* pbox,
                                                          double Lx, double Ly, double Lz, const int32_t* ci,
                                                          const int32_t* cj, const int32_t* cs, int64_t cap,
                                                          int64_t W, uint64_t* work, int64_t* ctr, int mp,
                                                          const float* vorg, const int64_t* voff,
                                                          stiv_pair_info* pinfo, double dm) {
  extern __shared__ float psm[];
  int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
  float* sbw = psm + (size_t)wid * 2 * mp * 6;                       // [2][mp][6]
  unsigned short* law = (unsigned short*)(psm + (size_t)4 * 2 * mp * 6) + (size_t)wid * 2 * mp;
  unsigned short* lbw = law + mp;
  int64_t npairs = ctr[STIV_C_PAIRS];
  if (npairs > cap) npairs = cap;
  double L[3] = {Lx, Ly, Lz};
  for (int64_t r = (int64_t)blockIdx.x * 4 + wid; r < npairs; r += (int64_t)gridDim.x * 4) {
    int i = ci[r], j = cj[r], code = cs[r];
    int s[3] = {code / 9 - 1, (code / 3) % 3 - 1, code % 3 - 1};
    int Pi = 2 * pv[i], Pj = 2 * pv[j];
    if (lane == 0) {
      // FP32 frame of the pair: origin of vesicle i; |FP32 position - exact
      // position| per component is bounded by 2^-22 (R_i + R_j + 2 |offset|)
      // (rounding of X0 - origin, of the offset and of the frame change)
      float o[3], dmax = 0.f;
      for (int c = 0; c < 3; ++c) {
        double d = ((double)vorg[4 * j + c] + s[c] * L[c]) - (double)vorg[4 * i + c];
        o[c] = (float)d;
        dmax = fmaxf(dmax, fabsf(o[c]));
      }
      stiv_pair_info p;
      p.frame = make_float4(o[0], o[1], o[2], 2.3841858e-7f * (vorg[4 * i + 3] + vorg[4 * j + 3] + 2.0f * dmax));
      p.vi = i; p.vj = j; p.code = code; p.Pij = Pi | (Pj << 16);
      p.voff_i = voff[i]; p.voff_j = voff[j];
      pinfo[r] = p;
    }
    int ni = stiv_npatches(Pi), nj = stiv_npatches(Pj);
    float shlo[3], shhi[3];
    for (int c = 0; c < 3; ++c) {
      double sh = s[c] * L[c];
      // d_m > 0: vesicle j's patch boxes widened by d_m (rounded outward)
      shlo[c] = __double2float_rd(__dsub_rd(sh, dm)); shhi[c] = __double2float_ru(__dadd_ru(sh, dm));
    }
    float bj[6];   // vesicle j's box at its image (A's patches are filtered against it)
    for (int c = 0; c < 3; ++c) {
      bj[c] = __fadd_rd(__double2float_rd(vbox[6 * j + c]), shlo[c]);
      bj[3 + c] = __fadd_ru(__double2float_ru(vbox[6 * j + 3 + c]), shhi[c]);
    }
    for (int k = lane; k < ni; k += 32)
      for (int c = 0; c < 6; ++c) sbw[(0 * mp + k) * 6 + c] = pbox[((size_t)i * mp + k) * STIV_PBOX + c];
    for (int k = lane; k < nj; k += 32)
      for (int c = 0; c < 3; ++c) {
        sbw[(1 * mp + k) * 6 + c] = __fadd_rd(pbox[((size_t)j * mp + k) * STIV_PBOX + c], shlo[c]);
        sbw[(1 * mp + k) * 6 + 3 + c] = __fadd_ru(pbox[((size_t)j * mp + k) * STIV_PBOX + 3 + c], shhi[c]);
      }
    __syncwarp();
    int na = 0, nb = 0;
    for (int k0 = 0; k0 < ni; k0 += 32) {
      int k = k0 + lane;
      bool hit = k < ni && fbox_hit(&sbw[(0 * mp + k) * 6], bj);
      unsigned m = __ballot_sync(0xffffffffu, hit);
      if (hit) law[na + __popc(m & ((1u << lane) - 1u))] = (unsigned short)k;
      na += __popc(m);
    }
    // union box of a list of staged patch boxes (side 0: A, 1: B)
    auto list_union = [&](const unsigned short* lst, int n, int side, float* u) {
      float lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
      for (int q = lane; q < n; q += 32) {
        const float* bx = &sbw[(side * mp + lst[q]) * 6];
        for (int c = 0; c < 3; ++c) { lo[c] = fminf(lo[c], bx[c]); hi[c] = fmaxf(hi[c], bx[3 + c]); }
      }
      for (int c = 0; c < 3; ++c) {
        u[c] = fkey_val(__reduce_min_sync(0xffffffffu, fkey32(lo[c])));
        u[3 + c] = fkey_val(__reduce_max_sync(0xffffffffu, fkey32(hi[c])));
      }
    };
    // B's patches against the union of A's kept patches (a patch of B that
    // meets a kept patch of A meets their union), then A's kept patches
    // against the union of B's
    __syncwarp();
    float ua[6], ub[6];
    list_union(law, na, 0, ua);
    for (int k0 = 0; k0 < nj; k0 += 32) {
      int k = k0 + lane;
      bool hit = k < nj && fbox_hit(&sbw[(1 * mp + k) * 6], ua);
      unsigned m = __ballot_sync(0xffffffffu, hit);
      if (hit) lbw[nb + __popc(m & ((1u << lane) - 1u))] = (unsigned short)k;
      nb += __popc(m);
    }
    __syncwarp();
    list_union(lbw, nb, 1, ub);
    {
      int na2 = 0;
      for (int q0 = 0; q0 < na; q0 += 32) {
        int q = q0 + lane;
        int k = q < na ? law[q] : 0;
        bool hit = q < na && fbox_hit(&sbw[(0 * mp + k) * 6], ub);
        unsigned m = __ballot_sync(0xffffffffu, hit);
        __syncwarp();
        if (hit) law[na2 + __popc(m & ((1u << lane) - 1u))] = (unsigned short)k;
        na2 += __popc(m);
      }
      na = na2;
    }
    __syncwarp();
    for (int e0 = 0; e0 < na * nb; e0 += 32) {
      int e = e0 + lane;
      bool hit = false;
      int pa = 0, pb = 0;
      if (e < na * nb) {
        pa = law[e / nb]; pb = lbw[e % nb];
        hit = fbox_hit(&sbw[(0 * mp + pa) * 6], &sbw[(1 * mp + pb) * 6]);
        if (hit) {
          // every primitive lies in one of its patch's four cells: some cell
          // of pa must meet some cell of pb (vesicle j's at its image,
          // widened by d_m, rounded outward as the patch boxes)
          const float4* ca = (const float4*)(pbox + ((size_t)i * mp + pa) * STIV_PBOX + STIV_PBOX_CELLS);
          const float4* cb = (const float4*)(pbox + ((size_t)j * mp + pb) * STIV_PBOX + STIV_PBOX_CELLS);
          float bB[4][6];
#pragma unroll
          for (int q = 0; q < 4; ++q) {
            float4 l = cb[2 * q], u = cb[2 * q + 1];
            bB[q][0] = __fadd_rd(l.x, shlo[0]); bB[q][1] = __fadd_rd(l.y, shlo[1]); bB[q][2] = __fadd_rd(l.z, shlo[2]);
            bB[q][3] = __fadd_ru(u.x, shhi[0]); bB[q][4] = __fadd_ru(u.y, shhi[1]); bB[q][5] = __fadd_ru(u.z, shhi[2]);
          }
          bool any = false;
#pragma unroll
          for (int q = 0; q < 4; ++q) {
            float4 l = ca[2 * q], u = ca[2 * q + 1];
            float bA[6] = {l.x, l.y, l.z, u.x, u.y, u.z};
#pragma unroll
            for (int w = 0; w < 4; ++w) any = any || fbox_hit(bA, bB[w]);
          }
          hit = any;
        }
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
  int pp_mult = h->tune[STIV_TUNE_PATCH_BLOCKS] > 0 ? h->tune[STIV_TUNE_PATCH_BLOCKS] : 4;
  if (blocks > pp_mult * num_sms) blocks = pp_mult * num_sms;
  if (blocks < 1) blocks = 1;
  int mp = stiv_npatches(2 * p_max);
  size_t psmem = (size_t)4 * 2 * mp * 6 * sizeof(float) + (size_t)4 * 2 * mp * sizeof(unsigned short);
  STIV_CUDA(h, cudaFuncSetAttribute(patch_pairs_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)psmem));
  {
    STIV_PROF(h, st, "patch_pairs");
    patch_pairs_kernel<<<blocks, 128, psmem, st>>>(p_dev, w.vbox, w.pbox, L[0], L[1], L[2], cand->i, cand->j,
                                                   cand->shift, cand->capacity, w.W, w.work, w.ctr, mp, w.vorg,
                                                   voff, w.pinfo, h->prm.d_m);
  }
  STIV_LAUNCH(h);
  narrow_args a;
  bool mixed = h->prm.precision == STIV_MIXED;
  a.pv = p_dev; a.voff = voff; a.X = X; a.mixed = mixed;
  a.pinfo = w.pinfo;
  a.L[0] = L[0]; a.L[1] = L[1]; a.L[2] = L[2];
  a.ci = cand->i; a.cj = cand->j; a.cs = cand->shift;
  a.work = w.work; a.W = w.W; a.include_ee = h->prm.include_ee; a.exact_only = w.exact_only;
  a.dm = h->prm.d_m;
  a.nlevel = h->tune[STIV_TUNE_PIECE_LEVELS] > 0 ? h->tune[STIV_TUNE_PIECE_LEVELS] : 2;
  if (a.nlevel > NLEVEL) a.nlevel = NLEVEL;
  if (a.nlevel < 1) a.nlevel = 1;
  a.vorg = w.vorg; a.fprep = w.fprep; a.fstride = w.fstride;
  a.q3 = w.q3; a.q2 = w.q2; a.Q3 = w.Q3; a.Q2 = w.Q2;
  a.C = w.C;
  a.rc_pair = w.tmp_i32; a.rc_type = w.tmp_i32 + w.C; a.rc_a = w.tmp_i32 + 2 * w.C; a.rc_b = w.tmp_i32 + 3 * w.C;
  a.rc_tau = w.tmp_f64; a.rc_w = w.tmp_f64 + w.C;
  a.ctr = w.ctr;
  // d_m > 0: widened boxes and the degree-six test, in kernels of their own
  bool dmk = h->prm.d_m > 0.0;
  size_t smem = stiv_narrow_smem();
  auto nk = mixed ? (dmk ? narrow_kernel<true, true> : narrow_kernel<true, false>)
                  : (dmk ? narrow_kernel<false, true> : narrow_kernel<false, false>);
  STIV_CUDA(h, cudaFuncSetAttribute(nk, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  int per_sm = 0;
  STIV_CUDA(h, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, nk, NW * 32, smem));
  if (h->tune[STIV_TUNE_NARROW_CTAS] > 0 && h->tune[STIV_TUNE_NARROW_CTAS] < per_sm) per_sm = h->tune[STIV_TUNE_NARROW_CTAS];
  if (per_sm < 1) per_sm = 1;
  {
    STIV_PROF(h, st, "narrow");
    nk<<<per_sm * num_sms, NW * 32, smem, st>>>(a);
  }
  STIV_LAUNCH(h);
  if (!w.exact_only) {
    size_t psm2 = sizeof(PieceWarp) * PW;
    auto pk = dmk ? pieces_kernel<true> : pieces_kernel<false>;
    STIV_CUDA(h, cudaFuncSetAttribute(pk, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)psm2));
    int per_sm2 = 0;
    STIV_CUDA(h, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm2, pk, PW * 32, psm2));
    if (h->tune[STIV_TUNE_PIECES_CTAS] > 0 && h->tune[STIV_TUNE_PIECES_CTAS] < per_sm2)
      per_sm2 = h->tune[STIV_TUNE_PIECES_CTAS];
    if (per_sm2 < 1) per_sm2 = 1;
    STIV_PROF(h, st, "pieces");
    pk<<<per_sm2 * num_sms, PW * 32, psm2, st>>>(a);
  }
  STIV_LAUNCH(h);
  {
    STIV_PROF(h, st, "fp64");
    auto fk = mixed ? (dmk ? fp64_kernel<true, true> : fp64_kernel<true, false>)
                    : (dmk ? fp64_kernel<false, true> : fp64_kernel<false, false>);
    int fm = h->tune[STIV_TUNE_FP64_BLOCKS] > 0 ? h->tune[STIV_TUNE_FP64_BLOCKS] : 16;
    fk<<<num_sms * fm, 128, 0, st>>>(a);
  }
  STIV_LAUNCH(h);
  return STIV_OK;
}

/*
 * libstiv: contact detection and space-time interference volumes (STIV) of
 * vesicle meshes on one GPU.
 *
 * Method: Lu, Rahimian & Zorin, "Parallel contact-aware simulations of
 * deformable particles in 3D Stokes flow" (arXiv 1812.04719):
 *   - each vesicle surface is a spherical-harmonic (SH) series of order p
 *     (Sec. 3.1.1), upsampled to order P = 2p and triangulated (Sec. 3.1.2,
 *     Fig. 3) at the start (X0, time t_n) and end (X1, time t_{n+1}) of a step;
 *   - candidate vesicle pairs come from space-time bounding boxes sorted on a
 *     Morton-ordered grid (Sec. 3.3.1, Alg. 1);
 *   - each vertex-triangle (and edge-edge) pair gets its earliest contact time
 *     from the coplanarity equation (Eq. 3.1, d_m = 0) under linear motion;
 *   - each contact gets the volume of Eq. 3.2 (App. A) and its gradient with
 *     respect to X1 (Sec. 3.1.2, Sec. 3.3.2), summed per vesicle pair (Alg. 2).
 *
 * Conventions for every entry point:
 *   - Array pointers are DEVICE pointers owned by the caller; the library never
 *     frees them and keeps none of them after the call returns.
 *   - Every call is asynchronous on the given CUDA stream (a cudaStream_t
 *     passed as void*, NULL = legacy default stream).  Counts are written to
 *     device memory; stiv_sync_counts copies them to the host.
 *   - The return value is a status: STIV_OK, or STIV_ERR_* for a bad argument
 *     or a CUDA launch/allocation failure.  Nothing traps or aborts.  Errors
 *     found by the kernels themselves (capacity overflow, invalid periodic
 *     box, non-finite input) are flags in counts[STIV_C_STATUS].
 *   - Scratch memory is owned by the handle (grown on demand with cudaMalloc).
 *
 * Layouts (N = number of vesicles, p_v = SH order of vesicle v, P_v = 2 p_v):
 *   coef:  per vesicle [2 time][3 coord][(p_v+1)^2] doubles at coef_off[v];
 *          real orthonormal SH without Condon-Shortley phase, entry n^2+n+m,
 *          m > 0 ~ cos(m phi), m < 0 ~ sin(|m| phi).
 *   verts: per vesicle [2 time][3 coord][n_v(P_v)] at vert_off[v] (elements),
 *          n_v(P) = 2P(P+1) + 2; doubles (STIV_FP64) or floats (STIV_MIXED).
 *          Vertex i*2P + j sits at polar angle arccos(x_i) (x_i the Gauss-
 *          Legendre nodes of order P+1, descending) and longitude 2 pi j/(2P);
 *          vertex 2P(P+1) is the north pole, 2P(P+1)+1 the south pole.
 *   mesh:  triangles and edges of stiv_mesh_topology; triangle ids and edge
 *          ids in the contact records refer to them.
 */
#ifndef STIV_H
#define STIV_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum stiv_status {
  STIV_OK = 0,
  STIV_ERR_ARG = 1,       /* bad argument (null pointer, size out of range) */
  STIV_ERR_CAPACITY = 2,  /* an output buffer was too small (counts say how big) */
  STIV_ERR_TIMEOUT = 3,   /* a bounded device wait gave up */
  STIV_ERR_CUDA = 4,      /* a CUDA call failed (see stiv_last_cuda_error) */
  STIV_ERR_INPUT = 5      /* kernels flagged the input (see counts[STIV_C_STATUS]) */
};

enum stiv_precision {
  STIV_FP64 = 0,   /* FP64 synthesis and vertices; FP64 contact arithmetic */
  STIV_MIXED = 1   /* FP32 synthesis and vertices; FP64 contact arithmetic */
};

/* Entries of the device counts array (int64, STIV_NCOUNTS entries). */
enum stiv_count {
  STIV_C_PAIRS = 0,    /* candidate vesicle pairs (i < j, image shift)        */
  STIV_C_PRIM = 1,     /* primitive pairs whose exact swept boxes overlap     */
  STIV_C_VF = 2,       /* vertex-triangle contacts                            */
  STIV_C_EE = 3,       /* edge-edge contacts                                  */
  STIV_C_CPAIRS = 4,   /* vesicle pairs with at least one contact             */
  STIV_C_DEGEN = 5,    /* primitive pairs skipped as degenerate               */
  STIV_C_STATUS = 6,   /* bit flags STIV_F_*                                  */
  STIV_C_PATCH = 7,    /* patch pairs examined by the narrow phase            */
  STIV_C_FLOPS = 8,    /* FP64 flops executed by the exact contact tests      */
  STIV_C_EXACT = 9,    /* primitive pairs that ran the FP64 contact test      */
  STIV_C_PIECE = 10,   /* primitive pairs the FP32 piece test examined        */
  STIV_NCOUNTS = 11
};

enum stiv_flag {
  STIV_F_PAIRS_OVERFLOW = 1,     /* candidate pairs exceeded stiv_pairs.capacity */
  STIV_F_CONTACTS_OVERFLOW = 2,  /* contacts exceeded stiv_contacts.capacity    */
  STIV_F_BOX_TOO_SMALL = 4,      /* a vesicle box spans >= L/2 on a periodic axis */
  STIV_F_NONFINITE = 8,          /* a vertex coordinate is NaN or infinite      */
  STIV_F_WORK_OVERFLOW = 16,     /* internal work list overflow (re-run)         */
  STIV_F_TIMEOUT = 32,           /* a bounded device wait gave up (mixed-form synthesis) */
  STIV_F_BAD_ORDER = 64          /* a vesicle's p_dev entry lies outside [1, p_max]: that
                                    vesicle is left out of synthesis, boxes and contacts */
};

typedef struct stiv_params {
  double d_m;          /* minimum separation; pads the vesicle boxes (Alg. 2 getBoundingBox) */
  double eps;          /* epsilon of the space-time metric (App. A), units of velocity */
  double dt;           /* time step Delta t; V depends on eps and dt only via eps*dt */
  double box_L[3];     /* periodic box lengths; 0 = free space on that axis */
  int32_t precision;   /* enum stiv_precision */
  int32_t include_ee;  /* 1: edge-edge contacts as well as vertex-triangle ones */
  int32_t exact_only;  /* 1: skip the certified FP32 rejection and run the FP64 contact
                          test on every primitive pair whose boxes overlap (same results,
                          slower; for cross-checks) */
  int32_t velocity;    /* enum stiv_velocity: the reading of U_k in Eq. 3.2 */
} stiv_params;

/* U_k in Eq. 3.2.  RELATIVE (default): the velocity of the contact point
 * relative to the opposite primitive (VF: D_p - sum beta_i D_i; EE:
 * D_q(u) - D_p(s)), Galilean-invariant.  ABSOLUTE: the literal reading, the
 * contact point's own velocity (VF: D_p; EE: D_p(s), the point on the first
 * edge).  Detection does not depend on it. */
enum stiv_velocity { STIV_VEL_RELATIVE = 0, STIV_VEL_ABSOLUTE = 1 };

/* Candidate vesicle pairs (Alg. 1 output, i < j), sorted by (i, j, shift).
 * shift = 9 (sx+1) + 3 (sy+1) + (sz+1): vesicle j is taken at X + s * box_L. */
typedef struct stiv_pairs {
  int64_t capacity;
  int32_t* i;
  int32_t* j;
  int32_t* shift;
} stiv_pairs;

/* Contacts (one record per primitive pair with a contact time in [0, 1]),
 * sorted by (pair, type, a, b).
 *   pair: index into the candidate pairs; type 0: vertex a of i vs triangle b
 *   of j; type 1: vertex a of j vs triangle b of i; type 2: edge a of i vs
 *   edge b of j.  tau: contact time in [0, 1] (fraction of the step).  w:
 *   [capacity][2], barycentric weights (beta1, beta2) of the contact point in
 *   the triangle (type 0/1), or the edge parameters (s on edge a, u on edge b). */
typedef struct stiv_contacts {
  int64_t capacity;
  int32_t* pair;
  int32_t* type;
  int32_t* a;
  int32_t* b;
  double* tau;
  double* w;
} stiv_contacts;

typedef struct stiv_handle stiv_handle;

/* Create a handle.  Fails with STIV_ERR_ARG for a negative box length,
 * non-positive eps or dt, or an unknown precision. */
int stiv_create(stiv_handle** h, const stiv_params* prm);
int stiv_destroy(stiv_handle* h);

/* Human-readable name of a status code. */
const char* stiv_status_string(int status);
/* The last CUDA error code the handle saw (cudaError_t as int). */
int stiv_last_cuda_error(const stiv_handle* h);

/* Mesh topology of order P (2 <= P <= 64), Sec. 3.1.2 / Fig. 3: each grid quad
 * (i,j),(i+1,j),(i+1,j+1),(i,j+1) split along (i,j)-(i+1,j+1) into
 * [(i,j),(i+1,j),(i+1,j+1)] and [(i,j),(i+1,j+1),(i,j+1)] (ids 2(i*2P+j) and
 * +1), north fan [N,(0,j),(0,j+1)] (id 4P^2+j), south fan [S,(P,j+1),(P,j)]
 * (id 4P^2+2P+j), normals outward.  tri_dev: [4P^2+4P][3]; edge_dev:
 * [6P^2+6P][2], the undirected edges as (min, max) sorted ascending. */
int stiv_mesh_topology(int32_t P, int32_t* tri_dev, int32_t* edge_dev, void* stream);

/* Sec. 3.1.2 upsampling: evaluate each vesicle's order-p series for X0 and X1
 * on its order-2p mesh (grid and poles).  p_dev[v] in [1, p_max], p_max <= 32;
 * a vesicle whose p_dev entry lies outside [1, p_max] is skipped (its vertices
 * are not written; stiv_detect then flags it as STIV_F_BAD_ORDER and leaves it
 * out of the boxes and contacts, stiv_mesh_fidelity reports NaN for it).
 * STIV_FP64: FP64 synthesis, doubles in verts_dev.  STIV_MIXED: the synthesis
 * runs on the tensor cores as one contraction per order with 3xTF32 split
 * products accumulated in FP32 (the degree-0 term added in the epilogue) and
 * writes floats; the handle keeps per-order tables and scratch (allocated on
 * the first call with a given n_ves and p_max).  A bounded wait that gives up
 * sets STIV_F_TIMEOUT in the next stiv_detect's counts. */
int stiv_upsample(stiv_handle* h, void* stream, int32_t n_ves, int32_t p_max, const int32_t* p_dev,
                  const int64_t* coef_off_dev, const double* coef_dev,
                  const int64_t* vert_off_dev, void* verts_dev);

/* Alg. 2's detection part without the distribution steps: vesicle space-time boxes,
 * candidate pairs (Alg. 1: Morton-grid sort and bbiCheck), then every
 * vertex-triangle pair (both directions) and edge-edge pair of each candidate
 * whose swept boxes overlap is tested with Eq. 3.1 (d_m = 0).  cand and out
 * are filled; counts_dev gets STIV_NCOUNTS int64 entries.  A periodic axis
 * requires every vesicle box to span less than half the box length. */
int stiv_detect(stiv_handle* h, void* stream, int32_t n_ves, int32_t p_max, const int32_t* p_dev,
                const int64_t* vert_off_dev, const void* verts_dev,
                const stiv_pairs* cand, const stiv_contacts* out, int64_t* counts_dev);

/* Eq. 3.2: V_k of every contact and the per-pair sums V_pair[r] (0 for a
 * candidate pair without contact).  V_contact_dev: [out->capacity];
 * V_pair_dev: [cand->capacity].  Either may be NULL. */
int stiv_stiv(stiv_handle* h, void* stream, int32_t n_ves, const int32_t* p_dev,
              const int64_t* vert_off_dev, const void* verts_dev, const stiv_pairs* cand,
              const stiv_contacts* contacts, const int64_t* counts_dev,
              double* V_contact_dev, double* V_pair_dev);

/* Eq. 3.2 and its gradient with respect to X1 (X0 fixed), through the contact
 * time (implicit function of Eq. 3.1) and the inside-test weights.  Per
 * contact k: grad_dev[k][4][3], and for each of the 4 points its vesicle
 * (g_ves_dev[k][4]) and local vertex id (g_vid_dev[k][4]).  Row r of the
 * Jacobian J = dV/dX1 (Sec. 3.2, Eq. 3.5-3.7) is the sum of the rows of the
 * contacts with pair == r. */
int stiv_stiv_grad(stiv_handle* h, void* stream, int32_t n_ves, const int32_t* p_dev,
                   const int64_t* vert_off_dev, const void* verts_dev, const stiv_pairs* cand,
                   const stiv_contacts* contacts, const int64_t* counts_dev,
                   double* V_contact_dev, double* V_pair_dev,
                   double* grad_dev, int32_t* g_ves_dev, int32_t* g_vid_dev);

/* dV_k/dX0 per contact (the start-of-step positions, X1 fixed): the same
 * layout and point order as the rows of stiv_stiv_grad (whose g_ves, g_vid
 * apply), [k][4][3].  With Y = X0 + tau (X1 - X0) and tau following
 * f(tau; X0) = 0, the rows satisfy dV/dX0 + dV/dX1 = 0 summed over the four
 * points (a rigid translation of both time levels leaves V unchanged). */
int stiv_stiv_grad_x0(stiv_handle* h, void* stream, int32_t n_ves, const int32_t* p_dev,
                      const int64_t* vert_off_dev, const void* verts_dev, const stiv_pairs* cand,
                      const stiv_contacts* contacts, const int64_t* counts_dev, double* grad_x0_dev);

/* Scatter-add per-contact gradient rows, each scaled by weight_pair[pair] (or
 * 1 if weight_pair is NULL), into a dense array in the vertex layout (only the
 * X1 block of each vesicle is written; the caller zeroes gX_dev). */
int stiv_grad_scatter(stiv_handle* h, void* stream, const int32_t* p_dev, const stiv_contacts* contacts,
                      const int64_t* counts_dev, const double* weight_pair_dev,
                      const double* grad_dev, const int32_t* g_ves_dev, const int32_t* g_vid_dev,
                      const int64_t* vert_off_dev, double* gX_dev);

/* Adjoint of the upsampling: gcoef = S^T gX for the X1 block of every vesicle
 * (S the synthesis matrix of stiv_upsample, grid and poles).  gX_dev in the
 * FP64 vertex layout; gcoef_dev in the coefficient layout (the X0 block is
 * set to zero).  STIV_FP64: FP64.  STIV_MIXED: on the tensor cores like the
 * mixed synthesis (3xTF32 split products, FP32 accumulation, FP64 output);
 * the first call with a given n_ves and p_max allocates scratch in the
 * handle. */
int stiv_grad_to_coef(stiv_handle* h, void* stream, int32_t n_ves, int32_t p_max, const int32_t* p_dev,
                      const int64_t* coef_off_dev, const int64_t* vert_off_dev,
                      const double* gX_dev, double* gcoef_dev);

/* Mesh fidelity (Sec. 3.1.2; Fig. 6): how far each vesicle's order-2p
 * triangle mesh (verts_dev as written by stiv_upsample, FP64 or FP32 per the
 * handle's precision) lies from its smooth order-p surface (coef_dev),
 * ||X^{q^up} - X(phi, theta)||_inf, estimated on the order-(factor 2p)
 * grid: its Gauss-Legendre rings and factor x 2 x 2p longitudes, poles
 * excluded.  The mesh is read as a map from parameter space: on the cell
 * [theta_i, theta_{i+1}] x [phi_j, phi_{j+1}] with fractions a (theta), b
 * (phi) it is the triangle (i,j), (i+1,j), (i+1,j+1) for a >= b and (i,j),
 * (i+1,j+1), (i,j+1) for a < b; beyond the first and last rings, the pole
 * fans.  err_dev [n_ves][2] (device, caller-owned) gets, per vesicle and time
 * level (X0, X1), the largest Euclidean distance between mesh and series at
 * those points; the paper asks for err < alpha d_m.  factor in [1, 8] (the
 * paper's estimate uses 4).  FP64 evaluation.  Returns STIV_ERR_ARG for a
 * NULL array or a parameter out of range. */
int stiv_mesh_fidelity(stiv_handle* h, void* stream, int32_t n_ves, int32_t p_max, const int32_t* p_dev,
                       const int64_t* coef_off_dev, const double* coef_dev, const int64_t* vert_off_dev,
                       const void* verts_dev, int32_t factor, double* err_dev);

/* The whole per-step path: upsample + detect + stiv_grad.  With use_graph = 1
 * the launches are captured into a CUDA graph on the first call and replayed
 * on later calls with the same arguments.  coef_dev = NULL skips the
 * upsampling: verts_dev then holds the input vertices (in the layout
 * stiv_upsample writes) and coef_off_dev is not read. */
int stiv_step(stiv_handle* h, void* stream, int32_t use_graph, int32_t n_ves, int32_t p_max,
              const int32_t* p_dev, const int64_t* coef_off_dev, const double* coef_dev,
              const int64_t* vert_off_dev, void* verts_dev, const stiv_pairs* cand,
              const stiv_contacts* out, int64_t* counts_dev, double* V_contact_dev,
              double* V_pair_dev, double* grad_dev, int32_t* g_ves_dev, int32_t* g_vid_dev);

/* Per-kernel timing with CUDA events recorded on the launching stream around
 * every kernel (or kernel group) the library launches.  Inside a captured
 * stiv_step graph the events are event-record nodes, re-recorded by each
 * replay.  stiv_profile_read waits for the recorded events and writes, per
 * stage name (32-byte NUL-terminated entries of names), the number of kernel
 * launches and the summed milliseconds, and sets *n_names; eager records are
 * then cleared, graph records are kept for the next replay (read once per
 * replay).  Stage names: synth, boxes, cells, sort_cells, cell_pairs,
 * sort_pairs, unique_pairs, patch_pairs, narrow, contact_order, finalize,
 * stiv, stiv_grad, vpair, grad_scatter, grad_to_coef. */
int stiv_profile(stiv_handle* h, int32_t enable);
int stiv_profile_read(stiv_handle* h, int32_t max_names, char* names, int64_t* launches, double* total_ms,
                      int32_t* n_names);

/* Wait for the stream, copy the counts to the host and return STIV_ERR_CAPACITY
 * if an overflow flag is set, STIV_ERR_INPUT for an input flag, else STIV_OK. */
int stiv_sync_counts(void* stream, const int64_t* counts_dev, int64_t* counts_host);

/* Contact LCP (Sec. 3.2, Eq. 3.7; Sec. 3.3.3, Alg. 3):
 *     0 <= q + B lambda  perp  lambda >= 0,   q = -V,  B = J M J^T,
 * one row per contact volume: each candidate pair (i, j, shift) with
 * contacts, in candidate-pair order; V its volume (V_pair of stiv_stiv_grad,
 * >= 0 for interference; the paper's constraint volume has the opposite sign,
 * which B does not see); J = dV/dX1, the gradient rows of stiv_stiv_grad
 * summed per vertex; M block-diagonal, a stand-in for the locally implicit
 * scheme's A^-1 G with its block structure: per vesicle i,
 * M_ii = m_i I + t_i (1 1^T (x) I_3), a local part plus a rigid translation
 * of the whole vesicle (m_ves_dev NULL: m_i = 1; t_ves_dev NULL: t_i = 0), so
 * B(j, k) = sum over vesicles i common to volumes j and k of
 * m_i g_j|i . g_k|i + t_i (sum g_j|i) . (sum g_k|i).  Entries are stored for
 * every pair of volumes that share a vesicle (a value may be 0), CSR with
 * columns ascending; B is symmetric bit for bit and positive semidefinite.
 * Caller-owned device arrays: */
typedef struct {
  int64_t row_capacity;   /* rows (contact volumes) the arrays hold              */
  int64_t nnz_capacity;   /* nonzeros of B the arrays hold                       */
  int32_t* row_pair;      /* [row_capacity] candidate-pair index of each row      */
  double* q;              /* [row_capacity] -V of each row                        */
  int64_t* row_ptr;       /* [row_capacity + 1]                                   */
  int32_t* col;           /* [nnz_capacity]                                       */
  double* val;            /* [nnz_capacity]                                       */
  int64_t* dims;          /* [8]: rows, nonzeros, status (1 rows over capacity, 2
                             nonzeros over capacity), internal counts             */
} stiv_lcp;
/* Forms B (Alg. 3) and q from the outputs of stiv_detect (cand, contacts,
 * counts) and stiv_stiv_grad (V_pair, grad, g_ves, g_vid) of the same step,
 * all on the device (m_ves_dev, t_ves_dev: [n_ves] or NULL).  Entries are
 * deterministic (every sum in a fixed order).  Scratch is handle-owned,
 * allocated on the first call with given capacities.  Returns STIV_ERR_ARG
 * for a NULL array or a capacity outside [1, 2^30); rows or nonzeros beyond
 * the capacities are not an error of the call: dims[2] reports them (after
 * the stream reaches the call), the arrays then hold the first row_capacity
 * rows and nnz_capacity nonzeros, and stiv_lcp_solve refuses the matrix. */
int stiv_lcp_matrix(stiv_handle* h, void* stream, int32_t n_ves, int32_t p_max, const stiv_pairs* cand,
                    const stiv_contacts* contacts, const int64_t* counts_dev, const double* V_pair_dev,
                    const double* grad_dev, const int32_t* g_ves_dev, const int32_t* g_vid_dev,
                    const double* m_ves_dev, const double* t_ves_dev, const stiv_lcp* lcp);
/* Minimum-map Newton method (Sec. 3.3.3) for the LCP above: Phi(lambda) =
 * min(lambda, q + B lambda); per Newton step the active set is
 * {q + B lambda < lambda}, the direction is -lambda off it and on it solves
 * the Newton system by a Jacobi-preconditioned conjugate gradient in FP32 to
 * a relative residual of 1e-6 (at most max_cg steps; an inexact Newton
 * method); Phi, the merit |Phi|^2 / 2 and its Armijo line search are FP64;
 * at most max_newton steps, stop when max |Phi| <= tol (FP64).  lambda_dev
 * [row_capacity] gets the multipliers; info_dev [4]: Newton steps, max |Phi|,
 * CG steps, status (0 converged, 1 matrix over capacity, 2 not converged).
 * One CTA (B and the vectors in its shared memory when they fit);
 * asynchronous.  Returns STIV_ERR_ARG for a NULL array, tol <= 0 or a
 * non-positive limit or capacity. */
int stiv_lcp_solve(stiv_handle* h, void* stream, const stiv_lcp* lcp, double tol, int32_t max_newton,
                   int32_t max_cg, double* lambda_dev, double* info_dev);

/* Launch-shape autotuner (not a step of the method: it changes how the
 * narrow phase's kernels are launched and how deep the certified FP32 piece
 * test refines before handing a pair to the FP64 test, never what the
 * detection returns).  Runs
 * stiv_detect on the given inputs (same arguments) under candidate launch
 * shapes, coordinate descent over the STIV_TUNE_* parameters, timing each
 * with CUDA events (the call synchronises the stream), and keeps the fastest
 * in the handle for later stiv_detect / stiv_step calls (a captured
 * stiv_step graph is re-captured).  choice_out (host, may be NULL) gets the
 * STIV_NTUNE chosen values; best_ms_out (host, may be NULL) the best time.
 * Outputs (cand, out, counts) hold the last run's results, identical for
 * every launch shape. */
enum stiv_tune_param {
  STIV_TUNE_NARROW_CTAS = 0,   /* narrow-kernel CTAs per SM (<= occupancy limit)  */
  STIV_TUNE_PIECES_CTAS = 1,   /* piece-test CTAs per SM                          */
  STIV_TUNE_FP64_BLOCKS = 2,   /* FP64 contact-test blocks per SM                 */
  STIV_TUNE_PATCH_BLOCKS = 3,  /* patch-pair blocks per SM                        */
  STIV_TUNE_PIECE_LEVELS = 4,  /* refinement levels of the FP32 piece test (2-6)  */
  STIV_NTUNE = 5
};
int stiv_autotune(stiv_handle* h, void* stream, int32_t n_ves, int32_t p_max, const int32_t* p_dev,
                  const int64_t* vert_off_dev, const void* verts_dev, const stiv_pairs* cand,
                  const stiv_contacts* out, int64_t* counts_dev, int32_t* choice_out, double* best_ms_out);
/* Set the STIV_NTUNE launch-shape values directly (host array; 0 = default;
 * STIV_TUNE_PIECE_LEVELS in [1, 6]); STIV_ERR_ARG for a value out of range. */
int stiv_set_tuning(stiv_handle* h, const int32_t* values);

/* Check of the bounded device waits (not a step of the method): one thread
 * waits on a shared-memory barrier that nothing completes, giving up after
 * limit_cycles SM clocks (0 <= limit_cycles <= the bound the tensor-core
 * synthesis uses, about a second at 2 GHz), and writes *status_dev = 1 when
 * it gave up, 0 otherwise.  The wait returns by itself; the context stays
 * usable.  STIV_ERR_ARG for a limit out of range. */
int stiv_wait_selftest(void* stream, int64_t limit_cycles, int32_t* status_dev);

/* Arithmetic-rate probe (not a step of the method; the paper has no
 * counterpart): the measured denominator of the FP64 and FP32 rooflines that
 * the benchmark reports.  Launches, on the current device, 8 blocks of 256
 * threads per SM; each thread runs 8 independent fused multiply-add chains of
 * `iters` steps in FP64 (kind 0) or FP32 (kind 1).  *flops_out (host) is set
 * to the operations the launch performs, 2 * 8 * iters * threads; time the
 * launch with events on `stream` to get the rate.  sink_dev: one device
 * double the kernel may write (it never does for the built-in constants; the
 * write only keeps the chains alive).  STIV_ERR_ARG for kind outside {0, 1},
 * iters outside [1, 2^32] or a null pointer. */
int stiv_peak_probe(void* stream, int32_t kind, int64_t iters, double* sink_dev, double* flops_out);

/* Stable LSD radix sort of (key, value) pairs on the low key_bits bits of the
 * 64-bit keys (Alg. 1's check-point sort, on one GPU).  scratch:
 * at least stiv_sort_scratch_bytes(n) bytes of device memory. */
size_t stiv_sort_scratch_bytes(int64_t n);
int stiv_sort_pairs(void* stream, int64_t n, int32_t key_bits, const uint64_t* keys_in,
                    const int32_t* vals_in, uint64_t* keys_out, int32_t* vals_out,
                    void* scratch, size_t scratch_bytes);

/* Allocation-free stiv_sort_pairs (the paper has no counterpart: this is an
 * interface for callers, not part of the method).  For callers that cannot
 * hand the library a scratch buffer or let it call cudaMalloc: code running
 * under another framework's device memory pool that owns all device memory,
 * latency-bound loops where cudaMalloc/cudaFree could synchronise the device,
 * or processes at their allocation limit.  Same sort and same result as
 * stiv_sort_pairs; its scratch is a fixed static device array inside the
 * library (about 13.6 MB, held on every GPU that loads the library until the
 * process exits).
 *   - n <= STIV_SORT_STATIC_MAX, else STIV_ERR_ARG (nothing is launched);
 *   - keys_in/vals_in are left intact; keys_out/vals_out receive the result;
 *   - calls no cudaMalloc, cudaFree or allocating library routine;
 *   - every call looks up the array's device address on the current device
 *     (cudaGetSymbolAddress); the first call on a device also makes the
 *     runtime load the library's device code there, so make that first call
 *     before any stream capture on the device;
 *   - all calls on a device share the one array, which keeps the previous
 *     call's contents: calls that overlap on the GPU (different streams, or
 *     concurrent host threads) race and must be serialised by the caller. */
#define STIV_SORT_STATIC_MAX (1 << 20)
int stiv_sort_pairs_static(void* stream, int64_t n, int32_t key_bits, const uint64_t* keys_in,
                           const int32_t* vals_in, uint64_t* keys_out, int32_t* vals_out);

#ifdef __cplusplus
}
#endif

#endif /* STIV_H */

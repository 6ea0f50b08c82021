// C-ABI entry points of libstiv: handle, scratch, mesh topology, the detect
// pipeline (Alg. 2) and the captured per-step graph.
#include "stiv_internal.cuh"

#include <stdlib.h>
#include <string.h>

#include <string>
#include <vector>

int stiv_broad_phase(stiv_handle* h, cudaStream_t st, int n, int p_max, const int32_t* p_dev, const int64_t* voff,
                     const void* X, const stiv_pairs* cand, detect_ws& w, int64_t* ctr);
int stiv_narrow_phase(stiv_handle* h, cudaStream_t st, const int32_t* p_dev, const int64_t* voff, const void* X,
                      const stiv_pairs* cand, detect_ws& w, int num_sms, int p_max);
int stiv_contact_order(stiv_handle* h, cudaStream_t st, const stiv_pairs* cand, const stiv_contacts* out,
                       detect_ws& w);

namespace {

__global__ void topology_kernel(int P, int32_t* tri, int32_t* edge) {
  int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k < stiv_ntris(P)) {
    int v[3];
    stiv_tri_verts(P, k, v);
    tri[3 * k] = v[0]; tri[3 * k + 1] = v[1]; tri[3 * k + 2] = v[2];
  }
  if (k < 2 * P * (P + 1)) {  // grid vertex k writes its forward edges
    int nb[5];
    int n = stiv_forward_nbrs(P, k, nb);
    int e0 = stiv_first_edge(P, k);
    for (int q = 0; q < n; ++q) { edge[2 * (e0 + q)] = k; edge[2 * (e0 + q) + 1] = nb[q]; }
  }
}

__global__ void finalize_kernel(int64_t* ctr, int64_t C, int64_t* counts, int* tc_status) {
  if (threadIdx.x == 0) {
    if (ctr[11] > C) ctr[STIV_C_STATUS] |= STIV_F_CONTACTS_OVERFLOW;
    if (tc_status && *tc_status) { ctr[STIV_C_STATUS] |= STIV_F_TIMEOUT; *tc_status = 0; }
    for (int k = 0; k < 8; ++k) counts[k] = ctr[k];
    counts[STIV_C_FLOPS] = ctr[12];
    counts[STIV_C_EXACT] = ctr[13];
    counts[STIV_C_PIECE] = ctr[14];
  }
}

inline size_t align_up(size_t x) { return (x + 255) & ~(size_t)255; }

}  // namespace

// ---------------------------------------------------------------------------
// per-kernel CUDA-event profiler
// ---------------------------------------------------------------------------
struct stiv_profiler {
  struct rec { std::string name; int nk; cudaEvent_t b, e; bool in_graph; bool valid; };
  std::vector<rec> recs;
  std::vector<cudaEvent_t> pool;
  std::vector<int> open;   // indices of stages begun but not ended
  cudaEvent_t get() {
    if (!pool.empty()) { cudaEvent_t ev = pool.back(); pool.pop_back(); return ev; }
    cudaEvent_t ev = nullptr;
    cudaEventCreate(&ev);
    return ev;
  }
};

static bool capturing(cudaStream_t st) {
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(st, &cs) != cudaSuccess) return false;
  return cs == cudaStreamCaptureStatusActive;
}

// While a stream is being captured the events become event-record nodes of
// the graph (re-recorded by every replay); otherwise plain records.
static void prof_record(cudaEvent_t ev, cudaStream_t st, bool graph) {
  if (graph) cudaEventRecordWithFlags(ev, st, cudaEventRecordExternal);
  else cudaEventRecord(ev, st);
}

void stiv_prof_begin(stiv_handle* h, cudaStream_t st, const char* name, int nk) {
  if (!h || !h->prof) return;
  stiv_profiler* P = (stiv_profiler*)h->prof;
  bool g = capturing(st);
  stiv_profiler::rec r{name, nk, P->get(), P->get(), g, !g};
  prof_record(r.b, st, g);
  P->recs.push_back(r);
  P->open.push_back((int)P->recs.size() - 1);
}

void stiv_prof_end(stiv_handle* h, cudaStream_t st) {
  if (!h || !h->prof) return;
  stiv_profiler* P = (stiv_profiler*)h->prof;
  if (P->open.empty()) return;
  int k = P->open.back();
  P->open.pop_back();
  prof_record(P->recs[k].e, st, P->recs[k].in_graph);
}

// Forget the records owned by a graph that is being destroyed.
void stiv_prof_drop_graph(stiv_handle* h) {
  if (!h || !h->prof) return;
  stiv_profiler* P = (stiv_profiler*)h->prof;
  std::vector<stiv_profiler::rec> keep;
  for (auto& r : P->recs) {
    if (r.in_graph) { P->pool.push_back(r.b); P->pool.push_back(r.e); }
    else keep.push_back(r);
  }
  P->recs.swap(keep);
}

extern "C" int stiv_profile(stiv_handle* h, int32_t enable) {
  if (!h) return STIV_ERR_ARG;
  if (enable && !h->prof) h->prof = new stiv_profiler();
  if (!enable && h->prof) {
    stiv_profiler* P = (stiv_profiler*)h->prof;
    cudaDeviceSynchronize();
    if (h->graph_exec) { cudaGraphExecDestroy(h->graph_exec); h->graph_exec = nullptr; h->graph_key = 0; }
    for (auto& r : P->recs) { cudaEventDestroy(r.b); cudaEventDestroy(r.e); }
    for (auto ev : P->pool) cudaEventDestroy(ev);
    delete P;
    h->prof = nullptr;
  }
  return STIV_OK;
}

extern "C" int stiv_profile_read(stiv_handle* h, int32_t max_names, char* names, int64_t* launches,
                                 double* total_ms, int32_t* n_names) {
  if (!h || !h->prof || !n_names || max_names < 0) return STIV_ERR_ARG;
  stiv_profiler* P = (stiv_profiler*)h->prof;
  std::vector<std::string> keys;
  std::vector<int64_t> cnt;
  std::vector<double> tot;
  std::vector<stiv_profiler::rec> keep;
  for (auto& r : P->recs) {
    if (!r.valid) { keep.push_back(r); continue; }   // captured but not replayed yet
    if (cudaEventSynchronize(r.e) != cudaSuccess) return STIV_ERR_CUDA;
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, r.b, r.e) != cudaSuccess) return STIV_ERR_CUDA;
    size_t k = 0;
    while (k < keys.size() && keys[k] != r.name) ++k;
    if (k == keys.size()) { keys.push_back(r.name); cnt.push_back(0); tot.push_back(0.0); }
    cnt[k] += r.nk; tot[k] += ms;
    if (r.in_graph) keep.push_back(r);
    else { P->pool.push_back(r.b); P->pool.push_back(r.e); }
  }
  P->recs.swap(keep);
  *n_names = (int32_t)keys.size();
  for (size_t k = 0; k < keys.size() && (int)k < max_names; ++k) {
    if (names) { strncpy(names + 32 * k, keys[k].c_str(), 31); names[32 * k + 31] = 0; }
    if (launches) launches[k] = cnt[k];
    if (total_ms) total_ms[k] = tot[k];
  }
  return STIV_OK;
}

extern "C" const char* stiv_status_string(int s) {
  switch (s) {
    case STIV_OK: return "ok";
    case STIV_ERR_ARG: return "invalid argument";
    case STIV_ERR_CAPACITY: return "output capacity exceeded";
    case STIV_ERR_TIMEOUT: return "device wait timed out";
    case STIV_ERR_CUDA: return "CUDA error";
    case STIV_ERR_INPUT: return "invalid input flagged by the kernels";
    default: return "unknown status";
  }
}

extern "C" int stiv_last_cuda_error(const stiv_handle* h) { return h ? h->last_cuda_error : 0; }

extern "C" int stiv_create(stiv_handle** out, const stiv_params* prm) {
  if (!out || !prm) return STIV_ERR_ARG;
  *out = nullptr;
  for (int c = 0; c < 3; ++c) if (!(prm->box_L[c] >= 0.0)) return STIV_ERR_ARG;
  if (!(prm->eps > 0.0) || !(prm->dt > 0.0) || !(prm->d_m >= 0.0)) return STIV_ERR_ARG;
  if (prm->precision != STIV_FP64 && prm->precision != STIV_MIXED) return STIV_ERR_ARG;
  if (prm->velocity != STIV_VEL_RELATIVE && prm->velocity != STIV_VEL_ABSOLUTE) return STIV_ERR_ARG;
  stiv_handle* h = (stiv_handle*)calloc(1, sizeof(stiv_handle));
  if (!h) return STIV_ERR_ARG;
  h->prm = *prm;
  cudaError_t e = cudaGetDevice(&h->device);
  if (e != cudaSuccess) { free(h); return STIV_ERR_CUDA; }
  *out = h;
  return STIV_OK;
}

extern "C" int stiv_destroy(stiv_handle* h) {
  if (!h) return STIV_ERR_ARG;
  for (int p = 0; p <= STIV_MAX_P; ++p) {
    if (h->tab_ready[p]) { cudaFree(h->tab[p].leg); cudaFree(h->tab[p].trig); cudaFree(h->tab[p].theta); }
    if (h->ytab[p]) cudaFree(h->ytab[p]);
    if (h->ytabT[p]) cudaFree(h->ytabT[p]);
  }
  if (h->tc_ws) cudaFree(h->tc_ws);
  if (h->tc_ws2) cudaFree(h->tc_ws2);
  if (h->tc_status) cudaFree(h->tc_status);
  if (h->lcp_ws) cudaFree(h->lcp_ws);
  if (h->lcp_ws2) cudaFree(h->lcp_ws2);
  if (h->fid_x) cudaFree(h->fid_x);
  if (h->graph_exec) cudaGraphExecDestroy(h->graph_exec);
  if (h->ws) cudaFree(h->ws);
  stiv_profile(h, 0);
  free(h);
  return STIV_OK;
}

int stiv_ws_reserve(stiv_handle* h, size_t bytes) {
  if (bytes <= h->ws_bytes) return STIV_OK;
  if (h->ws) { STIV_CUDA(h, cudaFree(h->ws)); h->ws = nullptr; h->ws_bytes = 0; }
  size_t nb = bytes + bytes / 4;
  STIV_CUDA(h, cudaMalloc(&h->ws, nb));
  h->ws_bytes = nb;
  return STIV_OK;
}

extern "C" int stiv_mesh_topology(int32_t P, int32_t* tri_dev, int32_t* edge_dev, void* stream) {
  if (P < 2 || P > STIV_MAX_PP || !tri_dev || !edge_dev) return STIV_ERR_ARG;
  int n = stiv_ntris(P);
  topology_kernel<<<(n + 255) / 256, 256, 0, (cudaStream_t)stream>>>(P, tri_dev, edge_dev);
  if (cudaGetLastError() != cudaSuccess) return STIV_ERR_CUDA;
  return STIV_OK;
}

// Scratch of stiv_detect, carved from the handle's buffer.
static int detect_layout(stiv_handle* h, int n, int p_max, const stiv_pairs* cand, const stiv_contacts* out,
                         detect_ws& w, bool carve) {
  w.R = (int64_t)n * 64 + 1024;
  w.Q = cand->capacity * 8 + 1024;
  w.W = cand->capacity * 64 + 1024;
  if (w.W < out->capacity) w.W = out->capacity;
  w.C = out->capacity > 0 ? out->capacity : 1;
  w.Q3 = 16 * w.C + 4096;
  w.Q2 = (h->prm.exact_only || h->prm.d_m > 0.0 ? 32 : 4) * w.C + 4096;
  int64_t smax = w.R > w.Q ? w.R : w.Q;
  if (w.C > smax) smax = w.C;
  w.sort_scratch_bytes = stiv_sort_scratch_impl(smax);
  size_t off = 0;
  size_t o_vbox = off; off = align_up(off + sizeof(double) * 6 * (size_t)n);
  w.pstride = stiv_npatches(2 * p_max);
  size_t o_pbox = off; off = align_up(off + sizeof(float) * STIV_PBOX * (size_t)w.pstride * n);
  w.fstride = 8 * (int64_t)stiv_nverts(2 * p_max);
  size_t o_vorg = off; off = align_up(off + sizeof(float) * 4 * (size_t)n);
  size_t o_fprep = off; off = align_up(off + sizeof(float) * (size_t)w.fstride * n);
  size_t o_grid = off; off = align_up(off + sizeof(double) * 16);
  size_t o_cc = off; off = align_up(off + sizeof(int32_t) * (size_t)(n + 1));
  size_t o_co = off; off = align_up(off + sizeof(int32_t) * (size_t)(n + 1));
  size_t o_rk = off; off = align_up(off + sizeof(uint64_t) * (size_t)w.R);
  size_t o_rv = off; off = align_up(off + sizeof(int32_t) * (size_t)w.R);
  size_t o_rk2 = off; off = align_up(off + sizeof(uint64_t) * (size_t)w.R);
  size_t o_rv2 = off; off = align_up(off + sizeof(int32_t) * (size_t)w.R);
  size_t o_rb = off; off = align_up(off + sizeof(int32_t) * (size_t)w.R);
  size_t o_rc = off; off = align_up(off + sizeof(int32_t) * (size_t)w.R);
  size_t o_pk = off; off = align_up(off + sizeof(uint64_t) * (size_t)w.Q);
  size_t o_pv = off; off = align_up(off + sizeof(int32_t) * (size_t)w.Q);
  size_t o_pk2 = off; off = align_up(off + sizeof(uint64_t) * (size_t)w.Q);
  size_t o_pv2 = off; off = align_up(off + sizeof(int32_t) * (size_t)w.Q);
  size_t o_wk = off; off = align_up(off + sizeof(uint64_t) * (size_t)w.W);
  size_t o_fr = off; off = align_up(off + sizeof(stiv_pair_info) * (size_t)cand->capacity);
  size_t o_q3 = off; off = align_up(off + sizeof(ulonglong2) * (size_t)w.Q3);
  size_t o_q2 = off; off = align_up(off + sizeof(ulonglong2) * (size_t)w.Q2);
  size_t o_pc = off; off = align_up(off + sizeof(int32_t) * (size_t)cand->capacity);
  size_t o_pf = off; off = align_up(off + sizeof(int32_t) * (size_t)cand->capacity);
  size_t o_po = off; off = align_up(off + sizeof(int32_t) * (size_t)(cand->capacity + 1));
  size_t o_sg = off; off = align_up(off + sizeof(uint64_t) * (size_t)w.C);
  size_t o_sg2 = off; off = align_up(off + sizeof(uint64_t) * (size_t)w.C);
  size_t o_ti = off; off = align_up(off + sizeof(int32_t) * 4 * (size_t)w.C);
  size_t o_tf = off; off = align_up(off + sizeof(double) * 3 * (size_t)w.C);
  size_t o_ctr = off; off = align_up(off + sizeof(int64_t) * 32);
  size_t o_ss = off; off = align_up(off + w.sort_scratch_bytes);
  if (!carve) return stiv_ws_reserve(h, off);
  char* b = (char*)h->ws;
  w.vbox = (double*)(b + o_vbox); w.pbox = (float*)(b + o_pbox); w.grid = (double*)(b + o_grid);
  w.vorg = (float*)(b + o_vorg); w.fprep = (float*)(b + o_fprep);
  w.exact_only = h->prm.exact_only;
  w.cell_count = (int32_t*)(b + o_cc); w.cell_off = (int32_t*)(b + o_co);
  w.rec_key = (uint64_t*)(b + o_rk); w.rec_val = (int32_t*)(b + o_rv);
  w.rec_key2 = (uint64_t*)(b + o_rk2); w.rec_val2 = (int32_t*)(b + o_rv2);
  w.rec_box = (int32_t*)(b + o_rb); w.rec_cell = (int32_t*)(b + o_rc);
  w.pkey = (uint64_t*)(b + o_pk); w.pval = (int32_t*)(b + o_pv);
  w.pkey2 = (uint64_t*)(b + o_pk2); w.pval2 = (int32_t*)(b + o_pv2);
  w.work = (uint64_t*)(b + o_wk);
  w.q3 = (ulonglong2*)(b + o_q3); w.q2 = (ulonglong2*)(b + o_q2);
  w.pinfo = (stiv_pair_info*)(b + o_fr);
  w.pair_cnt = (int32_t*)(b + o_pc); w.pair_fill = (int32_t*)(b + o_pf); w.pair_off = (int32_t*)(b + o_po);
  w.seg = (unsigned long long*)(b + o_sg); w.seg2 = (unsigned long long*)(b + o_sg2);
  w.tmp_i32 = (int32_t*)(b + o_ti); w.tmp_f64 = (double*)(b + o_tf);
  w.ctr = (int64_t*)(b + o_ctr);
  w.sort_scratch = b + o_ss;
  return STIV_OK;
}

extern "C" int stiv_detect(stiv_handle* h, void* stream, int32_t n_ves, int32_t p_max, const int32_t* p_dev,
                           const int64_t* vert_off_dev, const void* verts_dev, const stiv_pairs* cand,
                           const stiv_contacts* out, int64_t* counts_dev) {
  if (!h || n_ves < 0 || p_max < 1 || p_max > STIV_MAX_P || !cand || !out || !counts_dev) return STIV_ERR_ARG;
  if (cand->capacity < 1 || out->capacity < 1) return STIV_ERR_ARG;
  if (!cand->i || !cand->j || !cand->shift || !out->pair || !out->type || !out->a || !out->b || !out->tau || !out->w)
    return STIV_ERR_ARG;
  if (cand->capacity >= ((int64_t)1 << 31) || out->capacity >= ((int64_t)1 << 31) || n_ves >= (1 << 24))
    return STIV_ERR_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  if (n_ves < 2) {
    STIV_CUDA(h, cudaMemsetAsync(counts_dev, 0, sizeof(int64_t) * STIV_NCOUNTS, st));
    return STIV_OK;
  }
  if (!p_dev || !vert_off_dev || !verts_dev) return STIV_ERR_ARG;
  detect_ws w;
  int rc = detect_layout(h, n_ves, p_max, cand, out, w, false);
  if (rc) return rc;
  detect_layout(h, n_ves, p_max, cand, out, w, true);
  STIV_CUDA(h, cudaMemsetAsync(w.ctr, 0, sizeof(int64_t) * 32, st));
  STIV_CUDA(h, cudaMemsetAsync(w.pair_cnt, 0, sizeof(int32_t) * (size_t)cand->capacity, st));
  STIV_CUDA(h, cudaMemsetAsync(w.pair_fill, 0, sizeof(int32_t) * (size_t)cand->capacity, st));
  int sms = 152;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, h->device);
  rc = stiv_broad_phase(h, st, n_ves, p_max, p_dev, vert_off_dev, verts_dev, cand, w, w.ctr);
  if (rc) return rc;
  rc = stiv_narrow_phase(h, st, p_dev, vert_off_dev, verts_dev, cand, w, sms, p_max);
  if (rc) return rc;
  rc = stiv_contact_order(h, st, cand, out, w);
  if (rc) return rc;
  STIV_PROF(h, st, "finalize");
  finalize_kernel<<<1, 32, 0, st>>>(w.ctr, w.C, counts_dev, h->tc_status);
  STIV_LAUNCH(h);
  return STIV_OK;
}

extern "C" int stiv_autotune(stiv_handle* h, void* stream, int32_t n_ves, int32_t p_max, const int32_t* p_dev,
                             const int64_t* vert_off_dev, const void* verts_dev, const stiv_pairs* cand,
                             const stiv_contacts* out, int64_t* counts_dev, int32_t* choice_out,
                             double* best_ms_out) {
  if (!h || !counts_dev) return STIV_ERR_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  static const int32_t cands[STIV_NTUNE][4] = {{2, 3, 4, 0}, {1, 2, 3, 4}, {4, 8, 16, 32}, {2, 4, 8, 0}, {2, 3, 4, 0}};
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  STIV_CUDA(h, cudaEventCreate(&e0));
  STIV_CUDA(h, cudaEventCreate(&e1));
  int64_t host_counts[STIV_NCOUNTS];
  // one timed run of the detection with the handle's current launch shapes
  auto timed = [&](float& ms) -> int {
    float best = 1e30f;
    for (int rep = 0; rep < 2; ++rep) {
      if (cudaEventRecord(e0, st) != cudaSuccess) return STIV_ERR_CUDA;
      int rc = stiv_detect(h, stream, n_ves, p_max, p_dev, vert_off_dev, verts_dev, cand, out, counts_dev);
      if (rc) return rc;
      if (cudaEventRecord(e1, st) != cudaSuccess) return STIV_ERR_CUDA;
      if (cudaEventSynchronize(e1) != cudaSuccess) return STIV_ERR_CUDA;
      float t = 0.f;
      cudaEventElapsedTime(&t, e0, e1);
      if (t < best) best = t;
    }
    ms = best;
    return stiv_sync_counts(stream, counts_dev, host_counts);
  };
  int32_t saved[STIV_NTUNE];
  for (int k = 0; k < STIV_NTUNE; ++k) saved[k] = h->tune[k];
  float best_ms = 0.f;
  int rc = timed(best_ms);   // warm-up with the current shapes (sizes the workspace)
  if (!rc) rc = timed(best_ms);
  for (int k = 0; k < STIV_NTUNE && !rc; ++k) {
    int32_t keep = h->tune[k];
    for (int c = 0; c < 4 && !rc; ++c) {
      if (cands[k][c] == 0 || cands[k][c] == keep) continue;
      h->tune[k] = cands[k][c];
      float ms = 0.f;
      rc = timed(ms);
      if (!rc && ms < best_ms) { best_ms = ms; keep = cands[k][c]; }
    }
    h->tune[k] = keep;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (rc) {
    for (int k = 0; k < STIV_NTUNE; ++k) h->tune[k] = saved[k];
    return rc;
  }
  if (h->graph_exec) { cudaGraphExecDestroy(h->graph_exec); h->graph_exec = nullptr; h->graph_key = 0; }
  stiv_prof_drop_graph(h);
  if (choice_out) for (int k = 0; k < STIV_NTUNE; ++k) choice_out[k] = h->tune[k];
  if (best_ms_out) *best_ms_out = best_ms;
  return STIV_OK;
}

extern "C" int stiv_set_tuning(stiv_handle* h, const int32_t* values) {
  if (!h || !values) return STIV_ERR_ARG;
  for (int k = 0; k < STIV_NTUNE; ++k)
    if (values[k] < 0 || values[k] > 64 || (k == STIV_TUNE_PIECE_LEVELS && values[k] > 6)) return STIV_ERR_ARG;
  for (int k = 0; k < STIV_NTUNE; ++k) h->tune[k] = values[k];
  if (h->graph_exec) { cudaGraphExecDestroy(h->graph_exec); h->graph_exec = nullptr; h->graph_key = 0; }
  stiv_prof_drop_graph(h);
  return STIV_OK;
}

extern "C" int stiv_sync_counts(void* stream, const int64_t* counts_dev, int64_t* counts_host) {
  if (!counts_dev || !counts_host) return STIV_ERR_ARG;
  if (cudaStreamSynchronize((cudaStream_t)stream) != cudaSuccess) return STIV_ERR_CUDA;
  if (cudaMemcpy(counts_host, counts_dev, sizeof(int64_t) * STIV_NCOUNTS, cudaMemcpyDeviceToHost) != cudaSuccess)
    return STIV_ERR_CUDA;
  int64_t f = counts_host[STIV_C_STATUS];
  if (f & (STIV_F_PAIRS_OVERFLOW | STIV_F_CONTACTS_OVERFLOW | STIV_F_WORK_OVERFLOW)) return STIV_ERR_CAPACITY;
  if (f & (STIV_F_BOX_TOO_SMALL | STIV_F_NONFINITE | STIV_F_BAD_ORDER)) return STIV_ERR_INPUT;
  if (f & STIV_F_TIMEOUT) return STIV_ERR_TIMEOUT;
  return STIV_OK;
}

static int step_eager(stiv_handle* h, void* stream, int32_t n_ves, int32_t p_max, const int32_t* p_dev,
                      const int64_t* coef_off_dev, const double* coef_dev, const int64_t* vert_off_dev,
                      void* verts_dev, const stiv_pairs* cand, const stiv_contacts* out, int64_t* counts_dev,
                      double* Vc, double* Vp, double* grad, int32_t* gves, int32_t* gvid) {
  int rc = STIV_OK;
  if (coef_dev) {   // NULL: the vertices are the input
    rc = stiv_upsample(h, stream, n_ves, p_max, p_dev, coef_off_dev, coef_dev, vert_off_dev, verts_dev);
    if (rc) return rc;
  }
  rc = stiv_detect(h, stream, n_ves, p_max, p_dev, vert_off_dev, verts_dev, cand, out, counts_dev);
  if (rc) return rc;
  if (grad)
    return stiv_stiv_grad(h, stream, n_ves, p_dev, vert_off_dev, verts_dev, cand, out, counts_dev, Vc, Vp, grad,
                          gves, gvid);
  return stiv_stiv(h, stream, n_ves, p_dev, vert_off_dev, verts_dev, cand, out, counts_dev, Vc, Vp);
}

extern "C" int stiv_step(stiv_handle* h, void* stream, int32_t use_graph, int32_t n_ves, int32_t p_max,
                         const int32_t* p_dev, const int64_t* coef_off_dev, const double* coef_dev,
                         const int64_t* vert_off_dev, void* verts_dev, const stiv_pairs* cand,
                         const stiv_contacts* out, int64_t* counts_dev, double* V_contact_dev, double* V_pair_dev,
                         double* grad_dev, int32_t* g_ves_dev, int32_t* g_vid_dev) {
  if (!h || !cand || !out) return STIV_ERR_ARG;
  if (!use_graph || !stream)
    return step_eager(h, stream, n_ves, p_max, p_dev, coef_off_dev, coef_dev, vert_off_dev, verts_dev, cand, out,
                      counts_dev, V_contact_dev, V_pair_dev, grad_dev, g_ves_dev, g_vid_dev);
  // key of everything the captured launches depend on
  unsigned long long key = 1469598103934665603ull;
  auto mix = [&](unsigned long long x) { key = (key ^ x) * 1099511628211ull; };
  const void* ptrs[] = {p_dev, coef_off_dev, coef_dev, vert_off_dev, verts_dev, cand->i, cand->j, cand->shift,
                        out->pair, out->type, out->a, out->b, out->tau, out->w, counts_dev, V_contact_dev,
                        V_pair_dev, grad_dev, g_ves_dev, g_vid_dev, stream};
  for (const void* p : ptrs) mix((unsigned long long)(uintptr_t)p);
  mix((unsigned long long)n_ves); mix((unsigned long long)p_max);
  mix((unsigned long long)cand->capacity); mix((unsigned long long)out->capacity);
  if (h->graph_exec && key == h->graph_key) {
    STIV_CUDA(h, cudaGraphLaunch(h->graph_exec, (cudaStream_t)stream));
    if (h->prof)
      for (auto& r : ((stiv_profiler*)h->prof)->recs) if (r.in_graph) r.valid = true;
    return STIV_OK;
  }
  // first call with these arguments: run eagerly (allocates tables and scratch), then capture
  int rc = step_eager(h, stream, n_ves, p_max, p_dev, coef_off_dev, coef_dev, vert_off_dev, verts_dev, cand, out,
                      counts_dev, V_contact_dev, V_pair_dev, grad_dev, g_ves_dev, g_vid_dev);
  if (rc) return rc;
  if (h->graph_exec) { cudaGraphExecDestroy(h->graph_exec); h->graph_exec = nullptr; }
  stiv_prof_drop_graph(h);
  cudaStream_t st = (cudaStream_t)stream;
  STIV_CUDA(h, cudaStreamBeginCapture(st, cudaStreamCaptureModeRelaxed));
  void* ws_before = h->ws;
  rc = step_eager(h, stream, n_ves, p_max, p_dev, coef_off_dev, coef_dev, vert_off_dev, verts_dev, cand, out,
                  counts_dev, V_contact_dev, V_pair_dev, grad_dev, g_ves_dev, g_vid_dev);
  cudaGraph_t graph = nullptr;
  cudaError_t e = cudaStreamEndCapture(st, &graph);
  if (rc) { if (graph) cudaGraphDestroy(graph); return rc; }
  if (e != cudaSuccess || h->ws != ws_before) {
    if (graph) cudaGraphDestroy(graph);
    h->last_cuda_error = (int)e;
    return STIV_ERR_CUDA;
  }
  e = cudaGraphInstantiate(&h->graph_exec, graph, 0);
  cudaGraphDestroy(graph);
  if (e != cudaSuccess) { h->graph_exec = nullptr; h->last_cuda_error = (int)e; return STIV_ERR_CUDA; }
  h->graph_key = key;
  return STIV_OK;
}

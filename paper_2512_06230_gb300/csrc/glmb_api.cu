// C ABI of the multi-detection GLMB update (include/glmb.h): handle, device
// memory (allocated once at create), per-frame orchestration of the kernels
// on one stream, state import/export and inspection.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <string>
#include <unordered_map>
#include <vector>

#include "../../include/glmb.h"
#include "glmb_kernels.h"

using namespace glmb;

namespace {

constexpr unsigned long long kGolden = 0x9E3779B97F4A7C15ULL;

// stages timed by glmb_set_profiling
enum { kStagePredict = 0, kStageTable, kStageExpand, kStageSelect, kStageMat, kStageGc,
       kStageEstimates, kNumStages };

// device scalar slots
enum { S_ERR = 0, S_FP64 = 1, S_MAXT = 2, S_MAXK = 3, S_NUPD = 4, S_NKEEP = 5, S_K = 6, S_REDO = 7, S_STAGE = 8, S_KFULL = 9,
       S_N = 16 };

}  // namespace

namespace {
// launch sizes: eager (from the host-known sizes of this frame) or fixed by
// capacity (for a replayed graph)
struct Plan {
  bool fixed;
  int T, K, M;     // per-parent image plan: slots, gated pairs, detection rows
  bool thread;     // draws: one thread per child (many parents) or one warp per child
  bool smem;       // parents staged in shared memory (else in the image)
  int st_thr;      // threads per staging CTA
  int Gw, Gm;      // children per CTA of the warp kernel: expansion, regeneration
  int wg, mg;      // warps per child in them (1, 2, 4 or 8)
  int wc, mc;      // the part of wg, mg that follows the hypothesis count
};
}  // namespace

struct glmb_handle {
  glmb_config cfg{};
  Model md{};
  PartModel pm{};   // particle track model (md.particle)
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  std::string err;
  std::vector<void*> allocs;
  std::vector<void*> host_allocs;
  // capacities
  int cap_h = 0, cap_meas = 0, cap_births = 0, max_tracks = 0;
  long long cap_entries = 0, cap_comp = 0, cap_pairs = 0, cap_children = 0, cap_upd = 0;
  uint32_t hmask = 0;
  int smem_limit = 0, n_sm = 0, smem_per_sm = 0;
  // state (table A = comps[cur]) and working table (B)
  CompTable comps[2];
  int cur = 0;
  int n_comp = 0;
  HypTable hyps[2];
  int hcur = 0;
  int H = 1;
  long long n_entries = 0;
  int frame = 0;
  int stage = 0;            // 0 ready for predict, 1 predicted, 2 updated, 3 step in flight
  // last frame
  int nb = 0, T_work = 0, M = 0, H_par = 0, par_buf = 0, birth_base = 0;
  bool have_update = false, theta_M_valid = false, retained_valid = false;
  int theta_M = 0;
  double* d_births = nullptr;
  double* h_births = nullptr;
  float* d_Z = nullptr;
  const float* z_dev = nullptr;   // detections the kernels read: d_Z or the caller's device buffer
  float* h_Z = nullptr;
  PairTable pt{};
  // learned pair gate (glmb_set_gate): parameters on the device, the table
  // before the gate (PRUNE mode; shares logdetS with pt), per-pair keep flags
  // and logits of the last update, scratch of the training-data calls
  int gate_mode = 0, gate_mode_frame = 0;
  float gate_thr = 0.f;
  float* gate_params = nullptr;
  PairTable pt_full{};
  uint8_t* gate_keep = nullptr;
  float* gate_logit = nullptr;
  float* gate_X = nullptr;
  uint8_t* gate_used = nullptr;
  uint8_t* gate_hflag = nullptr;
  long long n_pairs_pregate = 0;
  uint32_t* scan_tmp32 = nullptr;
  long long scan_cap32 = 0;   // capacity scan_tmp32 was sized for
  long long* child_key = nullptr;
  unsigned long long* child_hash = nullptr;
  int8_t* child_status = nullptr;
  uint16_t* child_alive = nullptr;
  // per-parent images of the expansion (grown on demand) and the draws the
  // thread-per-child kernel hands to the warp kernel
  unsigned char* img = nullptr;
  size_t img_alloc = 0;
  uint32_t* redo_list = nullptr;
  PruneWork pw{};
  unsigned long long* hkeys = nullptr;
  uint32_t* hvals = nullptr;
  uint32_t* upd_src = nullptr;
  uint32_t* upd_slot = nullptr;   // update id -> hash slot
  unsigned* d_hprev = nullptr;     // updates the last materialisation inserted
  bool hash_dirty = false;         // a frame overflowed the update table: clear all of it
  uint32_t* upd_m = nullptr;
  long long* upd_se = nullptr;
  uint32_t* gc_flag = nullptr;
  uint32_t* gc_newpos = nullptr;
  // frame results, one device block copied back in one piece:
  // [scalars (S_N)][prune counters (8)][estimates], mirrored in pinned host
  // memory up to the end of the estimate records
  unsigned* d_scal = nullptr;
  unsigned* h_scal = nullptr;
  size_t res_off_cnt = 0, res_off_est = 0;
  // estimates: [nb (16 B)][pmf][tracks][done], mirrored on the host up to
  // est_off_end (the start of done); `done` holds the component bound and
  // the block counter of the existence sums, est_rcomp their per-component
  // sums followed by the per-track sums (all left zeroed by the kernels)
  unsigned char* d_est = nullptr;
  unsigned long long* est_rcomp = nullptr;
  unsigned char* h_est = nullptr;
  size_t est_off_pmf = 0, est_off_tr = 0, est_off_end = 0, est_off_done = 0;
  // state generation (bumped by every change of the filter state) and the
  // generation whose estimates h_est holds; glmb_step computes them in its
  // graph unless step_estimates is off
  long long gen = 0, est_gen = -1;
  bool step_estimates = true;
  unsigned launch_opts = 0;   // GLMB_OPT_* overrides
  glmb_tuning tune{4, 0, 16, 0};     // launch shapes (glmb_set_tuning)
  unsigned* h_cnt = nullptr;   // pinned copy of the prune counters
  double* d_ru = nullptr;
  // stage timing
  unsigned prof_mask = 0;
  cudaEvent_t ev[kNumStages][2] = {};
  bool ev_pending[kNumStages] = {};
  double stage_ms[kNumStages] = {};
  long long stage_calls[kNumStages] = {};
  // frame inputs, one device block [sizes][births][detections] that a frame
  // graph fills with one copy from its pinned image; the host block is
  // [sizes slot 0][the device block's image, whose sizes are slot 1]
  // (slot 0: glmb_predict, slot 1: glmb_update and glmb_step)
  size_t in_off_births = 0, in_off_Z = 0;
  FrameDev* d_fs = nullptr;
  FrameDev* h_fs = nullptr;
  // shared-memory plan of the expansion: exact slot maximum (from the last
  // prune), estimated pair maximum (from earlier frames; redone if exceeded)
  int alive_max = 0;
  int K_est = 256;
  int exp_smem = 0, exp_ctas = 0;
  int exp_plan[4] = {0, 0, 0, 0};   // T, K, M, threads of the last expansion
  int redo_count = 0;
  int lse_parts = 1;    // log-sum-exp partials the last expansion wrote
  // launch plan of the frame in progress, and captured frame graphs
  Plan plan{};
  // a kernel node of a captured graph that takes the frame's Philox key,
  // with the arguments it was captured with
  struct KeyNode {
    cudaGraphNode_t node;
    cudaKernelNodeParams p;
    ExpandArgs a;
  };
  struct CachedGraph {
    int hcur;
    unsigned prof;
    Plan plan;
    cudaGraphExec_t exec;
    long long n_kernels;
    int smem;              // shared memory per CTA of its expansion
    long long last_use;
    cudaGraph_t graph;     // kept while exec lives: its key nodes are set per replay
    std::vector<KeyNode> key_nodes;
  };
  std::vector<CachedGraph> graphs;
  bool capturing = false;
  long long n_captures = 0, n_graph_launches = 0;
  double capture_ms = 0.0;   // host time spent capturing and instantiating graphs
  // stats
  long long n_pairs = 0, n_unique = 0;
  int n_upd = 0, n_fp64 = 0;
  long long n_draw_overflow = 0;
  int T_max = 0, K_max = 0;
};

namespace {

// optional CUDA-event timing of the update's stages (glmb_set_profiling)
void prof_begin(glmb_handle* h, int st);
void prof_end(glmb_handle* h, int st);
void prof_collect(glmb_handle* h);

glmb_status fail(glmb_handle* h, glmb_status st, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  if (h) h->err = buf;
  return st;
}

void drop_graph(glmb_handle::CachedGraph& g) {
  cudaGraphExecDestroy(g.exec);
  if (g.graph) cudaGraphDestroy(g.graph);
  g.exec = nullptr;
  g.graph = nullptr;
}

#define CU(call)                                                                    \
  do {                                                                              \
    cudaError_t e_ = (call);                                                        \
    if (e_ != cudaSuccess)                                                          \
      return fail(h, GLMB_E_CUDA, "%s: %s", #call, cudaGetErrorString(e_));         \
  } while (0)

// device memory through the configured hook, else cudaMalloc / cudaFree
void* dev_alloc_raw(glmb_handle* h, size_t bytes) {
  if (h->cfg.dev_alloc) return h->cfg.dev_alloc(bytes, h->cfg.alloc_ctx);
  void* q = nullptr;
  if (cudaMalloc(&q, bytes) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  return q;
}

void dev_free_raw(glmb_handle* h, void* p) {
  if (!p) return;
  if (h->cfg.dev_alloc) h->cfg.dev_free(p, h->cfg.alloc_ctx);
  else cudaFree(p);
}

template <typename T>
bool dalloc(glmb_handle* h, T** p, long long n) {
  if (n <= 0) n = 1;
  void* q = dev_alloc_raw(h, (size_t)n * sizeof(T));
  if (!q) return false;
  // zero-filled, in the handle's stream order: no kernel ever reads
  // uninitialised memory, even a stale region of a frame being redone
  if (cudaMemsetAsync(q, 0, (size_t)n * sizeof(T), h->stream) != cudaSuccess) {
    dev_free_raw(h, q);
    return false;
  }
  h->allocs.push_back(q);
  *p = (T*)q;
  return true;
}

template <typename T>
bool halloc(glmb_handle* h, T** p, long long n) {
  void* q = nullptr;
  if (n <= 0) n = 1;
  if (cudaMallocHost(&q, (size_t)n * sizeof(T)) != cudaSuccess) return false;
  h->host_allocs.push_back(q);
  *p = (T*)q;
  return true;
}

bool alloc_comps(glmb_handle* h, CompTable& c, long long cap, int dx) {
  c.cap = (int)cap;
  c.px = nullptr;
  const int ncov = dx * (dx + 1) / 2;
  return dalloc(h, &c.mhi, cap * dx) && dalloc(h, &c.mlo, cap * dx) &&
         dalloc(h, &c.cov, cap * ncov) && dalloc(h, &c.lk, cap) && dalloc(h, &c.lb, cap) &&
         dalloc(h, &c.logp, cap) && dalloc(h, &c.log1mp, cap) &&
         (!h->md.particle || dalloc(h, &c.px, cap * 6 * (long long)h->pm.np));
}

bool alloc_hyps(glmb_handle* h, HypTable& y) {
  return dalloc(h, &y.ptr, h->cap_h + 1) && dalloc(h, &y.comp, h->cap_entries) &&
         dalloc(h, &y.logw, h->cap_h) && dalloc(h, &y.uid, h->cap_h) &&
         dalloc(h, &y.theta, (long long)h->cap_h * h->cap_meas);
}

void free_all(glmb_handle* h) {
  for (void* p : h->allocs) dev_free_raw(h, p);
  for (void* p : h->host_allocs) cudaFreeHost(p);
  h->allocs.clear();
  h->host_allocs.clear();
}

size_t round_up64(size_t x) { return (x + 63) / 64 * 64; }

// The frame's input and result blocks (layouts at their handle fields).
bool alloc_io(glmb_handle* h) {
  const size_t fs = sizeof(FrameDev);
  h->in_off_births = round_up64(fs);
  h->in_off_Z = h->in_off_births + round_up64((size_t)h->cap_births * kBirthRec * sizeof(double));
  const size_t in_bytes = h->in_off_Z + (size_t)h->cap_meas * h->md.dz * sizeof(float);
  unsigned char *din = nullptr, *hin = nullptr;
  if (!dalloc(h, &din, (long long)in_bytes) || !halloc(h, &hin, (long long)(fs + in_bytes))) return false;
  h->d_fs = reinterpret_cast<FrameDev*>(din);
  h->d_births = reinterpret_cast<double*>(din + h->in_off_births);
  h->d_Z = reinterpret_cast<float*>(din + h->in_off_Z);
  h->h_fs = reinterpret_cast<FrameDev*>(hin);
  h->h_births = reinterpret_cast<double*>(hin + fs + h->in_off_births);
  h->h_Z = reinterpret_cast<float*>(hin + fs + h->in_off_Z);

  const size_t pcap = (size_t)h->max_tracks + 1;
  h->est_off_pmf = 16;
  h->est_off_tr = h->est_off_pmf + 8 * pcap;
  h->est_off_end = h->est_off_tr + sizeof(glmb_track) * pcap;
  h->est_off_done = h->est_off_end;
  h->res_off_cnt = round_up64(S_N * sizeof(unsigned));
  h->res_off_est = h->res_off_cnt + 64;
  unsigned char *dres = nullptr, *hres = nullptr;
  if (!dalloc(h, &dres, (long long)(h->res_off_est + h->est_off_done + 16)) ||
      !halloc(h, &hres, (long long)(h->res_off_est + h->est_off_end)))
    return false;
  h->d_scal = reinterpret_cast<unsigned*>(dres);
  h->pw.counts = reinterpret_cast<unsigned*>(dres + h->res_off_cnt);
  h->d_est = dres + h->res_off_est;
  h->h_scal = reinterpret_cast<unsigned*>(hres);
  h->h_cnt = reinterpret_cast<unsigned*>(hres + h->res_off_cnt);
  h->h_est = hres + h->res_off_est;
  return true;
}

long long next_pow2(long long x) {
  long long p = 1;
  while (p < x) p <<= 1;
  return p;
}

bool spd_inverse(int n, const double* A, double* Ainv, double* logdet) {
  double L[9] = {0};
  for (int j = 0; j < n; ++j) {
    double s = A[j * n + j];
    for (int k = 0; k < j; ++k) s -= L[j * n + k] * L[j * n + k];
    if (!(s > 0)) return false;
    L[j * n + j] = std::sqrt(s);
    for (int i = j + 1; i < n; ++i) {
      double t = A[i * n + j];
      for (int k = 0; k < j; ++k) t -= L[i * n + k] * L[j * n + k];
      L[i * n + j] = t / L[j * n + j];
    }
  }
  *logdet = 0;
  for (int i = 0; i < n; ++i) *logdet += 2 * std::log(L[i * n + i]);
  for (int c = 0; c < n; ++c) {
    double y[3], x[3];
    for (int i = 0; i < n; ++i) {
      double s = (i == c);
      for (int k = 0; k < i; ++k) s -= L[i * n + k] * y[k];
      y[i] = s / L[i * n + i];
    }
    for (int i = n - 1; i >= 0; --i) {
      double s = y[i];
      for (int k = i + 1; k < n; ++k) s -= L[k * n + i] * x[k];
      x[i] = s / L[i * n + i];
    }
    for (int i = 0; i < n; ++i) Ainv[i * n + c] = x[i];
  }
  return true;
}


// every condition flagged in e, joined (a static buffer: the caller copies it)
const char* err_text(unsigned e) {
  static const struct { unsigned bit; const char* text; } kText[] = {
      {kErrPairs, "gated pairs exceed max_pairs"},
      {kErrSlots, "per-hypothesis staging exceeded its plan"},
      {kErrEntries, "hypothesis entries exceed h_max * max_tracks"},
      {kErrComps, "components exceed capacity"},
      {kErrUpdates, "distinct track updates exceed capacity"},
      {kErrHash, "update table full"},
      {kErrNumeric, "covariance not positive definite"},
      {kErrInput, "a detection is not finite"},
      {kErrGate, "learned gate: a tensor-core wait ran out of time"},
      {kErrTimeout, "a scan's look-back waited past its limit"},
      {kErrChkSurv, "internal check: a survivor index outside the frame's children"},
      {kErrChkComp, "internal check: a component index outside the working table"},
      {kErrChkRemap, "internal check: a new-hypothesis entry outside its tables"},
  };
  thread_local static char buf[512];
  buf[0] = 0;
  for (const auto& t : kText)
    if (e & t.bit) {
      if (buf[0]) std::strncat(buf, "; ", sizeof buf - std::strlen(buf) - 1);
      std::strncat(buf, t.text, sizeof buf - std::strlen(buf) - 1);
    }
  if (!buf[0]) std::snprintf(buf, sizeof buf, "device error 0x%x", e);
  return buf;
}

glmb_status set_initial(glmb_handle* h) {
  const uint32_t ptr0[2] = {0, 0};
  const double lw = 0.0;
  const unsigned long long uid = mix64(h->cfg.seed + kGolden);
  HypTable& y = h->hyps[h->hcur];
  CU(cudaMemcpyAsync(y.ptr, ptr0, sizeof ptr0, cudaMemcpyHostToDevice, h->stream));
  CU(cudaMemcpyAsync(y.logw, &lw, sizeof lw, cudaMemcpyHostToDevice, h->stream));
  CU(cudaMemcpyAsync(y.uid, &uid, sizeof uid, cudaMemcpyHostToDevice, h->stream));
  CU(cudaStreamSynchronize(h->stream));
  h->H = 1;
  h->n_entries = 0;
  h->n_comp = 0;
  h->frame = 0;
  h->stage = 0;
  h->alive_max = 0;
  h->K_est = 256;   // the planning state starts over with the filter
  h->have_update = false;
  h->theta_M_valid = false;
  return GLMB_OK;
}

void prof_begin(glmb_handle* h, int st) {
  if (!(h->prof_mask & (1u << st))) return;
  if (!h->ev[st][0]) {
    cudaEventCreate(&h->ev[st][0]);
    cudaEventCreate(&h->ev[st][1]);
  }
  // inside a graph capture the record becomes a node that fires on replay
  if (h->capturing) cudaEventRecordWithFlags(h->ev[st][0], h->stream, cudaEventRecordExternal);
  else cudaEventRecord(h->ev[st][0], h->stream);
}

void prof_end(glmb_handle* h, int st) {
  if (!(h->prof_mask & (1u << st)) || !h->ev[st][0]) return;
  if (h->capturing) {
    cudaEventRecordWithFlags(h->ev[st][1], h->stream, cudaEventRecordExternal);
    return;
  }
  cudaEventRecord(h->ev[st][1], h->stream);
  h->ev_pending[st] = true;
}

void prof_collect(glmb_handle* h) {
  for (int st = 0; st < kNumStages; ++st) {
    if (!h->ev_pending[st]) continue;
    float ms = 0.f;
    if (cudaEventSynchronize(h->ev[st][1]) == cudaSuccess &&
        cudaEventElapsedTime(&ms, h->ev[st][0], h->ev[st][1]) == cudaSuccess) {
      h->stage_ms[st] += ms;
      h->stage_calls[st] += 1;
    }
    h->ev_pending[st] = false;
  }
}

}  // namespace

extern "C" {

glmb_status glmb_set_launch_options(glmb_handle* h, unsigned opts) {
  if (!h) return GLMB_E_INVALID;
  if (opts & ~(GLMB_OPT_STAGE_GLOBAL | GLMB_OPT_DRAW_WARP | GLMB_OPT_DRAW_THREAD | GLMB_OPT_STAGE_SHARED |
               GLMB_OPT_STAGE_SCRATCH_ROWS | GLMB_OPT_STAGE_SCRATCH_NONE | GLMB_OPT_WARP_GROUPS))
    return fail(h, GLMB_E_INVALID, "set_launch_options: unknown option bits 0x%x", opts);
  if (opts != h->launch_opts) {
    cudaStreamSynchronize(h->stream);
    for (auto& g : h->graphs) drop_graph(g);
    h->graphs.clear();
  }
  h->launch_opts = opts;
  return GLMB_OK;
}

glmb_status glmb_set_wait_test(int mode, long long limit) {
  if (mode != 0 && mode != GLMB_WAIT_TEST_SCAN && mode != GLMB_WAIT_TEST_GATE) return GLMB_E_INVALID;
  if (mode != 0 && limit < 1) return GLMB_E_INVALID;
  set_wait_test(WaitTest{mode, mode ? limit : 0});
  return GLMB_OK;
}

glmb_status glmb_set_step_estimates(glmb_handle* h, int on) {
  if (!h) return GLMB_E_INVALID;
  if (h->step_estimates != (on != 0)) {
    // captured graphs were built with the other setting
    cudaStreamSynchronize(h->stream);
    for (auto& g : h->graphs) drop_graph(g);
    h->graphs.clear();
  }
  h->step_estimates = on != 0;
  return GLMB_OK;
}

glmb_status glmb_set_profiling(glmb_handle* h, unsigned stage_mask) {
  if (!h) return GLMB_E_INVALID;
  h->prof_mask = stage_mask;
  for (int st = 0; st < kNumStages; ++st) {
    h->stage_ms[st] = 0.0;
    h->stage_calls[st] = 0;
    h->ev_pending[st] = false;
    if ((stage_mask & (1u << st)) && !h->ev[st][0]) {
      CU(cudaEventCreate(&h->ev[st][0]));
      CU(cudaEventCreate(&h->ev[st][1]));
    }
  }
  return GLMB_OK;
}

glmb_status glmb_get_timing(glmb_handle* h, double* ms, long long* calls, int n) {
  if (!h || n < 0) return GLMB_E_INVALID;
  CU(cudaStreamSynchronize(h->stream));
  prof_collect(h);
  for (int st = 0; st < n; ++st) {
    if (ms) ms[st] = st < kNumStages ? h->stage_ms[st] : 0.0;
    if (calls) calls[st] = st < kNumStages ? h->stage_calls[st] : 0;
  }
  return GLMB_OK;
}

glmb_status glmb_create(const glmb_config* cfg, glmb_handle** out) {
  if (!cfg || !out) return GLMB_E_INVALID;
  *out = nullptr;
  const glmb_config& c = *cfg;
  if (c.model == 1) {
    if (!(c.dim_x == 5 && c.dim_z == 2 && c.score_mode == 1 && c.n_particles >= 1 && c.n_particles <= 4096 &&
          c.sigma_a >= 0 && c.sigma_w >= 0 && c.ess_frac >= 0 && c.ess_frac <= 1))
      return GLMB_E_INVALID;
  } else if (c.model != 0 || !((c.dim_x == 4 && c.dim_z == 2) || (c.dim_x == 6 && c.dim_z == 3))) {
    return GLMB_E_INVALID;
  }
  if (!(c.dt > 0) || !(c.q >= 0) || !(c.p_s >= 0 && c.p_s <= 1) || !(c.p_d >= 0 && c.p_d <= 1) ||
      !(c.lambda_d >= 0) || !(c.clutter_rate >= 0) || !(c.volume > 0) || !(c.gate > 0) ||
      c.h_max < 1 || c.h_up < 1 || c.h_up > 65535 || !(c.tau > 0) || c.score_mode < 0 || c.score_mode > 1)
    return GLMB_E_INVALID;
  if ((c.dev_alloc == nullptr) != (c.dev_free == nullptr)) return GLMB_E_INVALID;
  glmb_handle* h = new glmb_handle();
  h->cfg = c;
  const int dx = c.dim_x, dz = c.dim_z;
  h->cap_h = c.h_max;
  h->max_tracks = c.max_tracks > 0 ? c.max_tracks : 256;
  h->cap_meas = c.max_meas > 0 ? c.max_meas : 4096;
  h->cap_births = c.max_births > 0 ? c.max_births : 256;
  if (h->cap_meas > 65535 || h->max_tracks > 65535) {
    delete h;
    return GLMB_E_INVALID;
  }
  h->cap_entries = (long long)h->cap_h * h->max_tracks;
  h->cap_comp = c.max_components > 0 ? c.max_components : h->cap_entries + h->cap_births;
  h->cap_pairs = c.max_pairs > 0 ? c.max_pairs : 16 * h->cap_comp;
  h->cap_children = (long long)h->cap_h * c.h_up;
  h->cap_upd = std::min(h->cap_entries, h->cap_comp);
  const long long hcap = next_pow2(2 * h->cap_entries);
  h->hmask = (uint32_t)(hcap - 1);
  if (h->cap_comp >= (1LL << 31) || hcap > (1LL << 31) || h->cap_pairs >= (1LL << 32)) {
    delete h;
    return GLMB_E_INVALID;
  }

  // model constants (FP64 on the host, stored as FP32)
  Model& md = h->md;
  md.dx = dx;
  md.dz = dz;
  md.ncov = dx * (dx + 1) / 2;
  md.h_up = c.h_up;
  md.dt = c.dt;
  const double dt = c.dt;
  double Q[36] = {0};
  for (int a = 0; a < dz; ++a) {
    Q[a * dx + a] = c.q * dt * dt * dt / 3.0;
    Q[a * dx + dz + a] = c.q * dt * dt / 2.0;
    Q[(dz + a) * dx + a] = c.q * dt * dt / 2.0;
    Q[(dz + a) * dx + dz + a] = c.q * dt;
  }
  for (int i = 0; i < dx; ++i)
    for (int j = i; j < dx; ++j) md.Q[pidx(dx, i, j)] = (float)Q[i * dx + j];
  double Rinv[9], ldR;
  if (!spd_inverse(dz, c.R, Rinv, &ldR)) {
    delete h;
    return GLMB_E_INVALID;
  }
  for (int k = 0; k < dz * dz; ++k) {
    md.R[k] = (float)c.R[k];
    md.Rinv[k] = (float)Rinv[k];
  }
  md.logdetR = (float)ldR;
  md.log_pd = c.p_d > 0 ? (float)std::log(c.p_d) : -INFINITY;
  md.log_1mpd = c.p_d < 1 ? (float)std::log1p(-c.p_d) : -INFINITY;
  md.lambda_d = (float)c.lambda_d;
  md.log_lambda_d = c.lambda_d > 0 ? (float)std::log(c.lambda_d) : -INFINITY;
  const double kappa = c.clutter_rate / c.volume;
  md.kappa_zero = !(kappa > 0);
  md.score_mode = c.score_mode;
  md.log_kappa = md.kappa_zero ? -INFINITY : (float)std::log(kappa);
  md.fx_log_kappa = md.kappa_zero ? 0 : (long long)std::llrint((double)md.log_kappa * 4294967296.0);
  md.gate = std::isinf(c.gate) ? INFINITY : (float)c.gate;
  md.log_ps = c.p_s > 0 ? (float)std::log(c.p_s) : -INFINITY;
  md.log_1mps = c.p_s < 1 ? (float)std::log1p(-c.p_s) : -INFINITY;
  md.seed_lo = (uint32_t)c.seed;
  md.seed_hi = (uint32_t)(c.seed >> 32);
  md.particle = c.model == 1;
  if (md.particle) {
    PartModel& pm = h->pm;
    pm.np = c.n_particles;
    pm.dt = (double)c.dt;
    pm.sigma_a = c.sigma_a;
    pm.sigma_w = c.sigma_w;
    pm.ess_frac = c.ess_frac;
    for (int k = 0; k < 4; ++k) pm.Rinv[k] = Rinv[k];
    pm.lnorm = 0.5 * ldR + std::log(6.283185307179586476925);
    pm.log_pd = c.p_d > 0 ? std::log(c.p_d) : -INFINITY;
    pm.seed_lo = md.seed_lo;
    pm.seed_hi = md.seed_hi;
  }

  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) {
    delete h;
    return GLMB_E_CUDA;
  }
  cudaDeviceGetAttribute(&h->smem_limit, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  cudaDeviceGetAttribute(&h->smem_per_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
  cudaDeviceGetAttribute(&h->n_sm, cudaDevAttrMultiProcessorCount, dev);
  expand_init(h->smem_limit);
  if (c.stream) {
    h->stream = (cudaStream_t)c.stream;
  } else {
    if (cudaStreamCreateWithFlags(&h->stream, cudaStreamNonBlocking) != cudaSuccess) {
      delete h;
      return GLMB_E_CUDA;
    }
    h->own_stream = true;
  }
  const long long scan_n = std::max(h->cap_comp, h->cap_children);
  bool ok = alloc_comps(h, h->comps[0], h->cap_comp, dx) && alloc_comps(h, h->comps[1], h->cap_comp, dx) &&
            alloc_hyps(h, h->hyps[0]) && alloc_hyps(h, h->hyps[1]) &&
            alloc_io(h) && dalloc(h, &h->est_rcomp, h->cap_comp + h->max_tracks + 1) &&
            dalloc(h, &h->pt.cnt, h->cap_comp + 1) && dalloc(h, &h->pt.ptr, h->cap_comp + 1) &&
            dalloc(h, &h->pt.meas, h->cap_pairs) && dalloc(h, &h->pt.logC, h->cap_pairs) &&
            dalloc(h, &h->pt.q, h->cap_pairs) && dalloc(h, &h->pt.e, h->cap_pairs * dz) &&
            dalloc(h, &h->pt.dthr, h->cap_comp) && dalloc(h, &h->pt.dprob, h->cap_comp) &&
            dalloc(h, &h->pt.logdetS, h->cap_comp) &&
            dalloc(h, &h->scan_tmp32, scan_tmp_elems(scan_n)) &&
            dalloc(h, &h->child_key, h->cap_children) && dalloc(h, &h->child_status, h->cap_children) &&
            dalloc(h, &h->child_hash, h->cap_children) &&
            dalloc(h, &h->child_alive, h->cap_children) &&
            dalloc(h, &h->redo_list, h->cap_children) &&
            dalloc(h, &h->pw.blk_max, 4097) && dalloc(h, &h->pw.blk_sum, 4097) &&
            dalloc(h, &h->pw.blk_done, 4) && dalloc(h, &h->pw.lse, 2) && dalloc(h, &h->pw.thr, 1) &&
            dalloc(h, &h->pw.part_max, kMaxLseParts) && dalloc(h, &h->pw.part_sum, kMaxLseParts) &&
            dalloc(h, &h->pw.part_cnt, kMaxLseParts) &&
            dalloc(h, &h->pw.hist, 4096) && dalloc(h, &h->pw.sel, 4) &&
            dalloc(h, &h->pw.flags, h->cap_children) &&
            dalloc(h, &h->pw.flags_tmp, scan_tmp_elems(h->cap_children)) &&
            dalloc(h, &h->pw.surv_idx, h->cap_h) &&
            dalloc(h, &h->hkeys, hcap) && dalloc(h, &h->hvals, hcap) &&
            dalloc(h, &h->upd_src, h->cap_upd) && dalloc(h, &h->upd_m, h->cap_upd) &&
            dalloc(h, &h->upd_slot, h->cap_upd) && dalloc(h, &h->d_hprev, 1) &&
            dalloc(h, &h->upd_se, h->cap_upd * dz) && dalloc(h, &h->gc_flag, h->cap_comp) &&
            dalloc(h, &h->gc_newpos, h->cap_comp) && dalloc(h, &h->d_ru, h->cap_meas);
  if (ok) {
    h->pw.err = h->d_scal + S_ERR;
    h->pw.flags_tmp_cap = h->cap_children;
    h->scan_cap32 = scan_n;
    // scan work areas start zeroed (dalloc zero-fills them; each scan
    // leaves its own zeroed); every fill is ordered before the handle's work
    ok = cudaStreamSynchronize(h->stream) == cudaSuccess;
  }
  if (!ok) {
    free_all(h);
    if (h->own_stream) cudaStreamDestroy(h->stream);
    delete h;
    return GLMB_E_OOM;
  }
  h->pt.cap_pairs = h->cap_pairs;
  cudaMemsetAsync(h->pw.blk_done, 0, 4 * sizeof(unsigned), h->stream);
  cudaMemsetAsync(h->pw.hist, 0, 4096 * sizeof(unsigned), h->stream);
  if (set_initial(h) != GLMB_OK) {
    free_all(h);
    if (h->own_stream) cudaStreamDestroy(h->stream);
    delete h;
    return GLMB_E_CUDA;
  }
  *out = h;
  return GLMB_OK;
}

glmb_status glmb_destroy(glmb_handle* h) {
  if (!h) return GLMB_OK;
  cudaStreamSynchronize(h->stream);
  for (auto& g : h->graphs) drop_graph(g);
  dev_free_raw(h, h->img);
  dev_free_raw(h, h->pt.slm);
  dev_free_raw(h, h->pt.sln);
  for (int st = 0; st < kNumStages; ++st)
    if (h->ev[st][0]) {
      cudaEventDestroy(h->ev[st][0]);
      cudaEventDestroy(h->ev[st][1]);
    }
  free_all(h);
  if (h->own_stream) cudaStreamDestroy(h->stream);
  delete h;
  return GLMB_OK;
}

glmb_status glmb_reset(glmb_handle* h) {
  if (!h) return GLMB_E_INVALID;
  h->err.clear();
  ++h->gen;
  return set_initial(h);
}

const char* glmb_last_error(glmb_handle* h) { return h ? h->err.c_str() : "null handle"; }

namespace {

// validates and stages the births of a frame (host pinned buffer)
glmb_status stage_births(glmb_handle* h, const glmb_birth* births, int n_births) {
  if (n_births < 0 || (n_births > 0 && !births)) return fail(h, GLMB_E_INVALID, "predict: births");
  if (n_births > h->cap_births)
    return fail(h, GLMB_E_CAPACITY, "predict: %d births > max_births %d", n_births, h->cap_births);
  if ((long long)h->n_comp + n_births > h->cap_comp)
    return fail(h, GLMB_E_CAPACITY, "predict: components exceed capacity");
  const int dx = h->md.dx;
  for (int b = 0; b < n_births; ++b) {
    const glmb_birth& B = births[b];
    if (!(B.r >= 0 && B.r <= 1)) return fail(h, GLMB_E_INVALID, "predict: birth %d r", b);
    double* rec = h->h_births + (size_t)b * kBirthRec;
    rec[0] = B.r;
    for (int a = 0; a < 6; ++a) rec[1 + a] = a < dx ? B.mean[a] : 0.0;
    for (int k = 0; k < 36; ++k) rec[7 + k] = k < dx * dx ? B.cov[k] : 0.0;
    for (int k = 0; k < 1 + dx; ++k)
      if (!std::isfinite(rec[k])) return fail(h, GLMB_E_INVALID, "predict: birth %d not finite", b);
    for (int k = 0; k < dx * dx; ++k)
      if (!std::isfinite(rec[7 + k])) return fail(h, GLMB_E_INVALID, "predict: birth %d not finite", b);
    for (int k = kBirthChol; k < kBirthRec; ++k) rec[k] = 0.0;
    if (h->md.particle) {   // the particles are drawn through its Cholesky factor
      double L[25] = {0};
      for (int j = 0; j < 5; ++j) {
        double d = rec[7 + j * 5 + j];
        for (int k = 0; k < j; ++k) d -= L[j * 5 + k] * L[j * 5 + k];
        if (!(d > 0)) return fail(h, GLMB_E_INVALID, "predict: birth %d covariance not positive definite", b);
        L[j * 5 + j] = std::sqrt(d);
        for (int i = j + 1; i < 5; ++i) {
          double t = rec[7 + i * 5 + j];
          for (int k = 0; k < j; ++k) t -= L[i * 5 + k] * L[j * 5 + k];
          L[i * 5 + j] = t / L[j * 5 + j];
        }
      }
      for (int i = 0; i < 5; ++i)
        for (int j = 0; j <= i; ++j) rec[kBirthChol + i * (i + 1) / 2 + j] = L[i * 5 + j];
    }
  }
  return GLMB_OK;
}

// validates the detections: device ones are read in place by the kernels,
// host ones are staged in pinned memory and copied to d_Z (by this call,
// or by the frame graph when copy is false)
glmb_status stage_detections(glmb_handle* h, const float* Z, int M, int z_is_device, bool copy = true) {
  if (M < 0 || (M > 0 && !Z)) return fail(h, GLMB_E_INVALID, "update: detections");
  if (M > h->cap_meas) return fail(h, GLMB_E_CAPACITY, "update: M=%d > max_meas %d", M, h->cap_meas);
  const int dz = h->md.dz;
  h->z_dev = h->d_Z;
  if (M > 0 && !z_is_device)
    for (long long k = 0; k < (long long)M * dz; ++k)
      if (!std::isfinite(Z[k])) return fail(h, GLMB_E_INVALID, "update: non-finite detection");
  if (M > 0) {
    if (z_is_device) {
      // the kernels read device detections with global-memory loads: the
      // buffer must be device (or managed) memory of this handle's GPU,
      // 4-byte aligned
      cudaPointerAttributes pa{};
      int dev = -1;
      if (cudaPointerGetAttributes(&pa, Z) != cudaSuccess) {
        cudaGetLastError();
        return fail(h, GLMB_E_INVALID, "update: detections are not device memory");
      }
      CU(cudaGetDevice(&dev));
      if ((pa.type != cudaMemoryTypeDevice && pa.type != cudaMemoryTypeManaged) || pa.device != dev)
        return fail(h, GLMB_E_INVALID, "update: detections are not device memory of the handle's GPU");
      if ((reinterpret_cast<uintptr_t>(Z) & 3u) != 0u)
        return fail(h, GLMB_E_INVALID, "update: device detections not 4-byte aligned");
      h->z_dev = Z;
    } else {
      std::memcpy(h->h_Z, Z, (size_t)M * dz * sizeof(float));
      if (copy)
        CU(cudaMemcpyAsync(h->d_Z, h->h_Z, (size_t)M * dz * sizeof(float), cudaMemcpyHostToDevice, h->stream));
    }
  }
  return GLMB_OK;
}

// frame sizes to the device (pinned slot -> d_fs; by this call, or by the
// frame graph when copy is false)
glmb_status upload_sizes(glmb_handle* h, int slot, bool copy = true) {
  FrameDev& f = h->h_fs[slot];
  f = FrameDev{};
  f.n_comp = h->n_comp;
  f.nb = h->nb;
  f.T = h->T_work;
  f.M = h->M;
  f.H = h->H;
  f.frame = h->frame;
  f.Z = h->z_dev;
  if (copy) CU(cudaMemcpyAsync(h->d_fs, &f, sizeof f, cudaMemcpyHostToDevice, h->stream));
  return GLMB_OK;
}

int round_up(int x, int m) { return (x + m - 1) / m * m; }

glmb_status enqueue_predict(glmb_handle* h, const Plan& p) {
  const CompTable& A = h->comps[h->cur];
  const CompTable& B = h->comps[1 - h->cur];
  const int gp = p.fixed ? 2 * h->n_sm : std::max(1, std::min((h->T_work + 127) / 128, 8 * h->n_sm));
  prof_begin(h, kStagePredict);
  if (h->md.particle) {
    const int gpp = 4 * h->n_sm;
    launch_particle_predict(h->md, h->pm, A, B, h->d_fs, h->d_births, gpp, h->stream);
  } else {
    launch_predict(h->md, A, B, h->d_fs, h->d_births, gp, h->stream);
  }
  prof_end(h, kStagePredict);
  return GLMB_OK;
}

glmb_status enqueue_table(glmb_handle* h, const Plan& p) {
  const CompTable& B = h->comps[1 - h->cur];
  const int T = h->T_work, dz = h->md.dz;
  const long long cap = p.fixed ? h->cap_comp : std::max(T, 1);
  CU(cudaMemsetAsync(h->d_scal, 0, S_N * sizeof(unsigned), h->stream));
  prof_begin(h, kStageTable);
  const int gt = p.fixed ? 4 * h->n_sm : std::max(1, std::min((T * 32 + 255) / 256, 16 * h->n_sm));
  // with the gate pruning, the Mahalanobis-gated table goes to pt_full and
  // the gate compacts the pairs it keeps into pt
  const bool prune = h->gate_mode == GLMB_GATE_PRUNE;
  const PairTable& P0 = prune ? h->pt_full : h->pt;
  launch_table_count(h->md, B, P0, h->d_fs, h->d_scal + S_ERR, gt, h->stream);   // also checks Z is finite
  scan_u32(P0.cnt, P0.ptr, &h->d_fs->T, 1, cap, h->d_scal + (prune ? S_KFULL : S_K), true, h->scan_tmp32,
           h->scan_cap32, h->d_scal + S_ERR, h->stream);
  launch_table_write(h->md, B, P0, h->d_fs, h->d_scal + S_FP64, h->d_scal + S_ERR, gt,
                     h->stream);
  if (h->md.particle) launch_particle_logc(h->md, h->pm, B, P0, h->d_fs, gt, h->stream);
  if (h->gate_mode != GLMB_GATE_OFF) {
    launch_gate_forward_table(h->gate_params, h->gate_thr, h->md, B, P0, h->d_fs, h->gate_logit,
                              prune ? h->gate_keep : nullptr, h->d_scal + S_ERR, 2 * h->n_sm, h->stream);
    if (prune) {
      launch_gate_compact(h->md, B, P0, h->gate_keep, h->pt, h->d_fs, true, gt, h->stream);
      scan_u32(h->pt.cnt, h->pt.ptr, &h->d_fs->T, 1, cap, h->d_scal + S_K, true, h->scan_tmp32, h->scan_cap32,
               h->d_scal + S_ERR, h->stream);
      launch_gate_compact(h->md, B, P0, h->gate_keep, h->pt, h->d_fs, false, gt, h->stream);
    }
  }
  h->gate_mode_frame = h->gate_mode;
  // the largest slot and pair counts per parent are recorded by the
  // staging kernel (ExpandArgs::max_T / max_K)
  prof_end(h, kStageTable);
  return GLMB_OK;
}

ExpandArgs expand_args(glmb_handle* h, const Plan& p, bool mat) {
  ExpandArgs a{};
  a.md = h->md;
  a.ct = h->comps[1 - h->cur];
  a.pt = h->pt;
  a.parents = h->hyps[h->hcur];
  a.fs = h->d_fs;
  a.T_max = p.T;
  a.K_max = p.K;
  a.M_plan = p.M;
  a.img = h->img;
  a.img_stride = expand_image_bytes(h->md.dz, p.T, p.K, p.M);
  a.stage_smem = p.smem ? 1 : 0;
  a.warp_all = p.thread ? 0 : 1;
  a.redo_list = h->redo_list;
  a.redo_count = h->d_scal + S_REDO;
  a.stage_next = h->d_scal + S_STAGE;
  a.materialize = mat ? 1 : 0;
  a.err = h->d_scal + S_ERR;
  a.gc_flag = h->gc_flag;
  a.max_T = h->d_scal + S_MAXT;
  a.max_K = h->d_scal + S_MAXK;
  a.warp_group = 1;
  a.key_x = h->md.seed_lo;
  a.key_y = h->md.seed_hi ^ (uint32_t)h->frame;
  return a;
}

// the image buffer holds cap_h parents of plan p; growing it invalidates the
// captured graphs (they hold its address)
glmb_status ensure_img(glmb_handle* h, const Plan& p) {
  const size_t need = (size_t)h->cap_h * (size_t)expand_image_bytes(h->md.dz, p.T, p.K, p.M);
  if (need <= h->img_alloc) return GLMB_OK;
  CU(cudaStreamSynchronize(h->stream));
  for (auto& g : h->graphs) drop_graph(g);
  h->graphs.clear();
  dev_free_raw(h, h->img);
  h->img = nullptr;
  h->img_alloc = 0;
  const size_t want = need + need / 4;
  void* q = dev_alloc_raw(h, want);
  if (!q) return fail(h, GLMB_E_CAPACITY, "expansion images: %zu bytes not available", want);
  h->img = (unsigned char*)q;
  h->img_alloc = want;
  return GLMB_OK;
}

// the per-component table of m-only term parts holds the frame's working
// components (grown on demand, which drops the captured graphs: they hold
// its address).  Without room the terms are built per slot instead (the
// same values), so a failed allocation only costs time.
glmb_status ensure_slm(glmb_handle* h, long long need) {
  if (need <= h->pt.slm_cap || h->pt.slm_cap >= h->cap_comp) return GLMB_OK;
  const long long cap = std::min<long long>(h->cap_comp, ((need + need / 2 + 255) / 256) * 256);
  const int NP = h->md.dz * (h->md.dz + 1) / 2;
  CU(cudaStreamSynchronize(h->stream));
  for (auto& g : h->graphs) drop_graph(g);
  h->graphs.clear();
  dev_free_raw(h, h->pt.slm);
  dev_free_raw(h, h->pt.sln);
  h->pt.slm = (float*)dev_alloc_raw(h, (size_t)cap * kSlmM * (NP + 1) * sizeof(float));
  h->pt.sln = (int8_t*)dev_alloc_raw(h, (size_t)cap * kSlmM);
  h->pt.slm_cap = (h->pt.slm && h->pt.sln) ? (int)cap : 0;
  if (!h->pt.slm_cap) {
    dev_free_raw(h, h->pt.slm);
    dev_free_raw(h, h->pt.sln);
    h->pt.slm = nullptr;
    h->pt.sln = nullptr;
  }
  h->pt_full.slm = h->pt.slm;
  h->pt_full.sln = h->pt.sln;
  h->pt_full.slm_cap = h->pt.slm_cap;
  return GLMB_OK;
}

// scal_zeroed: the frame's table stage has just zeroed the scalar block
// (the redo counter and the staging counter with it)
glmb_status enqueue_expand(glmb_handle* h, const Plan& p, bool scal_zeroed = false) {
  cudaStream_t s = h->stream;
  const int n_sm = h->n_sm, h_up = h->cfg.h_up, dz = h->md.dz;
  ExpandArgs a = expand_args(h, p, false);
  a.child_key = h->child_key;
  a.child_hash = h->child_hash;
  a.child_status = h->child_status;
  a.child_alive = h->child_alive;
  const int img = (int)a.img_stride;
  // stage: CTAs of p.st_thr threads, each taking the next parent from a
  // counter (persistent grid)
  // staged in global memory: as much of its scratch in shared memory as fits
  a.stage_tail = 0;
  const int top = (h->launch_opts & GLMB_OPT_STAGE_SCRATCH_NONE)   ? 0
                  : (h->launch_opts & GLMB_OPT_STAGE_SCRATCH_ROWS) ? 1
                                                                   : 2;
  if (!p.smem)
    for (int m = top; m >= 1 && !a.stage_tail; --m)
      if (expand_stage_tail_bytes(dz, p.T, p.K, p.M, m) <= h->smem_limit) a.stage_tail = m;
  const int st_smem = (p.smem ? img : 0) + expand_stage_tail_bytes(dz, p.T, p.K, p.M, a.stage_tail);
  const int st_thr = p.st_thr;
  const int st_ctas = std::max(1, expand_occupancy(a, ExpandKernel::kStage, st_thr, st_smem));
  const int st_grid = p.fixed ? st_ctas * n_sm : std::max(1, std::min(h->H, st_ctas * n_sm));
  // draws: one thread per child over the frame's children in order
  // (persistent grid)
  // CTAs of 256 threads, or smaller ones when the frame's children would
  // not give every SM two of them (the mid scene's 32 000 children fill
  // only 125 CTAs of 256)
  int d_thr = h->tune.draw_threads;
  if (d_thr <= 0) {
    const long long kids = (long long)h->H * h_up;
    d_thr = 256;
    while (d_thr > 64 && kids < 2LL * n_sm * d_thr) d_thr >>= 1;
  }
  const int d_smem = expand_draw_smem(d_thr);
  const int d_ctas = std::max(1, expand_occupancy(a, ExpandKernel::kDraw, d_thr, d_smem));
  const long long d_need = ((long long)h->H * h_up + d_thr - 1) / d_thr;
  const int d_grid = p.fixed ? d_ctas * n_sm : (int)std::max(1LL, std::min(d_need, (long long)d_ctas * n_sm));
  // warp kernel: the overflow list, or every child
  int wg = p.wg;
  while (wg > 1 && p.Gw * wg > 16) wg >>= 1;   // a CTA holds at most 16 warps
  const int w_thr = 32 * p.Gw * wg;
  const int w_smem = expand_warp_smem(dz, 0, p.T, p.Gw, wg > 1);
  a.warp_group = wg;
  const int w_ctas = std::max(1, expand_occupancy(a, ExpandKernel::kWarp, w_thr, w_smem));
  int w_grid = w_ctas * n_sm;
  if (p.thread) w_grid = n_sm;
  else if (!p.fixed)
    w_grid = (int)std::max(1LL, std::min(((long long)h->H * h_up + p.Gw - 1) / p.Gw, (long long)w_grid));
  h->exp_smem = p.thread ? img : w_smem;
  h->exp_ctas = p.thread ? d_ctas : w_ctas;
  h->exp_plan[0] = p.T;
  h->exp_plan[1] = p.K;
  h->exp_plan[2] = p.M;
  h->exp_plan[3] = p.thread ? d_thr : w_thr;
  prof_begin(h, kStageExpand);
  if (!scal_zeroed) CU(cudaMemsetAsync(h->d_scal + S_REDO, 0, 2 * sizeof(unsigned), s));   // S_REDO, S_STAGE
  launch_expand_kernel(a, ExpandKernel::kStage, st_grid, st_thr, st_smem, s);
  if (p.thread) launch_expand_kernel(a, ExpandKernel::kDraw, d_grid, d_thr, d_smem, s);
  launch_expand_kernel(a, ExpandKernel::kWarp, w_grid, w_thr, w_smem, s);
  h->lse_parts = std::min(kMaxLseParts, p.fixed ? 8 * n_sm : std::max(1, std::min(h->H, 8 * n_sm)));
  launch_dedup(h->d_fs, h_up, h->child_key, h->child_hash, h->child_status, h->d_scal + S_ERR, h->pw,
               h->lse_parts, s);
  prof_end(h, kStageExpand);
  return GLMB_OK;
}

glmb_status enqueue_prune(glmb_handle* h, const Plan& p) {
  cudaStream_t s = h->stream;
  const int h_up = h->cfg.h_up;
  const long long n = p.fixed ? h->cap_children : (long long)h->H * h_up;
  const int nblk = (int)std::min<long long>(std::max(1LL, (n + 255) / 256), 2LL * h->n_sm);
  const double log_tau = std::log(h->cfg.tau);
  const double vmax = std::max(1.0, -log_tau) * 4294967296.0 + 2.0;
  const int nbits = std::max(1, (int)std::ceil(std::log2(vmax)));
  const HypTable& P = h->hyps[h->hcur];
  HypTable& O = h->hyps[1 - h->hcur];
  const CompTable& B = h->comps[1 - h->cur];
  CompTable& A = h->comps[h->cur];
  prof_begin(h, kStageSelect);
  // (the cluster kernel zeroes the prune counters itself)
  if (!launch_select_cluster(h->child_key, h->d_fs, h_up, h->pw, h->lse_parts, log_tau, h->cap_h, nbits,
                             h->child_alive, P, O,
                             h->d_scal + S_ERR, h->cap_entries, s)) {
    CU(cudaMemsetAsync(h->pw.counts, 0, 8 * sizeof(unsigned), s));
    launch_lse(h->child_key, h->d_fs, h_up, h->pw, log_tau, h->cap_h, nblk, s);
    launch_select(h->child_key, h->d_fs, h_up, nbits, h->pw, nblk, s);
    launch_compact(h->child_key, h->d_fs, h_up, n, h->pw, h->cap_h, nblk, s);
    launch_finalize(h->pw, h->child_key, h->child_alive, P, h_up, O, h->cap_h, h->d_scal + S_ERR,
                    h->cap_entries, s);
  }
  prof_end(h, kStageSelect);
  // the update hash table: only the slots the last materialisation filled
  // are cleared (the whole table is cleared after a frame that failed)
  launch_hash_reset(h->hkeys, h->upd_slot, h->d_hprev, (int)h->cap_upd, h->d_scal + S_NUPD, 2 * h->n_sm, s);
  const long long capT = p.fixed ? h->cap_comp : std::max(h->T_work, 1);
  ExpandArgs a = expand_args(h, p, true);
  a.surv_idx = h->pw.surv_idx;
  a.n_surv = h->pw.counts;
  a.out_ptr = O.ptr;
  a.out_comp = O.comp;
  a.out_theta = O.theta;
  a.hkeys = h->hkeys;
  a.hvals = h->hvals;
  a.hmask = h->hmask;
  a.upd_src = h->upd_src;
  a.upd_m = h->upd_m;
  a.upd_se = h->upd_se;
  a.upd_count = h->d_scal + S_NUPD;
  a.upd_slot = h->upd_slot;
  a.cap_upd = (int)h->cap_upd;
  int mg = p.mg;
  while (mg > 1 && p.Gm * mg > 16) mg >>= 1;   // a CTA holds at most 16 warps
  // (the areas were sized for one warp each; a group's area is 64 bytes larger)
  if (mg > 1 && expand_warp_smem(h->md.dz, 1, p.T, p.Gm, 1) > h->smem_limit) mg = 1;
  const int m_thr = 32 * p.Gm * mg;
  const int m_smem = expand_warp_smem(h->md.dz, 1, p.T, p.Gm, mg > 1);
  a.warp_group = mg;
  const int m_ctas = std::max(1, expand_occupancy(a, ExpandKernel::kWarp, m_thr, m_smem));
  const int m_grid = p.fixed ? m_ctas * h->n_sm
                             : std::max(1, std::min((h->cap_h + p.Gm - 1) / p.Gm, m_ctas * h->n_sm));
  prof_begin(h, kStageMat);
  launch_expand_kernel(a, ExpandKernel::kMatPrep, std::max(1, std::min((h->cap_h + 7) / 8, 2 * h->n_sm)),
                       256, 0, s);
  launch_expand_kernel(a, ExpandKernel::kWarp, m_grid, m_thr, m_smem, s);
  prof_end(h, kStageMat);
  const int T = h->T_work;
  prof_begin(h, kStageGc);
  scan_u32(h->gc_flag, h->gc_newpos, &h->d_fs->T, 1, capT, h->d_scal + S_NKEEP, false,
           h->scan_tmp32, h->scan_cap32, h->d_scal + S_ERR, s);
  const int ggc = p.fixed ? 4 * h->n_sm : std::max(1, std::min((T + 127) / 128 + 8, 8 * h->n_sm));
  if (h->md.particle)
    launch_particle_remap(h->md, h->pm, B, A, h->gc_newpos, h->gc_flag, h->d_fs, h->d_scal + S_NKEEP, h->upd_src,
                          h->upd_m, h->upd_se, (int)h->cap_upd, h->d_scal + S_NUPD, h->pw.counts,
                          h->d_scal + S_ERR, 4 * h->n_sm, s);
  launch_gc_remap(h->md, B, A, h->gc_newpos, h->gc_flag, h->d_fs, h->d_scal + S_NKEEP, h->upd_src, h->upd_m,
                  h->upd_se, (int)h->cap_upd, h->d_scal + S_NUPD, h->pw.counts, h->d_scal + S_ERR, O.comp,
                  h->pw.counts + 1, h->cap_entries, h->hvals, h->hmask, h->d_hprev, ggc, s);
  prof_end(h, kStageGc);
  CU(cudaGetLastError());
  return GLMB_OK;
}

// expansion plan of this frame: slots exactly (largest survivor of the last
// prune plus births), gated pairs from earlier frames (redone if exceeded)
// Warps per child on the warp path (expansion wg, regeneration mg) from
// the parts wc, mc that follow the hypothesis count: a child's work area in
// shared memory bounds how many warps an SM holds (16 at the kernel's
// registers); when the areas of a large plan leave fewer, a group of 2, 4
// or 8 warps shares each area (a child), so that the SM still holds up to
// 16 warps.  This part depends on the plan's slots alone, so a graph
// captured with headroom serves the frames that need fewer slots.
// GLMB_OPT_WARP_GROUPS forces groups of at least two (tests).
void set_groups(glmb_handle* h, Plan& p, int wc, int mc) {
  const int dz = h->md.dz;
  auto by_area = [&](int mat) {
    const int area = expand_warp_smem(dz, mat, p.T, 1, 1);
    const int areas_sm = std::max(1, std::min(16, h->smem_per_sm / std::max(area, 1)));
    int gw = 1;
    while (gw < 8 && areas_sm * gw * 2 <= 16) gw *= 2;
    return (h->launch_opts & GLMB_OPT_WARP_GROUPS) ? std::max(gw, 2) : gw;
  };
  p.wc = wc;
  p.mc = mc;
  p.wg = p.thread ? 1 : std::max(by_area(0), wc);
  p.mg = std::max(by_area(1), mc);
}

bool make_plan(glmb_handle* h, bool fixed, int T_plan, int K_plan, int M_plan, Plan& p) {
  p.fixed = fixed;
  p.T = std::max(1, T_plan);
  p.K = std::max(64, K_plan);
  p.M = std::max(1, M_plan);
  if (fixed) {
    p.T = round_up(p.T, 16);
    p.K = round_up(p.K, 64);
    p.M = round_up(p.M, 32);
  }
  const int dz = h->md.dz;
  // one thread per child once the children give every SM four warps (the
  // register lists address pairs with 16 bits); else one warp per child
  p.thread = (long long)h->H * h->cfg.h_up >= (long long)h->tune.thread_warps_per_sm * 32 * h->n_sm;
  if (h->launch_opts & GLMB_OPT_DRAW_THREAD) p.thread = true;
  if (h->launch_opts & GLMB_OPT_DRAW_WARP) p.thread = false;
  p.thread = p.thread && p.K <= 65536;
  // parents are staged in shared memory (then copied out to their image)
  // when eight staging CTAs fit on an SM; larger images are built in place
  // in global memory, where many CTAs per SM keep more parents in flight
  // (measured: on the 3-D sweep's N = 200 cell, 123 KB images, staging in
  // global memory with 64-thread CTAs ran the expansion in 2.41 ms against
  // 3.51 ms in shared memory at one CTA per SM; on the 2-D mid scene, 19 KB
  // images, shared memory stayed faster)
  const int img_bytes = expand_image_bytes(dz, p.T, p.K, p.M);
  p.smem = img_bytes + expand_stage_tail_bytes(dz, p.T, p.K, p.M, 0) <= h->smem_limit &&
           !(h->launch_opts & GLMB_OPT_STAGE_GLOBAL) &&
           (8LL * img_bytes <= (long long)h->smem_per_sm || (h->launch_opts & GLMB_OPT_STAGE_SHARED));
  // staging threads: 256 in shared memory, or for few parents (each parent's
  // work spread over more threads); else 128: with its scratch in shared
  // memory (about 29 KB for the 3-D sweep's plans) six such CTAs per SM keep
  // 24 warps in flight, where 64-thread CTAs would be limited to seven by
  // shared memory (measured on the N = 200, H_max = 20000 cell: expansion
  // 1.56 ms with 128, 1.87 ms with 64)
  p.st_thr = h->tune.stage_threads > 0 ? h->tune.stage_threads
             : (p.smem || (long long)h->H < 2LL * h->n_sm) ? 256 : 128;
  p.Gw = p.Gm = 0;
  for (int g = h->tune.warp_cta_warps; g >= 1 && !p.Gw; --g)
    if (expand_warp_smem(dz, 0, p.T, g, 1) <= h->smem_limit) p.Gw = g;
  // materialisation: the CTA size that keeps the most warps resident (its
  // per-warp work area is large, so eight-warp CTAs would leave an SM with
  // one CTA and shared memory unused)
  p.Gm = expand_warp_best_cta(dz, 1, p.T, 8, h->smem_limit);
  // warps per child, in two parts.  When the children are few (a few
  // hypotheses of many slots), several warps share a child, as long as all
  // the children's warps fit on the GPU at once (16 per SM).  This part
  // follows the hypothesis count, so it is kept to frames of 768 slots or
  // more, whose scenes hold their counts (smaller scenes sweep through the
  // thresholds as they grow and would spread their frames over more graphs:
  // measured, the N = 200 cell's regeneration 0.196 -> 0.208 ms).
  auto by_children = [&](long long children) {
    int gw = 1;
    if (p.T >= 768)
      while (gw < 8 && children * gw * 2 <= 16LL * h->n_sm) gw *= 2;
    return gw;
  };
  set_groups(h, p, p.thread ? 1 : by_children((long long)h->H * h->cfg.h_up), by_children(std::max(1, h->H)));
  return p.T <= 32767 && p.Gw > 0 && p.Gm > 0;
}

// footprint of a plan's per-parent image
int plan_smem(const glmb_handle* h, const Plan& p) {
  return expand_image_bytes(h->md.dz, p.T, p.K, p.M);
}

// the largest slot and pair counts over the frame's parents, computed from
// the table alone (a redo plans from these, whatever the failed pass staged)
glmb_status exact_maxima(glmb_handle* h, unsigned& max_T, unsigned& max_K) {
  CU(cudaMemsetAsync(h->d_scal + S_MAXT, 0, 2 * sizeof(unsigned), h->stream));
  launch_parent_stats(h->hyps[h->par_buf], h->d_fs, h->pt, h->d_scal + S_MAXT, h->d_scal + S_MAXK,
                      std::max(1, std::min((h->H + 127) / 128, 4 * h->n_sm)), h->stream);
  unsigned m[2] = {0, 0};
  CU(cudaMemcpyAsync(m, h->d_scal + S_MAXT, sizeof m, cudaMemcpyDeviceToHost, h->stream));
  CU(cudaStreamSynchronize(h->stream));
  max_T = m[0];
  max_K = m[1];
  return GLMB_OK;
}

// frame result: commit, abandon, or redo with exact maxima; `done` on return
// the frame's counters (and, with estimates, the estimate block) to pinned
// host memory, on the stream
glmb_status enqueue_results(glmb_handle* h, bool with_est) {
  // scalars and counters (and the estimates) in one copy of the result block
  const size_t bytes = with_est ? h->res_off_est + h->est_off_end : h->res_off_cnt + 8 * sizeof(unsigned);
  CU(cudaMemcpyAsync(h->h_scal, h->d_scal, bytes, cudaMemcpyDeviceToHost, h->stream));
  return GLMB_OK;
}

// estimates of table (Y, A) with Y's hypothesis count on the device
// (H_dev) or on the host
void enqueue_estimates(glmb_handle* h, const HypTable& Y, const CompTable& A, const unsigned* H_dev, int H) {
  const int pcap = h->max_tracks + 1;
  prof_begin(h, kStageEstimates);
  unsigned* work = reinterpret_cast<unsigned*>(h->d_est + h->est_off_done);   // [cmax, done]
  launch_estimates(Y, H, H_dev, H_dev ? h->cap_h : H, A, h->md.dx, (double*)(h->d_est + h->est_off_pmf), pcap,
                   (int*)h->d_est, h->est_rcomp, h->est_rcomp + h->cap_comp, h->d_est + h->est_off_tr, work,
                   work + 1, h->n_sm, H_dev ? h->d_scal + S_ERR : nullptr, h->stream);
  prof_end(h, kStageEstimates);
}

// the whole update hash table cleared (and the reset list emptied) after a
// frame whose updates overflowed it; stream-ordered before the next frame
glmb_status clear_hash_if_dirty(glmb_handle* h) {
  if (!h->hash_dirty) return GLMB_OK;
  CU(cudaMemsetAsync(h->hkeys, 0, ((size_t)h->hmask + 1) * sizeof(unsigned long long), h->stream));
  CU(cudaMemsetAsync(h->d_hprev, 0, sizeof(unsigned), h->stream));
  h->hash_dirty = false;
  return GLMB_OK;
}

// results: the counters were copied by the frame's launches when
// copies_enqueued (with the estimates when est_enqueued); redo, abandon or
// commit
glmb_status finish_frame(glmb_handle* h, bool copies_enqueued = false, bool est_enqueued = false) {
  auto abandon = [&](glmb_status st, const char* msg) {
    h->frame -= 1;
    h->stage = 0;
    return fail(h, st, "prune: %s", msg);
  };
  glmb_status st;
  if (!copies_enqueued && (st = enqueue_results(h, false)) != GLMB_OK) return st;
  CU(cudaStreamSynchronize(h->stream));
  const unsigned* cnt = h->h_cnt;
  unsigned e = h->h_scal[S_ERR];
  // updates beyond the table's capacity are not in the reset list
  if (e & (kErrUpdates | kErrHash)) h->hash_dirty = true;
  if ((e & kErrSlots) && !(e & (kErrFatal & ~kErrSlots))) {
    // a parent had more gated pairs than planned: redo the expansion and
    // the pruning with the exact maxima of this frame
    ++h->redo_count;
    unsigned mt = 0, mk = 0;
    if ((st = exact_maxima(h, mt, mk)) != GLMB_OK) return st;
    Plan p;
    if (!make_plan(h, false, std::max(1u, mt), std::max(1u, mk), h->M, p))
      return abandon(GLMB_E_CAPACITY, "per-hypothesis table exceeds the supported sizes");
    if ((st = ensure_img(h, p)) != GLMB_OK) return abandon(st, "expansion images do not fit");
    CU(cudaMemsetAsync(h->d_scal + S_ERR, 0, sizeof(unsigned), h->stream));
    if ((st = clear_hash_if_dirty(h)) != GLMB_OK) return st;
    if ((st = enqueue_expand(h, p)) != GLMB_OK) return st;
    if ((st = enqueue_prune(h, p)) != GLMB_OK) return st;
    if ((st = enqueue_results(h, false)) != GLMB_OK) return st;
    CU(cudaStreamSynchronize(h->stream));
    e = h->h_scal[S_ERR];
    if (e & (kErrUpdates | kErrHash)) h->hash_dirty = true;
    est_enqueued = false;   // the estimates copied with the first pass are stale
  }
  if (e & kErrInput) return abandon(GLMB_E_INVALID, "non-finite detection");
  if (e & (kErrGate | kErrTimeout)) return abandon(GLMB_E_TIMEOUT, err_text(e));
  if (e & kErrFatal) return abandon(e & kErrNumeric ? GLMB_E_NUMERIC : GLMB_E_CAPACITY, err_text(e));
  h->n_pairs = h->h_scal[S_K];
  h->n_pairs_pregate = h->gate_mode_frame == GLMB_GATE_PRUNE ? (long long)h->h_scal[S_KFULL] : h->n_pairs;
  h->n_fp64 = (int)h->h_scal[S_FP64];
  h->n_draw_overflow = h->plan.thread ? (long long)h->h_scal[S_REDO] : 0;
  const unsigned n_surv = cnt[0];
  if (n_surv == 0) return abandon(GLMB_E_NUMERIC, "no child has a finite weight above tau");
  const unsigned n_keep = h->h_scal[S_NKEEP], n_upd = h->h_scal[S_NUPD];
  if ((long long)n_keep + n_upd > h->cap_comp) return abandon(GLMB_E_CAPACITY, "components exceed capacity");
  prof_collect(h);
  // commit
  h->n_unique = cnt[2];
  h->alive_max = (int)cnt[3];
  h->K_est = round_up((int)(h->h_scal[S_MAXK] + h->h_scal[S_MAXK] / 8) + 16, 64);
  h->n_upd = (int)n_upd;
  h->n_comp = (int)(n_keep + n_upd);
  h->H = (int)n_surv;
  h->n_entries = cnt[1];
  h->hcur = 1 - h->hcur;
  h->theta_M = h->M;
  h->theta_M_valid = true;
  h->retained_valid = true;
  h->stage = 0;
  ++h->gen;
  if (est_enqueued) h->est_gen = h->gen;
  return GLMB_OK;
}

}  // namespace

glmb_status glmb_predict(glmb_handle* h, const glmb_birth* births, int n_births) {
  if (!h) return GLMB_E_INVALID;
  if (h->stage != 0) return fail(h, GLMB_E_STATE, "predict: previous frame not pruned");
  glmb_status st = stage_births(h, births, n_births);
  if (st != GLMB_OK) return st;
  if ((st = ensure_slm(h, (long long)h->n_comp + n_births)) != GLMB_OK) return st;
  h->frame += 1;
  h->nb = n_births;
  h->T_work = h->n_comp + n_births;
  h->M = 0;
  if ((st = upload_sizes(h, 0)) != GLMB_OK) return st;
  if (n_births)
    CU(cudaMemcpyAsync(h->d_births, h->h_births, (size_t)n_births * kBirthRec * sizeof(double),
                       cudaMemcpyHostToDevice, h->stream));
  Plan p{};
  p.fixed = false;
  enqueue_predict(h, p);
  CU(cudaGetLastError());
  h->stage = 1;
  h->have_update = false;
  return GLMB_OK;
}

glmb_status glmb_update(glmb_handle* h, const float* Z, int M, int z_is_device) {
  if (!h) return GLMB_E_INVALID;
  if (h->stage != 1) return fail(h, GLMB_E_STATE, "update: call glmb_predict first");
  glmb_status st = stage_detections(h, Z, M, z_is_device);
  if (st != GLMB_OK) {
    if (st == GLMB_E_INVALID && M > 0 && Z) {
      h->frame -= 1;
      h->stage = 0;
    }
    return st;
  }
  h->M = M;
  if ((st = upload_sizes(h, 1)) != GLMB_OK) return st;
  Plan p;
  if (!make_plan(h, false, h->alive_max + h->nb, h->K_est, h->M, p) || ensure_img(h, p) != GLMB_OK) {
    // the estimate does not fit; plan from the exact maxima of this frame
    h->err.clear();
    Plan q{};
    q.fixed = false;
    enqueue_table(h, q);
    launch_parent_stats(h->hyps[h->hcur], h->d_fs, h->pt, h->d_scal + S_MAXT, h->d_scal + S_MAXK,
                        std::max(1, std::min((h->H + 127) / 128, 4 * h->n_sm)), h->stream);
    CU(cudaStreamSynchronize(h->stream));
    unsigned mk = 0;
    CU(cudaMemcpy(&mk, h->d_scal + S_MAXK, sizeof mk, cudaMemcpyDeviceToHost));
    if (!make_plan(h, false, h->alive_max + h->nb, (int)mk, h->M, p) || ensure_img(h, p) != GLMB_OK) {
      h->frame -= 1;
      h->stage = 0;
      return fail(h, GLMB_E_CAPACITY, "update: per-hypothesis table exceeds the supported sizes");
    }
  } else {
    enqueue_table(h, p);
  }
  h->plan = p;
  enqueue_expand(h, p, true);
  CU(cudaGetLastError());
  // a parent with more gated pairs than the plan's estimate: redo the
  // expansion now with the frame's exact maxima, so that the children are
  // final when update returns (glmb_step redoes in its completion instead)
  CU(cudaStreamSynchronize(h->stream));
  unsigned sc[4] = {0, 0, 0, 0};
  CU(cudaMemcpy(sc, h->d_scal, sizeof sc, cudaMemcpyDeviceToHost));
  if ((sc[S_ERR] & kErrSlots) && !(sc[S_ERR] & (kErrFatal & ~kErrSlots))) {
    Plan q;
    unsigned mt = 0, mk = 0;
    h->par_buf = h->hcur;   // exact_maxima reads the parents of this update
    if ((st = exact_maxima(h, mt, mk)) != GLMB_OK) return st;
    if (make_plan(h, false, std::max(1u, mt), std::max(1u, mk), h->M, q) &&
        ensure_img(h, q) == GLMB_OK) {
      ++h->redo_count;
      CU(cudaMemsetAsync(h->d_scal + S_ERR, 0, sizeof(unsigned), h->stream));
      enqueue_expand(h, q);
      CU(cudaGetLastError());
      h->plan = q;
    }
  }
  h->H_par = h->H;
  h->par_buf = h->hcur;
  h->birth_base = h->n_comp;
  h->stage = 2;
  h->have_update = true;
  return GLMB_OK;
}

glmb_status glmb_prune(glmb_handle* h) {
  if (!h) return GLMB_E_INVALID;
  if (h->stage != 2) return fail(h, GLMB_E_STATE, "prune: call glmb_update first");
  h->retained_valid = false;
  glmb_status st = clear_hash_if_dirty(h);
  if (st != GLMB_OK) return st;
  st = enqueue_prune(h, h->plan);
  if (st != GLMB_OK) return st;
  return finish_frame(h);
}

glmb_status glmb_step_enqueue(glmb_handle* h, const glmb_birth* births, int n_births, const float* Z, int M,
                              int z_is_device) {
  if (!h) return GLMB_E_INVALID;
  if (h->stage != 0) return fail(h, GLMB_E_STATE, "step: a frame is in progress");
  glmb_status st = stage_births(h, births, n_births);
  if (st != GLMB_OK) return st;
  st = stage_detections(h, Z, M, z_is_device, false);
  if (st != GLMB_OK) return st;
  if ((st = ensure_slm(h, (long long)h->n_comp + n_births)) != GLMB_OK) return st;
  h->frame += 1;
  h->nb = n_births;
  h->T_work = h->n_comp + n_births;
  h->M = M;
  Plan p;
  // while a wait test is set, frames run eagerly (no graph is captured with
  // the test's launch settings)
  const bool graphs_ok = wait_test().mode == 0;
  if (!(graphs_ok && make_plan(h, true, h->alive_max + h->nb, h->K_est, h->M, p)) &&
      !make_plan(h, false, h->alive_max + h->nb, h->K_est, h->M, p)) {
    h->frame -= 1;
    return fail(h, GLMB_E_CAPACITY, "step: per-hypothesis table does not fit in shared memory");
  }
  if ((st = clear_hash_if_dirty(h)) != GLMB_OK) return st;
  // the frame's sizes, births and host detections go up with the frame: as
  // copy nodes of the graph when one is replayed, else as separate copies
  if ((st = upload_sizes(h, 1, !p.fixed)) != GLMB_OK) return st;
  if (!p.fixed) {
    if (n_births)
      CU(cudaMemcpyAsync(h->d_births, h->h_births, (size_t)n_births * kBirthRec * sizeof(double),
                         cudaMemcpyHostToDevice, h->stream));
    if (M > 0 && !z_is_device)
      CU(cudaMemcpyAsync(h->d_Z, h->h_Z, (size_t)M * h->md.dz * sizeof(float), cudaMemcpyHostToDevice,
                         h->stream));
  }
  h->retained_valid = false;
  h->plan = p;
  if (p.fixed) {
    // Replay the captured graph with the smallest per-parent image whose
    // plan covers this frame (same buffer parity and profiling mask; slots,
    // pairs and detections at least this frame's).  A cover more than three
    // times larger than this frame needs is replaced by a tighter capture;
    // captures take headroom so that a growing scene needs few of them.
    const int need_smem = plan_smem(h, p);
    int best = -1;
    for (int gi = 0; gi < (int)h->graphs.size(); ++gi) {
      const glmb_handle::CachedGraph& g = h->graphs[gi];
      if (g.hcur != h->hcur || g.prof != h->prof_mask || g.plan.thread != p.thread || g.plan.st_thr != p.st_thr ||
          g.plan.wc != p.wc || g.plan.mc != p.mc ||
          g.plan.T < p.T || g.plan.K < p.K || g.plan.M < p.M)
        continue;
      if (best < 0 || g.smem < h->graphs[best].smem) best = gi;
    }
    if (best >= 0 && (long long)h->graphs[best].smem > 3LL * need_smem) best = -1;
    if (best < 0) {
      Plan q = p;
      if (!make_plan(h, true, round_up(p.T + p.T / 2, 32), round_up(p.K + p.K / 2, 128), round_up(p.M + p.M / 4, 64), q) ||
          q.thread != p.thread ||
          (p.smem && !q.smem))
        q = p;
      set_groups(h, q, p.wc, p.mc);   // this frame's parts (q.T decides the rest)
      if ((st = ensure_img(h, q)) != GLMB_OK) {
        h->frame -= 1;
        return st;
      }
      cudaGraph_t graph = nullptr;
      cudaGraphExec_t exec = nullptr;
      const auto t_cap = std::chrono::steady_clock::now();
      CU(cudaStreamBeginCapture(h->stream, cudaStreamCaptureModeThreadLocal));
      h->capturing = true;
      // sizes, births and host detections in one copy of the input block
      cudaMemcpyAsync(h->d_fs, &h->h_fs[1],
                      h->in_off_Z + (size_t)std::min(q.M, h->cap_meas) * h->md.dz * sizeof(float),
                      cudaMemcpyHostToDevice, h->stream);
      enqueue_predict(h, q);
      enqueue_table(h, q);
      enqueue_expand(h, q, true);
      enqueue_prune(h, q);
      if (h->step_estimates)
        enqueue_estimates(h, h->hyps[1 - h->hcur], h->comps[h->cur], h->pw.counts, 0);
      enqueue_results(h, h->step_estimates);
      h->capturing = false;
      CU(cudaStreamEndCapture(h->stream, &graph));
      size_t n_nodes = 0;
      cudaGraphGetNodes(graph, nullptr, &n_nodes);
      std::vector<cudaGraphNode_t> nodes(n_nodes);
      long long n_kernels = 0;
      if (n_nodes && cudaGraphGetNodes(graph, nodes.data(), &n_nodes) == cudaSuccess)
        for (auto nd : nodes) {
          cudaGraphNodeType ty;
          if (cudaGraphNodeGetType(nd, &ty) == cudaSuccess && ty == cudaGraphNodeTypeKernel) ++n_kernels;
        }
      g_launches -= n_kernels;   // counted once per replay below, not at capture
      std::vector<glmb_handle::KeyNode> key_nodes;
      for (size_t ni = 0; ni < n_nodes; ++ni) {
        cudaGraphNodeType ty;
        cudaKernelNodeParams kp{};
        if (cudaGraphNodeGetType(nodes[ni], &ty) != cudaSuccess || ty != cudaGraphNodeTypeKernel ||
            cudaGraphKernelNodeGetParams(nodes[ni], &kp) != cudaSuccess || !expand_kernel_takes_key(kp.func))
          continue;
        glmb_handle::KeyNode kn;
        kn.node = nodes[ni];
        kn.p = kp;
        kn.p.kernelParams = nullptr;
        kn.p.extra = nullptr;
        std::memcpy(&kn.a, kp.kernelParams[0], sizeof(ExpandArgs));
        key_nodes.push_back(kn);
      }
      const cudaError_t ie = cudaGraphInstantiate(&exec, graph, 0);
      if (ie != cudaSuccess) {
        cudaGraphDestroy(graph);
        return fail(h, GLMB_E_CUDA, "step: graph instantiation: %s", cudaGetErrorString(ie));
      }
      if (h->graphs.size() >= 32) {
        // evict the least recently replayed graph
        int lru = 0;
        for (int gi = 1; gi < (int)h->graphs.size(); ++gi)
          if (h->graphs[gi].last_use < h->graphs[lru].last_use) lru = gi;
        drop_graph(h->graphs[lru]);
        h->graphs.erase(h->graphs.begin() + lru);
      }
      h->graphs.push_back(glmb_handle::CachedGraph{h->hcur, h->prof_mask, q, exec, n_kernels, plan_smem(h, q), 0,
                                                   graph, std::move(key_nodes)});
      ++h->n_captures;
      h->capture_ms += std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t_cap).count();
      best = (int)h->graphs.size() - 1;
    }
    h->graphs[best].last_use = h->frame;
    glmb_handle::CachedGraph& g = h->graphs[best];
    h->plan = g.plan;
    // this frame's Philox key in the nodes that draw
    const uint32_t key_y = h->md.seed_hi ^ (uint32_t)h->frame;
    for (auto& kn : g.key_nodes) {
      if (kn.a.key_y == key_y) continue;
      kn.a.key_y = key_y;
      void* args[1] = {&kn.a};
      cudaKernelNodeParams q = kn.p;
      q.kernelParams = args;
      CU(cudaGraphExecKernelNodeSetParams(g.exec, kn.node, &q));
    }
    g_launches += g.n_kernels;
    CU(cudaGraphLaunch(g.exec, h->stream));
    ++h->n_graph_launches;
    for (int s = 0; s <= kStageEstimates; ++s)
      if ((h->prof_mask & (1u << s)) && h->ev[s][0] && (s < kStageEstimates || h->step_estimates))
        h->ev_pending[s] = true;
  } else {
    enqueue_predict(h, p);
    enqueue_table(h, p);
    enqueue_expand(h, p, true);
    enqueue_prune(h, p);
    if (h->step_estimates)
      enqueue_estimates(h, h->hyps[1 - h->hcur], h->comps[h->cur], h->pw.counts, 0);
    enqueue_results(h, h->step_estimates);
  }
  CU(cudaGetLastError());
  h->H_par = h->H;
  h->par_buf = h->hcur;
  h->birth_base = h->n_comp;
  h->have_update = true;
  h->stage = 3;   // in flight: glmb_step_finish
  return GLMB_OK;
}

glmb_status glmb_step_finish(glmb_handle* h) {
  if (!h) return GLMB_E_INVALID;
  if (h->stage != 3) return fail(h, GLMB_E_STATE, "step_finish: no frame in flight");
  h->stage = 2;
  return finish_frame(h, true, h->step_estimates);
}

glmb_status glmb_step(glmb_handle* h, const glmb_birth* births, int n_births, const float* Z, int M,
                      int z_is_device) {
  glmb_status st = glmb_step_enqueue(h, births, n_births, Z, M, z_is_device);
  if (st != GLMB_OK) return st;
  return glmb_step_finish(h);
}

glmb_status glmb_step_batch(glmb_handle* const* hs, int n, const glmb_frame_in* frames, glmb_status* status) {
  if (n < 0 || (n > 0 && (!hs || !frames))) return GLMB_E_INVALID;
  glmb_status first = GLMB_OK;
  for (int i = 0; i < n; ++i) {
    const glmb_frame_in& f = frames[i];
    const glmb_status st = glmb_step_enqueue(hs[i], f.births, f.n_births, f.Z, f.M, f.z_is_device);
    if (status) status[i] = st;
    if (st != GLMB_OK && first == GLMB_OK) first = st;
  }
  for (int i = 0; i < n; ++i) {
    if (!hs[i] || hs[i]->stage != 3) continue;
    const glmb_status st = glmb_step_finish(hs[i]);
    if (status) status[i] = st;
    if (st != GLMB_OK && first == GLMB_OK) first = st;
  }
  return first;
}

glmb_status glmb_set_tuning(glmb_handle* h, const glmb_tuning* t) {
  if (!h || !t) return GLMB_E_INVALID;
  if (t->thread_warps_per_sm < 0 || t->warp_cta_warps < 1 || t->warp_cta_warps > 16 ||
      (t->draw_threads != 0 && (t->draw_threads < 32 || t->draw_threads > 256 || t->draw_threads % 32)) ||
      (t->stage_threads != 0 && (t->stage_threads < 32 || t->stage_threads > 256 || t->stage_threads % 32)))
    return fail(h, GLMB_E_INVALID, "set_tuning: a launch shape out of range");
  cudaStreamSynchronize(h->stream);
  for (auto& g : h->graphs) drop_graph(g);
  h->graphs.clear();
  h->tune = *t;
  return GLMB_OK;
}

glmb_status glmb_get_tuning(glmb_handle* h, glmb_tuning* t) {
  if (!h || !t) return GLMB_E_INVALID;
  *t = h->tune;
  return GLMB_OK;
}

glmb_status glmb_get_retained(glmb_handle* h, int64_t* child_idx, double* logw, int cap, int* n) {
  if (!h || !n) return GLMB_E_INVALID;
  if (!h->retained_valid) return fail(h, GLMB_E_STATE, "get_retained: no pruned frame");
  CU(cudaStreamSynchronize(h->stream));
  *n = h->H;
  if (h->H > cap) return fail(h, GLMB_E_CAPACITY, "get_retained: cap");
  if (child_idx)
    CU(cudaMemcpy(child_idx, h->pw.surv_idx, (size_t)h->H * sizeof(long long), cudaMemcpyDeviceToHost));
  if (logw)
    CU(cudaMemcpy(logw, h->hyps[h->hcur].logw, (size_t)h->H * sizeof(double), cudaMemcpyDeviceToHost));
  return GLMB_OK;
}

glmb_status glmb_get_info(glmb_handle* h, glmb_info* info) {
  if (!h || !info) return GLMB_E_INVALID;
  CU(cudaStreamSynchronize(h->stream));
  std::memset(info, 0, sizeof *info);
  info->frame = h->frame;
  info->n_hyp = h->H;
  info->n_entries = h->n_entries;
  info->n_components = h->n_comp;
  info->n_meas = h->M;
  info->n_pairs = h->n_pairs;
  if (h->have_update) {
    uint32_t K32 = 0;
    CU(cudaMemcpy(&K32, h->pt.ptr + h->T_work, sizeof K32, cudaMemcpyDeviceToHost));
    info->n_pairs = K32;
  }
  info->n_pairs_pregate = h->gate_mode_frame == GLMB_GATE_PRUNE ? h->n_pairs_pregate : info->n_pairs;
  info->n_children = h->have_update ? (long long)h->H_par * h->cfg.h_up : 0;
  info->n_unique = h->n_unique;
  info->n_updates = h->n_upd;
  info->n_fp64_chol = h->n_fp64;
  info->n_launches = g_launches;
  info->n_graph_captures = h->n_captures;
  info->n_graph_launches = h->n_graph_launches;
  info->n_redo = h->redo_count;
  info->expand_smem_bytes = h->exp_smem;
  info->expand_ctas_per_sm = h->exp_ctas;
  info->expand_plan_T = h->exp_plan[0];
  info->expand_plan_K = h->exp_plan[1];
  info->expand_plan_M = h->exp_plan[2];
  info->expand_threads = h->exp_plan[3];
  info->graph_capture_ms = h->capture_ms;
  info->n_draw_overflow = h->n_draw_overflow;
  return GLMB_OK;
}

glmb_status glmb_estimates(glmb_handle* h, glmb_track* out, int cap, int* n_out, double* card_pmf,
                           int pmf_cap) {
  if (!h || !n_out || (cap > 0 && !out)) return GLMB_E_INVALID;
  if (h->stage >= 2) return fail(h, GLMB_E_STATE, "estimates: call glmb_prune (or glmb_step_finish) first");
  cudaStream_t s = h->stream;
  const int pcap = h->max_tracks + 1;
  if (h->est_gen != h->gen) {   // not computed with this state's step
    enqueue_estimates(h, h->hyps[h->hcur], h->comps[h->cur], nullptr, h->H);
    CU(cudaGetLastError());
    CU(cudaMemcpyAsync(h->h_est, h->d_est, h->est_off_end, cudaMemcpyDeviceToHost, s));
    CU(cudaStreamSynchronize(s));
    h->est_gen = h->gen;
  }
  int nb[2];
  std::memcpy(nb, h->h_est, sizeof nb);
  const int nhat = nb[0];
  *n_out = nhat;
  const double* pmf = (const double*)(h->h_est + h->est_off_pmf);
  if (card_pmf)
    for (int k = 0; k < pmf_cap; ++k) card_pmf[k] = k < pcap ? pmf[k] : 0.0;
  if (nhat > cap) return fail(h, GLMB_E_CAPACITY, "estimates: %d tracks > cap %d", nhat, cap);
  if (nhat > 0) std::memcpy(out, h->h_est + h->est_off_tr, (size_t)nhat * sizeof(glmb_track));
  return GLMB_OK;
}

glmb_status glmb_meas_assoc(glmb_handle* h, double* r_u, int cap) {
  if (!h || (cap > 0 && !r_u)) return GLMB_E_INVALID;
  if (!h->theta_M_valid || h->stage >= 2) return fail(h, GLMB_E_STATE, "meas_assoc: no pruned frame");
  if (h->theta_M > cap) return fail(h, GLMB_E_CAPACITY, "meas_assoc: cap < M");
  launch_meas_assoc(h->hyps[h->hcur], h->H, h->theta_M, h->d_ru, h->stream);
  CU(cudaGetLastError());
  CU(cudaMemcpyAsync(r_u, h->d_ru, (size_t)h->theta_M * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
  CU(cudaStreamSynchronize(h->stream));
  return GLMB_OK;
}

// ---- state buffer ------------------------------------------------------------
namespace {
struct StateHeader {
  uint32_t magic, version;
  int32_t dim_x, frame, n_hyp, pad;
  int64_t n_tracks;
};
struct HypRec {
  double logw;
  uint64_t uid;
  int32_t n_tracks, pad;
};
}  // namespace

glmb_status glmb_export_state(glmb_handle* h, void* buf, size_t cap, size_t* n_out) {
  if (!h || !n_out) return GLMB_E_INVALID;
  if (h->stage != 0) return fail(h, GLMB_E_STATE, "export: frame in progress");
  const int dx = h->md.dx, ncov = h->md.ncov;
  const int np = h->md.particle ? h->pm.np : 0;
  const size_t trk = 8 + 8 * (size_t)dx + 8 * (size_t)dx * dx + 48 * (size_t)np;
  const size_t need = sizeof(StateHeader) + sizeof(HypRec) * h->H + trk * (size_t)h->n_entries;
  *n_out = need;
  if (!buf) return GLMB_OK;
  if (cap < need) return fail(h, GLMB_E_CAPACITY, "export: buffer too small");
  CU(cudaStreamSynchronize(h->stream));
  const HypTable& Y = h->hyps[h->hcur];
  const CompTable& A = h->comps[h->cur];
  std::vector<uint32_t> ptr(h->H + 1), comp(std::max<long long>(1, h->n_entries));
  std::vector<double> logw(h->H);
  std::vector<unsigned long long> uid(h->H);
  CU(cudaMemcpy(ptr.data(), Y.ptr, ptr.size() * 4, cudaMemcpyDeviceToHost));
  CU(cudaMemcpy(comp.data(), Y.comp, (size_t)h->n_entries * 4, cudaMemcpyDeviceToHost));
  CU(cudaMemcpy(logw.data(), Y.logw, (size_t)h->H * 8, cudaMemcpyDeviceToHost));
  CU(cudaMemcpy(uid.data(), Y.uid, (size_t)h->H * 8, cudaMemcpyDeviceToHost));
  const size_t nc = std::max(1, h->n_comp);
  std::vector<float> mh(nc * dx), ml(nc * dx), cv(nc * ncov);
  std::vector<uint32_t> lk(nc), lb(nc);
  for (int a = 0; a < dx; ++a) {
    CU(cudaMemcpy(mh.data() + a * nc, A.mhi + (size_t)a * A.cap, (size_t)h->n_comp * 4, cudaMemcpyDeviceToHost));
    CU(cudaMemcpy(ml.data() + a * nc, A.mlo + (size_t)a * A.cap, (size_t)h->n_comp * 4, cudaMemcpyDeviceToHost));
  }
  for (int k = 0; k < ncov; ++k)
    CU(cudaMemcpy(cv.data() + k * nc, A.cov + (size_t)k * A.cap, (size_t)h->n_comp * 4, cudaMemcpyDeviceToHost));
  CU(cudaMemcpy(lk.data(), A.lk, (size_t)h->n_comp * 4, cudaMemcpyDeviceToHost));
  CU(cudaMemcpy(lb.data(), A.lb, (size_t)h->n_comp * 4, cudaMemcpyDeviceToHost));
  std::vector<double> px(np ? nc * 6 * (size_t)np : 0);
  if (np && h->n_comp > 0)
    CU(cudaMemcpy(px.data(), A.px, (size_t)h->n_comp * 6 * np * 8, cudaMemcpyDeviceToHost));
  unsigned char* p = (unsigned char*)buf;
  StateHeader hd{0x424D4C47u, np ? 2u : 1u, dx, h->frame, h->H, 0, h->n_entries};
  std::memcpy(p, &hd, sizeof hd);
  p += sizeof hd;
  for (int y = 0; y < h->H; ++y) {
    HypRec r{logw[y], uid[y], (int32_t)(ptr[y + 1] - ptr[y]), 0};
    std::memcpy(p, &r, sizeof r);
    p += sizeof r;
  }
  for (long long e = 0; e < h->n_entries; ++e) {
    const size_t c = comp[e];
    std::memcpy(p, &lk[c], 4);
    std::memcpy(p + 4, &lb[c], 4);
    p += 8;
    for (int a = 0; a < dx; ++a) {
      const double v = (double)mh[a * nc + c] + (double)ml[a * nc + c];
      std::memcpy(p, &v, 8);
      p += 8;
    }
    for (int i = 0; i < dx; ++i)
      for (int k = 0; k < dx; ++k) {
        const double v = cv[(size_t)pidx(dx, std::min(i, k), std::max(i, k)) * nc + c];
        std::memcpy(p, &v, 8);
        p += 8;
      }
    for (int q = 0; q < np; ++q)
      for (int k = 0; k < 5; ++k) {
        std::memcpy(p, &px[(c * 6 + k) * (size_t)np + q], 8);
        p += 8;
      }
    if (np) {
      std::memcpy(p, &px[(c * 6 + 5) * (size_t)np], 8 * (size_t)np);
      p += 8 * (size_t)np;
    }
  }
  return GLMB_OK;
}

glmb_status glmb_import_state(glmb_handle* h, const void* buf, size_t n) {
  if (!h || !buf) return GLMB_E_INVALID;
  const int dx = h->md.dx, ncov = h->md.ncov;
  if (n < sizeof(StateHeader)) return fail(h, GLMB_E_STATE, "import: short buffer");
  StateHeader hd;
  std::memcpy(&hd, buf, sizeof hd);
  const int np = h->md.particle ? h->pm.np : 0;
  if (hd.magic != 0x424D4C47u || hd.version != (np ? 2u : 1u) || hd.dim_x != dx || hd.n_hyp < 1 ||
      hd.n_tracks < 0 || hd.frame < 0)
    return fail(h, GLMB_E_STATE, "import: bad header");
  if (hd.n_hyp > h->cap_h) return fail(h, GLMB_E_CAPACITY, "import: hypotheses exceed h_max");
  if (hd.n_tracks > h->cap_entries) return fail(h, GLMB_E_CAPACITY, "import: entries exceed capacity");
  const size_t trk = 8 + 8 * (size_t)dx + 8 * (size_t)dx * dx + 48 * (size_t)np;
  const size_t need = sizeof(StateHeader) + sizeof(HypRec) * hd.n_hyp + trk * (size_t)hd.n_tracks;
  if (n < need) return fail(h, GLMB_E_STATE, "import: truncated buffer");
  const unsigned char* p = (const unsigned char*)buf + sizeof hd;
  std::vector<uint32_t> ptr(hd.n_hyp + 1, 0);
  std::vector<double> logw(hd.n_hyp);
  std::vector<unsigned long long> uid(hd.n_hyp);
  for (int y = 0; y < hd.n_hyp; ++y) {
    HypRec r;
    std::memcpy(&r, p, sizeof r);
    p += sizeof r;
    if (r.n_tracks < 0 || r.n_tracks > h->max_tracks || !std::isfinite(r.logw))
      return fail(h, GLMB_E_STATE, "import: hypothesis %d", y);
    logw[y] = r.logw;
    uid[y] = r.uid;
    ptr[y + 1] = ptr[y] + (uint32_t)r.n_tracks;
  }
  if ((long long)ptr[hd.n_hyp] != hd.n_tracks) return fail(h, GLMB_E_STATE, "import: track count");
  // identical (label, mean, cov) records become one shared component
  std::unordered_map<std::string, uint32_t> seen;
  std::vector<uint32_t> comp(std::max<long long>(1, hd.n_tracks));
  std::vector<float> mh, ml, cv;
  std::vector<uint32_t> lk, lb;
  std::vector<double> px;   // particle model: per component 6 rows of np
  for (long long e = 0; e < hd.n_tracks; ++e) {
    std::string key((const char*)p, trk);
    auto it = seen.find(key);
    if (it != seen.end()) {
      comp[e] = it->second;
      p += trk;
      continue;
    }
    const uint32_t c = (uint32_t)lk.size();
    seen.emplace(std::move(key), c);
    comp[e] = c;
    uint32_t k0, b0;
    std::memcpy(&k0, p, 4);
    std::memcpy(&b0, p + 4, 4);
    lk.push_back(k0);
    lb.push_back(b0);
    p += 8;
    for (int a = 0; a < dx; ++a) {
      double v;
      std::memcpy(&v, p, 8);
      p += 8;
      if (!std::isfinite(v)) return fail(h, GLMB_E_STATE, "import: mean not finite");
      const float hi = (float)v;
      mh.push_back(hi);
      ml.push_back((float)(v - (double)hi));
    }
    double P[36];
    std::memcpy(P, p, 8 * dx * dx);
    p += 8 * dx * dx;
    if (!np) {
      for (int i = 0; i < dx; ++i)
        for (int k = i; k < dx; ++k) cv.push_back((float)(0.5 * (P[i * dx + k] + P[k * dx + i])));
      continue;
    }
    // particle model: the particles, and their weighted moments in place of
    // the record's (mean rounded to FP32 with a zero low part)
    const size_t base = px.size();
    px.resize(base + 6 * (size_t)np);
    for (int q = 0; q < np; ++q)
      for (int k = 0; k < 5; ++k) {
        std::memcpy(&px[base + (size_t)k * np + q], p, 8);
        p += 8;
      }
    std::memcpy(&px[base + 5 * (size_t)np], p, 8 * (size_t)np);
    p += 8 * (size_t)np;
    double m[5] = {0, 0, 0, 0, 0}, C2[15] = {0};
    for (int q = 0; q < np; ++q) {
      const double w = std::exp(px[base + 5 * (size_t)np + q]);
      if (!std::isfinite(w)) return fail(h, GLMB_E_STATE, "import: particle weight not finite");
      for (int k = 0; k < 5; ++k) m[k] += w * px[base + (size_t)k * np + q];
    }
    for (int q = 0; q < np; ++q) {
      const double w = std::exp(px[base + 5 * (size_t)np + q]);
      int k = 0;
      for (int i = 0; i < 5; ++i)
        for (int j = i; j < 5; ++j, ++k)
          C2[k] += w * (px[base + (size_t)i * np + q] - m[i]) * (px[base + (size_t)j * np + q] - m[j]);
    }
    for (int k = 0; k < 5; ++k) {
      if (!std::isfinite(m[k])) return fail(h, GLMB_E_STATE, "import: particle not finite");
      mh[mh.size() - 5 + k] = (float)m[k];
      ml[ml.size() - 5 + k] = 0.f;
    }
    for (int k = 0; k < 15; ++k) cv.push_back((float)C2[k]);
  }
  const int nc = (int)lk.size();
  if (nc > h->cap_comp) return fail(h, GLMB_E_CAPACITY, "import: components exceed capacity");
  CU(cudaStreamSynchronize(h->stream));
  const CompTable& A = h->comps[h->cur];
  if (nc > 0) {
    std::vector<float> col(nc);
    for (int a = 0; a < dx; ++a) {
      for (int c = 0; c < nc; ++c) col[c] = mh[(size_t)c * dx + a];
      CU(cudaMemcpyAsync(A.mhi + (size_t)a * A.cap, col.data(), nc * 4, cudaMemcpyHostToDevice, h->stream));
      for (int c = 0; c < nc; ++c) col[c] = ml[(size_t)c * dx + a];
      CU(cudaMemcpyAsync(A.mlo + (size_t)a * A.cap, col.data(), nc * 4, cudaMemcpyHostToDevice, h->stream));
    }
    for (int k = 0; k < ncov; ++k) {
      for (int c = 0; c < nc; ++c) col[c] = cv[(size_t)c * ncov + k];
      CU(cudaMemcpyAsync(A.cov + (size_t)k * A.cap, col.data(), nc * 4, cudaMemcpyHostToDevice, h->stream));
    }
    CU(cudaMemcpyAsync(A.lk, lk.data(), nc * 4, cudaMemcpyHostToDevice, h->stream));
    CU(cudaMemcpyAsync(A.lb, lb.data(), nc * 4, cudaMemcpyHostToDevice, h->stream));
    if (np) CU(cudaMemcpyAsync(A.px, px.data(), px.size() * 8, cudaMemcpyHostToDevice, h->stream));
  }
  const HypTable& Y = h->hyps[h->hcur];
  CU(cudaMemcpyAsync(Y.ptr, ptr.data(), ptr.size() * 4, cudaMemcpyHostToDevice, h->stream));
  if (hd.n_tracks > 0) CU(cudaMemcpyAsync(Y.comp, comp.data(), (size_t)hd.n_tracks * 4, cudaMemcpyHostToDevice, h->stream));
  CU(cudaMemcpyAsync(Y.logw, logw.data(), logw.size() * 8, cudaMemcpyHostToDevice, h->stream));
  CU(cudaMemcpyAsync(Y.uid, uid.data(), uid.size() * 8, cudaMemcpyHostToDevice, h->stream));
  // the copies read host vectors of this call: complete before returning
  CU(cudaStreamSynchronize(h->stream));
  h->n_comp = nc;
  h->H = hd.n_hyp;
  h->n_entries = hd.n_tracks;
  h->alive_max = 0;
  for (int y = 0; y < hd.n_hyp; ++y) h->alive_max = std::max(h->alive_max, (int)(ptr[y + 1] - ptr[y]));
  h->frame = hd.frame;
  h->stage = 0;
  h->have_update = false;
  h->theta_M_valid = false;
  h->retained_valid = false;
  ++h->gen;
  return GLMB_OK;
}

glmb_status glmb_get_hypotheses(glmb_handle* h, double* logw, uint64_t* uid, uint32_t* hyp_ptr,
                                uint32_t* label_k, uint32_t* label_b, uint16_t* theta, int cap_h,
                                int64_t cap_entries, int* n_h) {
  if (!h || !n_h) return GLMB_E_INVALID;
  if (h->stage != 0) return fail(h, GLMB_E_STATE, "get_hypotheses: frame in progress");
  CU(cudaStreamSynchronize(h->stream));
  *n_h = h->H;
  if (h->H > cap_h || h->n_entries > cap_entries) return fail(h, GLMB_E_CAPACITY, "get_hypotheses: caps");
  const HypTable& Y = h->hyps[h->hcur];
  const CompTable& A = h->comps[h->cur];
  if (logw) CU(cudaMemcpy(logw, Y.logw, (size_t)h->H * 8, cudaMemcpyDeviceToHost));
  if (uid) CU(cudaMemcpy(uid, Y.uid, (size_t)h->H * 8, cudaMemcpyDeviceToHost));
  if (hyp_ptr) CU(cudaMemcpy(hyp_ptr, Y.ptr, (size_t)(h->H + 1) * 4, cudaMemcpyDeviceToHost));
  if ((label_k || label_b) && h->n_entries > 0) {
    std::vector<uint32_t> comp(h->n_entries), lk(std::max(1, h->n_comp)), lb(std::max(1, h->n_comp));
    CU(cudaMemcpy(comp.data(), Y.comp, comp.size() * 4, cudaMemcpyDeviceToHost));
    CU(cudaMemcpy(lk.data(), A.lk, (size_t)h->n_comp * 4, cudaMemcpyDeviceToHost));
    CU(cudaMemcpy(lb.data(), A.lb, (size_t)h->n_comp * 4, cudaMemcpyDeviceToHost));
    for (long long e = 0; e < h->n_entries; ++e) {
      if (label_k) label_k[e] = lk[comp[e]];
      if (label_b) label_b[e] = lb[comp[e]];
    }
  }
  if (theta && h->theta_M_valid && h->theta_M > 0)
    CU(cudaMemcpy(theta, Y.theta, (size_t)h->H * h->theta_M * 2, cudaMemcpyDeviceToHost));
  return GLMB_OK;
}

glmb_status glmb_get_parents(glmb_handle* h, uint32_t* ptr, uint32_t* comp, int cap_parents,
                             int64_t cap_slots, int* n_parents) {
  if (!h || !n_parents) return GLMB_E_INVALID;
  if (!h->have_update) return fail(h, GLMB_E_STATE, "get_parents: no update");
  CU(cudaStreamSynchronize(h->stream));
  const HypTable& P = h->hyps[h->par_buf];
  const int H = h->H_par;
  *n_parents = H;
  std::vector<uint32_t> p(H + 1);
  CU(cudaMemcpy(p.data(), P.ptr, (H + 1) * 4, cudaMemcpyDeviceToHost));
  const long long total = (long long)p[H] + (long long)H * h->nb;
  if (H > cap_parents || total > cap_slots) return fail(h, GLMB_E_CAPACITY, "get_parents: caps");
  std::vector<uint32_t> c(std::max<uint32_t>(1, p[H]));
  if (p[H]) CU(cudaMemcpy(c.data(), P.comp, (size_t)p[H] * 4, cudaMemcpyDeviceToHost));
  long long o = 0;
  for (int y = 0; y < H; ++y) {
    if (ptr) ptr[y] = (uint32_t)o;
    for (uint32_t j = p[y]; j < p[y + 1]; ++j, ++o)
      if (comp) comp[o] = c[j];
    for (int b = 0; b < h->nb; ++b, ++o)
      if (comp) comp[o] = (uint32_t)(h->birth_base + b);
  }
  if (ptr) ptr[H] = (uint32_t)o;
  return GLMB_OK;
}


glmb_status glmb_get_components(glmb_handle* h, uint32_t* label_k, uint32_t* label_b,
                                double* mean, double* cov, double* p, double* dprob,
                                double* logdetS, int cap, int* n_comp) {
  if (!h || !n_comp) return GLMB_E_INVALID;
  if (!h->have_update) return fail(h, GLMB_E_STATE, "get_components: no update");
  CU(cudaStreamSynchronize(h->stream));
  const int T = h->T_work, dx = h->md.dx, ncov = h->md.ncov;
  *n_comp = T;
  if (T > cap) return fail(h, GLMB_E_CAPACITY, "get_components: cap");
  if (T == 0) return GLMB_OK;
  const CompTable& B = h->comps[1 - h->cur];
  std::vector<float> f(T);
  auto col = [&](const float* src) -> glmb_status {
    CU(cudaMemcpy(f.data(), src, (size_t)T * 4, cudaMemcpyDeviceToHost));
    return GLMB_OK;
  };
  if (label_k) CU(cudaMemcpy(label_k, B.lk, (size_t)T * 4, cudaMemcpyDeviceToHost));
  if (label_b) CU(cudaMemcpy(label_b, B.lb, (size_t)T * 4, cudaMemcpyDeviceToHost));
  if (mean) {
    std::vector<float> lo(T);
    for (int a = 0; a < dx; ++a) {
      if (col(B.mhi + (size_t)a * B.cap) != GLMB_OK) return GLMB_E_CUDA;
      CU(cudaMemcpy(lo.data(), B.mlo + (size_t)a * B.cap, (size_t)T * 4, cudaMemcpyDeviceToHost));
      for (int c = 0; c < T; ++c) mean[(size_t)c * dx + a] = (double)f[c] + (double)lo[c];
    }
  }
  if (cov) {
    for (int i = 0; i < dx; ++i)
      for (int k = i; k < dx; ++k) {
        if (col(B.cov + (size_t)pidx(dx, i, k) * B.cap) != GLMB_OK) return GLMB_E_CUDA;
        for (int c = 0; c < T; ++c)
          cov[(size_t)c * dx * dx + i * dx + k] = cov[(size_t)c * dx * dx + k * dx + i] = f[c];
      }
  }
  if (p) {
    if (col(B.logp) != GLMB_OK) return GLMB_E_CUDA;
    for (int c = 0; c < T; ++c) p[c] = std::exp((double)f[c]);
  }
  if (dprob) {
    if (col(h->pt.dprob) != GLMB_OK) return GLMB_E_CUDA;
    for (int c = 0; c < T; ++c) dprob[c] = f[c];
  }
  if (logdetS) {
    if (col(h->pt.logdetS) != GLMB_OK) return GLMB_E_CUDA;
    for (int c = 0; c < T; ++c) logdetS[c] = f[c];
  }
  (void)ncov;
  return GLMB_OK;
}

glmb_status glmb_get_pairs(glmb_handle* h, uint32_t* comp_ptr, uint32_t* meas, float* logC,
                           float* q, float* e, int cap_comp, int64_t cap_pairs, int64_t* n_pairs) {
  if (!h || !n_pairs) return GLMB_E_INVALID;
  if (!h->have_update) return fail(h, GLMB_E_STATE, "get_pairs: no update");
  CU(cudaStreamSynchronize(h->stream));
  const int T = h->T_work, dz = h->md.dz;
  uint32_t K32 = 0;
  CU(cudaMemcpy(&K32, h->pt.ptr + T, sizeof K32, cudaMemcpyDeviceToHost));
  const long long K = std::min<long long>(K32, h->cap_pairs);
  *n_pairs = K;
  if (T + 1 > cap_comp || K > cap_pairs) return fail(h, GLMB_E_CAPACITY, "get_pairs: caps");
  if (comp_ptr) CU(cudaMemcpy(comp_ptr, h->pt.ptr, (size_t)(T + 1) * 4, cudaMemcpyDeviceToHost));
  if (K == 0) return GLMB_OK;
  if (meas) CU(cudaMemcpy(meas, h->pt.meas, (size_t)K * 4, cudaMemcpyDeviceToHost));
  if (logC) CU(cudaMemcpy(logC, h->pt.logC, (size_t)K * 4, cudaMemcpyDeviceToHost));
  if (q) CU(cudaMemcpy(q, h->pt.q, (size_t)K * 4, cudaMemcpyDeviceToHost));
  if (e)
    for (int a = 0; a < dz; ++a) {
      std::vector<float> col(K);
      CU(cudaMemcpy(col.data(), h->pt.e + (size_t)a * h->cap_pairs, (size_t)K * 4, cudaMemcpyDeviceToHost));
      for (long long j = 0; j < K; ++j) e[j * dz + a] = col[j];
    }
  return GLMB_OK;
}

glmb_status glmb_get_children(glmb_handle* h, double* logw, int8_t* status, uint16_t* n_alive,
                              int64_t cap, int64_t* n_children) {
  if (!h || !n_children) return GLMB_E_INVALID;
  if (!h->have_update) return fail(h, GLMB_E_STATE, "get_children: no update");
  CU(cudaStreamSynchronize(h->stream));
  const long long n = (long long)h->H_par * h->cfg.h_up;
  *n_children = n;
  if (n > cap) return fail(h, GLMB_E_CAPACITY, "get_children: cap");
  if (logw) {
    std::vector<long long> k(n);
    CU(cudaMemcpy(k.data(), h->child_key, (size_t)n * 8, cudaMemcpyDeviceToHost));
    for (long long j = 0; j < n; ++j)
      logw[j] = k[j] == kKeyInvalid ? -INFINITY : (double)k[j] * kFxInv;
  }
  if (status) CU(cudaMemcpy(status, h->child_status, (size_t)n, cudaMemcpyDeviceToHost));
  if (n_alive) CU(cudaMemcpy(n_alive, h->child_alive, (size_t)n * 2, cudaMemcpyDeviceToHost));
  return GLMB_OK;
}

// ---------------------------------------------------------------------------
// learned pair gate
// ---------------------------------------------------------------------------
glmb_status glmb_set_gate(glmb_handle* h, const float* params, float threshold, int mode) {
  if (!h) return GLMB_E_INVALID;
  if (h->md.particle && mode != GLMB_GATE_OFF)
    return fail(h, GLMB_E_INVALID, "set_gate: the learned gate takes Gaussian features (track model 0)");
  if (mode != GLMB_GATE_OFF && mode != GLMB_GATE_PRUNE && mode != GLMB_GATE_SCORE)
    return fail(h, GLMB_E_INVALID, "set_gate: unknown mode %d", mode);
  if (mode != GLMB_GATE_OFF) {
    if (!params) return fail(h, GLMB_E_INVALID, "set_gate: no parameters");
    for (int i = 0; i < GLMB_GATE_NPARAM; ++i)
      if (!std::isfinite(params[i])) return fail(h, GLMB_E_INVALID, "set_gate: parameter %d is not finite", i);
    for (int j = 0; j < 5; ++j)
      if (!(params[kGateSd + j] > 0.f)) return fail(h, GLMB_E_INVALID, "set_gate: sd[%d] <= 0", j);
    if (std::isnan(threshold)) return fail(h, GLMB_E_INVALID, "set_gate: threshold is NaN");
  }
  CU(cudaStreamSynchronize(h->stream));
  const int dz = h->md.dz;
  if (mode != GLMB_GATE_OFF && !h->gate_params) {
    if (!(dalloc(h, &h->gate_params, GLMB_GATE_NPARAM) && dalloc(h, &h->gate_keep, h->cap_pairs) &&
          dalloc(h, &h->gate_logit, h->cap_pairs)))
      return fail(h, GLMB_E_OOM, "set_gate: gate buffers");
  }
  if (mode == GLMB_GATE_PRUNE && !h->pt_full.ptr) {
    PairTable& F = h->pt_full;
    if (!(dalloc(h, &F.cnt, h->cap_comp + 1) && dalloc(h, &F.ptr, h->cap_comp + 1) &&
          dalloc(h, &F.meas, h->cap_pairs) && dalloc(h, &F.logC, h->cap_pairs) && dalloc(h, &F.q, h->cap_pairs) &&
          dalloc(h, &F.e, h->cap_pairs * dz) && dalloc(h, &F.dthr, h->cap_comp) &&
          dalloc(h, &F.dprob, h->cap_comp))) {
      F.ptr = nullptr;
      return fail(h, GLMB_E_OOM, "set_gate: second pair table");
    }
    F.logdetS = h->pt.logdetS;
    F.cap_pairs = h->cap_pairs;
    F.slm = h->pt.slm;
    F.sln = h->pt.sln;
    F.slm_cap = h->pt.slm_cap;
  }
  if (mode != GLMB_GATE_OFF) {
    CU(cudaMemcpyAsync(h->gate_params, params, GLMB_GATE_NPARAM * sizeof(float), cudaMemcpyHostToDevice,
                       h->stream));
    CU(cudaStreamSynchronize(h->stream));
  }
  if (mode != h->gate_mode) {
    // captured frame graphs were built for the other table path
    for (auto& g : h->graphs) drop_graph(g);
    h->graphs.clear();
  }
  h->gate_mode = mode;
  h->gate_thr = threshold;
  return GLMB_OK;
}

namespace {
// the table of the last update before the learned gate
const PairTable& pregate_table(const glmb_handle* h) {
  return h->gate_mode_frame == GLMB_GATE_PRUNE ? h->pt_full : h->pt;
}
}  // namespace

glmb_status glmb_gate_features(glmb_handle* h, float* X, int64_t cap, int64_t* n) {
  if (!h || !n || (cap > 0 && !X)) return GLMB_E_INVALID;
  if (!h->have_update) return fail(h, GLMB_E_STATE, "gate_features: no update");
  CU(cudaStreamSynchronize(h->stream));
  const PairTable& P0 = pregate_table(h);
  uint32_t K32 = 0;
  CU(cudaMemcpy(&K32, P0.ptr + h->T_work, sizeof K32, cudaMemcpyDeviceToHost));
  *n = K32;
  if ((int64_t)K32 > cap) return fail(h, GLMB_E_CAPACITY, "gate_features: %u pairs, cap %lld", K32, (long long)cap);
  if (K32 == 0) return GLMB_OK;
  if (!h->gate_X && !dalloc(h, &h->gate_X, h->cap_pairs * 5)) return fail(h, GLMB_E_OOM, "gate_features: scratch");
  launch_gate_features(h->md, h->comps[1 - h->cur], P0, h->d_fs, h->gate_X, h->cap_pairs, 2 * h->n_sm, h->stream);
  CU(cudaMemcpyAsync(X, h->gate_X, (size_t)K32 * 5 * sizeof(float), cudaMemcpyDeviceToHost, h->stream));
  CU(cudaStreamSynchronize(h->stream));
  return GLMB_OK;
}

glmb_status glmb_gate_logits(glmb_handle* h, float* logit, int64_t cap, int64_t* n) {
  if (!h || !n || (cap > 0 && !logit)) return GLMB_E_INVALID;
  if (!h->have_update || h->gate_mode_frame == GLMB_GATE_OFF)
    return fail(h, GLMB_E_STATE, "gate_logits: no update with the gate on");
  CU(cudaStreamSynchronize(h->stream));
  uint32_t K32 = 0;
  CU(cudaMemcpy(&K32, pregate_table(h).ptr + h->T_work, sizeof K32, cudaMemcpyDeviceToHost));
  *n = K32;
  if ((int64_t)K32 > cap) return fail(h, GLMB_E_CAPACITY, "gate_logits: cap");
  if (K32) CU(cudaMemcpy(logit, h->gate_logit, (size_t)K32 * sizeof(float), cudaMemcpyDeviceToHost));
  return GLMB_OK;
}

glmb_status glmb_gate_usage(glmb_handle* h, uint8_t* used, int64_t cap_pairs, uint8_t* hyp_flag, int cap_h,
                            int64_t* n_pairs, int* n_hyp) {
  if (!h || !n_pairs || !n_hyp) return GLMB_E_INVALID;
  if (!h->retained_valid || !h->theta_M_valid || !h->have_update)
    return fail(h, GLMB_E_STATE, "gate_usage: no pruned frame");
  if (h->gate_mode_frame == GLMB_GATE_PRUNE) return fail(h, GLMB_E_STATE, "gate_usage: the gate pruned the table");
  CU(cudaStreamSynchronize(h->stream));
  uint32_t K32 = 0;
  CU(cudaMemcpy(&K32, h->pt.ptr + h->T_work, sizeof K32, cudaMemcpyDeviceToHost));
  *n_pairs = K32;
  *n_hyp = h->H;
  if ((used && (int64_t)K32 > cap_pairs) || (hyp_flag && h->H > cap_h))
    return fail(h, GLMB_E_CAPACITY, "gate_usage: arrays too short");
  if (!h->gate_used && !(dalloc(h, &h->gate_used, h->cap_pairs) && dalloc(h, &h->gate_hflag, h->cap_h)))
    return fail(h, GLMB_E_OOM, "gate_usage: scratch");
  CU(cudaMemsetAsync(h->gate_used, 0, std::max<size_t>(K32, 1), h->stream));
  CU(cudaMemsetAsync(h->gate_hflag, 0, std::max(h->H, 1), h->stream));
  const int capT = std::max(1, (int)h->h_scal[S_MAXT]);
  const bool score = h->gate_mode_frame == GLMB_GATE_SCORE;
  launch_gate_usage(h->hyps[h->par_buf], h->hyps[h->hcur], h->comps[h->cur], h->comps[1 - h->cur], h->pw.surv_idx,
                    h->H, h->cfg.h_up, h->theta_M, h->pt, h->d_fs, score ? h->gate_logit : nullptr, h->gate_thr,
                    h->gate_used, h->gate_hflag, capT, std::max(1, std::min(h->H, 8 * h->n_sm)), h->stream);
  if (used && K32) CU(cudaMemcpyAsync(used, h->gate_used, K32, cudaMemcpyDeviceToHost, h->stream));
  if (hyp_flag && h->H) CU(cudaMemcpyAsync(hyp_flag, h->gate_hflag, (size_t)h->H, cudaMemcpyDeviceToHost, h->stream));
  CU(cudaStreamSynchronize(h->stream));
  return GLMB_OK;
}

glmb_status glmb_mlp_forward(const float* params, const float* X, int64_t n, float* logit, uint32_t* err,
                             void* stream) {
  if (n < 0 || !params || !err || (n > 0 && (!X || !logit))) return GLMB_E_INVALID;
  if (n == 0) return GLMB_OK;
  int dev = 0, n_sm = 1;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev);
  const long long tiles = (n + 127) / 128;
  const int grid = (int)std::max(1LL, std::min(tiles, 4LL * n_sm));
  launch_gate_forward_rows(params, X, n, logit, err, grid, (cudaStream_t)stream);
  return cudaGetLastError() == cudaSuccess ? GLMB_OK : GLMB_E_CUDA;
}

glmb_status glmb_mlp_backward(const float* params, const float* X, const float* y, const float* wt, int64_t n,
                              float* grad, double* loss, uint32_t* err, void* stream) {
  if (n < 0 || !params || !grad || !loss || !err || (n > 0 && (!X || !y || !wt))) return GLMB_E_INVALID;
  cudaStream_t s = (cudaStream_t)stream;
  if (cudaMemsetAsync(grad, 0, GLMB_GATE_NPARAM * sizeof(float), s) != cudaSuccess ||
      cudaMemsetAsync(loss, 0, sizeof(double), s) != cudaSuccess)
    return GLMB_E_CUDA;
  if (n == 0) return GLMB_OK;
  int dev = 0, n_sm = 1;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev);
  const long long tiles = (n + 127) / 128;
  launch_gate_train(params, X, y, wt, n, grad, loss, err, (int)std::max(1LL, std::min(tiles, (long long)n_sm)), s);
  return cudaGetLastError() == cudaSuccess ? GLMB_OK : GLMB_E_CUDA;
}

glmb_status glmb_mlp_adam(float* params, const float* grad, float* m, float* v, int step, float lr, float beta1,
                          float beta2, float eps, void* stream) {
  if (!params || !grad || !m || !v || step < 1) return GLMB_E_INVALID;
  launch_gate_adam(params, grad, m, v, step, lr, beta1, beta2, eps, (cudaStream_t)stream);
  return cudaGetLastError() == cudaSuccess ? GLMB_OK : GLMB_E_CUDA;
}

}  // extern "C"

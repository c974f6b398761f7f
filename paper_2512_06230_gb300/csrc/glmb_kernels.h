// Host-side launch functions of the GLMB kernels (one GPU, one stream).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "glmb_dev.cuh"

namespace glmb {

// kernels launched by this library (all handles), for the benchmark's count
extern long long g_launches;

// Launches kernel k with programmatic stream serialisation: its blocks may
// start while the previous kernel in the stream finishes; every kernel of
// the library begins with pdl_enter(), which waits for that kernel first.
template <typename... KArgs, typename... Args>
inline void launch_k(void (*k)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t s,
                     Args... args) {
  cudaLaunchConfig_t cfg{};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  cudaLaunchKernelEx(&cfg, k, static_cast<KArgs>(args)...);
  ++g_launches;
}

// ---- prediction, births, table (kernels_table.cu) ----
// Sizes come from the device FrameDev; grid is the number of blocks of a
// grid-stride launch.
// prediction of fs->n_comp components from src into dst, then fs->nb births
// appended at dst[n_comp..) (births_dev: per birth [r, mean[6], cov[36]] FP64)
void launch_predict(const Model& md, const CompTable& src, const CompTable& dst, const FrameDev* fs,
                    const double* births_dev, int grid, cudaStream_t s);
// detections: fs->Z ([M][dz] floats on the device); the count kernel also
// sets kErrInput in *err when a detection coordinate is not finite
void launch_table_count(const Model& md, const CompTable& ct, const PairTable& pt,
                        const FrameDev* fs, unsigned* err, int grid, cudaStream_t s);
void launch_table_write(const Model& md, const CompTable& ct, const PairTable& pt,
                        const FrameDev* fs, unsigned* n_fp64, unsigned* err, int grid, cudaStream_t s);
void launch_parent_stats(const HypTable& hp, const FrameDev* fs, const PairTable& pt,
                         unsigned* max_T, unsigned* max_K, int grid, cudaStream_t s);

// exclusive scans of (*n_dev * mult) elements, at most cap, in one launch;
// tmp holds scan_tmp_elems(tmp_cap) elements (tmp_cap >= cap; one work area
// may serve scans of different capacities), zero before the first scan (each
// scan leaves it zero); total (nullable) receives the sum, and with
// total_at_end the sum is also written to out[n]; a look-back that waits too
// long sets kErrTimeout in *err
long long scan_tmp_elems(long long cap);
void scan_u32(const uint32_t* in, uint32_t* out, const int* n_dev, int mult, long long cap,
              uint32_t* total, bool total_at_end, uint32_t* tmp, long long tmp_cap, unsigned* err,
              cudaStream_t s);
void scan_u64(const unsigned long long* in, unsigned long long* out, const int* n_dev, int mult,
              long long cap, unsigned long long* total, bool total_at_end,
              unsigned long long* tmp, long long tmp_cap, unsigned* err, cudaStream_t s);

// A birth record on the device (FP64): r, mean[6], cov[36] (dim_x x dim_x
// row-major), and for the particle model the lower Cholesky factor of the
// 5 x 5 covariance, packed row-major, at kBirthChol (computed by the host,
// which refuses a covariance that is not positive definite).
constexpr int kBirthChol = 43;
constexpr int kBirthRec = 58;

// ---- particle track model (kernels_particle.cu) ----
// prediction of the working table: survivors' particles take a CTRV step,
// births are sampled from their Gaussian (a flat grid over components x
// particles), then the particles' moments (one warp per component); also
// writes the labels and existences
void launch_particle_predict(const Model& md, const PartModel& pm, const CompTable& src, const CompTable& dst,
                             const FrameDev* fs, const double* births_dev, int grid, cudaStream_t s);
// log C of every gated pair from the particles, then the death probability
// (after launch_table_write, which wrote the pairs)
void launch_particle_logc(const Model& md, const PartModel& pm, const CompTable& ct, const PairTable& pt,
                          const FrameDev* fs, int grid, cudaStream_t s);
// the regeneration's component work: kept components copied to their
// compacted positions, each distinct update's particle update (with
// resampling) after them; launch_gc_remap does the index remap
void launch_particle_remap(const Model& md, const PartModel& pm, const CompTable& src, const CompTable& dst,
                           const uint32_t* newpos, const uint32_t* flag, const FrameDev* fs,
                           const unsigned* n_keep_dev, const uint32_t* upd_src, const uint32_t* upd_m,
                           const long long* upd_se, int cap_upd, const unsigned* n_upd_dev,
                           const unsigned* n_surv_dev, unsigned* err, int grid, cudaStream_t s);
int particle_remap_smem(int np);

// ---- expansion / materialisation (kernels_expand.cu) ----
// Test hook of the bounded device-side waits (glmb_set_wait_test): mode 0
// runs with the normal limits; kWaitTestScan makes the first tile of every
// one-pass scan withhold its prefix, kWaitTestGate makes the gate's forward
// pass issue no tensor-core work for the first tile of its CTA 0, and in
// both the wait gives up after `limit` (polls for the scan, SM clock cycles
// for the gate).
struct WaitTest {
  int mode;
  long long limit;
};
constexpr int kWaitTestScan = 1, kWaitTestGate = 2;
constexpr long long kScanSpinLimit = 1LL << 22;        // look-back polls
constexpr long long kGateWaitLimit = 2000000000LL;     // SM clock cycles (about a second)
WaitTest wait_test();
void set_wait_test(WaitTest w);

struct ExpandArgs {
  Model md;
  CompTable ct;           // working (predicted) table
  PairTable pt;
  HypTable parents;       // hypotheses before the update
  const FrameDev* fs;     // H, M, births, frame
  // plan: largest slots, gated pairs and detections per parent (a parent
  // beyond it sets kErrSlots and the frame is redone with a larger plan)
  int T_max, K_max, M_plan;
  // per-parent images: parent h at img + h * img_stride
  unsigned char* img;
  long long img_stride;
  int stage_smem;         // staged in shared memory (else in the image itself)
  int warp_all;           // warp kernel: every child of every parent (else the overflow list)
  uint32_t* redo_list;    // children the draw kernel could not take
  unsigned* redo_count;
  unsigned* stage_next;   // staging: next parent to take (zero at the launch)
  int stage_tail;         // staging in global memory: what it keeps in shared memory (expand_stage_tail_bytes)
  int warp_group;         // warp kernel: warps per child (1, 2, 4 or 8; a CTA holds whole groups)
  // expansion outputs
  long long* child_key;   // [H * h_up] fixed-point log-weight or kKeyInvalid
  unsigned long long* child_hash;   // [H * h_up] order-free key of (deaths, associations)
  int8_t* child_status;   // 0 zero weight, 1 unique, 2 duplicate
  uint16_t* child_alive;  // surviving tracks
  // materialisation inputs / outputs
  int materialize;
  const long long* surv_idx;   // [n_surv] child index h*h_up + n, ascending
  const unsigned* n_surv;      // device count of survivors
  const uint32_t* out_ptr;     // [n_surv + 1]
  uint32_t* out_comp;          // entries: component index, or kNewTag | hash slot
  uint16_t* out_theta;         // [n_surv][M]
  unsigned long long* hkeys;   // hash table of (component, detection set) keys
  uint32_t* hvals;             // slot -> update id
  uint32_t hmask;
  uint32_t* upd_src;           // update id -> source component
  uint32_t* upd_m;             // update id -> |W|
  long long* upd_se;           // [dz][cap_upd] fixed-point sum of innovations
  uint32_t* upd_count;
  uint32_t* upd_slot;          // update id -> its hash slot (cleared by the next frame's reset)
  int cap_upd;
  uint32_t* gc_flag;           // [T] set for old components the new hypotheses keep
  unsigned* err;
  // largest slot and gated-pair counts over the staged parents (staging
  // records them for the next frame's plan and for a redo)
  unsigned* max_T;
  unsigned* max_K;
  // Philox key of the frame, (seed_lo, seed_hi ^ frame): a launch parameter,
  // so that the round keys are the same for every thread and stay out of
  // the per-thread registers (a replayed frame graph has it set per frame)
  uint32_t key_x, key_y;
};
// bytes of one parent's image (the staging kernel's shared memory when it
// stages there)
int expand_image_bytes(int dz, int T_max, int K_max, int M);
// shared memory the staging kernel needs beside (or, with the image in
// global memory, instead of) the image: next-parent word, scan sums, and
// the arrays it reads back many times when the image is in global memory
// (mode: 0 the two words only, 1 with the row offsets, 2 with every listed
// array; the image in shared memory takes mode 0)
int expand_stage_tail_bytes(int dz, int T_plan, int K_plan, int M_plan, int mode);
// shared memory of a draw-kernel CTA of `threads` threads
int expand_draw_smem(int threads);
// shared memory of a warp-kernel CTA of `warps` warps
int expand_warp_smem(int dz, int materialize, int T_max, int warps, int grp = 0);
enum class ExpandKernel { kStage, kDraw, kWarp, kMatPrep };
// resident CTAs per SM of one of the kernels
int expand_occupancy(const ExpandArgs& a, ExpandKernel k, int threads, int smem);
// allows the expansion kernels the device's opt-in shared memory (call once)
void expand_init(int smem_limit);
// stage: persistent CTAs over parents; draw: persistent over (parent, slice
// of blockDim draws); warp: persistent warps over a list of children;
// mat_prep: one warp per retained parent
void launch_expand_kernel(const ExpandArgs& a, ExpandKernel k, int grid, int threads, int smem,
                          cudaStream_t s);
// warps per CTA of the warp kernel (at most max_warps) that keep the most
// warps resident on an SM, for per-parent slot counts up to T (0: none fits)
int expand_warp_best_cta(int dz, int materialize, int T, int max_warps, int smem_limit);
// whether a kernel of a captured graph takes the frame's Philox key in its
// ExpandArgs (the draw and warp kernels)
bool expand_kernel_takes_key(const void* fn);
// clears the hash slots of the n_prev updates recorded in upd_slot (the
// previous materialisation's), instead of clearing the whole table, and
// zeroes the insert counter n_cur
void launch_hash_reset(unsigned long long* hkeys, const uint32_t* upd_slot, const unsigned* n_prev, int cap_upd,
                       unsigned* n_cur, int grid, cudaStream_t s);
struct PruneWork;
// marks duplicate children (status 2, key dropped), one block per parent
// and writes the log-sum-exp partial of its unique children per block
// (w.part_*; grid <= kMaxLseParts)
void launch_dedup(const FrameDev* fs, int HU, long long* child_key, const unsigned long long* child_hash,
                  int8_t* child_status, const unsigned* err, const PruneWork& w, int grid, cudaStream_t s);

// ---- normalisation, truncation, track update, estimates (kernels_prune.cu) ----
struct PruneWork {
  long long* blk_max;           // per-block partials
  double* blk_sum;
  unsigned* blk_done;           // last-block counters [4]
  double* lse;                  // [2]: LSE over unique children, LSE over retained
  long long* thr;               // fixed-point threshold log(tau) + LSE
  unsigned* hist;               // [4096]
  long long* sel;               // [4]: prefix, need, boundary key, flags
  unsigned long long* flags;    // [n_children] packed (gt, eq) prefix counts
  unsigned long long* flags_tmp;
  long long flags_tmp_cap;      // capacity flags_tmp was sized for
  long long* surv_idx;          // [cap_h]
  unsigned* counts;             // [8]: n_surv, n_entries, n_unique, max alive, [4..5] scan total
  unsigned* err;                // device error flags
  // log-sum-exp partials of the unique children, one per block of the
  // duplicate-marking kernel (kMaxLseParts at most): maximum key, sum of
  // exp(key - maximum), count
  long long* part_max;
  double* part_sum;
  unsigned* part_cnt;
};
constexpr int kMaxLseParts = 4096;
// the children are the fs->H * h_up entries of keys
void launch_lse(const long long* keys, const FrameDev* fs, int h_up, PruneWork w, double log_tau,
                int h_max, int nblk, cudaStream_t s);
void launch_select(const long long* keys, const FrameDev* fs, int h_up, int nbits, PruneWork w,
                   int nblk, cudaStream_t s);
void launch_compact(const long long* keys, const FrameDev* fs, int h_up, long long cap, PruneWork w,
                    int h_max, int nblk, cudaStream_t s);
// the whole of launch_lse + launch_select + launch_compact + launch_finalize
// in one launch of a thread-block cluster (select_cluster.cu); false when
// the device cannot run the cluster (the caller then launches the chain)
// (n_part: the duplicate-marking kernel's log-sum-exp partials)
bool launch_select_cluster(const long long* keys, const FrameDev* fs, int h_up, PruneWork w, int n_part,
                           double log_tau, int h_max, int nbits, const uint16_t* child_alive,
                           const HypTable& parents, const HypTable& out, unsigned* err, long long cap_entries,
                           cudaStream_t s);
// cluster size the fused selection runs with (0: cannot run)
int select_cluster_size();
void launch_finalize(PruneWork w, const long long* keys, const uint16_t* child_alive,
                     const HypTable& parents, int h_up, HypTable out, int h_max,
                     unsigned* err, long long cap_entries, cudaStream_t s);
// components of the new state into dst: every flagged old component c
// copied to newpos[c], then the distinct track updates (Kalman) after the
// n_keep kept ones; in the same launch the new hypothesis table's component
// indices out_comp[0 .. *n_entries_dev) are remapped, an old component c
// to newpos[c] and a new one (kNewTag | hash slot) to n_keep + hvals[slot]
void launch_gc_remap(const Model& md, const CompTable& src, const CompTable& dst, const uint32_t* newpos,
                     const uint32_t* flag, const FrameDev* fs, const unsigned* n_keep_dev, const uint32_t* upd_src,
                     const uint32_t* upd_m, const long long* upd_se, int cap_upd, const unsigned* n_upd_dev,
                     const unsigned* n_surv_dev, unsigned* err, uint32_t* out_comp, const unsigned* n_entries_dev,
                     long long cap_entries, const uint32_t* hvals, uint32_t hmask, unsigned* n_upd_prev, int grid,
                     cudaStream_t s);
// device error flags that abandon a frame (state left untouched)
constexpr unsigned kErrFatal = kErrPairs | kErrHash | kErrUpdates | kErrComps | kErrNumeric |
                               kErrEntries | kErrSlots | kErrInput | kErrGate | kErrTimeout | kErrChkSurv |
                               kErrChkComp | kErrChkRemap;

// ---- learned pair gate (gate_mlp.cu) ----
// parameter vector (floats): W1[64][5] b1[64] W2[64][64] b2[64] W3[64][64]
// b3[64] w4[64] b4 mu[5] sd[5]; the first kGateNTrain are trained
constexpr int kGateW1 = 0, kGateB1 = 320, kGateW2 = 384, kGateB2 = 4480, kGateW3 = 4544,
              kGateB3 = 8640, kGateW4 = 8704, kGateB4 = 8768, kGateMu = 8769, kGateSd = 8774;
constexpr int kGateNParam = 8779, kGateNTrain = 8769;
int gate_forward_smem();
int gate_train_smem();
// logits of n raw feature rows X[n][5] (persistent grid, 128 rows per tile)
void launch_gate_forward_rows(const float* P, const float* X, long long n, float* logit, unsigned* err,
                              int grid, cudaStream_t s);
// logits and keep flags (logit >= thr) of every pair of the table `full`
void launch_gate_forward_table(const float* P, float thr, const Model& md, const CompTable& ct,
                               const PairTable& full, const FrameDev* fs, float* logit, uint8_t* keep,
                               unsigned* err, int grid, cudaStream_t s);
// adds the gradient of sum wt (softplus(z) - y z) to grad and the loss to *loss
void launch_gate_train(const float* P, const float* X, const float* y, const float* wt, long long n,
                       float* grad, double* loss, unsigned* err, int grid, cudaStream_t s);
void launch_gate_adam(float* P, const float* G, float* m, float* v, int t, float lr, float b1, float b2,
                      float eps, cudaStream_t s);
// raw features of the pairs of table pt into X (at most cap rows)
void launch_gate_features(const Model& md, const CompTable& ct, const PairTable& pt, const FrameDev* fs,
                          float* X, long long cap, int grid, cudaStream_t s);
// count = true: kept pairs per component into gated.cnt; false: stable
// compaction into gated (whose ptr is the scan of cnt) and death probabilities
void launch_gate_compact(const Model& md, const CompTable& ct, const PairTable& full, const uint8_t* keep,
                         const PairTable& gated, const FrameDev* fs, bool count, int grid, cudaStream_t s);
// pairs of table pt used by the H_new retained hypotheses `out` (children
// surv[j] of parents `par`; A the new state's components, B the predicted
// ones; capT >= the largest retained track count), and per retained
// hypothesis whether it uses a pair with logit < thr (logit nullable)
void launch_gate_usage(const HypTable& par, const HypTable& out, const CompTable& A, const CompTable& B,
                       const long long* surv, int H_new, int h_up, int M, const PairTable& pt, const FrameDev* fs,
                       const float* logit, float thr, uint8_t* used, uint8_t* hflag, int capT, int grid,
                       cudaStream_t s);

// estimates: pmf[pcap], nb = {n_hat, MAP hypothesis}, tracks =
// glmb_track[pcap]; r_comp[ct.cap] (per-component weight sums), r_map[pcap]
// (per-track sums), cmax and done are zeroed work areas, left zeroed;
// H_dev (nullable) gives H on the device, H_bound an upper bound of H (the
// launch shape follows it); err (nullable): the frame's error flags, on
// which the kernels do nothing
void launch_estimates(const HypTable& hp, int H, const unsigned* H_dev, int H_bound, const CompTable& ct, int dx,
                      double* pmf, int pcap, int* nb, unsigned long long* r_comp, unsigned long long* r_map,
                      void* tracks, unsigned* cmax, unsigned* done, int n_sm, const unsigned* err, cudaStream_t s);
void launch_meas_assoc(const HypTable& hp, int H, int M, double* r_u, cudaStream_t s);

}  // namespace glmb

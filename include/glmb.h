/*
 * glmb.h - C ABI of the GB300 (sm_103a) multi-detection GLMB filter update.
 *
 * The method is the GLMB update of arXiv 2512.06230 ("GPU-GLMB"), Section 3:
 * every predicted track is compared with every detection (compatibility
 * matrix, Eq. 2), each retained hypothesis spawns H_up children by two-stage
 * sampling (Bernoulli track deaths, then an independent categorical draw per
 * detection row, possible because an object may yield several detections),
 * each unique child is weighted by its parent's weight times the joint
 * likelihood of its deaths and associations, and the set is truncated to the
 * H_max heaviest hypotheses above a threshold tau and renormalised.  Track
 * densities are Gaussian with a constant-velocity model (the paper uses
 * particles with a turn-rate model; this library uses linear Gaussian
 * tracks).
 *
 * Conventions shared by every call:
 *  - All pointers are host pointers unless the argument name says "device".
 *    The caller owns every buffer it passes; the library copies inputs
 *    before the call returns and writes outputs only on GLMB_OK.
 *  - The handle owns all device memory, from cudaMalloc or the allocation
 *    hook of glmb_config.  glmb_create allocates it from the capacities in
 *    glmb_config, with two exceptions: the per-hypothesis expansion images,
 *    grown by glmb_update / glmb_step when a frame needs more, and the
 *    learned gate's buffers, allocated by glmb_set_gate and the gate's data
 *    calls on first use.  Growth waits for the handle's stream first.
 *  - Work is issued on glmb_config.stream (a cudaStream_t; NULL means a
 *    stream owned by the handle).  glmb_predict only enqueues work (its host
 *    inputs are copied before it returns); glmb_update waits once, for its
 *    expansion, to check the expansion's plan (see glmb_update); glmb_prune
 *    and every call that returns sizes or host data synchronise that stream.
 *  - Host threads: the calls on one handle must not overlap.  The library
 *    also keeps a few process-wide launch settings (kernel shared-memory
 *    limits, the selection's cluster size), set on first use, so handles
 *    are created and stepped from one host thread at a time (the batched
 *    calls run many handles from one thread).
 *  - Call order per frame: glmb_predict -> glmb_update -> glmb_prune ->
 *    any number of glmb_estimates / glmb_meas_assoc / glmb_get_* calls.
 *    A call out of order returns GLMB_E_STATE and changes nothing.
 *  - No call throws or aborts.  On error the status is returned and a
 *    message is kept for glmb_last_error.  A failed glmb_update or
 *    glmb_prune leaves the filter state of the previous frame intact
 *    (call glmb_predict again to retry a frame).
 *  - Labels are (birth frame, birth index) pairs; they are unique within a
 *    hypothesis and persist across frames (Section 3).
 */
#ifndef GLMB_H
#define GLMB_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  GLMB_OK = 0,
  GLMB_E_INVALID = 1,   /* bad argument: null pointer, NaN/Inf input, bad size */
  GLMB_E_OOM = 2,       /* device or host allocation failed in glmb_create */
  GLMB_E_CAPACITY = 3,  /* a size exceeds a capacity fixed at glmb_create */
  GLMB_E_CUDA = 4,      /* a CUDA runtime call failed */
  GLMB_E_NUMERIC = 5,   /* no child has a finite weight, or a covariance lost definiteness */
  GLMB_E_STATE = 6,     /* call out of order, or a malformed state buffer */
  GLMB_E_TIMEOUT = 7    /* a bounded device-side wait ran out */
} glmb_status;

typedef struct glmb_handle glmb_handle;

/* Filter configuration (Section 3 model terms; Section 4.1 tracker
 * parameters H_max, H_up, tau). */
typedef struct {
  int32_t dim_x, dim_z;     /* 4/2 (2-D) or 6/3 (3-D) constant velocity; state
                               [positions, velocities], positions measured */
  float dt;                 /* frame period [s] */
  double q;                 /* white-acceleration power spectral density */
  double R[9];              /* dim_z x dim_z detection covariance, row-major, SPD */
  double p_s;               /* survival probability per frame */
  double p_d;               /* detection probability */
  double lambda_d;          /* a detected object yields 1 + Poisson(lambda_d) detections */
  double clutter_rate;      /* mean clutter detections per frame */
  double volume;            /* surveillance volume; kappa = clutter_rate / volume */
  double gate;              /* Mahalanobis gate on d^2 (INFINITY disables gating) */
  int32_t h_max;            /* hypotheses retained by glmb_prune */
  int32_t h_up;             /* children sampled per hypothesis (<= 65535) */
  double tau;               /* children with normalised weight < tau are dropped */
  uint64_t seed;            /* key of the counter-based random numbers */
  int32_t score_mode;       /* 0: joint likelihood of each track's detections (R3);
                               1: product of the Eq. 2 entries C[i, t] of the chosen
                               associations (the paper's factorised weighting) */
  int32_t max_tracks;       /* capacity: tracks per hypothesis incl. this frame's births */
  int32_t max_meas;         /* capacity: detections per frame (<= 65535) */
  int32_t max_births;       /* capacity: births per frame */
  int64_t max_pairs;        /* capacity: gated (component, detection) pairs per frame;
                               0 selects 16 per component */
  void* stream;             /* cudaStream_t, or NULL */
  int64_t max_components;   /* capacity: distinct Gaussian components (tracks are
                               shared between hypotheses); 0 selects
                               h_max * max_tracks + max_births */
  /* Device allocation hook (both NULL: cudaMalloc / cudaFree).  With it set,
   * every device buffer of the handle comes from dev_alloc(bytes, alloc_ctx),
   * which returns NULL on failure, and is returned through
   * dev_free(ptr, alloc_ctx) when the buffer is replaced or the handle is
   * destroyed (after the handle's stream has finished with it): for example
   * a framework's caching allocator.  Set both or neither. */
  void* (*dev_alloc)(size_t bytes, void* ctx);
  void (*dev_free)(void* ptr, void* ctx);
  void* alloc_ctx;
  /* Track model (Section 3).  0: Gaussian constant-velocity densities
   * (Kalman update), the fields above.  1: the paper's weighted particles
   * with constant-turn-rate-and-velocity motion: dim_x 5 (px, py, speed,
   * heading, turn rate), dim_z 2 (px, py measured), score_mode 1, no
   * learned gate; q is unused.  Each component holds n_particles FP64
   * particles (1..4096); survivors take one CTRV step per frame with
   * longitudinal and yaw accelerations ~ N(0, sigma_a^2), N(0, sigma_w^2);
   * births are sampled from their Gaussian (SPD covariance required);
   * Eq. 2's entry is P_D times the particle mixture likelihood, gated by
   * the Mahalanobis test under the particles' moments; a retained track
   * with detections W is reweighted by their likelihoods and resampled
   * (systematic) when its effective sample size falls below
   * ess_frac * n_particles.  Random numbers: Philox4x32-10 keyed by
   * (seed_lo ^ 0x5851F42D, seed_hi ^ frame), counter (label_k, label_b,
   * particle, stream << 24 | call); Box-Muller normals (streams 1 the
   * accelerations, 2 the birth draws, 3 the resampling offset).
   * Device memory: 2 x max_components x n_particles x 48 bytes. */
  int32_t model;
  int32_t n_particles;
  double sigma_a, sigma_w;
  double ess_frac;
} glmb_config;

/* An LMB birth component (Section 3): existence r, Gaussian density. */
typedef struct {
  double r;
  double mean[6];           /* first dim_x entries used */
  double cov[36];           /* dim_x x dim_x row-major in the first dim_x^2 entries */
} glmb_birth;

/* One estimated track. */
typedef struct {
  uint32_t label_k, label_b;
  double r;                 /* existence: total weight of hypotheses holding the label */
  double mean[6];
  double cov[36];           /* dim_x x dim_x row-major */
} glmb_track;

/* Sizes of the current state and of the last frame's work. */
typedef struct {
  int32_t frame;            /* frames predicted so far */
  int32_t n_hyp;            /* hypotheses */
  int64_t n_entries;        /* sum over hypotheses of their track counts */
  int32_t n_components;     /* distinct Gaussian components */
  int32_t n_meas;           /* detections of the last update */
  int64_t n_pairs;          /* gated pairs of the last update */
  int64_t n_children;       /* children drawn by the last update (parents x h_up) */
  int64_t n_unique;         /* unique children with finite weight */
  int32_t n_updates;        /* distinct (component, detection set) track updates */
  int32_t n_fp64_chol;      /* innovation covariances factorised in FP64 */
  int64_t n_launches;       /* CUDA kernels launched by the library so far (all handles) */
  int64_t n_graph_captures; /* frame graphs captured by glmb_step on this handle */
  int64_t n_graph_launches; /* frame graphs replayed by glmb_step on this handle */
  int64_t n_redo;           /* frames whose expansion was redone with a larger plan */
  int32_t expand_smem_bytes;   /* shared memory per CTA of the last expansion */
  int32_t expand_ctas_per_sm;  /* resident CTAs per SM of the last expansion */
  int32_t expand_plan_T;       /* slots per hypothesis the last expansion was planned for */
  int32_t expand_plan_K;       /* gated pairs per hypothesis it was planned for */
  int32_t expand_plan_M;       /* detection rows it was planned for */
  int32_t expand_threads;      /* threads per CTA of the last expansion */
  double graph_capture_ms;     /* host time spent capturing and instantiating frame graphs */
  int64_t n_pairs_pregate;     /* pairs that passed the Mahalanobis test (before the learned gate) */
  int64_t n_draw_overflow;     /* children of the last update that the one-thread-per-child draw
                                  handed to the one-warp-per-child kernel (a slot met twice) */
} glmb_info;

/* Creates a filter holding the initial GLMB: one hypothesis with no tracks
 * and weight one.  All device memory is allocated here from the capacities.
 * Errors: GLMB_E_INVALID (bad model or capacity), GLMB_E_OOM, GLMB_E_CUDA. */
glmb_status glmb_create(const glmb_config* cfg, glmb_handle** out);

/* Frees every resource of the handle.  Accepts NULL. */
glmb_status glmb_destroy(glmb_handle* h);

/* Returns the filter to the initial GLMB and frame 0. */
glmb_status glmb_reset(glmb_handle* h);

/* Prediction (Section 3): every track of every hypothesis is propagated with
 * the CV model and kept with prior existence p_s (its death is sampled in
 * glmb_update); the n_births birth components (host array, copied) are
 * appended to every hypothesis with existence r and label (frame, index).
 * Errors: GLMB_E_INVALID (r outside [0,1], NaN), GLMB_E_CAPACITY. */
glmb_status glmb_predict(glmb_handle* h, const glmb_birth* births, int n_births);

/* Update (Section 3, Eq. 2 and the two-stage sampling): Z holds M detections,
 * M x dim_z row-major float32, in host memory (z_is_device = 0; copied) or
 * device memory on the handle's GPU (z_is_device = 1; read in place by the
 * kernels, so it must stay valid and unchanged until glmb_prune returns, and
 * the handle's stream must be ordered after its writes).  Builds the gated
 * compatibility table, the posterior death probabilities, and the h_up
 * children of each hypothesis with their exact log-weights; unique children
 * stay on the device for glmb_prune.  The call waits once for the GPU, after
 * the expansion: a hypothesis with more gated pairs than the expansion was
 * planned for (from earlier frames) makes it redo the expansion with the
 * frame's exact maxima before it returns, so the children are final.
 * Errors: GLMB_E_STATE (no predict), GLMB_E_INVALID (M < 0, NaN/Inf in a
 * host Z, a device Z that is not device or managed memory of the handle's
 * GPU or not 4-byte aligned), GLMB_E_CAPACITY (M beyond max_meas, or a per-hypothesis table
 * that cannot fit in shared memory).  Errors found on the device (NaN/Inf in
 * a device Z, gated pairs beyond max_pairs) are returned by glmb_prune. */
glmb_status glmb_update(glmb_handle* h, const float* Z, int M, int z_is_device);

/* Pruning (Section 3): normalises the children's weights over all unique
 * children (FP64), drops those below tau, keeps the h_max heaviest (ties by
 * parent then draw index), renormalises, and builds the new hypotheses with
 * one Kalman update per distinct (component, detection set).  Waits for
 * the frame to finish (one synchronisation).
 * Errors: GLMB_E_STATE, GLMB_E_NUMERIC (no child with finite weight),
 * GLMB_E_INVALID (NaN/Inf in a device Z), GLMB_E_CAPACITY (pairs,
 * components or entries beyond capacity). */
glmb_status glmb_prune(glmb_handle* h);

/* One whole frame: glmb_predict + glmb_update + glmb_prune with the same
 * arguments and results, launched as one CUDA graph (captured on the first
 * call for a given launch plan and replayed afterwards) followed by one
 * synchronisation.  The graph also computes the frame's estimates (unless
 * glmb_set_step_estimates turned that off), so that a following
 * glmb_estimates only copies them out.  The handle's stream must not be the
 * legacy default stream.  The per-step inspection calls (glmb_get_parents,
 * _components, _pairs, _children) describe this frame afterwards as they do
 * after the separate calls.  Errors: those of the three calls. */
glmb_status glmb_step(glmb_handle* h, const glmb_birth* births, int n_births, const float* Z, int M,
                      int z_is_device);

/* Estimates: writes the tracks of the heaviest hypothesis among those with
 * the most probable cardinality into out[0..n_out) (n_out <= cap), each with
 * its existence r.  card_pmf (nullable) receives the cardinality
 * distribution for n = 0..pmf_cap-1.  Synchronises.
 * Errors: GLMB_E_INVALID, GLMB_E_CAPACITY (cap too small; n_out is set). */
glmb_status glmb_estimates(glmb_handle* h, glmb_track* out, int cap, int* n_out,
                           double* card_pmf, int pmf_cap);

/* For each detection i of the last update, the total weight of retained
 * hypotheses that assign it to clutter (r_u[i], i < M <= cap). Synchronises. */
glmb_status glmb_meas_assoc(glmb_handle* h, double* r_u, int cap);

/* Current sizes (synchronises). */
glmb_status glmb_get_info(glmb_handle* h, glmb_info* info);

/* State buffer (host memory), little-endian:
 *   u32 magic 0x424D4C47 ('GLMB'), u32 version (1; 2 with particles),
 *   i32 dim_x, i32 frame, i32 n_hyp, i32 pad, i64 n_tracks_total;
 *   per hypothesis: f64 logw, u64 uid, i32 n_tracks, i32 pad;
 *   per track (hypotheses in order): u32 label_k, u32 label_b,
 *     f64 mean[dim_x], f64 cov[dim_x * dim_x] (row-major), and with the
 *     particle model (version 2) f64 x[n_particles][5], f64
 *     logw[n_particles] (normalised; the mean and covariance are then
 *     recomputed from the particles on import).
 * glmb_export_state writes it into buf (cap bytes) and sets *n_out; with
 * buf == NULL it only sets *n_out.  glmb_import_state replaces the filter
 * state; the next call must be glmb_predict.  Log-weights must be
 * normalised.  Errors: GLMB_E_CAPACITY, GLMB_E_STATE (malformed buffer). */
glmb_status glmb_export_state(glmb_handle* h, void* buf, size_t cap, size_t* n_out);
glmb_status glmb_import_state(glmb_handle* h, const void* buf, size_t n);

/* Retained hypotheses after glmb_prune: logw[n_h], uid[n_h],
 * hyp_ptr[n_h + 1] (offsets into the label arrays), label_k/label_b per
 * track, and theta[n_h][M] (0 = clutter, j + 1 = the hypothesis's j-th
 * track).  Any output pointer may be NULL.  Synchronises.
 * Errors: GLMB_E_STATE, GLMB_E_CAPACITY (cap_h or cap_entries too small). */
glmb_status glmb_get_hypotheses(glmb_handle* h, double* logw, uint64_t* uid, uint32_t* hyp_ptr,
                                uint32_t* label_k, uint32_t* label_b, uint16_t* theta, int cap_h,
                                int64_t cap_entries, int* n_h);

/* The children retained by the last successful glmb_prune, in the order of
 * the hypotheses: child_idx[j] = parent * h_up + draw (parents in the order
 * they had during glmb_update), logw[j] their renormalised FP64
 * log-weights.  Either pointer may be NULL.  Synchronises.
 * Errors: GLMB_E_STATE (no pruned frame since create/reset/import),
 * GLMB_E_CAPACITY (cap < n; *n is still set). */
glmb_status glmb_get_retained(glmb_handle* h, int64_t* child_idx, double* logw, int cap, int* n);

/* Inspection of the last glmb_update, for checking each step on its own.
 *
 * glmb_get_parents: slot lists of the parents (the hypotheses before the
 * update, in order), births included: ptr[n_parents + 1], comp[] (component
 * index of each slot).
 * glmb_get_components: the predicted components the update used: labels,
 * mean (dim_x), cov (dim_x^2 row-major), existence prior p, posterior death
 * probability dprob, log det S.
 * glmb_get_pairs: the gated table, CSR by component: comp_ptr[n_comp + 1],
 * meas[], logC[] (log of the Eq. 2 entry), q[] (e^T R^-1 e), e[] (dim_z per
 * pair, e = z - H m).
 * glmb_get_children: for each child (parent-major, h_up per parent): its
 * unnormalised log-weight (FP64), status (0 zero weight, 1 unique,
 * 2 duplicate of a lower draw) and number of surviving tracks.
 * All synchronise; GLMB_E_STATE before the first update, GLMB_E_CAPACITY
 * when a cap is too small (the needed size is still written). */
glmb_status glmb_get_parents(glmb_handle* h, uint32_t* ptr, uint32_t* comp, int cap_parents,
                             int64_t cap_slots, int* n_parents);
glmb_status glmb_get_components(glmb_handle* h, uint32_t* label_k, uint32_t* label_b,
                                double* mean, double* cov, double* p, double* dprob,
                                double* logdetS, int cap, int* n_comp);
glmb_status glmb_get_pairs(glmb_handle* h, uint32_t* comp_ptr, uint32_t* meas, float* logC,
                           float* q, float* e, int cap_comp, int64_t cap_pairs, int64_t* n_pairs);
glmb_status glmb_get_children(glmb_handle* h, double* logw, int8_t* status, uint16_t* n_alive,
                              int64_t cap, int64_t* n_children);

/* Optional timing of the update's stages with CUDA events on the handle's
 * stream.  stage_mask bit s enables stage s: 0 predict, 1 compatibility
 * table and death probabilities, 2 child expansion and scoring, 3
 * normalisation and top-H selection, 4 regeneration of retained children,
 * 5 track update and component compaction, 6 estimates.  Setting the mask
 * clears the totals.  glmb_get_timing returns, per stage, total milliseconds
 * and the number of timed calls (n entries each; either pointer may be
 * NULL); it synchronises. */
glmb_status glmb_set_profiling(glmb_handle* h, unsigned stage_mask);

/* glmb_step in two halves, so that frames of several handles (each on its
 * own stream) run on the GPU at the same time: glmb_step_enqueue launches
 * the frame and returns; glmb_step_finish waits for it and commits it (or
 * redoes or abandons it, as glmb_step would).  No other call on the handle
 * is allowed in between.  Errors: as glmb_step; GLMB_E_STATE from finish
 * without an enqueued frame. */
glmb_status glmb_step_enqueue(glmb_handle* h, const glmb_birth* births, int n_births, const float* Z,
                              int M, int z_is_device);
glmb_status glmb_step_finish(glmb_handle* h);

/* One frame of n independent filters (scenes): every frame is enqueued,
 * then every frame finished.  Handles created with their own streams (the
 * default when glmb_config.stream is NULL) run concurrently.  status[i]
 * (nullable) receives scene i's result; the return value is the first
 * error, or GLMB_OK.  Not part of the paper's method: the batched form. */
typedef struct {
  const glmb_birth* births;
  int32_t n_births;
  int32_t z_is_device;
  const float* Z;
  int32_t M;
  int32_t pad;
} glmb_frame_in;
glmb_status glmb_step_batch(glmb_handle* const* hs, int n, const glmb_frame_in* frames, glmb_status* status);

/* Launch shapes (not part of the method; results do not depend on them):
 *   thread_warps_per_sm  draw one thread per child once the children give
 *                        every SM this many warps (default 4);
 *   draw_threads         threads per draw CTA (32..256, multiple of 32; 0:
 *                        256, halved down to 64 while the frame's children
 *                        would give an SM fewer than two CTAs; the draw
 *                        kernel takes the children in order, one per
 *                        thread, whatever the CTA size);
 *   warp_cta_warps       most warps per CTA of the one-warp-per-child kernel
 *                        (1..16, default 16);
 *   stage_threads        threads per staging CTA (32..256, multiple of 32; 0,
 *                        the default: 256 when parents are staged in shared
 *                        memory or are fewer than two per SM, else 64).
 * Setting them drops the captured graphs. */
typedef struct {
  int32_t thread_warps_per_sm;
  int32_t draw_threads;
  int32_t warp_cta_warps;
  int32_t stage_threads;
} glmb_tuning;
glmb_status glmb_set_tuning(glmb_handle* h, const glmb_tuning* t);
glmb_status glmb_get_tuning(glmb_handle* h, glmb_tuning* t);

/* Launch-path overrides, for tests and tuning (not part of the paper's
 * method).  The paths compute the same arithmetic, so children's keys,
 * hashes and statuses do not depend on them.
 *   GLMB_OPT_STAGE_GLOBAL  build the per-parent tables in global memory even
 *                          when they fit in shared memory;
 *   GLMB_OPT_DRAW_WARP     draw every child with one warp;
 *   GLMB_OPT_DRAW_THREAD   draw children one per thread whatever the number
 *                          of parents (children whose lists overflow still
 *                          go to the warp path).
 *   GLMB_OPT_STAGE_SHARED  build them in shared memory whenever a parent's
 *                          tables fit (GLMB_OPT_STAGE_GLOBAL wins if both
 *                          are set).
 *   GLMB_OPT_STAGE_SCRATCH_ROWS  when the tables are built in global memory,
 *                          keep only the row offsets in shared memory
 *                          while a parent is staged;
 *   GLMB_OPT_STAGE_SCRATCH_NONE  keep none of its scratch there (wins over
 *                          GLMB_OPT_STAGE_SCRATCH_ROWS);
 *   GLMB_OPT_WARP_GROUPS   on the one-warp-per-child path, let at least
 *                          two warps share each child (by default groups
 *                          form when the per-child work areas of a
 *                          large plan leave an SM fewer than 16 warps, or
 *                          when a plan of 768 slots or more has too few
 *                          children to fill the GPU's warps).
 * Default 0: shared-memory staging when eight staging CTAs fit on an SM
 * (else in global memory, with as much of the staging's scratch in shared
 * memory as fits), one thread per child once the children give every SM
 * four warps. */
#define GLMB_OPT_STAGE_GLOBAL 1u
#define GLMB_OPT_DRAW_WARP 2u
#define GLMB_OPT_DRAW_THREAD 4u
#define GLMB_OPT_STAGE_SHARED 8u
#define GLMB_OPT_STAGE_SCRATCH_ROWS 16u
#define GLMB_OPT_STAGE_SCRATCH_NONE 32u
#define GLMB_OPT_WARP_GROUPS 64u
glmb_status glmb_set_launch_options(glmb_handle* h, unsigned opts);

/* Whether glmb_step computes the frame's estimates in its graph (on by
 * default; with it off, glmb_estimates computes them when called).  Not part
 * of the paper's method: a launch option. */
glmb_status glmb_set_step_estimates(glmb_handle* h, int on);
glmb_status glmb_get_timing(glmb_handle* h, double* ms, long long* calls, int n);

/* ------------------------------------------------------------------------
 * Learned pair gate (an extension beyond the paper).  The paper gates the
 * compatibility matrix of Eq. 2 with a fixed test g_ijk (Section 3); this
 * library's test is d^2 <= cfg.gate.  The learned gate adds a 5-64-64-64-1
 * multilayer perceptron with GELU activations that scores every pair passing
 * that test from five features:
 *   d^2 (Mahalanobis), |e| (innovation norm), p (the slot's prior existence),
 *   age = frame - label_k, log det S.
 * In GLMB_GATE_PRUNE mode a pair enters the table only when its logit is at
 * or above the threshold, so the expansion draws over fewer candidates; the
 * death probability (reading R2) sums over the pairs that remain.
 *
 * Parameters: GLMB_GATE_NPARAM floats,
 *   W1[64][5] b1[64] W2[64][64] b2[64] W3[64][64] b3[64] w4[64] b4 mu[5] sd[5]
 * (row-major, output index first).  Features enter as (f - mu) / sd.  The
 * matrices W1, W2, W3 and w4 are used rounded to bf16; the standardised
 * features and the hidden activations are rounded to bf16 before each
 * matrix product; products accumulate in fp32.  The first GLMB_GATE_NTRAIN
 * values are the trained ones (mu and sd are fixed).
 * ---------------------------------------------------------------------- */
#define GLMB_GATE_NPARAM 8779
#define GLMB_GATE_NTRAIN 8769
#define GLMB_GATE_OFF 0     /* no learned gate (the default) */
#define GLMB_GATE_PRUNE 1   /* drop pairs whose logit < threshold */
#define GLMB_GATE_SCORE 2   /* score every pair, prune nothing (for evaluation) */

/* Sets the gate for the following updates.  params: host memory, copied
 * (ignored, and may be NULL, for GLMB_GATE_OFF).  Errors: GLMB_E_INVALID for
 * an unknown mode, missing params, a non-finite parameter or sd <= 0;
 * GLMB_E_OOM when the gate's buffers (two byte/float arrays of max_pairs
 * entries and, for PRUNE, a second pair table) cannot be allocated. */
glmb_status glmb_set_gate(glmb_handle* h, const float* params, float threshold, int mode);

/* Raw features (before standardisation) of the pairs of the last update's
 * table as it was before the learned gate, in table order (component, then
 * detection): X[n][5] floats, host memory.  *n receives the pair count;
 * GLMB_E_CAPACITY when it exceeds cap rows (nothing copied).  Valid from the
 * update until the next prediction.  GLMB_E_STATE without an update. */
glmb_status glmb_gate_features(glmb_handle* h, float* X, int64_t cap, int64_t* n);

/* Logits of those pairs (modes PRUNE and SCORE), host memory, same order. */
glmb_status glmb_gate_logits(glmb_handle* h, float* logit, int64_t cap, int64_t* n);

/* After a pruned frame with the gate OFF or in SCORE mode: used[k] = 1 when
 * a retained hypothesis assigns a detection to the track of pair k (the
 * gate's training label), else 0 (cap_pairs entries at least the pair
 * count); hyp_flag[j] = 1 when retained hypothesis j uses a pair whose logit
 * is below the threshold (SCORE mode; 0 otherwise; cap_h >= hypotheses).
 * Either array may be NULL.  Host memory.  Errors: GLMB_E_STATE without a
 * pruned frame or in PRUNE mode; GLMB_E_CAPACITY for short arrays. */
glmb_status glmb_gate_usage(glmb_handle* h, uint8_t* used, int64_t cap_pairs, uint8_t* hyp_flag, int cap_h,
                            int64_t* n_pairs, int* n_hyp);

/* Stateless MLP calls (no filter handle), device memory throughout, all
 * work enqueued on `stream` (a cudaStream_t, NULL for the default stream);
 * the caller owns every buffer.  err: one device uint32 to which a kernel
 * ORs 256 when a tensor-core wait ran out of time (its results are then
 * invalid); the caller zeroes and reads it.  GLMB_E_INVALID for n < 0 or a
 * NULL pointer (n = 0 launches nothing).
 *
 * glmb_mlp_forward: logit[i] for the raw feature rows X[n][5].
 * glmb_mlp_backward: zeroes grad[GLMB_GATE_NPARAM] and *loss (a double),
 *   then accumulates the loss sum_i wt[i] (softplus(z_i) - y[i] z_i) and its
 *   gradient with respect to the bf16-rounded weights (rounding passed
 *   straight through; zero for mu and sd).  y[i] in {0, 1}.
 * glmb_mlp_adam: one Adam step (Kingma and Ba 2015, bias-corrected,
 *   step = 1, 2, ...) of the first GLMB_GATE_NTRAIN parameters, moments m
 *   and v (GLMB_GATE_NTRAIN floats each, zero before the first step). */
glmb_status glmb_mlp_forward(const float* params, const float* X, int64_t n, float* logit, uint32_t* err,
                             void* stream);
glmb_status glmb_mlp_backward(const float* params, const float* X, const float* y, const float* wt, int64_t n,
                              float* grad, double* loss, uint32_t* err, void* stream);
glmb_status glmb_mlp_adam(float* params, const float* grad, float* m, float* v, int step, float lr, float beta1,
                          float beta2, float eps, void* stream);

/* Top-H selection without device allocation.  The paper has no counterpart:
 * this is the normalisation and truncation step of glmb_prune offered on
 * its own, for callers that may not allocate device memory while they run
 * (a tracking loop with a fixed memory budget and a frame deadline, where
 * cudaMalloc can synchronise the device and stall; a host application
 * whose memory policy forbids raw cudaMalloc).  It needs no handle and
 * allocates nothing: its scratch is a 41,216-byte array in the library's
 * device image, which every GPU that loads the library holds until the
 * process exits.
 *
 * Inputs (device memory, caller-owned): logw_dev[n] child log-weights in
 * FP64.  Valid log-weights lie in (-2^30, 2^30); anything else (-INFINITY,
 * +INFINITY, NaN, or a finite value outside that range) marks a child
 * without weight.  Computation, with the steps of glmb_prune's selection:
 * weights are rounded to 2^-32, normalised by their log-sum-exp (summed in
 * FP64), those below tau dropped, the h_max largest kept (ties to the lower
 * index).  glmb_prune sums its log-sum-exp in another order, so the two
 * agree up to its rounding: a child within that rounding of tau may be
 * decided either way.  Outputs (device memory, caller-owned):
 * idx_out_dev[h_max] the kept indices in ascending order,
 * logw_out_dev[h_max] their renormalised log-weights, *n_out_dev their
 * number.  Work is queued on stream (a cudaStream_t; NULL is the default
 * stream) and the call returns without waiting.
 *
 * The first call on a device looks up the scratch array's address for that
 * device (make it before any stream capture).  Every call uses the same
 * scratch and clears what it needs at its start, so calls that overlap on
 * the GPU (on different streams, or from several threads) race: serialise
 * them.  Limits: n <= 2^30, h_max <= 2^30.
 * Errors: GLMB_E_INVALID (null pointer, h_max < 1, tau <= 0),
 * GLMB_E_CAPACITY (n or h_max beyond the limits; nothing is launched),
 * GLMB_E_CUDA. */
glmb_status glmb_select_top_static(const double* logw_dev, int64_t n, int32_t h_max, double tau,
                                   int64_t* idx_out_dev, double* logw_out_dev, int32_t* n_out_dev,
                                   void* stream);

/* Failure-detection test hook (not part of the paper's method: it tests the
 * library's own error handling).  Every device-side wait of the library is
 * bounded; when a wait runs out, the kernel records the error, leaves its
 * work unfinished and returns, and the frame fails with GLMB_E_TIMEOUT,
 * leaving the previous frame's state intact.  This call makes one such
 * wait run out on purpose, without any GPU fault:
 *   GLMB_WAIT_TEST_SCAN  the first tile of every one-pass scan (used for
 *                        the pair-count scan of frames with more than 16384
 *                        components) withholds its prefix, so the look-back
 *                        waits of the later tiles give up after `limit`
 *                        polls;
 *   GLMB_WAIT_TEST_GATE  CTA 0 of the learned gate's forward pass issues no
 *                        tensor-core work for its first tile (nothing is in
 *                        flight), so its completion wait gives up after
 *                        `limit` SM clock cycles and the CTA frees its
 *                        tensor memory and returns;
 *   GLMB_WAIT_TEST_OFF   normal limits (`limit` ignored).
 * The setting is process-wide and applies to kernels launched after the
 * call; while it is set, glmb_step runs its frames without capturing a
 * graph.  Errors: GLMB_E_INVALID (unknown mode, limit < 1). */
#define GLMB_WAIT_TEST_OFF 0
#define GLMB_WAIT_TEST_SCAN 1
#define GLMB_WAIT_TEST_GATE 2
glmb_status glmb_set_wait_test(int mode, long long limit);

/* Message of the last error on this handle ("" if none). */
const char* glmb_last_error(glmb_handle* h);

#ifdef __cplusplus
}
#endif
#endif /* GLMB_H */

/*
 * FP64 CPU oracle of the multi-detection GLMB update (arXiv 2512.06230,
 * Section 3).  TEST INFRASTRUCTURE ONLY: the tests, the smoke check and the
 * benchmark's CPU-baseline leg call it; the library never does.  It shares
 * no code, header or constant with the CUDA path.
 *
 * Readings of the paper that this oracle fixes (the paper prints no
 * formula for them) are stated at each function in glmb_oracle.c.
 */
#ifndef GLMB_ORACLE_H
#define GLMB_ORACLE_H
#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct {
  int32_t dim_x, dim_z;          /* 4/2 or 6/3 constant velocity, positions measured */
  double dt, q;                  /* frame period, white-acceleration PSD */
  double R[9];                   /* dim_z x dim_z detection covariance, row-major */
  double p_s, p_d, lambda_d;     /* survival, detection, extra-detection Poisson mean */
  double clutter_rate, volume;   /* kappa = clutter_rate / volume */
  double gate;                   /* Mahalanobis gate on d^2 (INFINITY = off) */
  int32_t h_max, h_up;           /* retained hypotheses, draws per parent */
  double tau;                    /* weight threshold */
  uint64_t seed;
  int32_t score_mode;            /* 0 joint likelihood, 1 product of C entries */
  int32_t n_threads;             /* OpenMP threads over parents (<=0: 1) */
  /* track model: 0 Gaussian constant velocity (Kalman), 1 weighted
   * particles with constant turn rate and velocity (dim_x 5: px, py, v,
   * heading, turn rate; dim_z 2; score_mode 1) */
  int32_t model;
  int32_t n_particles;           /* particles per track (model 1) */
  double sigma_a, sigma_w;       /* std of the longitudinal and yaw accelerations */
  double ess_frac;               /* resample when ESS < ess_frac * n_particles */
} orc_config;

typedef struct {
  double r;
  double mean[6];
  double cov[36];                /* dim_x x dim_x row-major in the first dim_x^2 */
} orc_birth;

typedef struct orc_filter orc_filter;

orc_filter* orc_create(const orc_config* cfg);
void orc_destroy(orc_filter* f);
void orc_reset(orc_filter* f);
int orc_import(orc_filter* f, int frame, int H, const double* logw, const uint64_t* uid,
               const int32_t* n_tracks, const uint32_t* lk, const uint32_t* lb,
               const double* mean, const double* cov);
int orc_export_counts(const orc_filter* f, int* H, int* n_total, int* frame);
int orc_export(const orc_filter* f, double* logw, uint64_t* uid, int32_t* n_tracks,
               uint32_t* lk, uint32_t* lb, double* mean, double* cov);

int orc_predict(orc_filter* f, const orc_birth* births, int n_births);
int orc_update(orc_filter* f, const float* Z, int M);
int orc_prune(orc_filter* f);

/* introspection of the last predict/update/prune */
int orc_num_parents(const orc_filter* f);
int orc_parent_slots(const orc_filter* f, int h);
int orc_slot(const orc_filter* f, int h, int t, uint32_t* lk, uint32_t* lb, double* mean,
             double* cov, double* p, double* dprob, double* logdetS);
int orc_pair(const orc_filter* f, int h, int t, int i, double* d2, double* logC, double* e,
             double* q);
double orc_gate_margin(const orc_filter* f, int h);
/* parent h's gated-pair table (CSR by slot, detections ascending within a
 * slot): ptr[T+1], meas[K], logC[K], q[K], e[K][dim_z]; returns K (-1 on a
 * bad index); with meas NULL only K is returned */
int orc_parent_pairs(const orc_filter* f, int h, int32_t* ptr, int32_t* meas, double* logC, double* q,
                     double* e);
int orc_children(const orc_filter* f, int8_t* status, double* logw, double* margin,
                 int32_t* n_alive, uint64_t* uid);
int orc_child(const orc_filter* f, int h, int n, uint8_t* dead, uint16_t* theta);
int orc_kept(const orc_filter* f, int64_t* idx, double* logw_norm, double* lse_all);
int orc_kept_theta(const orc_filter* f, uint16_t* theta);
int orc_estimates(const orc_filter* f, int cap, int* n_out, uint32_t* lk, uint32_t* lb,
                  double* mean, double* cov, double* r, double* pmf, int pmf_cap,
                  int* map_index);
int orc_meas_assoc(const orc_filter* f, double* r_u);
int orc_bruteforce(const orc_filter* f, int h, int cap, uint8_t* dead, uint16_t* theta,
                   double* logw);
/* Learned gate: a 5-64-64-64-1 MLP with GELU activations on five features
 * of a gated (slot, detection) pair (Mahalanobis d^2, innovation norm,
 * prior existence, track age in frames, log det S).  A pair that passes the
 * Mahalanobis gate is kept only when its logit >= threshold.  params holds
 * ORC_GATE_NPARAM floats: W1[64][5] b1[64] W2[64][64] b2[64] W3[64][64]
 * b3[64] w4[64] b4 mu[5] sd[5] (weights used rounded to bf16; features
 * standardised as (f - mu) / sd).  NULL switches the gate off. */
#define ORC_GATE_NPARAM 8779
int orc_set_gate(orc_filter* f, const float* params, double threshold);
/* smallest |logit - threshold| over the pairs the gate judged for parent h
 * (INFINITY when the gate is off or judged none) */
double orc_mlp_margin(const orc_filter* f, int h);
/* features and logit of (parent h, slot t, detection i) */
int orc_gate_eval(const orc_filter* f, int h, int t, int i, double* feat, double* logit);
/* the MLP on one raw feature row; round_act = 1 rounds the standardised
 * features and every hidden activation to bf16 (the precision the library's
 * decision is taken in), 0 keeps them in double */
double orc_mlp_logit(const float* params, const double* feat, int round_act);
void orc_philox(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]);

/* Particle track model (model 1).  Particles of a track are [P][5]
 * states and [P] normalised log-weights; arrays over tracks follow the
 * order of orc_import / orc_export. */
int orc_import_particles(orc_filter* f, const double* x, const double* logw);
int orc_export_particles(const orc_filter* f, double* x, double* logw);
/* predicted particles of slot t of parent h of the last update */
int orc_slot_particles(const orc_filter* f, int h, int t, double* x, double* logw);
/* smallest distance between a resampling target and a cumulative weight
 * over the last prune's resamplings (INFINITY when none resampled) */
double orc_resample_margin(const orc_filter* f);
/* one CTRV step over dt with accelerations (a, alpha) held over it */
void orc_ctrv(const double x[5], double dt, double a, double alpha, double out[5]);
/* the two standard normal draws of particle p of label (lk, lb) in
 * stream s, call j, for the frame and seed of the filter */
void orc_particle_normals(const orc_filter* f, uint32_t lk, uint32_t lb, uint32_t p, uint32_t s,
                          uint32_t j, double out[2]);
uint64_t orc_mix64(uint64_t x);

#ifdef __cplusplus
}
#endif
#endif

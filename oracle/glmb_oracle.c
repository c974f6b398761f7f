/*
 * FP64 CPU oracle of the multi-detection GLMB filter update
 * (arXiv 2512.06230, "GPU-GLMB", Section 3), with Gaussian constant-velocity
 * track densities (model 0) or the paper's weighted particles moved by
 * constant-turn-rate-and-velocity kinematics (model 1, reading R15).
 *
 * TEST INFRASTRUCTURE ONLY.  Plain, slow and written to be read against the
 * paper: every step follows Section 3 in the paper's order, in double
 * precision, with no blocking, fusion or reordering.  It shares no code with
 * the CUDA library and is called only by the tests, the smoke check and the
 * benchmark's CPU-baseline leg.
 *
 * Steps (Section 3):
 *   predict      - CV prediction of every track, LMB births appended
 *   update       - compatibility matrix C_k (Eq. 2) with gate, posterior
 *                  death probabilities, two-stage sampling of H_up children
 *                  per parent (Bernoulli deaths, then an independent
 *                  categorical per detection row over the surviving columns
 *                  of C'_k), exact target weight of each child, retention of
 *                  unique children
 *   prune        - normalisation, threshold tau, top-H_max, renormalisation,
 *                  batched track update of the retained children
 *   estimates    - cardinality distribution and MAP hypothesis (reading)
 *
 * Readings where the paper is silent (each repeated at its function):
 *   R1  Eq. 2 entry for j >= 1 is P_D * N(z_i; H m_j, S_j), gated by a
 *       Mahalanobis test d^2 <= G; the clutter column is kappa = lambda_c/V.
 *   R2  posterior death probability of a slot with prior existence p:
 *       psi = (1 - P_D) + sum_{gated i} C[i,j] / kappa,
 *       d_prob = (1 - p) / ((1 - p) + p * psi).
 *   R3  child weight = parent weight x exact GLMB target weight of the
 *       sampled deaths and associations (no division by the proposal):
 *       dead slot: (1 - p); alive slot with W detections: p * rho(|W|) * |W|!
 *       * integral of prod_{i in W} N(z_i; Hx, R) against the predicted
 *       density; clutter detection: kappa.  rho(0) = 1 - P_D,
 *       rho(m >= 1) = P_D * Poisson(m - 1; lambda_d).
 *   R4  children of one parent are identical when (death mask, theta) are
 *       identical; the lowest draw index is kept.  Children of different
 *       parents are distinct hypotheses.
 *   R5  tau is applied to weights normalised over all unique children;
 *       ties in weight are broken by (parent, draw) ascending.
 *   R6  the retained track density of an alive slot with W detections is the
 *       Kalman update with the mean detection and covariance R/|W|
 *       (Joseph form); with W empty the predicted density is kept.
 *   R7  random numbers: Philox4x32-10 keyed by (seed_lo, seed_hi ^ frame)
 *       with counter (uid_lo, uid_hi, 2n + stream, idx >> 2), output word
 *       idx & 3, u = (word >> 8) * 2^-24.  Stream 0: death of slot idx;
 *       stream 1: association of detection row idx.  Row decision: the
 *       first option j (clutter first, then alive gated slots in slot order)
 *       with u * sum < cumulative weight through j.  Death: u < d_prob.
 *   R8  a child's uid is mix64(parent_uid + 0x9E3779B97F4A7C15 * (n + 1));
 *       the initial empty hypothesis has uid mix64(seed + 0x9E3779B97F4A7C15).
 *   R9  estimates: MAP cardinality, then the heaviest hypothesis of that
 *       cardinality; existence of a label = total weight of hypotheses that
 *       contain it.
 *   R10 learned gate (an extension, off unless orc_set_gate is called): a
 *       pair that passes the Mahalanobis test enters the table only when a
 *       5-64-64-64-1 GELU MLP on (d^2, |e|, p, age, log det S) scores it at
 *       or above a threshold.  The decision is taken on the forward pass
 *       with bf16 weights and bf16-rounded inputs and activations (the
 *       precision the library decides in), accumulated in double.
 *
 * R2 is pinned where the model reduces to the single-detection Bernoulli
 * filter (one track, lambda_d = 0): the death probability equals the exact
 * marginal over every enumerated child.  R9's sums (cardinality pmf, label
 * existence) and its choice (the MAP cardinality, then the heaviest
 * hypothesis of that cardinality) are pinned against the brute-force
 * posterior; the choice rule itself is a reading, which the paper does not
 * state.  Everything else is pinned by closed forms, brute force and
 * independent restatements (tests/test_oracle_pins.py).
 */
#include "glmb_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define LOG2PI 1.8378770664093454836
#define GOLDEN 0x9E3779B97F4A7C15ULL

/* ------------------------------------------------------------------ */
/* Counter-based generator: Philox4x32-10 from Salmon, Moraes, Dror and  */
/* Shaw, "Parallel random numbers: as easy as 1, 2, 3" (SC'11); pinned   */
/* to the known-answer vectors published with that definition.          */
/* ------------------------------------------------------------------ */
void orc_philox(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]) {
  uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
  uint32_t k0 = key[0], k1 = key[1];
  for (int round = 0; round < 10; ++round) {
    uint64_t p0 = (uint64_t)0xD2511F53u * (uint64_t)c0;
    uint64_t p1 = (uint64_t)0xCD9E8D57u * (uint64_t)c2;
    uint32_t n0 = (uint32_t)(p1 >> 32) ^ c1 ^ k0;
    uint32_t n1 = (uint32_t)p1;
    uint32_t n2 = (uint32_t)(p0 >> 32) ^ c3 ^ k1;
    uint32_t n3 = (uint32_t)p0;
    c0 = n0; c1 = n1; c2 = n2; c3 = n3;
    k0 += 0x9E3779B9u;
    k1 += 0xBB67AE85u;
  }
  out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* splitmix64 output function (Steele, Lea, Flood, OOPSLA 2014). */
uint64_t orc_mix64(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  return z ^ (z >> 31);
}

/* ------------------------------------------------------------------ */
/* small dense linear algebra (row-major, n <= 6)                      */
/* ------------------------------------------------------------------ */
static int chol(int n, const double* A, double* L) {
  memset(L, 0, sizeof(double) * n * n);
  for (int j = 0; j < n; ++j) {
    double s = A[j * n + j];
    for (int k = 0; k < j; ++k) s -= L[j * n + k] * L[j * n + k];
    if (!(s > 0.0)) return -1;
    double d = sqrt(s);
    L[j * n + j] = d;
    for (int i = j + 1; i < n; ++i) {
      double t = A[i * n + j];
      for (int k = 0; k < j; ++k) t -= L[i * n + k] * L[j * n + k];
      L[i * n + j] = t / d;
    }
  }
  return 0;
}

static void fwd_solve(int n, const double* L, const double* b, double* y) {
  for (int i = 0; i < n; ++i) {
    double s = b[i];
    for (int k = 0; k < i; ++k) s -= L[i * n + k] * y[k];
    y[i] = s / L[i * n + i];
  }
}

static void bwd_solve(int n, const double* L, const double* y, double* x) {
  /* solves L^T x = y */
  for (int i = n - 1; i >= 0; --i) {
    double s = y[i];
    for (int k = i + 1; k < n; ++k) s -= L[k * n + i] * x[k];
    x[i] = s / L[i * n + i];
  }
}

static double logdet_from_chol(int n, const double* L) {
  double s = 0.0;
  for (int i = 0; i < n; ++i) s += log(L[i * n + i]);
  return 2.0 * s;
}

/* x^T A^{-1} x with A = L L^T */
static double mahal(int n, const double* L, const double* x) {
  double y[6];
  fwd_solve(n, L, x, y);
  double s = 0.0;
  for (int i = 0; i < n; ++i) s += y[i] * y[i];
  return s;
}

static int spd_inverse(int n, const double* A, double* Ainv) {
  double L[36], e[6], y[6], x[6];
  if (chol(n, A, L)) return -1;
  for (int c = 0; c < n; ++c) {
    for (int i = 0; i < n; ++i) e[i] = (i == c);
    fwd_solve(n, L, e, y);
    bwd_solve(n, L, y, x);
    for (int i = 0; i < n; ++i) Ainv[i * n + c] = x[i];
  }
  return 0;
}

/* ------------------------------------------------------------------ */
/* state                                                                */
/* ------------------------------------------------------------------ */
typedef struct {
  double logw;
  uint64_t uid;
  int n;
  uint32_t *lk, *lb;
  double *m, *P;              /* n*dx, n*dx*dx (model 1: the particles' moments) */
  double *x, *pw;             /* model 1: particles n*Np*5, log-weights n*Np */
} hyp_t;

typedef struct {
  int T;                      /* slots: the parent's predicted tracks, then births */
  uint32_t *lk, *lb;
  double *m, *P, *p;          /* predicted mean, covariance, prior existence */
  double *x, *pw;             /* model 1: predicted particles T*Np*5, log-weights T*Np */
  double *S, *L, *logdetS;    /* innovation covariance, its Cholesky factor */
  double *dprob;
  int K;                      /* gated (slot, detection) pairs, CSR by slot */
  int *ptr, *meas;
  double *d2, *logC, *q, *e;
  double gate_margin;
  double mlp_margin;          /* smallest |logit - threshold| judged */
  int *rptr, *rslot, *rpair;  /* same pairs re-indexed by detection row */
  /* children */
  int8_t* status;             /* 0 zero weight, 1 unique, 2 duplicate */
  double *logw, *margin;
  int32_t *n_alive, *n_clutter;
  uint64_t* uid;
  uint16_t* theta;            /* H_up x M: 0 clutter, slot + 1 */
  uint8_t* dead;              /* H_up x T */
} par_t;

struct orc_filter {
  orc_config c;
  int mlp_on;                 /* learned gate (see orc_set_gate) */
  float mlp[8779];
  double mlp_thr;
  int dx, dz;
  int frame;
  double F[36], Q[36], Rinv[9], logdetR, kappa, log_kappa;
  int H;
  hyp_t* hyp;
  int nb;
  orc_birth* births;
  int stage;                  /* 0 idle, 1 predicted, 2 updated, 3 pruned */
  int M;
  double* Z;
  int Hold;
  par_t* par;
  hyp_t* old_hyp;             /* parents of the last update */
  int nkept;
  int64_t* kept_idx;
  double* kept_logw;
  double lse_all;
  uint16_t* kept_theta;       /* theta of retained children, in their own track indices */
  double resample_margin;     /* model 1: see orc_resample_margin */
};

static void free_hyp(hyp_t* h) {
  free(h->lk); free(h->lb); free(h->m); free(h->P); free(h->x); free(h->pw);
  memset(h, 0, sizeof(*h));
}

static void free_par(par_t* P) {
  free(P->lk); free(P->lb); free(P->m); free(P->P); free(P->p); free(P->x); free(P->pw);
  free(P->S); free(P->L); free(P->logdetS); free(P->dprob);
  free(P->ptr); free(P->meas); free(P->d2); free(P->logC); free(P->q); free(P->e);
  free(P->rptr); free(P->rslot); free(P->rpair);
  free(P->status); free(P->logw); free(P->margin); free(P->n_alive); free(P->n_clutter);
  free(P->uid); free(P->theta); free(P->dead);
  memset(P, 0, sizeof(*P));
}

static void clear_frame(orc_filter* f) {
  if (f->par) {
    for (int h = 0; h < f->Hold; ++h) free_par(&f->par[h]);
    free(f->par);
    f->par = NULL;
  }
  if (f->old_hyp) {
    for (int h = 0; h < f->Hold; ++h) free_hyp(&f->old_hyp[h]);
    free(f->old_hyp);
    f->old_hyp = NULL;
  }
  f->Hold = 0;
  free(f->births); f->births = NULL; f->nb = 0;
  free(f->Z); f->Z = NULL; f->M = 0;
  free(f->kept_idx); f->kept_idx = NULL;
  free(f->kept_logw); f->kept_logw = NULL;
  free(f->kept_theta); f->kept_theta = NULL;
  f->nkept = 0;
}

static void free_hyps(orc_filter* f) {
  for (int h = 0; h < f->H; ++h) free_hyp(&f->hyp[h]);
  free(f->hyp);
  f->hyp = NULL;
  f->H = 0;
}

/* Constant-velocity model matrices: F = [[I, dt I], [0, I]] and the
 * continuous white-acceleration process noise
 * Q = q [[dt^3/3 I, dt^2/2 I], [dt^2/2 I, dt I]]. */
static void cv_model(orc_filter* f) {
  int dx = f->dx, d = f->dz;
  double dt = f->c.dt, q = f->c.q;
  memset(f->F, 0, sizeof f->F);
  memset(f->Q, 0, sizeof f->Q);
  for (int i = 0; i < dx; ++i) f->F[i * dx + i] = 1.0;
  for (int a = 0; a < d; ++a) {
    f->F[a * dx + d + a] = dt;
    f->Q[a * dx + a] = q * dt * dt * dt / 3.0;
    f->Q[a * dx + d + a] = q * dt * dt / 2.0;
    f->Q[(d + a) * dx + a] = q * dt * dt / 2.0;
    f->Q[(d + a) * dx + d + a] = q * dt;
  }
}

/* ------------------------------------------------------------------ */
/* Particle track densities (model 1; Section 3: each labeled state is a */
/* set of P weighted particles moved by constant-turn-rate-and-velocity */
/* kinematics; births are sampled from the birth density; the retained */
/* tracks get a particle update with resampling).  Reading R15:         */
/*   a. state (px, py, v, psi, omega); over dt the heading turns by     */
/*      omega dt and the position moves along the arc; the longitudinal */
/*      acceleration a and yaw acceleration alpha (per particle, per    */
/*      frame) add (dt^2/2)(cos psi, sin psi) a, dt a, dt^2/2 alpha and */
/*      dt alpha to (px, py), v, psi and omega (psi the heading before  */
/*      the step); a ~ N(0, sigma_a^2), alpha ~ N(0, sigma_w^2).        */
/*   b. normals: Philox4x32-10 keyed by (seed_lo ^ 0x5851F42D,          */
/*      seed_hi ^ frame), counter (label_k, label_b, particle,          */
/*      stream << 24 | call); each call's words (w0..w3) give two       */
/*      normals, sqrt(-2 ln u(w0)) cos(2 pi u(w1)) and the same of      */
/*      (w2, w3), with u(w) = (w + 1/2) 2^-32.  Stream 1: the step's    */
/*      (a, alpha); stream 2: a birth particle's five normals (calls 0  */
/*      to 2), x = m_B + L xi with L L^T the birth covariance; stream   */
/*      3: the resampling offset u(w0) of call 0 of particle 0.         */
/*   c. C entry: P_D sum_p w_p N(z; (px, py)_p, R); gate: the           */
/*      Mahalanobis test of R1 under the particles' weighted mean and   */
/*      covariance.                                                     */
/*   d. weights: the product of the chosen C entries (score_mode 1).    */
/*   e. update with detections W: log w_p += sum_{z in W}               */
/*      log N(z; (px, py)_p, R), normalised; when the effective sample  */
/*      size 1 / sum w_p^2 falls below ess_frac * P, systematic         */
/*      resampling: target r = (u + r) / P takes the first particle     */
/*      whose cumulative weight exceeds it (the last when none does);   */
/*      resampled weights 1/P.  W empty: unchanged.                     */
/*   f. a track's mean and covariance are the particles' weighted       */
/*      moments (the gate, the estimates).                              */
/* ------------------------------------------------------------------ */
#define PI_D 3.14159265358979323846
static double quad_Rinv(const orc_filter* f, const double* e);
#define PKEY_XOR 0x5851F42Du

static double unit_open(uint32_t w) { return ((double)w + 0.5) * 2.3283064365386963e-10; }

void orc_particle_normals(const orc_filter* f, uint32_t lk, uint32_t lb, uint32_t p, uint32_t s,
                          uint32_t j, double out[2]) {
  uint32_t key[2] = {(uint32_t)f->c.seed ^ PKEY_XOR, (uint32_t)(f->c.seed >> 32) ^ (uint32_t)f->frame};
  uint32_t ctr[4] = {lk, lb, p, (s << 24) | j};
  uint32_t w[4];
  orc_philox(ctr, key, w);
  out[0] = sqrt(-2.0 * log(unit_open(w[0]))) * cos(2.0 * PI_D * unit_open(w[1]));
  out[1] = sqrt(-2.0 * log(unit_open(w[2]))) * cos(2.0 * PI_D * unit_open(w[3]));
}

/* The arc displacement (v / omega)(sin(psi + omega dt) - sin psi,
 * cos psi - cos(psi + omega dt)) written with the sum-to-product identity,
 * v dt sinc(omega dt / 2) (cos, sin)(psi + omega dt / 2), which holds at
 * omega = 0 too (the straight line). */
void orc_ctrv(const double x[5], double dt, double a, double alpha, double out[5]) {
  double px = x[0], py = x[1], v = x[2], psi = x[3], om = x[4];
  double half = 0.5 * om * dt;
  double sinc = half != 0.0 ? sin(half) / half : 1.0;
  out[0] = px + v * dt * sinc * cos(psi + half) + 0.5 * dt * dt * cos(psi) * a;
  out[1] = py + v * dt * sinc * sin(psi + half) + 0.5 * dt * dt * sin(psi) * a;
  out[2] = v + dt * a;
  out[3] = psi + om * dt + 0.5 * dt * dt * alpha;
  out[4] = om + dt * alpha;
}

/* weighted mean and covariance of Np particles (R15f) */
static void particle_moments(int Np, const double* x, const double* lw, double* m, double* P) {
  for (int a = 0; a < 5; ++a) m[a] = 0.0;
  for (int p = 0; p < Np; ++p) {
    double w = exp(lw[p]);
    for (int a = 0; a < 5; ++a) m[a] += w * x[p * 5 + a];
  }
  for (int k = 0; k < 25; ++k) P[k] = 0.0;
  for (int p = 0; p < Np; ++p) {
    double w = exp(lw[p]);
    for (int a = 0; a < 5; ++a)
      for (int b = 0; b < 5; ++b) P[a * 5 + b] += w * (x[p * 5 + a] - m[a]) * (x[p * 5 + b] - m[b]);
  }
}

/* log N(z; (px, py), R) of a particle */
static double particle_loglik(const orc_filter* f, const double* xp, const double* z) {
  double e[2] = {z[0] - xp[0], z[1] - xp[1]};
  return -0.5 * (quad_Rinv(f, e) + f->logdetR + 2.0 * LOG2PI);
}

/* log sum_p w_p N(z; (px, py)_p, R) (R15c) */
static double particle_logL(const orc_filter* f, const double* x, const double* lw, const double* z) {
  int Np = f->c.n_particles;
  double mx = -INFINITY, s = 0.0;
  for (int p = 0; p < Np; ++p) {
    double l = lw[p] + particle_loglik(f, x + p * 5, z);
    if (l > mx) mx = l;
  }
  if (mx == -INFINITY) return -INFINITY;
  for (int p = 0; p < Np; ++p) s += exp(lw[p] + particle_loglik(f, x + p * 5, z) - mx);
  return mx + log(s);
}

/* Particle update of one track with the detections rows[0..mc) (R15e):
 * writes x1, lw1 and lowers *margin to the closest resampling decision. */
static void particle_update(const orc_filter* f, uint32_t lk, uint32_t lb, const double* x0,
                            const double* lw0, const int* rows, int mc, double* x1, double* lw1,
                            double* margin) {
  int Np = f->c.n_particles;
  double* lw = (double*)malloc(sizeof(double) * Np);
  double mx = -INFINITY;
  for (int p = 0; p < Np; ++p) {
    double l = lw0[p];
    for (int r = 0; r < mc; ++r) l += particle_loglik(f, x0 + p * 5, f->Z + rows[r] * 2);
    lw[p] = l;
    if (l > mx) mx = l;
  }
  double s = 0.0;
  for (int p = 0; p < Np; ++p) s += exp(lw[p] - mx);
  double lse = mx + log(s), sw2 = 0.0;
  for (int p = 0; p < Np; ++p) {
    lw[p] -= lse;
    sw2 += exp(2.0 * lw[p]);
  }
  if (1.0 / sw2 < f->c.ess_frac * Np) {
    double u[2];
    uint32_t key[2] = {(uint32_t)f->c.seed ^ PKEY_XOR, (uint32_t)(f->c.seed >> 32) ^ (uint32_t)f->frame};
    uint32_t ctr[4] = {lk, lb, 0u, 3u << 24};
    uint32_t w[4];
    orc_philox(ctr, key, w);
    u[0] = unit_open(w[0]);
    int k = 0;
    double below = 0.0, cum = exp(lw[0]);   /* cumulative weight before and through k */
    for (int r = 0; r < Np; ++r) {
      double target = (u[0] + r) / Np;
      while (k < Np - 1 && cum <= target) {
        ++k;
        below = cum;
        cum += exp(lw[k]);
      }
      double d = fabs(cum - target);
      if (k > 0 && fabs(target - below) < d) d = fabs(target - below);
      if (d < *margin) *margin = d;
      memcpy(x1 + r * 5, x0 + k * 5, sizeof(double) * 5);
      lw1[r] = -log((double)Np);
    }
  } else {
    memcpy(x1, x0, sizeof(double) * 5 * Np);
    memcpy(lw1, lw, sizeof(double) * Np);
  }
  free(lw);
}

orc_filter* orc_create(const orc_config* cfg) {
  if (!cfg) return NULL;
  if (cfg->model == 1) {
    if (!(cfg->dim_x == 5 && cfg->dim_z == 2 && cfg->score_mode == 1 && cfg->n_particles >= 1 &&
          cfg->sigma_a >= 0.0 && cfg->sigma_w >= 0.0 && cfg->ess_frac >= 0.0 && cfg->ess_frac <= 1.0))
      return NULL;
  } else if (cfg->model != 0 ||
             !((cfg->dim_x == 4 && cfg->dim_z == 2) || (cfg->dim_x == 6 && cfg->dim_z == 3))) {
    return NULL;
  }
  if (cfg->h_up < 1 || cfg->h_max < 1) return NULL;
  orc_filter* f = (orc_filter*)calloc(1, sizeof(orc_filter));
  f->c = *cfg;
  f->dx = cfg->dim_x;
  f->dz = cfg->dim_z;
  if (cfg->model == 0) cv_model(f);
  double Lr[9];
  if (chol(f->dz, cfg->R, Lr) || spd_inverse(f->dz, cfg->R, f->Rinv)) {
    free(f);
    return NULL;
  }
  f->logdetR = logdet_from_chol(f->dz, Lr);
  f->kappa = cfg->clutter_rate / cfg->volume;
  f->log_kappa = log(f->kappa);
  orc_reset(f);
  return f;
}

void orc_destroy(orc_filter* f) {
  if (!f) return;
  clear_frame(f);
  free_hyps(f);
  free(f);
}

/* The initial GLMB: one hypothesis with no tracks and weight one (R8). */
void orc_reset(orc_filter* f) {
  clear_frame(f);
  free_hyps(f);
  f->H = 1;
  f->hyp = (hyp_t*)calloc(1, sizeof(hyp_t));
  f->hyp[0].logw = 0.0;
  f->hyp[0].uid = orc_mix64(f->c.seed + GOLDEN);
  f->frame = 0;
  f->stage = 0;
  f->resample_margin = INFINITY;
}

int orc_import(orc_filter* f, int frame, int H, const double* logw, const uint64_t* uid,
               const int32_t* n_tracks, const uint32_t* lk, const uint32_t* lb,
               const double* mean, const double* cov) {
  if (H < 1) return 1;
  clear_frame(f);
  free_hyps(f);
  int dx = f->dx;
  f->H = H;
  f->hyp = (hyp_t*)calloc(H, sizeof(hyp_t));
  size_t off = 0;
  for (int h = 0; h < H; ++h) {
    hyp_t* y = &f->hyp[h];
    y->logw = logw[h];
    y->uid = uid[h];
    y->n = n_tracks[h];
    y->lk = (uint32_t*)malloc(sizeof(uint32_t) * (y->n + 1));
    y->lb = (uint32_t*)malloc(sizeof(uint32_t) * (y->n + 1));
    y->m = (double*)malloc(sizeof(double) * (y->n * dx + 1));
    y->P = (double*)malloc(sizeof(double) * (y->n * dx * dx + 1));
    for (int t = 0; t < y->n; ++t, ++off) {
      y->lk[t] = lk[off];
      y->lb[t] = lb[off];
      memcpy(y->m + t * dx, mean + off * dx, sizeof(double) * dx);
      memcpy(y->P + t * dx * dx, cov + off * dx * dx, sizeof(double) * dx * dx);
    }
  }
  f->frame = frame;
  f->stage = 0;
  return 0;
}

int orc_export_counts(const orc_filter* f, int* H, int* n_total, int* frame) {
  int n = 0;
  for (int h = 0; h < f->H; ++h) n += f->hyp[h].n;
  *H = f->H;
  *n_total = n;
  *frame = f->frame;
  return 0;
}

int orc_export(const orc_filter* f, double* logw, uint64_t* uid, int32_t* n_tracks,
               uint32_t* lk, uint32_t* lb, double* mean, double* cov) {
  int dx = f->dx;
  size_t off = 0;
  for (int h = 0; h < f->H; ++h) {
    const hyp_t* y = &f->hyp[h];
    logw[h] = y->logw;
    uid[h] = y->uid;
    n_tracks[h] = y->n;
    for (int t = 0; t < y->n; ++t, ++off) {
      lk[off] = y->lk[t];
      lb[off] = y->lb[t];
      memcpy(mean + off * dx, y->m + t * dx, sizeof(double) * dx);
      memcpy(cov + off * dx * dx, y->P + t * dx * dx, sizeof(double) * dx * dx);
    }
  }
  return 0;
}

/* ------------------------------------------------------------------ */
/* Prediction (Section 3): survivors propagated with the CV model and    */
/* carried with prior existence P_S (their death is sampled in the       */
/* update); LMB births appended with existence r_B and label             */
/* (frame, birth index).                                                 */
/* ------------------------------------------------------------------ */
int orc_predict(orc_filter* f, const orc_birth* births, int n_births) {
  if (n_births < 0) return 1;
  for (int b = 0; b < n_births; ++b)
    if (!(births[b].r >= 0.0 && births[b].r <= 1.0)) return 1;
  clear_frame(f);
  f->frame += 1;
  f->nb = n_births;
  f->births = (orc_birth*)malloc(sizeof(orc_birth) * (n_births + 1));
  if (n_births) memcpy(f->births, births, sizeof(orc_birth) * n_births);
  f->stage = 1;
  return 0;
}

/* Particle prediction (R15a, b): survivors' particles take one CTRV step
 * with their own accelerations; a birth's particles are drawn from its
 * Gaussian; the moments follow (R15f).  Returns 5 when a birth covariance
 * is not positive definite. */
static int predict_particles(const orc_filter* f, const hyp_t* y, par_t* P) {
  int Np = f->c.n_particles, T = P->T;
  if (y->n > 0 && !y->x) return 5;   /* imported without particles */
  P->x = (double*)malloc(sizeof(double) * ((size_t)T * Np * 5 + 1));
  P->pw = (double*)malloc(sizeof(double) * ((size_t)T * Np + 1));
  for (int t = 0; t < y->n; ++t)
    for (int p = 0; p < Np; ++p) {
      double n[2];
      orc_particle_normals(f, P->lk[t], P->lb[t], (uint32_t)p, 1u, 0u, n);
      orc_ctrv(y->x + ((size_t)t * Np + p) * 5, f->c.dt, f->c.sigma_a * n[0], f->c.sigma_w * n[1],
               P->x + ((size_t)t * Np + p) * 5);
      P->pw[(size_t)t * Np + p] = y->pw[(size_t)t * Np + p];
    }
  for (int b = 0; b < f->nb; ++b) {
    int t = y->n + b;
    double L[25];
    if (chol(5, f->births[b].cov, L)) return 5;
    for (int p = 0; p < Np; ++p) {
      double xi[6];
      for (int j = 0; j < 3; ++j) orc_particle_normals(f, P->lk[t], P->lb[t], (uint32_t)p, 2u, (uint32_t)j, xi + 2 * j);
      double* xp = P->x + ((size_t)t * Np + p) * 5;
      for (int a = 0; a < 5; ++a) {
        double v = f->births[b].mean[a];
        for (int k = 0; k <= a; ++k) v += L[a * 5 + k] * xi[k];
        xp[a] = v;
      }
      P->pw[(size_t)t * Np + p] = -log((double)Np);
    }
  }
  for (int t = 0; t < T; ++t)
    particle_moments(Np, P->x + (size_t)t * Np * 5, P->pw + (size_t)t * Np, P->m + t * 5, P->P + t * 25);
  return 0;
}

static int predict_parent(const orc_filter* f, const hyp_t* y, par_t* P) {
  int dx = f->dx;
  int T = y->n + f->nb;
  P->T = T;
  P->lk = (uint32_t*)malloc(sizeof(uint32_t) * (T + 1));
  P->lb = (uint32_t*)malloc(sizeof(uint32_t) * (T + 1));
  P->m = (double*)calloc(T * dx + 1, sizeof(double));
  P->P = (double*)calloc(T * dx * dx + 1, sizeof(double));
  P->p = (double*)calloc(T + 1, sizeof(double));
  if (f->c.model == 1) {
    for (int t = 0; t < y->n; ++t) {
      P->lk[t] = y->lk[t];
      P->lb[t] = y->lb[t];
      P->p[t] = f->c.p_s;
    }
    for (int b = 0; b < f->nb; ++b) {
      P->lk[y->n + b] = (uint32_t)f->frame;
      P->lb[y->n + b] = (uint32_t)b;
      P->p[y->n + b] = f->births[b].r;
    }
    return predict_particles(f, y, P);
  }
  for (int t = 0; t < y->n; ++t) {
    const double* m0 = y->m + t * dx;
    const double* P0 = y->P + t * dx * dx;
    double* m1 = P->m + t * dx;
    double* P1 = P->P + t * dx * dx;
    double FP[36];
    for (int i = 0; i < dx; ++i) {
      double s = 0.0;
      for (int k = 0; k < dx; ++k) s += f->F[i * dx + k] * m0[k];
      m1[i] = s;
    }
    for (int i = 0; i < dx; ++i)
      for (int j = 0; j < dx; ++j) {
        double s = 0.0;
        for (int k = 0; k < dx; ++k) s += f->F[i * dx + k] * P0[k * dx + j];
        FP[i * dx + j] = s;
      }
    for (int i = 0; i < dx; ++i)
      for (int j = 0; j < dx; ++j) {
        double s = 0.0;
        for (int k = 0; k < dx; ++k) s += FP[i * dx + k] * f->F[j * dx + k];
        P1[i * dx + j] = s + f->Q[i * dx + j];
      }
    P->lk[t] = y->lk[t];
    P->lb[t] = y->lb[t];
    P->p[t] = f->c.p_s;
  }
  for (int b = 0; b < f->nb; ++b) {
    int t = y->n + b;
    memcpy(P->m + t * dx, f->births[b].mean, sizeof(double) * dx);
    memcpy(P->P + t * dx * dx, f->births[b].cov, sizeof(double) * dx * dx);
    P->lk[t] = (uint32_t)f->frame;
    P->lb[t] = (uint32_t)b;
    P->p[t] = f->births[b].r;
  }
  return 0;
}

/* ------------------------------------------------------------------ */
/* Compatibility matrix (Eq. 2, reading R1) and death probability (R2)  */
/* ------------------------------------------------------------------ */
static void innovation(const orc_filter* f, const double* m, const double* z, double* e) {
  for (int a = 0; a < f->dz; ++a) e[a] = z[a] - m[a];       /* H = [I 0] */
}

static double quad_Rinv(const orc_filter* f, const double* e) {
  int d = f->dz;
  double s = 0.0;
  for (int a = 0; a < d; ++a)
    for (int b = 0; b < d; ++b) s += e[a] * f->Rinv[a * d + b] * e[b];
  return s;
}

/* ------------------------------------------------------------------ */
/* Learned gate (an extension beyond the paper's gate g_ijk): an MLP on   */
/* five features of a pair, applied after the Mahalanobis test.           */
/* ------------------------------------------------------------------ */
enum { G_W1 = 0, G_B1 = 320, G_W2 = 384, G_B2 = 4480, G_W3 = 4544, G_B3 = 8640, G_W4 = 8704,
       G_B4 = 8768, G_MU = 8769, G_SD = 8774 };

/* round to the nearest bf16 (ties to even) through float */
static double to_bf16(double x) {
  float v = (float)x;
  uint32_t u;
  memcpy(&u, &v, 4);
  if ((u & 0x7f800000u) != 0x7f800000u) {
    u += 0x7fffu + ((u >> 16) & 1u);
    u &= 0xffff0000u;
  }
  memcpy(&v, &u, 4);
  return v;
}

/* GELU(x) = x * Phi(x), Phi the standard normal distribution function */
static double gelu(double x) { return 0.5 * x * (1.0 + erf(x / sqrt(2.0))); }

double orc_mlp_logit(const float* p, const double* feat, int round_act) {
  double x[5], h[64], g[64];
  for (int j = 0; j < 5; ++j) {
    x[j] = (feat[j] - (double)p[G_MU + j]) / (double)p[G_SD + j];
    if (round_act) x[j] = to_bf16(x[j]);
  }
  for (int o = 0; o < 64; ++o) {
    double z = p[G_B1 + o];
    for (int j = 0; j < 5; ++j) z += to_bf16(p[G_W1 + o * 5 + j]) * x[j];
    h[o] = round_act ? to_bf16(gelu(z)) : gelu(z);
  }
  for (int o = 0; o < 64; ++o) {
    double z = p[G_B2 + o];
    for (int j = 0; j < 64; ++j) z += to_bf16(p[G_W2 + o * 64 + j]) * h[j];
    g[o] = round_act ? to_bf16(gelu(z)) : gelu(z);
  }
  for (int o = 0; o < 64; ++o) {
    double z = p[G_B3 + o];
    for (int j = 0; j < 64; ++j) z += to_bf16(p[G_W3 + o * 64 + j]) * g[j];
    h[o] = round_act ? to_bf16(gelu(z)) : gelu(z);
  }
  double z = p[G_B4];
  for (int j = 0; j < 64; ++j) z += to_bf16(p[G_W4 + j]) * h[j];
  return z;
}

/* the gate's five features of slot t and a detection with innovation e */
static void gate_features(const orc_filter* f, const par_t* P, int t, const double* e, double d2,
                          double* feat) {
  double n2 = 0.0;
  for (int a = 0; a < f->dz; ++a) n2 += e[a] * e[a];
  feat[0] = d2;
  feat[1] = sqrt(n2);
  feat[2] = P->p[t];
  feat[3] = (double)((uint32_t)f->frame - P->lk[t]);
  feat[4] = P->logdetS[t];
}

int orc_set_gate(orc_filter* f, const float* params, double threshold) {
  if (!f) return 1;
  f->mlp_on = params != NULL;
  if (params) memcpy(f->mlp, params, sizeof f->mlp);
  f->mlp_thr = threshold;
  return 0;
}

/* whether the pair enters the table: the Mahalanobis test (R1), then, when
 * the learned gate is on, its logit against the threshold (decided on the
 * bf16-rounded forward pass) */
static int pair_gated(const orc_filter* f, const par_t* P, int t, const double* e, double d2,
                      double* margin) {
  if (!(d2 <= f->c.gate)) return 0;
  if (!f->mlp_on) return 1;
  double feat[5];
  gate_features(f, P, t, e, d2, feat);
  double lg = orc_mlp_logit(f->mlp, feat, 1);
  if (margin && fabs(lg - f->mlp_thr) < *margin) *margin = fabs(lg - f->mlp_thr);
  return lg >= f->mlp_thr;
}

static int build_table(const orc_filter* f, par_t* P) {
  int dx = f->dx, dz = f->dz, T = P->T, M = f->M;
  P->S = (double*)calloc(T * dz * dz + 1, sizeof(double));
  P->L = (double*)calloc(T * dz * dz + 1, sizeof(double));
  P->logdetS = (double*)calloc(T + 1, sizeof(double));
  P->dprob = (double*)calloc(T + 1, sizeof(double));
  P->ptr = (int*)calloc(T + 1, sizeof(int));
  P->gate_margin = INFINITY;
  P->mlp_margin = INFINITY;
  for (int t = 0; t < T; ++t) {
    double* S = P->S + t * dz * dz;
    for (int a = 0; a < dz; ++a)
      for (int b = 0; b < dz; ++b) S[a * dz + b] = P->P[t * dx * dx + a * dx + b] + f->c.R[a * dz + b];
    if (chol(dz, S, P->L + t * dz * dz)) return 5;
    P->logdetS[t] = logdet_from_chol(dz, P->L + t * dz * dz);
  }
  /* count gated pairs */
  int K = 0;
  double e[3];
  for (int t = 0; t < T; ++t) {
    P->ptr[t] = K;
    for (int i = 0; i < M; ++i) {
      innovation(f, P->m + t * dx, f->Z + i * dz, e);
      double d2 = mahal(dz, P->L + t * dz * dz, e);
      if (isfinite(f->c.gate)) {
        double mg = fabs(d2 - f->c.gate) / f->c.gate;
        if (mg < P->gate_margin) P->gate_margin = mg;
      }
      if (pair_gated(f, P, t, e, d2, &P->mlp_margin)) ++K;
    }
  }
  P->ptr[T] = K;
  P->K = K;
  P->meas = (int*)malloc(sizeof(int) * (K + 1));
  P->d2 = (double*)malloc(sizeof(double) * (K + 1));
  P->logC = (double*)malloc(sizeof(double) * (K + 1));
  P->q = (double*)malloc(sizeof(double) * (K + 1));
  P->e = (double*)malloc(sizeof(double) * (K * dz + 1));
  int k = 0;
  for (int t = 0; t < T; ++t) {
    for (int i = 0; i < M; ++i) {
      innovation(f, P->m + t * dx, f->Z + i * dz, e);
      double d2 = mahal(dz, P->L + t * dz * dz, e);
      if (!pair_gated(f, P, t, e, d2, NULL)) continue;
      P->meas[k] = i;
      P->d2[k] = d2;
      P->logC[k] = f->c.model == 1
                       ? log(f->c.p_d) + particle_logL(f, P->x + (size_t)t * f->c.n_particles * 5,
                                                      P->pw + (size_t)t * f->c.n_particles, f->Z + i * dz)
                       : log(f->c.p_d) - 0.5 * (d2 + P->logdetS[t] + dz * LOG2PI);
      P->q[k] = quad_Rinv(f, e);
      memcpy(P->e + k * dz, e, sizeof(double) * dz);
      ++k;
    }
  }
  /* posterior death probability (R2) */
  for (int t = 0; t < T; ++t) {
    double p = P->p[t];
    if (p <= 0.0) { P->dprob[t] = 1.0; continue; }
    if (p >= 1.0) { P->dprob[t] = 0.0; continue; }
    double sum_c = 0.0;
    for (int j = P->ptr[t]; j < P->ptr[t + 1]; ++j) sum_c += exp(P->logC[j]);
    double psi;
    if (sum_c > 0.0 && f->kappa <= 0.0) psi = INFINITY;
    else psi = (1.0 - f->c.p_d) + (sum_c > 0.0 ? sum_c / f->kappa : 0.0);
    P->dprob[t] = isinf(psi) ? 0.0 : (1.0 - p) / ((1.0 - p) + p * psi);
  }
  /* re-index the gated pairs by detection row; within a row slots ascend */
  P->rptr = (int*)calloc(M + 1, sizeof(int));
  P->rslot = (int*)malloc(sizeof(int) * (K + 1));
  P->rpair = (int*)malloc(sizeof(int) * (K + 1));
  for (int j = 0; j < K; ++j) P->rptr[P->meas[j] + 1]++;
  for (int i = 0; i < M; ++i) P->rptr[i + 1] += P->rptr[i];
  int* fill = (int*)calloc(M + 1, sizeof(int));
  for (int t = 0; t < T; ++t)
    for (int j = P->ptr[t]; j < P->ptr[t + 1]; ++j) {
      int i = P->meas[j];
      int pos = P->rptr[i] + fill[i]++;
      P->rslot[pos] = t;
      P->rpair[pos] = j;
    }
  free(fill);
  return 0;
}

/* ------------------------------------------------------------------ */
/* Exact child weight (reading R3) of (death mask, theta).              */
/* ------------------------------------------------------------------ */

/* log of the integral of prod_{i in W} N(z_i; Hx, R) against N(x; m, P)
 * for |W| = m >= 1, given sum of innovations e_i = z_i - H m and sum of
 * q_i = e_i^T R^{-1} e_i.  Uses prod N(z_i; Hx, R) = N(zbar; Hx, R/m) c(W). */
static double joint_loglik(const orc_filter* f, const double* Ppred, int m, const double* sum_e,
                           double sum_q) {
  int dx = f->dx, dz = f->dz;
  double ebar[3], Sm[9], Lm[9];
  for (int a = 0; a < dz; ++a) ebar[a] = sum_e[a] / m;
  for (int a = 0; a < dz; ++a)
    for (int b = 0; b < dz; ++b) Sm[a * dz + b] = Ppred[a * dx + b] + f->c.R[a * dz + b] / m;
  if (chol(dz, Sm, Lm)) return NAN;
  double spread = sum_q - m * quad_Rinv(f, ebar);
  return -0.5 * m * dz * LOG2PI - 0.5 * (m - 1) * f->logdetR - 0.5 * dz * log((double)m)
         - 0.5 * spread - 0.5 * logdet_from_chol(dz, Lm) - 0.5 * mahal(dz, Lm, ebar);
}

/* the table's log C[i, t] (-inf when the pair is not gated) */
static double pair_logC(const par_t* P, int t, int i) {
  for (int j = P->ptr[t]; j < P->ptr[t + 1]; ++j)
    if (P->meas[j] == i) return P->logC[j];
  return -INFINITY;
}

static double child_logw(const orc_filter* f, const par_t* P, double logw_parent,
                         const uint8_t* dead, const uint16_t* theta, int* n_alive_out,
                         int* n_clutter_out) {
  int dx = f->dx, dz = f->dz, T = P->T, M = f->M;
  double score = logw_parent;
  int n_clutter = 0, n_alive = 0;
  for (int i = 0; i < M; ++i) n_clutter += (theta[i] == 0);
  for (int t = 0; t < T; ++t) {
    if (dead[t]) {
      score += log(1.0 - P->p[t]);
      continue;
    }
    ++n_alive;
    int m = 0;
    double sum_e[3] = {0, 0, 0}, sum_q = 0.0, sum_logC = 0.0;
    for (int i = 0; i < M; ++i) {
      if (theta[i] != t + 1) continue;
      double e[3];
      innovation(f, P->m + t * dx, f->Z + i * dz, e);
      for (int a = 0; a < dz; ++a) sum_e[a] += e[a];
      sum_q += quad_Rinv(f, e);
      /* factorised mode: log C[i, t] of Eq. 2 */
      double d2 = mahal(dz, P->L + t * dz * dz, e);
      sum_logC += f->c.model == 1 ? pair_logC(P, t, i)
                                  : log(f->c.p_d) - 0.5 * (d2 + P->logdetS[t] + dz * LOG2PI);
      ++m;
    }
    score += log(P->p[t]);
    if (f->c.score_mode == 1) {
      score += (m == 0) ? log(1.0 - f->c.p_d) : sum_logC;
      continue;
    }
    if (m == 0) {
      score += log(1.0 - f->c.p_d);
    } else {
      /* log rho(m) + log m! = log P_D - lambda_d + (m-1) log lambda_d + log m */
      score += log(f->c.p_d) - f->c.lambda_d + (m > 1 ? (m - 1) * log(f->c.lambda_d) : 0.0)
               + log((double)m);
      score += joint_loglik(f, P->P + t * dx * dx, m, sum_e, sum_q);
    }
  }
  if (n_clutter > 0) score += n_clutter * f->log_kappa;
  if (n_alive_out) *n_alive_out = n_alive;
  if (n_clutter_out) *n_clutter_out = n_clutter;
  return score;
}

/* ------------------------------------------------------------------ */
/* Two-stage sampling of H_up children per parent (Section 3, R7)        */
/* ------------------------------------------------------------------ */
static double draw_u(const orc_filter* f, uint64_t uid, int n, int stream, int idx) {
  uint32_t ctr[4] = {(uint32_t)uid, (uint32_t)(uid >> 32), (uint32_t)(2 * n + stream),
                     (uint32_t)idx >> 2};
  uint32_t key[2] = {(uint32_t)f->c.seed, (uint32_t)(f->c.seed >> 32) ^ (uint32_t)f->frame};
  uint32_t out[4];
  orc_philox(ctr, key, out);
  return (double)(out[idx & 3] >> 8) * 0x1.0p-24;
}

static uint64_t child_key(int T, int M, const uint8_t* dead, const uint16_t* theta) {
  uint64_t h = 1469598103934665603ULL;            /* FNV-1a over the bytes */
  const uint8_t* b = (const uint8_t*)theta;
  for (int i = 0; i < T; ++i) { h ^= dead[i]; h *= 1099511628211ULL; }
  for (int i = 0; i < 2 * M; ++i) { h ^= b[i]; h *= 1099511628211ULL; }
  return h;
}

typedef struct { uint64_t key; int n; } keyidx_t;
static int cmp_keyidx(const void* a, const void* b) {
  const keyidx_t* x = (const keyidx_t*)a;
  const keyidx_t* y = (const keyidx_t*)b;
  if (x->key != y->key) return x->key < y->key ? -1 : 1;
  return x->n - y->n;
}

static void sample_children(const orc_filter* f, const hyp_t* y, par_t* P) {
  int T = P->T, M = f->M, HU = f->c.h_up;
  P->status = (int8_t*)calloc(HU, 1);
  P->logw = (double*)calloc(HU, sizeof(double));
  P->margin = (double*)calloc(HU, sizeof(double));
  P->n_alive = (int32_t*)calloc(HU, sizeof(int32_t));
  P->n_clutter = (int32_t*)calloc(HU, sizeof(int32_t));
  P->uid = (uint64_t*)calloc(HU, sizeof(uint64_t));
  P->theta = (uint16_t*)calloc((size_t)HU * M + 1, sizeof(uint16_t));
  P->dead = (uint8_t*)calloc((size_t)HU * T + 1, 1);
  for (int n = 0; n < HU; ++n) {
    uint8_t* dd = P->dead + (size_t)n * T;
    uint16_t* th = P->theta + (size_t)n * M;
    double mg = INFINITY;
    int ok = 1;
    P->uid[n] = orc_mix64(y->uid + GOLDEN * (uint64_t)(n + 1));
    /* stage 1: Bernoulli death of every slot with d_prob */
    for (int t = 0; t < T; ++t) {
      double dp = P->dprob[t];
      if (dp <= 0.0) { dd[t] = 0; continue; }
      if (dp >= 1.0) { dd[t] = 1; continue; }
      double u = draw_u(f, y->uid, n, 0, t);
      dd[t] = (u < dp);
      if (fabs(u - dp) < mg) mg = fabs(u - dp);
    }
    /* stage 2: each detection row draws clutter or a surviving gated slot
     * from its row of C'_k, normalised */
    for (int i = 0; i < M && ok; ++i) {
      double sum = f->kappa;
      int last = (f->kappa > 0.0) ? 0 : -1;
      for (int j = P->rptr[i]; j < P->rptr[i + 1]; ++j) {
        int t = P->rslot[j];
        if (dd[t]) continue;
        double w = exp(P->logC[P->rpair[j]]);
        sum += w;
        if (w > 0.0) last = t + 1;
      }
      if (!(sum > 0.0)) { ok = 0; break; }
      double u = draw_u(f, y->uid, n, 1, i);
      double x = u * sum;
      int choice = -1;
      double cum = f->kappa;
      if (f->kappa > 0.0) {
        if (x < cum) choice = 0;
        if (cum < sum && fabs(u - cum / sum) < mg) mg = fabs(u - cum / sum);
      }
      for (int j = P->rptr[i]; j < P->rptr[i + 1]; ++j) {
        int t = P->rslot[j];
        if (dd[t]) continue;
        double w = exp(P->logC[P->rpair[j]]);
        if (!(w > 0.0)) continue;
        cum += w;
        if (choice < 0 && x < cum) choice = t + 1;
        if (cum < sum && fabs(u - cum / sum) < mg) mg = fabs(u - cum / sum);
      }
      if (choice < 0) choice = last;
      th[i] = (uint16_t)choice;
    }
    P->margin[n] = mg;
    if (!ok) { P->status[n] = 0; P->logw[n] = -INFINITY; continue; }
    int na = 0, nc = 0;
    double s = child_logw(f, P, y->logw, dd, th, &na, &nc);
    P->n_alive[n] = na;
    P->n_clutter[n] = nc;
    P->logw[n] = s;
    P->status[n] = (isfinite(s) ? 1 : 0);
  }
  /* keep only unique children of this parent (R4) */
  keyidx_t* ks = (keyidx_t*)malloc(sizeof(keyidx_t) * HU);
  int nk = 0;
  for (int n = 0; n < HU; ++n)
    if (P->status[n] == 1) {
      ks[nk].key = child_key(T, M, P->dead + (size_t)n * T, P->theta + (size_t)n * M);
      ks[nk].n = n;
      ++nk;
    }
  qsort(ks, nk, sizeof(keyidx_t), cmp_keyidx);
  for (int a = 0; a < nk; ++a) {
    int na = ks[a].n;
    if (P->status[na] != 1) continue;
    for (int b = a + 1; b < nk && ks[b].key == ks[a].key; ++b) {
      int nb = ks[b].n;
      if (P->status[nb] != 1) continue;
      if (memcmp(P->dead + (size_t)na * T, P->dead + (size_t)nb * T, T) == 0 &&
          memcmp(P->theta + (size_t)na * M, P->theta + (size_t)nb * M, 2 * (size_t)M) == 0)
        P->status[nb] = 2;
    }
  }
  free(ks);
}

int orc_update(orc_filter* f, const float* Z, int M) {
  if (f->stage != 1) return 6;
  if (M < 0 || M > 65535) return 1;
  for (int i = 0; i < M * f->dz; ++i)
    if (!isfinite(Z[i])) return 1;
  f->M = M;
  f->Z = (double*)malloc(sizeof(double) * (M * f->dz + 1));
  for (int i = 0; i < M * f->dz; ++i) f->Z[i] = (double)Z[i];
  f->Hold = f->H;
  f->old_hyp = f->hyp;
  f->hyp = NULL;
  f->H = 0;
  f->par = (par_t*)calloc(f->Hold, sizeof(par_t));
  int err = 0;
  int nt = f->c.n_threads > 0 ? f->c.n_threads : 1;
  (void)nt;
#pragma omp parallel for schedule(dynamic, 1) num_threads(nt) reduction(| : err)
  for (int h = 0; h < f->Hold; ++h) {
    int e = predict_parent(f, &f->old_hyp[h], &f->par[h]);
    if (e) { err |= e; continue; }
    e = build_table(f, &f->par[h]);
    if (e) { err |= e; continue; }
    sample_children(f, &f->old_hyp[h], &f->par[h]);
  }
  if (err) return 5;
  f->stage = 2;
  return 0;
}

/* ------------------------------------------------------------------ */
/* Batched track update of a retained child (reading R6).               */
/* ------------------------------------------------------------------ */
static int kalman_multi(const orc_filter* f, const double* m0, const double* P0, const int* rows,
                        int mcount, double* m1, double* P1) {
  int dx = f->dx, dz = f->dz;
  double zbar[3] = {0, 0, 0}, nu[3], Rm[9], S[9], Sinv[9], K[18], A[36], AP[36];
  for (int r = 0; r < mcount; ++r)
    for (int a = 0; a < dz; ++a) zbar[a] += f->Z[rows[r] * dz + a];
  for (int a = 0; a < dz; ++a) {
    zbar[a] /= mcount;
    nu[a] = zbar[a] - m0[a];
  }
  for (int k = 0; k < dz * dz; ++k) Rm[k] = f->c.R[k] / mcount;
  for (int a = 0; a < dz; ++a)
    for (int b = 0; b < dz; ++b) S[a * dz + b] = P0[a * dx + b] + Rm[a * dz + b];
  if (spd_inverse(dz, S, Sinv)) return 5;
  for (int i = 0; i < dx; ++i)          /* K = P H^T S^{-1} */
    for (int b = 0; b < dz; ++b) {
      double s = 0.0;
      for (int a = 0; a < dz; ++a) s += P0[i * dx + a] * Sinv[a * dz + b];
      K[i * dz + b] = s;
    }
  for (int i = 0; i < dx; ++i) {
    double s = 0.0;
    for (int b = 0; b < dz; ++b) s += K[i * dz + b] * nu[b];
    m1[i] = m0[i] + s;
  }
  for (int i = 0; i < dx; ++i)          /* A = I - K H */
    for (int j = 0; j < dx; ++j) A[i * dx + j] = (i == j) - (j < dz ? K[i * dz + j] : 0.0);
  for (int i = 0; i < dx; ++i)
    for (int j = 0; j < dx; ++j) {
      double s = 0.0;
      for (int k = 0; k < dx; ++k) s += A[i * dx + k] * P0[k * dx + j];
      AP[i * dx + j] = s;
    }
  for (int i = 0; i < dx; ++i)          /* Joseph form */
    for (int j = 0; j < dx; ++j) {
      double s = 0.0;
      for (int k = 0; k < dx; ++k) s += AP[i * dx + k] * A[j * dx + k];
      for (int a = 0; a < dz; ++a)
        for (int b = 0; b < dz; ++b) s += K[i * dz + a] * Rm[a * dz + b] * K[j * dz + b];
      P1[i * dx + j] = s;
    }
  return 0;
}

/* ------------------------------------------------------------------ */
/* Pruning (Section 3, reading R5) and materialisation of the retained  */
/* children as the new hypothesis set, in (parent, draw) order.          */
/* ------------------------------------------------------------------ */
typedef struct { double l; int64_t idx; } cand_t;
static int cmp_cand(const void* a, const void* b) {
  const cand_t* x = (const cand_t*)a;
  const cand_t* y = (const cand_t*)b;
  if (x->l != y->l) return x->l > y->l ? -1 : 1;
  return x->idx < y->idx ? -1 : (x->idx > y->idx);
}
static int cmp_i64(const void* a, const void* b) {
  int64_t x = *(const int64_t*)a, y = *(const int64_t*)b;
  return x < y ? -1 : (x > y);
}

int orc_prune(orc_filter* f) {
  if (f->stage != 2) return 6;
  f->resample_margin = INFINITY;
  int HU = f->c.h_up, M = f->M, dx = f->dx;
  double mx = -INFINITY;
  int64_t nu = 0;
  for (int h = 0; h < f->Hold; ++h)
    for (int n = 0; n < HU; ++n)
      if (f->par[h].status[n] == 1) {
        ++nu;
        if (f->par[h].logw[n] > mx) mx = f->par[h].logw[n];
      }
  if (nu == 0) return 5;
  double s = 0.0;
  for (int h = 0; h < f->Hold; ++h)
    for (int n = 0; n < HU; ++n)
      if (f->par[h].status[n] == 1) s += exp(f->par[h].logw[n] - mx);
  f->lse_all = mx + log(s);
  double log_tau = log(f->c.tau);
  cand_t* cs = (cand_t*)malloc(sizeof(cand_t) * (nu + 1));
  int64_t nc = 0;
  for (int h = 0; h < f->Hold; ++h)
    for (int n = 0; n < HU; ++n)
      if (f->par[h].status[n] == 1) {
        double l = f->par[h].logw[n] - f->lse_all;
        if (l >= log_tau) {
          cs[nc].l = l;
          cs[nc].idx = (int64_t)h * HU + n;
          ++nc;
        }
      }
  qsort(cs, nc, sizeof(cand_t), cmp_cand);
  int nk = (int)(nc < f->c.h_max ? nc : f->c.h_max);
  if (nk == 0) { free(cs); return 5; }
  double mk = cs[0].l, sk = 0.0;
  for (int j = 0; j < nk; ++j) sk += exp(cs[j].l - mk);
  double lse_kept = mk + log(sk);
  int64_t* idx = (int64_t*)malloc(sizeof(int64_t) * nk);
  for (int j = 0; j < nk; ++j) idx[j] = cs[j].idx;
  qsort(idx, nk, sizeof(int64_t), cmp_i64);
  f->nkept = nk;
  f->kept_idx = idx;
  f->kept_logw = (double*)malloc(sizeof(double) * nk);
  f->kept_theta = (uint16_t*)calloc((size_t)nk * M + 1, sizeof(uint16_t));
  hyp_t* out = (hyp_t*)calloc(nk, sizeof(hyp_t));
  int* rows = (int*)malloc(sizeof(int) * (M + 1));
  for (int j = 0; j < nk; ++j) {
    int h = (int)(idx[j] / HU), n = (int)(idx[j] % HU);
    par_t* P = &f->par[h];
    int T = P->T;
    const uint8_t* dd = P->dead + (size_t)n * T;
    const uint16_t* th = P->theta + (size_t)n * M;
    double l = P->logw[n] - f->lse_all - lse_kept;
    f->kept_logw[j] = l;
    hyp_t* y = &out[j];
    y->logw = l;
    y->uid = P->uid[n];
    y->n = P->n_alive[n];
    y->lk = (uint32_t*)malloc(sizeof(uint32_t) * (y->n + 1));
    y->lb = (uint32_t*)malloc(sizeof(uint32_t) * (y->n + 1));
    y->m = (double*)malloc(sizeof(double) * (y->n * dx + 1));
    y->P = (double*)malloc(sizeof(double) * (y->n * dx * dx + 1));
    const int Np = f->c.n_particles;
    if (f->c.model == 1) {
      y->x = (double*)malloc(sizeof(double) * ((size_t)y->n * Np * 5 + 1));
      y->pw = (double*)malloc(sizeof(double) * ((size_t)y->n * Np + 1));
    }
    int* newpos = (int*)malloc(sizeof(int) * (T + 1));
    int a = 0;
    for (int t = 0; t < T; ++t) {
      if (dd[t]) { newpos[t] = -1; continue; }
      newpos[t] = a;
      int mc = 0;
      for (int i = 0; i < M; ++i)
        if (th[i] == t + 1) rows[mc++] = i;
      y->lk[a] = P->lk[t];
      y->lb[a] = P->lb[t];
      if (f->c.model == 1) {   /* particle update (R15e) and moments (R15f) */
        double* xa = y->x + (size_t)a * Np * 5;
        double* wa = y->pw + (size_t)a * Np;
        if (mc == 0) {
          memcpy(xa, P->x + (size_t)t * Np * 5, sizeof(double) * 5 * Np);
          memcpy(wa, P->pw + (size_t)t * Np, sizeof(double) * Np);
        } else {
          particle_update(f, P->lk[t], P->lb[t], P->x + (size_t)t * Np * 5, P->pw + (size_t)t * Np, rows, mc,
                          xa, wa, &f->resample_margin);
        }
        particle_moments(Np, xa, wa, y->m + a * dx, y->P + a * dx * dx);
      } else if (mc == 0) {
        memcpy(y->m + a * dx, P->m + t * dx, sizeof(double) * dx);
        memcpy(y->P + a * dx * dx, P->P + t * dx * dx, sizeof(double) * dx * dx);
      } else if (kalman_multi(f, P->m + t * dx, P->P + t * dx * dx, rows, mc, y->m + a * dx,
                              y->P + a * dx * dx)) {
        free(newpos); free(rows); free(cs);
        return 5;
      }
      ++a;
    }
    for (int i = 0; i < M; ++i)
      f->kept_theta[(size_t)j * M + i] = th[i] ? (uint16_t)(newpos[th[i] - 1] + 1) : 0;
    free(newpos);
  }
  free(rows);
  free(cs);
  f->hyp = out;
  f->H = nk;
  f->stage = 3;
  return 0;
}

/* ------------------------------------------------------------------ */
/* introspection                                                        */
/* ------------------------------------------------------------------ */
int orc_import_particles(orc_filter* f, const double* x, const double* logw) {
  if (f->c.model != 1) return 1;
  int Np = f->c.n_particles;
  size_t off = 0;
  for (int h = 0; h < f->H; ++h) {
    hyp_t* y = &f->hyp[h];
    free(y->x);
    free(y->pw);
    y->x = (double*)malloc(sizeof(double) * ((size_t)y->n * Np * 5 + 1));
    y->pw = (double*)malloc(sizeof(double) * ((size_t)y->n * Np + 1));
    for (int t = 0; t < y->n; ++t, ++off) {
      memcpy(y->x + (size_t)t * Np * 5, x + off * Np * 5, sizeof(double) * Np * 5);
      memcpy(y->pw + (size_t)t * Np, logw + off * Np, sizeof(double) * Np);
      particle_moments(Np, y->x + (size_t)t * Np * 5, y->pw + (size_t)t * Np, y->m + t * 5, y->P + t * 25);
    }
  }
  return 0;
}

int orc_export_particles(const orc_filter* f, double* x, double* logw) {
  if (f->c.model != 1) return 1;
  int Np = f->c.n_particles;
  size_t off = 0;
  for (int h = 0; h < f->H; ++h) {
    const hyp_t* y = &f->hyp[h];
    for (int t = 0; t < y->n; ++t, ++off) {
      memcpy(x + off * Np * 5, y->x + (size_t)t * Np * 5, sizeof(double) * Np * 5);
      memcpy(logw + off * Np, y->pw + (size_t)t * Np, sizeof(double) * Np);
    }
  }
  return 0;
}

int orc_slot_particles(const orc_filter* f, int h, int t, double* x, double* logw) {
  if (f->c.model != 1 || !f->par || h < 0 || h >= f->Hold || t < 0 || t >= f->par[h].T) return 1;
  int Np = f->c.n_particles;
  memcpy(x, f->par[h].x + (size_t)t * Np * 5, sizeof(double) * Np * 5);
  memcpy(logw, f->par[h].pw + (size_t)t * Np, sizeof(double) * Np);
  return 0;
}

double orc_resample_margin(const orc_filter* f) { return f->resample_margin; }

int orc_num_parents(const orc_filter* f) { return f->par ? f->Hold : 0; }
int orc_parent_slots(const orc_filter* f, int h) {
  return (f->par && h >= 0 && h < f->Hold) ? f->par[h].T : -1;
}

int orc_slot(const orc_filter* f, int h, int t, uint32_t* lk, uint32_t* lb, double* mean,
             double* cov, double* p, double* dprob, double* logdetS) {
  if (!f->par || h < 0 || h >= f->Hold || t < 0 || t >= f->par[h].T) return 1;
  const par_t* P = &f->par[h];
  int dx = f->dx;
  *lk = P->lk[t];
  *lb = P->lb[t];
  memcpy(mean, P->m + t * dx, sizeof(double) * dx);
  memcpy(cov, P->P + t * dx * dx, sizeof(double) * dx * dx);
  *p = P->p[t];
  *dprob = P->dprob ? P->dprob[t] : NAN;
  *logdetS = P->logdetS ? P->logdetS[t] : NAN;
  return 0;
}

int orc_pair(const orc_filter* f, int h, int t, int i, double* d2, double* logC, double* e,
             double* q) {
  if (!f->par || h < 0 || h >= f->Hold || t < 0 || t >= f->par[h].T || i < 0 || i >= f->M)
    return -1;
  const par_t* P = &f->par[h];
  int dx = f->dx, dz = f->dz;
  innovation(f, P->m + t * dx, f->Z + i * dz, e);
  *d2 = mahal(dz, P->L + t * dz * dz, e);
  *logC = f->c.model == 1 ? log(f->c.p_d) + particle_logL(f, P->x + (size_t)t * f->c.n_particles * 5,
                                                          P->pw + (size_t)t * f->c.n_particles, f->Z + i * dz)
                          : log(f->c.p_d) - 0.5 * (*d2 + P->logdetS[t] + dz * LOG2PI);
  *q = quad_Rinv(f, e);
  return pair_gated(f, P, t, e, *d2, NULL);
}

int orc_parent_pairs(const orc_filter* f, int h, int32_t* ptr, int32_t* meas, double* logC, double* q,
                     double* e) {
  if (!f->par || h < 0 || h >= f->Hold) return -1;
  const par_t* P = &f->par[h];
  if (meas) {
    for (int t = 0; t <= P->T; ++t) ptr[t] = P->ptr[t];
    for (int k = 0; k < P->K; ++k) {
      meas[k] = P->meas[k];
      logC[k] = P->logC[k];
      q[k] = P->q[k];
      for (int a = 0; a < f->dz; ++a) e[k * f->dz + a] = P->e[k * f->dz + a];
    }
  }
  return P->K;
}

double orc_mlp_margin(const orc_filter* f, int h) {
  if (!f->par || h < 0 || h >= f->Hold) return NAN;
  return f->par[h].mlp_margin;
}

int orc_gate_eval(const orc_filter* f, int h, int t, int i, double* feat, double* logit) {
  if (!f->par || h < 0 || h >= f->Hold || t < 0 || t >= f->par[h].T || i < 0 || i >= f->M)
    return -1;
  const par_t* P = &f->par[h];
  double e[3] = {0.0, 0.0, 0.0};
  innovation(f, P->m + t * f->dx, f->Z + i * f->dz, e);
  double d2 = mahal(f->dz, P->L + t * f->dz * f->dz, e);
  gate_features(f, P, t, e, d2, feat);
  *logit = f->mlp_on ? orc_mlp_logit(f->mlp, feat, 1) : NAN;
  return 0;
}

double orc_gate_margin(const orc_filter* f, int h) {
  if (!f->par || h < 0 || h >= f->Hold) return NAN;
  return f->par[h].gate_margin;
}

int orc_children(const orc_filter* f, int8_t* status, double* logw, double* margin,
                 int32_t* n_alive, uint64_t* uid) {
  if (!f->par || f->stage < 2) return 6;
  int HU = f->c.h_up;
  for (int h = 0; h < f->Hold; ++h) {
    const par_t* P = &f->par[h];
    size_t o = (size_t)h * HU;
    memcpy(status + o, P->status, HU);
    memcpy(logw + o, P->logw, sizeof(double) * HU);
    memcpy(margin + o, P->margin, sizeof(double) * HU);
    memcpy(n_alive + o, P->n_alive, sizeof(int32_t) * HU);
    memcpy(uid + o, P->uid, sizeof(uint64_t) * HU);
  }
  return 0;
}

int orc_child(const orc_filter* f, int h, int n, uint8_t* dead, uint16_t* theta) {
  if (!f->par || f->stage < 2 || h < 0 || h >= f->Hold || n < 0 || n >= f->c.h_up) return 1;
  const par_t* P = &f->par[h];
  memcpy(dead, P->dead + (size_t)n * P->T, P->T);
  memcpy(theta, P->theta + (size_t)n * f->M, sizeof(uint16_t) * f->M);
  return 0;
}

int orc_kept(const orc_filter* f, int64_t* idx, double* logw_norm, double* lse_all) {
  if (f->stage < 3 || !f->kept_idx) return -1;
  if (idx) memcpy(idx, f->kept_idx, sizeof(int64_t) * f->nkept);
  if (logw_norm) memcpy(logw_norm, f->kept_logw, sizeof(double) * f->nkept);
  if (lse_all) *lse_all = f->lse_all;
  return f->nkept;
}

int orc_kept_theta(const orc_filter* f, uint16_t* theta) {
  if (f->stage < 3 || !f->kept_theta) return -1;
  memcpy(theta, f->kept_theta, sizeof(uint16_t) * (size_t)f->nkept * f->M);
  return f->M;
}

/* ------------------------------------------------------------------ */
/* Estimates (reading R9) and per-detection unassigned probability       */
/* ------------------------------------------------------------------ */
int orc_estimates(const orc_filter* f, int cap, int* n_out, uint32_t* lk, uint32_t* lb,
                  double* mean, double* cov, double* r, double* pmf, int pmf_cap,
                  int* map_index) {
  int dx = f->dx;
  int nmax = 0;
  for (int h = 0; h < f->H; ++h)
    if (f->hyp[h].n > nmax) nmax = f->hyp[h].n;
  double* card = (double*)calloc(nmax + 1, sizeof(double));
  for (int h = 0; h < f->H; ++h) card[f->hyp[h].n] += exp(f->hyp[h].logw);
  int nhat = 0;
  for (int n = 1; n <= nmax; ++n)
    if (card[n] > card[nhat]) nhat = n;
  if (pmf)
    for (int n = 0; n < pmf_cap; ++n) pmf[n] = n <= nmax ? card[n] : 0.0;
  free(card);
  int best = -1;
  for (int h = 0; h < f->H; ++h)
    if (f->hyp[h].n == nhat && (best < 0 || f->hyp[h].logw > f->hyp[best].logw)) best = h;
  if (map_index) *map_index = best;
  *n_out = nhat;
  if (nhat > cap) return 3;
  const hyp_t* y = &f->hyp[best];
  for (int t = 0; t < nhat; ++t) {
    lk[t] = y->lk[t];
    lb[t] = y->lb[t];
    memcpy(mean + t * dx, y->m + t * dx, sizeof(double) * dx);
    memcpy(cov + t * dx * dx, y->P + t * dx * dx, sizeof(double) * dx * dx);
    double s = 0.0;
    for (int h = 0; h < f->H; ++h)
      for (int u = 0; u < f->hyp[h].n; ++u)
        if (f->hyp[h].lk[u] == y->lk[t] && f->hyp[h].lb[u] == y->lb[t]) {
          s += exp(f->hyp[h].logw);
          break;
        }
    r[t] = s;
  }
  return 0;
}

int orc_meas_assoc(const orc_filter* f, double* r_u) {
  if (f->stage < 3 || !f->kept_theta) return 6;
  for (int i = 0; i < f->M; ++i) {
    double s = 0.0;
    for (int j = 0; j < f->nkept; ++j)
      if (f->kept_theta[(size_t)j * f->M + i] == 0) s += exp(f->kept_logw[j]);
    r_u[i] = s;
  }
  return 0;
}

/* ------------------------------------------------------------------ */
/* Brute force: every death mask and every gated association of parent h */
/* with its exact weight (R3).  Tiny inputs only.                       */
/* ------------------------------------------------------------------ */
int orc_bruteforce(const orc_filter* f, int h, int cap, uint8_t* dead, uint16_t* theta,
                   double* logw) {
  if (!f->par || f->stage < 2 || h < 0 || h >= f->Hold) return -1;
  const par_t* P = &f->par[h];
  int T = P->T, M = f->M;
  if (T > 16) return -1;
  int count = 0;
  uint8_t dd[16];
  uint16_t* th = (uint16_t*)calloc(M + 1, sizeof(uint16_t));
  int* nopt = (int*)calloc(M + 1, sizeof(int));
  int* opt = (int*)calloc((size_t)(M + 1) * (T + 1), sizeof(int));
  int* digit = (int*)calloc(M + 1, sizeof(int));
  for (uint32_t mask = 0; mask < (1u << T); ++mask) {
    for (int t = 0; t < T; ++t) dd[t] = (mask >> t) & 1u;
    int empty_row = 0;
    for (int i = 0; i < M; ++i) {
      int k = 0;
      if (f->kappa > 0.0) opt[i * (T + 1) + k++] = 0;
      for (int j = P->rptr[i]; j < P->rptr[i + 1]; ++j)
        if (!dd[P->rslot[j]]) opt[i * (T + 1) + k++] = P->rslot[j] + 1;
      nopt[i] = k;
      if (k == 0) empty_row = 1;
    }
    if (empty_row) continue;
    memset(digit, 0, sizeof(int) * (M + 1));
    for (;;) {
      for (int i = 0; i < M; ++i) th[i] = (uint16_t)opt[i * (T + 1) + digit[i]];
      double s = child_logw(f, P, f->old_hyp[h].logw, dd, th, NULL, NULL);
      if (isfinite(s)) {
        if (count >= cap) { count = -2; goto done; }
        memcpy(dead + (size_t)count * T, dd, T);
        memcpy(theta + (size_t)count * M, th, sizeof(uint16_t) * M);
        logw[count] = s;
        ++count;
      }
      int i = 0;
      while (i < M && ++digit[i] == nopt[i]) digit[i++] = 0;
      if (i == M) break;
    }
  }
done:
  free(th); free(nopt); free(opt); free(digit);
  return count;
}

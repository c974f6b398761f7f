// Device-side data layout and arithmetic shared by the kernels of the
// multi-detection GLMB update (arXiv 2512.06230, Section 3).
//
// Layout in HBM (all structure-of-arrays, one GPU):
//   components  mean as two float32 words per coordinate (hi + lo, so a
//               position of 5 km keeps ~1e-9 m resolution while all
//               arithmetic stays FP32), packed upper-triangular FP32
//               covariance, labels, log prior existence;
//   table       gated (component, detection) pairs in CSR by component;
//   hypotheses  CSR of component indices, FP64 log-weights, 64-bit uids;
//   children    one int64 fixed-point log-weight per (parent, draw).
//
// Log-weights of children are sums of thousands of FP32 terms.  Each term is
// converted to int64 fixed point (2^-32 resolution) and the sums are exact
// integer sums, so identical terms cancel exactly between children and the
// result does not depend on summation order.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace glmb {

// device error flags (sticky per frame, read by the host at sync points)
enum : uint32_t {
  kErrPairs = 1u,       // gated pairs beyond capacity
  kErrHash = 2u,        // update hash table full
  kErrUpdates = 4u,     // distinct track updates beyond capacity
  kErrComps = 8u,       // components beyond capacity
  kErrNumeric = 16u,    // covariance not positive definite even in FP64
  kErrEntries = 32u,    // hypothesis entries beyond capacity
  kErrSlots = 64u,      // per-hypothesis staging beyond the planned size
  kErrInput = 128u,     // a detection is NaN or infinite
  kErrGate = 256u,      // a tensor-core wait of the learned gate ran out of time
  kErrTimeout = 512u,   // a scan's look-back waited past its limit
  // internal index checks (a violated invariant; the access is skipped)
  kErrChkSurv = 1024u,  // a survivor index outside the frame's children
  kErrChkComp = 2048u,  // a component index outside the working table
  kErrChkRemap = 4096u, // a new-hypothesis entry outside the tables it names
};

constexpr float kFxScale = 4294967296.0f;          // 2^32
constexpr double kFxInv = 2.3283064365386963e-10;  // 2^-32
constexpr long long kKeyInvalid = (long long)0x8000000000000000ULL;
constexpr uint32_t kNewTag = 0x80000000u;          // hypothesis entry -> hash-table slot
constexpr float kLog2Pi = 1.8378770664093453f;
constexpr uint32_t kOne24 = 1u << 24;

struct Model {
  int dx, dz, ncov;       // state dim, detection dim, packed covariance length
  int h_up;
  float dt;
  float Q[21];            // packed upper triangle, row-major
  float R[9], Rinv[9];    // dz x dz full
  float logdetR;
  float log_pd, log_1mpd; // log P_D, log(1 - P_D) (may be -inf)
  float lambda_d, log_lambda_d;
  float log_kappa;        // -inf when kappa == 0
  int kappa_zero;
  int score_mode;         // 0 joint likelihood of a track's detections, 1 product of C entries
  float gate;
  float log_ps, log_1mps;
  long long fx_log_kappa; // fixed-point log kappa (0 when kappa == 0)
  uint32_t seed_lo, seed_hi;
  int particle;           // track model: 0 Gaussian (Kalman), 1 weighted particles (CTRV)
};

// Particle track model (model 1): the constants its kernels use, in FP64.
struct PartModel {
  int np;                 // particles per component
  double dt, sigma_a, sigma_w, ess_frac;
  double Rinv[4];         // R^-1, 2 x 2 row-major
  double lnorm;           // (1/2) log det R + log 2 pi
  double log_pd;
  uint32_t seed_lo, seed_hi;
};

// Sizes of the current frame.  Kernels read them from device memory, so a
// frame's launches depend only on capacities (grids are grid-stride or
// persistent) and the host needs no synchronisation inside a frame.
struct FrameDev {
  int n_comp;             // components of the state table
  int nb;                 // births of this frame
  int T;                  // n_comp + nb: components of the working table
  int M;                  // detections
  int H;                  // parents (hypotheses before the update)
  int frame;              // frame number: birth labels and the random-number key
  const float* Z;         // detections [M][dz] (device memory)
};

struct CompTable {
  float* mhi;             // [dx][cap]
  float* mlo;             // [dx][cap]
  float* cov;             // [ncov][cap]
  uint32_t* lk;
  uint32_t* lb;
  float* logp;            // log prior existence
  float* log1mp;          // log(1 - prior existence)
  int cap;
  double* px;             // particle model: per component 6 rows of np values
                          // (px, py, v, heading, turn rate, log-weight)
};

struct PairTable {
  uint32_t* cnt;          // [comp] gated count (count pass)
  uint32_t* ptr;          // [comp + 1] CSR offsets
  uint32_t* meas;         // [pair]
  float* logC;            // [pair] log Eq. 2 entry
  float* q;               // [pair] e^T R^-1 e
  float* e;               // [dz][cap_pairs]
  uint32_t* dthr;         // [comp] death threshold on 24-bit uniforms
  float* dprob;           // [comp]
  float* logdetS;         // [comp]
  long long cap_pairs;
  // the parts of a component's alive term that depend only on (component,
  // m): S_m^-1 (packed) and the m-only constants, for m = 1 .. kSlmM, built
  // once per frame for the first slm_cap components (every parent holding
  // the component reads them): slm[((m - 1) * (NP + 1) + k) * slm_cap + c],
  // sln[(m - 1) * slm_cap + c] the infinite-term count
  float* slm;
  int8_t* sln;
  int slm_cap;
};
constexpr int kSlmM = 8;

struct HypTable {
  uint32_t* ptr;          // [cap_h + 1]
  uint32_t* comp;         // [cap_entries]
  double* logw;
  unsigned long long* uid;
  uint16_t* theta;        // [cap_h][max_meas]
};

__host__ __device__ __forceinline__ int pidx(int n, int i, int j) {
  // packed upper-triangular index, i <= j, row-major
  return i * n - (i * (i - 1)) / 2 + (j - i);
}

// splitmix64 output function (Steele, Lea, Flood, OOPSLA 2014)
__host__ __device__ __forceinline__ unsigned long long mix64(unsigned long long z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  return z ^ (z >> 31);
}

// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11): ten rounds of two
// 32x32->64 multiplies, with the Weyl key schedule.
__device__ __forceinline__ uint4 philox10(uint4 c, uint2 k) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    const uint32_t hi0 = __umulhi(0xD2511F53u, c.x), lo0 = 0xD2511F53u * c.x;
    const uint32_t hi1 = __umulhi(0xCD9E8D57u, c.z), lo1 = 0xCD9E8D57u * c.z;
    c = make_uint4(hi1 ^ c.y ^ k.x, lo1, hi0 ^ c.w ^ k.y, lo0);
    k.x += 0x9E3779B9u;
    k.y += 0xBB67AE85u;
  }
  return c;
}

// Philox4x32-10 of counters (c0, c1, c2, cc) in which only the last word
// varies (a child's draws of one stream: c0, c1 the parent's uid, c2 the
// draw and stream, cc the chunk of four slots or rows).  The first round
// multiplies c0 and c2, the second round's first product depends only on
// the first round's word 0 and the third round's second product only on
// the second round's word 2: none of these depends on cc.  PhiloxRun holds
// them (folded with the round keys), so a call costs 16 of the 20 wide
// multiplications and gives the same four words as philox10.
struct PhiloxRun {
  uint32_t w2;   // round-1 word 2 before the XOR with cc
  uint32_t y0;   // round-2 word 0 before the XOR with mulhi(M1, w2 ^ cc)
  uint32_t z0;   // round-3 word 0 before the XOR with mullo(M1, w2 ^ cc)
  uint32_t z1;   // round-3 word 1
  uint32_t z2;   // round-3 word 2 before the XOR with its mulhi(M0, .)
};

__device__ __forceinline__ PhiloxRun philox_run(uint32_t c0, uint32_t c1, uint32_t c2, uint2 k) {
  constexpr uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u, W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
  const uint32_t hiA = __umulhi(M0, c0), loA = M0 * c0;
  const uint32_t hiB = __umulhi(M1, c2), loB = M1 * c2;
  const uint32_t x0 = hiB ^ c1 ^ k.x;                       // round-1 words: x0, loB, hiA ^ cc ^ k.y, loA
  const uint32_t hiC = __umulhi(M0, x0), loC = M0 * x0;     // round 2, first product
  const uint32_t y2 = hiC ^ loA ^ (k.y + W1);               // round-2 words: ., ., y2, loC
  const uint32_t hiF = __umulhi(M1, y2), loF = M1 * y2;     // round 3, second product
  PhiloxRun p;
  p.w2 = hiA ^ k.y;
  p.y0 = loB ^ (k.x + W0);
  p.z0 = hiF ^ (k.x + 2u * W0);
  p.z1 = loF;
  p.z2 = loC ^ (k.y + 2u * W1);
  return p;
}

// The round keys k + r (W0, W1) are loop-invariant: with a key that is a
// launch parameter they are formed once per thread in uniform registers.
// Where the key is a per-thread value (an out-of-line function's argument),
// philox_at_rk forms them per call instead, so they take no registers
// across the caller's loop.
__device__ __forceinline__ uint4 philox_at(const PhiloxRun& p, uint32_t cc, uint2 k) {
  constexpr uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u;
  const uint32_t w2 = p.w2 ^ cc;
  const uint32_t hiD = __umulhi(M1, w2), loD = M1 * w2;     // round 2, second product
  const uint32_t y0 = hiD ^ p.y0;
  const uint32_t hiE = __umulhi(M0, y0), loE = M0 * y0;     // round 3, first product
  uint4 c = make_uint4(loD ^ p.z0, p.z1, hiE ^ p.z2, loE);
  k.x += 3u * 0x9E3779B9u;
  k.y += 3u * 0xBB67AE85u;
#pragma unroll
  for (int r = 3; r < 10; ++r) {
    const uint32_t hi0 = __umulhi(M0, c.x), lo0 = M0 * c.x;
    const uint32_t hi1 = __umulhi(M1, c.z), lo1 = M1 * c.z;
    c = make_uint4(hi1 ^ c.y ^ k.x, lo1, hi0 ^ c.w ^ k.y, lo0);
    k.x += 0x9E3779B9u;
    k.y += 0xBB67AE85u;
  }
  return c;
}

__device__ __forceinline__ uint4 philox_at_rk(const PhiloxRun& p, uint32_t cc, uint2 k) {
  asm volatile("" : "+r"(k.x), "+r"(k.y));
  return philox_at(p, cc, k);
}

__device__ __forceinline__ uint32_t word_of(const uint4& r, int b) {
  return b == 0 ? r.x : b == 1 ? r.y : b == 2 ? r.z : r.w;
}

// Programmatic dependent launch: wait until the kernel this one depends on
// has finished and its writes are visible (the next kernel is launched when
// this one completes, without a separate launch round trip).
__device__ __forceinline__ void pdl_enter() {
  asm volatile("griddepcontrol.wait;" ::: "memory");
}

__device__ __forceinline__ long long fx_of(float x) { return __float2ll_rn(x * kFxScale); }

// v * 2^-32 as a float, from the two 32-bit halves of v (no FP64 arithmetic,
// which runs at a small fraction of the FP32 rate on this part)
__device__ __forceinline__ float fx_to_f(long long v) {
  return (float)(int)(v >> 32) + (float)(uint32_t)v * 2.3283064365386963e-10f;
}

// One thread's running log-sum-exp of fixed-point keys: the largest key m
// and a compensated (Kahan) FP32 sum of exp(key - m), rescaled when m grows;
// n counts the keys.  Partials are combined in FP64 (lse_merge).
struct LseAcc {
  long long m;
  float s, c;
  unsigned n;
  __device__ __forceinline__ LseAcc() : m(kKeyInvalid), s(0.f), c(0.f), n(0u) {}
  __device__ __forceinline__ void add(long long k) {
    ++n;
    float term = 1.f;
    if (m == kKeyInvalid) {
      m = k;
    } else if (k > m) {
      const float sc = expf(fx_to_f(m - k));
      s *= sc;
      c *= sc;
      m = k;
    } else {
      term = expf(fx_to_f(k - m));
    }
    const float y = term - c;
    const float t = s + y;
    c = (t - s) - y;
    s = t;
  }
  __device__ __forceinline__ double sum() const { return (double)s - (double)c; }
};

// sum * exp(m - M): a partial (m, sum) rescaled to the overall maximum M
__device__ __forceinline__ double lse_rescale(long long m, double sum, long long M) {
  return (m == kKeyInvalid || !(sum > 0.0) || M == kKeyInvalid) ? 0.0 : sum * (double)expf(fx_to_f(m - M));
}

// a + b for hi/lo float pairs (Knuth two-sum, then renormalise)
__device__ __forceinline__ void df_add(float& hi, float& lo, float b) {
  const float s = hi + b;
  const float bb = s - hi;
  const float err = (hi - (s - bb)) + (b - bb);
  const float l = lo + err;
  hi = s + l;
  lo = l - (hi - s);
}

// Cholesky of an N x N SPD matrix (full, row-major) in type T; returns false
// when a pivot is not above 16 eps trace(S) (then the caller redoes the
// factorisation in FP64).
template <typename T, int N>
__device__ __forceinline__ bool chol_n(const T (&S)[N][N], T (&L)[N][N], T& logdet, T eps) {
  T tr = 0;
#pragma unroll
  for (int i = 0; i < N; ++i) tr += S[i][i];
  const T thr = T(16) * eps * tr;
  logdet = 0;
#pragma unroll
  for (int j = 0; j < N; ++j) {
    T s = S[j][j];
#pragma unroll
    for (int k = 0; k < j; ++k) s -= L[j][k] * L[j][k];
    if (!(s > thr)) return false;
    const T d = sqrt(s);
    L[j][j] = d;
    logdet += T(2) * log(d);
#pragma unroll
    for (int i = j + 1; i < N; ++i) {
      T t = S[i][j];
#pragma unroll
      for (int k = 0; k < j; ++k) t -= L[i][k] * L[j][k];
      L[i][j] = t / d;
    }
#pragma unroll
    for (int i = 0; i < j; ++i) L[i][j] = 0;
  }
  return true;
}

// x^T (L L^T)^-1 x by forward substitution
template <typename T, int N>
__device__ __forceinline__ T mahal_n(const T (&L)[N][N], const T (&x)[N]) {
  T y[N];
  T s = 0;
#pragma unroll
  for (int i = 0; i < N; ++i) {
    T t = x[i];
#pragma unroll
    for (int k = 0; k < i; ++k) t -= L[i][k] * y[k];
    y[i] = t / L[i][i];
    s += y[i] * y[i];
  }
  return s;
}

// logdet(S) and x^T S^-1 x with an FP64 fallback for ill-conditioned S.
// Returns 0 (FP32), 1 (FP64 used) or -1 (not positive definite).
template <int N>
__device__ __forceinline__ int logdet_mahal(const float (&S)[N][N], const float (&x)[N],
                                            float& logdet, float& d2) {
  float L[N][N];
  float ld;
  if (chol_n<float, N>(S, L, ld, 1.1920929e-7f)) {
    logdet = ld;
    d2 = mahal_n<float, N>(L, x);
    return 0;
  }
  double Sd[N][N], Ld[N][N], xd[N], ldd;
#pragma unroll
  for (int i = 0; i < N; ++i) {
    xd[i] = x[i];
#pragma unroll
    for (int j = 0; j < N; ++j) Sd[i][j] = S[i][j];
  }
  if (!chol_n<double, N>(Sd, Ld, ldd, 2.220446049250313e-16)) return -1;
  logdet = (float)ldd;
  d2 = (float)mahal_n<double, N>(Ld, xd);
  return 1;
}

// Per-track term of the child log-weight (exact GLMB target weight).
// alive with m >= 1 detections:
//   log p + log P_D - lambda_d + (m-1) log lambda_d + log m + J(W)
//   J = -(m dz/2) log 2pi - ((m-1)/2) log|R| - (dz/2) log m
//       - 1/2 (sum q - m ebar^T R^-1 ebar) - 1/2 log|S_m| - 1/2 ebar^T S_m^-1 ebar,
//   S_m = H P H^T + R/m, ebar = (sum e)/m  (prod_i N(z_i;Hx,R) = N(zbar;Hx,R/m) c(W));
// alive, undetected: log p + log(1 - P_D).
// The part that depends only on (track, m) -- S_m^-1, log|S_m| and the
// constant terms -- is SlotM; the rest is a quadratic form of the fixed-point
// sums.  Every evaluation goes through these two functions, so equal inputs
// give bit-identical terms.  The finite part is returned in fixed point;
// infinite parts are counted.
template <int DZ>
struct SlotM {
  float Sinv[DZ * (DZ + 1) / 2];   // packed upper triangle of S_m^-1
  float c;                         // all m-only terms, log|S_m| included
  int ninf;                        // infinite terms (or -1: S_m not positive definite)
};

template <int DZ>
__device__ __forceinline__ SlotM<DZ> make_slot_m(const Model& md, const float (&HPH)[DZ][DZ],
                                                 float logp, int m) {
  SlotM<DZ> s;
  s.ninf = 0;
  float c = 0.f;
  if (isinf(logp)) ++s.ninf; else c += logp;
  if (isinf(md.log_pd)) ++s.ninf; else c += md.log_pd;
  c -= md.lambda_d;
  if (m > 1) {
    if (md.lambda_d <= 0.f) ++s.ninf; else c += (float)(m - 1) * md.log_lambda_d;
  }
  const float fm = (float)m, inv_m = 1.f / fm, logm = logf(fm);
  c += logm;
  c += -0.5f * fm * (float)DZ * kLog2Pi - 0.5f * (fm - 1.f) * md.logdetR - 0.5f * (float)DZ * logm;
  float Sm[DZ][DZ];
#pragma unroll
  for (int a = 0; a < DZ; ++a)
#pragma unroll
    for (int b = 0; b < DZ; ++b) Sm[a][b] = HPH[a][b] + md.R[a * DZ + b] * inv_m;
  // S_m^-1 = L^-T L^-1 and log|S_m| from the Cholesky factor (FP64 when a
  // pivot falls below 16 eps trace)
  float L[DZ][DZ], ld;
  float Li[DZ][DZ];
  if (chol_n<float, DZ>(Sm, L, ld, 1.1920929e-7f)) {
#pragma unroll
    for (int j = 0; j < DZ; ++j)
#pragma unroll
      for (int i = 0; i < DZ; ++i) {
        float t = (i == j) ? 1.f : 0.f;
#pragma unroll
        for (int k = 0; k < i; ++k) t -= L[i][k] * Li[k][j];
        Li[i][j] = (i < j) ? 0.f : t / L[i][i];
      }
  } else {
    double Sd[DZ][DZ], Ld[DZ][DZ], ldd, Lid[DZ][DZ];
#pragma unroll
    for (int a = 0; a < DZ; ++a)
#pragma unroll
      for (int b = 0; b < DZ; ++b) Sd[a][b] = Sm[a][b];
    if (!chol_n<double, DZ>(Sd, Ld, ldd, 2.220446049250313e-16)) {
      s.ninf = -1;
      s.c = 0.f;
      return s;
    }
#pragma unroll
    for (int j = 0; j < DZ; ++j)
#pragma unroll
      for (int i = 0; i < DZ; ++i) {
        double t = (i == j) ? 1.0 : 0.0;
#pragma unroll
        for (int k = 0; k < i; ++k) t -= Ld[i][k] * Lid[k][j];
        Lid[i][j] = (i < j) ? 0.0 : t / Ld[i][i];
      }
#pragma unroll
    for (int i = 0; i < DZ; ++i)
#pragma unroll
      for (int j = 0; j < DZ; ++j) Li[i][j] = (float)Lid[i][j];
    ld = (float)ldd;
  }
  int k = 0;
#pragma unroll
  for (int i = 0; i < DZ; ++i)
#pragma unroll
    for (int j = i; j < DZ; ++j, ++k) {
      float t = 0.f;
#pragma unroll
      for (int q = 0; q < DZ; ++q) t += Li[q][i] * Li[q][j];
      s.Sinv[k] = t;
    }
  s.c = c - 0.5f * ld;
  return s;
}

template <int DZ>
__device__ __forceinline__ long long term_from(const Model& md, const SlotM<DZ>& s, int m,
                                               const long long* se, long long sq, int& ninf) {
  if (s.ninf < 0) { ninf = 1; return 0; }
  ninf = s.ninf;
  const float inv_m = 1.f / (float)m;
  float sum_e[DZ], ebar[DZ];
#pragma unroll
  for (int a = 0; a < DZ; ++a) {
    sum_e[a] = fx_to_f(se[a]);
    ebar[a] = sum_e[a] * inv_m;
  }
  float qR = 0.f;
#pragma unroll
  for (int a = 0; a < DZ; ++a)
#pragma unroll
    for (int b = 0; b < DZ; ++b) qR += sum_e[a] * md.Rinv[a * DZ + b] * sum_e[b];
  const float spread = fx_to_f(sq) - qR * inv_m;
  float d2 = 0.f;
  int k = 0;
#pragma unroll
  for (int i = 0; i < DZ; ++i)
#pragma unroll
    for (int j = i; j < DZ; ++j, ++k) d2 += (i == j ? 1.f : 2.f) * ebar[i] * s.Sinv[k] * ebar[j];
  return fx_of(s.c - 0.5f * spread - 0.5f * d2);
}

// Factorised mode (score_mode 1): a track alive with detection set W
// contributes log p + sum_{i in W} log C[i, t] (Eq. 2 entries, P_D included),
// or log p + log(1 - P_D) when W is empty; sq then carries the fixed-point
// sum of log C over W.
__device__ __forceinline__ long long factor_term(const Model& md, float logp, int m, long long sq, int& ninf) {
  ninf = 0;
  float t = 0.f;
  if (isinf(logp)) ++ninf; else t += logp;
  if (m == 0) {
    if (isinf(md.log_1mpd)) ++ninf; else t += md.log_1mpd;
    return fx_of(t);
  }
  return fx_of(t) + sq;
}

template <int DZ>
__device__ __forceinline__ long long alive_term(const Model& md, const float (&HPH)[DZ][DZ],
                                                float logp, int m, const long long* se,
                                                long long sq, int& ninf) {
  if (md.score_mode == 1) return factor_term(md, logp, m, sq, ninf);
  if (m == 0) {
    ninf = 0;
    float t = 0.f;
    if (isinf(logp)) ++ninf; else t += logp;
    if (isinf(md.log_1mpd)) ++ninf; else t += md.log_1mpd;
    return fx_of(t);
  }
  const SlotM<DZ> s = make_slot_m<DZ>(md, HPH, logp, m);
  return term_from<DZ>(md, s, m, se, sq, ninf);
}

__device__ __forceinline__ long long dead_term(float log1mp, int& ninf) {
  ninf = isinf(log1mp) ? 1 : 0;
  return ninf ? 0 : fx_of(log1mp);
}

template <int DZ>
__device__ __forceinline__ void load_HPH(const CompTable& ct, int ncov, int dx, int c,
                                         float (&HPH)[DZ][DZ]) {
#pragma unroll
  for (int a = 0; a < DZ; ++a)
#pragma unroll
    for (int b = a; b < DZ; ++b) {
      const float v = ct.cov[(size_t)pidx(dx, a, b) * ct.cap + c];
      HPH[a][b] = v;
      HPH[b][a] = v;
    }
}

// key of one association decision for the per-parent duplicate test
__device__ __forceinline__ unsigned long long row_key(int i, int theta) {
  return mix64(((unsigned long long)(uint32_t)i << 32) | (uint32_t)theta);
}
__device__ __forceinline__ unsigned long long dead_key(int t) {
  return mix64(0xFFFFFFFF00000000ULL | (uint32_t)t);
}
__device__ __forceinline__ unsigned long long wset_key(int i) {
  return mix64(0x5A5A5A5A00000000ULL ^ (unsigned long long)(uint32_t)i);
}

// ---- log-sum-exp and the posterior death probability (reading R2) ----
__device__ __forceinline__ void lse_push(float& m, float& s, float x) {
  if (x == -INFINITY) return;
  if (x > m) {
    s = (m == -INFINITY ? 0.f : s * __expf(m - x)) + 1.f;
    m = x;
  } else {
    s += __expf(x - m);
  }
}

// combines the (max, scaled sum) pairs of the 32 lanes of a warp
__device__ __forceinline__ void lse_warp(float& lm, float& ls) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const float m2 = __shfl_xor_sync(0xFFFFFFFFu, lm, o);
    const float s2 = __shfl_xor_sync(0xFFFFFFFFu, ls, o);
    const float m = fmaxf(lm, m2);
    if (m != -INFINITY) {
      ls = (lm == -INFINITY ? 0.f : ls * __expf(lm - m)) + (m2 == -INFINITY ? 0.f : s2 * __expf(m2 - m));
      lm = m;
    }
  }
}

// d_prob = (1 - p) / ((1 - p) + p psi), psi = (1 - P_D) + sum C / kappa,
// from the LSE (lm, ls) of log C - log kappa over the component's gated
// pairs (any: at least one pair), and its threshold on 24-bit uniforms
__device__ __forceinline__ void death_prob(const Model& md, float logp, float log1mp, float lm, float ls,
                                           bool any, float& d_out, uint32_t& thr_out) {
  float logpsi;
  if (md.kappa_zero && any) {
    logpsi = INFINITY;
  } else {
    float m = lm, s = ls;
    lse_push(m, s, md.log_1mpd);
    logpsi = (m == -INFINITY) ? -INFINITY : m + logf(s);
  }
  float d;
  if (logp == -INFINITY) d = 1.f;
  else if (log1mp == -INFINITY) d = 0.f;
  else if (logpsi == INFINITY) d = 0.f;
  else if (logpsi == -INFINITY) d = 1.f;
  else d = 1.f / (1.f + expf(logp + logpsi - log1mp));
  d_out = d;
  thr_out = d >= 1.f ? kOne24 : (d <= 0.f ? 0u : (uint32_t)ceilf(d * 16777216.f));
}

}  // namespace glmb

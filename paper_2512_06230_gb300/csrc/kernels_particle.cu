// Particle track model (Section 3 of arXiv 2512.06230: every labeled state
// is a set of P weighted particles moved by constant-turn-rate-and-velocity
// kinematics; births are sampled from their Gaussian; the retained tracks
// get a particle update with resampling).  A component's particles are
// FP64 states (px, py, v, heading, turn rate) and normalised log-weights,
// laid out per component as six rows of P values (CompTable::px).  The
// moment fields of the component (mean, covariance) hold the particles'
// weighted moments, with the mean rounded to FP32 (mlo = 0), so that a
// detection's innovation z - mhi (computed in FP32 by the table kernel) is
// exact and the fixed-point innovation sums of the regeneration give the
// mean detection to FP64 accuracy.
//
// Random numbers: Philox4x32-10 keyed by (seed_lo ^ 0x5851F42D,
// seed_hi ^ frame), counter (label_k, label_b, particle, stream << 24 |
// call); a call's words give two normals by the Box-Muller cosine branch.
// Stream 1: a survivor's accelerations (a, alpha); stream 2: a birth
// particle's five normals (calls 0-2); stream 3: the resampling offset.
#include <math.h>

#include "glmb_kernels.h"

namespace glmb {

namespace {

constexpr uint32_t kPartKeyXor = 0x5851F42Du;
constexpr int kPartThreads = 256;

__device__ __forceinline__ double unit_open(uint32_t w) { return ((double)w + 0.5) * 2.3283064365386963e-10; }

__device__ __forceinline__ uint4 part_words(const PartModel& pm, int frame, uint32_t lk, uint32_t lb, uint32_t p,
                                            uint32_t stream, uint32_t call) {
  return philox10(make_uint4(lk, lb, p, (stream << 24) | call),
                  make_uint2(pm.seed_lo ^ kPartKeyXor, pm.seed_hi ^ (uint32_t)frame));
}

// cos(2 pi u) as cospi(2 u): 2 u is exact, so no rounded multiple of pi
// enters the argument
__device__ __forceinline__ void normal_pair(const uint4& w, double& n0, double& n1) {
  n0 = sqrt(-2.0 * log(unit_open(w.x))) * cospi(2.0 * unit_open(w.y));
  n1 = sqrt(-2.0 * log(unit_open(w.z))) * cospi(2.0 * unit_open(w.w));
}

// one CTRV step over dt; the arc (v / w)(sin(psi + w dt) - sin psi, ...)
// as v dt sinc(h)(cos, sin)(psi + h), h = w dt / 2, valid at w = 0.  The
// half-angle terms sin h, cos h and sinc h come from their Taylor series
// when |h| < 0.03 (the first omitted terms, h^8 / 9! and h^8 / 8!, are
// below 1e-16 of the sums) and (cos, sin)(psi + h) from the angle sum, so
// a particle takes one sincos instead of three transcendental calls.
__device__ __forceinline__ void ctrv(const double (&x)[5], double dt, double a, double al, double (&y)[5]) {
  const double h = 0.5 * x[4] * dt;
  double sh, ch, sinc;
  if (fabs(h) < 0.03) {
    const double h2 = h * h;
    sinc = 1.0 - h2 / 6.0 * (1.0 - h2 / 20.0 * (1.0 - h2 / 42.0));
    sh = h * sinc;
    ch = 1.0 - 0.5 * h2 * (1.0 - h2 / 12.0 * (1.0 - h2 / 30.0));
  } else {
    sincos(h, &sh, &ch);
    sinc = sh / h;
  }
  const double vdt = x[2] * dt * sinc;
  double s0, c0;
  sincos(x[3], &s0, &c0);
  const double s1 = s0 * ch + c0 * sh, c1 = c0 * ch - s0 * sh;
  y[0] = x[0] + vdt * c1 + 0.5 * dt * dt * c0 * a;
  y[1] = x[1] + vdt * s1 + 0.5 * dt * dt * s0 * a;
  y[2] = x[2] + dt * a;
  y[3] = x[3] + x[4] * dt + 0.5 * dt * dt * al;
  y[4] = x[4] + dt * al;
}

__device__ __forceinline__ double* prow(const CompTable& ct, int np, int c, int k) {
  return ct.px + ((size_t)c * 6 + k) * np;
}

// sums of N values over the block (every thread gets the totals); red
// holds (threads / 32) * N doubles
template <int N>
__device__ void block_sum(double (&v)[N], double* red) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
  for (int k = 0; k < N; ++k)
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v[k] += __shfl_xor_sync(0xFFFFFFFFu, v[k], o);
  if (lane == 0)
#pragma unroll
    for (int k = 0; k < N; ++k) red[w * N + k] = v[k];
  __syncthreads();
#pragma unroll
  for (int k = 0; k < N; ++k) {
    double s = 0.0;
    for (int i = 0; i < nw; ++i) s += red[i * N + k];
    v[k] = s;
  }
  __syncthreads();
}

__device__ double block_max(double v, double* red) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xFFFFFFFFu, v, o));
  if (lane == 0) red[w] = v;
  __syncthreads();
  double m = -INFINITY;
  for (int i = 0; i < nw; ++i) m = fmax(m, red[i]);
  __syncthreads();
  return m;
}

// weighted mean and covariance of component c's particles into its moment
// fields (mean rounded to FP32, mlo = 0); wv holds the particles' weights
__device__ void write_moments(const CompTable& ct, int np, int c, const double* wv, double* red) {
  double s[5] = {0, 0, 0, 0, 0};
  for (int p = threadIdx.x; p < np; p += blockDim.x) {
    const double w = wv[p];
#pragma unroll
    for (int k = 0; k < 5; ++k) s[k] += w * prow(ct, np, c, k)[p];
  }
  block_sum<5>(s, red);
  double q[15];
#pragma unroll
  for (int k = 0; k < 15; ++k) q[k] = 0.0;
  for (int p = threadIdx.x; p < np; p += blockDim.x) {
    const double w = wv[p];
    double d[5];
#pragma unroll
    for (int k = 0; k < 5; ++k) d[k] = prow(ct, np, c, k)[p] - s[k];
    int k = 0;
#pragma unroll
    for (int i = 0; i < 5; ++i)
#pragma unroll
      for (int j = i; j < 5; ++j, ++k) q[k] += w * d[i] * d[j];
  }
  block_sum<15>(q, red);
  if (threadIdx.x == 0) {
    const size_t cap = ct.cap;
#pragma unroll
    for (int k = 0; k < 5; ++k) {
      ct.mhi[k * cap + c] = (float)s[k];
      ct.mlo[k * cap + c] = 0.f;
    }
#pragma unroll
    for (int k = 0; k < 15; ++k) ct.cov[(size_t)k * cap + c] = (float)q[k];
  }
  __syncthreads();   // wv is reused by the next component
}

// Prediction, particle by particle (a flat grid over the working table's
// components x particles, so that the FP64 work of one component runs on
// into the next without a barrier): a survivor's particle takes one CTRV
// step with its own accelerations; a birth's particle is drawn through the
// Cholesky factor that the host stored with the birth.  Particle 0 of each
// component writes its label and existence.
__global__ void __launch_bounds__(kPartThreads) particle_step_kernel(Model md, PartModel pm, CompTable src,
                                                                     CompTable dst, const FrameDev* fs,
                                                                     const double* __restrict__ births) {
  pdl_enter();
  const int n = fs->n_comp, nb = fs->nb, frame = fs->frame, np = pm.np;
  const long long total = (long long)(n + nb) * np;
  const double lw_b = -log((double)np);
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < total;
       i += (long long)gridDim.x * blockDim.x) {
    const int c = (int)(i / np), p = (int)(i - (long long)c * np);
    if (c < n) {
      const uint32_t lk = src.lk[c], lb = src.lb[c];
      double x[5], y[5], n0, n1;
#pragma unroll
      for (int k = 0; k < 5; ++k) x[k] = prow(src, np, c, k)[p];
      normal_pair(part_words(pm, frame, lk, lb, (uint32_t)p, 1u, 0u), n0, n1);
      ctrv(x, pm.dt, pm.sigma_a * n0, pm.sigma_w * n1, y);
#pragma unroll
      for (int k = 0; k < 5; ++k) prow(dst, np, c, k)[p] = y[k];
      prow(dst, np, c, 5)[p] = prow(src, np, c, 5)[p];
      if (p == 0) {
        dst.lk[c] = lk;
        dst.lb[c] = lb;
        dst.logp[c] = md.log_ps;
        dst.log1mp[c] = md.log_1mps;
      }
    } else {
      const int b = c - n;
      const double* rec = births + (size_t)b * kBirthRec;
      const double* L = rec + kBirthChol;   // lower triangle, row-major
      double xi[6];
#pragma unroll
      for (int j = 0; j < 3; ++j)
        normal_pair(part_words(pm, frame, (uint32_t)frame, (uint32_t)b, (uint32_t)p, 2u, (uint32_t)j), xi[2 * j],
                    xi[2 * j + 1]);
#pragma unroll
      for (int a = 0; a < 5; ++a) {
        double v = rec[1 + a];
#pragma unroll
        for (int k = 0; k <= a; ++k) v += L[a * (a + 1) / 2 + k] * xi[k];
        prow(dst, np, c, a)[p] = v;
      }
      prow(dst, np, c, 5)[p] = lw_b;
      if (p == 0) {
        const double r = rec[0];
        dst.lk[c] = (uint32_t)frame;
        dst.lb[c] = (uint32_t)b;
        dst.logp[c] = r > 0.0 ? (float)log(r) : -INFINITY;
        dst.log1mp[c] = r < 1.0 ? (float)log1p(-r) : -INFINITY;
      }
    }
  }
}

// The working table's moments: one block of 64 threads per component,
// threads over its particles, one pass with offsets from its particle 0, d_p = x_p - x_0:
// mean = x_0 + sum w d, covariance = sum w d d^T - (sum w d)(sum w d)^T
// (the weights sum to one), mean rounded to FP32 with a zero low part.
__global__ void __launch_bounds__(kPartThreads) particle_moments_kernel(PartModel pm, CompTable ct,
                                                                       const FrameDev* fs) {
  pdl_enter();
  __shared__ double part[kPartThreads / 32][20];
  const int T = fs->T, np = pm.np, lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  for (int c = blockIdx.x; c < T; c += gridDim.x) {
    double x0[5];
#pragma unroll
    for (int k = 0; k < 5; ++k) x0[k] = prow(ct, np, c, k)[0];
    double v[20];   // sum w d (5), sum w d d^T (15, packed)
#pragma unroll
    for (int k = 0; k < 20; ++k) v[k] = 0.0;
    for (int p = threadIdx.x; p < np; p += blockDim.x) {
      const double w = exp(prow(ct, np, c, 5)[p]);
      double d[5];
#pragma unroll
      for (int k = 0; k < 5; ++k) {
        d[k] = prow(ct, np, c, k)[p] - x0[k];
        v[k] += w * d[k];
      }
      int k = 5;
#pragma unroll
      for (int i = 0; i < 5; ++i)
#pragma unroll
        for (int j = i; j < 5; ++j, ++k) v[k] += w * d[i] * d[j];
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1)
#pragma unroll
      for (int k = 0; k < 20; ++k) v[k] += __shfl_xor_sync(0xFFFFFFFFu, v[k], o);
    if (lane == 0)
#pragma unroll
      for (int k = 0; k < 20; ++k) part[wid][k] = v[k];
    __syncthreads();
    if (threadIdx.x == 0) {
      const int nw = blockDim.x >> 5;
      double t[20];
      for (int k = 0; k < 20; ++k) {
        t[k] = 0.0;
        for (int i = 0; i < nw; ++i) t[k] += part[i][k];
      }
      const size_t cap = ct.cap;
      for (int k = 0; k < 5; ++k) {
        ct.mhi[k * cap + c] = (float)(x0[k] + t[k]);
        ct.mlo[k * cap + c] = 0.f;
      }
      int k = 0;
      for (int i = 0; i < 5; ++i)
        for (int j = i; j < 5; ++j, ++k) ct.cov[(size_t)k * cap + c] = (float)(t[5 + k] - t[i] * t[j]);
    }
    __syncthreads();
  }
}

// Compatibility entries: one warp per component, lanes over particles;
// log C = log P_D + log sum_p w_p N(z; (px, py)_p, R) for each of the
// component's gated pairs (the table kernels wrote the pairs, gated on
// the moments), then the death probability from these entries.  The
// offsets run in FP32: a particle's position relative to the component's
// FP32 mean, (px, py)_p - mhi, is formed once in FP64 and rounded, and a
// pair's innovation z - mhi is the table's (exact in FP32 when z and mhi
// are within a factor of two, as for any gated pair away from the
// origin); z - (px, py)_p is their difference.  The mixture's sum is in
// FP32 too (log C is stored in FP32).  Particles beyond kRegP per lane
// are re-read from the particle rows.
constexpr int kRegP = 8;   // particles held in registers per lane (256 per warp)

__global__ void __launch_bounds__(256) particle_logc_kernel(Model md, PartModel pm, CompTable ct, PairTable pt,
                                                            const FrameDev* fs) {
  pdl_enter();
  const int T = fs->T, np = pm.np, lane = threadIdx.x & 31;
  if (fs->M > 0 && !__isGlobal(fs->Z)) return;   // flagged by the count kernel
  const int nwarps = (gridDim.x * blockDim.x) >> 5;
  const unsigned cap_p = (unsigned)min(pt.cap_pairs, (long long)0xFFFFFFFF);
  const size_t capp = (size_t)pt.cap_pairs;
  const float r0 = (float)pm.Rinv[0], r1 = (float)(pm.Rinv[1] + pm.Rinv[2]), r3 = (float)pm.Rinv[3];
  const float lc0 = (float)(pm.log_pd - pm.lnorm);
  for (int c = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; c < T; c += nwarps) {
    const unsigned k0 = pt.ptr[c], k1 = min(pt.ptr[c + 1], cap_p);
    const double mx = (double)ct.mhi[c], my = (double)ct.mhi[(size_t)ct.cap + c];
    float ox[kRegP], oy[kRegP], ow[kRegP];
#pragma unroll
    for (int j = 0; j < kRegP; ++j) {
      const int p = lane + 32 * j;
      const bool in = p < np;
      ox[j] = in ? (float)(prow(ct, np, c, 0)[p] - mx) : 0.f;
      oy[j] = in ? (float)(prow(ct, np, c, 1)[p] - my) : 0.f;
      ow[j] = in ? (float)prow(ct, np, c, 5)[p] : -INFINITY;
    }
    float lm = -INFINITY, ls = 0.f;
    bool any = false;
    for (unsigned k = k0; k < k1; ++k) {
      const float ex = pt.e[k], ey = pt.e[capp + k];
      // the register-held particles' terms are independent: their maximum,
      // then the sum of their exponentials (no dependent chain through expf)
      float l[kRegP];
      float m = -INFINITY;
#pragma unroll
      for (int j = 0; j < kRegP; ++j) {
        const float dx = ex - ox[j], dy = ey - oy[j];
        l[j] = ow[j] - 0.5f * (r0 * dx * dx + r1 * dx * dy + r3 * dy * dy);
        m = fmaxf(m, l[j]);
      }
      float s = 0.f;
      if (m > -INFINITY) {
#pragma unroll
        for (int j = 0; j < kRegP; ++j) s += expf(l[j] - m);
      }
      auto push = [&](float dx, float dy, float w) {
        const float lv = w - 0.5f * (r0 * dx * dx + r1 * dx * dy + r3 * dy * dy);
        if (lv > m) {
          s = s * expf(m - lv) + 1.f;
          m = lv;
        } else if (lv > -INFINITY) {
          s += expf(lv - m);
        }
      };
      for (int p = lane + 32 * kRegP; p < np; p += 32)
        push(ex - (float)(prow(ct, np, c, 0)[p] - mx), ey - (float)(prow(ct, np, c, 1)[p] - my),
             (float)prow(ct, np, c, 5)[p]);
      // the warp's maximum, then each lane's sum rescaled to it once and
      // added across the warp
      float mw = m;
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) mw = fmaxf(mw, __shfl_xor_sync(0xFFFFFFFFu, mw, o));
      float sw = m == -INFINITY ? 0.f : s * expf(m - mw);
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) sw += __shfl_xor_sync(0xFFFFFFFFu, sw, o);
      const float logC = mw == -INFINITY ? -INFINITY : lc0 + mw + logf(sw);
      if (lane == 0) pt.logC[k] = logC;
      any = true;
      if (!md.kappa_zero) lse_push(lm, ls, logC - md.log_kappa);
    }
    if (lane == 0) death_prob(md, ct.logp[c], ct.log1mp[c], lm, ls, any, pt.dprob[c], pt.dthr[c]);
  }
}

// Regeneration: one block (64 threads) per kept component (copied to its compacted
// position) and per distinct (component, detection set) update (written
// after the kept ones): log w_p -= (m / 2) (zbar - h_p)^T R^-1 (zbar - h_p)
// (the product of the m detections' likelihoods up to a factor common to
// all particles), normalised; systematic resampling when the effective
// sample size is below ess_frac * P.  Dynamic shared memory: P doubles
// (cumulative weights).
__global__ void __launch_bounds__(kPartThreads) particle_remap_kernel(
    Model md, PartModel pm, CompTable src, CompTable dst, const uint32_t* __restrict__ newpos,
    const uint32_t* __restrict__ flag, const FrameDev* __restrict__ fs, const unsigned* __restrict__ n_keep_dev,
    const uint32_t* __restrict__ upd_src, const uint32_t* __restrict__ upd_m, const long long* __restrict__ upd_se,
    int cap_upd, const unsigned* __restrict__ n_upd_dev, const unsigned* __restrict__ n_surv_dev, unsigned* err) {
  pdl_enter();
  extern __shared__ double cum[];
  __shared__ double red[(kPartThreads / 32) * 15];
  __shared__ double runs[kPartThreads];
  if (*n_surv_dev == 0u || (*(volatile unsigned*)err & kErrFatal)) return;
  const int n_src = fs->T, np = pm.np, frame = fs->frame;
  const unsigned n_keep = *n_keep_dev;
  const unsigned n_upd = min(*n_upd_dev, (unsigned)cap_upd);
  if ((long long)n_keep + n_upd > dst.cap) return;   // flagged by the remap kernel
  for (long long x = blockIdx.x; x < (long long)n_src + n_upd; x += gridDim.x) {
    if (x < n_src) {
      const int c = (int)x;
      if (!flag[c]) continue;
      if (newpos[c] >= n_keep) {
        if (threadIdx.x == 0) atomicOr(err, kErrChkComp);
        continue;
      }
      const int d = (int)newpos[c];
      for (int k = 0; k < 6; ++k)
        for (int p = threadIdx.x; p < np; p += blockDim.x) prow(dst, np, d, k)[p] = prow(src, np, c, k)[p];
      if (threadIdx.x < 5) {
        dst.mhi[threadIdx.x * (size_t)dst.cap + d] = src.mhi[threadIdx.x * (size_t)src.cap + c];
        dst.mlo[threadIdx.x * (size_t)dst.cap + d] = 0.f;
      }
      if (threadIdx.x < 15) dst.cov[threadIdx.x * (size_t)dst.cap + d] = src.cov[threadIdx.x * (size_t)src.cap + c];
      if (threadIdx.x == 0) {
        dst.lk[d] = src.lk[c];
        dst.lb[d] = src.lb[c];
        dst.logp[d] = src.logp[c];
        dst.log1mp[d] = src.log1mp[c];
      }
      continue;
    }
    const int u = (int)(x - n_src);
    const int c = (int)upd_src[u];
    if (c >= n_src) {
      if (threadIdx.x == 0) atomicOr(err, kErrChkComp);
      continue;
    }
    const int d = (int)n_keep + u;
    const double m = (double)max(upd_m[u], 1u);   // an update holds at least one detection
    double zb[2];
#pragma unroll
    for (int a = 0; a < 2; ++a)
      zb[a] = (double)src.mhi[a * (size_t)src.cap + c] + (double)upd_se[(size_t)a * cap_upd + u] * kFxInv / m;
    // reweight (kept in the destination's weight row), then normalise
    double mx = -INFINITY;
    for (int p = threadIdx.x; p < np; p += blockDim.x) {
      const double ex = zb[0] - prow(src, np, c, 0)[p], ey = zb[1] - prow(src, np, c, 1)[p];
      const double l = prow(src, np, c, 5)[p] -
                       0.5 * m * (pm.Rinv[0] * ex * ex + (pm.Rinv[1] + pm.Rinv[2]) * ex * ey + pm.Rinv[3] * ey * ey);
      prow(dst, np, d, 5)[p] = l;
      mx = fmax(mx, l);
    }
    mx = block_max(mx, red);
    double sv[1] = {0.0};
    for (int p = threadIdx.x; p < np; p += blockDim.x) {
      const double e = exp(prow(dst, np, d, 5)[p] - mx);
      cum[p] = e;
      sv[0] += e;
    }
    block_sum<1>(sv, red);
    const double lse = mx + log(sv[0]), inv = 1.0 / sv[0];
    // normalised weights cum[p] = exp(l_p - mx) / sum; the log-weights
    // l_p - lse stay in the destination row
    double s2[1] = {0.0};
    for (int p = threadIdx.x; p < np; p += blockDim.x) {
      prow(dst, np, d, 5)[p] -= lse;
      const double w = cum[p] * inv;
      cum[p] = w;
      s2[0] += w * w;
    }
    block_sum<1>(s2, red);
    if (1.0 / s2[0] < pm.ess_frac * np) {
      // cumulative weights: each thread scans a contiguous run, then the
      // runs' totals are scanned by thread 0
      const int per = (np + blockDim.x - 1) / blockDim.x, b0 = threadIdx.x * per, b1 = min(np, b0 + per);
      double run = 0.0;
      for (int p = b0; p < b1; ++p) {
        run += cum[p];
        cum[p] = run;
      }
      runs[threadIdx.x] = run;
      __syncthreads();
      if (threadIdx.x == 0) {
        double acc = 0.0;
        for (int t = 0; t < (int)blockDim.x; ++t) {
          const double v = runs[t];
          runs[t] = acc;
          acc += v;
        }
      }
      __syncthreads();
      const double off = runs[threadIdx.x];
      for (int p = b0; p < b1; ++p) cum[p] += off;
      __syncthreads();
      const double u0 = unit_open(part_words(pm, frame, src.lk[c], src.lb[c], 0u, 3u, 0u).x);
      const double lw_r = -log((double)np);
      for (int r = threadIdx.x; r < np; r += blockDim.x) {
        const double target = (u0 + r) / np;
        int lo = 0, hi = np - 1;   // first k with cum[k] > target, else np - 1
        while (lo < hi) {
          const int mid = (lo + hi) >> 1;
          if (cum[mid] > target) hi = mid;
          else lo = mid + 1;
        }
#pragma unroll
        for (int k = 0; k < 5; ++k) prow(dst, np, d, k)[r] = prow(src, np, c, k)[lo];
      }
      __syncthreads();   // every cumulative weight read before it is overwritten
      for (int r = threadIdx.x; r < np; r += blockDim.x) {
        prow(dst, np, d, 5)[r] = lw_r;
        cum[r] = 1.0 / np;
      }
    } else {
      for (int k = 0; k < 5; ++k)
        for (int p = threadIdx.x; p < np; p += blockDim.x) prow(dst, np, d, k)[p] = prow(src, np, c, k)[p];
    }
    __syncthreads();
    write_moments(dst, np, d, cum, red);
    if (threadIdx.x == 0) {
      dst.lk[d] = src.lk[c];
      dst.lb[d] = src.lb[c];
      dst.logp[d] = src.logp[c];
      dst.log1mp[d] = src.log1mp[c];
    }
  }
}

}  // namespace

void launch_particle_predict(const Model& md, const PartModel& pm, const CompTable& src, const CompTable& dst,
                             const FrameDev* fs, const double* births_dev, int grid, cudaStream_t s) {
  launch_k(particle_step_kernel, grid, kPartThreads, 0, s, md, pm, src, dst, fs, births_dev);
  launch_k(particle_moments_kernel, 4 * grid, 64, 0, s, pm, dst, fs);
}

void launch_particle_logc(const Model& md, const PartModel& pm, const CompTable& ct, const PairTable& pt,
                          const FrameDev* fs, int grid, cudaStream_t s) {
  launch_k(particle_logc_kernel, grid, 256, 0, s, md, pm, ct, pt, fs);
}

void launch_particle_remap(const Model& md, const PartModel& pm, const CompTable& src, const CompTable& dst,
                           const uint32_t* newpos, const uint32_t* flag, const FrameDev* fs,
                           const unsigned* n_keep_dev, const uint32_t* upd_src, const uint32_t* upd_m,
                           const long long* upd_se, int cap_upd, const unsigned* n_upd_dev,
                           const unsigned* n_surv_dev, unsigned* err, int grid, cudaStream_t s) {
  // 64-thread blocks: several updates in flight per SM, each with short
  // block reductions
  launch_k(particle_remap_kernel, 4 * grid, 64, (size_t)pm.np * sizeof(double), s, md, pm, src, dst, newpos,
           flag, fs, n_keep_dev, upd_src, upd_m, upd_se, cap_upd, n_upd_dev, n_surv_dev, err);
}

int particle_remap_smem(int np) { return np * (int)sizeof(double); }

}  // namespace glmb

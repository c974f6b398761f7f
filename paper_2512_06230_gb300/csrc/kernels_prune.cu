// Normalisation, truncation and the batched track update of the retained
// children (arXiv 2512.06230, Section 3: weights below tau are discarded,
// the H_max most likely hypotheses are kept, and one update is run per
// distinct (track, detection set)), plus the estimate reductions.
#include <algorithm>

#include "../../include/glmb.h"
#include "glmb_kernels.h"

namespace glmb {

constexpr int kRedThreads = 256;

__device__ __forceinline__ long long warp_max_ll(long long v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = max(v, __shfl_xor_sync(0xFFFFFFFFu, v, o));
  return v;
}
__device__ __forceinline__ double warp_sum_d(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xFFFFFFFFu, v, o);
  return v;
}

// ---------------------------------------------------------------------------
// Global log-sum-exp over unique children, FP64.  Two grid passes (max, then
// sum of exp); each pass's last block combines the per-block partials in
// block order, so the result does not depend on scheduling.
// ---------------------------------------------------------------------------
// (max, sum of exp(x - max)) pairs in fixed-point keys
struct Lse {
  long long m;   // kKeyInvalid (the smallest 64-bit integer) when empty
  double s;
};
__device__ __forceinline__ long long warp_max_key(long long v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = max(v, __shfl_xor_sync(0xFFFFFFFFu, v, o));
  return v;
}
// Block-wide pair from per-thread pairs: the block maximum first (integer),
// then each thread's sum rescaled to it with one FP32 exponential of the key
// difference and summed in FP64; result valid in every thread.
__device__ Lse block_lse(Lse v) {
  __shared__ long long sm[32];
  __shared__ double ss[32];
  __shared__ long long s_max;
  __shared__ double s_sum;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
  long long mm = warp_max_key(v.m);
  __syncthreads();
  if (lane == 0) sm[w] = mm;
  __syncthreads();
  if (w == 0) {
    mm = warp_max_key(lane < nw ? sm[lane] : kKeyInvalid);
    if (lane == 0) s_max = mm;
  }
  __syncthreads();
  const long long M = s_max;
  double r = (v.m == kKeyInvalid || !(v.s > 0.0)) ? 0.0 : v.s * (double)expf(fx_to_f(v.m - M));
  r = warp_sum_d(r);
  if (lane == 0) ss[w] = r;
  __syncthreads();
  if (w == 0) {
    r = warp_sum_d(lane < nw ? ss[lane] : 0.0);
    if (lane == 0) s_sum = r;
  }
  __syncthreads();
  return Lse{M, s_sum};
}

// Global log-sum-exp over the unique children in one pass: each thread
// keeps a running (max, sum of shifted exponentials); blocks write
// partials; the last block combines them in a fixed tree, so the result does
// not depend on scheduling.  Also counts the unique children and sets the
// fixed-point threshold log(tau) + LSE.
__global__ void lse_kernel(const long long* __restrict__ keys, const FrameDev* __restrict__ fs,
                           int h_up, PruneWork w, double log_tau, int h_max) {
  pdl_enter();
  if (*(volatile const unsigned*)w.err & kErrFatal) return;   // children stale: frame redone or abandoned
  __shared__ bool last;
  const long long n = (long long)fs->H * h_up;
  // per thread: running maximum and a compensated FP32 sum of exp(key - max)
  // (FP32 exponentials of differences; FP64 only from the block partials on)
  long long m = kKeyInvalid;
  float sum = 0.f, comp = 0.f;
  unsigned valid = 0;
  for (long long j = (long long)blockIdx.x * blockDim.x + threadIdx.x; j < n;
       j += (long long)gridDim.x * blockDim.x) {
    const long long k = keys[j];
    if (k == kKeyInvalid) continue;
    ++valid;
    float term = 1.f;
    if (m == kKeyInvalid) {
      m = k;
    } else if (k > m) {
      const float sc = expf(fx_to_f(m - k));
      sum *= sc;
      comp *= sc;
      m = k;
    } else {
      term = expf(fx_to_f(k - m));
    }
    const float y = term - comp;   // Kahan summation
    const float t = sum + y;
    comp = (t - sum) - y;
    sum = t;
  }
  Lse v{m, (double)sum - (double)comp};
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) valid += __shfl_xor_sync(0xFFFFFFFFu, valid, o);
  if ((threadIdx.x & 31) == 0 && valid) atomicAdd(&w.counts[2], valid);
  v = block_lse(v);
  if (threadIdx.x == 0) {
    w.blk_max[blockIdx.x] = v.m;
    w.blk_sum[blockIdx.x] = v.s;
    __threadfence();
    last = atomicAdd(&w.blk_done[0], 1u) == gridDim.x - 1;
  }
  __syncthreads();
  if (!last) return;
  __threadfence();
  // block partials, each thread folding its share onto its own maximum
  Lse u{kKeyInvalid, 0.0};
  for (unsigned b = threadIdx.x; b < gridDim.x; b += blockDim.x) {
    const long long bm = ((volatile long long*)w.blk_max)[b];
    const double bs = ((volatile double*)w.blk_sum)[b];
    if (bm == kKeyInvalid || !(bs > 0.0)) continue;
    if (u.m == kKeyInvalid) {
      u = Lse{bm, bs};
    } else if (bm > u.m) {
      u = Lse{bm, bs + u.s * (double)expf(fx_to_f(u.m - bm))};
    } else {
      u.s += bs * (double)expf(fx_to_f(bm - u.m));
    }
  }
  u = block_lse(u);
  if (threadIdx.x == 0) {
    w.blk_done[0] = 0;
    if (u.m == kKeyInvalid || !(u.s > 0.0)) {
      w.lse[0] = -INFINITY;
      w.thr[0] = LLONG_MAX;
      w.sel[3] = 2;   // nothing to keep
    } else {
      const double lse = (double)u.m * kFxInv + log(u.s);
      w.lse[0] = lse;
      w.thr[0] = (long long)ceil((lse + log_tau) * 4294967296.0);
      w.sel[3] = 0;
    }
    w.sel[0] = 0;        // radix prefix
    w.sel[1] = h_max;    // still needed
    w.sel[2] = 0;        // boundary key
  }
}

void launch_lse(const long long* keys, const FrameDev* fs, int h_up, PruneWork w, double log_tau,
                int h_max, int nblk, cudaStream_t s) {
  launch_k(lse_kernel, nblk, kRedThreads, 0, s, keys, fs, h_up, w, log_tau, h_max);
}

// ---------------------------------------------------------------------------
// Top-H_max by 12-bit radix select on v = key - thr (>= 0 for candidates).
// sel[0] prefix of the selected digits, sel[1] elements still needed,
// sel[2] boundary key, sel[3] 0 running / 1 done-keep-all / 2 empty.
// ---------------------------------------------------------------------------
constexpr int kDigit = 12, kBins = 1 << kDigit;

__global__ void radix_hist_kernel(const long long* __restrict__ keys,
                                  const FrameDev* __restrict__ fs, int h_up, PruneWork w, int shift) {
  pdl_enter();
  if (*(volatile const unsigned*)w.err & kErrFatal) return;   // children stale: frame redone or abandoned
  __shared__ unsigned hist[kBins];
  const long long n = (long long)fs->H * h_up;
  if (w.sel[3] != 0) return;
  for (int b = threadIdx.x; b < kBins; b += blockDim.x) hist[b] = 0;
  __syncthreads();
  const long long thr = w.thr[0];
  const unsigned long long prefix = (unsigned long long)w.sel[0];
  for (long long j = (long long)blockIdx.x * blockDim.x + threadIdx.x; j < n;
       j += (long long)gridDim.x * blockDim.x) {
    const long long k = keys[j];
    if (k == kKeyInvalid || k < thr) continue;
    const unsigned long long v = (unsigned long long)(k - thr);
    if ((v >> (shift + kDigit)) != prefix) continue;
    atomicAdd(&hist[(v >> shift) & (kBins - 1)], 1u);
  }
  __syncthreads();
  for (int b = threadIdx.x; b < kBins; b += blockDim.x)
    if (hist[b]) atomicAdd(&w.hist[b], hist[b]);
}

__global__ void radix_find_kernel(PruneWork w, int shift, int first) {
  pdl_enter();
  if (*(volatile const unsigned*)w.err & kErrFatal) return;   // children stale: frame redone or abandoned
  // thread t owns bins [4t, 4t + 4) (blockDim.x == kBins / 4 == 1024);
  // the count of bins above a thread's range is total - inclusive prefix
  __shared__ unsigned wsum[32];
  const int t = threadIdx.x;
  const int lane = t & 31, wp = t >> 5;
  const bool running = w.sel[3] == 0;
  const long long need = w.sel[1];
  unsigned b4[4], mine = 0;
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    b4[k] = w.hist[4 * t + k];
    mine += b4[k];
    w.hist[4 * t + k] = 0;
  }
  unsigned x = mine;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const unsigned y = __shfl_up_sync(0xFFFFFFFFu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) wsum[wp] = x;
  __syncthreads();
  if (wp == 0) {
    unsigned s = wsum[lane];
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const unsigned y = __shfl_up_sync(0xFFFFFFFFu, s, o);
      if (lane >= o) s += y;
    }
    wsum[lane] = s;
  }
  __syncthreads();
  if (!running) return;
  const unsigned incl = x + (wp > 0 ? wsum[wp - 1] : 0u);
  const unsigned total = wsum[31];
  const unsigned above = total - incl;       // bins above this thread's range
  const unsigned upto = above + mine;
  if (first && (long long)total <= need) {
    if (t == 0) {
      w.sel[3] = 1;
      w.sel[2] = w.thr[0] - 1;   // every candidate is above the boundary
      w.sel[1] = 0;
    }
    return;
  }
  if ((long long)above < need && (long long)upto >= need) {
    unsigned cum = above;
    int b = 3;
    for (; b > 0; --b) {
      if ((long long)(cum + b4[b]) >= need) break;
      cum += b4[b];
    }
    w.sel[0] = (w.sel[0] << kDigit) | (4 * t + b);
    w.sel[1] = need - cum;
    if (shift == 0) w.sel[2] = w.thr[0] + w.sel[0];
  }
}

void launch_select(const long long* keys, const FrameDev* fs, int h_up, int nbits, PruneWork w,
                   int nblk, cudaStream_t s) {
  const int passes = (nbits + kDigit - 1) / kDigit;
  for (int p = 0; p < passes; ++p) {
    const int shift = (passes - 1 - p) * kDigit;
    launch_k(radix_hist_kernel, nblk, 256, 0, s, keys, fs, h_up, w, shift);
    launch_k(radix_find_kernel, 1, kBins / 4, 0, s, w, shift, p == 0);
  }
}

// ---------------------------------------------------------------------------
// Stable compaction of the retained children in (parent, draw) order:
// gt = key > boundary, eq = key == boundary (the first sel[1] of these in
// index order are kept).  One packed scan gives both prefix counts.
// ---------------------------------------------------------------------------
__device__ __forceinline__ unsigned long long keep_bits(long long k, long long thr, long long bnd,
                                                        long long need_eq, long long mode) {
  if (mode == 2 || k == kKeyInvalid || k < thr) return 0ULL;
  if (k > bnd) return 1ULL;
  if (k == bnd && need_eq > 0) return 1ULL << 32;
  return 0ULL;
}

__global__ void keep_flags_kernel(const long long* __restrict__ keys,
                                  const FrameDev* __restrict__ fs, int h_up, PruneWork w) {
  pdl_enter();
  if (*(volatile const unsigned*)w.err & kErrFatal) return;   // children stale: frame redone or abandoned
  const long long n = (long long)fs->H * h_up;
  const long long thr = w.thr[0], bnd = w.sel[2], need = w.sel[1], mode = w.sel[3];
  for (long long j = (long long)blockIdx.x * blockDim.x + threadIdx.x; j < n;
       j += (long long)gridDim.x * blockDim.x)
    w.flags[j] = keep_bits(keys[j], thr, bnd, need, mode);
}

__global__ void keep_write_kernel(const long long* __restrict__ keys,
                                  const FrameDev* __restrict__ fs, int h_up, PruneWork w, int h_max) {
  pdl_enter();
  if (*(volatile const unsigned*)w.err & kErrFatal) return;   // children stale: frame redone or abandoned
  const long long n = (long long)fs->H * h_up;
  const long long thr = w.thr[0], bnd = w.sel[2], need = w.sel[1], mode = w.sel[3];
  for (long long j = (long long)blockIdx.x * blockDim.x + threadIdx.x; j < n;
       j += (long long)gridDim.x * blockDim.x) {
    const unsigned long long f = keep_bits(keys[j], thr, bnd, need, mode);
    if (!f) continue;
    const unsigned long long pre = w.flags[j];
    const long long gt = (long long)(pre & 0xFFFFFFFFULL), eq = (long long)(pre >> 32);
    if ((f >> 32) && eq >= need) continue;
    const long long pos = gt + min(eq, need);
    if (pos < h_max) w.surv_idx[pos] = j;
  }
}

void launch_compact(const long long* keys, const FrameDev* fs, int h_up, long long cap, PruneWork w,
                    int h_max, int nblk, cudaStream_t s) {
  launch_k(keep_flags_kernel, nblk, 256, 0, s, keys, fs, h_up, w);
  scan_u64(w.flags, w.flags, &fs->H, h_up, cap, (unsigned long long*)(w.counts + 4), false,
           w.flags_tmp, w.flags_tmp_cap, w.err, s);
  launch_k(keep_write_kernel, nblk, 256, 0, s, keys, fs, h_up, w, h_max);
}

// ---------------------------------------------------------------------------
// Survivors: renormalised FP64 log-weights, child uids, CSR offsets.
// counts[0] survivors, counts[1] entries, counts[4..5] packed scan total.
// ---------------------------------------------------------------------------
__global__ void finalize_kernel(PruneWork w, const long long* __restrict__ keys,
                                const uint16_t* __restrict__ child_alive, HypTable parents,
                                int h_up, HypTable out, int h_max, unsigned* err,
                                long long cap_entries) {
  pdl_enter();
  if (*(volatile const unsigned*)err & kErrFatal) return;
  __shared__ long long s_n;
  __shared__ double s_lse;
  __shared__ uint32_t carry;
  const int tid = threadIdx.x, nthr = blockDim.x;
  if (tid == 0) {
    const unsigned long long tot = *(const unsigned long long*)(w.counts + 4);
    long long n = 0;
    if (w.sel[3] != 2) n = (long long)(tot & 0xFFFFFFFFULL) + min((long long)(tot >> 32), (long long)w.sel[1]);
    if (n > h_max) n = h_max;
    s_n = n;
    w.counts[0] = (unsigned)n;
    carry = 0;
  }
  __syncthreads();
  const long long n = s_n;
  const double lse_all = w.lse[0];
  // log-sum-exp of the retained keys: integer maximum, FP32 exponentials of
  // the key differences, FP64 sums
  Lse v{kKeyInvalid, 0.0};
  for (long long s = tid; s < n; s += nthr) {
    const long long k = keys[w.surv_idx[s]];
    if (v.m == kKeyInvalid) v = Lse{k, 1.0};
    else if (k > v.m) v = Lse{k, 1.0 + v.s * (double)expf(fx_to_f(v.m - k))};
    else v.s += (double)expf(fx_to_f(k - v.m));
  }
  v = block_lse(v);
  if (tid == 0) {
    s_lse = (double)v.m * kFxInv - lse_all + log(v.s);
    w.lse[1] = s_lse;
  }
  __syncthreads();
  for (long long base = 0; base < n; base += nthr) {
    const long long s = base + tid;
    uint32_t na = 0;
    if (s < n) {
      const long long j = w.surv_idx[s];
      out.logw[s] = (double)keys[j] * kFxInv - lse_all - s_lse;
      const long long hpar = j / h_up, nd = j % h_up;
      out.uid[s] = mix64(parents.uid[hpar] + 0x9E3779B97F4A7C15ULL * (unsigned long long)(nd + 1));
      na = child_alive[j];
      atomicMax(&w.counts[3], na);
    }
    // block exclusive scan of na
    uint32_t x = na;
    const int lane = tid & 31, wp = tid >> 5;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t y = __shfl_up_sync(0xFFFFFFFFu, x, o);
      if (lane >= o) x += y;
    }
    __shared__ uint32_t ws[32];
    if (lane == 31) ws[wp] = x;
    __syncthreads();
    if (tid < 32) {
      uint32_t v = tid < (nthr + 31) / 32 ? ws[tid] : 0u;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xFFFFFFFFu, v, o);
        if (tid >= o) v += y;
      }
      ws[tid] = v;
    }
    __syncthreads();
    const uint32_t excl = carry + (wp > 0 ? ws[wp - 1] : 0u) + x - na;
    if (s < n) out.ptr[s] = excl;
    __syncthreads();
    if (tid == 0) carry += ws[(nthr + 31) / 32 - 1];
    __syncthreads();
  }
  if (tid == 0) {
    out.ptr[n] = carry;
    w.counts[1] = carry;
    if ((long long)carry > cap_entries) atomicOr(err, kErrEntries);
  }
}

void launch_finalize(PruneWork w, const long long* keys, const uint16_t* child_alive,
                     const HypTable& parents, int h_up, HypTable out, int h_max, unsigned* err,
                     long long cap_entries, cudaStream_t s) {
  launch_k(finalize_kernel, 1, 1024, 0, s, w, keys, child_alive, parents, h_up, out, h_max, err,
                                     cap_entries);
}

// ---------------------------------------------------------------------------
// Garbage collection of components and the batched track update (Kalman
// with the mean detection and R/m, Joseph form), in one launch with the
// remapping of the new hypothesis table's component indices.
// ---------------------------------------------------------------------------

template <int DZ>
__device__ void copy_comp(const Model& md, const CompTable& src, int c, const CompTable& dst, int d) {
  constexpr int DX = 2 * DZ;
  const size_t cs = src.cap, cd = dst.cap;
#pragma unroll
  for (int a = 0; a < DX; ++a) {
    dst.mhi[a * cd + d] = src.mhi[a * cs + c];
    dst.mlo[a * cd + d] = src.mlo[a * cs + c];
  }
#pragma unroll
  for (int k = 0; k < DX * (DX + 1) / 2; ++k) dst.cov[k * cd + d] = src.cov[k * cs + c];
  dst.lk[d] = src.lk[c];
  dst.lb[d] = src.lb[c];
  dst.logp[d] = src.logp[c];
  dst.log1mp[d] = src.log1mp[c];
}

// Gain, mean and Joseph-form covariance of one track update in arithmetic F,
// from P, S^-1 = Si, R/m and the mean innovation; writes component d.
template <typename F, int DZ>
__device__ __forceinline__ void kalman_tail(const F (&P)[2 * DZ][2 * DZ], const F (&Si)[DZ][DZ],
                                            const F (&Rm)[DZ][DZ], const F (&ebar)[DZ], const CompTable& src,
                                            int c, const CompTable& dst, int d) {
  constexpr int DX = 2 * DZ;
  const size_t cs = src.cap, cd = dst.cap;
  F K[DX][DZ];
#pragma unroll
  for (int i = 0; i < DX; ++i)
#pragma unroll
    for (int b = 0; b < DZ; ++b) {
      F t = 0;
#pragma unroll
      for (int a = 0; a < DZ; ++a) t += P[i][a] * Si[a][b];
      K[i][b] = t;
    }
#pragma unroll
  for (int i = 0; i < DX; ++i) {
    F delta = 0;
#pragma unroll
    for (int b = 0; b < DZ; ++b) delta += K[i][b] * ebar[b];
    float hi = src.mhi[i * cs + c], lo = src.mlo[i * cs + c];
    if (sizeof(F) == sizeof(float)) {
      df_add(hi, lo, (float)delta);
    } else {
      const double v = ((double)hi + (double)lo) + (double)delta;
      hi = (float)v;
      lo = (float)(v - (double)hi);
    }
    dst.mhi[i * cd + d] = hi;
    dst.mlo[i * cd + d] = lo;
  }
  // Joseph form: (I - K H) P (I - K H)^T + K (R/m) K^T
  F AP[DX][DX];
#pragma unroll
  for (int i = 0; i < DX; ++i)
#pragma unroll
    for (int j = 0; j < DX; ++j) {
      F t = P[i][j];
#pragma unroll
      for (int a = 0; a < DZ; ++a) t -= K[i][a] * P[a][j];
      AP[i][j] = t;
    }
  F KR[DX][DZ];
#pragma unroll
  for (int i = 0; i < DX; ++i)
#pragma unroll
    for (int b = 0; b < DZ; ++b) {
      F t = 0;
#pragma unroll
      for (int a = 0; a < DZ; ++a) t += K[i][a] * Rm[a][b];
      KR[i][b] = t;
    }
#pragma unroll
  for (int i = 0; i < DX; ++i)
#pragma unroll
    for (int j = i; j < DX; ++j) {
      F t = AP[i][j], t2 = AP[j][i];
#pragma unroll
      for (int a = 0; a < DZ; ++a) {
        t -= AP[i][a] * K[j][a];
        t2 -= AP[j][a] * K[i][a];
      }
      F r = 0;
#pragma unroll
      for (int b = 0; b < DZ; ++b) r += KR[i][b] * K[j][b];
      dst.cov[(size_t)pidx(DX, i, j) * cd + d] = (float)(F(0.5) * (t + t2) + r);
    }
}

// The FP64 update of an ill-conditioned innovation covariance (rare; kept
// out of line so that its registers do not limit the kernel's occupancy).
template <int DZ>
__device__ __noinline__ bool kalman_fp64(const Model& md, const float (&P)[2 * DZ][2 * DZ], const long long (&se)[DZ],
                                         int m, const CompTable& src, int c, const CompTable& dst, int d) {
  constexpr int DX = 2 * DZ;
  double Pd[DX][DX], Sd[DZ][DZ], Ld[DZ][DZ], ldd, Li[DZ][DZ], Si[DZ][DZ], Rd[DZ][DZ], ed[DZ];
#pragma unroll
  for (int i = 0; i < DX; ++i)
#pragma unroll
    for (int j = 0; j < DX; ++j) Pd[i][j] = P[i][j];
#pragma unroll
  for (int a = 0; a < DZ; ++a) {
    ed[a] = (double)se[a] * kFxInv / (double)m;
#pragma unroll
    for (int b = 0; b < DZ; ++b) {
      Rd[a][b] = (double)md.R[a * DZ + b] / (double)m;
      Sd[a][b] = Pd[a][b] + Rd[a][b];
    }
  }
  if (!chol_n<double, DZ>(Sd, Ld, ldd, 2.220446049250313e-16)) return false;
#pragma unroll
  for (int j = 0; j < DZ; ++j)
#pragma unroll
    for (int i = 0; i < DZ; ++i) {
      double t = (i == j) ? 1.0 : 0.0;
#pragma unroll
      for (int k = 0; k < i; ++k) t -= Ld[i][k] * Li[k][j];
      Li[i][j] = (i < j) ? 0.0 : t / Ld[i][i];
    }
#pragma unroll
  for (int i = 0; i < DZ; ++i)
#pragma unroll
    for (int j = 0; j < DZ; ++j) {
      double t = 0.0;
#pragma unroll
      for (int k = 0; k < DZ; ++k) t += Li[k][i] * Li[k][j];
      Si[i][j] = t;
    }
  kalman_tail<double, DZ>(Pd, Si, Rd, ed, src, c, dst, d);
  return true;
}

// Kalman update of component c with m detections whose innovations sum to
// se (fixed point), into component d.  An innovation covariance whose FP32
// Cholesky factor fails the pivot test (a pivot at or below 16 eps32
// trace S) is factorised in FP64, and the gain, the mean and the Joseph
// form are then computed in FP64 too: with S that ill-conditioned the gain
// P H^T S^-1 cancels in FP32 (the posterior covariance is the difference of
// nearly equal O(|P|) terms).
template <int DZ>
__device__ bool kalman_comp(const Model& md, const CompTable& src, int c, int m,
                            const long long (&se)[DZ], const CompTable& dst, int d) {
  constexpr int DX = 2 * DZ;
  const size_t cs = src.cap;
  float P[DX][DX];
#pragma unroll
  for (int i = 0; i < DX; ++i)
#pragma unroll
    for (int j = i; j < DX; ++j) {
      const float v = src.cov[(size_t)pidx(DX, i, j) * cs + c];
      P[i][j] = v;
      P[j][i] = v;
    }
  const float inv_m = 1.f / (float)m;
  float ebar[DZ], S[DZ][DZ], Rm[DZ][DZ];
#pragma unroll
  for (int a = 0; a < DZ; ++a) {
    ebar[a] = (float)((double)se[a] * kFxInv) * inv_m;
#pragma unroll
    for (int b = 0; b < DZ; ++b) {
      Rm[a][b] = md.R[a * DZ + b] * inv_m;
      S[a][b] = P[a][b] + Rm[a][b];
    }
  }
  float L[DZ][DZ], ld;
  if (chol_n<float, DZ>(S, L, ld, 1.1920929e-7f)) {
    // S^-1 from the FP32 Cholesky factor
    float Li[DZ][DZ], Si[DZ][DZ];
#pragma unroll
    for (int j = 0; j < DZ; ++j)
#pragma unroll
      for (int i = 0; i < DZ; ++i) {
        float t = (i == j) ? 1.f : 0.f;
#pragma unroll
        for (int k = 0; k < i; ++k) t -= L[i][k] * Li[k][j];
        Li[i][j] = (i < j) ? 0.f : t / L[i][i];
      }
#pragma unroll
    for (int i = 0; i < DZ; ++i)
#pragma unroll
      for (int j = 0; j < DZ; ++j) {
        float t = 0.f;
#pragma unroll
        for (int k = 0; k < DZ; ++k) t += Li[k][i] * Li[k][j];
        Si[i][j] = t;
      }
    kalman_tail<float, DZ>(P, Si, Rm, ebar, src, c, dst, d);
  } else if (!kalman_fp64<DZ>(md, P, se, m, src, c, dst, d)) {
    return false;
  }
  dst.lk[d] = src.lk[c];
  dst.lb[d] = src.lb[c];
  dst.logp[d] = src.logp[c];
  dst.log1mp[d] = src.log1mp[c];
  return true;
}

template <int DZ>
__global__ void __launch_bounds__(256, DZ == 2 ? 3 : 2) gc_remap_kernel(Model md, CompTable src, CompTable dst, const uint32_t* __restrict__ newpos,
                                const uint32_t* __restrict__ flag, const FrameDev* __restrict__ fs,
                                const unsigned* __restrict__ n_keep_dev, const uint32_t* __restrict__ upd_src,
                                const uint32_t* __restrict__ upd_m, const long long* __restrict__ upd_se,
                                int cap_upd, const unsigned* __restrict__ n_upd_dev,
                                const unsigned* __restrict__ n_surv_dev, unsigned* err, uint32_t* out_comp,
                                const unsigned* __restrict__ n_entries, long long cap_entries,
                                const uint32_t* __restrict__ hvals, uint32_t hmask, unsigned* n_upd_prev) {
  pdl_enter();
  // the updates this frame inserted into the hash table, for the next
  // frame's reset (whatever happens below)
  if (blockIdx.x == 0 && threadIdx.x == 0) *n_upd_prev = *n_upd_dev;
  if (*n_surv_dev == 0u || (*(volatile unsigned*)err & kErrFatal)) return;
  const int n_src = fs->T;
  const unsigned n_keep = *n_keep_dev;
  const unsigned n_upd = min(*n_upd_dev, (unsigned)cap_upd);
  if ((long long)n_keep + n_upd > dst.cap) {
    if (blockIdx.x == 0 && threadIdx.x == 0) atomicOr(err, kErrComps);
    return;
  }
  // (the particle model's component work is particle_remap_kernel's)
  const long long total = md.particle ? 0 : (long long)n_src + n_upd;
  for (long long x = (long long)blockIdx.x * blockDim.x + threadIdx.x; x < total;
       x += (long long)gridDim.x * blockDim.x) {
    if (x < n_src) {
      const int c = (int)x;
      if (flag[c]) {
        if (newpos[c] >= n_keep) atomicOr(err, kErrChkComp);
        else copy_comp<DZ>(md, src, c, dst, (int)newpos[c]);
      }
    } else {
      const int u = (int)(x - n_src);
      if (upd_src[u] >= (uint32_t)n_src) {
        atomicOr(err, kErrChkComp);
        continue;
      }
      long long se[DZ];
#pragma unroll
      for (int a = 0; a < DZ; ++a) se[a] = upd_se[(size_t)a * cap_upd + u];
      if (!kalman_comp<DZ>(md, src, (int)upd_src[u], (int)upd_m[u], se, dst, (int)n_keep + u))
        atomicOr(err, kErrNumeric);
    }
  }
  // the new hypothesis table's component indices: an old component to its
  // compacted position, a new one (tagged hash slot) to its update's
  // position after the kept components (independent of the copies above)
  const long long n_e = min((long long)*n_entries, cap_entries);
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < n_e;
       e += (long long)gridDim.x * blockDim.x) {
    const uint32_t v = out_comp[e];
    if ((v & kNewTag) ? (v & ~kNewTag) > hmask : v >= (uint32_t)n_src) {
      atomicOr(err, kErrChkRemap);
      continue;
    }
    out_comp[e] = (v & kNewTag) ? n_keep + hvals[v & ~kNewTag] : newpos[v];
  }
}

void launch_gc_remap(const Model& md, const CompTable& src, const CompTable& dst, const uint32_t* newpos,
                     const uint32_t* flag, const FrameDev* fs, const unsigned* n_keep_dev, const uint32_t* upd_src,
                     const uint32_t* upd_m, const long long* upd_se, int cap_upd, const unsigned* n_upd_dev,
                     const unsigned* n_surv_dev, unsigned* err, uint32_t* out_comp, const unsigned* n_entries_dev,
                     long long cap_entries, const uint32_t* hvals, uint32_t hmask, unsigned* n_upd_prev, int grid,
                     cudaStream_t s) {
  if (md.dz == 2) {
    launch_k(gc_remap_kernel<2>, grid, 256, 0, s, md, src, dst, newpos, flag, fs, n_keep_dev, upd_src, upd_m,
             upd_se, cap_upd, n_upd_dev, n_surv_dev, err, out_comp, n_entries_dev, cap_entries, hvals, hmask,
             n_upd_prev);
  } else {
    launch_k(gc_remap_kernel<3>, grid, 256, 0, s, md, src, dst, newpos, flag, fs, n_keep_dev, upd_src, upd_m,
             upd_se, cap_upd, n_upd_dev, n_surv_dev, err, out_comp, n_entries_dev, cap_entries, hvals, hmask,
             n_upd_prev);
  }
}

// ---------------------------------------------------------------------------
// Estimates: cardinality distribution, MAP cardinality, heaviest hypothesis
// of that cardinality (ties to the lower index), label existence, and the
// clutter probability of each detection.
// ---------------------------------------------------------------------------
// Hypothesis weights enter the estimate sums as unsigned fixed point with 40
// fractional bits (FP32 exponential of the normalised log-weight), so the
// atomic sums are exact and independent of their order.
constexpr double kWfxInv = 9.094947017729282e-13;   // 2^-40
__device__ __forceinline__ unsigned long long w_fx(double logw) {
  return __float2ull_rn(expf((float)logw) * 1099511627776.0f);
}

// Cardinality distribution, MAP cardinality (ties to the smaller n) and the
// heaviest hypothesis of that cardinality (ties to the lower index), by one
// block: nb[0] = n_hat, nb[1] = MAP hypothesis.
__device__ __forceinline__ void est_card_block(const HypTable& hp, const int H, double* pmf, int pcap, int* nb) {
  extern __shared__ unsigned long long s_pmf[];   // [pcap]
  __shared__ unsigned long long bw[32];
  __shared__ int bi[32];
  __shared__ double lw_w[32];
  __shared__ int li_w[32];
  __shared__ int s_nhat;
  const int tid = threadIdx.x, nthr = blockDim.x, lane = tid & 31, wp = tid >> 5;
  const int nw = (nthr + 31) >> 5;
  for (int n = tid; n < pcap; n += nthr) s_pmf[n] = 0ull;
  __syncthreads();
  // one shared-memory atomic per distinct cardinality in a warp (most
  // hypotheses share a few cardinalities)
  for (int base = 0; base < H; base += nthr) {
    const int h = base + tid;
    int n = -1;
    unsigned long long w = 0ull;
    if (h < H) {
      n = (int)(hp.ptr[h + 1] - hp.ptr[h]);
      if (n < pcap) w = w_fx(hp.logw[h]);
      else n = -1;
    }
    const unsigned grp = __match_any_sync(0xFFFFFFFFu, n);
    // w < 2^41: the two 21-bit halves of 32 weights sum without overflow
    const unsigned lo = __reduce_add_sync(grp, (unsigned)(w & 0x1FFFFFull));
    const unsigned hi = __reduce_add_sync(grp, (unsigned)(w >> 21));
    if (n >= 0 && lane == __ffs(grp) - 1)
      atomicAdd(&s_pmf[n], ((unsigned long long)hi << 21) + lo);
  }
  __syncthreads();
  // argmax over bins (exact integer sums)
  unsigned long long v = 0ull;
  int vi = 0x7FFFFFFF;
  for (int n = tid; n < pcap; n += nthr) {
    const unsigned long long p = s_pmf[n];
    pmf[n] = (double)p * kWfxInv;
    if (vi == 0x7FFFFFFF || p > v) { v = p; vi = n; }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const unsigned long long v2 = __shfl_xor_sync(0xFFFFFFFFu, v, o);
    const int i2 = __shfl_xor_sync(0xFFFFFFFFu, vi, o);
    if (i2 != 0x7FFFFFFF && (vi == 0x7FFFFFFF || v2 > v || (v2 == v && i2 < vi))) { v = v2; vi = i2; }
  }
  if (lane == 0) { bw[wp] = v; bi[wp] = vi; }
  __syncthreads();
  if (tid == 0) {
    unsigned long long b = 0ull;
    int k = 0x7FFFFFFF;
    for (int w = 0; w < nw; ++w)
      if (bi[w] != 0x7FFFFFFF && (k == 0x7FFFFFFF || bw[w] > b || (bw[w] == b && bi[w] < k))) { b = bw[w]; k = bi[w]; }
    s_nhat = k == 0x7FFFFFFF ? 0 : k;
  }
  __syncthreads();
  const int nhat = s_nhat;
  double lw = -INFINITY;
  int li = -1;
  for (int h = tid; h < H; h += nthr) {
    if ((int)(hp.ptr[h + 1] - hp.ptr[h]) != nhat) continue;
    const double x = hp.logw[h];
    if (li < 0 || x > lw) { lw = x; li = h; }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const double w2 = __shfl_xor_sync(0xFFFFFFFFu, lw, o);
    const int i2 = __shfl_xor_sync(0xFFFFFFFFu, li, o);
    if (i2 >= 0 && (li < 0 || w2 > lw || (w2 == lw && i2 < li))) { lw = w2; li = i2; }
  }
  if (lane == 0) { lw_w[wp] = lw; li_w[wp] = li; }
  __syncthreads();
  if (tid == 0) {
    double b = -INFINITY;
    int k = -1;
    for (int w = 0; w < nw; ++w)
      if (li_w[w] >= 0 && (k < 0 || lw_w[w] > b || (lw_w[w] == b && li_w[w] < k))) { b = lw_w[w]; k = li_w[w]; }
    nb[0] = nhat;
    nb[1] = k;
  }
}

// Existence of the MAP tracks, first half, beside the cardinality block:
// every hypothesis adds its weight onto each of its components,
// r_comp[c] += w_h (one warp per hypothesis), and cmax records one past the
// largest component index met.  A label occurs at most once in a
// hypothesis, so the sum over the components of one label is the total
// weight of the hypotheses that hold it (the existence of Section 3's
// labelled tracks), reached without waiting for the MAP hypothesis.
constexpr int kEstPriv = 4096;   // components summed in shared memory per block

__global__ void est_sums_kernel(HypTable hp, int H_host, const unsigned* H_dev, double* pmf, int pcap, int* nb,
                                unsigned long long* r_comp, int ccap, unsigned* cmax, const unsigned* err) {
  pdl_enter();
  // a frame that failed left the new table incomplete: nothing to read
  if (err && (*(volatile const unsigned*)err & kErrFatal)) return;
  const int H = H_dev ? (int)*H_dev : H_host;
  if (blockIdx.x == 0) {
    est_card_block(hp, H, pmf, pcap, nb);
    return;
  }
  // hypotheses share most of their components, so the block sums the
  // first kEstPriv components in shared memory and adds each nonzero sum
  // to global memory once (fixed point: the sums do not depend on order)
  __shared__ unsigned long long s_acc[kEstPriv];
  __shared__ unsigned s_top;
  for (int c = threadIdx.x; c < kEstPriv; c += blockDim.x) s_acc[c] = 0ull;
  if (threadIdx.x == 0) s_top = 0u;
  __syncthreads();
  const int lane = threadIdx.x & 31;
  const int wpb = blockDim.x >> 5;
  unsigned top = 0u;
  for (int h = (blockIdx.x - 1) * wpb + (threadIdx.x >> 5); h < H; h += (gridDim.x - 1) * wpb) {
    const uint32_t lo = hp.ptr[h], hi = hp.ptr[h + 1];
    const unsigned long long wgt = w_fx(hp.logw[h]);
    for (uint32_t e = lo + lane; e < hi; e += 32) {
      const uint32_t c = min(hp.comp[e], (uint32_t)ccap - 1u);
      if (wgt) {
        if (c < (uint32_t)kEstPriv) atomicAdd(&s_acc[c], wgt);
        else atomicAdd(&r_comp[c], wgt);
      }
      top = max(top, c + 1u);
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) top = max(top, __shfl_xor_sync(0xFFFFFFFFu, top, o));
  if (lane == 0 && top) atomicMax(&s_top, top);
  __syncthreads();
  const unsigned nt = min(s_top, (unsigned)kEstPriv);
  for (unsigned c = threadIdx.x; c < nt; c += blockDim.x)
    if (s_acc[c]) atomicAdd(&r_comp[c], s_acc[c]);
  if (threadIdx.x == 0 && s_top) atomicMax(cmax, s_top);
}

// Existence of the MAP tracks, second half: the labels of the MAP
// hypothesis (in label order) go to each block's shared memory; every
// component with a nonzero sum adds it to its label's entry (binary search)
// and its sum is cleared, so r_comp is left zeroed.  One block writes the
// MAP tracks (glmb_track records: mean hi + lo in FP64, full covariance)
// from its own sums; with several blocks (large tables) each adds its sums
// into r_map once and the last block to finish writes the tracks.  cmax,
// done and r_map are left zeroed.
__global__ void est_tracks_kernel(HypTable hp, CompTable ct, int dx, const int* __restrict__ nb,
                                  unsigned long long* r_comp, unsigned* cmax, unsigned* done,
                                  unsigned long long* r_map, glmb_track* out, int cap, const unsigned* err) {
  pdl_enter();
  if (err && (*(volatile const unsigned*)err & kErrFatal)) return;
  extern __shared__ unsigned long long s_key[];   // [cap] MAP labels, then [cap] sums
  unsigned long long* s_r = s_key + cap;
  __shared__ bool last;
  const int best = nb[1];
  const uint32_t b0 = best >= 0 ? hp.ptr[best] : 0u;
  const int nmap = best >= 0 ? min((int)(hp.ptr[best + 1] - b0), cap) : 0;
  const uint32_t ccap = (uint32_t)ct.cap;
  const uint32_t nc = min(*(volatile unsigned*)cmax, ccap);
  for (int j = threadIdx.x; j < nmap; j += blockDim.x) {
    const uint32_t cm = min(hp.comp[b0 + j], ccap - 1u);
    s_key[j] = ((unsigned long long)ct.lk[cm] << 32) | ct.lb[cm];
    s_r[j] = 0ull;
  }
  __syncthreads();
  for (uint32_t c = blockIdx.x * blockDim.x + threadIdx.x; c < nc; c += gridDim.x * blockDim.x) {
    const unsigned long long v = r_comp[c];
    if (!v) continue;
    r_comp[c] = 0ull;
    const unsigned long long key = ((unsigned long long)ct.lk[c] << 32) | ct.lb[c];
    int l = 0, u = nmap;
    while (l < u) {
      const int mid = (l + u) >> 1;
      if (s_key[mid] < key) l = mid + 1; else u = mid;
    }
    if (l < nmap && s_key[l] == key) atomicAdd(&s_r[l], v);
  }
  __syncthreads();
  const bool multi = gridDim.x > 1;
  if (multi) {
    for (int j = threadIdx.x; j < nmap; j += blockDim.x)
      if (s_r[j]) atomicAdd(&r_map[j], s_r[j]);
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) last = atomicAdd(done, 1u) == gridDim.x - 1;
    __syncthreads();
    if (!last) return;
    __threadfence();
  }
  if (threadIdx.x == 0) {
    // every block has read cmax by now (the last block, or the only one)
    *cmax = 0u;
    if (multi) *done = 0u;
  }
  const size_t cc = ct.cap;
  for (int j = threadIdx.x; j < nmap; j += blockDim.x) {
    unsigned long long rs = s_r[j];
    if (multi) {
      rs = ((volatile unsigned long long*)r_map)[j];
      r_map[j] = 0ull;
    }
    const uint32_t c = min(hp.comp[b0 + j], ccap - 1u);
    glmb_track& t = out[j];
    t.label_k = ct.lk[c];
    t.label_b = ct.lb[c];
    t.r = (double)rs * kWfxInv;
    for (int a = 0; a < 6; ++a)
      t.mean[a] = a < dx ? (double)ct.mhi[a * cc + c] + (double)ct.mlo[a * cc + c] : 0.0;
    for (int k = 0; k < 36; ++k) t.cov[k] = 0.0;
    for (int i = 0; i < dx; ++i)
      for (int k = i; k < dx; ++k) {
        const double v = ct.cov[(size_t)pidx(dx, i, k) * cc + c];
        t.cov[i * dx + k] = v;
        t.cov[k * dx + i] = v;
      }
  }
}

void launch_estimates(const HypTable& hp, int H, const unsigned* H_dev, int H_bound, const CompTable& ct, int dx,
                      double* pmf, int pcap, int* nb, unsigned long long* r_comp, unsigned long long* r_map,
                      void* tracks, unsigned* cmax, unsigned* done, int n_sm, const unsigned* err, cudaStream_t s) {
  static int attr_pcap = 0;   // the limits only grow (graphs of larger filters stay valid)
  // (est_sums_kernel also holds kEstPriv sums in static shared memory, so
  // the opt-in is made whatever the dynamic size)
  if (pcap > attr_pcap) {
    cudaFuncSetAttribute(est_sums_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, pcap * 8);
    cudaFuncSetAttribute(est_tracks_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, pcap * 16);
    attr_pcap = pcap;
  }
  // block 0: the cardinality; blocks 1..: one warp per hypothesis
  const int sum_blocks = H_dev ? n_sm : std::max(1, std::min((H + 31) / 32, n_sm));
  launch_k(est_sums_kernel, 1 + sum_blocks, 1024, (size_t)pcap * 8, s, hp, H, H_dev, pmf, pcap, nb, r_comp,
           ct.cap, cmax, err);
  // the components in use grow with the hypotheses: one block while the
  // table holds at most 4096 hypotheses, else two blocks per SM
  const int track_blocks = H_bound <= 4096 ? 1 : 2 * n_sm;
  launch_k(est_tracks_kernel, track_blocks, 1024, (size_t)pcap * 16, s, hp, ct, dx, nb, r_comp, cmax, done, r_map,
           (glmb_track*)tracks, pcap, err);
}

__global__ void meas_assoc_kernel(HypTable hp, int H, int M, double* r_u) {
  pdl_enter();
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= M) return;
  unsigned long long s = 0ull;
  for (int h = 0; h < H; ++h)
    if (hp.theta[(size_t)h * M + i] == 0) s += w_fx(hp.logw[h]);
  r_u[i] = (double)s * kWfxInv;
}

void launch_meas_assoc(const HypTable& hp, int H, int M, double* r_u, cudaStream_t s) {
  if (M <= 0) return;
  launch_k(meas_assoc_kernel, (M + 127) / 128, 128, 0, s, hp, H, M, r_u);
}

}  // namespace glmb

// Normalisation, truncation to the top H_max and renormalisation of the
// children (arXiv 2512.06230, Section 3, pruning) in one launch: a cluster
// of CTAs on neighbouring SMs that combine their partial results through
// distributed shared memory, instead of a chain of grid-wide kernels.
//
//   1  log-sum-exp over the unique children (per-thread integer maximum and
//      compensated FP32 sums of FP32 exponentials, partials rescaled and
//      summed in FP64), the unique count, the fixed-point threshold
//      log(tau) + LSE;
//   2  top-H_max among the children at or above the threshold by 12-bit
//      radix select on key - threshold: every CTA histograms its slice,
//      each CTA sums one slice of bins over the cluster, every CTA gathers
//      the summed histogram and finds the boundary digit (all CTAs compute
//      the same result, so no broadcast is needed);
//   3  stable compaction in child order (parent, draw): per-CTA counts of
//      children above and at the boundary, an exclusive scan over the
//      cluster, then each thread writes its contiguous share;
//   4  the retained set (CTA 0): renormalised FP64 log-weights, child uids,
//      CSR offsets of the new hypothesis table.
// Results equal the multi-kernel chain's except for the summation order of
// the LSE (a different tree), which moves it by rounding only.
#include <cooperative_groups.h>

#include "../../include/glmb.h"
#include "glmb_kernels.h"

namespace cg = cooperative_groups;

namespace glmb {

namespace {

constexpr int kSelDigit = 12, kSelBins = 1 << kSelDigit;
constexpr int kSelThreads = 1024;

__device__ __forceinline__ long long warp_max_k(long long v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = max(v, __shfl_xor_sync(0xFFFFFFFFu, v, o));
  return v;
}
__device__ __forceinline__ double warp_sum_dd(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xFFFFFFFFu, v, o);
  return v;
}

struct SelShared {
  unsigned hist[kSelBins];        // this CTA's histogram of the current digit
  unsigned hsum[2][kSelBins];     // the cluster's histogram (this CTA sums one slice; rounds alternate)
  unsigned long long part[32];    // per-warp partials
  double dpart[32];
  long long pm;                   // CTA partial: maximum key
  double ps;                      //             sum of exp(key - pm)
  unsigned pc;                    //             unique children
  unsigned long long cnt;         // CTA count of (above | at << 32) the boundary
  // cluster-wide results (identical in every CTA)
  long long thr, prefix, need, bnd;
  int mode;                       // 0 selecting, 1 keep every candidate, 2 nothing
  double lse;
  unsigned long long before;      // children (above | at << 32) in lower-rank CTAs
  unsigned long long total;
};

__device__ __forceinline__ unsigned long long keep_flag(long long k, long long thr, long long bnd, long long need,
                                                        int mode) {
  if (mode == 2 || k == kKeyInvalid || k < thr) return 0ull;
  if (k > bnd) return 1ull;
  if (k == bnd && need > 0) return 1ull << 32;
  return 0ull;
}

}  // namespace

__global__ void __launch_bounds__(kSelThreads, 1)
select_cluster_kernel(const long long* __restrict__ keys, const FrameDev* __restrict__ fs, int h_up, PruneWork w,
                      double log_tau, int h_max, int nbits, const uint16_t* __restrict__ child_alive,
                      HypTable parents, HypTable out, unsigned* err, long long cap_entries) {
  pdl_enter();
  // a frame whose expansion was skipped (the staging flagged it, or the
  // table failed) holds stale children: nothing to select; every CTA of the
  // cluster reads the same flag and returns before any cluster barrier
  if (*(volatile const unsigned*)err & kErrFatal) return;
  extern __shared__ __align__(16) unsigned char sel_sm[];
  SelShared& S = *reinterpret_cast<SelShared*>(sel_sm);
  cg::cluster_group cl = cg::this_cluster();
  const int C = (int)cl.num_blocks(), rank = (int)cl.block_rank();
  const int tid = threadIdx.x, nthr = blockDim.x, lane = tid & 31, wp = tid >> 5, nw = nthr >> 5;
  const long long n = (long long)fs->H * h_up;
  const long long per = (n + C - 1) / C;
  const long long lo = min(n, (long long)rank * per), hi = min(n, lo + per);

  // ---- 1: log-sum-exp and unique count ----
  {
    long long m = kKeyInvalid;
    float sum = 0.f, comp = 0.f;
    unsigned valid = 0;
    for (long long j = lo + tid; j < hi; j += nthr) {
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
      const float y = term - comp;
      const float t = sum + y;
      comp = (t - sum) - y;
      sum = t;
    }
    const double s = (double)sum - (double)comp;
    long long mm = warp_max_k(m);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) valid += __shfl_xor_sync(0xFFFFFFFFu, valid, o);
    if (lane == 0) {
      S.part[wp] = (unsigned long long)mm;
      S.dpart[wp] = 0.0;
      S.hist[wp] = valid;
    }
    __syncthreads();
    if (wp == 0) {
      long long M = lane < nw ? (long long)S.part[lane] : kKeyInvalid;
      M = warp_max_k(M);
      unsigned c = lane < nw ? S.hist[lane] : 0u;
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xFFFFFFFFu, c, o);
      if (lane == 0) {
        S.pm = M;
        S.pc = c;
      }
    }
    __syncthreads();
    const long long M = S.pm;
    double r = (m == kKeyInvalid || !(s > 0.0)) ? 0.0 : s * (double)expf(fx_to_f(m - M));
    r = warp_sum_dd(r);
    if (lane == 0) S.dpart[wp] = r;
    __syncthreads();
    if (wp == 0) {
      double q = lane < nw ? S.dpart[lane] : 0.0;
      q = warp_sum_dd(q);
      if (lane == 0) S.ps = q;
    }
  }
  cl.sync();
  if (wp == 0) {
    // lane r holds CTA r's partial; maximum, rescale, sum over a fixed tree:
    // the same result in every CTA
    long long bm = kKeyInvalid;
    double bs = 0.0;
    unsigned cnt = 0;
    if (lane < C) {
      const SelShared* R = cl.map_shared_rank(&S, lane);
      bm = R->pm;
      bs = R->ps;
      cnt = R->pc;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) cnt += __shfl_xor_sync(0xFFFFFFFFu, cnt, o);
    const long long M = warp_max_k((bm == kKeyInvalid || !(bs > 0.0)) ? kKeyInvalid : bm);
    double r = (bm == kKeyInvalid || !(bs > 0.0) || M == kKeyInvalid) ? 0.0 : bs * (double)expf(fx_to_f(bm - M));
    const double sum = warp_sum_dd(r);
    if (lane == 0) {
      S.prefix = 0;
      S.need = h_max;
      S.bnd = 0;
      if (M == kKeyInvalid || !(sum > 0.0)) {
        S.lse = -INFINITY;
        S.thr = LLONG_MAX;
        S.mode = 2;
      } else {
        const double lse = (double)M * kFxInv + log(sum);
        S.lse = lse;
        S.thr = (long long)ceil((lse + log_tau) * 4294967296.0);
        S.mode = 0;
      }
      if (rank == 0) {
        w.lse[0] = S.lse;
        w.thr[0] = S.thr;
        w.counts[2] = cnt;
      }
    }
  }
  __syncthreads();

  // ---- 2: radix select of the H_max largest keys at or above thr ----
  const long long thr = S.thr;
  const int passes = (nbits + kSelDigit - 1) / kSelDigit;
  const int slice = (kSelBins + C - 1) / C;
  for (int p = 0; p < passes; ++p) {
    const int shift = (passes - 1 - p) * kSelDigit;
    const int mode = S.mode;   // identical in every CTA
    if (mode != 0) break;
    unsigned* hs = S.hsum[p & 1];
    for (int b = tid; b < kSelBins; b += nthr) S.hist[b] = 0u;
    __syncthreads();
    const unsigned long long prefix = (unsigned long long)S.prefix;
    // one shared-memory atomic per distinct bin of a warp (the keys near the
    // top crowd a few bins)
    for (long long base = lo; base < hi; base += nthr) {
      const long long j = base + tid;
      int bin = -1;
      if (j < hi) {
        const long long k = keys[j];
        if (k != kKeyInvalid && k >= thr) {
          const unsigned long long v = (unsigned long long)(k - thr);
          if ((v >> (shift + kSelDigit)) == prefix) bin = (int)((v >> shift) & (kSelBins - 1));
        }
      }
      const unsigned grp = __match_any_sync(0xFFFFFFFFu, bin);
      if (bin >= 0 && lane == __ffs(grp) - 1) atomicAdd(&S.hist[bin], (unsigned)__popc(grp));
    }
    cl.sync();
    // this CTA's slice of the summed histogram
    for (int b = rank * slice + tid; b < min(kSelBins, (rank + 1) * slice); b += nthr) {
      unsigned t = 0;
      for (int r = 0; r < C; ++r) t += cl.map_shared_rank(S.hist, r)[b];
      hs[b] = t;
    }
    cl.sync();
    // gather the other slices
    for (int b = tid; b < kSelBins; b += nthr) {
      const int owner = b / slice;
      if (owner != rank) hs[b] = cl.map_shared_rank(hs, owner)[b];
    }
    __syncthreads();
    // boundary digit: thread t owns bins [4t, 4t + 4); counts above a range =
    // total - inclusive prefix
    {
      unsigned b4[4], mine = 0;
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        b4[k] = hs[4 * tid + k];
        mine += b4[k];
      }
      unsigned x = mine;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const unsigned y = __shfl_up_sync(0xFFFFFFFFu, x, o);
        if (lane >= o) x += y;
      }
      if (lane == 31) S.part[wp] = x;
      __syncthreads();
      if (wp == 0) {
        unsigned long long s = S.part[lane];
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
          const unsigned long long y = __shfl_up_sync(0xFFFFFFFFu, s, o);
          if (lane >= o) s += y;
        }
        S.part[lane] = s;
      }
      __syncthreads();
      const unsigned incl = x + (wp > 0 ? (unsigned)S.part[wp - 1] : 0u);
      const unsigned total = (unsigned)S.part[31];
      const unsigned above = total - incl, upto = above + mine;
      const long long need = S.need;
      __syncthreads();   // everyone has read need before it changes
      if (p == 0 && (long long)total <= need) {
        if (tid == 0) {
          S.mode = 1;
          S.bnd = thr - 1;   // every candidate is above the boundary
          S.need = 0;
        }
      } else if ((long long)above < need && (long long)upto >= need) {
        unsigned cum = above;
        int b = 3;
        for (; b > 0; --b) {
          if ((long long)(cum + b4[b]) >= need) break;
          cum += b4[b];
        }
        S.prefix = (S.prefix << kSelDigit) | (4 * tid + b);
        S.need = need - cum;
        if (shift == 0) S.bnd = thr + S.prefix;
      }
      __syncthreads();
    }
  }
  cl.sync();   // the summed histograms are no longer read

  // ---- 3: stable compaction in child order ----
  const int mode = S.mode;
  const long long bnd = S.bnd, need = S.need;
  const long long chunk = hi - lo;
  const long long q = (chunk + nthr - 1) / nthr;
  const long long a0 = lo + (long long)tid * q, a1 = min(hi, a0 + q);
  unsigned long long mine = 0ull;
  for (long long j = a0; j < a1; ++j) mine += keep_flag(keys[j], thr, bnd, need, mode);
  // block exclusive scan of (above | at << 32)
  unsigned long long x = mine;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const unsigned long long y = __shfl_up_sync(0xFFFFFFFFu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) S.part[wp] = x;
  __syncthreads();
  if (wp == 0) {
    unsigned long long s = lane < nw ? S.part[lane] : 0ull;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const unsigned long long y = __shfl_up_sync(0xFFFFFFFFu, s, o);
      if (lane >= o) s += y;
    }
    S.part[lane] = s;
  }
  __syncthreads();
  const unsigned long long excl_blk = (wp > 0 ? S.part[wp - 1] : 0ull) + x - mine;
  if (tid == 0) S.cnt = S.part[nw - 1];
  cl.sync();
  if (wp == 0) {
    const unsigned long long c = lane < C ? cl.map_shared_rank(&S, lane)->cnt : 0ull;
    unsigned long long before = lane < rank ? c : 0ull, total = c;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      before += __shfl_xor_sync(0xFFFFFFFFu, before, o);
      total += __shfl_xor_sync(0xFFFFFFFFu, total, o);
    }
    if (lane == 0) {
      S.before = before;
      S.total = total;
    }
  }
  __syncthreads();
  {
    unsigned long long run = S.before + excl_blk;
    for (long long j = a0; j < a1; ++j) {
      const unsigned long long f = keep_flag(keys[j], thr, bnd, need, mode);
      if (!f) continue;
      const long long gt = (long long)(run & 0xFFFFFFFFull), eq = (long long)(run >> 32);
      run += f;
      if ((f >> 32) && eq >= need) continue;
      const long long pos = gt + min(eq, need);
      if (pos < h_max) w.surv_idx[pos] = j;
    }
  }
  cl.sync();   // every survivor index is written (the cluster barrier orders them)
  if (rank != 0) return;

  // ---- 4: the retained set ----
  __shared__ long long s_n;
  __shared__ double s_lse;
  __shared__ uint32_t carry;
  if (tid == 0) {
    const unsigned long long tot = S.total;
    long long ns = 0;
    if (mode != 2) ns = (long long)(tot & 0xFFFFFFFFull) + min((long long)(tot >> 32), need);
    if (ns > h_max) ns = h_max;
    s_n = ns;
    w.counts[0] = (unsigned)ns;
    w.sel[0] = S.prefix;
    w.sel[1] = need;
    w.sel[2] = bnd;
    w.sel[3] = mode;
    carry = 0;
  }
  __syncthreads();
  const long long ns = s_n;
  const double lse_all = S.lse;
  // each thread's survivors (one per thread when ns <= blockDim.x): every
  // load issued together
  constexpr int kPer = 4;
  long long sj[kPer], sk[kPer];
  uint32_t sna[kPer];
  unsigned long long suid[kPer];
  const int rounds = (int)((ns + nthr - 1) / nthr);
  const bool held = rounds <= kPer;
  {
    long long m = kKeyInvalid;
    double s = 0.0;
#pragma unroll
    for (int r = 0; r < kPer; ++r) {
      sj[r] = 0;
      sk[r] = 0;
      sna[r] = 0;
      suid[r] = 0;
    }
    for (int r = 0; r < rounds; ++r) {
      const long long t = (long long)r * nthr + tid;
      if (t >= ns) break;
      const long long j = w.surv_idx[t];
      if (j < 0 || j >= n) {   // invariant: every survivor index was written this frame
        atomicOr(err, kErrChkSurv);
        continue;
      }
      const long long k = keys[j];
      if (held) {
#pragma unroll
        for (int q = 0; q < kPer; ++q)
          if (q == r) {
            sj[q] = j;
            sk[q] = k;
            sna[q] = child_alive[j];
            suid[q] = parents.uid[j / h_up];
          }
      }
      if (m == kKeyInvalid) { m = k; s = 1.0; }
      else if (k > m) { s = 1.0 + s * (double)expf(fx_to_f(m - k)); m = k; }
      else s += (double)expf(fx_to_f(k - m));
    }
    long long mm = warp_max_k(m);
    if (lane == 0) S.part[wp] = (unsigned long long)mm;
    __syncthreads();
    if (wp == 0) {
      long long M = lane < nw ? (long long)S.part[lane] : kKeyInvalid;
      M = warp_max_k(M);
      if (lane == 0) S.pm = M;
    }
    __syncthreads();
    const long long M = S.pm;
    double r = (m == kKeyInvalid) ? 0.0 : s * (double)expf(fx_to_f(m - M));
    r = warp_sum_dd(r);
    if (lane == 0) S.dpart[wp] = r;
    __syncthreads();
    if (wp == 0) {
      double q2 = lane < nw ? S.dpart[lane] : 0.0;
      q2 = warp_sum_dd(q2);
      if (lane == 0) {
        s_lse = (double)M * kFxInv - lse_all + log(q2);
        w.lse[1] = s_lse;
      }
    }
    __syncthreads();
  }
  uint32_t amax = 0;
  for (int r = 0; r < rounds; ++r) {
    const long long t = (long long)r * nthr + tid;
    uint32_t na = 0;
    if (t < ns) {
      long long j, k;
      unsigned long long pu;
      if (held) {
        j = sj[0];
        k = sk[0];
        na = sna[0];
        pu = suid[0];
#pragma unroll
        for (int q = 1; q < kPer; ++q)
          if (q == r) {
            j = sj[q];
            k = sk[q];
            na = sna[q];
            pu = suid[q];
          }
      } else {
        j = w.surv_idx[t];
        if (j < 0 || j >= n) {
          atomicOr(err, kErrChkSurv);
          j = 0;
        }
        k = keys[j];
        na = child_alive[j];
        pu = parents.uid[j / h_up];
      }
      out.logw[t] = (double)k * kFxInv - lse_all - s_lse;
      out.uid[t] = mix64(pu + 0x9E3779B97F4A7C15ULL * (unsigned long long)(j % h_up + 1));
      amax = max(amax, na);
    }
    uint32_t y = na;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t z = __shfl_up_sync(0xFFFFFFFFu, y, o);
      if (lane >= o) y += z;
    }
    if (lane == 31) S.hist[wp] = y;
    __syncthreads();
    if (wp == 0) {
      uint32_t v = lane < nw ? S.hist[lane] : 0u;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const uint32_t z = __shfl_up_sync(0xFFFFFFFFu, v, o);
        if (lane >= o) v += z;
      }
      S.hist[lane] = v;
    }
    __syncthreads();
    const uint32_t excl = carry + (wp > 0 ? S.hist[wp - 1] : 0u) + y - na;
    if (t < ns) out.ptr[t] = excl;
    __syncthreads();
    if (tid == 0) carry += S.hist[nw - 1];
    __syncthreads();
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) amax = max(amax, __shfl_xor_sync(0xFFFFFFFFu, amax, o));
  if (lane == 0 && amax) atomicMax(&w.counts[3], amax);
  if (tid == 0) {
    out.ptr[ns] = carry;
    w.counts[1] = carry;
    if ((long long)carry > cap_entries) atomicOr(err, kErrEntries);
  }
}

int select_cluster_size() {
  static int size = -1;
  if (size >= 0) return size;
  size = 0;
  cudaFuncSetAttribute(select_cluster_kernel, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
  cudaFuncSetAttribute(select_cluster_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(SelShared));
  for (int c : {16, 8, 4}) {
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = dim3(c);
    cfg.blockDim = dim3(kSelThreads);
    cfg.dynamicSmemBytes = sizeof(SelShared);
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = c;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    int clusters = 0;
    if (cudaOccupancyMaxActiveClusters(&clusters, select_cluster_kernel, &cfg) == cudaSuccess && clusters > 0) {
      size = c;
      break;
    }
  }
  cudaGetLastError();
  return size;
}

bool launch_select_cluster(const long long* keys, const FrameDev* fs, int h_up, PruneWork w, double log_tau,
                           int h_max, int nbits, const uint16_t* child_alive, const HypTable& parents,
                           const HypTable& out, unsigned* err, long long cap_entries, cudaStream_t s) {
  const int c = select_cluster_size();
  if (c == 0) return false;
  cudaLaunchConfig_t cfg{};
  cfg.gridDim = dim3(c);
  cfg.blockDim = dim3(kSelThreads);
  cfg.dynamicSmemBytes = sizeof(SelShared);
  cfg.stream = s;
  cudaLaunchAttribute at[2];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = c;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  at[1].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[1].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = at;
  cfg.numAttrs = 2;
  if (cudaLaunchKernelEx(&cfg, select_cluster_kernel, keys, fs, h_up, w, log_tau, h_max, nbits, child_alive,
                         parents, out, err, cap_entries) != cudaSuccess)
    return false;
  ++g_launches;
  return true;
}

}  // namespace glmb

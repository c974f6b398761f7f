// Normalisation, truncation to the top H_max and renormalisation of the
// children (arXiv 2512.06230, Section 3, pruning) in one launch: a cluster
// of CTAs on neighbouring SMs that combine their partial results through
// distributed shared memory, instead of a chain of grid-wide kernels.
//
//   1  log-sum-exp over the unique children from the partials the
//      duplicate-marking kernel left per block (per-thread integer maximum
//      and compensated FP32 sums of FP32 exponentials, rescaled and summed
//      in FP64), the unique count, the fixed-point threshold log(tau) + LSE;
//   2  top-H_max among the children at or above the threshold by 12-bit
//      radix select on key - threshold: every CTA histograms its slice,
//      each CTA sums one slice of bins over the cluster, every CTA gathers
//      the summed histogram and finds the boundary digit (all CTAs compute
//      the same result, so no broadcast is needed).  The first pass also
//      counts each thread's children at or above the threshold: when the
//      cluster's count is within H_max every one of them is kept, and that
//      count is the compaction's, so no second pass is made;
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
                      int n_part, double log_tau, int h_max, int nbits, const uint16_t* __restrict__ child_alive,
                      HypTable parents, HypTable out, unsigned* err, long long cap_entries) {
  pdl_enter();
  cg::cluster_group cl = cg::this_cluster();
  const int C = (int)cl.num_blocks(), rank = (int)cl.block_rank();
  const int tid = threadIdx.x, nthr = blockDim.x, lane = tid & 31, wp = tid >> 5, nw = nthr >> 5;
  // the prune counters start at zero (this thread writes the first of them
  // below; the others are written after cluster barriers)
  if (rank == 0 && tid == 0)
    for (int i = 0; i < 8; ++i) w.counts[i] = 0u;
  // a frame whose expansion was skipped (the staging flagged it, or the
  // table failed) holds stale children: nothing to select; every CTA of the
  // cluster reads the same flag and returns before any cluster barrier
  if (*(volatile const unsigned*)err & kErrFatal) return;
  extern __shared__ __align__(16) unsigned char sel_sm[];
  SelShared& S = *reinterpret_cast<SelShared*>(sel_sm);
  const long long n = (long long)fs->H * h_up;
  const long long per = (n + C - 1) / C;
  const long long lo = min(n, (long long)rank * per), hi = min(n, lo + per);

  // ---- 1: log-sum-exp and unique count, from the per-block partials ----
  // (every CTA reduces all of them in the same order: the same result;
  // blocks beyond the parents wrote none)
  n_part = min(n_part, fs->H);
  {
    long long m = kKeyInvalid;
    for (int b = tid; b < n_part; b += nthr) m = max(m, w.part_max[b]);
    m = warp_max_k(m);
    if (lane == 0) S.part[wp] = (unsigned long long)m;
    __syncthreads();
    if (wp == 0) {
      long long M = lane < nw ? (long long)S.part[lane] : kKeyInvalid;
      M = warp_max_k(M);
      if (lane == 0) S.pm = M;
    }
    __syncthreads();
    const long long M = S.pm;
    double r = 0.0;
    unsigned c = 0;
    for (int b = tid; b < n_part; b += nthr) {
      r += lse_rescale(w.part_max[b], w.part_sum[b], M);
      c += w.part_cnt[b];
    }
    r = warp_sum_dd(r);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xFFFFFFFFu, c, o);
    if (lane == 0) {
      S.dpart[wp] = r;
      S.hist[wp] = c;
    }
    __syncthreads();
    if (wp == 0) {
      double q = lane < nw ? S.dpart[lane] : 0.0;
      q = warp_sum_dd(q);
      unsigned cc = lane < nw ? S.hist[lane] : 0u;
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) cc += __shfl_xor_sync(0xFFFFFFFFu, cc, o);
      if (lane == 0) {
        S.prefix = 0;
        S.need = h_max;
        S.bnd = 0;
        if (M == kKeyInvalid || !(q > 0.0)) {
          S.lse = -INFINITY;
          S.thr = LLONG_MAX;
          S.mode = 2;
        } else {
          const double lse = (double)M * kFxInv + log(q);
          S.lse = lse;
          S.thr = (long long)ceil((lse + log_tau) * 4294967296.0);
          S.mode = 0;
        }
        if (rank == 0) {
          w.lse[0] = S.lse;
          w.thr[0] = S.thr;
          w.counts[2] = cc;
        }
      }
    }
  }
  __syncthreads();

  // ---- 2: radix select of the H_max largest keys at or above thr ----
  const long long thr = S.thr;
  const int passes = (nbits + kSelDigit - 1) / kSelDigit;
  const int slice = (kSelBins + C - 1) / C;
  // each thread's contiguous share of the CTA's children (compaction order)
  const long long chunk = hi - lo;
  const long long q = (chunk + nthr - 1) / nthr;
  const long long a0 = lo + (long long)tid * q, a1 = min(hi, a0 + q);
  unsigned long long above0 = 0ull;   // this thread's children at or above thr (first pass)
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
    // the lanes with a bin (most children are below the threshold) add
    // their counts, one atomic per distinct bin
    auto add_bin = [&](int bin) {
      const unsigned act = __ballot_sync(0xFFFFFFFFu, bin >= 0);
      if (bin >= 0) {
        const unsigned grp = __match_any_sync(act, bin);
        if (lane == __ffs(grp) - 1) atomicAdd(&S.hist[bin], (unsigned)__popc(grp));
      }
    };
    if (p == 0) {
      // over the thread's own share, counting it as well; four loads in
      // flight per step (every lane runs the same steps, so the warp stays
      // converged for the ballots)
      for (long long t = 0; t < q; t += 4) {
        long long k4[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) k4[u] = a0 + t + u < a1 ? keys[a0 + t + u] : kKeyInvalid;
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          int bin = -1;
          if (k4[u] != kKeyInvalid && k4[u] >= thr) {
            ++above0;
            bin = (int)(((unsigned long long)(k4[u] - thr) >> shift) & (kSelBins - 1));
          }
          add_bin(bin);
        }
      }
    } else {
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
        add_bin(bin);
      }
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
  // every candidate kept (decided by the first pass), or none: the first
  // pass's count is the thread's; else count above and at the boundary
  unsigned long long mine = mode == 1 ? above0 : 0ull;
  if (mode == 0)
#pragma unroll 4
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
    // a share with nothing kept is not read again
    for (long long t = a0; mine && t < a1; t += 4) {
      long long k4[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) k4[u] = t + u < a1 ? keys[t + u] : kKeyInvalid;
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const unsigned long long f = keep_flag(k4[u], thr, bnd, need, mode);
        if (!f) continue;
        const long long gt = (long long)(run & 0xFFFFFFFFull), eq = (long long)(run >> 32);
        run += f;
        if ((f >> 32) && eq >= need) continue;
        const long long pos = gt + min(eq, need);
        if (pos < h_max) w.surv_idx[pos] = t + u;
      }
    }
  }
  cl.sync();   // every survivor index is written (the cluster barrier orders them)

  // ---- 4: the retained set, each CTA a contiguous share of it ----
  long long ns = 0;
  {
    const unsigned long long tot = S.total;
    if (mode != 2) ns = (long long)(tot & 0xFFFFFFFFull) + min((long long)(tot >> 32), need);
    if (ns > h_max) ns = h_max;
  }
  // shared over the cluster when it is larger than two rounds of one CTA;
  // else CTA 0 alone, without the cluster barriers
  const bool spread = ns > 2LL * nthr;
  if (!spread && rank != 0) return;
  const int Cs = spread ? C : 1;
  const long long sper = (ns + Cs - 1) / Cs;
  const long long r0 = min(ns, (long long)rank * sper), r1 = min(ns, r0 + sper);
  const double lse_all = S.lse;
  // each thread's survivors (up to kPer rounds held in registers; beyond
  // that they are read again for the writes)
  constexpr int kPer = 2;
  long long sj[kPer], sk[kPer];
  uint32_t sna[kPer];
  unsigned long long suid[kPer];
  const int rounds = (int)((r1 - r0 + nthr - 1) / nthr);
  const bool held = rounds <= kPer;
  auto load_survivor = [&](long long t, long long& j, long long& k, uint32_t& na, unsigned long long& pu) {
    j = w.surv_idx[t];
    if (j < 0 || j >= n) {   // invariant: every survivor index was written this frame
      atomicOr(err, kErrChkSurv);
      j = 0;
    }
    k = keys[j];
    na = child_alive[j];
    pu = parents.uid[j / h_up];
  };
  {
    // the share's maximum, sum of exp(key - maximum) and alive count
    long long m = kKeyInvalid;
    double sm_ = 0.0;
    unsigned long long alive = 0ull;
    uint32_t amax = 0;
#pragma unroll
    for (int r = 0; r < kPer; ++r) {
      sj[r] = 0;
      sk[r] = 0;
      sna[r] = 0;
      suid[r] = 0;
    }
    for (int r = 0; r < rounds; ++r) {
      const long long t = r0 + (long long)r * nthr + tid;
      if (t >= r1) break;
      long long j, k;
      uint32_t na;
      unsigned long long pu;
      load_survivor(t, j, k, na, pu);
      if (held) {
#pragma unroll
        for (int q2 = 0; q2 < kPer; ++q2)
          if (q2 == r) {
            sj[q2] = j;
            sk[q2] = k;
            sna[q2] = na;
            suid[q2] = pu;
          }
      }
      alive += na;
      amax = max(amax, na);
      if (m == kKeyInvalid) { m = k; sm_ = 1.0; }
      else if (k > m) { sm_ = 1.0 + sm_ * (double)expf(fx_to_f(m - k)); m = k; }
      else sm_ += (double)expf(fx_to_f(k - m));
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) amax = max(amax, __shfl_xor_sync(0xFFFFFFFFu, amax, o));
    if (lane == 0 && amax) atomicMax(&w.counts[3], amax);
    long long mm = warp_max_k(m);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) alive += __shfl_xor_sync(0xFFFFFFFFu, alive, o);
    if (lane == 0) {
      S.part[wp] = (unsigned long long)mm;
      S.hist[wp] = (unsigned)alive;
    }
    __syncthreads();
    if (wp == 0) {
      long long M = lane < nw ? (long long)S.part[lane] : kKeyInvalid;
      M = warp_max_k(M);
      unsigned long long a = lane < nw ? S.hist[lane] : 0u;
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) a += __shfl_xor_sync(0xFFFFFFFFu, a, o);
      if (lane == 0) {
        S.pm = M;
        S.before = a;   // this CTA's alive count, read by the cluster
      }
    }
    __syncthreads();
    double r = (m == kKeyInvalid) ? 0.0 : sm_ * (double)expf(fx_to_f(m - S.pm));
    r = warp_sum_dd(r);
    if (lane == 0) S.dpart[wp] = r;
    __syncthreads();
    if (wp == 0) {
      double q2 = lane < nw ? S.dpart[lane] : 0.0;
      q2 = warp_sum_dd(q2);
      if (lane == 0) S.ps = q2;
    }
  }
  if (spread) cl.sync();
  __shared__ double s_lse;
  __shared__ uint32_t carry;
  if (wp == 0) {
    // lane r holds CTA r's share: maximum, sum, alive count (a fixed tree:
    // the same log-sum-exp in every CTA)
    long long bm = kKeyInvalid;
    double bs = 0.0;
    unsigned long long ba = 0ull;
    if (lane < Cs) {
      const SelShared* R = spread ? cl.map_shared_rank(&S, lane) : &S;
      bm = R->pm;
      bs = R->ps;
      ba = R->before;
    }
    const long long M = warp_max_k(bm);
    const double q2 = warp_sum_dd(lse_rescale(bm, bs, M));
    unsigned long long before = lane < rank ? ba : 0ull, total = ba;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      before += __shfl_xor_sync(0xFFFFFFFFu, before, o);
      total += __shfl_xor_sync(0xFFFFFFFFu, total, o);
    }
    if (lane == 0) {
      s_lse = (M == kKeyInvalid) ? 0.0 : (double)M * kFxInv - lse_all + log(q2);
      carry = (uint32_t)before;
      if (rank == 0) {
        w.counts[0] = (unsigned)ns;
        w.counts[1] = (unsigned)total;
        w.sel[0] = S.prefix;
        w.sel[1] = need;
        w.sel[2] = bnd;
        w.sel[3] = mode;
        w.lse[1] = s_lse;
        out.ptr[ns] = (uint32_t)total;
        if ((long long)total > cap_entries) atomicOr(err, kErrEntries);
      }
    }
  }
  if (spread) cl.sync();   // no CTA leaves while another reads its shared memory
  else __syncthreads();
  const double lse_ret = s_lse;
  for (int r = 0; r < rounds; ++r) {
    const long long t = r0 + (long long)r * nthr + tid;
    uint32_t na = 0;
    if (t < r1) {
      long long j, k;
      unsigned long long pu;
      if (held) {
        j = sj[0];
        k = sk[0];
        na = sna[0];
        pu = suid[0];
#pragma unroll
        for (int q2 = 1; q2 < kPer; ++q2)
          if (q2 == r) {
            j = sj[q2];
            k = sk[q2];
            na = sna[q2];
            pu = suid[q2];
          }
      } else {
        load_survivor(t, j, k, na, pu);
      }
      out.logw[t] = (double)k * kFxInv - lse_all - lse_ret;
      out.uid[t] = mix64(pu + 0x9E3779B97F4A7C15ULL * (unsigned long long)(j % h_up + 1));
    }
    // CSR offsets: exclusive scan of the alive counts over the share
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
    if (t < r1) out.ptr[t] = excl;
    __syncthreads();
    if (tid == 0) carry += S.hist[nw - 1];
    __syncthreads();
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

bool launch_select_cluster(const long long* keys, const FrameDev* fs, int h_up, PruneWork w, int n_part,
                           double log_tau, int h_max, int nbits, const uint16_t* child_alive,
                           const HypTable& parents, const HypTable& out, unsigned* err, long long cap_entries,
                           cudaStream_t s) {
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
  if (cudaLaunchKernelEx(&cfg, select_cluster_kernel, keys, fs, h_up, w, n_part, log_tau, h_max, nbits,
                         child_alive, parents, out, err, cap_entries) != cudaSuccess)
    return false;
  ++g_launches;
  return true;
}

}  // namespace glmb

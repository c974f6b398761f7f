// glmb_select_top_static: top-H selection of child log-weights that makes no
// device allocation.  Its scratch is the file-scope array below (41,216
// bytes, sized for at most kMaxBlocks blocks); every GPU that loads the
// library holds it until the process exits.
//
// Who needs it: callers that may not allocate device memory while they run,
// such as a tracking loop with a fixed memory budget and a hard frame
// deadline (cudaMalloc can synchronise the device and stall for
// milliseconds), or code embedded in a host application whose memory policy
// forbids raw cudaMalloc.  The caller still passes the inputs and outputs.
//
// The steps are those of the selection inside glmb_prune: log-weights are
// converted to int64 with 2^-32 resolution, normalised by their log-sum-exp,
// children below tau are dropped, the h_max largest are kept (ties by
// index), the kept ones are listed in index order and their log-weights
// renormalised.  The log-sum-exp is summed differently (FP64 exponentials
// here, FP32 exponentials with compensated sums there), so the two agree up
// to its rounding: a child whose normalised weight lies within that rounding
// of tau may land on either side of the cut.
#include <algorithm>
#include <cmath>
#include <mutex>

#include "../../include/glmb.h"
#include "glmb_dev.cuh"

namespace {

using namespace glmb;

constexpr int kMaxBlocks = 1024;
constexpr int kThreads = 256;
constexpr int kDigitS = 12, kBinsS = 1 << kDigitS;
constexpr long long kMaxN = 1LL << 30;

// scratch layout (bytes)
constexpr size_t kOffBlkM = 0;                                   // long long[kMaxBlocks]
constexpr size_t kOffBlkS = kOffBlkM + 8 * kMaxBlocks;           // double[kMaxBlocks]
constexpr size_t kOffBlkGt = kOffBlkS + 8 * kMaxBlocks;          // uint32[kMaxBlocks]
constexpr size_t kOffBlkEq = kOffBlkGt + 4 * kMaxBlocks;         // uint32[kMaxBlocks]
constexpr size_t kOffHist = kOffBlkEq + 4 * kMaxBlocks;          // uint32[kBinsS]
constexpr size_t kOffScal = kOffHist + 4 * kBinsS;               // Scal
constexpr size_t kScratchBytes = kOffScal + 256;
// the size glmb.h states for the scratch array
static_assert(kScratchBytes == 41216, "scratch size changed: update glmb.h");

struct SelScal {
  unsigned done;        // last-block counter
  unsigned pad;
  double lse;           // log-sum-exp over valid children
  long long thr;        // fixed-point threshold
  long long prefix;     // radix prefix
  long long need;       // elements still needed at the boundary key
  long long bound;      // boundary key
  long long mode;       // 0 running, 1 keep all candidates, 2 nothing valid
  long long n_kept;
};

__device__ __align__(256) unsigned char g_select_scratch[kScratchBytes];

struct Ptrs {
  long long* blk_m;
  double* blk_s;
  unsigned* blk_gt;
  unsigned* blk_eq;
  unsigned* hist;
  SelScal* sc;
};

__host__ __device__ inline Ptrs ptrs_of(unsigned char* base) {
  return Ptrs{(long long*)(base + kOffBlkM), (double*)(base + kOffBlkS), (unsigned*)(base + kOffBlkGt),
              (unsigned*)(base + kOffBlkEq), (unsigned*)(base + kOffHist), (SelScal*)(base + kOffScal)};
}

__device__ __forceinline__ long long key_of(double lw) {
  // log-weights outside (-2^30, 2^30) -- -inf, +inf and NaN among them --
  // mark children without weight; inside, every key is below 2^62 in
  // magnitude, so the difference of two keys cannot overflow
  if (!(lw > -1073741824.0 && lw < 1073741824.0)) return kKeyInvalid;
  return __double2ll_rn(lw * 4294967296.0);
}

struct LseS {
  long long m;
  double s;
};
__device__ __forceinline__ LseS comb(LseS a, LseS b) {
  if (a.m == kKeyInvalid) return b;
  if (b.m == kKeyInvalid) return a;
  if (a.m >= b.m) return {a.m, a.s + b.s * exp((double)(b.m - a.m) * kFxInv)};
  return {b.m, b.s + a.s * exp((double)(a.m - b.m) * kFxInv)};
}
__device__ LseS block_comb(LseS v) {
  __shared__ long long sm[32];
  __shared__ double ss[32];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1)
    v = comb(v, LseS{__shfl_xor_sync(0xFFFFFFFFu, v.m, o), __shfl_xor_sync(0xFFFFFFFFu, v.s, o)});
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
  __syncthreads();
  if (lane == 0) { sm[w] = v.m; ss[w] = v.s; }
  __syncthreads();
  if (w == 0) {
    v = lane < nw ? LseS{sm[lane], ss[lane]} : LseS{kKeyInvalid, 0.0};
#pragma unroll
    for (int o = 16; o > 0; o >>= 1)
      v = comb(v, LseS{__shfl_xor_sync(0xFFFFFFFFu, v.m, o), __shfl_xor_sync(0xFFFFFFFFu, v.s, o)});
  }
  return v;
}

__device__ __forceinline__ void chunk_of(long long n, long long& lo, long long& hi) {
  const long long per = (n + gridDim.x - 1) / gridDim.x;
  lo = (long long)blockIdx.x * per;
  hi = lo + per < n ? lo + per : n;
}

// the previous call's contents are cleared here
__global__ void sel_init(unsigned char* base, int h_max) {
  Ptrs p = ptrs_of(base);
  for (int b = threadIdx.x; b < kBinsS; b += blockDim.x) p.hist[b] = 0u;
  if (threadIdx.x == 0) {
    p.sc->done = 0u;
    p.sc->need = h_max;
    p.sc->prefix = 0;
    p.sc->bound = 0;
    p.sc->mode = 0;
    p.sc->n_kept = 0;
  }
}

__global__ void sel_lse(const double* __restrict__ lw, long long n, double log_tau,
                        unsigned char* base) {
  __shared__ bool last;
  Ptrs p = ptrs_of(base);
  long long lo, hi;
  chunk_of(n, lo, hi);
  LseS v{kKeyInvalid, 0.0};
  for (long long j = lo + threadIdx.x; j < hi; j += blockDim.x) {
    const long long k = key_of(lw[j]);
    if (k != kKeyInvalid) v = comb(v, LseS{k, 1.0});
  }
  v = block_comb(v);
  if (threadIdx.x == 0) {
    p.blk_m[blockIdx.x] = v.m;
    p.blk_s[blockIdx.x] = v.s;
    __threadfence();
    last = atomicAdd(&p.sc->done, 1u) == gridDim.x - 1;
  }
  __syncthreads();
  if (!last) return;
  __threadfence();
  LseS u{kKeyInvalid, 0.0};
  for (unsigned b = threadIdx.x; b < gridDim.x; b += blockDim.x)
    u = comb(u, LseS{((volatile long long*)p.blk_m)[b], ((volatile double*)p.blk_s)[b]});
  u = block_comb(u);
  if (threadIdx.x == 0) {
    p.sc->done = 0u;
    if (u.m == kKeyInvalid || !(u.s > 0.0)) {
      p.sc->lse = -INFINITY;
      p.sc->thr = LLONG_MAX;
      p.sc->mode = 2;
    } else {
      p.sc->lse = (double)u.m * kFxInv + log(u.s);
      p.sc->thr = (long long)ceil((p.sc->lse + log_tau) * 4294967296.0);
    }
  }
}

__global__ void sel_hist(const double* __restrict__ lw, long long n, int shift, unsigned char* base) {
  __shared__ unsigned hist[kBinsS];
  Ptrs p = ptrs_of(base);
  if (p.sc->mode != 0) return;
  for (int b = threadIdx.x; b < kBinsS; b += blockDim.x) hist[b] = 0;
  __syncthreads();
  const long long thr = p.sc->thr;
  const unsigned long long prefix = (unsigned long long)p.sc->prefix;
  long long lo, hi;
  chunk_of(n, lo, hi);
  for (long long j = lo + threadIdx.x; j < hi; j += blockDim.x) {
    const long long k = key_of(lw[j]);
    if (k == kKeyInvalid || k < thr) continue;
    const unsigned long long v = (unsigned long long)(k - thr);
    if ((v >> (shift + kDigitS)) != prefix) continue;
    atomicAdd(&hist[(v >> shift) & (kBinsS - 1)], 1u);
  }
  __syncthreads();
  for (int b = threadIdx.x; b < kBinsS; b += blockDim.x)
    if (hist[b]) atomicAdd(&p.hist[b], hist[b]);
}

// one block of kBinsS / 4 threads; thread t owns bins [4t, 4t + 4)
__global__ void sel_find(int shift, int first, unsigned char* base) {
  __shared__ unsigned wsum[32];
  Ptrs p = ptrs_of(base);
  const int t = threadIdx.x, lane = t & 31, wp = t >> 5;
  const bool running = p.sc->mode == 0;
  const long long need = p.sc->need;
  unsigned b4[4], mine = 0;
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    b4[k] = p.hist[4 * t + k];
    mine += b4[k];
    p.hist[4 * t + k] = 0;
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
  const unsigned above = total - incl, upto = above + mine;
  if (first && (long long)total <= need) {
    if (t == 0) {
      p.sc->mode = 1;
      p.sc->bound = p.sc->thr - 1;
      p.sc->need = 0;
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
    p.sc->prefix = (p.sc->prefix << kDigitS) | (4 * t + b);
    p.sc->need = need - cum;
    if (shift == 0) p.sc->bound = p.sc->thr + p.sc->prefix;
  }
}

__device__ __forceinline__ void keep_kind(long long k, const SelScal& s, bool& gt, bool& eq) {
  gt = eq = false;
  if (s.mode == 2 || k == kKeyInvalid || k < s.thr) return;
  if (k > s.bound) gt = true;
  else if (k == s.bound && s.need > 0) eq = true;
}

__global__ void sel_count(const double* __restrict__ lw, long long n, unsigned char* base) {
  __shared__ unsigned cg, ce;
  Ptrs p = ptrs_of(base);
  if (threadIdx.x == 0) { cg = 0; ce = 0; }
  __syncthreads();
  const SelScal s = *p.sc;
  long long lo, hi;
  chunk_of(n, lo, hi);
  unsigned g = 0, e = 0;
  for (long long j = lo + threadIdx.x; j < hi; j += blockDim.x) {
    bool gt, eq;
    keep_kind(key_of(lw[j]), s, gt, eq);
    g += gt;
    e += eq;
  }
  if (g) atomicAdd(&cg, g);
  if (e) atomicAdd(&ce, e);
  __syncthreads();
  if (threadIdx.x == 0) {
    p.blk_gt[blockIdx.x] = cg;
    p.blk_eq[blockIdx.x] = ce;
  }
}

// exclusive offsets of the per-block counts (one block), total kept
__global__ void sel_offsets(int nblk, int h_max, int* n_out, unsigned char* base) {
  __shared__ unsigned long long carry;
  Ptrs p = ptrs_of(base);
  if (threadIdx.x == 0) carry = 0;
  __syncthreads();
  for (int b0 = 0; b0 < nblk; b0 += blockDim.x) {
    const int b = b0 + threadIdx.x;
    unsigned long long v = b < nblk ? ((unsigned long long)p.blk_eq[b] << 32) | p.blk_gt[b] : 0ULL;
    // block inclusive scan of packed (eq, gt) counts
    __shared__ unsigned long long ws[32];
    unsigned long long x = v;
    const int lane = threadIdx.x & 31, wp = threadIdx.x >> 5;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const unsigned long long y = __shfl_up_sync(0xFFFFFFFFu, x, o);
      if (lane >= o) x += y;
    }
    if (lane == 31) ws[wp] = x;
    __syncthreads();
    if (wp == 0) {
      unsigned long long s = lane < (int)((blockDim.x + 31) >> 5) ? ws[lane] : 0ULL;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const unsigned long long y = __shfl_up_sync(0xFFFFFFFFu, s, o);
        if (lane >= o) s += y;
      }
      ws[lane] = s;
    }
    __syncthreads();
    const unsigned long long excl = carry + (wp > 0 ? ws[wp - 1] : 0ULL) + x - v;
    if (b < nblk) {
      p.blk_gt[b] = (unsigned)(excl & 0xFFFFFFFFULL);
      p.blk_eq[b] = (unsigned)(excl >> 32);
    }
    __syncthreads();
    if (threadIdx.x == 0) carry += ws[((blockDim.x + 31) >> 5) - 1];
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    const long long gt = (long long)(carry & 0xFFFFFFFFULL), eq = (long long)(carry >> 32);
    long long kept = p.sc->mode == 2 ? 0 : gt + (eq < p.sc->need ? eq : p.sc->need);
    if (kept > h_max) kept = h_max;
    p.sc->n_kept = kept;
    *n_out = (int)kept;
  }
}

// kept children in index order; log-weights normalised over all children
__global__ void sel_write(const double* __restrict__ lw, long long n, int h_max, long long* idx_out,
                          double* lw_out, unsigned char* base) {
  __shared__ unsigned wg[kThreads / 32], we[kThreads / 32];
  __shared__ unsigned run_g, run_e;
  Ptrs p = ptrs_of(base);
  const SelScal s = *p.sc;
  long long lo, hi;
  chunk_of(n, lo, hi);
  if (threadIdx.x == 0) {
    run_g = p.blk_gt[blockIdx.x];
    run_e = p.blk_eq[blockIdx.x];
  }
  __syncthreads();
  const int lane = threadIdx.x & 31, wp = threadIdx.x >> 5;
  for (long long base_j = lo; base_j < hi; base_j += blockDim.x) {
    const long long j = base_j + threadIdx.x;
    bool gt = false, eq = false;
    long long k = kKeyInvalid;
    if (j < hi) {
      k = key_of(lw[j]);
      keep_kind(k, s, gt, eq);
    }
    const unsigned bg = __ballot_sync(0xFFFFFFFFu, gt), be = __ballot_sync(0xFFFFFFFFu, eq);
    if (lane == 0) { wg[wp] = __popc(bg); we[wp] = __popc(be); }
    __syncthreads();
    unsigned og = run_g, oe = run_e;
    for (int w = 0; w < wp; ++w) { og += wg[w]; oe += we[w]; }
    og += __popc(bg & ((1u << lane) - 1u));
    oe += __popc(be & ((1u << lane) - 1u));
    if (gt || (eq && (long long)oe < s.need)) {
      const long long pos = (long long)og + ((long long)oe < s.need ? (long long)oe : s.need);
      if (pos < h_max) {
        idx_out[pos] = j;
        lw_out[pos] = (double)k * kFxInv - s.lse;
      }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      for (int w = 0; w < (int)(blockDim.x >> 5); ++w) { run_g += wg[w]; run_e += we[w]; }
    }
    __syncthreads();
  }
}

// renormalise the kept log-weights (one block)
__global__ void sel_renorm(double* lw_out, unsigned char* base) {
  __shared__ double red[32];
  __shared__ double s_m, s_l;
  Ptrs p = ptrs_of(base);
  const long long n = p.sc->n_kept;
  double m = -INFINITY;
  for (long long j = threadIdx.x; j < n; j += blockDim.x) m = fmax(m, lw_out[j]);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xFFFFFFFFu, m, o));
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = m;
  __syncthreads();
  if (threadIdx.x == 0) {
    double g = -INFINITY;
    for (int w = 0; w < (int)((blockDim.x + 31) >> 5); ++w) g = fmax(g, red[w]);
    s_m = g;
  }
  __syncthreads();
  double sum = 0.0;
  for (long long j = threadIdx.x; j < n; j += blockDim.x) sum += exp(lw_out[j] - s_m);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) sum += __shfl_xor_sync(0xFFFFFFFFu, sum, o);
  __syncthreads();
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = sum;
  __syncthreads();
  if (threadIdx.x == 0) {
    double S = 0.0;
    for (int w = 0; w < (int)((blockDim.x + 31) >> 5); ++w) S += red[w];
    s_l = s_m + log(S);
  }
  __syncthreads();
  for (long long j = threadIdx.x; j < n; j += blockDim.x) lw_out[j] -= s_l;
}

// device address of the scratch array, looked up once per device
std::mutex g_setup_mutex;
unsigned char* g_scratch_ptr[128] = {};

glmb_status scratch_for_current_device(unsigned char** out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 128) return GLMB_E_CUDA;
  std::lock_guard<std::mutex> lock(g_setup_mutex);
  if (!g_scratch_ptr[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_select_scratch) != cudaSuccess || !p) return GLMB_E_CUDA;
    g_scratch_ptr[dev] = (unsigned char*)p;
  }
  *out = g_scratch_ptr[dev];
  return GLMB_OK;
}

}  // namespace

extern "C" glmb_status glmb_select_top_static(const double* logw_dev, int64_t n, int32_t h_max,
                                              double tau, int64_t* idx_out_dev, double* logw_out_dev,
                                              int32_t* n_out_dev, void* stream) {
  if (n < 0 || h_max < 1 || !(tau > 0.0) || !n_out_dev || (n > 0 && (!logw_dev || !idx_out_dev ||
                                                                      !logw_out_dev)))
    return GLMB_E_INVALID;
  if (n > kMaxN || h_max > (1 << 30)) return GLMB_E_CAPACITY;
  unsigned char* base = nullptr;
  const glmb_status st = scratch_for_current_device(&base);
  if (st != GLMB_OK) return st;
  cudaStream_t s = (cudaStream_t)stream;
  const int nblk = (int)(n == 0 ? 1 : std::min<long long>((n + kThreads - 1) / kThreads, kMaxBlocks));
  const double log_tau = std::log(tau);
  const double vmax = std::max(1.0, -log_tau) * 4294967296.0 + 2.0;
  const int nbits = std::max(1, (int)std::ceil(std::log2(vmax)));
  const int passes = (nbits + kDigitS - 1) / kDigitS;
  sel_init<<<1, 256, 0, s>>>(base, h_max);
  sel_lse<<<nblk, kThreads, 0, s>>>(logw_dev, n, log_tau, base);
  for (int q = 0; q < passes; ++q) {
    const int shift = (passes - 1 - q) * kDigitS;
    sel_hist<<<nblk, kThreads, 0, s>>>(logw_dev, n, shift, base);
    sel_find<<<1, kBinsS / 4, 0, s>>>(shift, q == 0, base);
  }
  sel_count<<<nblk, kThreads, 0, s>>>(logw_dev, n, base);
  sel_offsets<<<1, 1024, 0, s>>>(nblk, h_max, n_out_dev, base);
  sel_write<<<nblk, kThreads, 0, s>>>(logw_dev, n, h_max, (long long*)idx_out_dev, logw_out_dev,
                                      base);
  sel_renorm<<<1, 1024, 0, s>>>(logw_out_dev, base);
  return cudaGetLastError() == cudaSuccess ? GLMB_OK : GLMB_E_CUDA;
}

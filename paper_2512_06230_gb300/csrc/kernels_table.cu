// Prediction, births, and the gated compatibility table of Eq. 2 with the
// posterior death probability (arXiv 2512.06230, Section 3), plus the
// device-wide scans used across the update.
#include <algorithm>
#include <cfloat>

#include "glmb_kernels.h"

namespace glmb {

long long g_launches = 0;

namespace {
WaitTest g_wait_test{0, 0};
}
WaitTest wait_test() { return g_wait_test; }
void set_wait_test(WaitTest w) { g_wait_test = w; }

// ---------------------------------------------------------------------------
// Prediction: m <- F m, P <- F P F^T + Q for the constant-velocity model,
// F = [[I, dt I], [0, I]], from the state table into the working table
// (out of place, so a failed frame leaves the state untouched).  One
// thread per component; the mean's position
// coordinates advance in hi/lo arithmetic.  Survivors carry prior existence
// P_S (their death is sampled in the update).
// ---------------------------------------------------------------------------
__device__ void birth_comp(const Model& md, const CompTable& ct, int c, const double* __restrict__ rec,
                           int b, int frame);

template <int DZ>
__device__ void predict_comp(const Model& md, const CompTable& src, const CompTable& ct, int c);

template <int DZ>
__global__ void predict_kernel(Model md, CompTable src, CompTable ct, const FrameDev* __restrict__ fs,
                               const double* __restrict__ births) {
  pdl_enter();
  const int n = fs->n_comp, nb = fs->nb, frame = fs->frame;
  for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < n + nb; c += gridDim.x * blockDim.x) {
    if (c < n) predict_comp<DZ>(md, src, ct, c);
    else birth_comp(md, ct, c, births + (size_t)(c - n) * kBirthRec, c - n, frame);
  }
}

template <int DZ>
__device__ void predict_comp(const Model& md, const CompTable& src, const CompTable& ct, int c) {
  constexpr int DX = 2 * DZ;
  const size_t cap = ct.cap, scap = src.cap;
#pragma unroll
  for (int a = 0; a < DZ; ++a) {
    float hi = src.mhi[a * scap + c], lo = src.mlo[a * scap + c];
    const float vhi = src.mhi[(DZ + a) * scap + c], vlo = src.mlo[(DZ + a) * scap + c];
    ct.mhi[(DZ + a) * cap + c] = vhi;
    ct.mlo[(DZ + a) * cap + c] = vlo;
    const float p = md.dt * vhi;
    const float perr = fmaf(md.dt, vhi, -p);   // exact product error
    df_add(hi, lo, p);
    df_add(hi, lo, perr + md.dt * vlo);
    ct.mhi[a * cap + c] = hi;
    ct.mlo[a * cap + c] = lo;
  }
  float P[DX][DX];
#pragma unroll
  for (int i = 0; i < DX; ++i)
#pragma unroll
    for (int j = i; j < DX; ++j) {
      const float v = src.cov[(size_t)pidx(DX, i, j) * scap + c];
      P[i][j] = v;
      P[j][i] = v;
    }
  // blocks A (pos,pos), B (pos,vel), C (vel,vel):
  // F P F^T = [[A + dt (B + B^T) + dt^2 C, B + dt C], [B^T + dt C, C]]
  const float dt = md.dt;
  float Pn[DX][DX];
#pragma unroll
  for (int a = 0; a < DZ; ++a)
#pragma unroll
    for (int b = 0; b < DZ; ++b) {
      const float A = P[a][b], B = P[a][DZ + b], Bt = P[DZ + a][b], Cv = P[DZ + a][DZ + b];
      Pn[a][b] = A + dt * (B + Bt) + dt * dt * Cv;
      Pn[a][DZ + b] = B + dt * Cv;
      Pn[DZ + a][b] = Bt + dt * Cv;
      Pn[DZ + a][DZ + b] = Cv;
    }
#pragma unroll
  for (int i = 0; i < DX; ++i)
#pragma unroll
    for (int j = i; j < DX; ++j) {
      const int k = pidx(DX, i, j);
      ct.cov[(size_t)k * cap + c] = 0.5f * (Pn[i][j] + Pn[j][i]) + md.Q[k];
    }
  ct.lk[c] = src.lk[c];
  ct.lb[c] = src.lb[c];
  ct.logp[c] = md.log_ps;
  ct.log1mp[c] = md.log_1mps;
}

// LMB births: component c gets birth b's density, existence r and label
// (frame, b).  rec = [r, mean[6], cov[36]] (FP64).
__device__ void birth_comp(const Model& md, const CompTable& ct, int c, const double* __restrict__ rec,
                           int b, int frame) {
  const size_t cap = ct.cap;
  const double r = rec[0];
  const int dx = md.dx;
  for (int a = 0; a < dx; ++a) {
    const double m = rec[1 + a];
    const float hi = (float)m;
    ct.mhi[a * cap + c] = hi;
    ct.mlo[a * cap + c] = (float)(m - (double)hi);
  }
  for (int i = 0; i < dx; ++i)
    for (int j = i; j < dx; ++j)
      ct.cov[(size_t)pidx(dx, i, j) * cap + c] =
          (float)(0.5 * (rec[7 + i * dx + j] + rec[7 + j * dx + i]));
  ct.lk[c] = (uint32_t)frame;
  ct.lb[c] = (uint32_t)b;
  ct.logp[c] = r > 0.0 ? (float)log(r) : -INFINITY;
  ct.log1mp[c] = r < 1.0 ? (float)log1p(-r) : -INFINITY;
}

void launch_predict(const Model& md, const CompTable& src, const CompTable& dst, const FrameDev* fs,
                    const double* births_dev, int grid, cudaStream_t s) {
  if (md.dz == 2) {
    launch_k(predict_kernel<2>, grid, 128, 0, s, md, src, dst, fs, births_dev);
  } else {
    launch_k(predict_kernel<3>, grid, 128, 0, s, md, src, dst, fs, births_dev);
  }
}

// ---------------------------------------------------------------------------
// Eq. 2 with the gate: one warp per component, lanes over detections.
// S = H P H^T + R and its Cholesky factor are computed once per component
// (FP64 when a pivot falls below 16 eps trace(S)); each lane forms the
// innovation e = (z - m_hi) - m_lo, d^2 = e^T S^-1 e and the gate d^2 <= G.
// The count pass sizes the CSR; the write pass stores the gated entries in
// detection order (warp ballot compaction) and reduces
//   psi = (1 - P_D) + sum_gated C[i, j] / kappa
// into the death probability d = (1 - p) / ((1 - p) + p psi).
// ---------------------------------------------------------------------------
template <int DZ>
struct CompGeom {
  float mh[DZ], ml[DZ];
  float L[DZ][DZ];
  double Ld[DZ][DZ];
  float logdet;
  bool fp64;
  bool ok;
};

template <int DZ>
__device__ __forceinline__ void comp_geom(const Model& md, const CompTable& ct, int c,
                                          CompGeom<DZ>& g) {
  const size_t cap = ct.cap;
  float S[DZ][DZ];
  load_HPH<DZ>(ct, md.ncov, md.dx, c, S);
#pragma unroll
  for (int a = 0; a < DZ; ++a) {
    g.mh[a] = ct.mhi[a * cap + c];
    g.ml[a] = ct.mlo[a * cap + c];
#pragma unroll
    for (int b = 0; b < DZ; ++b) S[a][b] += md.R[a * DZ + b];
  }
  g.ok = true;
  g.fp64 = !chol_n<float, DZ>(S, g.L, g.logdet, 1.1920929e-7f);
  if (g.fp64) {
    double Sd[DZ][DZ], ld;
#pragma unroll
    for (int a = 0; a < DZ; ++a)
#pragma unroll
      for (int b = 0; b < DZ; ++b) Sd[a][b] = S[a][b];
    g.ok = chol_n<double, DZ>(Sd, g.Ld, ld, 2.220446049250313e-16);
    g.logdet = (float)ld;
  }
}

template <int DZ>
__device__ __forceinline__ bool pair_eval(const Model& md, const CompGeom<DZ>& g,
                                          const float* __restrict__ Z, int i, float (&e)[DZ],
                                          float& d2) {
#pragma unroll
  for (int a = 0; a < DZ; ++a) e[a] = (__ldg(Z + i * DZ + a) - g.mh[a]) - g.ml[a];
  if (!g.fp64) {
    d2 = mahal_n<float, DZ>(g.L, e);
  } else {
    double ed[DZ];
#pragma unroll
    for (int a = 0; a < DZ; ++a) ed[a] = e[a];
    d2 = (float)mahal_n<double, DZ>(g.Ld, ed);
  }
  return d2 <= md.gate;
}

template <int DZ>
__global__ void table_count_kernel(Model md, CompTable ct, PairTable pt, const FrameDev* __restrict__ fs,
                                   unsigned* err) {
  pdl_enter();
  const int T = fs->T, M = fs->M;
  const float* __restrict__ Z = fs->Z;
  // detections are read with global-memory loads: an address outside
  // global memory rejects the frame instead of being loaded
  if (M > 0 && !__isGlobal(Z)) {
    if (blockIdx.x == 0 && threadIdx.x == 0) atomicOr(err, kErrInput);
    return;
  }
  {
    // every detection coordinate finite, else the frame is rejected
    bool bad = false;
    for (long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x; k < (long long)M * DZ;
         k += (long long)gridDim.x * blockDim.x)
      bad |= !isfinite(Z[k]);
    if (__any_sync(0xFFFFFFFFu, bad) && (threadIdx.x & 31) == 0) atomicOr(err, kErrInput);
  }
  const int lane = threadIdx.x & 31;
  const int nwarps = (gridDim.x * blockDim.x) >> 5;
  for (int c = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; c < T; c += nwarps) {
  CompGeom<DZ> g;
  comp_geom<DZ>(md, ct, c, g);
  unsigned cnt = 0;
  if (g.ok) {
    for (int i0 = 0; i0 < M; i0 += 32) {
      const int i = i0 + lane;
      bool gated = false;
      if (i < M) {
        float e[DZ], d2;
        gated = pair_eval<DZ>(md, g, Z, i, e, d2);
      }
      cnt += __popc(__ballot_sync(0xFFFFFFFFu, gated));
    }
  }
  if (lane == 0) pt.cnt[c] = cnt;
  // the m-only parts of the component's alive term, m = lane + 1
  if (md.score_mode == 0 && (uint32_t)c < (uint32_t)pt.slm_cap && lane < kSlmM) {
    constexpr int NP = DZ * (DZ + 1) / 2;
    float HPH[DZ][DZ];
#pragma unroll
    for (int x = 0; x < DZ; ++x)
#pragma unroll
      for (int y = x; y < DZ; ++y) {
        const float v = ct.cov[(size_t)pidx(md.dx, x, y) * ct.cap + c];
        HPH[x][y] = v;
        HPH[y][x] = v;
      }
    const SlotM<DZ> sm = make_slot_m<DZ>(md, HPH, ct.logp[c], lane + 1);
    const size_t cap = (size_t)pt.slm_cap;
#pragma unroll
    for (int k = 0; k < NP; ++k) pt.slm[((size_t)lane * (NP + 1) + k) * cap + c] = sm.Sinv[k];
    pt.slm[((size_t)lane * (NP + 1) + NP) * cap + c] = sm.c;
    pt.sln[(size_t)lane * cap + c] = (int8_t)sm.ninf;
  }
  }
}

template <int DZ>
__device__ void table_write_comp(const Model& md, const CompTable& ct, const PairTable& pt, int c,
                                 const float* __restrict__ Z, int M, unsigned* n_fp64,
                                 unsigned* err);

template <int DZ>
__global__ void table_write_kernel(Model md, CompTable ct, PairTable pt, const FrameDev* __restrict__ fs,
                                   unsigned* n_fp64, unsigned* err) {
  pdl_enter();
  const int T = fs->T, M = fs->M;
  const float* __restrict__ Z = fs->Z;
  if (M > 0 && !__isGlobal(Z)) return;   // flagged by the count kernel
  const int nwarps = (gridDim.x * blockDim.x) >> 5;
  for (int c = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; c < T; c += nwarps)
    table_write_comp<DZ>(md, ct, pt, c, Z, M, n_fp64, err);
}

template <int DZ>
__device__ void table_write_comp(const Model& md, const CompTable& ct, const PairTable& pt, int c,
                                 const float* __restrict__ Z, int M, unsigned* n_fp64,
                                 unsigned* err) {
  const int lane = threadIdx.x & 31;
  CompGeom<DZ> g;
  comp_geom<DZ>(md, ct, c, g);
  if (!g.ok) {
    if (lane == 0) {
      atomicOr(err, kErrNumeric);
      pt.dthr[c] = kOne24;
      pt.dprob[c] = 1.f;
      pt.logdetS[c] = NAN;
    }
    return;
  }
  if (lane == 0 && g.fp64) atomicAdd(n_fp64, 1u);
  const unsigned base = pt.ptr[c];
  const size_t capp = (size_t)pt.cap_pairs;
  unsigned off = 0;
  float lm = -INFINITY, ls = 0.f;     // per-lane LSE of log C - log kappa
  bool any = false;
  const float c0 = md.log_pd - 0.5f * (g.logdet + (float)DZ * kLog2Pi);
  for (int i0 = 0; i0 < M; i0 += 32) {
    const int i = i0 + lane;
    bool gated = false;
    float e[DZ], d2 = 0.f;
    if (i < M) gated = pair_eval<DZ>(md, g, Z, i, e, d2);
    const unsigned bal = __ballot_sync(0xFFFFFFFFu, gated);
    if (gated) {
      const unsigned pos = base + off + __popc(bal & ((1u << lane) - 1u));
      if (pos < capp) {
        const float logC = c0 - 0.5f * d2;
        float q = 0.f;
#pragma unroll
        for (int a = 0; a < DZ; ++a)
#pragma unroll
          for (int b = 0; b < DZ; ++b) q += e[a] * md.Rinv[a * DZ + b] * e[b];
        pt.meas[pos] = (uint32_t)i;
        pt.logC[pos] = logC;
        pt.q[pos] = q;
#pragma unroll
        for (int a = 0; a < DZ; ++a) pt.e[a * capp + pos] = e[a];
        any = true;
        if (!md.kappa_zero) lse_push(lm, ls, logC - md.log_kappa);
      } else {
        atomicOr(err, kErrPairs);
      }
    }
    off += __popc(bal);
  }
  lse_warp(lm, ls);
  const bool any_w = __any_sync(0xFFFFFFFFu, any);
  if (lane == 0) {
    death_prob(md, ct.logp[c], ct.log1mp[c], lm, ls, any_w, pt.dprob[c], pt.dthr[c]);
    pt.logdetS[c] = g.logdet;
  }
}

void launch_table_count(const Model& md, const CompTable& ct, const PairTable& pt,
                        const FrameDev* fs, unsigned* err, int grid, cudaStream_t s) {
  if (md.dz == 2) { launch_k(table_count_kernel<2>, grid, 256, 0, s, md, ct, pt, fs, err); }
  else { launch_k(table_count_kernel<3>, grid, 256, 0, s, md, ct, pt, fs, err); }
}

void launch_table_write(const Model& md, const CompTable& ct, const PairTable& pt,
                        const FrameDev* fs, unsigned* n_fp64, unsigned* err, int grid, cudaStream_t s) {
  if (md.dz == 2) { launch_k(table_write_kernel<2>, grid, 256, 0, s, md, ct, pt, fs, n_fp64, err); }
  else { launch_k(table_write_kernel<3>, grid, 256, 0, s, md, ct, pt, fs, n_fp64, err); }
}


// per-parent slot and table sizes (max over parents), births included
__global__ void parent_stats_kernel(HypTable hp, const FrameDev* __restrict__ fs, PairTable pt,
                                    unsigned* max_T, unsigned* max_K) {
  pdl_enter();
  __shared__ unsigned kb;
  const int H = fs->H, nb = fs->nb, birth_base = fs->n_comp;
  if (threadIdx.x == 0) {
    unsigned s = 0;
    for (int b = 0; b < nb; ++b) s += pt.cnt[birth_base + b];
    kb = s;
  }
  __syncthreads();
  for (int h = blockIdx.x * blockDim.x + threadIdx.x; h < H; h += gridDim.x * blockDim.x) {
    const unsigned lo = hp.ptr[h], hi = hp.ptr[h + 1];
    unsigned k = kb;
    for (unsigned j = lo; j < hi; ++j) k += pt.cnt[hp.comp[j]];
    atomicMax(max_T, hi - lo + (unsigned)nb);
    atomicMax(max_K, k);
  }
}

void launch_parent_stats(const HypTable& hp, const FrameDev* fs, const PairTable& pt,
                         unsigned* max_T, unsigned* max_K, int grid, cudaStream_t s) {
  launch_k(parent_stats_kernel, grid, 128, 0, s, hp, fs, pt, max_T, max_K);
}

// ---------------------------------------------------------------------------
// Exclusive scan: tiles of 2048 elements (256 threads x 8), tile sums scanned
// by one block, then applied.
// ---------------------------------------------------------------------------
constexpr int kScanThreads = 256, kScanItems = 8, kScanTile = kScanThreads * kScanItems;

template <typename T>
__device__ __forceinline__ T block_exclusive_scan(T v, T& total) {
  __shared__ T warp_sums[kScanThreads / 32];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  T x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const T y = __shfl_up_sync(0xFFFFFFFFu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) warp_sums[w] = x;
  __syncthreads();
  if (w == 0) {
    T s = lane < kScanThreads / 32 ? warp_sums[lane] : T(0);
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const T y = __shfl_up_sync(0xFFFFFFFFu, s, o);
      if (lane >= o) s += y;
    }
    if (lane < kScanThreads / 32) warp_sums[lane] = s;
  }
  __syncthreads();
  const T before = (w > 0 ? warp_sums[w - 1] : T(0)) + x - v;
  total = warp_sums[kScanThreads / 32 - 1];
  __syncthreads();
  return before;
}

// length of a scan: count in device memory times a constant factor
__device__ __forceinline__ long long scan_len(const int* n_dev, int mult) {
  return (long long)(*n_dev) * mult;
}

// Single-pass scan with decoupled look-back (Merrill and Garland, "Single-pass
// parallel prefix scan with decoupled look-back", 2016): blocks take tiles in
// the order they start (an atomic counter), publish their tile's sum, and
// add up their predecessors' published sums back to the nearest published
// inclusive prefix.  A tile waits only on tiles taken before it, by blocks
// already running.  The grid is persistent (at most the blocks the GPU holds
// at once): a block takes tiles until none is left, so that a scan sized for
// a large capacity but short at run time costs no idle blocks.  Work area
// (elements of T), laid out for the largest scan it serves (nw tiles):
// counters [2], status [nw], aggregates [nw], inclusive prefixes [nw];
// counters and status are zero before the first use and left zero by the
// last block to finish.
constexpr unsigned kStAgg = 1u, kStInc = 2u;

template <typename T>
__global__ void scan_onepass(const T* in, T* out, const int* n_dev, int mult, T* total, int total_at_end,
                             T* work, int nw, int nt, unsigned* err, long long spin_limit, int withhold_first) {
  pdl_enter();
  __shared__ int s_tile;
  __shared__ T s_excl;
  T* ctr = work;
  T* st = work + 2;
  T* agg = work + 2 + nw;
  T* inc = work + 2 + 2 * nw;
  const long long n = scan_len(n_dev, mult);
  const int ntiles = (int)min((long long)nt, (n + kScanTile - 1) / kScanTile);
  for (;;) {
    if (threadIdx.x == 0) s_tile = (int)atomicAdd(&ctr[0], T(1));
    __syncthreads();
    const int tile = s_tile;
    __syncthreads();   // s_tile is read by all before the next take
    if (tile >= ntiles) {
      if (tile == 0 && threadIdx.x == 0) {   // empty input
        if (total) *total = 0;
        if (total_at_end) out[n] = 0;
      }
      break;
    }
    const long long base = (long long)tile * kScanTile + (long long)threadIdx.x * kScanItems;
    T vals[kScanItems];
    T sum = 0;
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
      vals[k] = base + k < n ? in[base + k] : T(0);
      sum += vals[k];
    }
    T tile_sum;
    T run = block_exclusive_scan<T>(sum, tile_sum);
    // warp 0 publishes the tile's sum and looks back 32 predecessors at a
    // time: it adds published sums until it meets a published prefix
    if (threadIdx.x < 32) {
      const int lane = threadIdx.x;
      T excl = 0;
      if (tile > 0) {
        if (lane == 0) {
          ((volatile T*)agg)[tile] = tile_sum;
          __threadfence();
          ((volatile T*)st)[tile] = (T)kStAgg;
        }
        int top = tile - 1;   // highest predecessor not yet added
        bool done = false, gave_up = false;
        while (!done && top >= 0) {
          const int p = top - lane;
          T f = p >= 0 ? ((volatile T*)st)[p] : (T)kStInc;
          long long spin = 0;
          while (__any_sync(0xFFFFFFFFu, f == 0) && ++spin < spin_limit)
            if (f == 0) f = ((volatile T*)st)[p];
          if (__any_sync(0xFFFFFFFFu, f == 0)) {   // a predecessor never published
            gave_up = true;
            break;
          }
          __threadfence();
          // the nearest predecessor with a published prefix (lowest lane)
          const unsigned inc_mask = __ballot_sync(0xFFFFFFFFu, p >= 0 && f == (T)kStInc);
          const int stop = inc_mask ? __ffs(inc_mask) - 1 : 31;
          T v = 0;
          if (p >= 0 && lane <= stop)
            v = (lane == stop && f == (T)kStInc) ? ((volatile T*)inc)[p] : ((volatile T*)agg)[p];
#pragma unroll
          for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xFFFFFFFFu, v, o);
          excl += v;
          done = inc_mask != 0u;
          top -= 32;
        }
        if (gave_up && lane == 0) atomicOr(err, kErrTimeout);
      }
      if (lane == 0) {
        ((volatile T*)inc)[tile] = excl + tile_sum;
        __threadfence();
        // (a failure-detection test withholds the first tile's prefix, so
        // that the later tiles' bounded waits run out)
        if (!(withhold_first && tile == 0)) ((volatile T*)st)[tile] = (T)kStInc;
        s_excl = excl;
        if (tile == ntiles - 1) {
          if (total) *total = excl + tile_sum;
          if (total_at_end) out[n] = excl + tile_sum;
        }
      }
    }
    __syncthreads();
    run += s_excl;
#pragma unroll
    for (int k = 0; k < kScanItems; ++k)
      if (base + k < n) {
        out[base + k] = run;
        run += vals[k];
      }
  }
  // the last block to finish clears the work area for the next scan
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    if (atomicAdd(&ctr[1], T(1)) == (T)(gridDim.x - 1)) {
      for (int t = 0; t < ntiles; ++t) st[t] = 0;
      ctr[0] = 0;
      ctr[1] = 0;
      __threadfence();
    }
  }
}

// whole scan in one block when the capacity is small (up to 64 items per thread)
constexpr long long kScanSmall = (long long)kScanThreads * 64;
template <typename T>
__global__ void scan_small(const T* in, T* out, const int* n_dev, int mult, T* total,
                           int total_at_end) {
  pdl_enter();
  const long long n = scan_len(n_dev, mult);
  const int per = (int)((n + kScanThreads - 1) / kScanThreads);
  const long long b = (long long)threadIdx.x * per;
  T s = 0;
  for (int k = 0; k < per; ++k)
    if (b + k < n) s += in[b + k];
  T tot;
  T run = block_exclusive_scan<T>(s, tot);
  for (int k = 0; k < per; ++k)
    if (b + k < n) {
      const T v = in[b + k];
      out[b + k] = run;
      run += v;
    }
  __syncthreads();
  if (threadIdx.x == 0) {
    if (total) *total = tot;
    if (total_at_end) out[n] = tot;
  }
}

static int scan_tiles(long long cap) { return (int)((cap + kScanTile - 1) / kScanTile + 1); }

// blocks of scan_onepass the GPU holds at once (the persistent grid)
template <typename T>
static int scan_resident_blocks() {
  static const int n = [] {
    int dev = 0, sms = 1, per = 1;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, scan_onepass<T>, kScanThreads, 0);
    return std::max(1, sms) * std::max(1, per);
  }();
  return n;
}
long long scan_tmp_elems(long long cap) { return 3LL * scan_tiles(cap) + 2; }

template <typename T>
static void scan_impl(const T* in, T* out, const int* n_dev, int mult, long long cap, T* total,
                      bool total_at_end, T* tmp, long long tmp_cap, unsigned* err, cudaStream_t s) {
  if (cap <= kScanSmall) {
    launch_k(scan_small<T>, 1, kScanThreads, 0, s, in, out, n_dev, mult, total, total_at_end ? 1 : 0);
    return;
  }
  const int nt = scan_tiles(cap), nw = scan_tiles(tmp_cap);
  if (nt > nw) {   // work area smaller than this capacity (a caller error): flag, no scan
    cudaMemsetAsync(err, (int)kErrNumeric, 1, s);
    return;
  }
  const WaitTest wt = wait_test();
  const bool test = wt.mode == kWaitTestScan;
  launch_k(scan_onepass<T>, std::min(nt, scan_resident_blocks<T>()), kScanThreads, 0, s, in, out, n_dev, mult,
           total, total_at_end ? 1 : 0, tmp, nw, nt, err, test ? wt.limit : kScanSpinLimit, test ? 1 : 0);
}

void scan_u32(const uint32_t* in, uint32_t* out, const int* n_dev, int mult, long long cap,
              uint32_t* total, bool total_at_end, uint32_t* tmp, long long tmp_cap, unsigned* err,
              cudaStream_t s) {
  scan_impl<uint32_t>(in, out, n_dev, mult, cap, total, total_at_end, tmp, tmp_cap, err, s);
}
void scan_u64(const unsigned long long* in, unsigned long long* out, const int* n_dev, int mult,
              long long cap, unsigned long long* total, bool total_at_end,
              unsigned long long* tmp, long long tmp_cap, unsigned* err, cudaStream_t s) {
  scan_impl<unsigned long long>(in, out, n_dev, mult, cap, total, total_at_end, tmp, tmp_cap, err, s);
}

}  // namespace glmb

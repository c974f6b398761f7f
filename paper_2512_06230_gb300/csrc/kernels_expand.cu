// Child expansion, scoring and per-parent deduplication (arXiv 2512.06230,
// Section 3: two-stage sampling of H_up children per hypothesis, weight =
// parent weight x joint likelihood of the sampled deaths and associations,
// retention of unique children), and the regeneration of the retained
// children for the batched track update.
//
// One CTA per parent hypothesis.  The CTA stages the parent's gated pairs in
// shared memory re-indexed by detection row (slots ascending within a row),
// with per-row integer thresholds of the categorical draw under "all slots
// alive", and a reference association (each row's most likely option) whose
// exact score is computed once.  Each warp then draws children:
//   phase 1  Philox words for the slots that can die; dead slots are marked;
//   phase 2  one Philox word per detection row; the row's option is the first
//            whose threshold exceeds the 24-bit uniform (rows with a dead
//            candidate fall back to the FP32 normalised row of C'_k); rows
//            that leave the reference move fixed-point sums (count, sum of
//            innovations, sum of e^T R^-1 e) between slots;
//   phase 3  only the touched slots are rescored; the child's log-weight is
//            the reference score plus the exact integer change.
// The duplicate test keys a child by the order-free sum of mix64 keys of its
// deviations and deaths.
#include "glmb_kernels.h"

namespace glmb {

struct Lay {
  int scal;
  int comp, dthr, logp, log1mp, mref, seref, sqref, termref, ninfref, hwref, refnew;
  int rowoff, rowfill, rowref, rowflag, rowthr0, roww0;
  int cslot, cthr, ceidx, cw, ce, cq, hph;
  int dpc;
  int redo;
  int grp, grp_bytes;
  int g_cnt, g_se, g_sq, g_hw, g_newval, g_tmask, g_dmask, g_dpre, g_tlist, g_nt;
  int total;
};

struct Bump {
  int off = 0;
  __host__ __device__ int take(long long bytes) {
    const int o = off;
    off += (int)((bytes + 15) & ~15LL);
    return o;
  }
};

struct Scal {
  long long ref_score;
  unsigned long long uid;
  double logw;
  int ninf_ref, nclut_ref, T, Town, K, ndpc, s_lo, s_hi, bad, nredo;
};

__host__ __device__ inline Lay make_lay(int dz, int mat, int T, int K, int M, int HU, int G) {
  Lay L;
  Bump b;
  const int W = (T + 31) / 32 + 1;
  L.scal = b.take(sizeof(Scal));
  L.seref = b.take(8LL * dz * T);
  L.sqref = b.take(8LL * T);
  L.termref = b.take(8LL * T);
  L.hwref = mat ? b.take(8LL * T) : 0;
  L.comp = b.take(4LL * T);
  L.dthr = b.take(4LL * T);
  L.logp = b.take(4LL * T);
  L.log1mp = b.take(4LL * T);
  L.mref = b.take(4LL * T);
  L.refnew = mat ? b.take(4LL * T) : 0;
  L.rowoff = b.take(4LL * (M + 1));
  L.rowfill = b.take(4LL * (M + 1));
  L.rowthr0 = b.take(4LL * M);
  L.roww0 = b.take(4LL * M);
  L.cthr = b.take(4LL * K);
  L.ceidx = b.take(4LL * K);
  L.cw = b.take(4LL * K);
  L.ce = b.take(4LL * dz * K);              // innovation of each candidate pair
  L.cq = b.take(4LL * K);                   // e^T R^-1 e of each candidate pair
  L.hph = b.take(4LL * (dz * (dz + 1) / 2) * T);   // H P H^T of each slot (packed)
  L.dpc = b.take(4LL * (T / 4 + 2));
  L.cslot = b.take(2LL * K);
  L.rowref = b.take(2LL * M);
  L.redo = b.take(2LL * HU);
  L.rowflag = b.take(M);
  L.ninfref = b.take(T);
  L.grp = b.off;
  Bump g;
  L.g_se = g.take(8LL * dz * T);
  L.g_sq = g.take(8LL * T);
  L.g_hw = mat ? g.take(8LL * T) : 0;
  L.g_cnt = g.take(4LL * T);
  L.g_newval = mat ? g.take(4LL * T) : 0;
  L.g_tmask = g.take(4LL * W);
  L.g_dmask = g.take(4LL * W);
  L.g_dpre = g.take(4LL * W);
  L.g_nt = g.take(16);
  L.g_tlist = g.take(2LL * T);
  L.grp_bytes = g.off;
  L.total = L.grp + G * L.grp_bytes;
  return L;
}

int expand_smem_bytes(int dz, int materialize, int T_max, int K_max, int M, int h_up,
                      int n_groups) {
  return make_lay(dz, materialize, T_max, K_max, M, h_up, n_groups).total;
}

int expand_plan_groups(int dz, int materialize, int T_max, int K_max, int M, int h_up,
                       int smem_limit, int max_groups) {
  for (int G = max_groups < 1 ? 1 : (max_groups > 16 ? 16 : max_groups); G >= 1; --G)
    if (expand_smem_bytes(dz, materialize, T_max, K_max, M, h_up, G) <= smem_limit) return G;
  return 0;
}

template <typename T>
__device__ __forceinline__ T* at(unsigned char* base, int off) {
  return reinterpret_cast<T*>(base + off);
}

__device__ __forceinline__ uint32_t thr_of(float frac) {
  // smallest integer k0 with k0 >= frac * 2^24, clamped to [0, 2^24]
  if (!(frac > 0.f)) return 0u;
  if (frac >= 1.f) return kOne24;
  return (uint32_t)ceilf(frac * 16777216.f);
}

__device__ __forceinline__ void touch(uint32_t* tmask, uint16_t* tlist, int* nt, int t) {
  const uint32_t bit = 1u << (t & 31);
  const uint32_t old = atomicOr(&tmask[t >> 5], bit);
  if (!(old & bit)) tlist[atomicAdd(nt, 1)] = (uint16_t)t;
}

template <int DZ>
__device__ __forceinline__ void slot_HPH(const float* s_hph, int T, int t, float (&HPH)[DZ][DZ]) {
  int k = 0;
#pragma unroll
  for (int x = 0; x < DZ; ++x)
#pragma unroll
    for (int y = x; y < DZ; ++y, ++k) {
      const float v = s_hph[k * T + t];
      HPH[x][y] = v;
      HPH[y][x] = v;
    }
}

__device__ __forceinline__ bool bit_of(const uint32_t* m, int t) {
  return (m[t >> 5] >> (t & 31)) & 1u;
}

// insert (component, detection-set key) into the update table; returns the
// tagged hash slot to be resolved to a component index after the kernel
template <int DZ>
__device__ uint32_t upd_insert(const ExpandArgs& a, uint32_t comp, unsigned long long hw, int m,
                               const long long (&se)[DZ]) {
  unsigned long long key = mix64(hw + 0x9E3779B97F4A7C15ULL * ((unsigned long long)comp + 1ULL));
  if (key == 0ULL) key = 1ULL;
  uint32_t slot = (uint32_t)key & a.hmask;
  for (uint32_t probe = 0; probe <= a.hmask; ++probe) {
    const unsigned long long prev = atomicCAS(&a.hkeys[slot], 0ULL, key);
    if (prev == 0ULL) {
      const uint32_t id = atomicAdd(a.upd_count, 1u);
      if (id < (uint32_t)a.cap_upd) {
        a.upd_src[id] = comp;
        a.upd_m[id] = (uint32_t)m;
#pragma unroll
        for (int d = 0; d < DZ; ++d) a.upd_se[(size_t)d * a.cap_upd + id] = se[d];
        a.hvals[slot] = id;
      } else {
        atomicOr(a.err, kErrUpdates);
        a.hvals[slot] = 0u;
      }
      return kNewTag | slot;
    }
    if (prev == key) return kNewTag | slot;
    slot = (slot + 1u) & a.hmask;
  }
  atomicOr(a.err, kErrHash);
  return kNewTag;
}

template <int DZ, bool MAT>
__device__ void expand_parent(const ExpandArgs& a, const int h, const int sl, const int S, const Lay& L,
                              unsigned char* sm);

// Persistent: each CTA takes parents blockIdx.x, blockIdx.x + gridDim.x, ...
template <int DZ, bool MAT>
__global__ void __launch_bounds__(512) expand_kernel(const ExpandArgs a) {
  extern __shared__ __align__(16) unsigned char sm[];
  const Lay L = make_lay(DZ, MAT, a.T_max, a.K_max, a.M_plan, a.md.h_up, a.n_fb_groups);
  const int H = a.fs->H;
  // draws of a parent are split into S slices when parents are too few to
  // fill the GPU (about target_warps warps in flight)
  int S = 1;
  if (!MAT) {
    const long long per = (long long)H * (blockDim.x >> 5);
    S = per > 0 ? (int)min((long long)a.max_slices, (a.target_warps + per - 1) / per) : 1;
    if (S < 1) S = 1;
  }
  for (int job = blockIdx.x; job < H * S; job += gridDim.x) {
    __syncthreads();   // the previous job's shared memory is free
    expand_parent<DZ, MAT>(a, job / S, job % S, S, L, sm);
  }
}

template <int DZ, bool MAT>
__device__ void expand_parent(const ExpandArgs& a, const int h, const int sl, const int S, const Lay& L,
                              unsigned char* sm) {
  const Model& md = a.md;
  const int HU = md.h_up;
  const int M = a.fs->M;
  const int birth_base = a.fs->n_comp, nb = a.fs->nb;
  const uint2 key = make_uint2(md.seed_lo, md.seed_hi ^ (uint32_t)a.fs->frame);
  Scal& sc = *at<Scal>(sm, L.scal);
  uint32_t* s_comp = at<uint32_t>(sm, L.comp);
  uint32_t* s_dthr = at<uint32_t>(sm, L.dthr);
  float* s_logp = at<float>(sm, L.logp);
  float* s_log1mp = at<float>(sm, L.log1mp);
  int* s_mref = at<int>(sm, L.mref);
  long long* s_seref = at<long long>(sm, L.seref);
  long long* s_sqref = at<long long>(sm, L.sqref);
  long long* s_termref = at<long long>(sm, L.termref);
  uint8_t* s_ninfref = at<uint8_t>(sm, L.ninfref);
  unsigned long long* s_hwref = at<unsigned long long>(sm, L.hwref);
  uint32_t* s_refnew = at<uint32_t>(sm, L.refnew);
  uint32_t* s_rowoff = at<uint32_t>(sm, L.rowoff);
  uint32_t* s_rowfill = at<uint32_t>(sm, L.rowfill);
  uint16_t* s_rowref = at<uint16_t>(sm, L.rowref);
  uint8_t* s_rowflag = at<uint8_t>(sm, L.rowflag);
  uint32_t* s_rowthr0 = at<uint32_t>(sm, L.rowthr0);
  float* s_roww0 = at<float>(sm, L.roww0);
  uint16_t* s_cslot = at<uint16_t>(sm, L.cslot);
  uint32_t* s_cthr = at<uint32_t>(sm, L.cthr);
  uint32_t* s_ceidx = at<uint32_t>(sm, L.ceidx);
  float* s_cw = at<float>(sm, L.cw);
  float* s_ce = at<float>(sm, L.ce);
  float* s_cq = at<float>(sm, L.cq);
  float* s_hph = at<float>(sm, L.hph);
  const int Kp = a.K_max;                   // stride of the candidate arrays
  uint32_t* s_dpc = at<uint32_t>(sm, L.dpc);
  const CompTable& ct = a.ct;
  const PairTable& pt = a.pt;
  const size_t capp = (size_t)pt.cap_pairs;
  const int tid = threadIdx.x, nthr = blockDim.x;

  // ---- parent header ----
  if (tid == 0) {
    const uint32_t lo = a.parents.ptr[h], hi = a.parents.ptr[h + 1];
    sc.Town = (int)(hi - lo);
    sc.T = sc.Town + nb;
    sc.ref_score = 0;
    sc.ninf_ref = 0;
    sc.nclut_ref = 0;
    sc.ndpc = 0;
    sc.bad = 0;
    sc.nredo = 0;
    sc.uid = a.parents.uid[h];
    sc.logw = a.parents.logw[h];
    sc.s_lo = sc.s_hi = 0;
    if (MAT) {
      // survivors of this parent: child indices in [h*HU, (h+1)*HU)
      const long long lo_key = (long long)h * HU, hi_key = lo_key + HU;
      const int ns = (int)*a.n_surv;
      int l = 0, r = ns;
      while (l < r) { const int mid = (l + r) >> 1; if (a.surv_idx[mid] < lo_key) l = mid + 1; else r = mid; }
      sc.s_lo = l;
      r = ns;
      while (l < r) { const int mid = (l + r) >> 1; if (a.surv_idx[mid] < hi_key) l = mid + 1; else r = mid; }
      sc.s_hi = l;
    }
    if (sc.T > a.T_max || M > a.M_plan) { sc.bad = 1; atomicOr(a.err, kErrSlots); }
    // a frame already abandoned (e.g. entries beyond capacity) writes nothing
    if (MAT && (*(volatile unsigned*)a.err & (kErrEntries | kErrSlots | kErrPairs))) sc.bad = 1;
  }
  __syncthreads();
  if (sc.bad) return;
  if (MAT && sc.s_lo == sc.s_hi) return;
  const int T = sc.T, Town = sc.Town;
  const uint32_t plo = a.parents.ptr[h];

  // ---- slots ----
  for (int t = tid; t < T; t += nthr) {
    const uint32_t c = t < Town ? a.parents.comp[plo + t] : (uint32_t)(birth_base + (t - Town));
    s_comp[t] = c;
    {
      int k = 0;
#pragma unroll
      for (int x = 0; x < DZ; ++x)
#pragma unroll
        for (int y = x; y < DZ; ++y, ++k) s_hph[k * T + t] = ct.cov[(size_t)pidx(md.dx, x, y) * ct.cap + c];
    }
    s_dthr[t] = pt.dthr[c];
    s_logp[t] = ct.logp[c];
    s_log1mp[t] = ct.log1mp[c];
    s_mref[t] = 0;
#pragma unroll
    for (int d = 0; d < DZ; ++d) s_seref[d * T + t] = 0;
    s_sqref[t] = 0;
    if (MAT) s_hwref[t] = 0;
  }
  for (int i = tid; i <= M; i += nthr) s_rowfill[i] = 0;
  __syncthreads();
  for (int t = tid; t < T; t += nthr) {
    const uint32_t c = s_comp[t];
    for (uint32_t j = pt.ptr[c], je = pt.ptr[c + 1]; j < je; ++j) atomicAdd(&s_rowfill[pt.meas[j]], 1u);
  }
  __syncthreads();
  // exclusive scan of the row counts (single warp, serial carry over chunks)
  if (tid < 32) {
    uint32_t carry = 0;
    for (int base = 0; base < M; base += 32) {
      const int i = base + tid;
      const uint32_t v = i < M ? s_rowfill[i] : 0u;
      uint32_t x = v;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xFFFFFFFFu, x, o);
        if (tid >= o) x += y;
      }
      if (i < M) s_rowoff[i] = carry + x - v;
      carry += __shfl_sync(0xFFFFFFFFu, x, 31);
    }
    if (tid == 0) {
      s_rowoff[M] = carry;
      sc.K = (int)carry;
      if ((int)carry > a.K_max) { sc.bad = 1; atomicOr(a.err, kErrSlots); }
    }
  }
  __syncthreads();
  if (sc.bad) return;
  for (int i = tid; i < M; i += nthr) s_rowfill[i] = 0;
  __syncthreads();
  for (int t = tid; t < T; t += nthr) {
    const uint32_t c = s_comp[t];
    for (uint32_t j = pt.ptr[c], je = pt.ptr[c + 1]; j < je; ++j) {
      const uint32_t i = pt.meas[j];
      const uint32_t pos = s_rowoff[i] + atomicAdd(&s_rowfill[i], 1u);
      s_cslot[pos] = (uint16_t)t;
      s_ceidx[pos] = j;
    }
  }
  __syncthreads();

  // ---- rows: order, weights, thresholds, reference option ----
  {
    int my_clut = 0;
    for (int i = tid; i < M; i += nthr) {
      const uint32_t off = s_rowoff[i];
      const int nc = (int)(s_rowoff[i + 1] - off);
      for (int x = 1; x < nc; ++x) {   // insertion sort by slot
        const uint16_t ks = s_cslot[off + x];
        const uint32_t ke = s_ceidx[off + x];
        int y = x - 1;
        while (y >= 0 && s_cslot[off + y] > ks) {
          s_cslot[off + y + 1] = s_cslot[off + y];
          s_ceidx[off + y + 1] = s_ceidx[off + y];
          --y;
        }
        s_cslot[off + y + 1] = ks;
        s_ceidx[off + y + 1] = ke;
      }
      if (nc == 0) {
        s_rowref[i] = 0;
        s_rowflag[i] = 0;
        s_rowthr0[i] = kOne24;
        s_roww0[i] = 1.f;
        ++my_clut;
        continue;
      }
      float smax = md.kappa_zero ? -INFINITY : md.log_kappa;
      for (int j = 0; j < nc; ++j) {
        const uint32_t ei = s_ceidx[off + j];
        smax = fmaxf(smax, pt.logC[ei]);
#pragma unroll
        for (int d = 0; d < DZ; ++d) s_ce[d * Kp + off + j] = pt.e[d * capp + ei];
        s_cq[off + j] = pt.q[ei];
      }
      const float w0 = md.kappa_zero ? 0.f : expf(md.log_kappa - smax);
      float sum = w0;
      for (int j = 0; j < nc; ++j) {
        const float w = expf(pt.logC[s_ceidx[off + j]] - smax);
        s_cw[off + j] = w;
        sum += w;
      }
      float cum = w0, best = w0;
      int ref = 0;
      bool flag = false;
      s_rowthr0[i] = (nc == 0) ? kOne24 : thr_of(cum / sum);
      for (int j = 0; j < nc; ++j) {
        const float w = s_cw[off + j];
        cum += w;
        s_cthr[off + j] = (j == nc - 1) ? kOne24 : thr_of(cum / sum);
        if (w > best) { best = w; ref = j + 1; }
        flag |= s_dthr[s_cslot[off + j]] > 0u;
      }
      s_rowref[i] = (uint16_t)ref;
      s_rowflag[i] = flag ? 1 : 0;
      s_roww0[i] = w0;
      if (ref == 0) {
        ++my_clut;
      } else {
        const int r = s_cslot[off + ref - 1];
        const uint32_t pos = off + ref - 1;
        atomicAdd(&s_mref[r], 1);
#pragma unroll
        for (int d = 0; d < DZ; ++d)
          atomicAdd((unsigned long long*)&s_seref[d * T + r], (unsigned long long)fx_of(s_ce[d * Kp + pos]));
        atomicAdd((unsigned long long*)&s_sqref[r], (unsigned long long)fx_of(s_cq[pos]));
        if (MAT) atomicAdd(&s_hwref[r], wset_key(i));
      }
    }
    if (my_clut) atomicAdd(&sc.nclut_ref, my_clut);
  }
  __syncthreads();

  // ---- reference terms, death-possible chunks ----
  {
    long long my_term = 0;
    int my_ninf = 0;
    for (int t = tid; t < T; t += nthr) {
      float HPH[DZ][DZ];
      slot_HPH<DZ>(s_hph, T, t, HPH);
      long long se[DZ];
#pragma unroll
      for (int d = 0; d < DZ; ++d) se[d] = s_seref[d * T + t];
      int ninf;
      const long long term = alive_term<DZ>(md, HPH, s_logp[t], s_mref[t], se, s_sqref[t], ninf);
      s_termref[t] = term;
      s_ninfref[t] = (uint8_t)ninf;
      my_term += term;
      my_ninf += ninf;
      if (MAT) {
        s_refnew[t] = s_mref[t] >= 1 ? upd_insert<DZ>(a, s_comp[t], s_hwref[t], s_mref[t], se)
                                     : s_comp[t];
      }
    }
    if (my_term) atomicAdd((unsigned long long*)&sc.ref_score, (unsigned long long)my_term);
    if (my_ninf) atomicAdd(&sc.ninf_ref, my_ninf);
    const int nch = (T + 3) >> 2;
    for (int cc = tid; cc < nch; cc += nthr) {
      uint32_t mask = 0;
#pragma unroll
      for (int b = 0; b < 4; ++b) {
        const int t = 4 * cc + b;
        if (t < T && s_dthr[t] > 0u) mask |= 1u << b;
      }
      if (mask) s_dpc[atomicAdd(&sc.ndpc, 1)] = ((uint32_t)cc << 4) | mask;
    }
  }
  __syncthreads();
  if (tid == 0) {
    sc.ref_score += __double2ll_rn(sc.logw * 4294967296.0);
    if (md.kappa_zero) sc.ninf_ref += sc.nclut_ref;
    else sc.ref_score += (long long)sc.nclut_ref * md.fx_log_kappa;
  }
  __syncthreads();

  // ---- draws, one thread per child ----
  // Every thread walks the same rows (broadcast shared-memory reads) with its
  // own random words, keeps its deaths and deviating rows in short local
  // lists, and rescores only the slots they touch.  Children whose lists
  // overflow (or parents with more than kTwMax * 32 slots) are redone below
  // by one warp each.
  uint16_t* s_redo = at<uint16_t>(sm, L.redo);
  const int chunk = (HU + S - 1) / S;
  const int n_lo = MAT ? 0 : sl * chunk;
  const int n_items = MAT ? (sc.s_hi - sc.s_lo) : max(0, min(HU, n_lo + chunk) - n_lo);
  const uint32_t uid_lo = (uint32_t)sc.uid, uid_hi = (uint32_t)(sc.uid >> 32);
  const int ndpc = sc.ndpc;
  const int nrc = (M + 3) >> 2;
  const long long ref_score = sc.ref_score;
  const int ninf_ref = sc.ninf_ref;
  const int W = (T + 31) >> 5;
  {
    constexpr int kTwMax = 64, kDeadMax = 64, kDevMax = 128, kTouchMax = 2 * kDevMax + kDeadMax;
    for (int it = tid; it < n_items; it += nthr) {
      if (MAT || !a.thread_path || W > kTwMax) {
        s_redo[atomicAdd(&sc.nredo, 1)] = (uint16_t)it;
        continue;
      }
      const int n = MAT ? (int)(a.surv_idx[sc.s_lo + it] - (long long)h * HU) : n_lo + it;
      const int s_out = MAT ? sc.s_lo + it : 0;
      uint32_t deadw[kTwMax];
      uint16_t dl[kDeadMax];
      uint32_t dv[kDevMax];
      for (int w = 0; w < W; ++w) deadw[w] = 0u;
      int nd = 0, ndv = 0, dclut = 0;
      bool over = false, bad_row = false;
      unsigned long long hsh = 0;
      // stage 1: deaths
      for (int x = 0; x < ndpc; ++x) {
        const uint32_t ent = s_dpc[x];
        const uint32_t cc = ent >> 4, mask = ent & 15u;
        const uint4 r = philox10(make_uint4(uid_lo, uid_hi, 2u * (uint32_t)n, cc), key);
#pragma unroll
        for (int b = 0; b < 4; ++b) {
          if (!((mask >> b) & 1u)) continue;
          const int t = 4 * (int)cc + b;
          if ((word_of(r, b) >> 8) < s_dthr[t]) {
            deadw[t >> 5] |= 1u << (t & 31);
            if (nd < kDeadMax) dl[nd] = (uint16_t)t;
            ++nd;
          }
        }
      }
      over |= nd > kDeadMax;
      // dead slots below each 32-slot word (child track index = slot - dead below)
      uint32_t dpw[kTwMax];
      if (MAT) {
        uint32_t run = 0;
        for (int w = 0; w < W; ++w) {
          dpw[w] = run;
          run += __popc(deadw[w]);
        }
      }
      // stage 2: one categorical draw per detection row
      for (int cc = 0; cc < nrc; ++cc) {
        const int i0 = 4 * cc;
        const int i1 = min(i0 + 4, M);
        if (s_rowoff[i1] == s_rowoff[i0]) {
          if (MAT)
            for (int i = i0; i < i1; ++i) a.out_theta[(size_t)s_out * M + i] = 0;
          continue;
        }
        const uint4 r = philox10(make_uint4(uid_lo, uid_hi, 2u * (uint32_t)n + 1u, (uint32_t)cc), key);
#pragma unroll
        for (int b = 0; b < 4; ++b) {
          const int i = i0 + b;
          if (i >= i1) break;
          const uint32_t off = s_rowoff[i];
          const int nc = (int)(s_rowoff[i + 1] - off);
          if (nc == 0) {
            if (MAT) a.out_theta[(size_t)s_out * M + i] = 0;
            continue;
          }
          const uint32_t k = word_of(r, b) >> 8;
          bool fast = true;
          if (s_rowflag[i])
            for (int j = 0; j < nc; ++j) {
              const int t = s_cslot[off + j];
              if ((deadw[t >> 5] >> (t & 31)) & 1u) { fast = false; break; }
            }
          int opt;
          if (fast) {
            if (k < s_rowthr0[i]) {
              opt = 0;
            } else {
              int j = 0;
              while (j < nc - 1 && k >= s_cthr[off + j]) ++j;
              opt = j + 1;
            }
          } else {
            const float w0 = md.kappa_zero ? 0.f : s_roww0[i];
            float sum = w0;
            for (int j = 0; j < nc; ++j) {
              const int t = s_cslot[off + j];
              if (!((deadw[t >> 5] >> (t & 31)) & 1u)) sum += s_cw[off + j];
            }
            if (!(sum > 0.f)) {
              bad_row = true;
              opt = 0;
            } else {
              const float xk = (float)k * 5.9604644775390625e-8f * sum;
              float cum = w0;
              int last = w0 > 0.f ? 0 : -1;
              opt = -1;
              if (w0 > 0.f && xk < cum) opt = 0;
              for (int j = 0; j < nc; ++j) {
                const int t = s_cslot[off + j];
                if ((deadw[t >> 5] >> (t & 31)) & 1u) continue;
                const float w = s_cw[off + j];
                if (!(w > 0.f)) continue;
                cum += w;
                last = j + 1;
                if (opt < 0 && xk < cum) opt = j + 1;
              }
              if (opt < 0) opt = last < 0 ? 0 : last;
            }
          }
          // deviations are rare and differ between lanes: only record them here
          if (opt != s_rowref[i]) {
            if (ndv < kDevMax) dv[ndv] = ((uint32_t)i << 16) | (uint32_t)opt;
            ++ndv;
          }
          if (MAT) {
            const int ns = opt > 0 ? (int)s_cslot[off + opt - 1] : -1;
            uint16_t th = 0;
            if (ns >= 0)
              th = (uint16_t)(ns - (int)(dpw[ns >> 5] + __popc(deadw[ns >> 5] & ((1u << (ns & 31)) - 1u))) + 1);
            a.out_theta[(size_t)s_out * M + i] = th;
          }
        }
      }
      over |= ndv > kDevMax;
      if (over) {
        s_redo[atomicAdd(&sc.nredo, 1)] = (uint16_t)it;
        continue;
      }
      // duplicate-test key and clutter count of the deaths and deviations
      for (int j = 0; j < nd; ++j) hsh += dead_key(dl[j]);
      for (int q = 0; q < ndv; ++q) {
        const int iq = (int)(dv[q] >> 16), oq = (int)(dv[q] & 0xFFFFu);
        const uint32_t offq = s_rowoff[iq];
        const int refq = s_rowref[iq];
        const int nsq = oq > 0 ? (int)s_cslot[offq + oq - 1] : -1;
        const int rsq = refq > 0 ? (int)s_cslot[offq + refq - 1] : -1;
        dclut += (oq == 0) - (refq == 0);
        hsh += row_key(iq, oq > 0 ? nsq + 1 : 0) - row_key(iq, refq > 0 ? rsq + 1 : 0);
      }
      // stage 3: rescore the touched slots (exact fixed-point deltas)
      long long delta = 0;
      int dninf = 0;
      uint16_t tsl[kTouchMax];
      uint32_t tval[MAT ? kTouchMax : 1];
      int ntouch = 0;
      for (int j = 0; j < nd; ++j) {
        const int t = dl[j];
        int ninf;
        const long long term = dead_term(s_log1mp[t], ninf);
        delta += term - s_termref[t];
        dninf += ninf - (int)s_ninfref[t];
        tsl[ntouch++] = (uint16_t)t;
      }
      for (int q = 0; q < ndv; ++q) {
        const int iq = (int)(dv[q] >> 16), oq = (int)(dv[q] & 0xFFFFu);
        const uint32_t offq = s_rowoff[iq];
        const int refq = s_rowref[iq];
#pragma unroll
        for (int side = 0; side < 2; ++side) {
          const int o = side == 0 ? refq : oq;
          if (o <= 0) continue;
          const int t = s_cslot[offq + o - 1];
          if ((deadw[t >> 5] >> (t & 31)) & 1u) continue;
          bool seen = false;
          for (int u = nd; u < ntouch; ++u)
            if (tsl[u] == t) { seen = true; break; }
          if (seen) continue;
          // all deviating rows that leave or join slot t
          int dcnt = 0;
          long long dse[DZ], dsq = 0;
          unsigned long long dhw = 0;
#pragma unroll
          for (int d = 0; d < DZ; ++d) dse[d] = 0;
          for (int q2 = 0; q2 < ndv; ++q2) {
            const int i2 = (int)(dv[q2] >> 16), o2 = (int)(dv[q2] & 0xFFFFu);
            const uint32_t off2 = s_rowoff[i2];
            const int r2 = s_rowref[i2];
            if (r2 > 0 && (int)s_cslot[off2 + r2 - 1] == t) {
              const uint32_t pos = off2 + r2 - 1;
              --dcnt;
#pragma unroll
              for (int d = 0; d < DZ; ++d) dse[d] -= fx_of(s_ce[d * Kp + pos]);
              dsq -= fx_of(s_cq[pos]);
              if (MAT) dhw -= wset_key(i2);
            }
            if (o2 > 0 && (int)s_cslot[off2 + o2 - 1] == t) {
              const uint32_t pos = off2 + o2 - 1;
              ++dcnt;
#pragma unroll
              for (int d = 0; d < DZ; ++d) dse[d] += fx_of(s_ce[d * Kp + pos]);
              dsq += fx_of(s_cq[pos]);
              if (MAT) dhw += wset_key(i2);
            }
          }
          float HPH[DZ][DZ];
          slot_HPH<DZ>(s_hph, T, t, HPH);
          const int m = s_mref[t] + dcnt;
          long long se[DZ];
#pragma unroll
          for (int d = 0; d < DZ; ++d) se[d] = s_seref[d * T + t] + dse[d];
          int ninf;
          const long long term = alive_term<DZ>(md, HPH, s_logp[t], m, se, s_sqref[t] + dsq, ninf);
          delta += term - s_termref[t];
          dninf += ninf - (int)s_ninfref[t];
          if (MAT) tval[ntouch] = m >= 1 ? upd_insert<DZ>(a, s_comp[t], s_hwref[t] + dhw, m, se) : s_comp[t];
          tsl[ntouch++] = (uint16_t)t;
        }
      }
      if (MAT) {
        // the child's track list: alive slots in slot order
        const uint32_t base = a.out_ptr[s_out];
        for (int t = 0; t < T; ++t) {
          if ((deadw[t >> 5] >> (t & 31)) & 1u) continue;
          uint32_t v = s_refnew[t];
          for (int u = nd; u < ntouch; ++u)
            if (tsl[u] == t) { v = tval[u]; break; }
          a.out_comp[base + (uint32_t)t - (dpw[t >> 5] + __popc(deadw[t >> 5] & ((1u << (t & 31)) - 1u)))] = v;
        }
      } else {
        const long long score = ref_score + delta + (md.kappa_zero ? 0LL : (long long)dclut * md.fx_log_kappa);
        const int ninf = ninf_ref + dninf + (md.kappa_zero ? dclut : 0);
        const bool valid = !bad_row && ninf == 0;
        const size_t j = (size_t)h * HU + n;
        a.child_key[j] = valid ? score : kKeyInvalid;
        a.child_hash[j] = hsh;
        a.child_status[j] = valid ? 1 : 0;
        a.child_alive[j] = (uint16_t)(T - nd);
      }
    }
  }
  __syncthreads();
  const int n_redo = sc.nredo;

  // ---- redone children: one warp per child ----
  const int g = tid >> 5, lane = tid & 31;
  unsigned char* gb = sm + L.grp + g * L.grp_bytes;
  int* acc_cnt = at<int>(gb, L.g_cnt);
  long long* acc_se = at<long long>(gb, L.g_se);
  long long* acc_sq = at<long long>(gb, L.g_sq);
  unsigned long long* acc_hw = at<unsigned long long>(gb, L.g_hw);
  uint32_t* newval = at<uint32_t>(gb, L.g_newval);
  uint32_t* tmask = at<uint32_t>(gb, L.g_tmask);
  uint32_t* dmask = at<uint32_t>(gb, L.g_dmask);
  uint32_t* dpre = at<uint32_t>(gb, L.g_dpre);
  uint16_t* tlist = at<uint16_t>(gb, L.g_tlist);
  int* ntp = at<int>(gb, L.g_nt);
  for (int t = lane; g < a.n_fb_groups && t < T; t += 32) {
    acc_cnt[t] = 0;
#pragma unroll
    for (int d = 0; d < DZ; ++d) acc_se[d * T + t] = 0;
    acc_sq[t] = 0;
    if (MAT) acc_hw[t] = 0;
  }
  for (int w = lane; g < a.n_fb_groups && w < W; w += 32) { tmask[w] = 0; dmask[w] = 0; }
  if (lane == 0 && g < a.n_fb_groups) *ntp = 0;
  __syncwarp();

  for (int rr = g; g < a.n_fb_groups && rr < n_redo; rr += a.n_fb_groups) {
    const int it = s_redo[rr];
    const int n = MAT ? (int)(a.surv_idx[sc.s_lo + it] - (long long)h * HU) : n_lo + it;
    const int s_out = MAT ? sc.s_lo + it : 0;
    // phase 1: deaths
    int my_dead = 0;
    unsigned long long hsh = 0;
    for (int x = lane; x < ndpc; x += 32) {
      const uint32_t ent = s_dpc[x];
      const uint32_t cc = ent >> 4, mask = ent & 15u;
      const uint4 r = philox10(make_uint4(uid_lo, uid_hi, 2u * (uint32_t)n, cc), key);
#pragma unroll
      for (int b = 0; b < 4; ++b) {
        if (!((mask >> b) & 1u)) continue;
        const int t = 4 * (int)cc + b;
        if ((word_of(r, b) >> 8) < s_dthr[t]) {
          atomicOr(&dmask[t >> 5], 1u << (t & 31));
          touch(tmask, tlist, ntp, t);
          ++my_dead;
          hsh += dead_key(t);
        }
      }
    }
    __syncwarp();
    if (MAT) {
      uint32_t carry = 0;
      for (int base = 0; base < W; base += 32) {
        const int w = base + lane;
        const uint32_t v = w < W ? (uint32_t)__popc(dmask[w]) : 0u;
        uint32_t x = v;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
          const uint32_t y = __shfl_up_sync(0xFFFFFFFFu, x, o);
          if (lane >= o) x += y;
        }
        if (w < W) dpre[w] = carry + x - v;
        carry += __shfl_sync(0xFFFFFFFFu, x, 31);
      }
      __syncwarp();
    }
    // phase 2: one categorical draw per detection row
    int my_dclut = 0;
    bool bad_row = false;
    for (int cc = lane; cc < nrc; cc += 32) {
      const int i0 = 4 * cc;
      const int i1 = min(i0 + 4, M);
      if (s_rowoff[i1] == s_rowoff[i0]) {
        if (MAT)
          for (int i = i0; i < i1; ++i) a.out_theta[(size_t)s_out * M + i] = 0;
        continue;
      }
      const uint4 r = philox10(make_uint4(uid_lo, uid_hi, 2u * (uint32_t)n + 1u, (uint32_t)cc), key);
#pragma unroll
      for (int b = 0; b < 4; ++b) {
        const int i = i0 + b;
        if (i >= i1) break;
        const uint32_t off = s_rowoff[i];
        const int nc = (int)(s_rowoff[i + 1] - off);
        if (nc == 0) {
          if (MAT) a.out_theta[(size_t)s_out * M + i] = 0;
          continue;
        }
        const uint32_t k = word_of(r, b) >> 8;
        bool fast = true;
        if (s_rowflag[i])
          for (int j = 0; j < nc; ++j)
            if (bit_of(dmask, s_cslot[off + j])) { fast = false; break; }
        int opt;
        if (fast) {
          if (k < s_rowthr0[i]) {
            opt = 0;
          } else {
            int j = 0;
            while (j < nc - 1 && k >= s_cthr[off + j]) ++j;
            opt = j + 1;
          }
        } else {
          const float w0 = md.kappa_zero ? 0.f : s_roww0[i];
          float sum = w0;
          for (int j = 0; j < nc; ++j)
            if (!bit_of(dmask, s_cslot[off + j])) sum += s_cw[off + j];
          if (!(sum > 0.f)) {
            bad_row = true;
            opt = 0;
          } else {
            const float xk = (float)k * 5.9604644775390625e-8f * sum;
            float cum = w0;
            int last = w0 > 0.f ? 0 : -1;
            opt = -1;
            if (w0 > 0.f && xk < cum) opt = 0;
            for (int j = 0; j < nc; ++j) {
              if (bit_of(dmask, s_cslot[off + j])) continue;
              const float w = s_cw[off + j];
              if (!(w > 0.f)) continue;
              cum += w;
              last = j + 1;
              if (opt < 0 && xk < cum) opt = j + 1;
            }
            if (opt < 0) opt = last < 0 ? 0 : last;
          }
        }
        const int ref = s_rowref[i];
        int ns = -1;
        if (opt > 0) ns = s_cslot[off + opt - 1];
        if (opt != ref) {
          int rs = -1;
          if (ref > 0) {
            rs = s_cslot[off + ref - 1];
            const uint32_t pos = off + ref - 1;
            atomicSub(&acc_cnt[rs], 1);
#pragma unroll
            for (int d = 0; d < DZ; ++d)
              atomicAdd((unsigned long long*)&acc_se[d * T + rs], (unsigned long long)(-fx_of(s_ce[d * Kp + pos])));
            atomicAdd((unsigned long long*)&acc_sq[rs], (unsigned long long)(-fx_of(s_cq[pos])));
            if (MAT) atomicAdd(&acc_hw[rs], (unsigned long long)(0ULL - wset_key(i)));
            touch(tmask, tlist, ntp, rs);
          } else {
            --my_dclut;
          }
          if (opt > 0) {
            const uint32_t pos = off + opt - 1;
            atomicAdd(&acc_cnt[ns], 1);
#pragma unroll
            for (int d = 0; d < DZ; ++d)
              atomicAdd((unsigned long long*)&acc_se[d * T + ns], (unsigned long long)fx_of(s_ce[d * Kp + pos]));
            atomicAdd((unsigned long long*)&acc_sq[ns], (unsigned long long)fx_of(s_cq[pos]));
            if (MAT) atomicAdd(&acc_hw[ns], wset_key(i));
            touch(tmask, tlist, ntp, ns);
          } else {
            ++my_dclut;
          }
          hsh += row_key(i, opt > 0 ? ns + 1 : 0) - row_key(i, ref > 0 ? rs + 1 : 0);
        }
        if (MAT) {
          uint16_t th = 0;
          if (ns >= 0) {
            const uint32_t below = dpre[ns >> 5] + __popc(dmask[ns >> 5] & ((1u << (ns & 31)) - 1u));
            th = (uint16_t)(ns - (int)below + 1);
          }
          a.out_theta[(size_t)s_out * M + i] = th;
        }
      }
    }
    __syncwarp();
    // phase 3: rescore touched slots
    const int nt = *((volatile int*)ntp);
    long long my_delta = 0;
    int my_dninf = 0;
    for (int x = lane; x < nt; x += 32) {
      const int t = tlist[x];
      int ninf;
      long long term;
      long long se[DZ];
      int m = 0;
      const bool dead = bit_of(dmask, t);
      if (dead) {
        term = dead_term(s_log1mp[t], ninf);
      } else {
        float HPH[DZ][DZ];
        slot_HPH<DZ>(s_hph, T, t, HPH);
        m = s_mref[t] + acc_cnt[t];
#pragma unroll
        for (int d = 0; d < DZ; ++d) se[d] = s_seref[d * T + t] + acc_se[d * T + t];
        term = alive_term<DZ>(md, HPH, s_logp[t], m, se, s_sqref[t] + acc_sq[t], ninf);
      }
      my_delta += term - s_termref[t];
      my_dninf += ninf - (int)s_ninfref[t];
      if (MAT && !dead)
        newval[t] = m >= 1 ? upd_insert<DZ>(a, s_comp[t], s_hwref[t] + acc_hw[t], m, se) : s_comp[t];
      acc_cnt[t] = 0;
#pragma unroll
      for (int d = 0; d < DZ; ++d) acc_se[d * T + t] = 0;
      acc_sq[t] = 0;
      if (MAT) acc_hw[t] = 0;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      my_delta += __shfl_xor_sync(0xFFFFFFFFu, my_delta, o);
      my_dninf += __shfl_xor_sync(0xFFFFFFFFu, my_dninf, o);
      my_dclut += __shfl_xor_sync(0xFFFFFFFFu, my_dclut, o);
      my_dead += __shfl_xor_sync(0xFFFFFFFFu, my_dead, o);
      hsh += __shfl_xor_sync(0xFFFFFFFFu, hsh, o);
    }
    const bool any_bad = __any_sync(0xFFFFFFFFu, bad_row);
    __syncwarp();
    if (MAT) {
      const uint32_t base = a.out_ptr[s_out];
      for (int t = lane; t < T; t += 32) {
        if (bit_of(dmask, t)) continue;
        const uint32_t below = dpre[t >> 5] + __popc(dmask[t >> 5] & ((1u << (t & 31)) - 1u));
        a.out_comp[base + (uint32_t)t - below] = bit_of(tmask, t) ? newval[t] : s_refnew[t];
      }
      __syncwarp();
    }
    for (int w = lane; w < W; w += 32) { tmask[w] = 0; dmask[w] = 0; }
    if (lane == 0) {
      *ntp = 0;
      if (!MAT) {
        const long long score = ref_score + my_delta + (md.kappa_zero ? 0LL : (long long)my_dclut * md.fx_log_kappa);
        const int ninf = ninf_ref + my_dninf + (md.kappa_zero ? my_dclut : 0);
        const bool valid = !any_bad && ninf == 0;
        const size_t j = (size_t)h * HU + n;
        a.child_key[j] = valid ? score : kKeyInvalid;
        a.child_hash[j] = hsh;
        a.child_status[j] = valid ? 1 : 0;
        a.child_alive[j] = (uint16_t)(T - my_dead);
      }
    }
    __syncwarp();
  }
}

// Unique children of each parent (Section 3: only unique hypotheses are
// retained): a valid child whose key equals a lower valid draw's is a
// duplicate; its weight is dropped.  One block per parent.
__global__ void dedup_kernel(const FrameDev* __restrict__ fs, int HU, long long* child_key,
                             const unsigned long long* __restrict__ child_hash, int8_t* child_status) {
  extern __shared__ unsigned long long s_h[];
  uint8_t* s_v = reinterpret_cast<uint8_t*>(s_h + HU);
  const int H = fs->H;
  for (int h = blockIdx.x; h < H; h += gridDim.x) {
    const size_t base = (size_t)h * HU;
    __syncthreads();
    for (int n = threadIdx.x; n < HU; n += blockDim.x) {
      s_h[n] = child_hash[base + n];
      s_v[n] = child_status[base + n] != 0;
    }
    __syncthreads();
    for (int n = threadIdx.x; n < HU; n += blockDim.x) {
      if (!s_v[n]) continue;
      const unsigned long long hv = s_h[n];
      bool dup = false;
      for (int n2 = 0; n2 < n; ++n2)
        if (s_v[n2] && s_h[n2] == hv) { dup = true; break; }
      if (dup) {
        child_status[base + n] = 2;
        child_key[base + n] = kKeyInvalid;
      }
    }
  }
}

void launch_dedup(const FrameDev* fs, int HU, long long* child_key, const unsigned long long* child_hash,
                  int8_t* child_status, int grid, cudaStream_t s) {
  const int smem = HU * 9 + 16;
  if (smem > 48 * 1024) cudaFuncSetAttribute(dedup_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  dedup_kernel<<<grid, 128, smem, s>>>(fs, HU, child_key, child_hash, child_status);
  ++g_launches;
}

template <int DZ, bool MAT>
static void launch_one(const ExpandArgs& a, int grid, cudaStream_t s) {
  expand_kernel<DZ, MAT><<<grid, 32 * a.n_groups, a.smem_bytes, s>>>(a);
  ++g_launches;
}

void expand_init(int smem_limit) {
  cudaFuncSetAttribute(expand_kernel<2, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem_limit);
  cudaFuncSetAttribute(expand_kernel<2, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem_limit);
  cudaFuncSetAttribute(expand_kernel<3, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem_limit);
  cudaFuncSetAttribute(expand_kernel<3, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem_limit);
}

int expand_max_ctas(const ExpandArgs& a) {
  int per_sm = 0;
  const int threads = 32 * a.n_groups;
  cudaError_t e;
  if (a.md.dz == 2)
    e = a.materialize ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, expand_kernel<2, true>, threads, a.smem_bytes)
                      : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, expand_kernel<2, false>, threads, a.smem_bytes);
  else
    e = a.materialize ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, expand_kernel<3, true>, threads, a.smem_bytes)
                      : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, expand_kernel<3, false>, threads, a.smem_bytes);
  return e == cudaSuccess ? per_sm : 0;
}

void launch_expand(const ExpandArgs& a, int grid, cudaStream_t s) {
  if (grid <= 0) return;
  if (a.md.dz == 2) {
    if (a.materialize) launch_one<2, true>(a, grid, s);
    else launch_one<2, false>(a, grid, s);
  } else {
    if (a.materialize) launch_one<3, true>(a, grid, s);
    else launch_one<3, false>(a, grid, s);
  }
}

}  // namespace glmb

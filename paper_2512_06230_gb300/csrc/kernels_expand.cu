// Child expansion, scoring and per-parent deduplication (arXiv 2512.06230,
// Section 3: two-stage sampling of H_up children per hypothesis, weight =
// parent weight x joint likelihood of the sampled deaths and associations,
// retention of unique children), and the regeneration of the retained
// children for the batched track update.
//
// Four kernels share one per-parent image in global memory:
//   stage     one CTA per parent builds the parent's tables (in shared memory
//             when they fit, then copied out; else in place): its gated pairs
//             re-indexed by detection row (slots ascending within a row), per
//             row integer thresholds of the categorical draw under "all slots
//             alive", a reference association (each row's most likely option)
//             with its exact score, and per slot the m-only part of the track
//             term for m_ref - 2 .. m_ref + 2 detections;
//             The stage also tabulates the exact score change of every single
//             deviation from the reference: a detection joining a candidate
//             pair's slot, leaving its reference slot, a slot dying;
//   draw      one thread per child: Philox words for the slots that can die
//             (stage 1) and one per detection row (stage 2); the row's option
//             is the first whose threshold exceeds the 24-bit uniform (rows
//             with a dead candidate fall back to the FP32 normalised row of
//             C'_k); deaths and rows that leave the reference are listed in
//             shared memory; the child's log-weight is the reference score
//             plus the tabulated changes, or, when a slot is met twice, the
//             exact rescoring of every met slot (stage 3), in fixed point;
//   warp      one warp per child, rows split over the lanes and per-slot sums
//             in shared memory: children whose lists overflow the draw
//             kernel's, every child when parents are too few to fill
//             the GPU with threads, and the regeneration of retained children
//             (association rows, track lists, updated-component requests);
//   mat_prep  the updated components of each retained parent's reference
//             association, requested once per parent.
// The duplicate test keys a child by the order-free sum of mix64 keys of its
// deviations and deaths.
#include <algorithm>
#include <map>
#include <mutex>
#include <tuple>

#include "glmb_kernels.h"

namespace glmb {

// ---- per-parent image ----

struct Lay {
  int scal;
  int row, rowbl, seref, sqref, termref, hwref, deadd;
  int rowrk, rch, rowoff, rowfill, roww0, rowthr0;
  int comp, dthr, logp, log1mp, mref, refnew, hph, dpc;
  int cthr, ceidx, cw, ce, cq, cslot;
  int ninfref, dninf, srow;
  int total;
};

// Chunk of four detection rows with candidates, as the thread-per-child
// draw reads it: head = (chunk index, bit b set when row 4 cc + b has a
// candidate slot that can die, low and high words of the bloom of those
// slots over the four rows), then the four rows' reference intervals
// [lo, hi) of the 24-bit uniform u = word >> 8 (rows without candidates, or
// beyond the detections: [0, 2^24)), held as base = lo << 8 and
// span = ((hi - lo) << 8) - 1 (mod 2^32): u is in [lo, hi) exactly when
// word - base <= span, as unsigned 32-bit arithmetic (hi - lo >= 1).
struct RowChunk {
  uint4 head;
  uint4 base;
  uint4 span;
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
  int ninf_ref, nclut_ref, T, Town, K, ndpc, nrca, bad;
};

// T, K, M: the plan's slots, gated pairs and detection rows per parent.
// Per-slot arrays are indexed with the parent's own slot count as stride,
// per-pair arrays with K.
__host__ __device__ inline Lay make_lay(int dz, int T, int K, int M) {
  Lay L;
  Bump b;
  const int NP = dz * (dz + 1) / 2;
  L.scal = b.take(sizeof(Scal));
  L.row = b.take(16LL * M);                 // packed row descriptors (uint4)
  L.rowbl = b.take(8LL * M);                // bit (slot mod 64) of each candidate slot
  L.seref = b.take(8LL * dz * T);           // reference sums of innovations (fixed point)
  L.sqref = b.take(8LL * T);                // reference sums of e^T R^-1 e
  L.termref = b.take(8LL * T);              // reference track terms
  L.hwref = b.take(8LL * T);                // reference detection-set keys
  // exact score change of a slot dying (deadd[t]) and of its infinite-term
  // count (dninf); a row's deviations are scored by the child that makes them
  L.deadd = b.take(8LL * T);
  L.rowrk = b.take(4LL * M);                // reference option's slot and pair
  L.rch = b.take(48LL * ((M + 3) / 4 + 1)); // chunks of 4 rows with candidates (RowChunk)
  L.rowoff = b.take(4LL * (M + 1));
  L.rowfill = b.take(4LL * (M + 1));
  L.roww0 = b.take(4LL * M);
  L.rowthr0 = b.take(4LL * M);              // clutter option's threshold
  L.comp = b.take(4LL * T);
  L.dthr = b.take(4LL * T);
  L.logp = b.take(4LL * T);
  L.log1mp = b.take(4LL * T);
  L.mref = b.take(4LL * T);
  L.refnew = b.take(4LL * T);
  L.hph = b.take(4LL * NP * T);             // H P H^T of each slot (packed)
  L.dpc = b.take(4LL * (T / 4 + 2));        // chunks of 4 slots that can die
  L.cthr = b.take(4LL * K);
  L.ceidx = b.take(4LL * K);
  L.cw = b.take(4LL * K);
  L.ce = b.take(4LL * dz * K);              // innovation of each candidate pair
  L.cq = b.take(4LL * K);                   // e^T R^-1 e of each candidate pair
  L.cslot = b.take(2LL * K);
  L.ninfref = b.take(T);
  L.dninf = b.take(T);
  L.srow = b.take(T);                       // slot can die and is a candidate of some row
  L.total = b.off;
  return L;
}

// The staging kernel's shared scratch beside the image: the next-parent
// word (16 B) and the scan's warp sums (32 B); then, when the image is
// built in global memory, the arrays the staging reads back many times:
// mode >= 1 the row offsets and fill cursors, mode 2 also the candidates'
// slots and pair indices and the per-slot reference counts, sums, terms
// and infinite-term counts (copied to the image at the end of the parent).
// Offsets from its base.
struct StageTail {
  int rowoff, rowfill, cslot, ceidx, mref, seref, sqref, hwref, termref, ninfref, dthr, total;
};
__host__ __device__ inline StageTail make_stage_tail(int dz, int T, int K, int M, int mode) {
  StageTail S{};
  Bump b;
  b.take(16);   // next-parent word
  b.take(32);   // warp sums of the row-count scan
  if (mode >= 1) {
    S.rowoff = b.take(4LL * (M + 1));
    S.rowfill = b.take(4LL * (M + 1));
  }
  if (mode >= 2) {
    S.cslot = b.take(2LL * K);
    S.ceidx = b.take(4LL * K);
    S.mref = b.take(4LL * T);
    S.seref = b.take(8LL * dz * T);
    S.sqref = b.take(8LL * T);
    S.hwref = b.take(8LL * T);
    S.termref = b.take(8LL * T);
    S.ninfref = b.take(T);
    S.dthr = b.take(4LL * T);
  }
  S.total = b.off;
  return S;
}

int expand_image_bytes(int dz, int T, int K, int M) {
  return (make_lay(dz, T, K, M).total + 127) & ~127;
}

// per-warp work area of the warp kernel
struct WLay {
  int se, sq, hw, cnt, newval, tmask, dmask, dpre, nt, tlist, red, total;
};

__host__ __device__ inline WLay make_wlay(int dz, int mat, int T, int grp = 0) {
  WLay L;
  Bump b;
  const int W = (T + 31) / 32 + 1;
  L.se = b.take(8LL * dz * T);
  L.sq = b.take(8LL * T);
  L.hw = mat ? b.take(8LL * T) : 0;
  L.cnt = b.take(4LL * T);
  L.newval = mat ? b.take(4LL * T) : 0;
  L.tmask = b.take(4LL * W);
  L.dmask = b.take(4LL * W);
  L.dpre = b.take(4LL * W);
  L.nt = b.take(16);
  L.tlist = b.take(2LL * T);
  L.red = grp ? b.take(64) : 0;   // a multi-warp group's reductions
  L.total = b.off;
  return L;
}

int expand_warp_smem(int dz, int materialize, int T, int warps, int grp) {
  return warps * make_wlay(dz, materialize, T, grp).total;
}

template <typename T>
__device__ __forceinline__ T* at(unsigned char* base, int off) {
  return reinterpret_cast<T*>(base + off);
}
template <typename T>
__device__ __forceinline__ const T* at(const unsigned char* base, int off) {
  return reinterpret_cast<const T*>(base + off);
}

__device__ __forceinline__ uint32_t thr_of(float frac) {
  // smallest integer k0 with k0 >= frac * 2^24, clamped to [0, 2^24]
  if (!(frac > 0.f)) return 0u;
  if (frac >= 1.f) return kOne24;
  return (uint32_t)ceilf(frac * 16777216.f);
}

// A child of the warp path is handled by a group of gsz threads (one warp,
// or several consecutive warps of the CTA that share one work area and
// synchronise on named barrier gid + 1).
__device__ __forceinline__ void group_sync(int gsz, int gid) {
  if (gsz == 32) __syncwarp();
  else asm volatile("bar.sync %0, %1;" ::"r"(gid + 1), "r"(gsz) : "memory");
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

// The m-only parts of component c's alive term with m detections, from the
// frame's per-component table (built by the table's count kernel).
template <int DZ>
__device__ __forceinline__ SlotM<DZ> load_cslm(const float* slm, const int8_t* sln, int cap, int m, uint32_t c) {
  constexpr int NP = DZ * (DZ + 1) / 2;
  SlotM<DZ> s;
  const size_t base = (size_t)(m - 1) * (NP + 1);
#pragma unroll
  for (int k = 0; k < NP; ++k) s.Sinv[k] = slm[(base + k) * cap + c];
  s.c = slm[(base + NP) * cap + c];
  s.ninf = sln[(size_t)(m - 1) * cap + c];
  return s;
}

// Term of slot t alive with m detections, built from H P H^T (kept out of
// line: it is rare and needs many registers)
struct TermOut {
  long long term;
  int ninf;
};
template <int DZ>
struct SeVec {
  long long v[DZ];
};

template <int DZ>
__device__ __noinline__ TermOut slot_term_full(const Model& md, const float* s_hph, const float* s_logp, int T,
                                               int t, int m, const SeVec<DZ> se, long long sq) {
  // the sums come and the result goes by value, so a caller keeps them in
  // registers (an array passed by reference would live in local memory)
  float HPH[DZ][DZ];
  slot_HPH<DZ>(s_hph, T, t, HPH);
  TermOut o;
  o.term = alive_term<DZ>(md, HPH, s_logp[t], m, se.v, sq, o.ninf);
  return o;
}

// read-only view of a staged parent
struct View {
  const Scal* sc;
  const uint4* row;
  const unsigned long long* rowbl;
  const long long *seref, *sqref, *termref, *deadd;
  const unsigned long long* hwref;
  const RowChunk* rch;
  const uint32_t *rowrk, *rowthr0, *comp, *dthr, *refnew, *dpc, *cthr;
  const float *roww0, *logp, *log1mp, *hph, *cw, *ce, *cq;
  const float* cslm;      // per-component m-only term parts (PairTable::slm)
  const int8_t* csln;
  int slm_cap;
  const int* mref;
  const uint16_t* cslot;
  const uint8_t* ninfref;
  const int8_t* dninf;
  const uint8_t* srow;
};

__device__ __forceinline__ View make_view(const unsigned char* b, const Lay& L, const PairTable& pt) {
  View v;
  v.sc = at<Scal>(b, L.scal);
  v.row = at<uint4>(b, L.row);
  v.rowbl = at<unsigned long long>(b, L.rowbl);
  v.seref = at<long long>(b, L.seref);
  v.sqref = at<long long>(b, L.sqref);
  v.termref = at<long long>(b, L.termref);
  v.deadd = at<long long>(b, L.deadd);
  v.dninf = at<int8_t>(b, L.dninf);
  v.hwref = at<unsigned long long>(b, L.hwref);
  v.rowrk = at<uint32_t>(b, L.rowrk);
  v.rch = at<RowChunk>(b, L.rch);
  v.srow = at<uint8_t>(b, L.srow);
  v.rowthr0 = at<uint32_t>(b, L.rowthr0);
  v.comp = at<uint32_t>(b, L.comp);
  v.dthr = at<uint32_t>(b, L.dthr);
  v.refnew = at<uint32_t>(b, L.refnew);
  v.dpc = at<uint32_t>(b, L.dpc);
  v.cthr = at<uint32_t>(b, L.cthr);
  v.roww0 = at<float>(b, L.roww0);
  v.logp = at<float>(b, L.logp);
  v.log1mp = at<float>(b, L.log1mp);
  v.hph = at<float>(b, L.hph);
  v.cslm = pt.slm;
  v.csln = pt.sln;
  v.slm_cap = pt.slm_cap;
  v.cw = at<float>(b, L.cw);
  v.ce = at<float>(b, L.ce);
  v.cq = at<float>(b, L.cq);
  v.mref = at<int>(b, L.mref);
  v.cslot = at<uint16_t>(b, L.cslot);
  v.ninfref = at<uint8_t>(b, L.ninfref);
  return v;
}

// a view for code that evaluates no track term (no per-component table)
__device__ __forceinline__ View make_view(const unsigned char* b, const Lay& L) {
  PairTable none{};
  return make_view(b, L, none);
}

// Term of slot t alive with m detections whose sums are (se, sq): the m-only
// parts from the per-component table when it holds (component, m), else
// built from H P H^T (the same function, so the same values).
template <int DZ>
__device__ __forceinline__ long long slot_term(const Model& md, const View& v, int T, int t, int m,
                                               const long long (&se)[DZ], long long sq, int& ninf) {
  if (md.score_mode == 1) return factor_term(md, v.logp[t], m, sq, ninf);
  if (m >= 1 && m <= kSlmM) {
    const uint32_t c = v.comp[t];
    if (c < (uint32_t)v.slm_cap) return term_from<DZ>(md, load_cslm<DZ>(v.cslm, v.csln, v.slm_cap, m, c), m, se, sq, ninf);
  }
  SeVec<DZ> sv;
#pragma unroll
  for (int d = 0; d < DZ; ++d) sv.v[d] = se[d];
  const TermOut o = slot_term_full<DZ>(md, v.hph, v.logp, T, t, m, sv, sq);
  ninf = o.ninf;
  return o.term;
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
        a.upd_slot[id] = slot;
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

// ====================== stage: one CTA per parent ======================
// Detection rows with at most this many candidate slots are sorted and
// weighed in registers (nearly all rows: a detection gates to one track or
// a few).
constexpr int kRowReg = 4;
template <int N>
struct FVec {
  float v[N];
};
// Builds parent h's image at `sm` (shared memory, or the image itself).
// `tb`: the shared scratch beside the image (StageTail).  With the image in
// global memory (in_tail) the arrays it lists live there while the parent
// is staged, so that their atomics and read-backs stay on chip, and are
// copied to the image at the end.
template <int DZ>
__device__ void stage_parent(const ExpandArgs& a, const int h, const Lay& L, unsigned char* sm, unsigned char* tb,
                             int mode) {
  const StageTail TS = make_stage_tail(DZ, a.T_max, a.K_max, a.M_plan, mode);
  const bool in_tail = mode >= 2;
  const Model& md = a.md;
  const int M = a.fs->M;
  const int birth_base = a.fs->n_comp, nb = a.fs->nb;
  Scal& sc = *at<Scal>(sm, L.scal);
  uint4* s_row = at<uint4>(sm, L.row);
  unsigned long long* s_rowbl = at<unsigned long long>(sm, L.rowbl);
  long long* s_seref = in_tail ? at<long long>(tb, TS.seref) : at<long long>(sm, L.seref);
  long long* s_sqref = in_tail ? at<long long>(tb, TS.sqref) : at<long long>(sm, L.sqref);
  long long* s_termref = in_tail ? at<long long>(tb, TS.termref) : at<long long>(sm, L.termref);
  unsigned long long* s_hwref = in_tail ? at<unsigned long long>(tb, TS.hwref) : at<unsigned long long>(sm, L.hwref);
  uint32_t* s_rowrk = at<uint32_t>(sm, L.rowrk);
  RowChunk* s_rch = at<RowChunk>(sm, L.rch);
  uint8_t* s_srow = at<uint8_t>(sm, L.srow);
  uint32_t* s_rowthr0 = at<uint32_t>(sm, L.rowthr0);
  uint32_t* s_wsum = at<uint32_t>(tb, 16);
  uint32_t* s_rowoff = mode >= 1 ? at<uint32_t>(tb, TS.rowoff) : at<uint32_t>(sm, L.rowoff);
  uint32_t* s_rowfill = mode >= 1 ? at<uint32_t>(tb, TS.rowfill) : at<uint32_t>(sm, L.rowfill);
  float* s_roww0 = at<float>(sm, L.roww0);
  uint32_t* s_comp = at<uint32_t>(sm, L.comp);
  // death thresholds: written to the image, read back on chip
  uint32_t* g_dthr = at<uint32_t>(sm, L.dthr);
  uint32_t* s_dthr = in_tail ? at<uint32_t>(tb, TS.dthr) : g_dthr;
  float* s_logp = at<float>(sm, L.logp);
  float* s_log1mp = at<float>(sm, L.log1mp);
  int* s_mref = in_tail ? at<int>(tb, TS.mref) : at<int>(sm, L.mref);
  float* s_hph = at<float>(sm, L.hph);
  uint32_t* s_dpc = at<uint32_t>(sm, L.dpc);
  uint32_t* s_cthr = at<uint32_t>(sm, L.cthr);
  uint32_t* s_ceidx = in_tail ? at<uint32_t>(tb, TS.ceidx) : at<uint32_t>(sm, L.ceidx);
  float* s_cw = at<float>(sm, L.cw);
  float* s_ce = at<float>(sm, L.ce);
  float* s_cq = at<float>(sm, L.cq);
  uint16_t* s_cslot = in_tail ? at<uint16_t>(tb, TS.cslot) : at<uint16_t>(sm, L.cslot);
  uint8_t* s_ninfref = in_tail ? at<uint8_t>(tb, TS.ninfref) : at<uint8_t>(sm, L.ninfref);
  const int Kp = a.K_max;                   // stride of the candidate arrays
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
    sc.nrca = 0;
    sc.bad = 0;
    sc.K = 0;
    sc.uid = a.parents.uid[h];
    sc.logw = a.parents.logw[h];
    // the block reads its sizes and counts on chip (the scan's words are
    // free until the scan)
    s_wsum[2] = (uint32_t)sc.T;
    s_wsum[3] = (uint32_t)sc.Town;
    s_wsum[4] = 0u;   // gated pairs
    s_wsum[5] = 0u;   // bad
  }
  __syncthreads();
  const int T = (int)s_wsum[2], Town = (int)s_wsum[3];
  const uint32_t plo = a.parents.ptr[h];
  // the parent's gated pairs, counted for every parent (also one beyond the
  // plan): the frame's maxima plan the next frame, or this frame's redo
  {
    unsigned kp = 0;
    for (int t = tid; t < T; t += nthr) {
      const uint32_t c = t < Town ? a.parents.comp[plo + t] : (uint32_t)(birth_base + (t - Town));
      if (c >= (uint32_t)(birth_base + nb)) {   // invariant: slots name the working table
        atomicOr(a.err, kErrChkComp);
        continue;
      }
      kp += pt.cnt[c];
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) kp += __shfl_xor_sync(0xFFFFFFFFu, kp, o);
    if ((tid & 31) == 0 && kp) atomicAdd(&s_wsum[4], kp);
  }
  __syncthreads();
  if (tid == 0) {
    const int K = (int)s_wsum[4];
    sc.K = K;
    int bad = (*(volatile const unsigned*)a.err & kErrChkComp) ? 1 : 0;
    if (a.max_T) atomicMax(a.max_T, (unsigned)T);
    if (a.max_K) atomicMax(a.max_K, (unsigned)K);
    if (T > a.T_max || M > a.M_plan || K > a.K_max) {
      bad = 1;
      atomicOr(a.err, kErrSlots);
    }
    sc.bad = bad;
    s_wsum[5] = (uint32_t)bad;
  }
  __syncthreads();
  if (s_wsum[5]) return;

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
    {
      const uint32_t dt = pt.dthr[c];
      s_dthr[t] = dt;
      if (in_tail) g_dthr[t] = dt;
    }
    s_logp[t] = ct.logp[c];
    s_log1mp[t] = ct.log1mp[c];
    s_mref[t] = 0;
#pragma unroll
    for (int d = 0; d < DZ; ++d) s_seref[d * T + t] = 0;
    s_sqref[t] = 0;
    s_hwref[t] = 0;
  }
  for (int i = tid; i <= M; i += nthr) s_rowfill[i] = 0;
  __syncthreads();
  for (int t = tid; t < T; t += nthr) {
    const uint32_t c = s_comp[t];
    for (uint32_t j = pt.ptr[c], je = pt.ptr[c + 1]; j < je; ++j) atomicAdd(&s_rowfill[pt.meas[j]], 1u);
    s_srow[t] = (pt.ptr[c + 1] > pt.ptr[c] && s_dthr[t] > 0u) ? 1 : 0;
  }
  __syncthreads();
  // exclusive scan of the row counts over the block: each thread a
  // contiguous run of rows, a scan of the runs' totals across the warps;
  // the offsets are also the fill cursors
  {
    const int per = (M + nthr - 1) / nthr;
    const int b0 = min(M, tid * per), b1 = min(M, b0 + per);
    uint32_t run = 0;
    for (int i = b0; i < b1; ++i) run += s_rowfill[i];
    const int lane = tid & 31, wp = tid >> 5;
    uint32_t x = run;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t y = __shfl_up_sync(0xFFFFFFFFu, x, o);
      if (lane >= o) x += y;
    }
    if (lane == 31) s_wsum[wp] = x;
    __syncthreads();
    uint32_t base = x - run;
    for (int w = 0; w < wp; ++w) base += s_wsum[w];
    for (int i = b0; i < b1; ++i) {
      const uint32_t v = s_rowfill[i];
      s_rowoff[i] = base;
      s_rowfill[i] = base;
      base += v;
    }
    if (tid == nthr - 1) {
      // the last thread's run ends at M (or is empty, with base the total)
      s_rowoff[M] = base;
      sc.K = (int)base;
      const bool over = (int)base > a.K_max;
      if (over) {
        sc.bad = 1;
        atomicOr(a.err, kErrSlots);
      }
      s_wsum[7] = over ? 1u : 0u;   // no warp's scan reads the last word
    }
  }
  __syncthreads();
  if (s_wsum[7]) return;
  for (int t = tid; t < T; t += nthr) {
    const uint32_t c = s_comp[t];
    for (uint32_t j = pt.ptr[c], je = pt.ptr[c + 1]; j < je; ++j) {
      const uint32_t i = pt.meas[j];
      const uint32_t pos = atomicAdd(&s_rowfill[i], 1u);
      s_cslot[pos] = (uint16_t)t;
      s_ceidx[pos] = j;
    }
  }
  __syncthreads();

  // ---- rows: order, weights, thresholds, reference option ----
  // (the scan's sums are read; their words count the chunk lists next)
  if (tid == 0) {
    s_wsum[0] = 0u;
    s_wsum[1] = 0u;
  }
  {
    int my_clut = 0;
    // every thread runs the same rounds, so that the four rows of a chunk
    // (four neighbouring lanes: nthr is a multiple of 32) can pass their
    // parts of the chunk's record to its first lane
    for (int rb = 0; rb < M; rb += nthr) {
    const int i = rb + tid;
    bool r_has = false, r_flag = false;
    uint32_t r_lo = 0u, r_hi = kOne24;
    unsigned long long r_bl = 0ull;
    auto row_body = [&]() {
      if (i >= M) return;
      const uint32_t off = s_rowoff[i];
      const int nc = (int)(s_rowoff[i + 1] - off);
      if (nc == 0) {
        s_row[i] = make_uint4(off, 0u, 0u, kOne24);
        s_rowthr0[i] = kOne24;
        s_rowbl[i] = 0ull;
        s_rowrk[i] = 0u;
        s_roww0[i] = 1.f;
        ++my_clut;
        return;
      }
      // row i: x = first candidate, y = count | may-die flag << 15 |
      // reference option << 16, [z, w) = the uniforms that pick the reference
      // option when every candidate is alive; the reference slot's sums
      auto finish_row = [&](int ref, bool flag, uint32_t thr0, uint32_t lo, uint32_t hi, unsigned long long bl,
                            float w0, int r, const FVec<DZ> e_ref, float q_ref) {
        s_row[i] = make_uint4(off, (uint32_t)nc | (flag ? 0x8000u : 0u) | ((uint32_t)ref << 16), lo, hi);
        s_rowthr0[i] = thr0;
        s_rowbl[i] = bl;
        s_rowrk[i] = ref > 0 ? (((uint32_t)r + 1u) << 16) | (off + ref - 1) : 0u;
        s_roww0[i] = w0;
        r_has = true;
        r_flag = flag;
        r_lo = lo;
        r_hi = hi;
        r_bl = bl;
        if (ref == 0) {
          ++my_clut;
        } else {
          atomicAdd(&s_mref[r], 1);
#pragma unroll
          for (int d = 0; d < DZ; ++d)
            atomicAdd((unsigned long long*)&s_seref[d * T + r], (unsigned long long)fx_of(e_ref.v[d]));
          atomicAdd((unsigned long long*)&s_sqref[r], (unsigned long long)fx_of(q_ref));
          atomicAdd(&s_hwref[r], wset_key(i));
        }
      };
      if (nc <= kRowReg) {
        // the candidates in registers: sorted, weighed and thresholded with
        // the same operations in the same order as the general path below
        uint32_t cs[kRowReg], ce[kRowReg];
#pragma unroll
        for (int x = 0; x < kRowReg; ++x) {
          cs[x] = x < nc ? s_cslot[off + x] : 0xFFFFu;
          ce[x] = x < nc ? s_ceidx[off + x] : 0u;
        }
#pragma unroll
        for (int x = 1; x < kRowReg; ++x)
#pragma unroll
          for (int y = x; y > 0; --y)
            if (cs[y - 1] > cs[y]) {   // unused entries (0xFFFF) stay last
              const uint32_t ts = cs[y - 1], te = ce[y - 1];
              cs[y - 1] = cs[y];
              ce[y - 1] = ce[y];
              cs[y] = ts;
              ce[y] = te;
            }
        float lc[kRowReg];
        float smax = md.kappa_zero ? -INFINITY : md.log_kappa;
#pragma unroll
        for (int x = 0; x < kRowReg; ++x) {
          if (x >= nc) break;
          s_cslot[off + x] = (uint16_t)cs[x];
          s_ceidx[off + x] = ce[x];
          lc[x] = pt.logC[ce[x]];
          smax = fmaxf(smax, lc[x]);
#pragma unroll
          for (int d = 0; d < DZ; ++d) s_ce[d * Kp + off + x] = pt.e[d * capp + ce[x]];
          s_cq[off + x] = md.score_mode == 1 ? lc[x] : pt.q[ce[x]];
        }
        const float w0 = md.kappa_zero ? 0.f : expf(md.log_kappa - smax);
        float wv[kRowReg];
        float sum = w0;
#pragma unroll
        for (int x = 0; x < kRowReg; ++x) {
          if (x >= nc) break;
          wv[x] = expf(lc[x] - smax);
          s_cw[off + x] = wv[x];
          sum += wv[x];
        }
        float cum = w0, best = w0;
        int ref = 0;
        bool flag = false;
        const uint32_t thr0 = thr_of(cum / sum);
        uint32_t lo = 0u, hi = thr0, prev = thr0;
        unsigned long long bl = 0ull;
        int r = 0;
        uint32_t rce = 0u;
        float rlc = 0.f;
#pragma unroll
        for (int x = 0; x < kRowReg; ++x) {
          if (x >= nc) break;
          const bool can_die = s_dthr[cs[x]] > 0u;
          if (can_die) bl |= 1ull << (cs[x] & 63);
          cum += wv[x];
          const uint32_t th = (x == nc - 1) ? kOne24 : thr_of(cum / sum);
          s_cthr[off + x] = th;
          if (wv[x] > best) {
            best = wv[x];
            ref = x + 1;
            lo = prev;
            hi = th;
            r = (int)cs[x];
            rce = ce[x];
            rlc = lc[x];
          }
          prev = th;
          flag |= can_die;
        }
        // the reference pair's innovation and q, read again (L1)
        FVec<DZ> e_ref;
        float q_ref = 0.f;
#pragma unroll
        for (int d = 0; d < DZ; ++d) e_ref.v[d] = ref > 0 ? pt.e[d * capp + rce] : 0.f;
        if (ref > 0) q_ref = md.score_mode == 1 ? rlc : pt.q[rce];
        finish_row(ref, flag, thr0, lo, hi, bl, w0, r, e_ref, q_ref);
        return;
      }
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
      float smax = md.kappa_zero ? -INFINITY : md.log_kappa;
      for (int j = 0; j < nc; ++j) {
        const uint32_t ei = s_ceidx[off + j];
        smax = fmaxf(smax, pt.logC[ei]);
#pragma unroll
        for (int d = 0; d < DZ; ++d) s_ce[d * Kp + off + j] = pt.e[d * capp + ei];
        // e^T R^-1 e of the pair; the factorised mode sums log C instead
        s_cq[off + j] = md.score_mode == 1 ? pt.logC[ei] : pt.q[ei];
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
      const uint32_t thr0 = thr_of(cum / sum);
      unsigned long long bl = 0ull;
      for (int j = 0; j < nc; ++j) {
        const float w = s_cw[off + j];
        const bool can_die = s_dthr[s_cslot[off + j]] > 0u;
        if (can_die) bl |= 1ull << (s_cslot[off + j] & 63);
        cum += w;
        s_cthr[off + j] = (j == nc - 1) ? kOne24 : thr_of(cum / sum);
        if (w > best) { best = w; ref = j + 1; }
        flag |= can_die;
      }
      const uint32_t lo = ref == 0 ? 0u : (ref == 1 ? thr0 : s_cthr[off + ref - 2]);
      const uint32_t hi = ref == 0 ? thr0 : s_cthr[off + ref - 1];
      FVec<DZ> e_ref;
      float q_ref = 0.f;
      int r = 0;
#pragma unroll
      for (int d = 0; d < DZ; ++d) e_ref.v[d] = 0.f;
      if (ref > 0) {
        const uint32_t pos = off + ref - 1;
        r = s_cslot[pos];
#pragma unroll
        for (int d = 0; d < DZ; ++d) e_ref.v[d] = s_ce[d * Kp + pos];
        q_ref = s_cq[pos];
      }
      finish_row(ref, flag, thr0, lo, hi, bl, w0, r, e_ref, q_ref);
    };
    row_body();
    // the chunk's record, at its first lane
    {
      const int lane = tid & 31, lead = lane & ~3;
      uint32_t cmask = 0u, cdmask = 0u, blo = 0u, bhi = 0u, lo4[4], hi4[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const uint32_t has = __shfl_sync(0xFFFFFFFFu, r_has ? 1u : 0u, lead + q);
        const uint32_t fl = __shfl_sync(0xFFFFFFFFu, r_flag ? 1u : 0u, lead + q);
        const uint32_t bl0 = __shfl_sync(0xFFFFFFFFu, (uint32_t)r_bl, lead + q);
        const uint32_t bl1 = __shfl_sync(0xFFFFFFFFu, (uint32_t)(r_bl >> 32), lead + q);
        lo4[q] = __shfl_sync(0xFFFFFFFFu, r_lo, lead + q);
        hi4[q] = __shfl_sync(0xFFFFFFFFu, r_hi, lead + q);
        cmask |= has << q;
        if (fl) {
          cdmask |= 1u << q;
          blo |= bl0;
          bhi |= bl1;
        }
      }
      if (lane == lead && cmask) {
        RowChunk rc;
        rc.head = make_uint4((uint32_t)(i >> 2), cdmask, blo, bhi);
        rc.base = make_uint4(lo4[0] << 8, lo4[1] << 8, lo4[2] << 8, lo4[3] << 8);
        rc.span = make_uint4(((hi4[0] - lo4[0]) << 8) - 1u, ((hi4[1] - lo4[1]) << 8) - 1u,
                             ((hi4[2] - lo4[2]) << 8) - 1u, ((hi4[3] - lo4[3]) << 8) - 1u);
        s_rch[atomicAdd(&s_wsum[1], 1u)] = rc;
      }
    }
    }
    if (my_clut) atomicAdd(&sc.nclut_ref, my_clut);
  }
  __syncthreads();

  // ---- chunk lists ----
  {
    const int nch = (T + 3) >> 2;
    for (int cc = tid; cc < nch; cc += nthr) {
      uint32_t mask = 0;
#pragma unroll
      for (int b = 0; b < 4; ++b) {
        const int t = 4 * cc + b;
        if (t < T && s_dthr[t] > 0u) mask |= 1u << b;
      }
      if (mask) s_dpc[atomicAdd(&s_wsum[0], 1u)] = ((uint32_t)cc << 4) | mask;
    }
  }
  __syncthreads();
  if (tid == 0) {
    sc.ndpc = (int)s_wsum[0];
    sc.nrca = (int)s_wsum[1];
  }

  // ---- reference terms ----
  {
    long long my_term = 0;
    int my_ninf = 0;
    for (int t = tid; t < T; t += nthr) {
      long long se[DZ];
#pragma unroll
      for (int d = 0; d < DZ; ++d) se[d] = s_seref[d * T + t];
      const int mr = s_mref[t];
      int ninf;
      long long term;
      if (md.score_mode == 0 && mr >= 1 && mr <= kSlmM && s_comp[t] < (uint32_t)a.pt.slm_cap) {
        term = term_from<DZ>(md, load_cslm<DZ>(a.pt.slm, a.pt.sln, a.pt.slm_cap, mr, s_comp[t]), mr, se, s_sqref[t],
                             ninf);
      } else {
        float HPH[DZ][DZ];
        slot_HPH<DZ>(s_hph, T, t, HPH);
        term = alive_term<DZ>(md, HPH, s_logp[t], mr, se, s_sqref[t], ninf);
      }
      s_termref[t] = term;
      s_ninfref[t] = (uint8_t)ninf;
      my_term += term;
      my_ninf += ninf;
    }
    if (my_term) atomicAdd((unsigned long long*)&sc.ref_score, (unsigned long long)my_term);
    if (my_ninf) atomicAdd(&sc.ninf_ref, my_ninf);
  }
  __syncthreads();

  // ---- death deltas: a slot dying changes its term to the dead term (the
  // rows' single deviations are scored by the children that make them) ----
  {
    long long* s_deadd = at<long long>(sm, L.deadd);
    int8_t* s_dninf = at<int8_t>(sm, L.dninf);
    for (int t = tid; t < T; t += nthr) {
      int ninf;
      const long long term = dead_term(s_log1mp[t], ninf);
      s_deadd[t] = term - s_termref[t];
      s_dninf[t] = (int8_t)(ninf - (int)s_ninfref[t]);
    }
  }
  if (in_tail) {
    // the arrays staged on chip go to the image
    __syncthreads();
    const int K = sc.K;
    uint16_t* g_cslot = at<uint16_t>(sm, L.cslot);
    uint32_t* g_ceidx = at<uint32_t>(sm, L.ceidx);
    for (int i = tid; i < K; i += nthr) {
      g_cslot[i] = s_cslot[i];
      g_ceidx[i] = s_ceidx[i];
    }
    int* g_mref = at<int>(sm, L.mref);
    long long* g_seref = at<long long>(sm, L.seref);
    long long* g_sqref = at<long long>(sm, L.sqref);
    unsigned long long* g_hwref = at<unsigned long long>(sm, L.hwref);
    long long* g_termref = at<long long>(sm, L.termref);
    uint8_t* g_ninfref = at<uint8_t>(sm, L.ninfref);
    for (int t = tid; t < T; t += nthr) {
      g_mref[t] = s_mref[t];
#pragma unroll
      for (int d = 0; d < DZ; ++d) g_seref[d * T + t] = s_seref[d * T + t];
      g_sqref[t] = s_sqref[t];
      g_hwref[t] = s_hwref[t];
      g_termref[t] = s_termref[t];
      g_ninfref[t] = s_ninfref[t];
    }
  }
  if (tid == 0) {
    sc.ref_score += __double2ll_rn(sc.logw * 4294967296.0);
    if (md.kappa_zero) sc.ninf_ref += sc.nclut_ref;
    else sc.ref_score += (long long)sc.nclut_ref * md.fx_log_kappa;
  }
}

// Persistent: CTA b stages parent b first (the launch spreads CTAs over the
// SMs, so a frame with few parents gets one SM each), then takes the next
// parent from a counter until none is left (parents differ in slots and
// pairs, so a fixed share per CTA would leave SMs idle at the end).
// SMEM: staged in shared memory and copied to the image (16-byte words).
template <int DZ, bool SMEM>
__global__ void __launch_bounds__(256, 3) stage_kernel(const __grid_constant__ ExpandArgs a) {
  pdl_enter();
  extern __shared__ __align__(16) unsigned char sm[];
  const Lay L = make_lay(DZ, a.T_max, a.K_max, a.M_plan);
  // after the staged image (SMEM) or alone: the next-parent word, then the
  // staging's shared scratch (expand_stage_tail_bytes)
  unsigned char* tb = sm + (SMEM ? L.total : 0);
  int& s_next = *reinterpret_cast<int*>(tb);
  const int H = a.fs->H;
  // a table that failed (e.g. pairs beyond capacity, whose offsets then run
  // past the pair arrays) is not staged; the frame is abandoned.  The flags
  // this kernel raises itself (a parent beyond the plan, a bad slot index)
  // are set by its CTAs while others start, so they must not stop a CTA:
  // every parent's counts are recorded
  if (*(volatile const unsigned*)a.err & (kErrFatal & ~(kErrSlots | kErrChkComp))) return;
  for (int h = blockIdx.x; h < H;) {
    unsigned char* img = a.img + (size_t)h * a.img_stride;
    stage_parent<DZ>(a, h, L, SMEM ? sm : img, tb, SMEM ? 0 : a.stage_tail);
    __syncthreads();
    if (SMEM) {
      // a parent whose staging failed copies only its header
      const int bytes = at<Scal>(sm, L.scal)->bad ? (int)sizeof(Scal) : L.total;
      const uint4* src = reinterpret_cast<const uint4*>(sm);
      uint4* dst = reinterpret_cast<uint4*>(img);
      for (int w = threadIdx.x; w < (bytes + 15) / 16; w += blockDim.x) dst[w] = src[w];
    }
    __syncthreads();   // the copy-out has read shared memory, s_next is free
    if (threadIdx.x == 0) s_next = (int)gridDim.x + (int)atomicAdd(a.stage_next, 1u);
    __syncthreads();
    h = s_next;
  }
}

// ====================== draw: one thread per child ======================
// A child's deaths come first: one Philox4x32-10 call per chunk of four
// slots that can die.  Then one categorical draw per detection row with
// candidates, one call per chunk of four rows.  A row keeps its reference
// option when its 24-bit uniform falls in the reference interval and none
// of its candidates died -- nearly always -- so the common path reads one
// 48-byte chunk record and tests four intervals per call, and holds only
// the chunk loop's state in registers.  Everything else about a row is out
// of line (slow_rows): a row with a candidate that may have died is drawn
// among the living, and a row that leaves the reference adds the staged
// change of a single deviation.  Whether a slot died is answered by its
// bloom bit and, when that is set, by regenerating the slot's death draw,
// so a thread keeps no lists.  The slots a child's deviations meet are
// kept as a 64-bit mask (bit slot mod 64): when a bit is met again (a slot
// met twice, or two slots sharing a bit), the slots met more than once are
// rescored exactly after the rows (slow_rows).

// Whether slot t of the child whose death stream is pd died.
__device__ __forceinline__ bool slot_died(const uint32_t* __restrict__ dthr, const PhiloxRun& pd, uint2 key,
                                          uint32_t t) {
  const uint4 r = philox_at_rk(pd, t >> 2, key);
  return (word_of(r, (int)(t & 3u)) >> 8) < dthr[t];
}

// The rows a child's chunk loop noted, in one out-of-line call (the
// parent's layout, view and generators are built once per child): each
// row's uniform is regenerated; a row whose candidates' bloom meets the
// child's dead slots is drawn among the living candidates in proportion to
// their weights (clutter first), in the FP32 arithmetic of the warp kernel;
// otherwise its option is the first whose cumulative threshold exceeds the
// uniform.  A row that leaves its reference option adds the staged changes
// of the slots it leaves and joins (a dead reference slot is not met: its
// change is the death's).  When the deviations meet a slot more than once,
// that slot's change is not the sum of the single changes but the exact
// rescoring of the slot with every detection that joins and leaves it: the
// slots met more than once are rescored with the warp kernel's functions
// and inputs, so the keys are bit-identical.
struct SlowSum {
  long long d;
  unsigned long long hw;
  int ninf, clut, bad;
};

// The score change of one deviation, alone: candidate pair `pos` joining
// (sg = 1) or leaving (sg = -1) slot t, from the slot's reference sums (the
// same function and inputs as an exact rescoring of the slot, so the sums
// are bit-identical); term = the change, ninf = the infinite-term count's.
template <int DZ>
__device__ __noinline__ TermOut single_deviation(const Model* md, const View* vp, int T, int Kp, int t, uint32_t pos,
                                                 int sg) {
  const View& v = *vp;
  long long se[DZ];
#pragma unroll
  for (int d = 0; d < DZ; ++d) se[d] = v.seref[d * T + t] + (long long)sg * fx_of(v.ce[d * Kp + pos]);
  int ninf;
  const long long term =
      slot_term<DZ>(*md, v, T, t, v.mref[t] + sg, se, v.sqref[t] + (long long)sg * fx_of(v.cq[pos]), ninf);
  TermOut o;
  o.term = term - v.termref[t];
  o.ninf = ninf - (int)v.ninfref[t];
  return o;
}

template <int DZ>
__device__ __noinline__ SlowSum slow_rows(const Model* md, const PairTable* pt, const unsigned char* img,
                                          const int Tp, const int Kp, const int Mp, const uint16_t* s_slow,
                                          const int nslow, const int stride, const unsigned long long bloom,
                                          const uint32_t n, const uint2 key) {
  constexpr int kE = 2 * 24;
  const Lay L = make_lay(DZ, Tp, Kp, Mp);
  const View v = make_view(img, L, *pt);
  const Scal& sc = *v.sc;
  const int T = sc.T;
  const uint32_t uid_lo = (uint32_t)sc.uid, uid_hi = (uint32_t)(sc.uid >> 32);
  const PhiloxRun pd = philox_run(uid_lo, uid_hi, 2u * n, key);
  const PhiloxRun pr = philox_run(uid_lo, uid_hi, 2u * n + 1u, key);
  SlowSum o{0, 0ull, 0, 0, 0};
  uint16_t ep_slot[kE];
  uint32_t ep_pos[kE];
  int8_t ep_sg[kE], ep_dn[kE];
  long long ep_d[kE];
  int ne = 0;
  auto single_dev = [&](int t, uint32_t pos, int sg, long long& d, int& dn) {
    const TermOut r = single_deviation<DZ>(md, &v, T, Kp, t, pos, sg);
    d = r.term;
    dn = r.ninf;
  };
  unsigned long long metm = 0ull;
  bool twice = false;
  for (int q = 0; q < nslow; ++q) {
    const int i = s_slow[q * stride];
    const uint4 rr = philox_at_rk(pr, (uint32_t)i >> 2, key);
    const uint32_t k = word_of(rr, i & 3) >> 8;
    const uint4 R = v.row[i];
    const uint32_t off = R.x;
    const int nc = (int)(R.y & 0x7FFFu);
    const int ref = (int)(R.y >> 16);
    int opt = -1;
    if (v.rowbl[i] & bloom) {
      auto is_dead = [&](int j) -> bool {
        const uint32_t t = v.cslot[off + j];
        return ((bloom >> (t & 63u)) & 1ull) && slot_died(v.dthr, pd, key, t);
      };
      uint32_t dm = 0u;
      bool any = false;
      for (int j = 0; j < nc; ++j)
        if (is_dead(j)) {
          any = true;
          if (j < 32) dm |= 1u << j;
        }
      if (any) {
        auto dead_j = [&](int j) -> bool { return j < 32 ? ((dm >> j) & 1u) != 0u : is_dead(j); };
        const float w0 = md->kappa_zero ? 0.f : v.roww0[i];
        float sum = w0;
        for (int j = 0; j < nc; ++j)
          if (!dead_j(j)) sum += v.cw[off + j];
        if (!(sum > 0.f)) {
          o.bad = 1;
          opt = 0;
        } else {
          const float xk = (float)k * 5.9604644775390625e-8f * sum;
          float cum = w0;
          int last = w0 > 0.f ? 0 : -1;
          if (w0 > 0.f && xk < cum) opt = 0;
          for (int j = 0; j < nc; ++j) {
            if (dead_j(j)) continue;
            const float w = v.cw[off + j];
            if (!(w > 0.f)) continue;
            cum += w;
            last = j + 1;
            if (opt < 0 && xk < cum) opt = j + 1;
          }
          if (opt < 0) opt = last < 0 ? 0 : last;
        }
      }
    }
    if (opt < 0) {
      if (k - R.z < R.w - R.z) continue;   // the reference option
      if (k < v.rowthr0[i]) {
        opt = 0;
      } else {
        int j = 0;
        while (j < nc - 1 && k >= v.cthr[off + j]) ++j;
        opt = j + 1;
      }
    }
    if (opt == ref) continue;
    uint32_t rs1 = ref > 0 ? (uint32_t)v.cslot[off + ref - 1] + 1u : 0u;
    const uint32_t ns1 = opt > 0 ? (uint32_t)v.cslot[off + opt - 1] + 1u : 0u;
    o.hw += row_key(i, (int)ns1) - row_key(i, (int)rs1);
    o.clut += (opt == 0) - (ref == 0);
    if (rs1 && ((bloom >> ((rs1 - 1u) & 63u)) & 1ull) && slot_died(v.dthr, pd, key, rs1 - 1u)) rs1 = 0u;
    unsigned long long m1 = 0ull, m2 = 0ull;
    if (rs1) {
      long long d;
      int dn;
      single_dev((int)rs1 - 1, off + (uint32_t)ref - 1u, -1, d, dn);
      o.d += d;
      o.ninf += dn;
      m1 = 1ull << ((rs1 - 1u) & 63u);
      if (ne < kE) {
        ep_slot[ne] = (uint16_t)rs1;
        ep_sg[ne] = -1;
        ep_pos[ne] = off + (uint32_t)ref - 1u;
        ep_d[ne] = d;
        ep_dn[ne] = (int8_t)dn;
        ++ne;
      }
    }
    if (ns1) {
      long long d;
      int dn;
      single_dev((int)ns1 - 1, off + (uint32_t)opt - 1u, 1, d, dn);
      o.d += d;
      o.ninf += dn;
      m2 = 1ull << ((ns1 - 1u) & 63u);
      if (ne < kE) {
        ep_slot[ne] = (uint16_t)ns1;
        ep_sg[ne] = 1;
        ep_pos[ne] = off + (uint32_t)opt - 1u;
        ep_d[ne] = d;
        ep_dn[ne] = (int8_t)dn;
        ++ne;
      }
    }
    twice |= (metm & (m1 | m2)) || (m1 & m2);
    metm |= m1 | m2;
  }
  if (!twice) return o;
  // slots met more than once: exact term minus reference term minus the
  // single changes added above
  for (int w = 0; w < ne; ++w) {
    const uint16_t sp = ep_slot[w];
    int cnt = 0;
    bool first = true;
    for (int w2 = 0; w2 < ne; ++w2)
      if (ep_slot[w2] == sp) {
        ++cnt;
        if (w2 < w) first = false;
      }
    if (cnt < 2 || !first) continue;
    int dcnt = 0, sninf = 0;
    long long dse[DZ], dsq = 0, single = 0;
#pragma unroll
    for (int d = 0; d < DZ; ++d) dse[d] = 0;
    for (int w2 = w; w2 < ne; ++w2) {
      if (ep_slot[w2] != sp) continue;
      const uint32_t pos = ep_pos[w2];
      const int sg = ep_sg[w2];
      single += ep_d[w2];
      sninf += ep_dn[w2];
      dcnt += sg;
#pragma unroll
      for (int d = 0; d < DZ; ++d) dse[d] += sg * fx_of(v.ce[d * Kp + pos]);
      dsq += sg * fx_of(v.cq[pos]);
    }
    const int t = (int)sp - 1;
    long long se[DZ];
#pragma unroll
    for (int d = 0; d < DZ; ++d) se[d] = v.seref[d * T + t] + dse[d];
    int ninf;
    const long long term = slot_term<DZ>(*md, v, T, t, v.mref[t] + dcnt, se, v.sqref[t] + dsq, ninf);
    o.d += term - v.termref[t] - single;
    o.ninf += ninf - (int)v.ninfref[t] - sninf;
  }
  return o;
}

// Rows a child's chunk loop sets aside for slow_rows (per-thread list in
// shared memory, entry q at [q * blockDim.x]); a child with more goes to
// the warp kernel.
constexpr int kDrawSlow = 24;
// Dead slots the first death pass records for the score pass (the same
// kind of per-thread list, after the noted rows); a child with more
// regenerates its death draws instead.
constexpr int kDrawDead = 8;
// chunks per iteration of the draw loop's rows: three (1) or one (0)
constexpr int kDrawPairs = 1;

// Draws child n of the parent staged at img.  The chunk loop only tests the
// reference intervals and notes the rows that need more (their uniform is
// regenerated afterwards), so it holds nothing but its own state in
// registers.  Slots its deviations meet more than once are rescored exactly
// (slow_rows).  Returns false when the child must be drawn by the warp
// kernel: more noted rows than the list holds.
template <int DZ>
__device__ __forceinline__ bool thread_child(const ExpandArgs& a, const unsigned char* img, const Lay& L,
                                             const int h, const int n, const uint2 key, uint16_t* s_slow,
                                             uint16_t* s_dead) {
  const Model& md = a.md;
  const Scal& sc = *at<Scal>(img, L.scal);
  unsigned long long bloom = 0ull;
  int nd = 0;
  {
    // stage 1: deaths; only their bloom (slots with candidate rows) is kept
    // through the chunk loop, their score and key changes are summed after
    const uint32_t* dpc = at<uint32_t>(img, L.dpc);
    const uint32_t* dthr = at<uint32_t>(img, L.dthr);
    const uint8_t* srow = at<uint8_t>(img, L.srow);
    const PhiloxRun pd = philox_run((uint32_t)sc.uid, (uint32_t)(sc.uid >> 32), 2u * (uint32_t)n, key);
    const int ndpc = sc.ndpc;
    auto test_deaths = [&](uint32_t ent, const uint4& r) {
      const uint32_t cc = ent >> 4, mask = ent & 15u;
      const uint4 th = *reinterpret_cast<const uint4*>(dthr + 4 * cc);
#pragma unroll
      for (int b = 0; b < 4; ++b) {
        const uint32_t thb = b == 0 ? th.x : b == 1 ? th.y : b == 2 ? th.z : th.w;
        if (((mask >> b) & 1u) && (word_of(r, b) >> 8) < thb) {
          const uint32_t t = 4u * cc + (uint32_t)b;
          if (nd < kDrawDead) s_dead[nd * (int)blockDim.x] = (uint16_t)t;
          ++nd;
          if (srow[t]) bloom |= 1ull << (t & 63u);
        }
      }
    };
    // two chunks per iteration: two independent Philox chains in flight
    int x = 0;
    for (; x + 1 < ndpc; x += 2) {
      const uint32_t e0 = dpc[x], e1 = dpc[x + 1];
      const uint4 r0 = philox_at(pd, e0 >> 4, key);
      const uint4 r1 = philox_at(pd, e1 >> 4, key);
      test_deaths(e0, r0);
      test_deaths(e1, r1);
    }
    if (x < ndpc) {
      const uint32_t e = dpc[x];
      test_deaths(e, philox_at(pd, e >> 4, key));
    }
  }
  // stage 2: one categorical draw per detection row with candidates; rows
  // outside their reference interval, or whose candidates' bloom meets the
  // dead slots', are noted
  int nslow = 0;
  {
    const PhiloxRun pr = philox_run((uint32_t)sc.uid, (uint32_t)(sc.uid >> 32), 2u * (uint32_t)n + 1u, key);
    const RowChunk* rch = at<RowChunk>(img, L.rch);
    const int nrca = sc.nrca;
    // the interval tests of chunk x with its four words r
    auto test_chunk = [&](int x, uint32_t cc, const uint4& r) {
      const uint4 hd = rch[x].head, base = rch[x].base, span = rch[x].span;
      const uint32_t hit = ((((unsigned long long)hd.w << 32) | hd.z) & bloom) ? hd.y : 0u;
      // bit b: row 4 cc + b left its reference interval
      uint32_t out = 0u;
#pragma unroll
      for (int b = 0; b < 4; ++b)
        if (word_of(r, b) - word_of(base, b) > word_of(span, b)) out |= 1u << b;
      uint32_t look = out | hit;   // nearly always 0: all four keep the reference
      while (look) {
        const int b = __ffs(look) - 1;
        look &= look - 1u;
        const uint32_t i = 4u * cc + (uint32_t)b;
        // a row of a chunk whose bloom meets the dead slots', still in its
        // reference interval: noted only if its own candidates' bloom does
        if (!((out >> b) & 1u) && !(at<unsigned long long>(img, L.rowbl)[i] & bloom)) continue;
        if (nslow < kDrawSlow) s_slow[nslow * (int)blockDim.x] = (uint16_t)i;
        ++nslow;
      }
    };
    int x = 0;
    if (kDrawPairs) {
      // three chunks per iteration: three independent Philox chains in flight
      for (; x + 2 < nrca; x += 3) {
        const uint32_t c0 = rch[x].head.x, c1 = rch[x + 1].head.x, c2 = rch[x + 2].head.x;
        const uint4 r0 = philox_at(pr, c0, key);
        const uint4 r1 = philox_at(pr, c1, key);
        const uint4 r2 = philox_at(pr, c2, key);
        test_chunk(x, c0, r0);
        test_chunk(x + 1, c1, r1);
        test_chunk(x + 2, c2, r2);
      }
    }
    uint32_t cc_next = x < nrca ? rch[x].head.x : 0u;   // one iteration ahead
    for (; x < nrca; ++x) {
      const uint32_t cc = cc_next;
      if (x + 1 < nrca) cc_next = rch[x + 1].head.x;
      test_chunk(x, cc, philox_at(pr, cc, key));
    }
  }
  if (nslow > kDrawSlow) return false;
  // the deaths' score and key changes (a dead slot's change is its dead term)
  unsigned long long hsh = 0ull;
  long long delta = 0;
  int dclut = 0, dninf = 0;
  bool bad_row = false;
  if (nd && nd <= kDrawDead) {
    const long long* deadd = at<long long>(img, L.deadd);
    const int8_t* dninf8 = at<int8_t>(img, L.dninf);
    for (int q = 0; q < nd; ++q) {
      const int t = s_dead[q * (int)blockDim.x];
      hsh += dead_key(t);
      delta += deadd[t];
      dninf += dninf8[t];
    }
  } else if (nd) {
    // more deaths than the list holds: their draws again
    const uint32_t* dpc = at<uint32_t>(img, L.dpc);
    const uint32_t* dthr = at<uint32_t>(img, L.dthr);
    const PhiloxRun pd = philox_run((uint32_t)sc.uid, (uint32_t)(sc.uid >> 32), 2u * (uint32_t)n, key);
    const int ndpc = sc.ndpc;
    int left = nd;
    for (int x = 0; x < ndpc && left; ++x) {
      const uint32_t ent = dpc[x];
      const uint32_t cc = ent >> 4, mask = ent & 15u;
      const uint4 r = philox_at(pd, cc, key);
#pragma unroll
      for (int b = 0; b < 4; ++b) {
        const uint32_t t = 4u * cc + (uint32_t)b;
        if (((mask >> b) & 1u) && (word_of(r, b) >> 8) < dthr[t]) {
          --left;
          hsh += dead_key((int)t);
          delta += at<long long>(img, L.deadd)[t];
          dninf += at<int8_t>(img, L.dninf)[t];
        }
      }
    }
  }
  // the noted rows (out of line, once per child)
  if (nslow) {
    const SlowSum o = slow_rows<DZ>(&md, &a.pt, img, a.T_max, a.K_max, a.M_plan, s_slow, nslow, (int)blockDim.x, bloom,
                                    (uint32_t)n, key);
    hsh += o.hw;
    dclut += o.clut;
    delta += o.d;
    dninf += o.ninf;
    bad_row |= o.bad != 0;
  }
  const long long score = sc.ref_score + delta + (md.kappa_zero ? 0LL : (long long)dclut * md.fx_log_kappa);
  const int ninf = sc.ninf_ref + dninf + (md.kappa_zero ? dclut : 0);
  const bool valid = !bad_row && ninf == 0;
  const size_t j = (size_t)h * md.h_up + n;
  a.child_key[j] = valid ? score : kKeyInvalid;
  a.child_hash[j] = hsh;
  a.child_status[j] = valid ? 1 : 0;
  a.child_alive[j] = (uint16_t)(sc.T - nd);
  return true;
}

int expand_stage_tail_bytes(int dz, int T_plan, int K_plan, int M_plan, int mode) {
  return make_stage_tail(dz, T_plan, K_plan, M_plan, mode).total;
}

int expand_draw_smem(int threads) { return threads * (kDrawSlow + kDrawDead) * (int)sizeof(uint16_t); }

// Persistent over the children of the frame, one thread per child in the
// order parent * h_up + draw (a warp holds 32 consecutive children, of at
// most two parents when h_up >= 32); no block-level synchronisation.
template <int DZ>
__global__ void __launch_bounds__(256, 3) draw_kernel(const __grid_constant__ ExpandArgs a) {
  pdl_enter();
  extern __shared__ __align__(16) unsigned char sm[];
  uint16_t* s_slow = reinterpret_cast<uint16_t*>(sm) + threadIdx.x;
  uint16_t* s_dead = s_slow + kDrawSlow * blockDim.x;
  const Lay L = make_lay(DZ, a.T_max, a.K_max, a.M_plan);
  const int H = a.fs->H, HU = a.md.h_up;
  const uint2 key = make_uint2(a.key_x, a.key_y);
  // a failed table or staging (the frame is redone or abandoned): the
  // images may be stale, so nothing is drawn
  if (*(volatile const unsigned*)a.err & kErrFatal) return;
  const long long total = (long long)H * HU;
  for (long long j = (long long)blockIdx.x * blockDim.x + threadIdx.x; j < total;
       j += (long long)gridDim.x * blockDim.x) {
    const int h = (int)(j / HU);
    const int n = (int)(j - (long long)h * HU);
    const unsigned char* img = a.img + (size_t)h * a.img_stride;
    if (at<Scal>(img, L.scal)->bad) continue;
    if (!thread_child<DZ>(a, img, L, h, n, key, s_slow, s_dead))
      a.redo_list[atomicAdd(a.redo_count, 1u)] = (uint32_t)j;
  }
}

// ====================== warp: one warp per child ======================
// The work area's sums, masks and touched list are zero on entry and are
// left zero on return.
template <int DZ, bool MAT, bool GRP>
__device__ void warp_child(const ExpandArgs& a, const View& v, const int T, const int Kp, const int M,
                           const int h, const int n, const int s_out, const uint2 key, unsigned char* gb,
                           const WLay& WL, const int gsz_in, const int gid) {
  const int gsz = GRP ? gsz_in : 32;   // one warp: the group code folds away
  const Model& md = a.md;
  const Scal& sc = *v.sc;
  const int HU = md.h_up;
  const int lane = threadIdx.x & 31;
  const int gl = (int)threadIdx.x % gsz;   // the thread's index in its group
  unsigned long long* red = at<unsigned long long>(gb, WL.red);
  const int W = (T + 31) >> 5;
  const int nrc = (M + 3) >> 2;
  const uint32_t uid_lo = (uint32_t)sc.uid, uid_hi = (uint32_t)(sc.uid >> 32);
  const int ndpc = sc.ndpc;
  int* acc_cnt = at<int>(gb, WL.cnt);
  long long* acc_se = at<long long>(gb, WL.se);
  long long* acc_sq = at<long long>(gb, WL.sq);
  unsigned long long* acc_hw = at<unsigned long long>(gb, WL.hw);
  uint32_t* newval = at<uint32_t>(gb, WL.newval);
  uint32_t* tmask = at<uint32_t>(gb, WL.tmask);
  uint32_t* dmask = at<uint32_t>(gb, WL.dmask);
  uint32_t* dpre = at<uint32_t>(gb, WL.dpre);
  uint16_t* tlist = at<uint16_t>(gb, WL.tlist);
  int* ntp = at<int>(gb, WL.nt);

  // phase 1: deaths
  int my_dead = 0;
  unsigned long long hsh = 0;
  for (int x = gl; x < ndpc; x += gsz) {
    const uint32_t ent = v.dpc[x];
    const uint32_t cc = ent >> 4, mask = ent & 15u;
    const uint4 r = philox10(make_uint4(uid_lo, uid_hi, 2u * (uint32_t)n, cc), key);
#pragma unroll
    for (int b = 0; b < 4; ++b) {
      if (!((mask >> b) & 1u)) continue;
      const int t = 4 * (int)cc + b;
      if ((word_of(r, b) >> 8) < v.dthr[t]) {
        atomicOr(&dmask[t >> 5], 1u << (t & 31));
        touch(tmask, tlist, ntp, t);
        ++my_dead;
        hsh += dead_key(t);
      }
    }
  }
  group_sync(gsz, gid);
  if (MAT) {
    if (gl < 32) {   // the group's first warp
      uint32_t carry = 0;
      for (int base = 0; base < W; base += 32) {
        const int w = base + lane;
        const uint32_t val = w < W ? (uint32_t)__popc(dmask[w]) : 0u;
        uint32_t x = val;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
          const uint32_t y = __shfl_up_sync(0xFFFFFFFFu, x, o);
          if (lane >= o) x += y;
        }
        if (w < W) dpre[w] = carry + x - val;
        carry += __shfl_sync(0xFFFFFFFFu, x, 31);
      }
    }
    group_sync(gsz, gid);
  }
  // phase 2: one categorical draw per detection row.  The dead slots'
  // bloom (slot mod 64) screens a row's candidates before the exact check;
  // a row none of whose candidates died whose uniform is in its reference
  // interval keeps its reference option without its thresholds
  int my_dclut = 0;
  bool bad_row = false;
  unsigned long long dbl = 0ull;
  for (int w = gl; w < W; w += gsz)
    for (uint32_t m = dmask[w]; m; m &= m - 1u) dbl |= 1ull << ((32 * w + __ffs(m) - 1) & 63);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) dbl |= __shfl_xor_sync(0xFFFFFFFFu, dbl, o);
  if (gsz > 32) {
    if (lane == 0 && dbl) atomicOr(&red[0], dbl);
    group_sync(gsz, gid);
    dbl = red[0];
  }
  const PhiloxRun pr = philox_run(uid_lo, uid_hi, 2u * (uint32_t)n + 1u, key);
  for (int cc = gl; cc < nrc; cc += gsz) {
    const int i0 = 4 * cc;
    const int i1 = min(i0 + 4, M);
    const uint4 r = philox_at(pr, (uint32_t)cc, key);
#pragma unroll
    for (int b = 0; b < 4; ++b) {
      const int i = i0 + b;
      if (i >= i1) break;
      const uint4 R = v.row[i];
      const unsigned long long rbl = v.rowbl[i];
      const uint32_t off = R.x;
      const int nc = (int)(R.y & 0x7FFFu);
      if (nc == 0) {
        if (MAT) a.out_theta[(size_t)s_out * M + i] = 0;
        continue;
      }
      const uint32_t k = word_of(r, b) >> 8;
      bool fast = true;
      if ((R.y & 0x8000u) && (rbl & dbl))
        for (int j = 0; j < nc; ++j)
          if (bit_of(dmask, v.cslot[off + j])) { fast = false; break; }
      int opt;
      if (fast && k - R.z < R.w - R.z) {
        opt = (int)(R.y >> 16);   // the reference option
      } else if (fast) {
        if (k < v.rowthr0[i]) {
          opt = 0;
        } else {
          int j = 0;
          while (j < nc - 1 && k >= v.cthr[off + j]) ++j;
          opt = j + 1;
        }
      } else {
        const float w0 = md.kappa_zero ? 0.f : v.roww0[i];
        float sum = w0;
        for (int j = 0; j < nc; ++j)
          if (!bit_of(dmask, v.cslot[off + j])) sum += v.cw[off + j];
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
            if (bit_of(dmask, v.cslot[off + j])) continue;
            const float w = v.cw[off + j];
            if (!(w > 0.f)) continue;
            cum += w;
            last = j + 1;
            if (opt < 0 && xk < cum) opt = j + 1;
          }
          if (opt < 0) opt = last < 0 ? 0 : last;
        }
      }
      const int ref = (int)(R.y >> 16);
      int ns = -1;
      if (opt > 0) ns = v.cslot[off + opt - 1];
      if (opt != ref) {
        int rs = -1;
        if (ref > 0) {
          rs = v.cslot[off + ref - 1];
          const uint32_t pos = off + ref - 1;
          atomicSub(&acc_cnt[rs], 1);
#pragma unroll
          for (int d = 0; d < DZ; ++d)
            atomicAdd((unsigned long long*)&acc_se[d * T + rs], (unsigned long long)(-fx_of(v.ce[d * Kp + pos])));
          atomicAdd((unsigned long long*)&acc_sq[rs], (unsigned long long)(-fx_of(v.cq[pos])));
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
            atomicAdd((unsigned long long*)&acc_se[d * T + ns], (unsigned long long)fx_of(v.ce[d * Kp + pos]));
          atomicAdd((unsigned long long*)&acc_sq[ns], (unsigned long long)fx_of(v.cq[pos]));
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
  group_sync(gsz, gid);
  // phase 3: rescore touched slots
  const int nt = *((volatile int*)ntp);
  long long my_delta = 0;
  int my_dninf = 0;
  for (int x = gl; x < nt; x += gsz) {
    const int t = tlist[x];
    int ninf;
    long long term;
    long long se[DZ];
    int m = 0;
    const bool is_dead = bit_of(dmask, t);
    if (is_dead) {
      term = dead_term(v.log1mp[t], ninf);
    } else {
      m = v.mref[t] + acc_cnt[t];
#pragma unroll
      for (int d = 0; d < DZ; ++d) se[d] = v.seref[d * T + t] + acc_se[d * T + t];
      term = slot_term<DZ>(md, v, T, t, m, se, v.sqref[t] + acc_sq[t], ninf);
    }
    my_delta += term - v.termref[t];
    my_dninf += ninf - (int)v.ninfref[t];
    if (MAT && !is_dead)
      newval[t] = m >= 1 ? upd_insert<DZ>(a, v.comp[t], v.hwref[t] + acc_hw[t], m, se) : v.comp[t];
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
  bool any_bad = __any_sync(0xFFFFFFFFu, bad_row);
  if (gsz > 32 && !MAT) {
    // the group's totals (integers: the same whatever the order)
    if (lane == 0) {
      atomicAdd(&red[1], (unsigned long long)my_delta);
      atomicAdd(&red[2], (unsigned long long)(long long)my_dninf);
      atomicAdd(&red[3], (unsigned long long)(long long)my_dclut);
      atomicAdd(&red[4], (unsigned long long)(long long)my_dead);
      atomicAdd(&red[5], hsh);
      if (any_bad) atomicOr(&red[6], 1ull);
    }
    group_sync(gsz, gid);
    my_delta = (long long)red[1];
    my_dninf = (int)(long long)red[2];
    my_dclut = (int)(long long)red[3];
    my_dead = (int)(long long)red[4];
    hsh = red[5];
    any_bad = red[6] != 0ull;
  }
  group_sync(gsz, gid);
  if (MAT) {
    const uint32_t base = a.out_ptr[s_out];
    for (int t = gl; t < T; t += gsz) {
      if (bit_of(dmask, t)) continue;
      const uint32_t below = dpre[t >> 5] + __popc(dmask[t >> 5] & ((1u << (t & 31)) - 1u));
      const uint32_t val = bit_of(tmask, t) ? newval[t] : v.refnew[t];
      a.out_comp[base + (uint32_t)t - below] = val;
      if (!(val & kNewTag)) {   // an old component stays
        if (val < (uint32_t)a.fs->T) a.gc_flag[val] = 1u;
        else atomicOr(a.err, kErrChkRemap);
      }
    }
    group_sync(gsz, gid);
  }
  for (int w = gl; w < W; w += gsz) { tmask[w] = 0; dmask[w] = 0; }
  if (GRP && gl < 8) red[gl] = 0ull;   // every reader has passed a barrier since
  if (gl == 0) {
    *ntp = 0;
    if (!MAT) {
      const long long score = sc.ref_score + my_delta + (md.kappa_zero ? 0LL : (long long)my_dclut * md.fx_log_kappa);
      const int ninf = sc.ninf_ref + my_dninf + (md.kappa_zero ? my_dclut : 0);
      const bool valid = !any_bad && ninf == 0;
      const size_t j = (size_t)h * HU + n;
      a.child_key[j] = valid ? score : kKeyInvalid;
      a.child_hash[j] = hsh;
      a.child_status[j] = valid ? 1 : 0;
      a.child_alive[j] = (uint16_t)(T - my_dead);
    }
  }
  group_sync(gsz, gid);
}

// Persistent over a list of children, one group of a.warp_group warps each
// (several when the children are few and long): the survivors (MAT), every
// child of every parent (a.warp_all), or the draw kernel's overflow.
template <int DZ, bool MAT, bool GRP>
__global__ void __launch_bounds__(512) warp_kernel(const __grid_constant__ ExpandArgs a) {
  pdl_enter();
  extern __shared__ __align__(16) unsigned char sm[];
  const Lay L = make_lay(DZ, a.T_max, a.K_max, a.M_plan);
  const WLay WL = make_wlay(DZ, MAT, a.T_max, GRP ? 1 : 0);
  // groups of a.warp_group warps per child, one work area each
  const int gsz = GRP ? 32 * a.warp_group : 32, groups = (int)blockDim.x / gsz;
  const int g = (int)threadIdx.x / gsz, gl = (int)threadIdx.x % gsz;
  const int HU = a.md.h_up, M = a.fs->M;
  const uint2 key = make_uint2(a.key_x, a.key_y);
  // a frame already abandoned (e.g. entries beyond capacity) writes
  // nothing; a failed table or staging leaves the images stale
  if (MAT && (*(volatile unsigned*)a.err & (kErrEntries | kErrSlots | kErrPairs))) return;
  if (!MAT && (*(volatile const unsigned*)a.err & kErrFatal)) return;
  const long long count = MAT ? (long long)*a.n_surv
                              : (a.warp_all ? (long long)a.fs->H * HU : (long long)*a.redo_count);
  // an empty list (the usual overflow case) costs no work-area set-up
  if ((long long)blockIdx.x * groups >= count) return;
  unsigned char* gb = sm + g * WL.total;
  {
    // the sums are indexed d * T + t with each parent's own T <= T_max
    const int Wm = (a.T_max + 31) / 32 + 1;
    int* acc_cnt = at<int>(gb, WL.cnt);
    long long* acc_se = at<long long>(gb, WL.se);
    long long* acc_sq = at<long long>(gb, WL.sq);
    unsigned long long* acc_hw = at<unsigned long long>(gb, WL.hw);
    for (int t = gl; t < a.T_max; t += gsz) {
      acc_cnt[t] = 0;
#pragma unroll
      for (int d = 0; d < DZ; ++d) acc_se[d * a.T_max + t] = 0;
      acc_sq[t] = 0;
      if (MAT) acc_hw[t] = 0;
    }
    for (int w = gl; w < Wm; w += gsz) {
      at<uint32_t>(gb, WL.tmask)[w] = 0;
      at<uint32_t>(gb, WL.dmask)[w] = 0;
    }
    if (gl == 0) *at<int>(gb, WL.nt) = 0;
    if (GRP && gl < 8) at<unsigned long long>(gb, WL.red)[gl] = 0ull;
    group_sync(gsz, g);
  }
  const long long nw = (long long)gridDim.x * groups;
  for (long long c = (long long)blockIdx.x * groups + g; c < count; c += nw) {
    const long long ci = MAT ? a.surv_idx[c] : (a.warp_all ? c : (long long)a.redo_list[c]);
    const int h = (int)(ci / HU), n = (int)(ci % HU);
    const View v = make_view(a.img + (size_t)h * a.img_stride, L, a.pt);
    if (v.sc->bad) continue;
    warp_child<DZ, MAT, GRP>(a, v, v.sc->T, a.K_max, M, h, n, (int)c, key, gb, WL, gsz, g);
  }
}

// The reference association's updated components of every retained parent,
// requested once per parent (one warp per first survivor of a parent).
template <int DZ>
__global__ void __launch_bounds__(256) mat_prep_kernel(const __grid_constant__ ExpandArgs a) {
  pdl_enter();
  const Lay L = make_lay(DZ, a.T_max, a.K_max, a.M_plan);
  const int lane = threadIdx.x & 31;
  const int HU = a.md.h_up;
  // the kept-component flags the materialisation sets: cleared here over
  // the working table only (the next kernel waits for this one)
  for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < a.fs->T; c += gridDim.x * blockDim.x) a.gc_flag[c] = 0u;
  if (*(volatile unsigned*)a.err & (kErrEntries | kErrSlots | kErrPairs)) return;
  const long long count = (long long)*a.n_surv;
  const long long nw = (long long)gridDim.x * (blockDim.x >> 5);
  for (long long c = (long long)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); c < count; c += nw) {
    const int h = (int)(a.surv_idx[c] / HU);
    if (c > 0 && (int)(a.surv_idx[c - 1] / HU) == h) continue;
    unsigned char* img = a.img + (size_t)h * a.img_stride;
    const Scal& sc = *at<Scal>(img, L.scal);
    if (sc.bad) continue;
    const int T = sc.T;
    const int* mref = at<int>(img, L.mref);
    const uint32_t* comp = at<uint32_t>(img, L.comp);
    const long long* seref = at<long long>(img, L.seref);
    const unsigned long long* hwref = at<unsigned long long>(img, L.hwref);
    uint32_t* refnew = at<uint32_t>(img, L.refnew);
    for (int t = lane; t < T; t += 32) {
      long long se[DZ];
#pragma unroll
      for (int d = 0; d < DZ; ++d) se[d] = seref[d * T + t];
      refnew[t] = mref[t] >= 1 ? upd_insert<DZ>(a, comp[t], hwref[t], mref[t], se) : comp[t];
    }
  }
}

// Unique children of each parent (Section 3: only unique hypotheses are
// retained): a valid child whose key equals a lower valid draw's is a
// duplicate; its weight is dropped.  One block per parent: every valid child
// enters an open-addressing table in shared memory (key -> lowest draw).
__device__ __forceinline__ int dedup_table_size(int HU) {
  int ts = 64;
  while (ts < 2 * HU) ts <<= 1;
  return ts;
}

__global__ void __launch_bounds__(128) dedup_kernel(const FrameDev* __restrict__ fs, int HU, long long* child_key,
                                                   const unsigned long long* __restrict__ child_hash,
                                                   int8_t* child_status, const unsigned* err, long long* part_max,
                                                   double* part_sum, unsigned* part_cnt) {
  pdl_enter();
  if (*(volatile const unsigned*)err & kErrFatal) return;   // the draws were skipped
  extern __shared__ unsigned long long s_k[];   // [ts] keys, 0 = empty
  const int ts = dedup_table_size(HU);
  uint32_t* s_n = reinterpret_cast<uint32_t*>(s_k + ts);   // [ts] lowest draw
  __shared__ uint32_t s_zero;                                // lowest draw whose key is 0
  __shared__ long long s_pm[4];
  __shared__ double s_ps[4];
  __shared__ unsigned s_pc[4];
  const int H = fs->H;
  // a block beyond the parents (fixed launches are sized for the most
  // parents a frame can have) holds an empty partial; the selection reads
  // only the first H partials
  if (blockIdx.x >= H) return;
  LseAcc acc;   // this thread's unique children
  for (int h = blockIdx.x; h < H; h += gridDim.x) {
    const size_t base = (size_t)h * HU;
    __syncthreads();
    for (int i = threadIdx.x; i < ts; i += blockDim.x) {
      s_k[i] = 0ull;
      s_n[i] = 0xFFFFFFFFu;
    }
    if (threadIdx.x == 0) s_zero = 0xFFFFFFFFu;
    __syncthreads();
    for (int n = threadIdx.x; n < HU; n += blockDim.x) {
      if (child_status[base + n] == 0) continue;
      const unsigned long long hv = child_hash[base + n];
      if (hv == 0ull) {
        atomicMin(&s_zero, (uint32_t)n);
        continue;
      }
      uint32_t slot = (uint32_t)(hv ^ (hv >> 32)) & (uint32_t)(ts - 1);
      for (int probe = 0; probe < ts; ++probe) {   // ts > entries: a slot is found
        const unsigned long long prev = atomicCAS(&s_k[slot], 0ull, hv);
        if (prev == 0ull || prev == hv) {
          atomicMin(&s_n[slot], (uint32_t)n);
          break;
        }
        slot = (slot + 1u) & (uint32_t)(ts - 1);
      }
    }
    __syncthreads();
    for (int n = threadIdx.x; n < HU; n += blockDim.x) {
      if (child_status[base + n] == 0) continue;
      const unsigned long long hv = child_hash[base + n];
      uint32_t low = s_zero;
      if (hv != 0ull) {
        uint32_t slot = (uint32_t)(hv ^ (hv >> 32)) & (uint32_t)(ts - 1);
        for (int probe = 0; probe < ts && s_k[slot] != hv; ++probe) slot = (slot + 1u) & (uint32_t)(ts - 1);
        low = s_n[slot];
      }
      if (low < (uint32_t)n) {
        child_status[base + n] = 2;
        child_key[base + n] = kKeyInvalid;
      } else {
        acc.add(child_key[base + n]);
      }
    }
  }
  // the block's partial: maximum, sum rescaled to it (FP64), count
  const int lane = threadIdx.x & 31, wp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  long long M = acc.m;
  unsigned c = acc.n;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    M = max(M, __shfl_xor_sync(0xFFFFFFFFu, M, o));
    c += __shfl_xor_sync(0xFFFFFFFFu, c, o);
  }
  if (lane == 0) {
    s_pm[wp] = M;
    s_pc[wp] = c;
  }
  __syncthreads();
  M = s_pm[0];
  c = s_pc[0];
  for (int w = 1; w < nw; ++w) {
    M = max(M, s_pm[w]);
    c += s_pc[w];
  }
  double r = lse_rescale(acc.m, acc.sum(), M);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) r += __shfl_xor_sync(0xFFFFFFFFu, r, o);
  if (lane == 0) s_ps[wp] = r;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < nw; ++w) t += s_ps[w];
    part_max[blockIdx.x] = M;
    part_sum[blockIdx.x] = t;
    part_cnt[blockIdx.x] = c;
  }
}

__global__ void hash_reset_kernel(unsigned long long* hkeys, const uint32_t* __restrict__ upd_slot,
                                  const unsigned* __restrict__ n_prev, int cap_upd, unsigned* n_cur) {
  pdl_enter();
  if (blockIdx.x == 0 && threadIdx.x == 0) *n_cur = 0u;   // this frame's insert counter
  const unsigned n = min(*n_prev, (unsigned)cap_upd);
  for (unsigned i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
    hkeys[upd_slot[i]] = 0ull;
}

void launch_hash_reset(unsigned long long* hkeys, const uint32_t* upd_slot, const unsigned* n_prev, int cap_upd,
                       unsigned* n_cur, int grid, cudaStream_t s) {
  launch_k(hash_reset_kernel, grid, 256, 0, s, hkeys, upd_slot, n_prev, cap_upd, n_cur);
}

void launch_dedup(const FrameDev* fs, int HU, long long* child_key, const unsigned long long* child_hash,
                  int8_t* child_status, const unsigned* err, const PruneWork& w, int grid, cudaStream_t s) {
  int ts = 64;
  while (ts < 2 * HU) ts <<= 1;
  const int smem = ts * 12;
  if (smem > 48 * 1024) cudaFuncSetAttribute(dedup_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  launch_k(dedup_kernel, std::min(grid, kMaxLseParts), 128, smem, s, fs, HU, child_key, child_hash, child_status,
           err, w.part_max, w.part_sum, w.part_cnt);
}

// ---- host side ----
using KernelFn = void (*)(const ExpandArgs);

static KernelFn stage_fn(int dz, bool smem) {
  if (dz == 2) return smem ? stage_kernel<2, true> : stage_kernel<2, false>;
  return smem ? stage_kernel<3, true> : stage_kernel<3, false>;
}
static KernelFn draw_fn(int dz) { return dz == 2 ? draw_kernel<2> : draw_kernel<3>; }
static KernelFn warp_fn(int dz, bool mat, bool grp = false) {
  if (grp) {
    if (dz == 2) return mat ? warp_kernel<2, true, true> : warp_kernel<2, false, true>;
    return mat ? warp_kernel<3, true, true> : warp_kernel<3, false, true>;
  }
  if (dz == 2) return mat ? warp_kernel<2, true, false> : warp_kernel<2, false, false>;
  return mat ? warp_kernel<3, true, false> : warp_kernel<3, false, false>;
}
static KernelFn prep_fn(int dz) { return dz == 2 ? mat_prep_kernel<2> : mat_prep_kernel<3>; }

void expand_init(int smem_limit) {
  for (int dz = 2; dz <= 3; ++dz) {
    cudaFuncSetAttribute(stage_fn(dz, true), cudaFuncAttributeMaxDynamicSharedMemorySize, smem_limit);
    cudaFuncSetAttribute(stage_fn(dz, false), cudaFuncAttributeMaxDynamicSharedMemorySize, smem_limit);
    cudaFuncSetAttribute(draw_fn(dz), cudaFuncAttributeMaxDynamicSharedMemorySize, smem_limit);
    for (int grp = 0; grp < 2; ++grp) {
      cudaFuncSetAttribute(warp_fn(dz, false, grp), cudaFuncAttributeMaxDynamicSharedMemorySize, smem_limit);
      cudaFuncSetAttribute(warp_fn(dz, true, grp), cudaFuncAttributeMaxDynamicSharedMemorySize, smem_limit);
    }
  }
}

static KernelFn kernel_of(const ExpandArgs& a, ExpandKernel k) {
  switch (k) {
    case ExpandKernel::kStage: return stage_fn(a.md.dz, a.stage_smem != 0);
    case ExpandKernel::kDraw: return draw_fn(a.md.dz);
    case ExpandKernel::kWarp: return warp_fn(a.md.dz, a.materialize != 0, a.warp_group > 1);
    default: return prep_fn(a.md.dz);
  }
}

int expand_occupancy(const ExpandArgs& a, ExpandKernel k, int threads, int smem) {
  int per_sm = 0;
  const cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel_of(a, k), threads, smem);
  return e == cudaSuccess ? per_sm : 0;
}

void launch_expand_kernel(const ExpandArgs& a, ExpandKernel k, int grid, int threads, int smem,
                          cudaStream_t s) {
  if (grid <= 0) return;
  launch_k(kernel_of(a, k), grid, threads, smem, s, a);
}

int expand_warp_best_cta(int dz, int materialize, int T, int max_warps, int smem_limit) {
  static std::mutex mu;
  static std::map<std::tuple<int, int, int, int, int>, int> memo;
  const auto key = std::make_tuple(dz, materialize, T, max_warps, smem_limit);
  std::lock_guard<std::mutex> lock(mu);
  auto it = memo.find(key);
  if (it != memo.end()) return it->second;
  int best = 0, best_res = 0;
  for (int g = 1; g <= max_warps; ++g) {
    const int smem = expand_warp_smem(dz, materialize, T, g, 0);
    if (smem > smem_limit) break;
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, warp_fn(dz, materialize != 0), 32 * g, smem) !=
        cudaSuccess)
      per_sm = 0;
    if (per_sm * g >= best_res && per_sm > 0) {   // ties: the larger CTA
      best_res = per_sm * g;
      best = g;
    }
  }
  cudaGetLastError();
  memo[key] = best;
  return best;
}

bool expand_kernel_takes_key(const void* fn) {
  for (int dz = 2; dz <= 3; ++dz)
    if (fn == (const void*)draw_fn(dz) || fn == (const void*)warp_fn(dz, false) || fn == (const void*)warp_fn(dz, true) ||
        fn == (const void*)warp_fn(dz, false, true) || fn == (const void*)warp_fn(dz, true, true))
      return true;
  return false;
}

}  // namespace glmb

// Learned pair gate: a 5-64-64-64-1 multilayer perceptron with GELU
// activations, bf16 weights and fp32 accumulation, scoring every pair of
// the compatibility table (Eq. 2) that passes the Mahalanobis test; with
// the gate on, a pair stays in the table only when its logit reaches the
// threshold.  This extends the paper's gate g_ijk (Section 3), a plain
// threshold, with a model trained on which pairs the retained hypotheses of
// the ungated filter use.
//
// Layers 1-3 run on the 5th-generation tensor cores: 128 pairs per tile
// (one row per thread of a 128-thread CTA), operands staged in shared
// memory in the canonical no-swizzle K-major layout, tcgen05.mma issued by
// one thread with the accumulator (128 lanes x 64 fp32 columns) in tensor
// memory, completion signalled on an mbarrier, tcgen05.ld back to
// registers for the bias + GELU epilogue.  The output layer is a 64-term
// dot product per row.  Training runs the same forward pass, then the
// backward pass: activation gradients through the tensor cores (dz * W with
// W transposed in shared memory), weight gradients on the CUDA cores from
// the tile's activations, accumulated per CTA and added once to global
// memory; Adam updates the fp32 master parameters.
#include <cuda_bf16.h>

#include "glmb_kernels.h"

namespace glmb {

namespace {

constexpr int kTile = 128;        // rows (pairs) per tile = MMA M
constexpr int kHid = 64;          // hidden width = MMA N
constexpr int kIn = 5;            // features
constexpr int kIn16 = 16;         // layer-1 K, padded to one bf16 MMA step
constexpr int kZPitch = 65;       // fp32 row pitch of the saved pre-activations

// canonical no-swizzle K-major layout of a bf16 operand with kc8 = K / 8
// core matrices per row group: element (r, k) of core matrix (r/8, k/8),
// each core matrix 8 rows x 16 bytes stored contiguously
__device__ __forceinline__ uint32_t core_off(int r, int k, int kc8) {
  return (uint32_t)((((r >> 3) * kc8 + (k >> 3)) << 7) + ((r & 7) << 4) + ((k & 7) << 1));
}

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

// shared-memory matrix descriptor of tcgen05: start address, leading
// (K-direction core matrix) byte offset, stride (8-row group) byte offset,
// descriptor version 1, no swizzle
__device__ __forceinline__ uint64_t mdesc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
  return (uint64_t)((addr & 0x3FFFFu) >> 4) | ((uint64_t)((lbo & 0x3FFFFu) >> 4) << 16) |
         ((uint64_t)((sbo & 0x3FFFFu) >> 4) << 32) | (1ull << 46);
}

// instruction descriptor of kind::f16: fp32 accumulator, bf16 A and B,
// both K-major, N = 64, M = 128
constexpr uint32_t kIdesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(kHid >> 3) << 17) |
                            ((uint32_t)(kTile >> 4) << 24);

__device__ __forceinline__ void mma_issue(uint32_t tmem, uint64_t a, uint64_t b, uint32_t acc) {
  asm volatile(
      "{\n\t.reg .pred p;\n\tsetp.ne.u32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(tmem),
      "l"(a), "l"(b), "r"(kIdesc), "r"(acc));
}

__device__ __forceinline__ void mma_commit(uint32_t mbar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(mbar)
               : "memory");
}

__device__ __forceinline__ void fence_before() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void fence_after() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}
// generic-proxy shared-memory writes made visible to the tensor cores
__device__ __forceinline__ void fence_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// waits for the mbarrier phase with the given parity; gives up after
// `limit` SM clock cycles, about a second by default (returns false)
__device__ __forceinline__ bool mbar_wait(uint32_t mbar, uint32_t parity, long long limit = kGateWaitLimit) {
  const long long t0 = clock64();
  for (;;) {
    uint32_t done;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}\n"
        : "=r"(done)
        : "r"(mbar), "r"(parity)
        : "memory");
    if (done) return true;
    if (clock64() - t0 > limit) return false;
  }
}

// 16 consecutive fp32 columns of this thread's TMEM lane
__device__ __forceinline__ void tmem_ld16(uint32_t addr, float (&v)[16]) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, "
      "%12, %13, %14, %15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
        "=r"(r[14]), "=r"(r[15])
      : "r"(addr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int j = 0; j < 16; ++j) v[j] = __uint_as_float(r[j]);
}

__device__ __forceinline__ float bf16r(float x) { return __bfloat162float(__float2bfloat16_rn(x)); }

__device__ __forceinline__ float gelu_f(float x) { return 0.5f * x * (1.f + erff(x * 0.70710678118654752f)); }

__device__ __forceinline__ float gelu_grad_f(float x) {
  return 0.5f * (1.f + erff(x * 0.70710678118654752f)) + x * 0.39894228040143268f * expf(-0.5f * x * x);
}

// eight values as bf16 into one 16-byte core-matrix row
__device__ __forceinline__ void st_core8(unsigned char* base, uint32_t off, const float* v) {
  __nv_bfloat162 p[4];
#pragma unroll
  for (int j = 0; j < 4; ++j) p[j] = __floats2bfloat162_rn(v[2 * j], v[2 * j + 1]);
  *reinterpret_cast<uint4*>(base + off) = *reinterpret_cast<const uint4*>(p);
}

__device__ __forceinline__ void ld_core8(const unsigned char* base, uint32_t off, float* v) {
  const uint4 q = *reinterpret_cast<const uint4*>(base + off);
  const __nv_bfloat162* p = reinterpret_cast<const __nv_bfloat162*>(&q);
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    const float2 f = __bfloat1622float2(p[j]);
    v[2 * j] = f.x;
    v[2 * j + 1] = f.y;
  }
}

// shared-memory plan (bytes); matrices on 1024-byte boundaries
struct GLay {
  static constexpr int W1 = 0, W2 = 2048, W3 = W2 + 8192;
  static constexpr int W2T = W3 + 8192, W3T = W2T + 8192;       // training only
  static constexpr int A0 = W3T + 8192;                          // 128 x 16 bf16
  static constexpr int H1 = A0 + 4096, H2 = H1 + 16384;          // 128 x 64 bf16
  static constexpr int DZ = H2 + 16384;                          // training only
  static constexpr int Z1 = DZ + 16384;                          // fp32 128 x 65, training only
  static constexpr int Z2 = Z1 + kTile * kZPitch * 4, Z3 = Z2 + kTile * kZPitch * 4;
  static constexpr int CST = Z3 + kTile * kZPitch * 4;           // b1 b2 b3 w4(bf16) mu sd b4
  static constexpr int DL = CST + 272 * 4;                       // per-row output gradient
  static constexpr int MBAR = DL + kTile * 4;
  static constexpr int TSLOT = MBAR + 8, FLAG = TSLOT + 4;
  static constexpr int TOTAL = FLAG + 12;
};
// the forward kernel uses W1..W3, A0, H1 (both hidden layers) and the constants
struct FLay {
  static constexpr int W1 = 0, W2 = 2048, W3 = W2 + 8192, A0 = W3 + 8192, H1 = A0 + 4096;
  static constexpr int CST = H1 + 16384, MBAR = CST + 272 * 4, TSLOT = MBAR + 8, FLAG = TSLOT + 4;
  static constexpr int TOTAL = FLAG + 12;
};

constexpr int kCB1 = 0, kCB2 = 64, kCB3 = 128, kCW4 = 192, kCMu = 256, kCSd = 261, kCB4 = 266;

// stages the weights (rounded to bf16) into the operand layouts and the
// vectors into the constant block; transposed copies of W2 and W3 when
// w2t/w3t are given
__device__ void stage_weights(const float* __restrict__ P, unsigned char* sm, int w1, int w2, int w3,
                              int w2t, int w3t, float* cst) {
  for (int idx = threadIdx.x; idx < kHid * kIn16; idx += blockDim.x) {
    const int o = idx / kIn16, j = idx % kIn16;
    const float v = j < kIn ? P[kGateW1 + o * kIn + j] : 0.f;
    *reinterpret_cast<__nv_bfloat16*>(sm + w1 + core_off(o, j, 2)) = __float2bfloat16_rn(v);
  }
  for (int idx = threadIdx.x; idx < kHid * kHid; idx += blockDim.x) {
    const int o = idx / kHid, j = idx % kHid;
    const __nv_bfloat16 a = __float2bfloat16_rn(P[kGateW2 + idx]);
    const __nv_bfloat16 b = __float2bfloat16_rn(P[kGateW3 + idx]);
    *reinterpret_cast<__nv_bfloat16*>(sm + w2 + core_off(o, j, 8)) = a;
    *reinterpret_cast<__nv_bfloat16*>(sm + w3 + core_off(o, j, 8)) = b;
    if (w2t >= 0) *reinterpret_cast<__nv_bfloat16*>(sm + w2t + core_off(j, o, 8)) = a;
    if (w3t >= 0) *reinterpret_cast<__nv_bfloat16*>(sm + w3t + core_off(j, o, 8)) = b;
  }
  for (int idx = threadIdx.x; idx < kHid; idx += blockDim.x) {
    cst[kCB1 + idx] = P[kGateB1 + idx];
    cst[kCB2 + idx] = P[kGateB2 + idx];
    cst[kCB3 + idx] = P[kGateB3 + idx];
    cst[kCW4 + idx] = bf16r(P[kGateW4 + idx]);
  }
  if (threadIdx.x < kIn) {
    cst[kCMu + threadIdx.x] = P[kGateMu + threadIdx.x];
    cst[kCSd + threadIdx.x] = P[kGateSd + threadIdx.x];
  }
  if (threadIdx.x == 0) cst[kCB4] = P[kGateB4];
}

// TMEM: warp 0 allocates 64 columns for the CTA, then lets the other CTAs
// of the SM allocate
__device__ __forceinline__ void tmem_alloc(uint32_t* slot) {
  if (threadIdx.x < 32) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(slot)),
                 "r"(kHid));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
}
__device__ __forceinline__ void tmem_free(uint32_t taddr) {
  if (threadIdx.x < 32) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(kHid));
}

__device__ __forceinline__ void mbar_init(uint32_t mbar) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(mbar) : "memory");
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

// one layer on the tensor cores: D[128 x 64] = A[128 x 16 ksteps] * B^T,
// A and B K-major with kc8 = 2 * ksteps core matrices per row group;
// issued by thread 0, completion on mbar
__device__ __forceinline__ void layer_mma(uint32_t tmem, uint32_t a, uint32_t b, int ksteps, uint32_t mbar) {
  if (threadIdx.x == 0) {
    fence_after();
    const uint32_t sbo = (uint32_t)(ksteps * 2) << 7;
    for (int k = 0; k < ksteps; ++k)
      mma_issue(tmem, mdesc(a + (uint32_t)k * 256u, 128u, sbo), mdesc(b + (uint32_t)k * 256u, 128u, sbo),
                k > 0 ? 1u : 0u);
    mma_commit(mbar);
  }
}

// every thread waits for the layer; a time-out anywhere aborts the CTA
__device__ __forceinline__ bool layer_wait(uint32_t mbar, uint32_t& parity, int* flag,
                                           long long limit = kGateWaitLimit) {
  const bool ok = mbar_wait(mbar, parity, limit);
  parity ^= 1u;
  if (!ok) atomicOr(flag, 1);
  fence_after();
  return __syncthreads_or(!ok) == 0;
}

// epilogue of a hidden layer for this thread's row: z = acc + b, GELU,
// bf16 into the next layer's operand; z saved (fp32) when zrow is given
__device__ __forceinline__ void hidden_epilogue(uint32_t trow, const float* b, float* zrow, unsigned char* dst,
                                                int m) {
#pragma unroll 1
  for (int c0 = 0; c0 < kHid; c0 += 16) {
    float v[16];
    tmem_ld16(trow + (uint32_t)c0, v);
#pragma unroll
    for (int j = 0; j < 16; ++j) {
      const float z = v[j] + b[c0 + j];
      if (zrow) zrow[c0 + j] = z;
      v[j] = gelu_f(z);
    }
    st_core8(dst, core_off(m, c0, 8), v);
    st_core8(dst, core_off(m, c0 + 8, 8), v + 8);
  }
}

// standardised features of one row as bf16 into the layer-1 operand
__device__ __forceinline__ void write_input(unsigned char* a0, int m, const float* f, bool valid,
                                            const float* cst) {
  float v[16];
#pragma unroll
  for (int j = 0; j < 16; ++j) v[j] = 0.f;
  if (valid) {
#pragma unroll
    for (int j = 0; j < kIn; ++j) v[j] = (f[j] - cst[kCMu + j]) / cst[kCSd + j];
  }
  st_core8(a0, core_off(m, 0, 2), v);
  st_core8(a0, core_off(m, 8, 2), v + 8);
}

// component of pair p: the c with ptr[c] <= p < ptr[c + 1]
__device__ __forceinline__ int pair_comp(const uint32_t* __restrict__ ptr, int T, uint32_t p) {
  int lo = 0, hi = T;  // invariant ptr[lo] <= p < ptr[hi]
  while (hi - lo > 1) {
    const int mid = (lo + hi) >> 1;
    if (__ldg(ptr + mid) <= p) lo = mid;
    else hi = mid;
  }
  return lo;
}

}  // namespace

// the gate's raw features of pair p: d^2 (recovered from log C and log det
// S), innovation norm, prior existence, age in frames, log det S
__device__ __forceinline__ void pair_features(const Model& md, const CompTable& ct, const PairTable& pt,
                                              const FrameDev& fs, uint32_t p, int c, float* f) {
  const float ld = pt.logdetS[c];
  const float c0 = md.log_pd - 0.5f * (ld + (float)md.dz * kLog2Pi);
  float n2 = 0.f;
  for (int a = 0; a < md.dz; ++a) {
    const float e = pt.e[(size_t)a * (size_t)pt.cap_pairs + p];
    n2 += e * e;
  }
  f[0] = fmaxf(2.f * (c0 - pt.logC[p]), 0.f);
  f[1] = sqrtf(n2);
  f[2] = expf(ct.logp[c]);
  f[3] = (float)((uint32_t)fs.frame - ct.lk[c]);
  f[4] = ld;
}

// ---------------------------------------------------------------------------
// forward pass: rows from a feature array (X [n][5]) or from the pair table
// ---------------------------------------------------------------------------
struct GateFwdArgs {
  const float* P;
  const float* X;
  long long n;
  // table mode
  Model md;
  CompTable ct;
  PairTable pt;
  const FrameDev* fs;
  float thr;
  uint8_t* keep;
  float* logit;
  unsigned* err;
  long long wait_limit;   // SM clock cycles a completion wait may take
  int skip_first_mma;     // failure-detection test: CTA 0 issues no MMA for its first tile
};

template <bool kTable>
__global__ void __launch_bounds__(kTile) gate_forward_kernel(GateFwdArgs g) {
  pdl_enter();
  extern __shared__ __align__(1024) unsigned char sm[];
  float* cst = reinterpret_cast<float*>(sm + FLay::CST);
  uint32_t* tslot = reinterpret_cast<uint32_t*>(sm + FLay::TSLOT);
  int* flag = reinterpret_cast<int*>(sm + FLay::FLAG);
  const uint32_t mbar = smem_u32(sm + FLay::MBAR);
  const int m = threadIdx.x, warp = m >> 5;
  long long n = g.n;
  int T = 0;
  if (kTable) {
    // a table that overflowed its capacity (the frame is abandoned) is
    // scored only up to the capacity
    T = g.fs->T;
    n = min((long long)g.pt.ptr[T], g.pt.cap_pairs);
  }
  const long long tiles = (n + kTile - 1) / kTile;
  if ((long long)blockIdx.x >= tiles) return;
  if (m == 0) {
    *flag = 0;
    mbar_init(mbar);
  }
  tmem_alloc(tslot);
  stage_weights(g.P, sm, FLay::W1, FLay::W2, FLay::W3, -1, -1, cst);
  fence_async_smem();
  fence_before();
  __syncthreads();
  fence_after();
  const uint32_t tmem = *tslot;
  const uint32_t trow = tmem + ((uint32_t)(warp * 32) << 16);
  const uint32_t a0 = smem_u32(sm + FLay::A0), h1 = smem_u32(sm + FLay::H1);
  uint32_t parity = 0;
  bool ok = true;
  for (long long tile = blockIdx.x; tile < tiles && ok; tile += gridDim.x) {
    const long long row = tile * kTile + m;
    const bool valid = row < n;
    float f[kIn] = {0.f, 0.f, 0.f, 0.f, 0.f};
    if (valid) {
      if (kTable) {
        const int c = pair_comp(g.pt.ptr, T, (uint32_t)row);
        pair_features(g.md, g.ct, g.pt, *g.fs, (uint32_t)row, c, f);
      } else {
#pragma unroll
        for (int j = 0; j < kIn; ++j) f[j] = g.X[row * kIn + j];
      }
    }
    write_input(sm + FLay::A0, m, f, valid, cst);
    fence_async_smem();
    __syncthreads();
    if (!(g.skip_first_mma && blockIdx.x == 0 && tile == blockIdx.x))
      layer_mma(tmem, a0, smem_u32(sm + FLay::W1), 1, mbar);
    if (!(ok = layer_wait(mbar, parity, flag, g.wait_limit))) break;
    hidden_epilogue(trow, cst + kCB1, nullptr, sm + FLay::H1, m);
    fence_before();
    fence_async_smem();
    __syncthreads();
    layer_mma(tmem, h1, smem_u32(sm + FLay::W2), 4, mbar);
    if (!(ok = layer_wait(mbar, parity, flag, g.wait_limit))) break;
    // layer 2's activations overwrite its own operand once the MMA is done
    hidden_epilogue(trow, cst + kCB2, nullptr, sm + FLay::H1, m);
    fence_before();
    fence_async_smem();
    __syncthreads();
    layer_mma(tmem, h1, smem_u32(sm + FLay::W3), 4, mbar);
    if (!(ok = layer_wait(mbar, parity, flag, g.wait_limit))) break;
    float z = cst[kCB4];
#pragma unroll 1
    for (int c0 = 0; c0 < kHid; c0 += 16) {
      float v[16];
      tmem_ld16(trow + (uint32_t)c0, v);
#pragma unroll
      for (int j = 0; j < 16; ++j) z += bf16r(gelu_f(v[j] + cst[kCB3 + c0 + j])) * cst[kCW4 + c0 + j];
    }
    if (valid) {
      if (g.logit) g.logit[row] = z;
      if (kTable && g.keep) g.keep[row] = z >= g.thr ? 1 : 0;
    }
    fence_before();
    __syncthreads();
  }
  if (!ok) {
    // an MMA may still be in flight: give it one more bounded wait
    mbar_wait(mbar, parity ^ 1u, g.wait_limit);
    if (m == 0) atomicOr(g.err, kErrGate);
  }
  fence_before();
  __syncthreads();
  fence_after();
  tmem_free(tmem);
}

// ---------------------------------------------------------------------------
// training: forward, weighted binary cross-entropy, backward
// ---------------------------------------------------------------------------
struct GateTrainArgs {
  const float* P;
  const float* X;
  const float* y;
  const float* wt;
  long long n;
  float* grad;
  double* loss;
  unsigned* err;
};

__global__ void __launch_bounds__(kTile, 1) gate_train_kernel(GateTrainArgs g) {
  pdl_enter();
  extern __shared__ __align__(1024) unsigned char sm[];
  float* cst = reinterpret_cast<float*>(sm + GLay::CST);
  float* dl = reinterpret_cast<float*>(sm + GLay::DL);
  float* Z1 = reinterpret_cast<float*>(sm + GLay::Z1);
  float* Z2 = reinterpret_cast<float*>(sm + GLay::Z2);
  float* Z3 = reinterpret_cast<float*>(sm + GLay::Z3);
  uint32_t* tslot = reinterpret_cast<uint32_t*>(sm + GLay::TSLOT);
  int* flag = reinterpret_cast<int*>(sm + GLay::FLAG);
  const uint32_t mbar = smem_u32(sm + GLay::MBAR);
  const int m = threadIdx.x, warp = m >> 5;
  const long long tiles = (g.n + kTile - 1) / kTile;
  if ((long long)blockIdx.x >= tiles) return;
  if (m == 0) {
    *flag = 0;
    mbar_init(mbar);
  }
  tmem_alloc(tslot);
  stage_weights(g.P, sm, GLay::W1, GLay::W2, GLay::W3, GLay::W2T, GLay::W3T, cst);
  fence_async_smem();
  fence_before();
  __syncthreads();
  fence_after();
  const uint32_t tmem = *tslot;
  const uint32_t trow = tmem + ((uint32_t)(warp * 32) << 16);
  // weight-gradient ownership: output unit o, inputs [i0, i0 + 32)
  const int o = m >> 1, i0 = (m & 1) * 32;
  float gW3[32], gW2[32], gW1[3];
#pragma unroll
  for (int j = 0; j < 32; ++j) gW3[j] = gW2[j] = 0.f;
  gW1[0] = gW1[1] = gW1[2] = 0.f;
  float gB1 = 0.f, gB2 = 0.f, gB3 = 0.f, gW4 = 0.f, gB4 = 0.f;
  double loss = 0.0;
  uint32_t parity = 0;
  bool ok = true;
  for (long long tile = blockIdx.x; tile < tiles && ok; tile += gridDim.x) {
    const long long row = tile * kTile + m;
    const bool valid = row < g.n;
    const int nv = (int)min((long long)kTile, g.n - tile * kTile);
    float f[kIn] = {0.f, 0.f, 0.f, 0.f, 0.f};
    if (valid) {
#pragma unroll
      for (int j = 0; j < kIn; ++j) f[j] = g.X[row * kIn + j];
    }
    write_input(sm + GLay::A0, m, f, valid, cst);
    fence_async_smem();
    __syncthreads();
    // ---- forward ----
    layer_mma(tmem, smem_u32(sm + GLay::A0), smem_u32(sm + GLay::W1), 1, mbar);
    if (!(ok = layer_wait(mbar, parity, flag))) break;
    hidden_epilogue(trow, cst + kCB1, Z1 + m * kZPitch, sm + GLay::H1, m);
    fence_before();
    fence_async_smem();
    __syncthreads();
    layer_mma(tmem, smem_u32(sm + GLay::H1), smem_u32(sm + GLay::W2), 4, mbar);
    if (!(ok = layer_wait(mbar, parity, flag))) break;
    hidden_epilogue(trow, cst + kCB2, Z2 + m * kZPitch, sm + GLay::H2, m);
    fence_before();
    fence_async_smem();
    __syncthreads();
    layer_mma(tmem, smem_u32(sm + GLay::H2), smem_u32(sm + GLay::W3), 4, mbar);
    if (!(ok = layer_wait(mbar, parity, flag))) break;
    float z = cst[kCB4];
#pragma unroll 1
    for (int c0 = 0; c0 < kHid; c0 += 16) {
      float v[16];
      tmem_ld16(trow + (uint32_t)c0, v);
#pragma unroll
      for (int j = 0; j < 16; ++j) {
        const float zz = v[j] + cst[kCB3 + c0 + j];
        Z3[m * kZPitch + c0 + j] = zz;
        z += bf16r(gelu_f(zz)) * cst[kCW4 + c0 + j];
      }
    }
    // ---- loss and output gradient ----
    float d = 0.f;
    if (valid) {
      const float yy = g.y[row], w = g.wt[row];
      const float sp = fmaxf(z, 0.f) + log1pf(expf(-fabsf(z)));
      loss += (double)w * (double)(sp - yy * z);
      d = w * (1.f / (1.f + expf(-z)) - yy);
    }
    dl[m] = d;
    fence_before();
    __syncthreads();
    // ---- output layer gradients (h3 recomputed from z3) ----
    {
      const int nn = m & 63, half = m >> 6;
      const int r0 = half * 64, r1 = min(nv, r0 + 64);
      for (int r = r0; r < r1; ++r) gW4 += dl[r] * bf16r(gelu_f(Z3[r * kZPitch + nn]));
      if (m == 0)
        for (int r = 0; r < nv; ++r) gB4 += dl[r];
    }
    __syncthreads();
    // ---- layer 3: dz3 = dl * w4 * GELU'(z3); dh2 = dz3 W3 on the tensor cores ----
    {
      float v[8];
#pragma unroll 1
      for (int c0 = 0; c0 < kHid; c0 += 8) {
#pragma unroll
        for (int j = 0; j < 8; ++j) {
          const float dz = dl[m] * cst[kCW4 + c0 + j] * gelu_grad_f(Z3[m * kZPitch + c0 + j]);
          Z3[m * kZPitch + c0 + j] = dz;
          v[j] = dz;
        }
        st_core8(sm + GLay::DZ, core_off(m, c0, 8), v);
      }
    }
    fence_async_smem();
    __syncthreads();
    layer_mma(tmem, smem_u32(sm + GLay::DZ), smem_u32(sm + GLay::W3T), 4, mbar);
    for (int r = 0; r < nv; ++r) {           // dW3, db3 while the MMA runs
      const float dz = Z3[r * kZPitch + o];
      float h[32];
#pragma unroll
      for (int q = 0; q < 4; ++q) ld_core8(sm + GLay::H2, core_off(r, i0 + 8 * q, 8), h + 8 * q);
#pragma unroll
      for (int j = 0; j < 32; ++j) gW3[j] += dz * h[j];
      if (i0 == 0) gB3 += dz;
    }
    if (!(ok = layer_wait(mbar, parity, flag))) break;
#pragma unroll 1
    for (int c0 = 0; c0 < kHid; c0 += 16) {
      float v[16];
      tmem_ld16(trow + (uint32_t)c0, v);
#pragma unroll
      for (int j = 0; j < 16; ++j) {
        v[j] *= gelu_grad_f(Z2[m * kZPitch + c0 + j]);
        Z2[m * kZPitch + c0 + j] = v[j];
      }
      st_core8(sm + GLay::DZ, core_off(m, c0, 8), v);
      st_core8(sm + GLay::DZ, core_off(m, c0 + 8, 8), v + 8);
    }
    fence_before();
    fence_async_smem();
    __syncthreads();
    // ---- layer 2: dh1 = dz2 W2; dW2, db2 ----
    layer_mma(tmem, smem_u32(sm + GLay::DZ), smem_u32(sm + GLay::W2T), 4, mbar);
    for (int r = 0; r < nv; ++r) {
      const float dz = Z2[r * kZPitch + o];
      float h[32];
#pragma unroll
      for (int q = 0; q < 4; ++q) ld_core8(sm + GLay::H1, core_off(r, i0 + 8 * q, 8), h + 8 * q);
#pragma unroll
      for (int j = 0; j < 32; ++j) gW2[j] += dz * h[j];
      if (i0 == 0) gB2 += dz;
    }
    if (!(ok = layer_wait(mbar, parity, flag))) break;
#pragma unroll 1
    for (int c0 = 0; c0 < kHid; c0 += 16) {
      float v[16];
      tmem_ld16(trow + (uint32_t)c0, v);
#pragma unroll
      for (int j = 0; j < 16; ++j) Z1[m * kZPitch + c0 + j] = v[j] * gelu_grad_f(Z1[m * kZPitch + c0 + j]);
    }
    fence_before();
    __syncthreads();
    // ---- layer 1: dW1, db1 ----
    {
      const int j0 = (m & 1) ? 3 : 0, nj = (m & 1) ? 2 : 3;
      for (int r = 0; r < nv; ++r) {
        const float dz = Z1[r * kZPitch + o];
        float x[8];
        ld_core8(sm + GLay::A0, core_off(r, 0, 2), x);
        for (int j = 0; j < nj; ++j) gW1[j] += dz * x[j0 + j];
        if (i0 == 0) gB1 += dz;
      }
    }
    __syncthreads();
  }
  if (!ok) {
    mbar_wait(mbar, parity ^ 1u);
    if (m == 0) atomicOr(g.err, kErrGate);
  } else {
#pragma unroll 4
    for (int j = 0; j < 32; ++j) {
      atomicAdd(g.grad + kGateW3 + o * kHid + i0 + j, gW3[j]);
      atomicAdd(g.grad + kGateW2 + o * kHid + i0 + j, gW2[j]);
    }
    const int j0 = (m & 1) ? 3 : 0, nj = (m & 1) ? 2 : 3;
    for (int j = 0; j < nj; ++j) atomicAdd(g.grad + kGateW1 + o * kIn + j0 + j, gW1[j]);
    if (i0 == 0) {
      atomicAdd(g.grad + kGateB1 + o, gB1);
      atomicAdd(g.grad + kGateB2 + o, gB2);
      atomicAdd(g.grad + kGateB3 + o, gB3);
    }
    atomicAdd(g.grad + kGateW4 + (m & 63), gW4);
    if (m == 0) atomicAdd(g.grad + kGateB4, gB4);
    // loss: warp sums, then one atomic per warp
    for (int off = 16; off > 0; off >>= 1) loss += __shfl_xor_sync(0xFFFFFFFFu, loss, off);
    if ((m & 31) == 0) atomicAdd(g.loss, loss);
  }
  fence_before();
  __syncthreads();
  fence_after();
  tmem_free(tmem);
}

// Adam (Kingma and Ba 2015) on the trained parameters, bias-corrected
__global__ void gate_adam_kernel(float* __restrict__ P, const float* __restrict__ G, float* __restrict__ mo,
                                 float* __restrict__ ve, int t, float lr, float b1, float b2, float eps) {
  pdl_enter();
  const float c1 = 1.f - powf(b1, (float)t), c2 = 1.f - powf(b2, (float)t);
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < kGateNTrain; i += gridDim.x * blockDim.x) {
    const float gi = G[i];
    const float mi = b1 * mo[i] + (1.f - b1) * gi;
    const float vi = b2 * ve[i] + (1.f - b2) * gi * gi;
    mo[i] = mi;
    ve[i] = vi;
    P[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
  }
}

// raw features of every pair of the table (rows for training)
__global__ void gate_features_kernel(Model md, CompTable ct, PairTable pt, const FrameDev* __restrict__ fs,
                                     float* __restrict__ X, long long cap) {
  pdl_enter();
  const int T = fs->T;
  const long long n = min((long long)pt.ptr[T], cap);
  for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < n;
       p += (long long)gridDim.x * blockDim.x) {
    float f[kIn];
    pair_features(md, ct, pt, *fs, (uint32_t)p, pair_comp(pt.ptr, T, (uint32_t)p), f);
    for (int j = 0; j < kIn; ++j) X[p * kIn + j] = f[j];
  }
}

// kept pairs per component (warp per component)
__global__ void gate_count_kernel(PairTable full, const uint8_t* __restrict__ keep, PairTable gated,
                                  const FrameDev* __restrict__ fs) {
  pdl_enter();
  const int T = fs->T, lane = threadIdx.x & 31;
  const int nw = (gridDim.x * blockDim.x) >> 5;
  for (int c = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; c < T; c += nw) {
    const uint32_t cap = (uint32_t)full.cap_pairs;
    const uint32_t lo = min(full.ptr[c], cap), hi = min(full.ptr[c + 1], cap);
    unsigned k = 0;
    for (uint32_t j = lo + lane; j < hi; j += 32) k += keep[j];
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) k += __shfl_xor_sync(0xFFFFFFFFu, k, off);
    if (lane == 0) gated.cnt[c] = k;
  }
}

// stable compaction of the kept pairs into the gated table, and the death
// probability (reading R2) over the pairs that remain
__global__ void gate_compact_kernel(Model md, CompTable ct, PairTable full, const uint8_t* __restrict__ keep,
                                    PairTable gated, const FrameDev* __restrict__ fs) {
  pdl_enter();
  const int T = fs->T, lane = threadIdx.x & 31, dz = md.dz;
  const int nw = (gridDim.x * blockDim.x) >> 5;
  const size_t cf = (size_t)full.cap_pairs, cg = (size_t)gated.cap_pairs;
  for (int c = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; c < T; c += nw) {
    const uint32_t lo = min(full.ptr[c], (uint32_t)cf), hi = min(full.ptr[c + 1], (uint32_t)cf);
    uint32_t out = gated.ptr[c];
    float lm = -INFINITY, ls = 0.f;
    bool any = false;
    for (uint32_t j0 = lo; j0 < hi; j0 += 32) {
      const uint32_t j = j0 + lane;
      const bool k = j < hi && keep[j];
      const unsigned bal = __ballot_sync(0xFFFFFFFFu, k);
      const uint32_t q = out + __popc(bal & ((1u << lane) - 1u));
      if (k && q < cg) {
        const float lc = full.logC[j];
        gated.meas[q] = full.meas[j];
        gated.logC[q] = lc;
        gated.q[q] = full.q[j];
        for (int a = 0; a < dz; ++a) gated.e[a * cg + q] = full.e[a * cf + j];
        any = true;
        if (!md.kappa_zero) lse_push(lm, ls, lc - md.log_kappa);
      }
      out += __popc(bal);
    }
    lse_warp(lm, ls);
    const bool any_w = __any_sync(0xFFFFFFFFu, any);
    if (lane == 0) death_prob(md, ct.logp[c], ct.log1mp[c], lm, ls, any_w, gated.dprob[c], gated.dthr[c]);
  }
}

// Which pairs of the last update's table the retained hypotheses use (the
// gate's training labels), and which retained hypotheses use a pair whose
// logit is below the threshold.  One block per retained hypothesis: its new
// tracks are its parent's surviving slots in slot order, so walking both
// lists by label recovers each track's predicted component; theta then names
// the pair (component, detection), found by binary search in the component's
// slice (detections ascend within it).
__global__ void gate_usage_kernel(HypTable par, HypTable out, CompTable A, CompTable B,
                                  const long long* __restrict__ surv, int H_new, int h_up, int M,
                                  PairTable pt, const FrameDev* __restrict__ fs, const float* __restrict__ logit,
                                  float thr, uint8_t* __restrict__ used, uint8_t* __restrict__ hflag, int capT) {
  pdl_enter();
  extern __shared__ int kc[];
  const int n_comp = fs->n_comp, nb = fs->nb;
  for (int j = blockIdx.x; j < H_new; j += gridDim.x) {
    if (threadIdx.x == 0) {
      const int p = (int)(surv[j] / h_up);
      const uint32_t plo = par.ptr[p];
      const int Tp = (int)(par.ptr[p + 1] - plo), Ts = Tp + nb;
      const uint32_t lo = out.ptr[j], hi = out.ptr[j + 1];
      int s = 0;
      for (uint32_t e = lo; e < hi && (int)(e - lo) < capT; ++e) {
        const uint32_t ca = out.comp[e];
        const uint32_t lk = A.lk[ca], lb = A.lb[ca];
        int c = -1;
        while (s < Ts) {
          const int cs = s < Tp ? (int)par.comp[plo + s] : n_comp + (s - Tp);
          ++s;
          if (B.lk[cs] == lk && B.lb[cs] == lb) {
            c = cs;
            break;
          }
        }
        kc[e - lo] = c;
      }
    }
    __syncthreads();
    const int nt = min((int)(out.ptr[j + 1] - out.ptr[j]), capT);
    int bad = 0;
    for (int i = threadIdx.x; i < M; i += blockDim.x) {
      const int t = out.theta[(size_t)j * M + i];
      if (t == 0 || t > nt) continue;
      const int c = kc[t - 1];
      if (c < 0) continue;
      uint32_t lo = pt.ptr[c], hi = pt.ptr[c + 1];
      const uint32_t end = hi;
      while (lo < hi) {
        const uint32_t mid = (lo + hi) >> 1;
        if (pt.meas[mid] < (uint32_t)i) lo = mid + 1;
        else hi = mid;
      }
      if (lo < end && pt.meas[lo] == (uint32_t)i) {
        if (used) used[lo] = 1;
        if (logit && logit[lo] < thr) bad = 1;
      }
    }
    bad = __syncthreads_or(bad);
    if (threadIdx.x == 0 && hflag) hflag[j] = (uint8_t)bad;
  }
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
int gate_forward_smem() { return FLay::TOTAL; }
int gate_train_smem() { return GLay::TOTAL; }

static bool gate_attrs_set = false;
static void gate_attrs() {
  if (gate_attrs_set) return;
  cudaFuncSetAttribute(gate_train_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, GLay::TOTAL);
  cudaFuncSetAttribute(gate_forward_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, FLay::TOTAL);
  cudaFuncSetAttribute(gate_forward_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, FLay::TOTAL);
  gate_attrs_set = true;
}

void launch_gate_forward_rows(const float* P, const float* X, long long n, float* logit, unsigned* err, int grid,
                              cudaStream_t s) {
  gate_attrs();
  GateFwdArgs g{};
  g.P = P;
  g.X = X;
  g.n = n;
  g.logit = logit;
  g.err = err;
  const WaitTest wt = wait_test();
  g.wait_limit = wt.mode == kWaitTestGate ? wt.limit : kGateWaitLimit;
  g.skip_first_mma = wt.mode == kWaitTestGate ? 1 : 0;
  launch_k(gate_forward_kernel<false>, grid, kTile, FLay::TOTAL, s, g);
}

void launch_gate_forward_table(const float* P, float thr, const Model& md, const CompTable& ct,
                               const PairTable& full, const FrameDev* fs, float* logit, uint8_t* keep,
                               unsigned* err, int grid, cudaStream_t s) {
  gate_attrs();
  GateFwdArgs g{};
  g.P = P;
  g.md = md;
  g.ct = ct;
  g.pt = full;
  g.fs = fs;
  g.thr = thr;
  g.keep = keep;
  g.logit = logit;
  g.err = err;
  const WaitTest wt = wait_test();
  g.wait_limit = wt.mode == kWaitTestGate ? wt.limit : kGateWaitLimit;
  g.skip_first_mma = wt.mode == kWaitTestGate ? 1 : 0;
  launch_k(gate_forward_kernel<true>, grid, kTile, FLay::TOTAL, s, g);
}

void launch_gate_train(const float* P, const float* X, const float* y, const float* wt, long long n,
                       float* grad, double* loss, unsigned* err, int grid, cudaStream_t s) {
  gate_attrs();
  GateTrainArgs g{P, X, y, wt, n, grad, loss, err};
  launch_k(gate_train_kernel, grid, kTile, GLay::TOTAL, s, g);
}

void launch_gate_adam(float* P, const float* G, float* m, float* v, int t, float lr, float b1, float b2,
                      float eps, cudaStream_t s) {
  launch_k(gate_adam_kernel, (kGateNTrain + 255) / 256, 256, 0, s, P, G, m, v, t, lr, b1, b2, eps);
}

void launch_gate_features(const Model& md, const CompTable& ct, const PairTable& pt, const FrameDev* fs,
                          float* X, long long cap, int grid, cudaStream_t s) {
  launch_k(gate_features_kernel, grid, 256, 0, s, md, ct, pt, fs, X, cap);
}

void launch_gate_compact(const Model& md, const CompTable& ct, const PairTable& full, const uint8_t* keep,
                         const PairTable& gated, const FrameDev* fs, bool count, int grid, cudaStream_t s) {
  if (count) launch_k(gate_count_kernel, grid, 256, 0, s, full, keep, gated, fs);
  else launch_k(gate_compact_kernel, grid, 256, 0, s, md, ct, full, keep, gated, fs);
}

void launch_gate_usage(const HypTable& par, const HypTable& out, const CompTable& A, const CompTable& B,
                       const long long* surv, int H_new, int h_up, int M, const PairTable& pt, const FrameDev* fs,
                       const float* logit, float thr, uint8_t* used, uint8_t* hflag, int capT, int grid,
                       cudaStream_t s) {
  const size_t smem = (size_t)capT * sizeof(int);
  if (smem > 48 * 1024) cudaFuncSetAttribute(gate_usage_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  launch_k(gate_usage_kernel, grid, 128, smem, s, par, out, A, B, surv, H_new, h_up, M, pt, fs, logit, thr, used,
           hflag, capT);
}

}  // namespace glmb

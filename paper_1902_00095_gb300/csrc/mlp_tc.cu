// Inference of the learned Schur correction's MLP (24 -> 64 -> 64 -> 8, GELU)
// on the fifth-generation tensor cores: tcgen05.mma with BF16 operands in
// shared memory and FP32 accumulators in tensor memory (TMEM).
//
// One CTA of 128 threads takes a tile of 128 cells (the MMA's M). The
// weights (packed once in the operand layout) and the tile's FP32 features
// arrive by bulk copy (cp.async.bulk) on an mbarrier; operands are staged in
// the no-swizzle K-major layout of 8-row x 16-byte core
// matrices: element (r, k) of an R x K tile sits at byte
// ((r / 8) * (K / 8) + k / 8) * 128 + (r % 8) * 16 + (k % 8) * 2, so core
// matrices adjacent along K are 128 bytes apart (the descriptor's leading
// byte offset) and those adjacent along M or N are K * 16 bytes apart (its
// stride byte offset); one MMA with K = 16 reads two core matrices along K.
// Layer l's accumulator occupies its own TMEM columns (0-63, 64-127,
// 128-143 of 256 allocated); thread t of warp w reads TMEM lane 32 w + t,
// i.e. cell t of the warp's 32, adds the bias, applies GELU and writes the
// BF16 activation as the next layer's A operand. One elected thread issues
// the MMAs and commits them to an mbarrier that all threads wait on, with a
// bounded spin that records a timeout in an error word.
#include <cstdint>
#include <atomic>

#include "learned.cuh"

namespace tp {

namespace {

constexpr int kTcRows = 128;
constexpr int kTcThreads = 128;
constexpr uint32_t kTcCols = 256;
// shared-memory map (bytes)
constexpr uint32_t kOffX = 0;                         // [128 x 32]
constexpr uint32_t kOffH1 = kOffX + 128 * 32 * 2;     // [128 x 64]
constexpr uint32_t kOffH2 = kOffH1 + 128 * 64 * 2;    // [128 x 64]
constexpr uint32_t kOffW1 = kOffH2 + 128 * 64 * 2;    // [64 x 32]
constexpr uint32_t kOffW2 = kOffW1 + 64 * 32 * 2;     // [64 x 64]
constexpr uint32_t kOffW3 = kOffW2 + 64 * 64 * 2;     // [16 x 64]
constexpr uint32_t kOffXf = kOffW3 + 16 * 64 * 2;     // [128 x 24] FP32 features (bulk copy)
constexpr uint32_t kOffBar = kOffXf + 128 * 24 * 4;   // MMA mbarrier, copy mbarrier, TMEM base
constexpr uint32_t kTcSmemUsed = kOffBar + 32;
static_assert(kOffW2 - kOffW1 == 64 * 32 * 2 && kOffW3 - kOffW1 == (64 * 32 + 64 * 64) * 2,
              "weights must be laid out as in MlpDev::Wtc");
// requested dynamic shared memory: more than a third of the SM's, so at
// most two CTAs share an SM and their TMEM (2 x 256 of 512 columns)
constexpr uint32_t kTcSmem = 96 * 1024;
static_assert(kTcSmemUsed <= kTcSmem, "shared-memory map exceeds the request");

__device__ __forceinline__ uint32_t core_off(int r, int k, int K) { return mlp_core_off(r, k, K); }

// one-dimensional bulk copy global -> shared, completing on an mbarrier
// (addresses and size multiples of 16 bytes)
__device__ __forceinline__ void bulk_copy(uint32_t dst, const void* src, uint32_t bytes,
                                          uint32_t bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];\n" ::"r"(
          dst),
      "l"(src), "r"(bytes), "r"(bar)
      : "memory");
}

__device__ __forceinline__ uint64_t smem_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
  uint64_t d = (uint64_t)((saddr >> 4) & 0x3FFFu);
  d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
  d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
  d |= (uint64_t)1 << 46;  // descriptor version of the tcgen05 family; no swizzle
  return d;
}

// kind::f16 instruction descriptor: FP32 accumulate, BF16 A and B, both
// K-major, shape M x N
__host__ __device__ constexpr uint32_t instr_desc(int M, int N) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) |
         ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void mma_bf16(uint32_t dtmem, uint64_t adesc, uint64_t bdesc,
                                         uint32_t idesc, uint32_t accumulate) {
  asm volatile(
      "{\n"
      ".reg .pred p;\n"
      "setp.ne.b32 p, %4, 0;\n"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n"
      "}\n" ::"r"(dtmem),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate));
}

__device__ __forceinline__ void mma_commit(uint32_t bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(
                   bar)
               : "memory");
}

__device__ __forceinline__ bool bar_try_wait(uint32_t bar, uint32_t parity) {
  uint32_t ok = 0;
  asm volatile(
      "{\n"
      ".reg .pred p;\n"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
      "selp.u32 %0, 1, 0, p;\n"
      "}\n"
      : "=r"(ok)
      : "r"(bar), "r"(parity)
      : "memory");
  return ok != 0;
}

// wait for the given phase parity, at most ~2^22 polls; a timeout sets err
__device__ __forceinline__ void bar_wait(uint32_t bar, uint32_t parity, int* err) {
  for (int it = 0; it < (1 << 22); ++it)
    if (bar_try_wait(bar, parity)) return;
  atomicOr(err, 1);
}

__device__ __forceinline__ void fence_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
}
__device__ __forceinline__ void tc_fence_before() {
  asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() {
  asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
}

// 16 consecutive FP32 accumulator columns of this thread's TMEM lane
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float* v) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,"
      "%15}, [%16];\n"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
        "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
#pragma unroll
  for (int j = 0; j < 16; ++j) v[j] = __uint_as_float(r[j]);
}

__device__ __forceinline__ float gelu_tc(float x) {
  const float c = 0.7978845608028654f;  // sqrt(2 / pi)
  return 0.5f * x * (1.0f + tanhf(c * (x + 0.044715f * x * x * x)));
}

__global__ void __launch_bounds__(kTcThreads) k_mlp_forward_tc(MlpDev m, int n,
                                                               const float* __restrict__ X,
                                                               int x_bulk,
                                                               float* __restrict__ O,
                                                               int* __restrict__ err) {
  extern __shared__ __align__(1024) unsigned char smem[];
  const int tid = threadIdx.x, warp = tid >> 5;
  const uint32_t sbase = (uint32_t)__cvta_generic_to_shared(smem);
  const uint32_t bar = sbase + kOffBar;        // MMA completions
  const uint32_t cbar = sbase + kOffBar + 8;   // bulk copies
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(smem + kOffBar + 16);
  const int row0 = blockIdx.x * kTcRows;
  const int rows = min(kTcRows, n - row0);
  const uint32_t xbytes = x_bulk ? (uint32_t)rows * kMlpIn * 4 : 0u;  // multiple of 16

  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(bar) : "memory");
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(cbar) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    // weights (already in the operand layout) and this tile's features by
    // the bulk-copy engine, both completing on cbar
    const uint32_t wbytes = (uint32_t)kMlpTcWeights * 2;
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(cbar),
                 "r"(wbytes + xbytes)
                 : "memory");
    bulk_copy(sbase + kOffW1, m.Wtc, wbytes, cbar);
    if (xbytes) bulk_copy(sbase + kOffXf, X + (size_t)row0 * kMlpIn, xbytes, cbar);
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(
                     sbase + kOffBar + 16),
                 "r"(kTcCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::: "memory");
  }
  __syncthreads();  // barrier initialisation visible before anyone waits on it
  bar_wait(cbar, 0, err);
  // this thread's cell: features as BF16, K padded to 32 with zeros
  const int row = row0 + tid;
  const float* xf = reinterpret_cast<const float*>(smem + kOffXf) + tid * kMlpIn;
  __nv_bfloat16* sX = reinterpret_cast<__nv_bfloat16*>(smem + kOffX);
  for (int k = 0; k < 32; ++k) {
    float v = 0.f;
    if (row < n && k < kMlpIn) v = x_bulk ? xf[k] : X[(size_t)row * kMlpIn + k];
    sX[core_off(tid, k, 32) / 2] = __float2bfloat16_rn(v);
  }
  fence_async_smem();
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;
  const uint32_t lane_addr = tmem + ((uint32_t)(warp * 32) << 16);

  __nv_bfloat16* sH1 = reinterpret_cast<__nv_bfloat16*>(smem + kOffH1);
  __nv_bfloat16* sH2 = reinterpret_cast<__nv_bfloat16*>(smem + kOffH2);
  const float* b1 = m.params + kOffB1;
  const float* b2 = m.params + kOffB2;
  const float* b3 = m.params + kOffB3;

  // layer 1: [128 x 32] x [32 x 64] -> TMEM columns 0..63
  if (tid == 0) {
    for (int kk = 0; kk < 2; ++kk)
      mma_bf16(tmem, smem_desc(sbase + kOffX + kk * 256, 128, 4 * 128),
               smem_desc(sbase + kOffW1 + kk * 256, 128, 4 * 128), instr_desc(128, 64), kk > 0);
    mma_commit(bar);
  }
  bar_wait(bar, 0, err);
  tc_fence_after();
  for (int c0 = 0; c0 < 64; c0 += 16) {
    float v[16];
    tmem_ld16(lane_addr + c0, v);
#pragma unroll
    for (int j = 0; j < 16; ++j)
      sH1[core_off(tid, c0 + j, 64) / 2] = __float2bfloat16_rn(gelu_tc(v[j] + b1[c0 + j]));
  }
  fence_async_smem();
  tc_fence_before();
  __syncthreads();
  tc_fence_after();

  // layer 2: [128 x 64] x [64 x 64] -> TMEM columns 64..127
  if (tid == 0) {
    for (int kk = 0; kk < 4; ++kk)
      mma_bf16(tmem + 64, smem_desc(sbase + kOffH1 + kk * 256, 128, 8 * 128),
               smem_desc(sbase + kOffW2 + kk * 256, 128, 8 * 128), instr_desc(128, 64), kk > 0);
    mma_commit(bar);
  }
  bar_wait(bar, 1, err);
  tc_fence_after();
  for (int c0 = 0; c0 < 64; c0 += 16) {
    float v[16];
    tmem_ld16(lane_addr + 64 + c0, v);
#pragma unroll
    for (int j = 0; j < 16; ++j)
      sH2[core_off(tid, c0 + j, 64) / 2] = __float2bfloat16_rn(gelu_tc(v[j] + b2[c0 + j]));
  }
  fence_async_smem();
  tc_fence_before();
  __syncthreads();
  tc_fence_after();

  // layer 3: [128 x 64] x [64 x 16] -> TMEM columns 128..143 (8 used)
  if (tid == 0) {
    for (int kk = 0; kk < 4; ++kk)
      mma_bf16(tmem + 128, smem_desc(sbase + kOffH2 + kk * 256, 128, 8 * 128),
               smem_desc(sbase + kOffW3 + kk * 256, 128, 8 * 128), instr_desc(128, 16), kk > 0);
    mma_commit(bar);
  }
  bar_wait(bar, 0, err);
  tc_fence_after();
  {
    float v[16];
    tmem_ld16(lane_addr + 128, v);
    if (row < n) {
#pragma unroll
      for (int j = 0; j < kMlpOut; ++j) O[(size_t)row * kMlpOut + j] = v[j] + b3[j];
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem),
                 "r"(kTcCols)
                 : "memory");
}

}  // namespace

void mlp_forward_tc(const MlpDev& m, int n, const float* X, float* O, int* err, cudaStream_t s) {
  if (n <= 0) return;
  // the large dynamic shared memory is an opt-in of the current device:
  // set once per device ordinal
  static std::atomic<bool> opted[64];
  int dev = 0;
  TP_CUDA_TRY(cudaGetDevice(&dev));
  if (dev < 0 || dev >= 64 || !opted[dev].load(std::memory_order_acquire)) {
    TP_CUDA_TRY(cudaFuncSetAttribute(k_mlp_forward_tc, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)kTcSmem));
    if (dev >= 0 && dev < 64) opted[dev].store(true, std::memory_order_release);
  }
  const int blocks = (n + kTcRows - 1) / kTcRows;
  // the features' tile is bulk-copied when X is 16-byte aligned (every
  // tile then starts on a 96-byte row boundary and spans whole rows)
  const int x_bulk = (reinterpret_cast<uintptr_t>(X) & 15) == 0 ? 1 : 0;
  k_mlp_forward_tc<<<blocks, kTcThreads, kTcSmem, s>>>(m, n, X, x_bulk, O, err);
  TP_LAUNCH_CHECK();
}

}  // namespace tp

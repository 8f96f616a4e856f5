// Inference of the learned Schur correction's MLP (24 -> 64 -> 64 -> 8, GELU)
// on the fifth-generation tensor cores: tcgen05.mma with BF16 operands in
// shared memory and FP32 accumulators in tensor memory (TMEM).
//
// One CTA of 128 threads takes a tile of 128 cells (the MMA's M). Operands
// are staged in the no-swizzle K-major layout of 8-row x 16-byte core
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
constexpr uint32_t kOffBar = kOffW3 + 16 * 64 * 2;    // mbarrier (8 B) + TMEM base (4 B)
constexpr uint32_t kTcSmemUsed = kOffBar + 16;
// requested dynamic shared memory: more than a third of the SM's, so at
// most two CTAs share an SM and their TMEM (2 x 256 of 512 columns)
constexpr uint32_t kTcSmem = 96 * 1024;
static_assert(kTcSmemUsed <= kTcSmem, "shared-memory map exceeds the request");

__device__ __forceinline__ uint32_t core_off(int r, int k, int K) {
  return (uint32_t)(((r >> 3) * (K >> 3) + (k >> 3)) * 128 + (r & 7) * 16 + (k & 7) * 2);
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
                                                               float* __restrict__ O,
                                                               int* __restrict__ err) {
  extern __shared__ __align__(1024) unsigned char smem[];
  const int tid = threadIdx.x, warp = tid >> 5;
  const uint32_t sbase = (uint32_t)__cvta_generic_to_shared(smem);
  const uint32_t bar = sbase + kOffBar;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(smem + kOffBar + 8);

  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(bar) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(
                     sbase + kOffBar + 8),
                 "r"(kTcCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::: "memory");
  }
  // weights into the core-matrix layout (W3 padded to 16 rows with zeros)
  __nv_bfloat16* sW1 = reinterpret_cast<__nv_bfloat16*>(smem + kOffW1);
  __nv_bfloat16* sW2 = reinterpret_cast<__nv_bfloat16*>(smem + kOffW2);
  __nv_bfloat16* sW3 = reinterpret_cast<__nv_bfloat16*>(smem + kOffW3);
  for (int p = tid; p < 64 * 32; p += kTcThreads) {
    const int r = p / 32, k = p % 32;
    sW1[core_off(r, k, 32) / 2] = m.W1[p];
  }
  for (int p = tid; p < 64 * 64; p += kTcThreads) {
    const int r = p / 64, k = p % 64;
    sW2[core_off(r, k, 64) / 2] = m.W2[p];
  }
  for (int p = tid; p < 16 * 64; p += kTcThreads) {
    const int r = p / 64, k = p % 64;
    sW3[core_off(r, k, 64) / 2] = r < kMlpOut ? m.W3[r * 64 + k] : __float2bfloat16_rn(0.f);
  }
  // this thread's cell: features as BF16, K padded to 32 with zeros
  const int row = blockIdx.x * kTcRows + tid;
  __nv_bfloat16* sX = reinterpret_cast<__nv_bfloat16*>(smem + kOffX);
  for (int k = 0; k < 32; ++k) {
    const float v = (row < n && k < kMlpIn) ? X[(size_t)row * kMlpIn + k] : 0.f;
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
  static const bool attr = []() {
    TP_CUDA_TRY(cudaFuncSetAttribute(k_mlp_forward_tc, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)kTcSmem));
    return true;
  }();
  (void)attr;
  const int blocks = (n + kTcRows - 1) / kTcRows;
  k_mlp_forward_tc<<<blocks, kTcThreads, kTcSmem, s>>>(m, n, X, O, err);
  TP_LAUNCH_CHECK();
}

}  // namespace tp

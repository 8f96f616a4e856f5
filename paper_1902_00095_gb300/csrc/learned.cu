// Learned correction of the Schur approximation: per-cell features, the
// training of a 24 -> 64 -> 64 -> 8 GELU MLP (forward and backward of
// 16-sample warp tiles with mma.sync m16n8k16, BF16 operands, FP32
// accumulation), Adam, and the corrected S~_T (Eq. Se) with a per-row
// guard. Inference over all cells runs on tcgen05 (mlp_tc.cu).
//
// Row i of S~_T becomes S_ii <- S~_ii exp(o_0) + o_7 S~_ii and
// S_ij <- S~_ij exp(o_d) for face direction d = 1..6 of neighbour j; the
// network is trained on exact Schur complement entries (Eq. Afact) with the
// loss mean(((S_learned,ij - S_ij) / S_ii)^2).
//
// One warp owns 16 samples (rows of the M = 16 tile). Activations stay in
// registers between layers: the accumulator layout of m16n8 tiles n and n+1
// is the A-operand layout of one k16 chunk. Weight gradients reduce over
// the warp's 16 samples with the same instruction (A = dZ^T, B = H, staged
// through shared memory), one partial per warp, summed in a fixed order.
#include <cuda_bf16.h>
#include "learned.cuh"

namespace tp {

namespace {

constexpr float kGeluC = 0.7978845608028654f;  // sqrt(2 / pi)

__device__ __forceinline__ float gelu_f(float x) {
  return 0.5f * x * (1.0f + tanhf(kGeluC * (x + 0.044715f * x * x * x)));
}

__device__ __forceinline__ float gelu_grad_f(float x) {
  const float u = kGeluC * (x + 0.044715f * x * x * x);
  const float t = tanhf(u);
  return 0.5f * (1.0f + t) + 0.5f * x * (1.0f - t * t) * kGeluC * (1.0f + 3.0f * 0.044715f * x * x);
}

__device__ __forceinline__ unsigned pack_bf16(float lo, float hi) {
  __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
  return *reinterpret_cast<unsigned*>(&v);
}

__device__ __forceinline__ unsigned pack_raw(__nv_bfloat16 lo, __nv_bfloat16 hi) {
  __nv_bfloat162 v;
  v.x = lo;
  v.y = hi;
  return *reinterpret_cast<unsigned*>(&v);
}

// D = A (16x16 bf16, row) * B (16x8 bf16, col) + C, FP32 accumulate
__device__ __forceinline__ void mma16816(float* d, unsigned a0, unsigned a1, unsigned a2,
                                         unsigned a3, unsigned b0, unsigned b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, "
      "{%8,%9}, {%0,%1,%2,%3};\n"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
}

// B fragment of a row-major weight W[N][K] (bf16) used as the col-major K x N
// operand: column n = n0 + g, rows k = k0 + 2t, 2t+1 and k0 + 2t + 8, +9
__device__ __forceinline__ void load_b(const __nv_bfloat16* __restrict__ W, int ldk, int n0,
                                       int k0, int g, int t, unsigned& b0, unsigned& b1) {
  const __nv_bfloat16* p = W + (size_t)(n0 + g) * ldk + k0 + 2 * t;
  b0 = *reinterpret_cast<const unsigned*>(p);
  b1 = *reinterpret_cast<const unsigned*>(p + 8);
}

struct Tile {
  float z1[8][4], z2[8][4], o[4];
  unsigned h1[4][4], h2[4][4];  // A fragments of gelu(z1), gelu(z2)
  unsigned x[2][4];             // A fragments of the features (K padded to 32)
};

// forward pass of 16 samples starting at row r0 (rows >= n read as zero)
__device__ __forceinline__ void mlp_forward_tile(const MlpDev& m, const float* __restrict__ X,
                                                 int n, int r0, int g, int t, Tile& T) {
  // features -> A fragments (rows g, g + 8; cols 2t, 2t+1, +8, +9 per k16)
  const int ra = r0 + g, rb = r0 + g + 8;
#pragma unroll
  for (int kc = 0; kc < 2; ++kc) {
    float v[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      const int row = (q & 2) ? rb : ra;
      const int c = kc * 16 + 2 * t + (q & 1) + ((q & 4) ? 8 : 0);
      v[q] = (row < n && c < kMlpIn) ? X[(size_t)row * kMlpIn + c] : 0.0f;
    }
    T.x[kc][0] = pack_bf16(v[0], v[1]);
    T.x[kc][1] = pack_bf16(v[2], v[3]);
    T.x[kc][2] = pack_bf16(v[4], v[5]);
    T.x[kc][3] = pack_bf16(v[6], v[7]);
  }
  const float* b1 = m.params + kOffB1;
  const float* b2 = m.params + kOffB2;
  const float* b3 = m.params + kOffB3;
  // layer 1
#pragma unroll
  for (int nt = 0; nt < 8; ++nt) {
    const float bl = b1[nt * 8 + 2 * t], bh = b1[nt * 8 + 2 * t + 1];
    T.z1[nt][0] = bl; T.z1[nt][1] = bh; T.z1[nt][2] = bl; T.z1[nt][3] = bh;
#pragma unroll
    for (int kc = 0; kc < 2; ++kc) {
      unsigned bb0, bb1;
      load_b(m.W1, kMlpInPad, nt * 8, kc * 16, g, t, bb0, bb1);
      mma16816(T.z1[nt], T.x[kc][0], T.x[kc][1], T.x[kc][2], T.x[kc][3], bb0, bb1);
    }
  }
#pragma unroll
  for (int kc = 0; kc < 4; ++kc) {
    T.h1[kc][0] = pack_bf16(gelu_f(T.z1[2 * kc][0]), gelu_f(T.z1[2 * kc][1]));
    T.h1[kc][1] = pack_bf16(gelu_f(T.z1[2 * kc][2]), gelu_f(T.z1[2 * kc][3]));
    T.h1[kc][2] = pack_bf16(gelu_f(T.z1[2 * kc + 1][0]), gelu_f(T.z1[2 * kc + 1][1]));
    T.h1[kc][3] = pack_bf16(gelu_f(T.z1[2 * kc + 1][2]), gelu_f(T.z1[2 * kc + 1][3]));
  }
  // layer 2
#pragma unroll
  for (int nt = 0; nt < 8; ++nt) {
    const float bl = b2[nt * 8 + 2 * t], bh = b2[nt * 8 + 2 * t + 1];
    T.z2[nt][0] = bl; T.z2[nt][1] = bh; T.z2[nt][2] = bl; T.z2[nt][3] = bh;
#pragma unroll
    for (int kc = 0; kc < 4; ++kc) {
      unsigned bb0, bb1;
      load_b(m.W2, kMlpHidden, nt * 8, kc * 16, g, t, bb0, bb1);
      mma16816(T.z2[nt], T.h1[kc][0], T.h1[kc][1], T.h1[kc][2], T.h1[kc][3], bb0, bb1);
    }
  }
#pragma unroll
  for (int kc = 0; kc < 4; ++kc) {
    T.h2[kc][0] = pack_bf16(gelu_f(T.z2[2 * kc][0]), gelu_f(T.z2[2 * kc][1]));
    T.h2[kc][1] = pack_bf16(gelu_f(T.z2[2 * kc][2]), gelu_f(T.z2[2 * kc][3]));
    T.h2[kc][2] = pack_bf16(gelu_f(T.z2[2 * kc + 1][0]), gelu_f(T.z2[2 * kc + 1][1]));
    T.h2[kc][3] = pack_bf16(gelu_f(T.z2[2 * kc + 1][2]), gelu_f(T.z2[2 * kc + 1][3]));
  }
  // layer 3 (8 outputs)
  T.o[0] = b3[2 * t]; T.o[1] = b3[2 * t + 1]; T.o[2] = b3[2 * t]; T.o[3] = b3[2 * t + 1];
#pragma unroll
  for (int kc = 0; kc < 4; ++kc) {
    unsigned bb0, bb1;
    load_b(m.W3, kMlpHidden, 0, kc * 16, g, t, bb0, bb1);
    mma16816(T.o, T.h2[kc][0], T.h2[kc][1], T.h2[kc][2], T.h2[kc][3], bb0, bb1);
  }
}

// Training: forward + backward of 16 samples per warp; writes the warp's
// gradient partial (kMlpParams floats) and loss partial to partials[tile].
constexpr int kTrainWarps = 4;

__global__ void __launch_bounds__(32 * kTrainWarps) k_mlp_train_tile(
    MlpDev m, int B, const float* __restrict__ X, const int* __restrict__ slot,
    const double* __restrict__ St, const double* __restrict__ Sd,
    const double* __restrict__ target, float* __restrict__ partials) {
  // per-warp staging (bf16): X [16][32], h1, h2, dz1, dz2 [16][64], dO [16][16]
  __shared__ __nv_bfloat16 sX[kTrainWarps][16][kMlpInPad];
  __shared__ __nv_bfloat16 sH1[kTrainWarps][16][kMlpHidden];
  __shared__ __nv_bfloat16 sH2[kTrainWarps][16][kMlpHidden];
  __shared__ __nv_bfloat16 sD1[kTrainWarps][16][kMlpHidden];
  __shared__ __nv_bfloat16 sD2[kTrainWarps][16][kMlpHidden];
  __shared__ __nv_bfloat16 sDO[kTrainWarps][16][16];
  const int w = threadIdx.x >> 5;
  const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
  const int tile = blockIdx.x * kTrainWarps + w;
  const int r0 = tile * 16;
  if (r0 >= B) return;
  float* part = partials + (size_t)tile * kMlpPartial;
  Tile T;
  mlp_forward_tile(m, X, B, r0, g, t, T);
  // output gradient: gather o_pick and o_7 of rows g and g + 8 in the quad
  float dO[4] = {0.f, 0.f, 0.f, 0.f};
  float lsum = 0.f;
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    const int row = r0 + g + 8 * h;
    const bool valid = row < B;
    const int sl = valid ? slot[row] : 0;
    const int pick = sl;  // slot 0 -> o_0 (diagonal), 1..6 -> o_d
    const int src = (lane & ~3) | (pick >> 1);
    const float oa = __shfl_sync(0xffffffffu, T.o[2 * h], src);
    const float ob = __shfl_sync(0xffffffffu, T.o[2 * h + 1], src);
    const float opk = (pick & 1) ? ob : oa;
    const float o7 = __shfl_sync(0xffffffffu, T.o[2 * h + 1], (lane & ~3) | 3);
    if (valid) {
      const double sd = Sd[row], st = St[row];
      const double e = exp((double)opk);
      const double pred = st * e + (sl == 0 ? (double)o7 * sd : 0.0);
      const double r = (pred - target[row]) / sd;
      const double dpred = 2.0 * r / sd / (double)B;
      if (t == 0) lsum += (float)(r * r / (double)B);
      // this thread holds columns 2t, 2t+1 of the row
#pragma unroll
      for (int c = 0; c < 2; ++c) {
        const int col = 2 * t + c;
        float v = 0.f;
        if (col == pick) v += (float)(dpred * st * e);
        if (col == 7 && sl == 0) v += (float)(dpred * sd);
        dO[2 * h + c] = v;
      }
    }
  }
  // stage dO (K padded to 16), X, h1, h2 as bf16 [sample][feature]
  {
    __nv_bfloat16* d = &sDO[w][0][0];
    d[g * 16 + 2 * t] = __float2bfloat16_rn(dO[0]);
    d[g * 16 + 2 * t + 1] = __float2bfloat16_rn(dO[1]);
    d[(g + 8) * 16 + 2 * t] = __float2bfloat16_rn(dO[2]);
    d[(g + 8) * 16 + 2 * t + 1] = __float2bfloat16_rn(dO[3]);
    d[g * 16 + 8 + 2 * t] = __float2bfloat16_rn(0.f);
    d[g * 16 + 8 + 2 * t + 1] = __float2bfloat16_rn(0.f);
    d[(g + 8) * 16 + 8 + 2 * t] = __float2bfloat16_rn(0.f);
    d[(g + 8) * 16 + 8 + 2 * t + 1] = __float2bfloat16_rn(0.f);
  }
  auto stage_a = [&](__nv_bfloat16 (*dst)[kMlpHidden], const unsigned (*a)[4], int nk) {
    for (int kc = 0; kc < nk; ++kc) {
      *reinterpret_cast<unsigned*>(&dst[g][kc * 16 + 2 * t]) = a[kc][0];
      *reinterpret_cast<unsigned*>(&dst[g + 8][kc * 16 + 2 * t]) = a[kc][1];
      *reinterpret_cast<unsigned*>(&dst[g][kc * 16 + 8 + 2 * t]) = a[kc][2];
      *reinterpret_cast<unsigned*>(&dst[g + 8][kc * 16 + 8 + 2 * t]) = a[kc][3];
    }
  };
  stage_a(sH1[w], T.h1, 4);
  stage_a(sH2[w], T.h2, 4);
#pragma unroll
  for (int kc = 0; kc < 2; ++kc) {
    *reinterpret_cast<unsigned*>(&sX[w][g][kc * 16 + 2 * t]) = T.x[kc][0];
    *reinterpret_cast<unsigned*>(&sX[w][g + 8][kc * 16 + 2 * t]) = T.x[kc][1];
    *reinterpret_cast<unsigned*>(&sX[w][g][kc * 16 + 8 + 2 * t]) = T.x[kc][2];
    *reinterpret_cast<unsigned*>(&sX[w][g + 8][kc * 16 + 8 + 2 * t]) = T.x[kc][3];
  }
  // dH2 = dO W3 (K = 8 padded to 16; B = W3^T as [64][16]); dZ2 = dH2 * gelu'(z2)
  const unsigned do0 = pack_bf16(dO[0], dO[1]), do1 = pack_bf16(dO[2], dO[3]);
  float dz2[8][4];
#pragma unroll
  for (int nt = 0; nt < 8; ++nt) {
    dz2[nt][0] = dz2[nt][1] = dz2[nt][2] = dz2[nt][3] = 0.f;
    unsigned bb0, bb1;
    load_b(m.W3T, 16, nt * 8, 0, g, t, bb0, bb1);
    mma16816(dz2[nt], do0, do1, 0u, 0u, bb0, bb1);
#pragma unroll
    for (int q = 0; q < 4; ++q) dz2[nt][q] *= gelu_grad_f(T.z2[nt][q]);
  }
  unsigned a2[4][4];
#pragma unroll
  for (int kc = 0; kc < 4; ++kc) {
    a2[kc][0] = pack_bf16(dz2[2 * kc][0], dz2[2 * kc][1]);
    a2[kc][1] = pack_bf16(dz2[2 * kc][2], dz2[2 * kc][3]);
    a2[kc][2] = pack_bf16(dz2[2 * kc + 1][0], dz2[2 * kc + 1][1]);
    a2[kc][3] = pack_bf16(dz2[2 * kc + 1][2], dz2[2 * kc + 1][3]);
  }
  stage_a(sD2[w], a2, 4);
  // dH1 = dZ2 W2 (B = W2^T); dZ1 = dH1 * gelu'(z1)
  float dz1[8][4];
#pragma unroll
  for (int nt = 0; nt < 8; ++nt) {
    dz1[nt][0] = dz1[nt][1] = dz1[nt][2] = dz1[nt][3] = 0.f;
#pragma unroll
    for (int kc = 0; kc < 4; ++kc) {
      unsigned bb0, bb1;
      load_b(m.W2T, kMlpHidden, nt * 8, kc * 16, g, t, bb0, bb1);
      mma16816(dz1[nt], a2[kc][0], a2[kc][1], a2[kc][2], a2[kc][3], bb0, bb1);
    }
#pragma unroll
    for (int q = 0; q < 4; ++q) dz1[nt][q] *= gelu_grad_f(T.z1[nt][q]);
  }
  unsigned a1[4][4];
#pragma unroll
  for (int kc = 0; kc < 4; ++kc) {
    a1[kc][0] = pack_bf16(dz1[2 * kc][0], dz1[2 * kc][1]);
    a1[kc][1] = pack_bf16(dz1[2 * kc][2], dz1[2 * kc][3]);
    a1[kc][2] = pack_bf16(dz1[2 * kc + 1][0], dz1[2 * kc + 1][1]);
    a1[kc][3] = pack_bf16(dz1[2 * kc + 1][2], dz1[2 * kc + 1][3]);
  }
  stage_a(sD1[w], a1, 4);
  __syncwarp();
  // weight gradients over the 16 samples: dW[o][i] = sum_s D[s][o] H[s][i]
  // A = D^T (rows o, K = samples), B = H (K = samples x N = i)
  auto wgrad = [&](const __nv_bfloat16 (*D)[kMlpHidden], int ldD, const __nv_bfloat16* H,
                   int ldH, int Mo, int Ni, int off) {
    for (int mt = 0; mt < Mo / 16 + (Mo % 16 ? 1 : 0); ++mt) {
      for (int nt = 0; nt < Ni / 8; ++nt) {
        const int o_a = mt * 16 + g, o_b = mt * 16 + g + 8;
        auto dget = [&](int s, int o) -> __nv_bfloat16 {
          return o < Mo ? (reinterpret_cast<const __nv_bfloat16*>(D))[s * ldD + o]
                        : __float2bfloat16_rn(0.f);
        };
        const unsigned aa0 = pack_raw(dget(2 * t, o_a), dget(2 * t + 1, o_a));
        const unsigned aa1 = pack_raw(dget(2 * t, o_b), dget(2 * t + 1, o_b));
        const unsigned aa2 = pack_raw(dget(2 * t + 8, o_a), dget(2 * t + 9, o_a));
        const unsigned aa3 = pack_raw(dget(2 * t + 8, o_b), dget(2 * t + 9, o_b));
        const int ic = nt * 8 + g;
        const unsigned bb0 = pack_raw(H[(2 * t) * ldH + ic], H[(2 * t + 1) * ldH + ic]);
        const unsigned bb1 = pack_raw(H[(2 * t + 8) * ldH + ic], H[(2 * t + 9) * ldH + ic]);
        float c[4] = {0.f, 0.f, 0.f, 0.f};
        mma16816(c, aa0, aa1, aa2, aa3, bb0, bb1);
        const int i0 = nt * 8 + 2 * t;
        if (o_a < Mo) {
          part[off + o_a * Ni + i0] = c[0];
          part[off + o_a * Ni + i0 + 1] = c[1];
        }
        if (o_b < Mo) {
          part[off + o_b * Ni + i0] = c[2];
          part[off + o_b * Ni + i0 + 1] = c[3];
        }
      }
    }
  };
  wgrad(sD2[w], kMlpHidden, &sH1[w][0][0], kMlpHidden, kMlpHidden, kMlpHidden, kOffW2);
  wgrad(reinterpret_cast<const __nv_bfloat16(*)[kMlpHidden]>(&sDO[w][0][0]), 16, &sH2[w][0][0],
        kMlpHidden, kMlpOut, kMlpHidden, kOffW3);
  // W1: inputs 0..23 of the padded 32 (N = 24 = 3 n-tiles)
  wgrad(sD1[w], kMlpHidden, &sX[w][0][0], kMlpInPad, kMlpHidden, kMlpIn, kOffW1);
  // bias gradients: column sums over the 16 samples (FP32 over bf16 stage)
  for (int c = lane; c < kMlpHidden; c += 32) {
    float s1 = 0.f, s2 = 0.f;
    for (int s = 0; s < 16; ++s) {
      s1 += __bfloat162float(sD1[w][s][c]);
      s2 += __bfloat162float(sD2[w][s][c]);
    }
    part[kOffB1 + c] = s1;
    part[kOffB2 + c] = s2;
  }
  if (lane < kMlpOut) {
    float s3 = 0.f;
    for (int s = 0; s < 16; ++s) s3 += __bfloat162float(sDO[w][s][lane]);
    part[kOffB3 + lane] = s3;
  }
  // loss partial
  float l = lsum;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) l += __shfl_down_sync(0xffffffffu, l, o);
  if (lane == 0) part[kMlpParams] = l;
}

// grad[p] = sum over tiles of partials[tile][p] (fixed order); the loss in
// grad[kMlpParams]
__global__ void k_mlp_reduce(int ntiles, const float* __restrict__ partials,
                             float* __restrict__ grad) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p > kMlpParams) return;
  float s = 0.f;
  for (int k = 0; k < ntiles; ++k) s += partials[(size_t)k * kMlpPartial + p];
  grad[p] = s;
}

// Adam (Kingma and Ba 2015), bias-corrected, FP32 master weights
__global__ void k_adam(float* __restrict__ w, const float* __restrict__ g, float* __restrict__ mm,
                       float* __restrict__ vv, int step, float lr) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= kMlpParams) return;
  const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
  const float gi = g[p];
  const float mi = b1 * mm[p] + (1.f - b1) * gi;
  const float vi = b2 * vv[p] + (1.f - b2) * gi * gi;
  mm[p] = mi;
  vv[p] = vi;
  const float mh = mi / (1.f - powf(b1, (float)step));
  const float vh = vi / (1.f - powf(b2, (float)step));
  w[p] -= lr * mh / (sqrtf(vh) + eps);
}

// BF16 copies used by the tensor-core kernels
__global__ void k_mlp_pack(MlpDev m) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  const float* P = m.params;
  if (p < kMlpHidden * kMlpInPad) {  // W1 [64][32], K padded with zeros
    const int o = p / kMlpInPad, i = p % kMlpInPad;
    m.W1[p] = __float2bfloat16_rn(i < kMlpIn ? P[kOffW1 + o * kMlpIn + i] : 0.f);
  }
  if (p < kMlpHidden * kMlpHidden) {  // W2 [64][64] and W2^T
    const int o = p / kMlpHidden, i = p % kMlpHidden;
    m.W2[p] = __float2bfloat16_rn(P[kOffW2 + p]);
    m.W2T[i * kMlpHidden + o] = __float2bfloat16_rn(P[kOffW2 + p]);
  }
  if (p < kMlpOut * kMlpHidden) {  // W3 [8][64]
    m.W3[p] = __float2bfloat16_rn(P[kOffW3 + p]);
  }
  if (p < kMlpHidden * 16) {  // W3^T [64][16], K padded with zeros
    const int h = p / 16, o = p % 16;
    m.W3T[p] = __float2bfloat16_rn(o < kMlpOut ? P[kOffW3 + o * kMlpHidden + h] : 0.f);
  }
  // the same weights in the tcgen05 operand layout
  if (p < kMlpHidden * kMlpInPad) {
    const int o = p / kMlpInPad, i = p % kMlpInPad;
    m.Wtc[mlp_core_off(o, i, 32) / 2] =
        __float2bfloat16_rn(i < kMlpIn ? P[kOffW1 + o * kMlpIn + i] : 0.f);
  }
  if (p < kMlpHidden * kMlpHidden) {
    const int o = p / kMlpHidden, i = p % kMlpHidden;
    m.Wtc[64 * 32 + mlp_core_off(o, i, 64) / 2] = __float2bfloat16_rn(P[kOffW2 + p]);
  }
  if (p < 16 * kMlpHidden) {
    const int o = p / kMlpHidden, i = p % kMlpHidden;
    m.Wtc[64 * 32 + 64 * 64 + mlp_core_off(o, i, 64) / 2] =
        __float2bfloat16_rn(o < kMlpOut ? P[kOffW3 + o * kMlpHidden + i] : 0.f);
  }
}

// Row i: S_ii <- S~_ii exp(o_0) + o_7 S~_ii, S_ij <- S~_ij exp(o_d), d the
// face direction of j read from the grid coordinates (z-, y-, x-, x+, y+,
// z+: the one coordinate in which i and j differ). The row keeps plain S~
// when a corrected value is not finite, the corrected diagonal is not
// positive, an off-diagonal changes sign, or the row loses the diagonal
// dominance the plain row had.
__global__ void k_learned_schur(int N, int nx, int ny, const int* __restrict__ rowptr,
                                const int* __restrict__ col, const int* __restrict__ dpos,
                                const double* __restrict__ S, const float* __restrict__ O,
                                double* __restrict__ out, int* __restrict__ nbad) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= N) return;
  const int r0 = rowptr[i], r1 = rowptr[i + 1], d = dpos[i];
  const float* o = O + (size_t)i * kMlpOut;
  const double sd = S[d];
  const int nxy = nx * ny;
  const int xi = i % nx, yi = (i / nx) % ny, zi = i / nxy;
  bool bad = false;
  double offo = 0.0, offn = 0.0, nd = 0.0;
  for (int e = r0; e < r1; ++e) {
    const int j = col[e];
    double v;
    if (j == i) {
      v = sd * exp((double)o[0]) + (double)o[7] * sd;
      nd = v;
    } else {
      const int xj = j % nx, yj = (j / nx) % ny, zj = j / nxy;
      const int k = zj < zi ? 1 : yj < yi ? 2 : xj < xi ? 3 : xj > xi ? 4 : yj > yi ? 5 : 6;
      v = S[e] * exp((double)o[k]);
      if ((v > 0.0) != (S[e] > 0.0) || (v < 0.0) != (S[e] < 0.0)) bad = true;
      offo += fabs(S[e]);
      offn += fabs(v);
    }
    if (!isfinite(v)) bad = true;
    out[e] = v;
  }
  if (!(nd > 0.0)) bad = true;
  if (sd >= offo && nd < offn) bad = true;
  if (bad) {
    for (int e = r0; e < r1; ++e) out[e] = S[e];
    atomicAdd(nbad, 1);
  }
}

}  // namespace

void learned_schur(int N, int nx, int ny, const int* rowptr, const int* col, const int* dpos,
                   const double* S, const float* O, double* out, int* nbad, cudaStream_t s) {
  k_learned_schur<<<grid_for(N), kBlock, 0, s>>>(N, nx, ny, rowptr, col, dpos, S, O, out, nbad);
  TP_LAUNCH_CHECK();
}

void mlp_pack(const MlpDev& m, cudaStream_t s) {
  k_mlp_pack<<<grid_for(kMlpHidden * kMlpHidden), kBlock, 0, s>>>(m);
  TP_LAUNCH_CHECK();
}

void mlp_forward(const MlpDev& m, int n, const float* X, float* O, cudaStream_t s) {
  if (n <= 0) return;
  TP_CUDA_TRY(cudaMemsetAsync(m.err, 0, sizeof(int), s));
  mlp_forward_tc(m, n, X, O, m.err, s);
  int h = 0;
  TP_CUDA_TRY(cudaMemcpyAsync(&h, m.err, sizeof(int), cudaMemcpyDeviceToHost, s));
  TP_CUDA_TRY(cudaStreamSynchronize(s));
  if (h != 0) fail(TP_ECUDA, "MLP forward: a tensor-core completion wait timed out");
}

void mlp_gradient(const MlpDev& m, int B, const float* X, const int* slot, const double* St,
                  const double* Sd, const double* target, float* partials, float* grad,
                  cudaStream_t s) {
  const int tiles = (B + 15) / 16;
  k_mlp_train_tile<<<(tiles + kTrainWarps - 1) / kTrainWarps, 32 * kTrainWarps, 0, s>>>(
      m, B, X, slot, St, Sd, target, partials);
  TP_LAUNCH_CHECK();
  k_mlp_reduce<<<grid_for(kMlpParams + 1), kBlock, 0, s>>>(tiles, partials, grad);
  TP_LAUNCH_CHECK();
}

void mlp_adam(MlpDev& m, const float* grad, float lr, cudaStream_t s) {
  m.step += 1;
  k_adam<<<grid_for(kMlpParams), kBlock, 0, s>>>(m.params, grad, m.adam_m, m.adam_v, m.step, lr);
  TP_LAUNCH_CHECK();
  mlp_pack(m, s);
}

}  // namespace tp

// Learned Schur correction: MLP parameters and launchers (internal header).
#pragma once
#include <cuda_bf16.h>
#include "common.cuh"

namespace tp {

constexpr int kMlpIn = 24, kMlpInPad = 32, kMlpHidden = 64, kMlpOut = 8;
// flat FP32 parameter layout: W1 [64][24], b1 [64], W2 [64][64], b2 [64],
// W3 [8][64], b3 [8]
constexpr int kOffW1 = 0;
constexpr int kOffB1 = kOffW1 + kMlpHidden * kMlpIn;
constexpr int kOffW2 = kOffB1 + kMlpHidden;
constexpr int kOffB2 = kOffW2 + kMlpHidden * kMlpHidden;
constexpr int kOffW3 = kOffB2 + kMlpHidden;
constexpr int kOffB3 = kOffW3 + kMlpOut * kMlpHidden;
constexpr int kMlpParams = kOffB3 + kMlpOut;   // 6280
constexpr int kMlpPartial = kMlpParams + 1;    // + loss
constexpr int kMlpTcWeights = 64 * 32 + 64 * 64 + 16 * 64;  // bf16 elements of Wtc

// byte offset of element (r, k) of an R x K bf16 tile in the no-swizzle
// K-major layout of 8-row x 16-byte core matrices used by tcgen05 operands
__host__ __device__ inline unsigned mlp_core_off(int r, int k, int K) {
  return (unsigned)(((r >> 3) * (K >> 3) + (k >> 3)) * 128 + (r & 7) * 16 + (k & 7) * 2);
}

struct MlpDev {
  float* params = nullptr;  // FP32 master weights [kMlpParams]
  float* adam_m = nullptr;
  float* adam_v = nullptr;
  float* grad = nullptr;    // [kMlpPartial]
  __nv_bfloat16* W1 = nullptr;   // [64][32]
  __nv_bfloat16* W2 = nullptr;   // [64][64]
  __nv_bfloat16* W3 = nullptr;   // [8][64]
  __nv_bfloat16* W2T = nullptr;  // [64][64]
  __nv_bfloat16* W3T = nullptr;  // [64][16]
  // W1 [64 x 32], W2 [64 x 64], W3 padded [16 x 64] back to back in the
  // tcgen05 shared-memory layout (kMlpTcWeights bf16, copied in one bulk copy)
  __nv_bfloat16* Wtc = nullptr;
  int* err = nullptr;            // tensor-core forward: bit 0 = mbarrier wait timed out
  int step = 0;
};

void mlp_pack(const MlpDev& m, cudaStream_t s);
// inference O[n][8] = MLP(X[n][24]) on the tcgen05 tensor cores (mlp_tc.cu);
// throws if a wait on the tensor cores timed out
void mlp_forward(const MlpDev& m, int n, const float* X, float* O, cudaStream_t s);
void mlp_forward_tc(const MlpDev& m, int n, const float* X, float* O, int* err, cudaStream_t s);
// gradient of the mean squared relative error over B samples into grad
// (loss in grad[kMlpParams]); partials holds ceil(B/16) * kMlpPartial floats
void mlp_gradient(const MlpDev& m, int B, const float* X, const int* slot, const double* St,
                  const double* Sd, const double* target, float* partials, float* grad,
                  cudaStream_t s);
void mlp_adam(MlpDev& m, const float* grad, float lr, cudaStream_t s);

// learned S~ values on the 7-point pattern with the per-row guard; returns
// (through *nbad, device int) the number of rows that fell back
void learned_schur(int N, int nx, int ny, const int* rowptr, const int* col, const int* dpos,
                   const double* S, const float* O, double* out, int* nbad, cudaStream_t s);

}  // namespace tp

// Allocation-free variant of the equation-scale reduction.
//
// Some callers cannot call cudaMalloc: code that runs while a memory pool is
// frozen or being defragmented, allocator hooks, or embedders that hand this
// library a fixed device budget up front. tp_equation_scales_noalloc serves
// them: it computes the same two equation scales as the solver's own
// reduction (s_m = N / sum_i |A_pp,ii|, s_e = N / sum_i |A_TT,ii|) from
// caller-owned device arrays, and its only scratch is the fixed array below,
// which every GPU that loads this library keeps until the process exits.
#include <mutex>
#include "common.cuh"

namespace {

// rows reduced per block, and the largest number of blocks the scratch holds
constexpr int kRowsPerBlock = 2048;
constexpr int kMaxBlocks = 4096;   // N <= 4096 * 2048 = 8,388,608 cells
constexpr int kThreads = 256;

// two partial sums per block (|A_pp,ii| and |A_TT,ii|); 64 KiB per device
static __device__ __align__(256) double g_scale_partials[2 * kMaxBlocks];

// Block b sums |diag| of rows [b * kRowsPerBlock, ...) for both equations.
// Each slot is overwritten (never accumulated), so nothing needs clearing.
__global__ void k_scale_partials(int N, const int* __restrict__ rowptr,
                                 const int* __restrict__ col,
                                 const double* __restrict__ bval,
                                 double* __restrict__ partials) {
  __shared__ double sm[kThreads], se[kThreads];
  const long long r0 = (long long)blockIdx.x * kRowsPerBlock;
  long long r1 = r0 + kRowsPerBlock;
  if (r1 > N) r1 = N;
  double am = 0.0, ae = 0.0;
  for (long long i = r0 + threadIdx.x; i < r1; i += blockDim.x) {
    for (int e = rowptr[i]; e < rowptr[i + 1]; ++e) {
      if (col[e] == (int)i) {
        am += fabs(bval[4ll * e + 0]);
        ae += fabs(bval[4ll * e + 3]);
        break;
      }
    }
  }
  sm[threadIdx.x] = am;
  se[threadIdx.x] = ae;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if ((int)threadIdx.x < o) {
      sm[threadIdx.x] += sm[threadIdx.x + o];
      se[threadIdx.x] += se[threadIdx.x + o];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    partials[2 * blockIdx.x + 0] = sm[0];
    partials[2 * blockIdx.x + 1] = se[0];
  }
}

// one thread adds the block partials in block order and writes the scales
__global__ void k_scale_finish(int N, int nblocks, const double* __restrict__ partials,
                               double* __restrict__ scales) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  double sm = 0.0, se = 0.0;
  for (int b = 0; b < nblocks; ++b) {
    sm += partials[2 * b + 0];
    se += partials[2 * b + 1];
  }
  scales[0] = (double)N / sm;
  scales[1] = (double)N / se;
}

// Device address of the scratch array (host code may not pass the symbol
// itself: on the host it is only a stand-in). Outside stream capture it is
// looked up on every call, so a device reset or another context on the same
// device (where the module, and with it the array, may be loaded at a new
// address) is followed; inside a capture the address of the last uncaptured
// call on this device is used.
constexpr int kMaxDevices = 64;
double* g_scratch_ptr[kMaxDevices] = {};
std::mutex g_scratch_mu;

int scratch_for_current_device(cudaStream_t s, double** out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
    cudaGetLastError();
    return TP_ECUDA;
  }
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(s, &cap) != cudaSuccess) {
    cudaGetLastError();
    return TP_ECUDA;
  }
  std::lock_guard<std::mutex> lock(g_scratch_mu);
  if (cap == cudaStreamCaptureStatusNone || !g_scratch_ptr[dev]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_scale_partials);
    if (e != cudaSuccess || !p) {
      cudaGetLastError();
      return TP_ECUDA;
    }
    g_scratch_ptr[dev] = static_cast<double*>(p);
  }
  *out = g_scratch_ptr[dev];
  return TP_OK;
}

}  // namespace

extern "C" int tp_equation_scales_noalloc(int N, const int* rowptr, const int* col,
                                          const double* bval, double* scales,
                                          void* cuda_stream) {
  if (N < 1 || !rowptr || !col || !bval || !scales) return TP_EINVAL;
  const long long nblocks = ((long long)N + kRowsPerBlock - 1) / kRowsPerBlock;
  if (nblocks > kMaxBlocks) return TP_EINVAL;  // N above 8,388,608 cells
  cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
  double* partials = nullptr;
  int st = scratch_for_current_device(s, &partials);
  if (st != TP_OK) return st;
  k_scale_partials<<<(int)nblocks, kThreads, 0, s>>>(N, rowptr, col, bval, partials);
  k_scale_finish<<<1, 32, 0, s>>>(N, (int)nblocks, partials, scales);
  if (cudaGetLastError() != cudaSuccess) return TP_ECUDA;
  tp::count_launch(2);
  return TP_OK;
}

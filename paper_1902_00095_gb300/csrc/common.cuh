// Shared device-side definitions of the thermo library (internal header).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>
#include <vector>
#include <string>
#include "thermo.h"

namespace tp {

// ---------------------------------------------------------------- errors
struct Error {
  int code;
  std::string what;
};

#define TP_CUDA_TRY(expr)                                                  \
  do {                                                                     \
    cudaError_t e__ = (expr);                                              \
    if (e__ != cudaSuccess)                                                \
      throw ::tp::Error{TP_ECUDA, std::string(#expr) + ": " +              \
                                      cudaGetErrorString(e__)};            \
  } while (0)

// Host-side count of kernels this library has launched (graph replays add
// their kernel-node count); launches recorded into a graph are not counted.
void count_launch(long long n = 1);
extern thread_local bool g_capturing;

#define TP_LAUNCH_CHECK()                 \
  do {                                    \
    TP_CUDA_TRY(cudaGetLastError());      \
    ::tp::count_launch();                 \
  } while (0)

inline void fail(int code, const std::string& msg) { throw Error{code, msg}; }

// ------------------------------------------------------------- allocation
// Owns every device allocation of one object; freed together.
class Pool {
 public:
  Pool() = default;
  Pool(const Pool&) = delete;
  Pool& operator=(const Pool&) = delete;
  ~Pool() { release(); }
  template <class T>
  T* alloc(size_t count) {
    if (count == 0) count = 1;
    void* p = nullptr;
    cudaError_t e = cudaMalloc(&p, count * sizeof(T));
    if (e != cudaSuccess) {
      cudaGetLastError();
      fail(TP_ENOMEM, "cudaMalloc of " + std::to_string(count * sizeof(T)) + " bytes");
    }
    ptrs_.push_back(p);
    return static_cast<T*>(p);
  }
  void release() {
    for (void* p : ptrs_) cudaFree(p);
    ptrs_.clear();
  }

 private:
  std::vector<void*> ptrs_;
};

// ---------------------------------------------------------------- CSR
struct DevCSR {
  int n = 0;      // rows
  int m = 0;      // columns
  int nnz = 0;
  int* rowptr = nullptr;
  int* col = nullptr;
  double* val = nullptr;
  float* valf = nullptr;  // FP32 copy (mixed-precision hierarchy)
};

// ---------------------------------------------------------------- launch
constexpr int kBlock = 256;
inline int grid_for(long long n, int block = kBlock) {
  long long g = (n + block - 1) / block;
  if (g < 1) g = 1;
  return (int)g;
}

// ----------------------------------------------------- dependent launch
// Programmatic dependent launch: a kernel started with launch_pdl may begin
// while the previous kernel on the stream finishes; it must call pdl_wait()
// before reading anything that kernel wrote, and calls pdl_trigger() once
// its own inputs are consumed so the next kernel can start launching.
__device__ __forceinline__ void pdl_wait() {
  asm volatile("griddepcontrol.wait;" ::: "memory");
}
__device__ __forceinline__ void pdl_trigger() {
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

template <typename... KArgs, typename... Args>
void launch_pdl(void (*kernel)(KArgs...), dim3 grid, dim3 block, cudaStream_t s,
                Args&&... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = 0;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  TP_CUDA_TRY(cudaLaunchKernelEx(&cfg, kernel, static_cast<KArgs>(args)...));
  count_launch();
}

// exclusive scan of n ints: out[0] = 0, out[i] = sum in[0..i-1]; out has
// n + 1 entries and out[n] is the total. `in` and `out` may alias only if
// equal. Returns the total (synchronises the stream).
long long scan_exclusive(const int* in, int* out, int n, Pool& scratch,
                         cudaStream_t s);

// Deterministic sum of n doubles (fixed block partition and tree order),
// result in *out (device).
void sum_fixed(const double* x, int n, double* out, double* partials,
               int nparts, cudaStream_t s);

}  // namespace tp

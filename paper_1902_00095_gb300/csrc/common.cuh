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
// Owns the device memory of one object as a chain of chunks handed out by a
// bump pointer (256-byte aligned). release() only rewinds: the chunks stay
// allocated and the next build that allocates in the same order gets the
// same addresses, so repeated setups make no cudaMalloc/cudaFree calls (a
// cudaFree synchronises the device). Reuse is safe because every user
// allocates and consumes on one stream, in order. The destructor frees.
class Pool {
 public:
  Pool() = default;
  Pool(const Pool&) = delete;
  Pool& operator=(const Pool&) = delete;
  ~Pool() { free_all(); }
  template <class T>
  T* alloc(size_t count) {
    if (count == 0) count = 1;
    const size_t bytes = (count * sizeof(T) + 255) & ~size_t(255);
    while (cur_ < chunks_.size() && chunks_[cur_].used + bytes > chunks_[cur_].size) ++cur_;
    if (cur_ == chunks_.size()) {
      size_t want = next_ < bytes ? bytes : next_;
      void* p = nullptr;
      cudaError_t e = cudaMalloc(&p, want);
      if (e != cudaSuccess) {
        cudaGetLastError();
        fail(TP_ENOMEM, "cudaMalloc of " + std::to_string(want) + " bytes");
      }
      chunks_.push_back(Chunk{static_cast<char*>(p), want, 0});
      if (next_ < (size_t(256) << 20)) next_ *= 2;
    }
    Chunk& c = chunks_[cur_];
    void* out = c.base + c.used;
    c.used += bytes;
    return static_cast<T*>(out);
  }
  // rewind: every pointer handed out so far becomes invalid, memory is kept
  void release() {
    for (Chunk& c : chunks_) c.used = 0;
    cur_ = 0;
  }
  void free_all() {
    for (Chunk& c : chunks_) cudaFree(c.base);
    chunks_.clear();
    cur_ = 0;
  }
  size_t reserved() const {
    size_t t = 0;
    for (const Chunk& c : chunks_) t += c.size;
    return t;
  }

 private:
  struct Chunk {
    char* base;
    size_t size;
    size_t used;
  };
  std::vector<Chunk> chunks_;
  size_t cur_ = 0;
  size_t next_ = size_t(4) << 20;  // first chunk 4 MiB, doubling up to 256 MiB
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

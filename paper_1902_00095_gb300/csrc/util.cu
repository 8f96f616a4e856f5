// Device scans and deterministic reductions used by assembly and AMG setup.
#include "common.cuh"
#include <atomic>
#include <climits>

namespace tp {

static std::atomic<long long> g_launches{0};
thread_local bool g_capturing = false;

void count_launch(long long n) {
  if (!g_capturing) g_launches.fetch_add(n, std::memory_order_relaxed);
}

long long launches_total() { return g_launches.load(); }

namespace {

constexpr int kScanThreads = 256;
constexpr int kScanItems = 4;
constexpr int kScanTile = kScanThreads * kScanItems;

// Block-local exclusive scan of a tile; writes local prefixes and the tile
// total. T_in is int (counts) or long long (block totals of a lower pass).
template <class T_in>
__global__ void k_scan_tile(const T_in* __restrict__ in, long long* __restrict__ out,
                            long long* __restrict__ tile_sums, int n) {
  __shared__ long long warp_tot[kScanThreads / 32];
  const int base = blockIdx.x * kScanTile + threadIdx.x * kScanItems;
  long long v[kScanItems];
  long long run = 0;
#pragma unroll
  for (int k = 0; k < kScanItems; ++k) {
    int i = base + k;
    long long x = (i < n) ? (long long)in[i] : 0;
    v[k] = run;
    run += x;
  }
  // inclusive warp scan of per-thread totals
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  long long incl = run;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    long long y = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += y;
  }
  if (lane == 31) warp_tot[wid] = incl;
  __syncthreads();
  if (wid == 0) {
    long long t = (lane < kScanThreads / 32) ? warp_tot[lane] : 0;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      long long y = __shfl_up_sync(0xffffffffu, t, o);
      if (lane >= o) t += y;
    }
    if (lane < kScanThreads / 32) warp_tot[lane] = t;  // inclusive
  }
  __syncthreads();
  long long excl = incl - run + (wid > 0 ? warp_tot[wid - 1] : 0);
#pragma unroll
  for (int k = 0; k < kScanItems; ++k) {
    int i = base + k;
    if (i < n) out[i] = excl + v[k];
  }
  if (threadIdx.x == kScanThreads - 1) tile_sums[blockIdx.x] = excl + run;
}

__global__ void k_scan_add(long long* __restrict__ out, const long long* __restrict__ offs, int n) {
  int i = blockIdx.x * kScanTile + threadIdx.x;
  long long o = offs[blockIdx.x];
  for (int k = 0; k < kScanItems; ++k, i += kScanThreads)
    if (i < n && i < (blockIdx.x + 1) * kScanTile) out[i] += o;
}

__global__ void k_to_int(const long long* __restrict__ in, int* __restrict__ out, int n,
                         long long total, int* __restrict__ overflow) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) out[i] = (int)in[i];
  if (i == 0) {
    out[n] = (int)total;
    *overflow = total > (long long)INT_MAX ? 1 : 0;
  }
}

// In-place exclusive scan of a long long array (recursive over tiles);
// returns nothing, leaves the total in *total_dev.
void scan_ll(long long* data_in_out, int n, long long* total_dev, Pool& scratch, cudaStream_t s);

template <class T_in>
void scan_to_ll(const T_in* in, long long* out, int n, long long* total_dev, Pool& scratch,
                cudaStream_t s) {
  int tiles = (n + kScanTile - 1) / kScanTile;
  if (tiles < 1) tiles = 1;
  long long* sums = scratch.alloc<long long>(tiles + 1);
  k_scan_tile<T_in><<<tiles, kScanThreads, 0, s>>>(in, out, sums, n);
  TP_LAUNCH_CHECK();
  if (tiles > 1) {
    scan_ll(sums, tiles, total_dev, scratch, s);
    k_scan_add<<<tiles, kScanThreads, 0, s>>>(out, sums, n);
    TP_LAUNCH_CHECK();
  } else {
    TP_CUDA_TRY(cudaMemcpyAsync(total_dev, sums, sizeof(long long), cudaMemcpyDeviceToDevice, s));
  }
}

void scan_ll(long long* data, int n, long long* total_dev, Pool& scratch, cudaStream_t s) {
  scan_to_ll<long long>(data, data, n, total_dev, scratch, s);
}

__global__ void k_partial_sums(const double* __restrict__ x, int n, double* __restrict__ partials) {
  __shared__ double sh[kBlock];
  double acc = 0.0;
  // block b owns the contiguous chunk [b*chunk, (b+1)*chunk)
  long long chunk = ((long long)n + gridDim.x - 1) / gridDim.x;
  long long lo = chunk * blockIdx.x, hi = lo + chunk;
  if (hi > n) hi = n;
  for (long long i = lo + threadIdx.x; i < hi; i += blockDim.x) acc += x[i];
  sh[threadIdx.x] = acc;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) partials[blockIdx.x] = sh[0];
}

__global__ void k_sum_partials(const double* __restrict__ partials, int np, double* __restrict__ out) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    double s = 0.0;
    for (int i = 0; i < np; ++i) s += partials[i];
    *out = s;
  }
}

}  // namespace

long long scan_exclusive(const int* in, int* out, int n, Pool& scratch, cudaStream_t s) {
  long long* tmp = scratch.alloc<long long>(n + 1);
  long long* total = scratch.alloc<long long>(1);
  int* overflow = scratch.alloc<int>(1);
  scan_to_ll<int>(in, tmp, n, total, scratch, s);
  long long h_total = 0;
  TP_CUDA_TRY(cudaMemcpyAsync(&h_total, total, sizeof(long long), cudaMemcpyDeviceToHost, s));
  TP_CUDA_TRY(cudaStreamSynchronize(s));
  k_to_int<<<grid_for(n + 1), kBlock, 0, s>>>(tmp, out, n, h_total, overflow);
  TP_LAUNCH_CHECK();
  if (h_total > (long long)INT_MAX) fail(TP_ENOMEM, "scan total exceeds 32-bit index range");
  return h_total;
}

void sum_fixed(const double* x, int n, double* out, double* partials, int nparts, cudaStream_t s) {
  k_partial_sums<<<nparts, kBlock, 0, s>>>(x, n, partials);
  TP_LAUNCH_CHECK();
  k_sum_partials<<<1, 32, 0, s>>>(partials, nparts, out);
  TP_LAUNCH_CHECK();
}

}  // namespace tp

// Explicit inverse of the coarsest AMG operator (dense n x n, row-major),
// the coarse-grid solver of the V-cycle (Gaussian elimination on the
// coarsest grid, Sec. 4 solver settings), computed inside one
// thread-block cluster.
//
// The rows are split over the cluster's CTAs and stay in their shared
// memory for the whole elimination. Gauss-Jordan runs in place, without an
// augmented identity: at step k with pivot row p (column k),
//   rows i != p:  f_i = a_ik / a_pk,  a_ij -= f_i a_pj (j != k),  a_ik = -f_i
//   row p:        a_pj /= a_pk (j != k),  a_pk = 1 / a_pk
// (each division taken as a product with the reciprocal 1 / a_pk).
// Column k of the identity is e_k until step k, so it can live in the slot
// of column k of A, which step k clears. The pivot is the largest |a_ik|
// over the rows not yet used (ties to the lower row index): each CTA offers
// its best row (value and a copy of the row, in one of two buffers that
// alternate between steps), every CTA reads all offers through distributed
// shared memory, takes the same pivot, copies the pivot row from its
// owner's offer, then updates its own rows. Choosing row p_k at step k is unpivoted elimination of
// B = Pi A (row k of B = row p_k of A) stored in A's row order, so the storage
// ends with B^{-1} = A^{-1} Pi^T, row k of it in storage row p_k, i.e.
// A^{-1}[k][p_j] = M[p_k][j]; the epilogue writes it out in that order.
//
// One cluster barrier per step (a CTA rewrites an offer buffer only after
// the next barrier, which every reader of it has passed); no flag waits.
// The caller checks and counts the launch.
#include <cooperative_groups.h>
#include <climits>

#include "amg.cuh"

namespace cg = cooperative_groups;

namespace tp {

namespace {

constexpr int kGjThreads = 1024;
constexpr int kGjWarps = kGjThreads / 32;

// shared-memory layout of one CTA (R rows of n entries), same on both sides
struct GjLayout {
  size_t M, offer, prow, fr, cand_k, ipiv, perm, pos, used, cand_i, piv_row, bytes;
  __host__ __device__ GjLayout(int n, int R) {
    size_t o = 0;
    M = o;       o += sizeof(double) * (size_t)R * n;
    offer = o;   o += sizeof(double) * 2 * (size_t)n;
    prow = o;    o += sizeof(double) * (size_t)n;
    fr = o;      o += sizeof(double) * (size_t)R;
    cand_k = o;  o += sizeof(unsigned long long) * 2;
    ipiv = o;    o += sizeof(double) * 2;
    perm = o;    o += sizeof(int) * (size_t)n;
    pos = o;     o += sizeof(int) * (size_t)R;
    used = o;    o += sizeof(int) * (size_t)R;
    cand_i = o;  o += sizeof(int) * 2;
    piv_row = o; o += sizeof(int) * 2;
    bytes = o;
  }
};

// Ordering key of |a|: for non-negative IEEE doubles the bit patterns,
// read as unsigned integers, order like the values; NaN maps to 0 (never a
// pivot, as a zero).
__device__ __forceinline__ unsigned long long abs_key(double a) {
  const unsigned long long u = (unsigned long long)__double_as_longlong(a) & 0x7fffffffffffffffull;
  return u > 0x7ff0000000000000ull ? 0ull : u;
}

// larger key wins; equal keys go to the lower row index
__device__ __forceinline__ void better_key(unsigned long long& best, int& bi,
                                           unsigned long long ob, int oi) {
  if (ob > best || (ob == best && oi < bi)) {
    best = ob;
    bi = oi;
  }
}

__device__ __forceinline__ void warp_best_key(unsigned long long& best, int& bi) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const unsigned long long ob = __shfl_down_sync(0xffffffffu, best, o);
    const int oi = __shfl_down_sync(0xffffffffu, bi, o);
    better_key(best, bi, ob, oi);
  }
}

__global__ void __launch_bounds__(kGjThreads) k_gj_cluster(int n, int R,
                                                           const double* __restrict__ A,
                                                           double* __restrict__ inv,
                                                           int* __restrict__ err) {
  cg::cluster_group cluster = cg::this_cluster();
  const int C = (int)cluster.num_blocks();
  const int c = (int)cluster.block_rank();
  extern __shared__ __align__(16) unsigned char smem[];
  const GjLayout lay(n, R);
  double* M = reinterpret_cast<double*>(smem + lay.M);
  double* prow = reinterpret_cast<double*>(smem + lay.prow);
  double* fr = reinterpret_cast<double*>(smem + lay.fr);
  unsigned long long* cand_k = reinterpret_cast<unsigned long long*>(smem + lay.cand_k);
  double* offer = reinterpret_cast<double*>(smem + lay.offer);
  double* s_ipiv = reinterpret_cast<double*>(smem + lay.ipiv);
  int* perm = reinterpret_cast<int*>(smem + lay.perm);
  int* pos = reinterpret_cast<int*>(smem + lay.pos);
  int* used = reinterpret_cast<int*>(smem + lay.used);
  int* cand_i = reinterpret_cast<int*>(smem + lay.cand_i);
  int* piv_row = reinterpret_cast<int*>(smem + lay.piv_row);

  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int r0 = c * R;
  const int rc = max(0, min(R, n - r0));  // rows this CTA owns
  for (int r = warp; r < rc; r += kGjWarps)
    for (int j = lane; j < n; j += 32) M[(size_t)r * n + j] = A[(size_t)(r0 + r) * n + j];
  for (int r = tid; r < R; r += kGjThreads) used[r] = 0;
  __syncthreads();

  for (int k = 0; k < n; ++k) {
    const int b = k & 1;  // offer buffers alternate between steps
    // this CTA's offer: its unused row with the largest |a_rk|, searched by
    // one warp on the magnitudes' bit patterns (integer compares; the FP64
    // pipe is narrow on this part), which then copies the row
    if (warp == 0) {
      unsigned long long best = 0ull;
      int bi = INT_MAX;
      for (int r = lane; r < rc; r += 32)
        if (!used[r]) better_key(best, bi, abs_key(M[(size_t)r * n + k]), r0 + r);
      warp_best_key(best, bi);
      if (lane == 0) {
        cand_k[b] = best;
        cand_i[b] = bi;
      }
      bi = __shfl_sync(0xffffffffu, bi, 0);
      if (bi != INT_MAX) {
        const double* w = M + (size_t)(bi - r0) * n;
        for (int j = lane; j < n; j += 32) offer[(size_t)b * n + j] = w[j];
      }
    }
    // every offer is visible cluster-wide; the buffers of step k - 1 are no
    // longer read by anyone
    cluster.sync();
    if (warp == 0) {
      unsigned long long best = 0ull;
      int bi = INT_MAX;
      if (lane < C) {
        best = cluster.map_shared_rank(cand_k, (unsigned)lane)[b];
        bi = cluster.map_shared_rank(cand_i, (unsigned)lane)[b];
      }
      warp_best_key(best, bi);
      // a zero (or NaN-only) column among the unused rows: singular
      if (lane == 0) piv_row[0] = (best > 0ull) ? bi : -1;
    }
    __syncthreads();
    const int p = piv_row[0];
    if (p < 0) {
      if (c == 0 && tid == 0) *err = 1;
      cluster.sync();  // no CTA leaves while another may still read its offer
      return;
    }
    const double* src = cluster.map_shared_rank(offer, (unsigned)(p / R)) + (size_t)b * n;
    for (int j = tid; j < n; j += kGjThreads) prow[j] = src[j];
    // FP64 division is slow on this part: one warp forms 1 / a_pk and the
    // row factors (meanwhile the others copy the pivot row), the update
    // multiplies
    if (warp == 0) {
      const double ipiv = 1.0 / src[k];
      if (lane == 0) {
        s_ipiv[0] = ipiv;
        perm[k] = p;
      }
      for (int r = lane; r < rc; r += 32) fr[r] = (r0 + r == p) ? 0.0 : M[(size_t)r * n + k] * ipiv;
    }
    __syncthreads();
    const double ipiv = s_ipiv[0];
    for (int r = warp; r < rc; r += kGjWarps) {
      double* m = M + (size_t)r * n;
      if (r0 + r == p) {
        for (int j = lane; j < n; j += 32) m[j] = (j == k) ? ipiv : prow[j] * ipiv;
      } else {
        const double f = fr[r];
        for (int j = lane; j < n; j += 32) m[j] = (j == k) ? -f : m[j] - f * prow[j];
      }
    }
    if (tid == 0 && p >= r0 && p < r0 + rc) used[p - r0] = 1;
    __syncthreads();
  }
  cluster.sync();  // the last offers have been read

  // A^{-1}[k][p_j] = M[p_k][j]
  for (int k = tid; k < n; k += kGjThreads) {
    const int g = perm[k];
    if (g >= r0 && g < r0 + rc) pos[g - r0] = k;
  }
  __syncthreads();
  for (int r = warp; r < rc; r += kGjWarps) {
    double* out = inv + (size_t)pos[r] * n;
    for (int j = lane; j < n; j += 32) out[perm[j]] = M[(size_t)r * n + j];
  }
}

struct GjConfig {
  int cluster = 0;   // 0: cluster launch unavailable
  size_t smem_max = 0;
};

// largest cluster (16, else 8) that can be resident with the largest shared
// memory a CTA may take on this device
GjConfig probe_gj() {
  GjConfig g;
  int dev = 0, optin = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) !=
          cudaSuccess) {
    cudaGetLastError();
    return g;
  }
  if (cudaFuncSetAttribute(k_gj_cluster, cudaFuncAttributeMaxDynamicSharedMemorySize, optin) !=
      cudaSuccess) {
    cudaGetLastError();
    return g;
  }
  for (int c : {16, 8}) {
    if (c > 8 && cudaFuncSetAttribute(k_gj_cluster, cudaFuncAttributeNonPortableClusterSizeAllowed,
                                      1) != cudaSuccess) {
      cudaGetLastError();
      continue;
    }
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute attr[1];
    cfg.gridDim = dim3(c);
    cfg.blockDim = dim3(kGjThreads);
    cfg.dynamicSmemBytes = (size_t)optin;
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = c;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    int nclusters = 0;
    if (cudaOccupancyMaxActiveClusters(&nclusters, k_gj_cluster, &cfg) == cudaSuccess &&
        nclusters >= 1) {
      g.cluster = c;
      g.smem_max = (size_t)optin;
      return g;
    }
    cudaGetLastError();
  }
  return g;
}

}  // namespace

bool coarse_inverse_cluster(int n, const double* A, double* inv, int* err, cudaStream_t s) {
  static const GjConfig g = probe_gj();
  if (g.cluster == 0 || n < 1) return false;
  const int R = (n + g.cluster - 1) / g.cluster;
  const GjLayout lay(n, R);
  if (lay.bytes > g.smem_max) return false;
  cudaLaunchConfig_t cfg = {};
  cudaLaunchAttribute attr[1];
  cfg.gridDim = dim3(g.cluster);
  cfg.blockDim = dim3(kGjThreads);
  cfg.dynamicSmemBytes = lay.bytes;
  cfg.stream = s;
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = g.cluster;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  TP_CUDA_TRY(cudaLaunchKernelEx(&cfg, k_gj_cluster, n, R, A, inv, err));
  return true;
}

}  // namespace tp

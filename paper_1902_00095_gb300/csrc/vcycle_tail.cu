// Coarse tail of the AMG V-cycle as one thread-block-cluster kernel.
//
// On the coarse Galerkin levels every phase of the V-cycle (smoothing,
// residual, restriction, the dense coarsest solve, prolongation) touches a
// few hundred kilobytes, so a chain of one kernel per phase costs mostly
// launch and drain latency. Here the levels from `first` down to the
// coarsest run inside one cluster of CTAs (16 where the device allows,
// else 8), separated by cluster barriers (release/acquire at cluster scope)
// instead of kernel boundaries. The arithmetic per row is that of the
// multi-kernel V-cycle (l1-Jacobi sweeps, the first two fused from a zero
// guess; r = b - A x; b_c = R r; x_c = A_c^{-1} b_c; x += P e), with rows
// split over groups of 8 lanes; the ping-pong order of the work vectors is
// the same, so the result lands in the buffer the host expects.
//
// Measured on GB300 (FGMRES time per iteration, 64x64x32 and 128x128x64
// hierarchies): slower than the per-phase kernels replayed in a CUDA graph
// with programmatic dependent launches at every threshold tried (levels of
// at most 256 rows: +4 % / +1 %; 12288 rows: +50 % / +11 %), because one
// cluster of 16 SMs streams the larger levels far slower than the whole GPU
// and even the tiny levels gain nothing over back-to-back dependent
// launches. It is therefore off by default (tail_rows = 0) and kept as an
// option.
//
// Vectors written inside the kernel are read with ld.global.cg (L2, never a
// stale L1 line) and written with st.global.cg; matrix values are
// read-only. Every thread of every CTA executes the same sequence of
// barriers: loop bounds depend only on level sizes.
#include "amg.cuh"

namespace tp {

namespace {

constexpr int kTailThreads = 1024;
constexpr int kTailLanes = 8;

// arrive.release / wait.acquire order every thread's global writes before
// the barrier with every thread's reads after it, at cluster scope
__device__ __forceinline__ void cluster_barrier() {
  asm volatile(
      "barrier.cluster.arrive.release;\n"
      "barrier.cluster.wait.acquire;\n" ::: "memory");
}

__device__ __forceinline__ float widen_h(__nv_bfloat16 v) { return __bfloat162float(v); }

template <class TV>
__device__ __forceinline__ TV lanes_sum(TV v) {
#pragma unroll
  for (int o = kTailLanes / 2; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o, kTailLanes);
  return v;
}

// sum_j a_ij x_j over the row owned by this lane group; values of type TV
template <class TV>
__device__ __forceinline__ TV dot_row(const int* rp, const int* col, const TV* val, const TV* x,
                                      int row, bool valid, int lane) {
  TV acc = TV(0);
  if (valid) {
    const int e1 = __ldg(rp + row + 1);
    for (int e = __ldg(rp + row) + lane; e < e1; e += kTailLanes)
      acc += __ldg(val + e) * __ldcg(x + __ldg(col + e));
  }
  return lanes_sum<TV>(acc);
}

// the same with BF16 values (precision 2 interpolation / restriction)
template <class TV>
__device__ __forceinline__ TV dot_row_h(const int* rp, const int* col, const __nv_bfloat16* val,
                                        const TV* x, int row, bool valid, int lane) {
  TV acc = TV(0);
  if (valid) {
    const int e1 = __ldg(rp + row + 1);
    for (int e = __ldg(rp + row) + lane; e < e1; e += kTailLanes)
      acc += (TV)widen_h(val[e]) * __ldcg(x + __ldg(col + e));
  }
  return lanes_sum<TV>(acc);
}

template <class TV>
__global__ void __launch_bounds__(kTailThreads) k_vcycle_tail(const TailLevel* __restrict__ D,
                                                              int first, int last,
                                                              const double* __restrict__ cinv,
                                                              int nc, int nu_pre, int nu_post) {
  const int T = gridDim.x * blockDim.x;
  const int g = blockIdx.x * blockDim.x + threadIdx.x;
  const int lane32 = g & 31;
  const int lane = g & (kTailLanes - 1);
  const int sub = lane32 / kTailLanes;            // row slot within the warp
  const int warp = g >> 5, nwarps = T >> 5;
  constexpr int kRowsPerWarp = 32 / kTailLanes;
  TV* curp[kMaxTailLevels];

  // ---------------------------------------------------------------- down
  for (int l = first; l < last; ++l) {
    const TailLevel Lv = D[l];
    const int n = Lv.n;
    const int* rp = Lv.Arp;
    const int* col = Lv.Acol;
    const TV* A = static_cast<const TV*>(Lv.Aval);
    const TV* dv = static_cast<const TV*>(Lv.dinv);
    TV* b = static_cast<TV*>(Lv.b);
    TV* x = static_cast<TV*>(Lv.x);
    TV* t = static_cast<TV*>(Lv.t);
    TV* r = static_cast<TV*>(Lv.r);
    int done = 1;
    if (nu_pre >= 2) {
      // x = d b + d (b - A (d b)): two sweeps from a zero guess
      for (int base = warp * kRowsPerWarp; base < n; base += nwarps * kRowsPerWarp) {
        const int row = base + sub;
        const bool valid = row < n;
        TV acc = TV(0);
        if (valid) {
          const int e1 = __ldg(rp + row + 1);
          for (int e = __ldg(rp + row) + lane; e < e1; e += kTailLanes) {
            const int j = __ldg(col + e);
            acc += __ldg(A + e) * (__ldg(dv + j) * __ldcg(b + j));
          }
        }
        acc = lanes_sum<TV>(acc);
        if (valid && lane == 0) {
          const TV d = __ldg(dv + row), bi = __ldcg(b + row);
          __stcg(x + row, d * bi + d * (bi - acc));
        }
      }
      done = 2;
    } else {
      for (int i = g; i < n; i += T) __stcg(x + i, __ldg(dv + i) * __ldcg(b + i));
    }
    cluster_barrier();
    TV* cur = x;
    TV* oth = t;
    for (int k = done; k < nu_pre; ++k) {
      for (int base = warp * kRowsPerWarp; base < n; base += nwarps * kRowsPerWarp) {
        const int row = base + sub;
        const bool valid = row < n;
        const TV ax = dot_row<TV>(rp, col, A, cur, row, valid, lane);
        if (valid && lane == 0)
          __stcg(oth + row, __ldcg(cur + row) + __ldg(dv + row) * (__ldcg(b + row) - ax));
      }
      cluster_barrier();
      TV* tmp = cur;
      cur = oth;
      oth = tmp;
    }
    // residual
    for (int base = warp * kRowsPerWarp; base < n; base += nwarps * kRowsPerWarp) {
      const int row = base + sub;
      const bool valid = row < n;
      const TV ax = dot_row<TV>(rp, col, A, cur, row, valid, lane);
      if (valid && lane == 0) __stcg(r + row, __ldcg(b + row) - ax);
    }
    cluster_barrier();
    // restriction into the next level's right-hand side
    TV* bn = static_cast<TV*>(D[l + 1].b);
    const int nn = Lv.nnext;
    for (int base = warp * kRowsPerWarp; base < nn; base += nwarps * kRowsPerWarp) {
      const int row = base + sub;
      const bool valid = row < nn;
      const TV v = Lv.Rh ? dot_row_h<TV>(Lv.Rrp, Lv.Rcol, Lv.Rh, r, row, valid, lane)
                         : dot_row<TV>(Lv.Rrp, Lv.Rcol, static_cast<const TV*>(Lv.Rval), r, row,
                                       valid, lane);
      if (valid && lane == 0) __stcg(bn + row, v);
    }
    cluster_barrier();
    curp[l - first] = cur;
  }

  // ------------------------------------------------------------ coarsest
  {
    const TV* bc = static_cast<const TV*>(D[last].b);
    TV* xc = static_cast<TV*>(D[last].x);
    for (int row = warp; row < nc; row += nwarps) {
      double acc = 0.0;
      for (int j = lane32; j < nc; j += 32)
        acc += __ldg(cinv + (long long)row * nc + j) * (double)__ldcg(bc + j);
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
      if (lane32 == 0) __stcg(xc + row, (TV)acc);
    }
    cluster_barrier();
  }

  // ------------------------------------------------------------------ up
  const TV* e = static_cast<const TV*>(D[last].x);
  for (int l = last - 1; l >= first; --l) {
    const TailLevel Lv = D[l];
    const int n = Lv.n;
    const int* rp = Lv.Arp;
    const int* col = Lv.Acol;
    const TV* A = static_cast<const TV*>(Lv.Aval);
    const TV* dv = static_cast<const TV*>(Lv.dinv);
    const TV* b = static_cast<const TV*>(Lv.b);
    TV* x = static_cast<TV*>(Lv.x);
    TV* t = static_cast<TV*>(Lv.t);
    TV* cur = curp[l - first];
    TV* oth = (cur == x) ? t : x;
    // x += P e
    for (int base = warp * kRowsPerWarp; base < n; base += nwarps * kRowsPerWarp) {
      const int row = base + sub;
      const bool valid = row < n;
      const TV pe = Lv.Ph ? dot_row_h<TV>(Lv.Prp, Lv.Pcol, Lv.Ph, e, row, valid, lane)
                          : dot_row<TV>(Lv.Prp, Lv.Pcol, static_cast<const TV*>(Lv.Pval), e, row,
                                        valid, lane);
      if (valid && lane == 0) __stcg(cur + row, __ldcg(cur + row) + pe);
    }
    cluster_barrier();
    for (int k = 1; k <= nu_post; ++k) {
      for (int base = warp * kRowsPerWarp; base < n; base += nwarps * kRowsPerWarp) {
        const int row = base + sub;
        const bool valid = row < n;
        const TV ax = dot_row<TV>(rp, col, A, cur, row, valid, lane);
        if (valid && lane == 0)
          __stcg(oth + row, __ldcg(cur + row) + __ldg(dv + row) * (__ldcg(b + row) - ax));
      }
      cluster_barrier();
      TV* tmp = cur;
      cur = oth;
      oth = tmp;
    }
    e = cur;
  }
}

template <class TV>
cudaLaunchConfig_t tail_config(int cluster, cudaStream_t s, cudaLaunchAttribute* attr) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(cluster);
  cfg.blockDim = dim3(kTailThreads);
  cfg.dynamicSmemBytes = 0;
  cfg.stream = s;
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = cluster;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cfg;
}

// largest cluster (16, else 8) of which at least one can be resident, for
// both value types; 0 when clusters cannot be launched
int probe_cluster_size() {
  for (int c : {16, 8}) {
    bool ok = true;
    for (int f = 0; f < 2 && ok; ++f) {
      const void* fn = f == 0 ? (const void*)k_vcycle_tail<double> : (const void*)k_vcycle_tail<float>;
      if (c > 8 &&
          cudaFuncSetAttribute(fn, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) !=
              cudaSuccess) {
        cudaGetLastError();
        ok = false;
        break;
      }
      cudaLaunchAttribute attr[1];
      cudaLaunchConfig_t cfg = tail_config<double>(c, nullptr, attr);
      int nclusters = 0;
      if (cudaOccupancyMaxActiveClusters(&nclusters, fn, &cfg) != cudaSuccess || nclusters < 1) {
        cudaGetLastError();
        ok = false;
      }
    }
    if (ok) return c;
  }
  return 0;
}

}  // namespace

int tail_cluster_size() {
  static const int c = probe_cluster_size();
  return c;
}

template <class TV>
void launch_vcycle_tail(const TailLevel* desc, int first, int last, const double* cinv, int nc,
                        int nu_pre, int nu_post, int cluster, cudaStream_t s) {
  cudaLaunchAttribute attr[1];
  cudaLaunchConfig_t cfg = tail_config<TV>(cluster, s, attr);
  TP_CUDA_TRY(cudaLaunchKernelEx(&cfg, k_vcycle_tail<TV>, desc, first, last, cinv, nc, nu_pre,
                                 nu_post));
  count_launch();
}

template void launch_vcycle_tail<double>(const TailLevel*, int, int, const double*, int, int, int,
                                         int, cudaStream_t);
template void launch_vcycle_tail<float>(const TailLevel*, int, int, const double*, int, int, int,
                                        int, cudaStream_t);

}  // namespace tp

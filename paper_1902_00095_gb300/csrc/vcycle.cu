// AMG V-cycle kernels (l1-Jacobi smoothing, residual, restriction,
// prolongation, coarsest dense solve) in FP64 or FP32.
//
// CSR rows are processed by groups of LANES consecutive threads (LANES a
// power of two chosen from the mean row length), reduced with warp shuffles.
// On the finest level of an FP32 hierarchy the right-hand side is read in
// FP64 and the final post-smoothing sweep writes the FP64 result directly,
// so no conversion passes are needed at the preconditioner boundary.
//
// Every kernel is launched as a programmatic dependent launch. The level
// operators (pattern, values, l1 scaling, coarsest inverse) do not change
// during a V-cycle, so each kernel loads its share of them before
// griddepcontrol.wait, while the previous kernel is still running, and only
// the vectors the previous kernels wrote after it. The first kernel of a
// V-cycle (level 0 pre-smoothing) waits first: the kernel before it may be a
// setup kernel that wrote those operators.
#include "amg.cuh"

namespace tp {

namespace {

// value conversion (BF16 interpolation weights are widened to the vector type)
template <class TV, class TP>
__device__ __forceinline__ TV widen(TP v) {
  return (TV)v;
}
template <>
__device__ __forceinline__ float widen<float, __nv_bfloat16>(__nv_bfloat16 v) {
  return __bfloat162float(v);
}
template <>
__device__ __forceinline__ double widen<double, __nv_bfloat16>(__nv_bfloat16 v) {
  return (double)__bfloat162float(v);
}

template <int LANES, class T>
__device__ __forceinline__ T group_sum(T v) {
#pragma unroll
  for (int o = LANES / 2; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o, LANES);
  return v;
}

// The part of one CSR row a lane owns (entries rp[row] + lane + k LANES):
// the column indices and values of its first K entries are held in
// registers (loaded before the dependency wait), the rest are read in the
// dot itself. Summation order is the plain lane-strided order. K is 4 for
// 8-byte values and 8 for narrower ones (about the same registers; measured
// on the 64x64x32 and 128x128x64 hierarchies: FP64 sweeps slower with 8,
// FP32 ones faster).

template <class TP>
constexpr int row_pre() {
  return sizeof(TP) >= 8 ? 4 : 8;
}

template <int LANES, class TP>
struct RowPre {
  static constexpr int K = row_pre<TP>();
  int e = 0, e1 = 0;
  int c[K];
  TP v[K];

  __device__ __forceinline__ void load(const int* __restrict__ rp, const int* __restrict__ col,
                                       const TP* __restrict__ val, int row, bool valid,
                                       int lane) {
    if (valid) {
      e = rp[row] + lane;
      e1 = rp[row + 1];
    }
#pragma unroll
    for (int k = 0; k < K; ++k) {
      const int q = e + k * LANES;
      c[k] = 0;
      v[k] = TP{};
      if (q < e1) {
        c[k] = col[q];
        v[k] = val[q];
      }
    }
  }

  // sum_j a_ij x_j over the lane's entries, reduced over the row's lanes
  template <class TV, class TX>
  __device__ __forceinline__ TV dot(const int* __restrict__ col, const TP* __restrict__ val,
                                    const TX* __restrict__ x) const {
    TV acc = TV(0);
#pragma unroll
    for (int k = 0; k < K; ++k)
      if (e + k * LANES < e1) acc += widen<TV, TP>(v[k]) * (TV)x[c[k]];
    for (int q = e + K * LANES; q < e1; q += LANES)
      acc += widen<TV, TP>(val[q]) * (TV)x[col[q]];
    return group_sum<LANES>(acc);
  }
};

// x_out = x_in + dinv (b - A x_in)
template <int LANES, class TV, class TB, class TO>
__global__ void __launch_bounds__(256) k_jacobi(int n, const int* __restrict__ rp,
                                                const int* __restrict__ col,
                                                const TV* __restrict__ val,
                                                const TV* __restrict__ dinv,
                                                const TB* __restrict__ b,
                                                const TV* __restrict__ xin, TO* __restrict__ xout) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  const int row = t / LANES, lane = t % LANES;
  const bool valid = row < n;
  RowPre<LANES, TV> a;
  a.load(rp, col, val, row, valid, lane);
  TV di = TV(0);
  if (valid && lane == 0) di = dinv[row];
  pdl_wait();
  pdl_trigger();
  // the row's own vector entries are loaded before the dot so their latency
  // overlaps the gathers instead of following the reduction
  TV xi = TV(0), bi = TV(0);
  if (valid && lane == 0) {
    xi = xin[row];
    bi = (TV)b[row];
  }
  TV ax = a.template dot<TV, TV>(col, val, xin);
  if (valid && lane == 0) xout[row] = (TO)(xi + di * (bi - ax));
}

// x = dinv b (first sweep from a zero guess)
template <class TV, class TB>
__global__ void k_jacobi0(int n, const TV* __restrict__ dinv, const TB* __restrict__ b,
                          TV* __restrict__ x, int first) {
  if (first) pdl_wait();
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const TV d = i < n ? dinv[i] : TV(0);
  pdl_wait();
  pdl_trigger();
  if (i < n) x[i] = d * (TV)b[i];
}

// y = d b (rounded as in the sweeps): the first sweep from a zero guess,
// read by the fused two-sweep kernels below instead of forming d_j b_j for
// every matrix entry (two FP64 operations per entry on a pipe that bounds
// these sweeps). first: the kernel opens a V-cycle (waits before any read).
template <class TV, class TB>
__global__ void k_scale_db(int n, const TV* __restrict__ dinv, const TB* __restrict__ b,
                           TV* __restrict__ y, int first) {
  if (first) pdl_wait();
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const TV d = i < n ? dinv[i] : TV(0);
  pdl_wait();
  pdl_trigger();
  if (i < n) y[i] = d * (TV)b[i];
}

// two sweeps from a zero guess in one pass, y = d b from k_scale_db:
// x = d b + d (b - A y)
template <int LANES, class TV, class TB>
__global__ void __launch_bounds__(256) k_jacobi2z(int n, const int* __restrict__ rp,
                                                  const int* __restrict__ col,
                                                  const TV* __restrict__ val,
                                                  const TV* __restrict__ dinv,
                                                  const TB* __restrict__ b,
                                                  const TV* __restrict__ y,
                                                  TV* __restrict__ x) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  const int row = t / LANES, lane = t % LANES;
  const bool valid = row < n;
  RowPre<LANES, TV> a;
  a.load(rp, col, val, row, valid, lane);
  TV d = TV(0);
  if (valid && lane == 0) d = dinv[row];
  constexpr int K = RowPre<LANES, TV>::K;
  pdl_wait();
  pdl_trigger();
  TV bi = TV(0);
  if (valid && lane == 0) bi = (TV)b[row];
  TV acc = TV(0);
#pragma unroll
  for (int k = 0; k < K; ++k)
    if (a.e + k * LANES < a.e1) acc += a.v[k] * y[a.c[k]];
  for (int q = a.e + K * LANES; q < a.e1; q += LANES) acc += val[q] * y[col[q]];
  acc = group_sum<LANES>(acc);
  if (valid && lane == 0) x[row] = d * bi + d * (bi - acc);
}

// column of slot k of row `row` in an ELL copy by grid direction (offsets
// -nxy, -nx, -1, 0, +1, +nx, +nxy), clamped to [0, n): an absent neighbour's
// slot holds 0, so any column in range adds an exact zero
__device__ __forceinline__ int stencil_col(int k, int row, int n, int nx, int nxy) {
  const int o = k == 0 ? -nxy : k == 1 ? -nx : k == 2 ? -1 : k == 3 ? 0 : k == 4 ? 1
              : k == 5 ? nx : nxy;
  const int c = row + o;
  return c < 0 ? 0 : (c >= n ? n - 1 : c);
}

// ELL forms (slot-major, one thread per row, coalesced over rows); a row's
// slots are held in registers, loaded before the dependency wait. ecol null:
// the slots are the grid directions of an nx x ny x nz grid (nxy = nx ny)
template <class TV>
struct EllRow {
  int c[kEllMaxW];
  TV v[kEllMaxW];

  __device__ __forceinline__ void load(int n, int w, const int* __restrict__ ecol,
                                       const TV* __restrict__ eval, int row, int nx, int nxy) {
#pragma unroll
    for (int k = 0; k < kEllMaxW; ++k) {
      c[k] = 0;
      v[k] = TV(0);
      if (k < w) {
        const long long q = (long long)k * n + row;
        c[k] = ecol ? ecol[q] : stencil_col(k, row, n, nx, nxy);
        v[k] = eval[q];
      }
    }
  }

  template <class TX>
  __device__ __forceinline__ TV dot(int w, const TX* __restrict__ x) const {
    TV acc = TV(0);
#pragma unroll
    for (int k = 0; k < kEllMaxW; ++k)
      if (k < w) acc += v[k] * (TV)x[c[k]];
    return acc;
  }
};

template <class TV, class TB, class TO>
__global__ void __launch_bounds__(256) k_jacobi_ell(int n, int w, const int* __restrict__ ecol, int snx, int snxy,
                                                    const TV* __restrict__ eval,
                                                    const TV* __restrict__ dinv,
                                                    const TB* __restrict__ b,
                                                    const TV* __restrict__ xin,
                                                    TO* __restrict__ xout) {
  const int row = blockIdx.x * blockDim.x + threadIdx.x;
  EllRow<TV> a;
  TV di = TV(0);
  if (row < n) {
    a.load(n, w, ecol, eval, row, snx, snxy);
    di = dinv[row];
  }
  pdl_wait();
  pdl_trigger();
  if (row >= n) return;
  const TV xi = xin[row], bi = (TV)b[row];
  const TV ax = a.dot(w, xin);
  xout[row] = (TO)(xi + di * (bi - ax));
}

template <class TV, class TB>
__global__ void __launch_bounds__(256) k_residual_ell(int n, int w, const int* __restrict__ ecol, int snx, int snxy,
                                                      const TV* __restrict__ eval,
                                                      const TB* __restrict__ b,
                                                      const TV* __restrict__ x,
                                                      TV* __restrict__ r) {
  const int row = blockIdx.x * blockDim.x + threadIdx.x;
  EllRow<TV> a;
  if (row < n) a.load(n, w, ecol, eval, row, snx, snxy);
  pdl_wait();
  pdl_trigger();
  if (row >= n) return;
  const TV bi = (TV)b[row];
  r[row] = bi - a.dot(w, x);
}

template <class TV, class TB>
__global__ void __launch_bounds__(256) k_jacobi2z_ell(int n, int w, const int* __restrict__ ecol,
                                                      int snx, int snxy,
                                                      const TV* __restrict__ eval,
                                                      const TV* __restrict__ dinv,
                                                      const TB* __restrict__ b,
                                                      const TV* __restrict__ y,
                                                      TV* __restrict__ x) {
  const int row = blockIdx.x * blockDim.x + threadIdx.x;
  EllRow<TV> a;
  TV d = TV(0);
  if (row < n) {
    a.load(n, w, ecol, eval, row, snx, snxy);
    d = dinv[row];
  }
  pdl_wait();
  pdl_trigger();
  if (row >= n) return;
  const TV bi = (TV)b[row];
  TV acc = TV(0);
#pragma unroll
  for (int k = 0; k < kEllMaxW; ++k)
    if (k < w) acc += a.v[k] * y[a.c[k]];
  x[row] = d * bi + d * (bi - acc);
}

// r = b - A x
template <int LANES, class TV, class TB>
__global__ void __launch_bounds__(256) k_residual(int n, const int* __restrict__ rp,
                                                  const int* __restrict__ col,
                                                  const TV* __restrict__ val,
                                                  const TB* __restrict__ b,
                                                  const TV* __restrict__ x, TV* __restrict__ r) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  const int row = t / LANES, lane = t % LANES;
  const bool valid = row < n;
  RowPre<LANES, TV> a;
  a.load(rp, col, val, row, valid, lane);
  pdl_wait();
  pdl_trigger();
  TV bi = TV(0);
  if (valid && lane == 0) bi = (TV)b[row];
  TV ax = a.template dot<TV, TV>(col, val, x);
  if (valid && lane == 0) r[row] = bi - ax;
}

// y = R x (restriction; R values of type TP)
template <int LANES, class TP, class TV>
// y = A x (the restriction); with dsc, also ysc = dsc y, rounded as in the
// coarse level's first sweep from zero (d b: its k_jacobi0 result or the y of
// its fused two sweeps), which then needs no kernel of its own
__global__ void __launch_bounds__(256) k_spmv(int n, const int* __restrict__ rp,
                                              const int* __restrict__ col,
                                              const TP* __restrict__ val,
                                              const TV* __restrict__ x, TV* __restrict__ y,
                                              const TV* __restrict__ dsc,
                                              TV* __restrict__ ysc) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  const int row = t / LANES, lane = t % LANES;
  const bool valid = row < n;
  RowPre<LANES, TP> a;
  a.load(rp, col, val, row, valid, lane);
  const TV d = (dsc && valid && lane == 0) ? dsc[row] : TV(0);
  pdl_wait();
  pdl_trigger();
  TV ax = a.template dot<TV, TV>(col, val, x);
  if (valid && lane == 0) {
    y[row] = ax;
    if (dsc) ysc[row] = d * ax;
  }
}

// x += P e (prolongation; P values of type TP)
template <int LANES, class TP, class TV>
__global__ void __launch_bounds__(256) k_prolong(int n, const int* __restrict__ rp,
                                                 const int* __restrict__ col,
                                                 const TP* __restrict__ val,
                                                 const TV* __restrict__ e, TV* __restrict__ x) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  const int row = t / LANES, lane = t % LANES;
  const bool valid = row < n;
  RowPre<LANES, TP> a;
  a.load(rp, col, val, row, valid, lane);
  pdl_wait();
  pdl_trigger();
  TV xi = TV(0);
  if (valid && lane == 0) xi = x[row];
  TV pe = a.template dot<TV, TV>(col, val, e);
  if (valid && lane == 0) x[row] = xi + pe;
}

// x = Ainv b on the coarsest level (dense FP64 inverse), one warp per row
template <class TB, class TO>
__global__ void k_coarse(int n, const double* __restrict__ inv, const TB* __restrict__ b,
                         TO* __restrict__ x) {
  const int row = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  constexpr int kPre = 4;  // columns j = lane + 32 k, k < kPre, held before the wait
  double a[kPre];
#pragma unroll
  for (int k = 0; k < kPre; ++k) {
    const int j = lane + 32 * k;
    a[k] = (row < n && j < n) ? inv[(long long)row * n + j] : 0.0;
  }
  pdl_wait();
  pdl_trigger();
  if (row >= n) return;
  double acc = 0.0;
#pragma unroll
  for (int k = 0; k < kPre; ++k)
    if (lane + 32 * k < n) acc += a[k] * (double)b[lane + 32 * k];
  for (int j = lane + 32 * kPre; j < n; j += 32) acc += inv[(long long)row * n + j] * (double)b[j];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
  if (lane == 0) x[row] = (TO)acc;
}

// Vertical-line step x_out = x_in + T^-1 (b - A x_in) (x_in null: x_out =
// T^-1 b) with the twisted factorisation of k_line_factor: two threads per
// column c of the nxy x nz grid (cell c + nxy k), adjacent lanes. With mid =
// nz / 2 the even lane eliminates the top rows downwards and the odd lane
// the bottom rows upwards, in the same instructions (the stored coefficients
// make the two recurrences one: g = (r - lo g_prev) minv), each forming its
// residual rows on the way (ELL slots when the level has them, else the CSR
// row) and parking g in x_out. The even lane then solves the middle row with
// the odd lane's last g (a shuffle), and both substitute back towards their
// ends, e = g - cp e_prev. Half the serial chain of a one-thread Thomas
// solve, twice the threads.
template <class TV, class TB, class TO>
__global__ void __launch_bounds__(128) k_line_sweep(
    int nxy, int nz, int n, int ell_w, const int* __restrict__ ecol, int snx, int snxy,
    const TV* __restrict__ eval,
    const int* __restrict__ rp, const int* __restrict__ col, const TV* __restrict__ val,
    const TV* __restrict__ lo, const TV* __restrict__ minv, const TV* __restrict__ cp,
    const TB* __restrict__ b, const TV* __restrict__ xin, TO* __restrict__ xout) {
  pdl_wait();
  pdl_trigger();
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  const int c = t >> 1, role = t & 1;  // role 0: top rows, 1: bottom rows
  const bool act = c < nxy;
  const int mid = nz >> 1;
  const int nsteps = role ? nz - 1 - mid : mid;
  auto rrow = [&](int i) -> TV {
    TV r = (TV)b[i];
    if (xin) {
      TV ax = TV(0);
      if (ell_w > 0) {
#pragma unroll
        for (int q = 0; q < kEllMaxW; ++q)
          if (q < ell_w) {
            const long long e = (long long)q * n + i;
            ax += eval[e] * xin[ecol ? ecol[e] : stencil_col(q, i, n, snx, snxy)];
          }
      } else {
        for (int e = rp[i]; e < rp[i + 1]; ++e) ax += val[e] * xin[col[e]];
      }
      r -= ax;
    }
    return r;
  };
  TV gprev = TV(0);
#pragma unroll 2
  for (int s = 0; s < mid; ++s) {
    if (act && s < nsteps) {
      const int i = c + (role ? nz - 1 - s : s) * nxy;
      const TV g = (rrow(i) - lo[i] * gprev) * minv[i];
      xout[i] = (TO)g;
      gprev = g;
    }
  }
  // middle row: the top lane takes the bottom lane's last g
  const TV gb = __shfl_down_sync(0xffffffffu, gprev, 1);
  TV xm = TV(0);
  if (act && role == 0) {
    const int i = c + mid * nxy;
    const TV gt = mid > 0 ? gprev : TV(0);
    const TV gu = mid + 1 < nz ? gb : TV(0);
    xm = (rrow(i) - lo[i] * gt - cp[i] * gu) * minv[i];
    xout[i] = (TO)(xin ? xin[i] + xm : xm);
  }
  TV enext = __shfl_sync(0xffffffffu, xm, (threadIdx.x & 31) & ~1);
#pragma unroll 2
  for (int s = 0; s < mid; ++s) {
    if (act && s < nsteps) {
      const int i = c + (role ? mid + 1 + s : mid - 1 - s) * nxy;
      const TV e = (TV)xout[i] - cp[i] * enext;
      xout[i] = (TO)(xin ? xin[i] + e : e);
      enext = e;
    }
  }
}

// Sliced-ELL forms (levels below the finest with long rows): one thread per
// row in length-sorted order, one warp per 32-row slice, so a warp loads 32
// consecutive entries at each step and its lanes idle only on the slice's
// padding; a row's sum runs over its entries in CSR order. The row of each
// slot, the slice extent and the first K entries are loaded before the
// dependency wait.
template <class TV>
struct SellRow {
  static constexpr int K = sizeof(TV) >= 8 ? 4 : 8;
  int row = -1, q0 = 0, w = 0;
  int c[K];
  TV v[K];

  __device__ __forceinline__ void load(int nslots, const int* __restrict__ ptr,
                                       const int* __restrict__ perm, const int* __restrict__ col,
                                       const TV* __restrict__ val, int t) {
    if (t < nslots) {
      const int sl = t >> 5;
      row = perm[t];
      q0 = ptr[sl] + (t & 31);
      w = (ptr[sl + 1] - ptr[sl]) >> 5;
    }
#pragma unroll
    for (int k = 0; k < K; ++k) {
      c[k] = 0;
      v[k] = TV(0);
      if (k < w) {
        c[k] = col[q0 + 32 * k];
        v[k] = val[q0 + 32 * k];
      }
    }
  }

  // FP64: the next group's K entries are loaded while the current group's
  // gathers are in flight (one DRAM round trip per group instead of two);
  // FP32 rows hold 2K entries in the first group and keep the plain loop
  // (measured faster there)
  template <class TX>
  __device__ __forceinline__ TV dot(const int* __restrict__ col, const TV* __restrict__ val,
                                    const TX* __restrict__ x) const {
    TV acc = TV(0);
    if constexpr (sizeof(TV) >= 8) {
      int cc[K];
      TV vv[K];
#pragma unroll
      for (int k = 0; k < K; ++k) {
        cc[k] = c[k];
        vv[k] = v[k];
      }
      for (int k0 = 0; k0 < w; k0 += K) {
        TV xv[K];
#pragma unroll
        for (int j = 0; j < K; ++j) xv[j] = (k0 + j < w) ? (TV)x[cc[j]] : TV(0);
        int cn[K];
        TV vn[K];
#pragma unroll
        for (int j = 0; j < K; ++j) {
          const int k = k0 + K + j;
          cn[j] = 0;
          vn[j] = TV(0);
          if (k < w) {
            cn[j] = col[q0 + 32 * k];
            vn[j] = val[q0 + 32 * k];
          }
        }
#pragma unroll
        for (int j = 0; j < K; ++j)
          if (k0 + j < w) acc += vv[j] * xv[j];
#pragma unroll
        for (int j = 0; j < K; ++j) {
          cc[j] = cn[j];
          vv[j] = vn[j];
        }
      }
    } else {
#pragma unroll
      for (int k = 0; k < K; ++k)
        if (k < w) acc += v[k] * (TV)x[c[k]];
      for (int k = K; k < w; ++k) acc += val[q0 + 32 * k] * (TV)x[col[q0 + 32 * k]];
    }
    return acc;
  }
};

template <class TV, class TB, class TO>
__global__ void __launch_bounds__(256) k_sell_jacobi(int nslots, const int* __restrict__ ptr,
                                                     const int* __restrict__ perm,
                                                     const int* __restrict__ col,
                                                     const TV* __restrict__ val,
                                                     const TV* __restrict__ dinv,
                                                     const TB* __restrict__ b,
                                                     const TV* __restrict__ xin,
                                                     TO* __restrict__ xout) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  SellRow<TV> a;
  a.load(nslots, ptr, perm, col, val, t);
  const TV di = a.row >= 0 ? dinv[a.row] : TV(0);
  pdl_wait();
  pdl_trigger();
  if (a.row < 0) return;
  const TV xi = xin[a.row], bi = (TV)b[a.row];
  const TV ax = a.dot(col, val, xin);
  xout[a.row] = (TO)(xi + di * (bi - ax));
}

template <class TV, class TB>
__global__ void __launch_bounds__(256) k_sell_residual(int nslots, const int* __restrict__ ptr,
                                                       const int* __restrict__ perm,
                                                       const int* __restrict__ col,
                                                       const TV* __restrict__ val,
                                                       const TB* __restrict__ b,
                                                       const TV* __restrict__ x,
                                                       TV* __restrict__ r) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  SellRow<TV> a;
  a.load(nslots, ptr, perm, col, val, t);
  pdl_wait();
  pdl_trigger();
  if (a.row < 0) return;
  const TV bi = (TV)b[a.row];
  r[a.row] = bi - a.dot(col, val, x);
}

// two sweeps from a zero guess, y = d b from k_scale_db: x = d b + d (b - A y)
template <class TV, class TB>
__global__ void __launch_bounds__(256) k_sell_jacobi2z(int nslots, const int* __restrict__ ptr,
                                                       const int* __restrict__ perm,
                                                       const int* __restrict__ col,
                                                       const TV* __restrict__ val,
                                                       const TV* __restrict__ dinv,
                                                       const TB* __restrict__ b,
                                                       const TV* __restrict__ y,
                                                       TV* __restrict__ x) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  SellRow<TV> a;
  a.load(nslots, ptr, perm, col, val, t);
  const TV d = a.row >= 0 ? dinv[a.row] : TV(0);
  pdl_wait();
  pdl_trigger();
  if (a.row < 0) return;
  const TV bi = (TV)b[a.row];
  TV acc = TV(0);
  constexpr int K = SellRow<TV>::K;
#pragma unroll
  for (int k = 0; k < K; ++k)
    if (k < a.w) acc += a.v[k] * y[a.c[k]];
  for (int k = K; k < a.w; ++k) acc += val[a.q0 + 32 * k] * y[col[a.q0 + 32 * k]];
  x[a.row] = d * bi + d * (bi - acc);
}

template <class TV, class TB, class TO>
void jacobi(int lanes, const DevCSR& A, const TV* val, const TV* dinv, const TB* b, const TV* xin,
            TO* xout, cudaStream_t s) {
  const long long threads = (long long)A.n * lanes;
  const int g = grid_for(threads);
  switch (lanes) {
#define TP_CASE(L)                                                                          \
  case L:                                                                                   \
    launch_pdl(k_jacobi<L, TV, TB, TO>, g, kBlock, s, A.n, A.rowptr, A.col, val, dinv, b,  \
               xin, xout);                                                                  \
    break;
    TP_CASE(1) TP_CASE(2) TP_CASE(4) TP_CASE(8) TP_CASE(16) TP_CASE(32)
#undef TP_CASE
  }
}

template <class TV, class TB>
void jacobi2z(int lanes, const DevCSR& A, const TV* val, const TV* dinv, const TB* b,
              const TV* y, TV* x, cudaStream_t s) {
  const int g = grid_for((long long)A.n * lanes);
  switch (lanes) {
#define TP_CASE(L)                                                                         \
  case L:                                                                                  \
    launch_pdl(k_jacobi2z<L, TV, TB>, g, kBlock, s, A.n, A.rowptr, A.col, val, dinv, b, y, \
               x);                                                                         \
    break;
    TP_CASE(1) TP_CASE(2) TP_CASE(4) TP_CASE(8) TP_CASE(16) TP_CASE(32)
#undef TP_CASE
  }
}

template <class TV, class TB>
void residual(int lanes, const DevCSR& A, const TV* val, const TB* b, const TV* x, TV* r,
              cudaStream_t s) {
  const int g = grid_for((long long)A.n * lanes);
  switch (lanes) {
#define TP_CASE(L)                                                                      \
  case L:                                                                               \
    launch_pdl(k_residual<L, TV, TB>, g, kBlock, s, A.n, A.rowptr, A.col, val, b, x, r);  \
    break;
    TP_CASE(1) TP_CASE(2) TP_CASE(4) TP_CASE(8) TP_CASE(16) TP_CASE(32)
#undef TP_CASE
  }
}

template <class TP, class TV>
void spmv(int lanes, const DevCSR& A, const TP* val, const TV* x, TV* y, cudaStream_t s,
          const TV* dsc = nullptr, TV* ysc = nullptr) {
  const int g = grid_for((long long)A.n * lanes);
  switch (lanes) {
#define TP_CASE(L)                                                                           \
  case L:                                                                                    \
    launch_pdl(k_spmv<L, TP, TV>, g, kBlock, s, A.n, A.rowptr, A.col, val, x, y, dsc, ysc);  \
    break;
    TP_CASE(1) TP_CASE(2) TP_CASE(4) TP_CASE(8) TP_CASE(16) TP_CASE(32)
#undef TP_CASE
  }
}

template <class TP, class TV>
void prolong(int lanes, const DevCSR& P, const TP* val, const TV* e, TV* x, cudaStream_t s) {
  const int g = grid_for((long long)P.n * lanes);
  switch (lanes) {
#define TP_CASE(L)                                                                      \
  case L:                                                                               \
    launch_pdl(k_prolong<L, TP, TV>, g, kBlock, s, P.n, P.rowptr, P.col, val, e, x);    \
    break;
    TP_CASE(1) TP_CASE(2) TP_CASE(4) TP_CASE(8) TP_CASE(16) TP_CASE(32)
#undef TP_CASE
  }
}

template <class TB, class TO>
void coarse(int n, const double* inv, const TB* b, TO* x, cudaStream_t s) {
  launch_pdl(k_coarse<TB, TO>, grid_for((long long)n * 32), kBlock, s, n, inv, b, x);
}

template <class TV>
struct Vals {
  static const TV* A(const Level& l);
  static const TV* P(const Level& l);
  static const TV* R(const Level& l);
  static const TV* dinv(const Level& l);
};
template <>
struct Vals<double> {
  static const double* S(const Level& l) { return l.sell_val; }
  static const double* lo(const Level& l) { return l.line_lo; }
  static const double* minv(const Level& l) { return l.line_minv; }
  static const double* cp(const Level& l) { return l.line_cp; }
  static const double* E(const Level& l) { return l.ell_val; }
  static const double* A(const Level& l) { return l.A.val; }
  static const double* P(const Level& l) { return l.P.val; }
  static const double* R(const Level& l) { return l.R.val; }
  static const double* dinv(const Level& l) { return l.dinv; }
};
template <>
struct Vals<float> {
  static const float* S(const Level& l) { return l.sell_valf; }
  static const float* lo(const Level& l) { return l.line_lof; }
  static const float* minv(const Level& l) { return l.line_minvf; }
  static const float* cp(const Level& l) { return l.line_cpf; }
  static const float* E(const Level& l) { return l.ell_valf; }
  static const float* A(const Level& l) { return l.A.valf; }
  static const float* P(const Level& l) { return l.P.valf; }
  static const float* R(const Level& l) { return l.R.valf; }
  static const float* dinv(const Level& l) { return l.dinvf; }
};

// One V-cycle on level l for right-hand side b (type TB). The result goes to
// `final_out` (type TO) when non-null, else to one of the level's work
// vectors, whose address is returned.
// level operations: ELL when the level has an ELL copy, CSR otherwise
template <class TV, class TB, class TO>
void level_sweep(const Level& v, const TV* dinv, const TB* b, const TV* xin, TO* xout,
                 cudaStream_t s) {
  if (v.sell_slices > 0) {
    const int nslots = v.sell_slices * 32;
    launch_pdl(k_sell_jacobi<TV, TB, TO>, grid_for(nslots), kBlock, s, nslots, v.sell_ptr,
               v.sell_perm, v.sell_col, Vals<TV>::S(v), dinv, b, xin, xout);
  } else if (v.ell_w > 0) {
    launch_pdl(k_jacobi_ell<TV, TB, TO>, grid_for(v.A.n), kBlock, s, v.A.n, v.ell_w, v.ell_col,
               v.ell_nx, v.ell_nxy, Vals<TV>::E(v), dinv, b, xin, xout);
  } else {
    jacobi<TV, TB, TO>(v.lanes_A, v.A, Vals<TV>::A(v), dinv, b, xin, xout, s);
  }
}

template <class TV, class TB>
void level_residual(const Level& v, const TB* b, const TV* x, TV* r, cudaStream_t s) {
  if (v.sell_slices > 0) {
    const int nslots = v.sell_slices * 32;
    launch_pdl(k_sell_residual<TV, TB>, grid_for(nslots), kBlock, s, nslots, v.sell_ptr,
               v.sell_perm, v.sell_col, Vals<TV>::S(v), b, x, r);
  } else if (v.ell_w > 0) {
    launch_pdl(k_residual_ell<TV, TB>, grid_for(v.A.n), kBlock, s, v.A.n, v.ell_w, v.ell_col,
               v.ell_nx, v.ell_nxy, Vals<TV>::E(v), b, x, r);
  } else {
    residual<TV, TB>(v.lanes_A, v.A, Vals<TV>::A(v), b, x, r, s);
  }
}

// y: work vector of the level (holds d b); first: the sweeps open a V-cycle
// (the first kernel waits before any read)
template <class TV, class TB>
void level_two_sweeps_from_zero(const Level& v, const TV* dinv, const TB* b, TV* y, TV* x,
                                int first, cudaStream_t s, bool y_ready = false) {
  if (!y_ready)
    launch_pdl(k_scale_db<TV, TB>, grid_for(v.A.n), kBlock, s, v.A.n, dinv, b, y, first);
  if (v.sell_slices > 0) {
    const int nslots = v.sell_slices * 32;
    launch_pdl(k_sell_jacobi2z<TV, TB>, grid_for(nslots), kBlock, s, nslots, v.sell_ptr,
               v.sell_perm, v.sell_col, Vals<TV>::S(v), dinv, b, (const TV*)y, x);
  } else if (v.ell_w > 0) {
    launch_pdl(k_jacobi2z_ell<TV, TB>, grid_for(v.A.n), kBlock, s, v.A.n, v.ell_w, v.ell_col,
               v.ell_nx, v.ell_nxy, Vals<TV>::E(v), dinv, b, (const TV*)y, x);
  } else {
    jacobi2z<TV, TB>(v.lanes_A, v.A, Vals<TV>::A(v), dinv, b, y, x, s);
  }
}

// algorithmic bytes of one sweep x_out = x_in + dinv (b - A x_in)
template <class TV, class TB, class TO>
double sweep_bytes(const Level& v) {
  const DevCSR& A = v.A;
  // an ELL copy by grid direction holds values only (7 per row, zeros at
  // the boundary included): its column indices are implicit
  const double amat = v.ell_nxy > 0 ? (double)A.n * v.ell_w * sizeof(TV)
                                    : (double)A.nnz * (sizeof(TV) + sizeof(int)) + 4.0 * (A.n + 1);
  return amat + (double)A.n * (2 * sizeof(TV) + sizeof(TB) + sizeof(TO));
}

template <class TV, class TB, class TO>
void sweep_probed(Probe* pr, const Level& v, const TV* dinv, const TB* b, const TV* xin,
                  TO* xout, cudaStream_t s) {
  if (pr) pr->before(s);
  level_sweep<TV, TB, TO>(v, dinv, b, xin, xout, s);
  if (pr) pr->after(s, sweep_bytes<TV, TB, TO>(v));
}

// smoother selection of one V-cycle: 0 l1-Jacobi, 1 Chebyshev of `degree`;
// tail_first >= 0: levels from tail_first down run as one cluster kernel;
// line_nz > 1: the finest level takes nu_line vertical-line steps instead
struct Smooth {
  int kind = 0, degree = 2;
  int tail_first = -1, tail_cluster = 0, nc = 0;
  const TailLevel* tail_desc = nullptr;
  int line_nxy = 0, line_nz = 0, nu_line = 1;
  int probe_level = 0;  // level whose smoothing sweeps the probe times
};

// algorithmic bytes of one line step: the level operator (ELL slots or CSR
// row pattern), the three factor arrays, b, x_in (when present) and x_out
template <class TV, class TB, class TO>
double line_bytes(const Level& v, bool from_zero) {
  const double n = v.A.n;
  double bytes = n * (3 * sizeof(TV) + sizeof(TB) + sizeof(TO));
  if (!from_zero) {
    bytes += n * sizeof(TV);
    if (v.ell_w > 0) bytes += n * v.ell_w * ((v.ell_nxy > 0 ? 0 : sizeof(int)) + sizeof(TV));
    else bytes += (double)v.A.nnz * (sizeof(int) + sizeof(TV)) + 4.0 * (n + 1);
  }
  return bytes;
}

template <class TV, class TB, class TO>
void line_step(const Smooth& sm, const Level& v, const TB* b, const TV* xin, TO* xout,
               cudaStream_t s) {
  // two threads per column; small blocks spread a few thousand columns over
  // every SM
  const long long lanes = 2ll * sm.line_nxy;
  const int threads = lanes >= 152 * 128 * 2 ? 128 : 32;
  const int grid = (int)((lanes + threads - 1) / threads);
  launch_pdl(k_line_sweep<TV, TB, TO>, grid, threads, s, sm.line_nxy, sm.line_nz, v.A.n,
             v.ell_w, v.ell_col, v.ell_nx, v.ell_nxy, Vals<TV>::E(v), v.A.rowptr, v.A.col,
             Vals<TV>::A(v),
             Vals<TV>::lo(v), Vals<TV>::minv(v), Vals<TV>::cp(v), b, xin, xout);
}

// one smoothing step xin -> xout (xin null: zero initial guess, Chebyshev only)
template <class TV, class TB, class TO>
void smooth_step(const Smooth& sm, Probe* pr, const Level& v, const TV* dinv, const TB* b,
                 const TV* xin, TO* xout, cudaStream_t s) {
  if (sm.kind == 1) {
    chebyshev_apply<TV, TB, TO>(v, Vals<TV>::A(v), dinv, sm.degree, b, xin, xout, s);
  } else {
    sweep_probed<TV, TB, TO>(pr, v, dinv, b, xin, xout, s);
  }
}

// bc = R r for level l + 1. When that level smooths with l1-Jacobi by the
// per-kernel path (not the coarsest, not the cluster tail) the restriction
// also writes its first sweep from zero, d b: into t for the fused two
// sweeps, into x for a single one. Returns whether it did.
template <class TV>
bool restrict_to(std::vector<Level>& L, size_t l, const Smooth& sm, int nu_pre, const TV* r,
                 TV* bc, cudaStream_t s) {
  Level& v = L[l];
  Level& c = L[l + 1];
  const bool fuse = sm.kind == 0 && l + 2 < L.size() && (int)(l + 1) != sm.tail_first;
  const TV* dsc = fuse ? Vals<TV>::dinv(c) : nullptr;
  TV* ysc = fuse ? static_cast<TV*>(nu_pre >= 2 ? c.t : c.x) : nullptr;
  if (v.Rh) spmv<__nv_bfloat16, TV>(v.lanes_R, v.R, v.Rh, r, bc, s, dsc, ysc);
  else spmv<TV, TV>(v.lanes_R, v.R, Vals<TV>::R(v), r, bc, s, dsc, ysc);
  return fuse;
}

template <class TV, class TB, class TO>
TV* run_level(std::vector<Level>& L, const double* cinv, size_t l, const TB* b, TO* final_out,
              int nu_pre, int nu_post, const Smooth& sm, cudaStream_t s,
              Probe* probe = nullptr, bool pre_done = false) {
  Level& v = L[l];
  const int n = v.A.n;
  TV* x = static_cast<TV*>(v.x);
  TV* t = static_cast<TV*>(v.t);
  if (l + 1 == L.size()) {
    if (final_out) {
      coarse<TB, TO>(n, cinv, b, final_out, s);
      return nullptr;
    }
    coarse<TB, TV>(n, cinv, b, x, s);
    return x;
  }
  if ((int)l == sm.tail_first && !final_out) {
    // the whole coarse tail in one cluster kernel; the result buffer follows
    // the same ping-pong of x and t as the per-kernel path below
    launch_vcycle_tail<TV>(sm.tail_desc, (int)l, (int)L.size() - 1, cinv, sm.nc, nu_pre, nu_post,
                           sm.tail_cluster, s);
    TV* cur = x;
    TV* oth = t;
    for (int k = (nu_pre >= 2 ? 2 : 1); k < nu_pre; ++k) std::swap(cur, oth);
    for (int k = 1; k <= nu_post; ++k) std::swap(cur, oth);
    return cur;
  }
  const TV* dinv = Vals<TV>::dinv(v);
  Probe* pr = ((int)l == sm.probe_level) ? probe : nullptr;
  TV* cur = x;
  TV* oth = t;
  if (l == 0 && sm.line_nz > 1 && v.line_minv) {
    // vertical-line smoothing of the finest level
    line_step<TV, TB, TV>(sm, v, b, (const TV*)nullptr, cur, s);
    for (int k = 1; k < sm.nu_line; ++k) {
      line_step<TV, TB, TV>(sm, v, b, cur, oth, s);
      std::swap(cur, oth);
    }
    TV* r = static_cast<TV*>(v.r);
    level_residual<TV, TB>(v, b, cur, r, s);
    Level& c = L[l + 1];
    TV* bc = static_cast<TV*>(c.b);
    const bool fuse = restrict_to<TV>(L, l, sm, nu_pre, r, bc, s);
    TV* ec = run_level<TV, TV, TV>(L, cinv, l + 1, bc, (TV*)nullptr, nu_pre, nu_post, sm, s,
                                   probe, fuse);
    if (v.Ph) prolong<__nv_bfloat16, TV>(v.lanes_P, v.P, v.Ph, ec, cur, s);
    else prolong<TV, TV>(v.lanes_P, v.P, Vals<TV>::P(v), ec, cur, s);
    double span_bytes = 0.0;
    if (pr) pr->before(s);
    for (int k = 1; k <= sm.nu_line; ++k) {
      if (k == sm.nu_line && final_out) {
        line_step<TV, TB, TO>(sm, v, b, cur, final_out, s);
        span_bytes += line_bytes<TV, TB, TO>(v, false);
        if (pr) pr->after(s, span_bytes, sm.nu_line);
        return nullptr;
      }
      line_step<TV, TB, TV>(sm, v, b, cur, oth, s);
      span_bytes += line_bytes<TV, TB, TV>(v, false);
      std::swap(cur, oth);
    }
    if (pr) pr->after(s, span_bytes, sm.nu_line);
    return cur;
  }
  int done = 1;
  if (sm.kind == 1) {
    // pre-smoothing from a zero guess
    smooth_step<TV, TB, TV>(sm, nullptr, v, dinv, b, (const TV*)nullptr, x, s);
  } else if (nu_pre >= 2) {
    // the first two l1-Jacobi sweeps from a zero guess fused (y = d b in t,
    // written by the restriction when pre_done)
    level_two_sweeps_from_zero<TV, TB>(v, dinv, b, t, x, l == 0 ? 1 : 0, s, pre_done);
    done = 2;
  } else if (!pre_done) {
    launch_pdl(k_jacobi0<TV, TB>, grid_for(n), kBlock, s, n, dinv, b, x, l == 0 ? 1 : 0);
  }
  for (int k = done; k < nu_pre; ++k) {
    smooth_step<TV, TB, TV>(sm, pr, v, dinv, b, cur, oth, s);
    std::swap(cur, oth);
  }
  // coarse-grid correction
  TV* r = static_cast<TV*>(v.r);
  level_residual<TV, TB>(v, b, cur, r, s);
  Level& c = L[l + 1];
  TV* bc = static_cast<TV*>(c.b);
  const bool fuse = restrict_to<TV>(L, l, sm, nu_pre, r, bc, s);
  TV* ec = run_level<TV, TV, TV>(L, cinv, l + 1, bc, (TV*)nullptr, nu_pre, nu_post, sm, s,
                                 probe, fuse);
  if (v.Ph) prolong<__nv_bfloat16, TV>(v.lanes_P, v.P, v.Ph, ec, cur, s);
  else prolong<TV, TV>(v.lanes_P, v.P, Vals<TV>::P(v), ec, cur, s);
  // post-smoothing; on the probed level one event pair spans all sweeps
  // (one pair per launch would put an event node between every two kernels)
  Probe* span = (pr && sm.kind == 0) ? pr : nullptr;
  double span_bytes = 0.0;
  if (span) span->before(s);
  for (int k = 1; k <= nu_post; ++k) {
    if (k == nu_post && final_out) {
      smooth_step<TV, TB, TO>(sm, nullptr, v, dinv, b, cur, final_out, s);
      span_bytes += sweep_bytes<TV, TB, TO>(v);
      if (span) span->after(s, span_bytes, nu_post);
      return nullptr;
    }
    smooth_step<TV, TB, TV>(sm, nullptr, v, dinv, b, cur, oth, s);
    span_bytes += sweep_bytes<TV, TB, TV>(v);
    std::swap(cur, oth);
  }
  if (span) span->after(s, span_bytes, nu_post);
  return cur;
}

}  // namespace

void Hierarchy::vcycle(cudaStream_t s) {
  if (opts.precision >= 1) vcycle_fp32(s);
  else vcycle_fp64(s);
}

void Hierarchy::vcycle_fp64(cudaStream_t s) {
  Smooth sm{opts.smoother, opts.cheb_degree, tail_first, tail_cluster, nc, tail_desc,
            opts.line_nxy, opts.line_nz, opts.nu_line, probe_level};
  run_level<double, double, double>(L, coarse_inv, 0, in, out, opts.nu_pre, opts.nu_post, sm, s,
                                    probe);
}

void Hierarchy::vcycle_fp32(cudaStream_t s) {
  Smooth sm{opts.smoother, opts.cheb_degree, tail_first, tail_cluster, nc, tail_desc,
            opts.line_nxy, opts.line_nz, opts.nu_line, probe_level};
  run_level<float, double, double>(L, coarse_inv, 0, in, out, opts.nu_pre, opts.nu_post, sm, s,
                                   probe);
}

// ------------------------------------------------- V-cycle byte count
// Algorithmic bytes of one V-cycle as run_level executes it: every matrix
// entry, index and vector element each kernel touches counted once per
// kernel (level operator, smoother scaling or line factors, right-hand side,
// input and output vectors; R and P with their row pointers; the coarsest
// inverse and its two vectors). Values and vectors in the hierarchy's
// precision; level 0 reads its right-hand side and writes its result in FP64.
double Hierarchy::vcycle_bytes() const {
  const bool f32 = opts.precision >= 1;
  const double sv = f32 ? 4.0 : 8.0;
  const double spr = opts.precision == 2 ? 2.0 : sv;  // P and R values
  double total = 0.0;
  const size_t nl = L.size();
  for (size_t l = 0; l < nl; ++l) {
    const Level& v = L[l];
    const double n = v.A.n;
    const double sb = (l == 0) ? 8.0 : sv;  // right-hand side
    if (l + 1 == nl) {
      total += n * n * 8.0 + n * sb + n * (l == 0 ? 8.0 : sv);
      break;
    }
    const double amat = v.ell_w > 0 ? n * v.ell_w * ((v.ell_nxy > 0 ? 0.0 : 4.0) + sv)
                                    : (double)v.A.nnz * (4.0 + sv) + 4.0 * (n + 1);
    const double sweep = amat + n * (sv /*dinv*/ + sb + sv /*x in*/ + sv /*x out*/);
    const double resid = amat + n * (sb + sv + sv);
    const double nc = L[l + 1].A.n;
    const double restr = (double)v.R.nnz * (4.0 + spr) + 4.0 * (nc + 1) + n * sv + nc * sv;
    const double prol = (double)v.P.nnz * (4.0 + spr) + 4.0 * (n + 1) + nc * sv + 2.0 * n * sv;
    double smooth = 0.0;
    if (l == 0 && opts.line_nz > 1 && v.line_minv) {
      const double fac = 3.0 * sv;
      const double zero = n * (fac + sb + sv);
      const double step = amat + n * (fac + sb + sv + sv);
      smooth = zero + (opts.nu_line - 1) * step + opts.nu_line * step;
    } else {
      const int pre = opts.nu_pre, post = opts.nu_post;
      const double deg = opts.smoother == 1 ? (double)opts.cheb_degree : 1.0;
      if (opts.smoother == 0 && pre >= 2) smooth += sweep + (pre - 2) * sweep;
      else smooth += deg * pre * sweep;
      smooth += deg * post * sweep;
    }
    total += smooth + resid + restr + prol;
  }
  return total;
}

// ------------------------------------------------------------------ probe
void Probe::create() {
  if (created) return;
  for (int q = 0; q < 2; ++q)
    for (int k = 0; k < 2 * kMaxPairs; ++k) TP_CUDA_TRY(cudaEventCreate(&ev[q][k]));
  created = true;
}

void Probe::destroy() {
  if (!created) return;
  for (int q = 0; q < 2; ++q)
    for (int k = 0; k < 2 * kMaxPairs; ++k) cudaEventDestroy(ev[q][k]);
  created = false;
}

void Probe::before(cudaStream_t s) {
  if (npairs >= kMaxPairs) return;
  cudaEvent_t e = ev[active][2 * npairs];
  if (g_capturing) TP_CUDA_TRY(cudaEventRecordWithFlags(e, s, cudaEventRecordExternal));
  else TP_CUDA_TRY(cudaEventRecord(e, s));
}

void Probe::after(cudaStream_t s, double algorithmic_bytes, int launches_in_span) {
  if (npairs >= kMaxPairs) return;
  cudaEvent_t e = ev[active][2 * npairs + 1];
  if (g_capturing) TP_CUDA_TRY(cudaEventRecordWithFlags(e, s, cudaEventRecordExternal));
  else TP_CUDA_TRY(cudaEventRecord(e, s));
  bytes[npairs] = algorithmic_bytes;
  nlaunch[npairs] = launches_in_span;
  ++npairs;
}

void Probe::read_and_accumulate(int set) {
  for (int k = 0; k < npairs; ++k) {
    float ms = 0.f;
    TP_CUDA_TRY(cudaEventElapsedTime(&ms, ev[set][2 * k], ev[set][2 * k + 1]));
    total_ms += ms;
    total_bytes += bytes[k];
    launches += nlaunch[k];
  }
}

}  // namespace tp

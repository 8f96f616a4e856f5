// Chebyshev polynomial smoother on D^{-1} A, D = diag(A), as the alternative
// to l1-Jacobi in the AMG V-cycle.
//
// Setup: lambda_max(D^{-1} A) by 10 power iterations from the seeded start
// vector x_i = h_i / 2^32 + 1/2 (h_i the splitmix64 tie-break hash of row i
// with seed + 1); the polynomial targets [lambda/30, 1.1 lambda]. Norms are
// summed over a fixed block partition, and lambda and the recurrence
// coefficients stay on the device, so setup needs no host round trip and
// the captured V-cycle reads them at replay.
//
// Apply (three-term recurrence, Saad, Iterative Methods for Sparse Linear
// Systems, Alg. 12.1): theta = (hi + lo)/2, delta = (hi - lo)/2, sigma =
// theta/delta, rho_0 = 1/sigma;
//   r = D^{-1}(b - A x), d = r / theta, x += d;
//   then per further degree k: r -= D^{-1} A d, rho_k = 1/(2 sigma - rho_{k-1}),
//   d = rho_k rho_{k-1} d + (2 rho_k / delta) r, x += d.
// One kernel per degree (each one SpMV), rows split over groups of LANES
// threads as in the other CSR kernels.
#include "amg.cuh"

namespace tp {

namespace {

constexpr int kPowerIters = 10;
constexpr int kNormParts = 256;   // fixed partition of the norm partial sums

template <int LANES, class T>
__device__ __forceinline__ T lane_sum(T v) {
#pragma unroll
  for (int o = LANES / 2; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o, LANES);
  return v;
}

template <int LANES, class TV, class TX>
__device__ __forceinline__ TV csr_row_dot(const int* __restrict__ rp, const int* __restrict__ col,
                                          const TV* __restrict__ val, const TX* __restrict__ x,
                                          int row, bool valid, int lane) {
  TV acc = TV(0);
  if (valid) {
    const int e1 = rp[row + 1];
    for (int e = rp[row] + lane; e < e1; e += LANES) acc += val[e] * (TV)x[col[e]];
  }
  return lane_sum<LANES>(acc);
}

// dinv_i = 1 / a_ii
__global__ void k_diag_inv(int n, const int* __restrict__ rp, const int* __restrict__ col,
                           const double* __restrict__ val, double* __restrict__ dinv,
                           float* __restrict__ dinvf, int* __restrict__ err) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  double d = 0.0;
  for (int e = rp[i]; e < rp[i + 1]; ++e)
    if (col[e] == i) d = val[e];
  if (d == 0.0 || !isfinite(d)) {
    atomicOr(err, 4);
    d = 1.0;
  }
  dinv[i] = 1.0 / d;
  if (dinvf) dinvf[i] = (float)(1.0 / d);
}

// power-iteration start vector x_i = h_i / 2^32 + 1/2
__global__ void k_power_start(int n, unsigned long long seed, double* __restrict__ x,
                              double* __restrict__ scal) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) x[i] = (double)pmis_hash(seed, i) / 4294967296.0 + 0.5;
  if (i == 0) scal[0] = 1.0;  // scale of x (1 / ||y_prev|| after the first step)
}

// y = D^{-1} A (s x), partial sums of |y|^2 and |s x|^2 over a fixed
// partition of the rows (one row per thread)
__global__ void __launch_bounds__(256) k_power_step(int n, const int* __restrict__ rp,
                                                    const int* __restrict__ col,
                                                    const double* __restrict__ val,
                                                    const double* __restrict__ dinv,
                                                    const double* __restrict__ x,
                                                    const double* __restrict__ scal,
                                                    double* __restrict__ y,
                                                    double* __restrict__ partials) {
  __shared__ double sy[8], sx[8];
  const double s = scal[0];
  const long long chunk = ((long long)n + gridDim.x - 1) / gridDim.x;
  const long long lo = chunk * blockIdx.x;
  long long hi = lo + chunk;
  if (hi > n) hi = n;
  double ay = 0.0, ax = 0.0;
  for (long long i = lo + threadIdx.x; i < hi; i += blockDim.x) {
    double acc = 0.0;
    for (int e = rp[i]; e < rp[i + 1]; ++e) acc += val[e] * (s * x[col[e]]);
    const double yi = dinv[i] * acc;
    y[i] = yi;
    const double xi = s * x[i];
    ay += yi * yi;
    ax += xi * xi;
  }
  ay = lane_sum<32>(ay);
  ax = lane_sum<32>(ax);
  if ((threadIdx.x & 31) == 0) {
    sy[threadIdx.x >> 5] = ay;
    sx[threadIdx.x >> 5] = ax;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double ty = 0.0, tx = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
      ty += sy[w];
      tx += sx[w];
    }
    partials[2 * blockIdx.x] = ty;
    partials[2 * blockIdx.x + 1] = tx;
  }
}

// lambda = ||y|| / ||s x||, next scale 1 / ||y||; on the last iteration the
// recurrence coefficients: coef[0] = 1/theta, coef[2k-1] = rho_k rho_{k-1},
// coef[2k] = 2 rho_k / delta for k = 1..degree-1
__global__ void k_power_finish(const double* __restrict__ partials, int B,
                               double* __restrict__ scal, double* __restrict__ lam, int last,
                               int degree, double* __restrict__ coef,
                               float* __restrict__ coeff, int* __restrict__ err) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  double ty = 0.0, tx = 0.0;
  for (int b = 0; b < B; ++b) {
    ty += partials[2 * b];
    tx += partials[2 * b + 1];
  }
  const double ny = sqrt(ty), nx = sqrt(tx);
  const double l = ny / nx;
  if (!(ny > 0.0) || !isfinite(l)) {
    atomicOr(err, 8);
    scal[0] = 1.0;
    lam[0] = 1.0;
  } else {
    scal[0] = 1.0 / ny;
    lam[0] = l;
  }
  if (!last) return;
  const double lo = lam[0] / 30.0, hi = 1.1 * lam[0];
  const double theta = 0.5 * (hi + lo), delta = 0.5 * (hi - lo);
  const double sigma = theta / delta;
  double rho = 1.0 / sigma;
  coef[0] = 1.0 / theta;
  for (int k = 1; k < degree; ++k) {
    const double rn = 1.0 / (2.0 * sigma - rho);
    coef[2 * k - 1] = rn * rho;
    coef[2 * k] = 2.0 * rn / delta;
    rho = rn;
  }
  for (int k = 0; k < 2 * degree - 1; ++k) coeff[k] = (float)coef[k];
}

template <class TV>
__device__ __forceinline__ const TV* pick_coef(const double* c, const float* cf);
template <>
__device__ __forceinline__ const double* pick_coef<double>(const double* c, const float*) {
  return c;
}
template <>
__device__ __forceinline__ const float* pick_coef<float>(const double*, const float* cf) {
  return cf;
}

// first degree: r = D^{-1}(b - A x) (x = 0 when xin is null), d = r / theta,
// x1 = x + d; with degree 1 x1 goes to xout, else x1, d, r are stored
template <int LANES, class TV, class TB, class TO>
__global__ void __launch_bounds__(256) k_cheb_first(
    int n, const int* __restrict__ rp, const int* __restrict__ col, const TV* __restrict__ val,
    const TV* __restrict__ dinv, const TB* __restrict__ b, const TV* __restrict__ xin,
    const double* __restrict__ coef, const float* __restrict__ coeff, int last,
    TO* __restrict__ xout, TV* __restrict__ xw, TV* __restrict__ dk, TV* __restrict__ r) {
  pdl_wait();
  pdl_trigger();
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  const int row = t / LANES, lane = t % LANES;
  const bool valid = row < n;
  TV ax = TV(0);
  if (xin) ax = csr_row_dot<LANES, TV, TV>(rp, col, val, xin, row, valid, lane);
  if (!valid || lane != 0) return;
  const TV* c = pick_coef<TV>(coef, coeff);
  const TV ri = dinv[row] * ((TV)b[row] - ax);
  const TV di = ri * c[0];
  const TV xi = (xin ? xin[row] : TV(0)) + di;
  if (last) {
    xout[row] = (TO)xi;
  } else {
    xw[row] = xi;
    dk[row] = di;
    r[row] = ri;
  }
}

// degree k >= 1: r -= D^{-1} A d, d' = a_k d + c_k r, x += d'
template <int LANES, class TV, class TO>
__global__ void __launch_bounds__(256) k_cheb_step(
    int n, const int* __restrict__ rp, const int* __restrict__ col, const TV* __restrict__ val,
    const TV* __restrict__ dinv, const TV* __restrict__ din, const double* __restrict__ coef,
    const float* __restrict__ coeff, int k, int last, TV* __restrict__ r, TV* __restrict__ xw,
    TV* __restrict__ dout, TO* __restrict__ xout) {
  pdl_wait();
  pdl_trigger();
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  const int row = t / LANES, lane = t % LANES;
  const bool valid = row < n;
  const TV ad = csr_row_dot<LANES, TV, TV>(rp, col, val, din, row, valid, lane);
  if (!valid || lane != 0) return;
  const TV* c = pick_coef<TV>(coef, coeff);
  const TV ri = r[row] - dinv[row] * ad;
  const TV di = c[2 * k - 1] * din[row] + c[2 * k] * ri;
  const TV xi = xw[row] + di;
  if (last) {
    xout[row] = (TO)xi;
  } else {
    r[row] = ri;
    dout[row] = di;
    xw[row] = xi;
  }
}

}  // namespace

// Plain-diagonal scaling and Chebyshev bounds/coefficients of one level
// (no host synchronisation).
void chebyshev_setup(Level& v, Pool& pool, int degree, unsigned long long seed,
                     double* partials, int* err, bool allocate, cudaStream_t s) {
  const int n = v.A.n;
  if (allocate) {
    v.cheb = pool.alloc<double>(2 * kMaxChebDegree + 2);
    v.chebf = pool.alloc<float>(2 * kMaxChebDegree);
    v.pw0 = pool.alloc<double>(n);
    v.pw1 = pool.alloc<double>(n);
  }
  k_diag_inv<<<grid_for(n), kBlock, 0, s>>>(n, v.A.rowptr, v.A.col, v.A.val, v.dinv, v.dinvf,
                                            err);
  TP_LAUNCH_CHECK();
  double* x = v.pw0;
  double* y = v.pw1;
  double* scal = v.cheb + 2 * kMaxChebDegree;
  double* lam = scal + 1;
  k_power_start<<<grid_for(n), kBlock, 0, s>>>(n, seed + 1, x, scal);
  TP_LAUNCH_CHECK();
  for (int it = 0; it < kPowerIters; ++it) {
    k_power_step<<<kNormParts, kBlock, 0, s>>>(n, v.A.rowptr, v.A.col, v.A.val, v.dinv, x, scal,
                                               y, partials);
    TP_LAUNCH_CHECK();
    k_power_finish<<<1, 32, 0, s>>>(partials, kNormParts, scal, lam, it == kPowerIters - 1,
                                    degree, v.cheb, v.chebf, err);
    TP_LAUNCH_CHECK();
    std::swap(x, y);
  }
}

int chebyshev_norm_parts() { return kNormParts; }

template <class TV, class TB, class TO>
void chebyshev_apply(const Level& v, const TV* val, const TV* dinv, int degree, const TB* b,
                     const TV* xin, TO* xout, cudaStream_t s) {
  const int lanes = v.lanes_A;
  const int g = grid_for((long long)v.A.n * lanes);
  TV* xw = static_cast<TV*>(v.cw);
  TV* d0 = static_cast<TV*>(v.cd0);
  TV* d1 = static_cast<TV*>(v.cd1);
  TV* r = static_cast<TV*>(v.cr);
  switch (lanes) {
#define TP_CASE(L)                                                                            \
  case L: {                                                                                   \
    launch_pdl(k_cheb_first<L, TV, TB, TO>, g, kBlock, s, v.A.n, v.A.rowptr, v.A.col, val,   \
               dinv, b, xin, (const double*)v.cheb, (const float*)v.chebf, degree == 1 ? 1 : 0, \
               xout, xw, d0, r);                                                              \
    for (int k = 1; k < degree; ++k) {                                                        \
      launch_pdl(k_cheb_step<L, TV, TO>, g, kBlock, s, v.A.n, v.A.rowptr, v.A.col, val, dinv, \
                 (const TV*)d0, (const double*)v.cheb, (const float*)v.chebf, k,              \
                 k == degree - 1 ? 1 : 0, r, xw, d1, xout);                                  \
      std::swap(d0, d1);                                                                      \
    }                                                                                         \
    break;                                                                                    \
  }
    TP_CASE(1) TP_CASE(2) TP_CASE(4) TP_CASE(8) TP_CASE(16) TP_CASE(32)
#undef TP_CASE
  }
  TP_LAUNCH_CHECK();
}

template void chebyshev_apply<double, double, double>(const Level&, const double*, const double*,
                                                      int, const double*, const double*, double*,
                                                      cudaStream_t);
template void chebyshev_apply<float, double, double>(const Level&, const float*, const float*, int,
                                                     const double*, const float*, double*,
                                                     cudaStream_t);
template void chebyshev_apply<float, double, float>(const Level&, const float*, const float*, int,
                                                    const double*, const float*, float*,
                                                    cudaStream_t);
template void chebyshev_apply<float, float, float>(const Level&, const float*, const float*, int,
                                                   const float*, const float*, float*,
                                                   cudaStream_t);

}  // namespace tp

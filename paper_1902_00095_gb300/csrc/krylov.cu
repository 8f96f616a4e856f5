// Block preconditioner (Sec. 3.2) and flexible GMRES (Sec. 4 solver
// settings: right preconditioning, restart 30).
//
// Krylov vectors are split [p (N) | T (N)]. The solve works on the
// equation-scaled system D A x = D b, D = diag(s_m I, s_e I) (the mass and
// energy rows differ by ~10 orders of magnitude in SI units); the block
// preconditioner of D A is M^{-1} D^{-1} because each V-cycle is linear and
// scale-homogeneous. Orthogonalisation is classical Gram-Schmidt with a
// re-orthogonalisation pass when the first pass cancelled most of w (the
// criterion of Daniel, Gragg, Kaufman and Stewart 1976: ||w'|| < ||w|| /
// sqrt(2), ||w||^2 = ||w'||^2 + sum h^2), decided on the device so the host
// never waits; all reductions use a fixed block partition and tree order, so
// results are deterministic.
#include <cmath>
#include <chrono>
#include "solver.cuh"

namespace tp {

namespace {

// vectors per multi-dot launch: 16 while the basis vectors are short (the
// launches dominate), 4 for long ones (fewer concurrent DRAM streams).
// FGMRES time measured on 262k / 2.1M / 8.4M unknowns: 16 vectors 34.0 /
// 49.0 / 4988 ms, 8 vectors 34.5 / 50.2 / 5583 ms, 4 vectors 34.8 / 48.3 /
// 4827 ms.
constexpr int kDotWide = 16, kDotNarrow = 4;
constexpr long long kDotWideMaxN = 1ll << 20;  // vector length up to which 16 are taken
constexpr int kEstSlot = 16;  // pinned-buffer offset of the two convergence-estimate slots

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  return v;
}

__device__ __forceinline__ void chunk_of(long long n, long long& lo, long long& hi) {
  long long chunk = (n + gridDim.x - 1) / gridDim.x;
  lo = chunk * blockIdx.x;
  hi = lo + chunk;
  if (hi > n) hi = n;
}

// block-level sum of one value per thread -> out (thread 0 writes)
__device__ __forceinline__ void block_sum_store(double v, double* out) {
  __shared__ double sh[32];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  v = warp_sum(v);
  if (lane == 0) sh[wid] = v;
  __syncthreads();
  if (wid == 0) {
    double t = (lane < (int)(blockDim.x >> 5)) ? sh[lane] : 0.0;
    t = warp_sum(t);
    if (lane == 0) *out = t;
  }
  __syncthreads();
}

// ------------------------------------------------------ preconditioner pieces
__global__ void k_precond_in(int N, const double* __restrict__ vp, const double* __restrict__ vT,
                             const double* __restrict__ scales, double* __restrict__ bp_s,
                             double* __restrict__ bT_s, double* __restrict__ hin) {
  pdl_wait();
  pdl_trigger();
  // 1 / s_m and 1 / s_e once per block: an FP64 instruction occupies the
  // GB300's FP64 pipe for the whole warp however few lanes run it, so a
  // division per element (or per warp) would bound the kernel
  __shared__ double rs[2];
  if (threadIdx.x == 0) {
    rs[0] = 1.0 / scales[0];
    rs[1] = 1.0 / scales[1];
  }
  __syncthreads();
  const double r0 = rs[0], r1 = rs[1];
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= N) return;
  const double a = vp[i] * r0;
  bp_s[i] = a;
  hin[i] = a;
  bT_s[i] = vT[i] * r1;
}

// out = b - A x over the shared 7-point pattern (steps 2 and 4 of Sec. 3.2)
__global__ void k_rhs_minus(int N, const int* __restrict__ rp, const int* __restrict__ col,
                            const double* __restrict__ val, const double* __restrict__ b,
                            const double* __restrict__ x, double* __restrict__ out) {
  pdl_wait();
  pdl_trigger();
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= N) return;
  const double bi = b[i];  // issued before the gathers
  double acc = 0.0;
  for (int e = rp[i]; e < rp[i + 1]; ++e) acc += val[e] * x[col[e]];
  out[i] = bi - acc;
}

// w = D A z (block-CSR, Eq. AXR); optionally stores z into Z_j.
__global__ void __launch_bounds__(256) k_block_spmv(int N, const int* __restrict__ rp,
                                                    const int* __restrict__ col,
                                                    const double4_32a* __restrict__ bval,
                                                    const double* __restrict__ zp,
                                                    const double* __restrict__ zT,
                                                    double* __restrict__ Zp,
                                                    double* __restrict__ ZT,
                                                    double* __restrict__ wp,
                                                    double* __restrict__ wT,
                                                    const double* __restrict__ scales) {
  // programmatic dependent launch: the row's pattern (the matrix does not
  // change during the solve) is loaded before the wait; its 2x2 blocks are
  // not (held in registers they cost occupancy on large grids)
  constexpr int kPre = 7;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  int e0 = 0, e1 = 0;
  int c[kPre];
  if (i < N) {
    e0 = rp[i];
    e1 = rp[i + 1];
  }
#pragma unroll
  for (int k = 0; k < kPre; ++k) c[k] = (e0 + k < e1) ? col[e0 + k] : 0;
  pdl_wait();
  pdl_trigger();
  if (i >= N) return;
  const double zpi = zp[i], zTi = zT[i];  // issued before the gathers
  double ap = 0.0, aT = 0.0;
#pragma unroll
  for (int k = 0; k < kPre; ++k) {
    if (e0 + k < e1) {
      const double4_32a b = bval[e0 + k];
      const double xp = zp[c[k]], xT = zT[c[k]];
      // two chained FMAs per component: 4 FP64 instructions per block (a
      // sum of two products added to the accumulator would take 6)
      ap = fma(b.y, xT, fma(b.x, xp, ap));
      aT = fma(b.w, xT, fma(b.z, xp, aT));
    }
  }
  for (int e = e0 + kPre; e < e1; ++e) {
    const int j = col[e];
    const double4_32a b = bval[e];
    const double xp = zp[j], xT = zT[j];
    ap = fma(b.y, xT, fma(b.x, xp, ap));
    aT = fma(b.w, xT, fma(b.z, xp, aT));
  }
  if (Zp) {
    Zp[i] = zpi;
    ZT[i] = zTi;
  }
  const double s0 = scales ? scales[0] : 1.0, s1 = scales ? scales[1] : 1.0;
  wp[i] = s0 * ap;
  wT[i] = s1 * aT;
}

// ------------------------------------------------------------ Gram-Schmidt
// partial dot products V_k . w, k0 <= k < k0 + nv (nv <= NV), of this
// block's element chunk: per-thread sums, then warp sums, then the block's
// warps in order (one barrier)
template <int NV>
__global__ void __launch_bounds__(256) k_mdot(long long n2, const double* __restrict__ V,
                                              long long stride, int k0, int nv,
                                              const double* __restrict__ w,
                                              double* __restrict__ partials,
                                              const int* __restrict__ gate) {
  __shared__ double sh[8][NV];
  pdl_wait();
  pdl_trigger();
  if (gate && *gate == 0) return;  // re-orthogonalisation not needed
  long long lo, hi;
  chunk_of(n2, lo, hi);
  double acc[NV];
#pragma unroll
  for (int q = 0; q < NV; ++q) acc[q] = 0.0;
  for (long long i = lo + threadIdx.x; i < hi; i += blockDim.x) {
    const double wi = w[i];
#pragma unroll
    for (int q = 0; q < NV; ++q)
      if (q < nv) acc[q] += wi * V[(long long)(k0 + q) * stride + i];
  }
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
  for (int q = 0; q < NV; ++q) {
    if (q < nv) {
      const double t = warp_sum(acc[q]);
      if (lane == 0) sh[wid][q] = t;
    }
  }
  __syncthreads();
  if (threadIdx.x < nv) {
    double t = 0.0;
    for (int u = 0; u < (int)(blockDim.x >> 5); ++u) t += sh[u][threadIdx.x];
    partials[(long long)(k0 + threadIdx.x) * gridDim.x + blockIdx.x] = t;
  }
}

// out[k] = sum_b partials[k * B + b], k < count (fixed order); 0 when gated off
__global__ void k_reduce_rows(int count, int B, const double* __restrict__ partials,
                              double* __restrict__ out, const int* __restrict__ gate) {
  pdl_wait();
  pdl_trigger();
  const int k = blockIdx.x;
  if (k >= count) return;
  if (gate && *gate == 0) {
    if (threadIdx.x == 0) out[k] = 0.0;
    return;
  }
  double v = 0.0;
  for (int b = threadIdx.x; b < B; b += blockDim.x) v += partials[(long long)k * B + b];
  block_sum_store(v, &out[k]);
}

// w -= sum_k h_k V_k; optionally per-block partial sums of w^2. Grid-stride
// over elements (fixed grid, so the partition of the partial sums is fixed);
// the k loop is unrolled by 8 so every thread keeps 8 independent loads of
// V in flight.
__global__ void __launch_bounds__(256) k_orth_update(long long n2, const double* __restrict__ V,
                                                     long long stride, int count,
                                                     const double* __restrict__ h,
                                                     double* __restrict__ w,
                                                     double* __restrict__ norm_partials,
                                                     const int* __restrict__ gate) {
  pdl_wait();
  pdl_trigger();
  if (gate && *gate == 0) return;  // w and the first pass's norm partials stand
  const long long step = (long long)gridDim.x * blockDim.x;
  double nrm = 0.0;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n2; i += step) {
    double a = w[i];
    int k = 0;
    for (; k + 8 <= count; k += 8) {
      double v[8];
#pragma unroll
      for (int q = 0; q < 8; ++q) v[q] = V[(long long)(k + q) * stride + i];
#pragma unroll
      for (int q = 0; q < 8; ++q) a -= h[k + q] * v[q];
    }
    for (; k < count; ++k) a -= h[k] * V[(long long)k * stride + i];
    w[i] = a;
    nrm += a * a;
  }
  if (norm_partials) block_sum_store(nrm, &norm_partials[blockIdx.x]);
}

// Arnoldi column j: H(:, j) = h1 + h2, H(j+1, j) = ||w|| (the block sums the
// B norm partials in a fixed tree order), Givens update by thread 0.
__global__ void __launch_bounds__(256) k_arnoldi(int j, int ldh, double* __restrict__ H,
                                                 double* __restrict__ cs,
                                                 double* __restrict__ sn,
                                                 double* __restrict__ g,
                                                 const double* __restrict__ h1,
                                                 const double* __restrict__ h2,
                                                 const double* __restrict__ npart, int B,
                                                 double* __restrict__ hn_out,
                                                 double* __restrict__ est) {
  __shared__ double tot;
  pdl_wait();
  pdl_trigger();
  double part = 0.0;
  for (int b = threadIdx.x; b < B; b += blockDim.x) part += npart[b];
  block_sum_store(part, &tot);
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  double* Hj = H + (long long)j * ldh;
  for (int k = 0; k <= j; ++k) Hj[k] = h1[k] + h2[k];
  const double hn = sqrt(tot);
  Hj[j + 1] = hn;
  for (int k = 0; k < j; ++k) {
    const double t = cs[k] * Hj[k] + sn[k] * Hj[k + 1];
    Hj[k + 1] = -sn[k] * Hj[k] + cs[k] * Hj[k + 1];
    Hj[k] = t;
  }
  const double den = hypot(Hj[j], Hj[j + 1]);
  if (den > 0.0) {
    cs[j] = Hj[j] / den;
    sn[j] = Hj[j + 1] / den;
  } else {
    cs[j] = 1.0;
    sn[j] = 0.0;
  }
  Hj[j] = den;
  Hj[j + 1] = 0.0;
  g[j + 1] = -sn[j] * g[j];
  g[j] = cs[j] * g[j];
  hn_out[0] = hn;
  hn_out[1] = 1.0 / hn;  // for k_normalize: one division here, not one per element
  est[0] = fabs(g[j + 1]);
  est[1] = hn;
  est[2] = den;
}

// re-orthogonalise iff ||w'||^2 < (||w'||^2 + sum_k h_k^2) / 2 after the
// first pass (fixed-order sums)
__global__ void __launch_bounds__(256) k_reorth_gate(int count, const double* __restrict__ h,
                                                     const double* __restrict__ npart, int B,
                                                     int* __restrict__ gate) {
  __shared__ double tot;
  pdl_wait();
  pdl_trigger();
  double part = 0.0;
  for (int b = threadIdx.x; b < B; b += blockDim.x) part += npart[b];
  block_sum_store(part, &tot);
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  double hh = 0.0;
  for (int k = 0; k < count; ++k) hh += h[k] * h[k];
  *gate = (2.0 * tot < tot + hh || !(tot == tot)) ? 1 : 0;
}

// v = w / h_{j+1,j} as w * (1 / h_{j+1,j}) (hn[1], written by k_arnoldi): an
// FP64 division per element would keep the GB300's FP64 pipe busy for
// longer than the vector takes to stream
__global__ void k_normalize(long long n2, const double* __restrict__ w,
                            const double* __restrict__ hn, double* __restrict__ v) {
  pdl_wait();
  pdl_trigger();
  long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i < n2) v[i] = w[i] * hn[1];
}

// first basis vector and Givens right-hand side: v0 = r / beta (as r times
// beta[1] = 1 / beta, from k_sqrt_inplace), g = beta e1
__global__ void k_start_cycle(long long n2, const double* __restrict__ r,
                              const double* __restrict__ beta, double* __restrict__ v0,
                              double* __restrict__ g, int restart) {
  long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i < n2) v0[i] = r[i] * beta[1];
  if (i <= restart) g[i] = (i == 0) ? beta[0] : 0.0;
}

// y = H(0:m, 0:m)^{-1} g (upper triangular back substitution)
__global__ void k_hsolve(int m, int ldh, const double* __restrict__ H,
                         const double* __restrict__ g, double* __restrict__ y) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  for (int i = m - 1; i >= 0; --i) {
    double s = g[i];
    for (int k = i + 1; k < m; ++k) s -= H[(long long)k * ldh + i] * y[k];
    y[i] = s / H[(long long)i * ldh + i];
  }
}

// x += sum_k y_k Z_k
__global__ void k_update_x(long long n2, const double* __restrict__ Z, long long stride, int m,
                           const double* __restrict__ y, double* __restrict__ x) {
  long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i >= n2) return;
  double a = x[i];
  for (int k = 0; k < m; ++k) a += y[k] * Z[(long long)k * stride + i];
  x[i] = a;
}

// bs = D b and partial ||bs||^2
__global__ void __launch_bounds__(256) k_scale_rhs(int N, const double* __restrict__ bp,
                                                   const double* __restrict__ bT,
                                                   const double* __restrict__ scales,
                                                   double* __restrict__ bs,
                                                   double* __restrict__ partials) {
  long long lo, hi;
  chunk_of(2ll * N, lo, hi);
  double s = 0.0;
  for (long long i = lo + threadIdx.x; i < hi; i += blockDim.x) {
    double v = (i < N) ? scales[0] * bp[i] : scales[1] * bT[i - N];
    bs[i] = v;
    s += v * v;
  }
  block_sum_store(s, &partials[blockIdx.x]);
}

// r = bs - D A x and partial ||r||^2 (row-parallel over the 2N rows)
__global__ void __launch_bounds__(256) k_true_residual(int N, const int* __restrict__ rp,
                                                       const int* __restrict__ col,
                                                       const double4_32a* __restrict__ bval,
                                                       const double* __restrict__ x,
                                                       const double* __restrict__ bs,
                                                       const double* __restrict__ scales,
                                                       double* __restrict__ r,
                                                       double* __restrict__ partials) {
  long long lo, hi;
  chunk_of(N, lo, hi);
  double s = 0.0;
  for (long long i = lo + threadIdx.x; i < hi; i += blockDim.x) {
    double ap = 0.0, aT = 0.0;
    for (int e = rp[i]; e < rp[i + 1]; ++e) {
      const int j = col[e];
      const double4_32a b = bval[e];
      const double xp = x[j], xT = x[N + j];
      ap = fma(b.y, xT, fma(b.x, xp, ap));
      aT = fma(b.w, xT, fma(b.z, xp, aT));
    }
    const double rp_ = bs[i] - scales[0] * ap, rT_ = bs[N + i] - scales[1] * aT;
    r[i] = rp_;
    r[N + i] = rT_;
    s += rp_ * rp_ + rT_ * rT_;
  }
  block_sum_store(s, &partials[blockIdx.x]);
}

// unscaled per-block residual sums: ||r_p||^2, ||r_T||^2, ||b_p||^2, ||b_T||^2
__global__ void __launch_bounds__(256) k_unscaled_sums(int N, const int* __restrict__ rp,
                                                       const int* __restrict__ col,
                                                       const double4_32a* __restrict__ bval,
                                                       const double* __restrict__ x,
                                                       const double* __restrict__ bp,
                                                       const double* __restrict__ bT,
                                                       double* __restrict__ partials) {
  long long lo, hi;
  chunk_of(N, lo, hi);
  double s[4] = {0.0, 0.0, 0.0, 0.0};
  for (long long i = lo + threadIdx.x; i < hi; i += blockDim.x) {
    double ap = 0.0, aT = 0.0;
    for (int e = rp[i]; e < rp[i + 1]; ++e) {
      const int j = col[e];
      const double4_32a b = bval[e];
      const double xp = x[j], xT = x[N + j];
      ap = fma(b.y, xT, fma(b.x, xp, ap));
      aT = fma(b.w, xT, fma(b.z, xp, aT));
    }
    const double a = bp[i] - ap, c = bT[i] - aT;
    s[0] += a * a;
    s[1] += c * c;
    s[2] += bp[i] * bp[i];
    s[3] += bT[i] * bT[i];
  }
  for (int q = 0; q < 4; ++q) block_sum_store(s[q], &partials[(long long)q * gridDim.x + blockIdx.x]);
}

__global__ void k_sum_to(const double* __restrict__ partials, int B, double* __restrict__ out) {
  double v = 0.0;
  for (int b = threadIdx.x; b < B; b += blockDim.x) v += partials[b];
  block_sum_store(v, out);
}

// v[0] = sqrt(v[0]), v[1] = 1 / v[0] (for k_start_cycle)
__global__ void k_sqrt_inplace(double* v) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    v[0] = sqrt(v[0]);
    v[1] = 1.0 / v[0];
  }
}

void mdot_all(long long n2, const double* V, long long stride, int count, const double* w,
              double* partials, int B, double* out, cudaStream_t s,
              const int* gate = nullptr) {
  const int nvmax = n2 <= kDotWideMaxN ? kDotWide : kDotNarrow;
  for (int k0 = 0; k0 < count; k0 += nvmax) {
    const int nv = count - k0 < nvmax ? count - k0 : nvmax;
    if (nvmax == kDotWide)
      launch_pdl(k_mdot<kDotWide>, B, 256, s, n2, V, stride, k0, nv, w, partials, gate);
    else
      launch_pdl(k_mdot<kDotNarrow>, B, 256, s, n2, V, stride, k0, nv, w, partials, gate);
  }
  launch_pdl(k_reduce_rows, count, 256, s, count, B, partials, out, gate);
}

// grid of the multi-dots of the FGMRES basis: 8 blocks per SM (the
// partition of their partial sums; with 2 per SM, the context's partition,
// the 8.4 M-element dots left most of each SM idle: layered 256x256x64
// FGMRES 144.4 ms with 2, 142.9 with 4, 140.5 with 8, 141.1 with 16)
int mdot_grid(const tp_ctx* c, long long n) {
  const long long want = (n + 255) / 256;
  const long long cap = 8ll * c->num_sms;
  return (int)std::max(1ll, std::min(want, cap));
}

// grid of k_orth_update: enough blocks for 8 resident per SM, at most one
// element per thread
int orth_grid(const tp_ctx* c, long long n) {
  const long long want = (n + 255) / 256;
  const long long cap = 8ll * c->num_sms;
  return (int)std::max(1ll, std::min(want, cap));
}

double read_double(const double* d, double* host_pinned, cudaStream_t s) {
  TP_CUDA_TRY(cudaMemcpyAsync(host_pinned, d, sizeof(double), cudaMemcpyDeviceToHost, s));
  TP_CUDA_TRY(cudaStreamSynchronize(s));
  return *host_pinned;
}

void ensure_workspace(tp_ctx* c, int restart) {
  if (c->restart_alloc >= restart && c->Vb) return;
  c->kpool.release();
  const long long n2 = 2ll * c->N;
  c->Vb = c->kpool.alloc<double>((size_t)(restart + 1) * n2);
  c->Zb = c->kpool.alloc<double>((size_t)restart * n2);
  c->w = c->kpool.alloc<double>(n2);
  c->xs = c->kpool.alloc<double>(n2);
  c->bs = c->kpool.alloc<double>(n2);
  const int ldh = restart + 1;
  c->H = c->kpool.alloc<double>((size_t)ldh * (restart + 1));
  c->cs = c->kpool.alloc<double>(restart + 1);
  c->sn = c->kpool.alloc<double>(restart + 1);
  c->g = c->kpool.alloc<double>(restart + 2);
  c->yv = c->kpool.alloc<double>(restart + 1);
  c->hn = c->kpool.alloc<double>(4);
  c->est = c->kpool.alloc<double>(4);
  c->h2 = c->kpool.alloc<double>(2 * (restart + 2));
  c->kparts = c->kpool.alloc<double>(
      (size_t)(restart + 2) * std::max(4 * c->nparts, mdot_grid(c, 2ll * c->N)) + 16);
  c->oparts = c->kpool.alloc<double>((size_t)orth_grid(c, 2ll * c->N) + 16);
  c->reorth = c->kpool.alloc<int>(4);
  c->restart_alloc = restart;
}

// y = A x (scalar CSR, one thread per row)
__global__ void k_csr_spmv(int n, const int* __restrict__ rp, const int* __restrict__ col,
                           const double* __restrict__ val, const double* __restrict__ x,
                           double* __restrict__ y) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  double a = 0.0;
  for (int e = rp[i]; e < rp[i + 1]; ++e) a += val[e] * x[col[e]];
  y[i] = a;
}

// r = b - A x with partial ||r||^2 over a fixed block partition
__global__ void __launch_bounds__(256) k_csr_residual(int n, const int* __restrict__ rp,
                                                      const int* __restrict__ col,
                                                      const double* __restrict__ val,
                                                      const double* __restrict__ x,
                                                      const double* __restrict__ b,
                                                      double* __restrict__ r,
                                                      double* __restrict__ partials) {
  long long lo, hi;
  chunk_of(n, lo, hi);
  double s = 0.0;
  for (long long i = lo + threadIdx.x; i < hi; i += blockDim.x) {
    double a = 0.0;
    for (int e = rp[i]; e < rp[i + 1]; ++e) a += val[e] * x[col[e]];
    const double v = b[i] - a;
    r[i] = v;
    s += v * v;
  }
  block_sum_store(s, &partials[blockIdx.x]);
}

// column j of A_pT as a dense vector (rows of column j = rows of row j's
// pattern, the pattern being symmetric)
__global__ void k_column_rhs(int n, const int* __restrict__ rp, const int* __restrict__ col,
                             const double* __restrict__ ApT, int j, double* __restrict__ rhs) {
  long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i < n) rhs[i] = 0.0;
}

__global__ void k_column_fill(const int* __restrict__ rp, const int* __restrict__ col,
                              const double* __restrict__ ApT, int j, double* __restrict__ rhs) {
  const int q = threadIdx.x;
  const int e_j = rp[j] + q;
  if (e_j >= rp[j + 1]) return;
  const int i = col[e_j];
  for (int e = rp[i]; e < rp[i + 1]; ++e)
    if (col[e] == j) rhs[i] = ApT[e];
}

// S_ij = A_TT[i][j] - (A_Tp z)_i for the rows i of column j; writes the
// pattern entry index of (i, j) and the value
__global__ void k_column_schur(const int* __restrict__ rp, const int* __restrict__ col,
                               const double* __restrict__ ATp, const double* __restrict__ ATT,
                               int j, const double* __restrict__ z, int* __restrict__ entry,
                               double* __restrict__ value) {
  const int q = threadIdx.x;
  if (q >= 7) return;
  const int e_j = rp[j] + q;
  if (e_j >= rp[j + 1]) {
    entry[q] = -1;
    value[q] = 0.0;
    return;
  }
  const int i = col[e_j];
  double a = 0.0;
  int eij = -1;
  for (int e = rp[i]; e < rp[i + 1]; ++e) {
    a += ATp[e] * z[col[e]];
    if (col[e] == j) eij = e;
  }
  entry[q] = eij;
  value[q] = ATT[eij] - a;
}

}  // namespace

// FGMRES(restart) on a scalar CSR system A x = b, right-preconditioned by
// one V-cycle of h, x0 = 0, stop at ||b - A x|| <= rtol ||b||. Uses the
// context's Krylov workspace. Returns the iteration count (negative when
// rtol was not reached within maxit).
int scalar_fgmres(tp_ctx* c, Hierarchy& h, const DevCSR& A, const double* b, double* x,
                  double rtol, int maxit, int restart) {
  cudaStream_t s = c->s;
  ensure_workspace(c, restart);
  const int n = A.n;
  const int B = c->nparts;
  const int ldh = restart + 1;
  double* hp_host = c->host_est;
  double* r = c->w;
  TP_CUDA_TRY(cudaMemsetAsync(x, 0, sizeof(double) * n, s));
  k_csr_residual<<<B, 256, 0, s>>>(n, A.rowptr, A.col, A.val, x, b, r, c->kparts);
  TP_LAUNCH_CHECK();
  k_sum_to<<<1, 256, 0, s>>>(c->kparts, B, c->hn + 2);
  TP_LAUNCH_CHECK();
  const double bnorm = std::sqrt(read_double(c->hn + 2, hp_host, s));
  if (bnorm == 0.0) return 0;
  int its = 0;
  double beta = bnorm;
  TP_CUDA_TRY(cudaMemcpyAsync(c->hn, c->hn + 2, sizeof(double), cudaMemcpyDeviceToDevice, s));
  k_sqrt_inplace<<<1, 32, 0, s>>>(c->hn);
  TP_LAUNCH_CHECK();
  while (true) {
    if (beta <= rtol * bnorm) return its;
    if (its >= maxit) return -its;
    k_start_cycle<<<grid_for(n), kBlock, 0, s>>>(n, r, c->hn, c->Vb, c->g, restart);
    TP_LAUNCH_CHECK();
    int m = 0;
    for (int j = 0; j < restart; ++j) {
      double* vj = c->Vb + (long long)j * n;
      double* zj = c->Zb + (long long)j * n;
      TP_CUDA_TRY(cudaMemcpyAsync(h.in, vj, sizeof(double) * n, cudaMemcpyDeviceToDevice, s));
      h.vcycle(s);
      TP_CUDA_TRY(cudaMemcpyAsync(zj, h.out, sizeof(double) * n, cudaMemcpyDeviceToDevice, s));
      k_csr_spmv<<<grid_for(n), kBlock, 0, s>>>(n, A.rowptr, A.col, A.val, zj, c->w);
      TP_LAUNCH_CHECK();
      double* h1 = c->h2;
      double* h2 = c->h2 + (restart + 2);
      const int G = orth_grid(c, n);
      mdot_all(n, c->Vb, n, j + 1, c->w, c->kparts, B, h1, s);
      k_orth_update<<<G, 256, 0, s>>>(n, c->Vb, n, j + 1, h1, c->w, nullptr, nullptr);
      TP_LAUNCH_CHECK();
      mdot_all(n, c->Vb, n, j + 1, c->w, c->kparts, B, h2, s);
      k_orth_update<<<G, 256, 0, s>>>(n, c->Vb, n, j + 1, h2, c->w, c->oparts, nullptr);
      TP_LAUNCH_CHECK();
      k_arnoldi<<<1, 256, 0, s>>>(j, ldh, c->H, c->cs, c->sn, c->g, h1, h2, c->oparts, G, c->hn,
                                  c->est);
      TP_LAUNCH_CHECK();
      TP_CUDA_TRY(cudaMemcpyAsync(hp_host, c->est, 3 * sizeof(double), cudaMemcpyDeviceToHost, s));
      TP_CUDA_TRY(cudaStreamSynchronize(s));
      ++its;
      m = j + 1;
      if (!std::isfinite(hp_host[0]) || !(hp_host[2] > 0.0)) {
        m = j;
        break;
      }
      if (hp_host[0] <= rtol * bnorm || its >= maxit || hp_host[1] == 0.0) break;
      k_normalize<<<grid_for(n), kBlock, 0, s>>>(n, c->w, c->hn, c->Vb + (long long)(j + 1) * n);
      TP_LAUNCH_CHECK();
    }
    if (m > 0) {
      k_hsolve<<<1, 32, 0, s>>>(m, ldh, c->H, c->g, c->yv);
      TP_LAUNCH_CHECK();
      k_update_x<<<grid_for(n), kBlock, 0, s>>>(n, c->Zb, n, m, c->yv, x);
      TP_LAUNCH_CHECK();
    } else {
      return -its;
    }
    k_csr_residual<<<B, 256, 0, s>>>(n, A.rowptr, A.col, A.val, x, b, r, c->kparts);
    TP_LAUNCH_CHECK();
    k_sum_to<<<1, 256, 0, s>>>(c->kparts, B, c->hn);
    TP_LAUNCH_CHECK();
    k_sqrt_inplace<<<1, 32, 0, s>>>(c->hn);
    TP_LAUNCH_CHECK();
    beta = read_double(c->hn, hp_host, s);
    if (!std::isfinite(beta)) return -its;
  }
}

// Exact Schur complement column j restricted to the pattern (Eq. Afact):
// z = A_pp^{-1} A_pT e_j by scalar FGMRES, then S_ij = A_TT e_j - A_Tp z.
int probe_schur_column(tp_ctx* c, int j, double rtol, int maxit, int* entry, double* value) {
  cudaStream_t s = c->s;
  const int N = c->N;
  double* rhs = c->io0;
  double* z = c->io1;
  k_column_rhs<<<grid_for(N), kBlock, 0, s>>>(N, c->rowptr, c->col, c->ApT, j, rhs);
  TP_LAUNCH_CHECK();
  k_column_fill<<<1, 32, 0, s>>>(c->rowptr, c->col, c->ApT, j, rhs);
  TP_LAUNCH_CHECK();
  DevCSR A{N, N, c->nnzb, c->rowptr, c->col, c->App, nullptr};
  int its = scalar_fgmres(c, *c->hpp, A, rhs, z, rtol, maxit, 30);
  k_column_schur<<<1, 32, 0, s>>>(c->rowptr, c->col, c->ATp, c->ATT, j, z, entry, value);
  TP_LAUNCH_CHECK();
  return its;
}

void launch_block_spmv(int N, const int* rowptr, const int* col, const double* bval,
                       const double* xp, const double* xT, double* yp, double* yT,
                       const double* scales, cudaStream_t s) {
  k_block_spmv<<<grid_for(N), kBlock, 0, s>>>(N, rowptr, col,
                                              reinterpret_cast<const double4_32a*>(bval), xp, xT,
                                              nullptr, nullptr, yp, yT, scales);
  TP_LAUNCH_CHECK();
}

void precond_record(tp_ctx* c, cudaStream_t s) {
  c->probe.npairs = 0;
  Hierarchy& hp = *c->hpp;
  Hierarchy& hs = *c->hS;
  const int N = c->N;
  hp.vcycle(s);  // step 1: x_p = V_pp(b_p)
  launch_pdl(k_rhs_minus, grid_for(N), kBlock, s, N, c->rowptr, c->col, c->ATp, c->bT_s, hp.out,
             hs.in);  // step 2
  hs.vcycle(s);  // step 3: d_T = V_S(bt_T)
  if (c->opts.variant == 0) {
    launch_pdl(k_rhs_minus, grid_for(N), kBlock, s, N, c->rowptr, c->col, c->ApT, c->bp_s,
               hs.out, hp.in);  // step 4
    hp.vcycle(s);  // step 5: d_p = V_pp(bt_p)
  }
}

void precond_apply(tp_ctx* c, const double* vp, const double* vT, const double* scales,
                   cudaStream_t s, int set) {
  const int N = c->N;
  launch_pdl(k_precond_in, grid_for(N), kBlock, s, N, vp, vT, scales, c->bp_s, c->bT_s,
             c->hpp->in);
  if (c->pc_graph) {
    // point the graph's probe event nodes at this iteration's event set
    if (!c->probe_nodes.empty() && c->probe_set != set) {
      for (const auto& pn : c->probe_nodes)
        TP_CUDA_TRY(cudaGraphExecEventRecordNodeSetEvent(c->pc_graph, pn.first,
                                                         c->probe.ev[set][pn.second]));
      c->probe_set = set;
    }
    TP_CUDA_TRY(cudaGraphLaunch(c->pc_graph, s));
    count_launch(c->pc_graph_kernels);
  } else {
    c->probe.active = set;
    precond_record(c, s);
    c->probe.active = 0;
  }
}

int fgmres_solve(tp_ctx* c, const double* bp, const double* bT, double* xp, double* xT,
                 double rtol, int maxit, int restart, tp_solve_info* info) {
  cudaStream_t s = c->s;
  ensure_workspace(c, restart);
  const int N = c->N;
  const long long n2 = 2ll * N;
  const int B = c->nparts;
  const int Bm = mdot_grid(c, 2ll * c->N);
  const int ldh = restart + 1;
  double* hp_host = c->host_est;
  auto t0 = std::chrono::steady_clock::now();

  k_scale_rhs<<<B, 256, 0, s>>>(N, bp, bT, c->scales, c->bs, c->kparts);
  TP_LAUNCH_CHECK();
  k_sum_to<<<1, 256, 0, s>>>(c->kparts, B, c->hn + 2);
  TP_LAUNCH_CHECK();
  const double bnorm = std::sqrt(read_double(c->hn + 2, hp_host, s));
  TP_CUDA_TRY(cudaMemsetAsync(c->xs, 0, sizeof(double) * n2, s));
  int its = 0, restarts = 0, status = TP_NOT_CONVERGED;
  double beta = bnorm;
  bool breakdown = false;
  if (!std::isfinite(bnorm)) fail(TP_ENONFINITE, "right-hand side is not finite");
  if (bnorm == 0.0) {
    status = TP_OK;
  } else {
    bool first = true;
    double* r = c->w;  // residual shares the w buffer at cycle start
    while (true) {
      if (first) {
        TP_CUDA_TRY(cudaMemcpyAsync(r, c->bs, sizeof(double) * n2, cudaMemcpyDeviceToDevice, s));
        TP_CUDA_TRY(cudaMemcpyAsync(c->hn, c->hn + 2, sizeof(double), cudaMemcpyDeviceToDevice, s));
        k_sqrt_inplace<<<1, 32, 0, s>>>(c->hn);
        TP_LAUNCH_CHECK();
        first = false;
      } else {
        k_true_residual<<<B, 256, 0, s>>>(N, c->rowptr, c->col,
                                          reinterpret_cast<const double4_32a*>(c->bval), c->xs,
                                          c->bs, c->scales, r, c->kparts);
        TP_LAUNCH_CHECK();
        k_sum_to<<<1, 256, 0, s>>>(c->kparts, B, c->hn);
        TP_LAUNCH_CHECK();
        k_sqrt_inplace<<<1, 32, 0, s>>>(c->hn);
        TP_LAUNCH_CHECK();
        beta = read_double(c->hn, hp_host, s);
      }
      if (!std::isfinite(beta)) {
        breakdown = true;
        break;
      }
      if (beta <= rtol * bnorm) {
        status = TP_OK;
        break;
      }
      if (its >= maxit || breakdown) break;
      k_start_cycle<<<grid_for(n2), kBlock, 0, s>>>(n2, r, c->hn, c->Vb, c->g, restart);
      TP_LAUNCH_CHECK();
      // Iteration j is enqueued before the host looks at iteration j - 1's
      // convergence estimate (copied to pinned memory behind an event), so
      // the GPU never idles on the host; an iteration enqueued past the
      // stopping point is discarded (m counts checked columns only, and it
      // touches nothing that columns < m use).
      int m = 0;
      auto enqueue = [&](int j) {
        double* vj = c->Vb + (long long)j * n2;
        double* zj = c->Zb + (long long)j * n2;
        precond_apply(c, vj, vj + N, c->scales, s, j & 1);
        const bool probe_spmv = c->probe_which == 2;
        if (probe_spmv) {
          c->probe.npairs = 0;
          c->probe.active = j & 1;
          c->probe.before(s);
        }
        launch_pdl(k_block_spmv, grid_for(N), kBlock, s, N, c->rowptr, c->col,
                   reinterpret_cast<const double4_32a*>(c->bval), c->hpp->out, c->hS->out, zj,
                   zj + N, c->w, c->w + N, c->scales);
        if (probe_spmv) {
          c->probe.after(s, 36.0 * c->nnzb + 4.0 * (N + 1) + 48.0 * N);
          c->probe.active = 0;
        }
        // classical Gram-Schmidt against V_0..V_j, a second pass when the
        // first cancelled most of w
        double* h1 = c->h2;
        double* h2 = c->h2 + (restart + 2);
        const int G = orth_grid(c, n2);
        mdot_all(n2, c->Vb, n2, j + 1, c->w, c->kparts, Bm, h1, s);
        launch_pdl(k_orth_update, G, 256, s, n2, c->Vb, n2, j + 1, h1, c->w, c->oparts,
                   (const int*)nullptr);
        launch_pdl(k_reorth_gate, 1, 256, s, j + 1, h1, c->oparts, G, c->reorth);
        mdot_all(n2, c->Vb, n2, j + 1, c->w, c->kparts, Bm, h2, s, c->reorth);
        launch_pdl(k_orth_update, G, 256, s, n2, c->Vb, n2, j + 1, h2, c->w, c->oparts,
                   (const int*)c->reorth);
        launch_pdl(k_arnoldi, 1, 256, s, j, ldh, c->H, c->cs, c->sn, c->g, h1, h2, c->oparts, G,
                   c->hn, c->est);
        TP_CUDA_TRY(cudaMemcpyAsync(hp_host + kEstSlot + 4 * (j & 1), c->est, 3 * sizeof(double),
                                    cudaMemcpyDeviceToHost, s));
        TP_CUDA_TRY(cudaEventRecord(c->ev_est[j & 1], s));
        if (j + 1 < restart) {
          launch_pdl(k_normalize, grid_for(n2), kBlock, s, n2, c->w, c->hn,
                     c->Vb + (long long)(j + 1) * n2);
        }
      };
      // returns true when the cycle stops after column j (m set)
      auto check = [&](int j) {
        TP_CUDA_TRY(cudaEventSynchronize(c->ev_est[j & 1]));
        if (c->probe_which >= 0) c->probe.read_and_accumulate(j & 1);
        const double* e = hp_host + kEstSlot + 4 * (j & 1);
        const double est = e[0], hnv = e[1], den = e[2];
        ++its;
        m = j + 1;
        if (!std::isfinite(est) || !std::isfinite(hnv) || !(den > 0.0)) {
          breakdown = true;  // drop the singular or non-finite column j
          m = j;
          return true;
        }
        if (est <= rtol * bnorm || its >= maxit) return true;
        if (hnv == 0.0) return true;  // happy breakdown: the solution is in the space
        return false;
      };
      for (int j = 0; j < restart; ++j) {
        if (j == 0) enqueue(0);
        if (j + 1 < restart && its + 1 < maxit) enqueue(j + 1);
        if (check(j)) break;
      }
      if (m > 0) {
        k_hsolve<<<1, 32, 0, s>>>(m, ldh, c->H, c->g, c->yv);
        TP_LAUNCH_CHECK();
        k_update_x<<<grid_for(n2), kBlock, 0, s>>>(n2, c->Zb, n2, m, c->yv, c->xs);
        TP_LAUNCH_CHECK();
      }
      ++restarts;
      if (breakdown) break;
    }
  }
  // final true residual (scaled) and unscaled per-block residuals
  k_true_residual<<<B, 256, 0, s>>>(N, c->rowptr, c->col,
                                    reinterpret_cast<const double4_32a*>(c->bval), c->xs, c->bs,
                                    c->scales, c->w, c->kparts);
  TP_LAUNCH_CHECK();
  k_sum_to<<<1, 256, 0, s>>>(c->kparts, B, c->hn);
  TP_LAUNCH_CHECK();
  const double rfin = std::sqrt(read_double(c->hn, hp_host, s));
  k_unscaled_sums<<<B, 256, 0, s>>>(N, c->rowptr, c->col,
                                    reinterpret_cast<const double4_32a*>(c->bval), c->xs, bp,
                                    bT, c->kparts);
  TP_LAUNCH_CHECK();
  for (int q = 0; q < 4; ++q) {
    k_sum_to<<<1, 256, 0, s>>>(c->kparts + (long long)q * B, B, c->est + q);
    TP_LAUNCH_CHECK();
  }
  TP_CUDA_TRY(cudaMemcpyAsync(hp_host, c->est, 4 * sizeof(double), cudaMemcpyDeviceToHost, s));
  TP_CUDA_TRY(cudaMemcpyAsync(xp, c->xs, sizeof(double) * N, cudaMemcpyDeviceToDevice, s));
  TP_CUDA_TRY(cudaMemcpyAsync(xT, c->xs + N, sizeof(double) * N, cudaMemcpyDeviceToDevice, s));
  TP_CUDA_TRY(cudaStreamSynchronize(s));
  auto t1 = std::chrono::steady_clock::now();
  const double rp2 = hp_host[0], rT2 = hp_host[1], bp2 = hp_host[2], bT2 = hp_host[3];
  const double rel = bnorm > 0.0 ? rfin / bnorm : 0.0;
  if (status != TP_OK && bnorm > 0.0 && rel <= rtol) status = TP_OK;
  if (breakdown && status != TP_OK) status = TP_BREAKDOWN;
  if (info) {
    info->iters = its;
    info->restarts = restarts;
    info->status = status;
    info->rel_res = rel;
    info->rel_res_unscaled = (bp2 + bT2) > 0 ? std::sqrt((rp2 + rT2) / (bp2 + bT2)) : 0.0;
    info->rel_res_p = bp2 > 0 ? std::sqrt(rp2 / bp2) : std::sqrt(rp2);
    info->rel_res_T = bT2 > 0 ? std::sqrt(rT2 / bT2) : std::sqrt(rT2);
    info->t_solve_ms = std::chrono::duration<double, std::milli>(t1 - t0).count();
    info->levels_pp = (int)c->hpp->L.size();
    info->levels_S = (int)c->hS->L.size();
    info->opc_pp = c->hpp->operator_complexity();
    info->opc_S = c->hS->operator_complexity();
  }
  return status;
}

}  // namespace tp

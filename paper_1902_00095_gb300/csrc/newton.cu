// Newton iteration with line search of one backward-Euler step (Sec. 3:
// linearise G(x) = 0 at x_k and solve Eq. AXR for the increment; Sec. 4:
// line search, relative function-norm and relative step tolerances). The first iteration builds the preconditioner;
// later ones optionally keep the AMG structure (C/F splits, P, R, patterns)
// and refresh only the Galerkin values, so the captured graph is reused.
#include <chrono>
#include <cmath>
#include "solver.cuh"

namespace tp {

namespace {

__device__ __forceinline__ double wsum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  return v;
}

// partial sums of (sa a)^2 + (sb b)^2 over a fixed block partition
__global__ void __launch_bounds__(256) k_sumsq2(int N, const double* __restrict__ a,
                                                const double* __restrict__ b,
                                                const double* __restrict__ sa,
                                                const double* __restrict__ sb,
                                                double* __restrict__ partials) {
  __shared__ double sh[8];
  long long chunk = ((long long)N + gridDim.x - 1) / gridDim.x;
  long long lo = chunk * blockIdx.x, hi = lo + chunk;
  if (hi > N) hi = N;
  const double ka = sa ? sa[0] : 1.0, kb = sb ? sb[1] : 1.0;
  double s = 0.0;
  for (long long i = lo + threadIdx.x; i < hi; i += blockDim.x) {
    const double x = ka * a[i], y = kb * b[i];
    s += x * x + y * y;
  }
  s = wsum(s);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += sh[w];
    partials[blockIdx.x] = t;
  }
}

__global__ void k_finish_sum(const double* __restrict__ partials, int B, double* __restrict__ out) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    double s = 0.0;
    for (int b = 0; b < B; ++b) s += partials[b];
    *out = s;
  }
}

// (p, T) = (p0, T0) + alpha (dp, dT)
__global__ void k_axpby2(int N, const double* __restrict__ p0, const double* __restrict__ T0,
                         double alpha, const double* __restrict__ dp,
                         const double* __restrict__ dT, double* __restrict__ p,
                         double* __restrict__ T) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < N) {
    p[i] = p0[i] + alpha * dp[i];
    T[i] = T0[i] + alpha * dT[i];
  }
}

double sumsq2(tp_ctx* c, const double* a, const double* b, const double* scales) {
  cudaStream_t s = c->s;
  const int B = c->nparts;
  k_sumsq2<<<B, 256, 0, s>>>(c->N, a, b, scales, scales, c->partials);
  TP_LAUNCH_CHECK();
  k_finish_sum<<<1, 32, 0, s>>>(c->partials, B, c->tmpN);
  TP_LAUNCH_CHECK();
  TP_CUDA_TRY(cudaMemcpyAsync(c->host_est + 8, c->tmpN, sizeof(double), cudaMemcpyDeviceToHost, s));
  TP_CUDA_TRY(cudaStreamSynchronize(s));
  return c->host_est[8];
}

}  // namespace

int newton_step(tp_ctx* c, double dt, const tp_precond_opts& popts, const tp_newton_opts& no,
                tp_newton_info* info) {
  cudaStream_t s = c->s;
  const int N = c->N;
  auto t0 = std::chrono::steady_clock::now();
  double G0 = -1.0, relf = 1.0, reldx = 1.0;
  int k = 0, lin_its = 0, lin_status = TP_OK, status = TP_NOT_CONVERGED, ls_total = 0;
  double* dp = c->io2;
  double* dT = c->io3;
  if (!c->xsave_p) {
    c->xsave_p = c->pool.alloc<double>(N);
    c->xsave_T = c->pool.alloc<double>(N);
  }
  // linearise at x_0
  int st = assemble_device(c, dt);
  if (st != TP_OK) return st;
  launch_extract_blocks(c->nnzb, c->bval, c->App, c->ApT, c->ATp, c->ATT, s);
  launch_equation_scales(N, c->dpos, c->App, c->ATT, c->tmpN, c->partials, c->nparts,
                         c->scales, s);
  // the first linearisation fixes the scaling of the function norm
  TP_CUDA_TRY(cudaMemcpyAsync(c->fscale, c->scales, 2 * sizeof(double), cudaMemcpyDeviceToDevice, s));
  double G = std::sqrt(sumsq2(c, c->Rm, c->Re, c->fscale));
  G0 = G;
  for (k = 0;; ++k) {
    if (!std::isfinite(G)) {
      status = TP_ENONFINITE;
      break;
    }
    relf = G0 > 0.0 ? G / G0 : 0.0;
    if (G == 0.0 || (k > 0 && relf <= no.tol_f)) {
      status = TP_OK;
      break;
    }
    if (k >= no.max_newton) break;
    if (k == 0 || !no.reuse || !c->built) {
      build_device(c, popts);
    } else {
      refresh_device(c);
    }
    negated_residual(c);  // b = -G(x_k) into io0, io1
    tp_solve_info si{};
    lin_status = fgmres_solve(c, c->io0, c->io1, dp, dT, no.rtol, no.maxit, no.restart, &si);
    lin_its += si.iters;
    if (lin_status < 0) return lin_status;
    // line search (Sec. 4 names Newton with line search without its form;
    // taken as backtracking on the scaled function norm): x_k + alpha dx,
    // alpha = 1, 1/2, ... until ||G|| <= (1 - 1e-4 alpha) ||G(x_k)||, at most
    // max_ls halvings; a non-finite trial state counts as a rejected step
    TP_CUDA_TRY(cudaMemcpyAsync(c->xsave_p, c->p, sizeof(double) * N, cudaMemcpyDeviceToDevice, s));
    TP_CUDA_TRY(cudaMemcpyAsync(c->xsave_T, c->T, sizeof(double) * N, cudaMemcpyDeviceToDevice, s));
    double alpha = 1.0, Gt = G;
    const int max_ls = no.line_search ? 6 : 0;
    for (int ls = 0;; ++ls) {
      k_axpby2<<<grid_for(N), kBlock, 0, s>>>(N, c->xsave_p, c->xsave_T, alpha, dp, dT, c->p, c->T);
      TP_LAUNCH_CHECK();
      st = assemble_device(c, dt);
      if (st != TP_OK && st != TP_ENONFINITE) return st;
      const bool finite = st == TP_OK;
      if (finite) {
        launch_extract_blocks(c->nnzb, c->bval, c->App, c->ApT, c->ATp, c->ATT, s);
        launch_equation_scales(N, c->dpos, c->App, c->ATT, c->tmpN, c->partials, c->nparts,
                               c->scales, s);
        Gt = std::sqrt(sumsq2(c, c->Rm, c->Re, c->fscale));
      }
      if ((finite && std::isfinite(Gt) && Gt <= (1.0 - 1e-4 * alpha) * G) || ls >= max_ls) {
        if (!finite) return st;
        break;
      }
      alpha *= 0.5;
      ++ls_total;
    }
    G = Gt;
    const double dx = alpha * std::sqrt(sumsq2(c, dp, dT, nullptr));
    const double xn = std::sqrt(sumsq2(c, c->p, c->T, nullptr));
    reldx = xn > 0.0 ? dx / xn : 0.0;
    if (reldx <= no.tol_dx) {
      status = TP_OK;
      ++k;
      relf = G0 > 0.0 ? G / G0 : 0.0;
      break;
    }
  }
  TP_CUDA_TRY(cudaStreamSynchronize(s));
  auto t1 = std::chrono::steady_clock::now();
  if (info) {
    info->newton_iters = k;
    info->linear_iters = lin_its;
    info->status = status;
    info->last_linear_status = lin_status;
    info->rel_f = relf;
    info->rel_dx = reldx;
    info->t_ms = std::chrono::duration<double, std::milli>(t1 - t0).count();
    info->line_search_halvings = ls_total;
  }
  return status;
}

}  // namespace tp

// TPFA Newton-system assembly: cell properties, block-CSR Jacobian,
// residual and the Schur approximation S~_T (Sec. 2.2, Sec. 3, Eq. Se).
//
// One thread per cell writes its own block row (gather form): every face is
// evaluated by both of its cells, with the face always oriented from the
// lower to the higher cell index so that both evaluations agree bit for bit
// (and the upwind tie dPhi = 0 goes to the lower index, the "E1" side of the
// upwind rule in Sec. 2.2.1). No atomics; the result is deterministic.
#include "kernels.cuh"

namespace tp {

namespace {

__device__ __forceinline__ double density(double p, double T, const FluidDev& f) {
  return f.rho0 * exp(f.c * (p - f.p0)) * exp(f.beta * (T - f.T0));
}

// 7-point block pattern, columns ascending (z-1, y-1, x-1, self, x+1, y+1,
// z+1). The start of row i is i (diagonals of earlier rows) plus, for each
// axis, the faces whose lower cell is below i (upper entries of earlier
// rows) and the faces whose upper cell is below i (lower entries).
__device__ __forceinline__ long long faces_below(long long r, long long per_group,
                                                 long long group, long long n_total_lo) {
  // number of face lower-cells a < r when lower cells are the first
  // per_group of every `group` consecutive indices, capped by n_total_lo
  if (r <= 0) return 0;
  long long full = r / group, rem = r % group;
  long long v = full * per_group + (rem < per_group ? rem : per_group);
  return v < n_total_lo ? v : n_total_lo;
}

__global__ void k_pattern(GridDev g, int* __restrict__ rowptr, int* __restrict__ col,
                          int* __restrict__ dpos) {
  const int N = g.nx * g.ny * g.nz;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= N) return;
  const int nxy = g.nx * g.ny;
  const int x = i % g.nx, y = (i / g.nx) % g.ny, z = i / nxy;
  const long long nfx = (long long)(g.nx - 1) * g.ny * g.nz;
  const long long nfy = (long long)g.nx * (g.ny - 1) * g.nz;
  const long long nfz = (long long)nxy * (g.nz - 1);
  long long before = i;
  before += faces_below(i, g.nx - 1, g.nx, nfx) + faces_below(i - 1, g.nx - 1, g.nx, nfx);
  before += faces_below(i, nxy - g.nx, nxy, nfy) + faces_below(i - g.nx, nxy - g.nx, nxy, nfy);
  before += faces_below(i, N - nxy, N, nfz) + faces_below(i - nxy, N - nxy, N, nfz);
  int e = (int)before;
  rowptr[i] = e;
  if (z > 0) col[e++] = i - nxy;
  if (y > 0) col[e++] = i - g.nx;
  if (x > 0) col[e++] = i - 1;
  dpos[i] = e;
  col[e++] = i;
  if (x < g.nx - 1) col[e++] = i + 1;
  if (y < g.ny - 1) col[e++] = i + g.nx;
  if (z < g.nz - 1) col[e++] = i + nxy;
  if (i == N - 1) rowptr[N] = e;
}

__global__ void k_mix_conductivity(int N, const double* __restrict__ phi,
                                   const double* __restrict__ kTr, FluidDev f,
                                   double* __restrict__ kT) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= N) return;
  double ph = phi[i];
  kT[i] = (f.kT_mix == 0) ? ph * kTr[i] + (1.0 - ph) * f.kTf : (1.0 - ph) * kTr[i] + ph * f.kTf;
}

// Bennison heavy-oil viscosity coefficients (Table 1)
constexpr double kBennA1 = -0.8021, kBennA2 = 23.8765, kBennA3 = 0.31458, kBennA4 = -9.21592;
constexpr double kLn10 = 2.302585092994046;

// A1: rho, lam = rho/mu and the p/T derivatives of lam per cell.
__global__ void k_cell_props(int N, const double* __restrict__ p, const double* __restrict__ T,
                             FluidDev f, double* __restrict__ rho, double* __restrict__ lam,
                             double* __restrict__ lam_p, double* __restrict__ lam_T) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= N) return;
  double r = density(p[i], T[i], f);
  double mu, mlog_T;  // viscosity and d(ln mu)/dT
  if (f.mu_law == 1) {
    // Bennison (Eq. bennison, Table 1): mu in cp of T in degrees Fahrenheit
    const double tf = (T[i] - 273.15) * 1.8 + 32.0;
    const double ex = kBennA3 * f.api + kBennA4;
    mu = 1e-3 * exp(kLn10 * (kBennA1 * f.api + kBennA2) + ex * log(tf));
    mlog_T = ex * 1.8 / tf;
  } else {
    mu = f.mu0 * exp(-f.mu_coef * (T[i] - f.T_mu0));
    mlog_T = -f.mu_coef;
  }
  double l = r / mu;
  rho[i] = r;
  lam[i] = l;
  lam_p[i] = (f.c * r) / mu;
  // d(rho/mu)/dT = rho_T/mu - (rho/mu) d(ln mu)/dT
  lam_T[i] = (f.beta * r) / mu - mlog_T * l;
}

struct Face {
  double dF[4], dE[4], F, E, adv, Tcf;
  bool up_lo;
};

// Face transmissibilities (Sec. 2.2, Eq. Fm, Eq. Fe): for cell lo and each
// axis towards its upper neighbour hi, T_f = |e|/d 2 K_lo K_hi / (K_lo + K_hi)
// and Tc_f the same for the mixture conductivity; axis-major [3][N], 0 on the
// last layer of an axis. They depend on the fields only, so they are computed
// when the fields are set, not at every assembly (two FP64 divisions per face
// and side there).
__global__ void k_face_trans(GridDev g, const double* __restrict__ Kx,
                             const double* __restrict__ Ky, const double* __restrict__ Kz,
                             const double* __restrict__ kT, double* __restrict__ Tf,
                             double* __restrict__ Tc) {
  const int N = g.nx * g.ny * g.nz;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= N) return;
  const int nxy = g.nx * g.ny;
  const int x = i % g.nx, y = (i / g.nx) % g.ny, z = i / nxy;
  const bool has[3] = {x < g.nx - 1, y < g.ny - 1, z < g.nz - 1};
  const int step[3] = {1, g.nx, nxy};
#pragma unroll
  for (int ax = 0; ax < 3; ++ax) {
    double tf = 0.0, tc = 0.0;
    if (has[ax]) {
      const int hi = i + step[ax];
      const double area_over_d = ax == 0 ? (g.dy * g.dz) / g.dx
                                 : ax == 1 ? (g.dx * g.dz) / g.dy
                                           : (g.dx * g.dy) / g.dz;
      const double* K = ax == 0 ? Kx : ax == 1 ? Ky : Kz;
      const double Klo = K[i], Khi = K[hi], kTlo = kT[i], kThi = kT[hi];
      tf = area_over_d * __ddiv_rn(__dmul_rn(__dmul_rn(2.0, Klo), Khi), __dadd_rn(Klo, Khi));
      tc = area_over_d * __ddiv_rn(__dmul_rn(__dmul_rn(2.0, kTlo), kThi), __dadd_rn(kTlo, kThi));
    }
    Tf[(long long)ax * N + i] = tf;
    Tc[(long long)ax * N + i] = tc;
  }
}

// Face between cells lo < hi (quantities oriented lo -> hi).
__device__ __forceinline__ void face_terms(int lo, int hi, double Tf, double Tcf, double dzf,
                                           const double* __restrict__ p,
                                           const double* __restrict__ T,
                                           const double* __restrict__ rho,
                                           const double* __restrict__ lam,
                                           const double* __restrict__ lam_p,
                                           const double* __restrict__ lam_T,
                                           const FluidDev& f, double g, Face& o) {
  const double rlo = rho[lo], rhi = rho[hi];
  const double rhobar = __dmul_rn(0.5, __dadd_rn(rlo, rhi));
  const double dphi = __dsub_rn(__dsub_rn(p[lo], p[hi]), __dmul_rn(__dmul_rn(rhobar, g), dzf));
  const bool up_lo = dphi >= 0.0;
  const double lam_u = up_lo ? lam[lo] : lam[hi];
  const double Tlo = T[lo], Thi = T[hi];
  const double Tu = up_lo ? Tlo : Thi;
  const double F = Tf * lam_u * dphi;
  const double rho_p_lo = f.c * rlo, rho_p_hi = f.c * rhi;
  const double rho_T_lo = f.beta * rlo, rho_T_hi = f.beta * rhi;
  const double dPhi[4] = {1.0 - 0.5 * rho_p_lo * g * dzf, -0.5 * rho_T_lo * g * dzf,
                          -1.0 - 0.5 * rho_p_hi * g * dzf, -0.5 * rho_T_hi * g * dzf};
  const double dLam[4] = {up_lo ? lam_p[lo] : 0.0, up_lo ? lam_T[lo] : 0.0,
                          up_lo ? 0.0 : lam_p[hi], up_lo ? 0.0 : lam_T[hi]};
  const double dTup[4] = {0.0, up_lo ? 1.0 : 0.0, 0.0, up_lo ? 0.0 : 1.0};
  const double dTd[4] = {0.0, 1.0, 0.0, -1.0};
#pragma unroll
  for (int a = 0; a < 4; ++a) {
    o.dF[a] = Tf * (dLam[a] * dphi + lam_u * dPhi[a]);
    o.dE[a] = f.cv * (Tu * o.dF[a] + F * dTup[a]) + Tcf * dTd[a];
  }
  o.F = F;
  o.E = f.cv * Tu * F + Tcf * (Tlo - Thi);
  o.adv = f.cv * Tf * lam_u * dphi;
  o.Tcf = Tcf;
  o.up_lo = up_lo;
}

__global__ void __launch_bounds__(128) k_assemble(
    GridDev g, FluidDev f, const int* __restrict__ rowptr, const int* __restrict__ dpos,
    const double* __restrict__ Tf3, const double* __restrict__ Tc3,
    const double* __restrict__ phi, const double* __restrict__ p,
    const double* __restrict__ T, const double* __restrict__ p_n, const double* __restrict__ T_n,
    const double* __restrict__ rho, const double* __restrict__ lam,
    const double* __restrict__ lam_p, const double* __restrict__ lam_T, double dt,
    double* __restrict__ bval, double* __restrict__ Sval, double* __restrict__ Rm,
    double* __restrict__ Re) {
  const int N = g.nx * g.ny * g.nz;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= N) return;
  const int nxy = g.nx * g.ny;
  const int x = i % g.nx, y = (i / g.nx) % g.ny, z = i / nxy;
  const int d = dpos[i];
  double J[4] = {0.0, 0.0, 0.0, 0.0};
  double Sd = 0.0, rm = 0.0, re = 0.0;
  // neighbours in ascending column order; position of the block in the row
  int e = rowptr[i];
  const int nb[6] = {i - nxy, i - g.nx, i - 1, i + 1, i + g.nx, i + nxy};
  const bool has[6] = {z > 0, y > 0, x > 0, x < g.nx - 1, y < g.ny - 1, z < g.nz - 1};
  const int axis[6] = {2, 1, 0, 0, 1, 2};
#pragma unroll 1
  for (int q = 0; q < 6; ++q) {
    if (q == 3) e = d + 1;  // upper neighbours follow the diagonal
    if (!has[q]) continue;
    const int j = nb[q];
    const int lo = i < j ? i : j, hi = i < j ? j : i;
    const int ax = axis[q];
    const long long fidx = (long long)ax * N + lo;
    const double dzf = ax == 2 ? g.dz : 0.0;
    Face o;
    face_terms(lo, hi, Tf3[fidx], Tc3[fidx], dzf, p, T, rho, lam, lam_p, lam_T, f, g.g, o);
    double* blk = bval + 4ll * e;
    if (i == lo) {
      rm += o.F;
      re += o.E;
      J[0] += o.dF[0]; J[1] += o.dF[1]; J[2] += o.dE[0]; J[3] += o.dE[1];
      blk[0] = o.dF[2]; blk[1] = o.dF[3]; blk[2] = o.dE[2]; blk[3] = o.dE[3];
      double off = -o.Tcf;
      if (o.up_lo) Sd += o.adv; else off += o.adv;
      Sd += o.Tcf;
      Sval[e] = off;
    } else {
      rm -= o.F;
      re -= o.E;
      J[0] -= o.dF[2]; J[1] -= o.dF[3]; J[2] -= o.dE[2]; J[3] -= o.dE[3];
      blk[0] = -o.dF[0]; blk[1] = -o.dF[1]; blk[2] = -o.dE[0]; blk[3] = -o.dE[1];
      double off = -o.Tcf;
      if (o.up_lo) off -= o.adv; else Sd -= o.adv;
      Sd += o.Tcf;
      Sval[e] = off;
    }
    ++e;
  }
  // accumulation (backward Euler)
  const double V = g.dx * g.dy * g.dz;
  const double ph = phi[i];
  const double r = rho[i], Ti = T[i];
  const double rho_p = f.c * r, rho_T = f.beta * r;
  const double rn = density(p_n[i], T_n[i], f);
  const double Tn = T_n[i];
  const double rock = (1.0 - ph) * f.rho_r * f.cr;
  const double vdt = V / dt;  // one FP64 division per cell, not seven
  rm += vdt * (ph * (r - rn));
  re += vdt * (ph * f.cv * (r * Ti - rn * Tn) + rock * (Ti - Tn));
  J[0] += vdt * (ph * rho_p);
  J[1] += vdt * (ph * rho_T);
  J[2] += vdt * (ph * f.cv * rho_p * Ti);
  J[3] += vdt * (ph * f.cv * (rho_T * Ti + r) + rock);
  Sd += vdt * (ph * f.cv * r + rock);
  double* blk = bval + 4ll * d;
  blk[0] = J[0]; blk[1] = J[1]; blk[2] = J[2]; blk[3] = J[3];
  Sval[d] = Sd;
  Rm[i] = rm;
  Re[i] = re;
}

__device__ __forceinline__ double peaceman_wi(double kx, double ky) {
  const double Dx = 5.0, Dy = 5.0, h = 5.0, rw = 0.1;
  const double Ke = sqrt(kx * ky);
  const double ryx = sqrt(ky / kx), rxy = sqrt(kx / ky);
  const double re = 0.14 * sqrt(ryx * Dx * Dx + rxy * Dy * Dy) / (0.5 * (sqrt(ryx) + sqrt(rxy)));
  return 2.0 * 3.141592653589793 * h * Ke / log(re / rw);
}

// Wells and heaters (Eq. f, Eq. fT, Peaceman model, heater law): one thread
// per completed cell, completions in input order.
__global__ void k_wells(int ncells, const int* __restrict__ wcell, const int* __restrict__ woff,
                        const int* __restrict__ kind, const int* __restrict__ nl,
                        const double* __restrict__ value, const double* __restrict__ Tinj,
                        const double* __restrict__ Uh, FluidDev f, const int* __restrict__ dpos,
                        const double* __restrict__ Kx, const double* __restrict__ Ky,
                        const double* __restrict__ p, const double* __restrict__ T,
                        const double* __restrict__ rho, const double* __restrict__ lam,
                        const double* __restrict__ lam_p, const double* __restrict__ lam_T,
                        double* __restrict__ bval, double* __restrict__ Sval,
                        double* __restrict__ Rm, double* __restrict__ Re) {
  int gi = blockIdx.x * blockDim.x + threadIdx.x;
  if (gi >= ncells) return;
  const int c = wcell[gi];
  const int d = dpos[c];
  double* blk = bval + 4ll * d;
  for (int k = woff[gi]; k < woff[gi + 1]; ++k) {
    const int kd = kind[k];
    const double pc = p[c], Tc = T[c];
    if (kd == 0) {
      const double q = value[k] / nl[k];
      const double ti = Tinj[k];
      const double rho_inj = density(pc, ti, f);
      const double rho_inj_p = f.c * rho_inj;
      Rm[c] -= q * rho_inj;
      Re[c] -= q * rho_inj * f.cv * ti;
      blk[0] -= q * rho_inj_p;
      blk[2] -= q * rho_inj_p * f.cv * ti;
    } else if (kd == 1) {
      const double wi = peaceman_wi(Kx[c], Ky[c]);
      const double dp = pc - value[k];
      if (dp > 0.0) {
        const double l = lam[c], lp = lam_p[c], lT = lam_T[c];
        Rm[c] += wi * dp * l;
        Re[c] += wi * dp * l * f.cv * Tc;
        blk[0] += wi * (l + dp * lp);
        blk[1] += wi * dp * lT;
        blk[2] += wi * f.cv * Tc * (l + dp * lp);
        blk[3] += wi * dp * f.cv * (lT * Tc + l);
        Sval[d] += f.cv * wi * dp * l;
      }
    } else if (kd == 2) {
      const double U = Uh[k];
      Re[c] -= U * (Tinj[k] - Tc);
      blk[3] += U;
      Sval[d] += U;
    } else if (kd == 3) {
      const double q = value[k] / nl[k];
      const double r = rho[c];
      const double rp = f.c * r, rT = f.beta * r;
      Rm[c] += q * r;
      Re[c] += q * r * f.cv * Tc;
      blk[0] += q * rp;
      blk[1] += q * rT;
      blk[2] += q * f.cv * rp * Tc;
      blk[3] += q * f.cv * (rT * Tc + r);
      Sval[d] += f.cv * q * r;
    }
  }
}

__global__ void k_extract(int nnzb, const double4_32a* __restrict__ bval, double* __restrict__ App,
                          double* __restrict__ ApT, double* __restrict__ ATp,
                          double* __restrict__ ATT) {
  int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= nnzb) return;
  double4_32a b = bval[e];
  App[e] = b.x;
  ApT[e] = b.y;
  ATp[e] = b.z;
  ATT[e] = b.w;
}

__global__ void k_abs_diag(int N, const int* __restrict__ dpos, const double* __restrict__ A,
                           double* __restrict__ out) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < N) out[i] = fabs(A[dpos[i]]);
}

__global__ void k_scales(int N, const double* __restrict__ sums, double* __restrict__ scales) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    scales[0] = (double)N / sums[0];
    scales[1] = (double)N / sums[1];
  }
}

// 24 learned-correction features per cell (FP32 [N][24]):
// 0-5 log10(T_f/1e-12), 6-11 log10(Tc_f), 12 log10(lam/1e6), 13-18 outward
// advective face coefficient / S~_ii, 19 A_pT A_Tp / (A_pp A_TT) at the
// diagonal, 20 log10(A_pp,ii s_m), 21 log10(A_TT,ii s_e),
// 22 (A_TT,ii - S~_ii) / S~_ii, 23 accumulation / S~_ii.
__global__ void __launch_bounds__(128) k_features(
    GridDev g, FluidDev f, const int* __restrict__ dpos, const double* __restrict__ Tf3,
    const double* __restrict__ Tc3, const double* __restrict__ phi,
    const double* __restrict__ p, const double* __restrict__ T,
    const double* __restrict__ rho, const double* __restrict__ lam,
    const double* __restrict__ lam_p, const double* __restrict__ lam_T,
    const double* __restrict__ bval, const double* __restrict__ Sval,
    const double* __restrict__ scales, double dt, float* __restrict__ F) {
  const int N = g.nx * g.ny * g.nz;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= N) return;
  const int nxy = g.nx * g.ny;
  const int x = i % g.nx, y = (i / g.nx) % g.ny, z = i / nxy;
  const int d = dpos[i];
  const double Sd = Sval[d];
  float* out = F + (size_t)i * 24;
  const int nb[6] = {i - nxy, i - g.nx, i - 1, i + 1, i + g.nx, i + nxy};
  const bool has[6] = {z > 0, y > 0, x > 0, x < g.nx - 1, y < g.ny - 1, z < g.nz - 1};
  const int axis[6] = {2, 1, 0, 0, 1, 2};
#pragma unroll 1
  for (int q = 0; q < 6; ++q) {
    if (!has[q]) {
      out[q] = 0.f;
      out[6 + q] = 0.f;
      out[13 + q] = 0.f;
      continue;
    }
    const int j = nb[q];
    const int lo = i < j ? i : j, hi = i < j ? j : i;
    const int ax = axis[q];
    const long long fidx = (long long)ax * N + lo;
    const double dzf = ax == 2 ? g.dz : 0.0;
    Face o;
    face_terms(lo, hi, Tf3[fidx], Tc3[fidx], dzf, p, T, rho, lam, lam_p, lam_T, f, g.g, o);
    out[q] = (float)log10(Tf3[fidx] / 1e-12);
    out[6 + q] = (float)log10(o.Tcf);
    out[13 + q] = (float)((i == lo ? o.adv : -o.adv) / Sd);
  }
  const double4_32a b = reinterpret_cast<const double4_32a*>(bval)[d];
  out[12] = (float)log10(lam[i] / 1e6);
  out[19] = (float)(b.y * b.z / (b.x * b.w));
  out[20] = (float)log10(fabs(b.x) * scales[0]);
  out[21] = (float)log10(fabs(b.w) * scales[1]);
  out[22] = (float)((b.w - Sd) / Sd);
  const double V = g.dx * g.dy * g.dz;
  const double ph = phi[i];
  out[23] = (float)(V * (ph * f.cv * rho[i] + (1.0 - ph) * f.rho_r * f.cr) / dt / Sd);
}

}  // namespace

void launch_features(const GridDev& g, const FluidDev& f, const int* dpos, const double* Tf3,
                     const double* Tc3, const double* phi, const double* p, const double* T,
                     const double* rho, const double* lam, const double* lam_p,
                     const double* lam_T, const double* bval, const double* Sval,
                     const double* scales, double dt, float* F, cudaStream_t s) {
  int N = g.nx * g.ny * g.nz;
  k_features<<<grid_for(N, 128), 128, 0, s>>>(g, f, dpos, Tf3, Tc3, phi, p, T, rho, lam, lam_p,
                                              lam_T, bval, Sval, scales, dt, F);
  TP_LAUNCH_CHECK();
}

void launch_pattern(const GridDev& g, int* rowptr, int* col, int* dpos, cudaStream_t s) {
  int N = g.nx * g.ny * g.nz;
  k_pattern<<<grid_for(N), kBlock, 0, s>>>(g, rowptr, col, dpos);
  TP_LAUNCH_CHECK();
}

void launch_mix_conductivity(int N, const double* phi, const double* kTr, const FluidDev& f,
                             double* kT, cudaStream_t s) {
  k_mix_conductivity<<<grid_for(N), kBlock, 0, s>>>(N, phi, kTr, f, kT);
  TP_LAUNCH_CHECK();
}

void launch_cell_props(int N, const double* p, const double* T, const FluidDev& f, double* rho,
                       double* lam, double* lam_p, double* lam_T, cudaStream_t s) {
  k_cell_props<<<grid_for(N), kBlock, 0, s>>>(N, p, T, f, rho, lam, lam_p, lam_T);
  TP_LAUNCH_CHECK();
}

void launch_face_trans(const GridDev& g, const double* Kx, const double* Ky, const double* Kz,
                       const double* kT, double* Tf3, double* Tc3, cudaStream_t s) {
  const int N = g.nx * g.ny * g.nz;
  k_face_trans<<<grid_for(N), kBlock, 0, s>>>(g, Kx, Ky, Kz, kT, Tf3, Tc3);
  TP_LAUNCH_CHECK();
}

void launch_assemble(const GridDev& g, const FluidDev& f, const int* rowptr, const int* dpos,
                     const double* Tf3, const double* Tc3, const double* phi, const double* p,
                     const double* T, const double* p_n, const double* T_n, const double* rho,
                     const double* lam, const double* lam_p, const double* lam_T, double dt,
                     double* bval, double* Sval, double* Rm, double* Re, cudaStream_t s) {
  int N = g.nx * g.ny * g.nz;
  k_assemble<<<grid_for(N, 128), 128, 0, s>>>(g, f, rowptr, dpos, Tf3, Tc3, phi, p, T, p_n, T_n,
                                               rho, lam, lam_p, lam_T, dt, bval, Sval, Rm, Re);
  TP_LAUNCH_CHECK();
}

void launch_wells(const GridDev& g, const FluidDev& f, const WellsDev& w, const int* dpos,
                  const double* Kx, const double* Ky, const double* p, const double* T,
                  const double* rho, const double* lam, const double* lam_p, const double* lam_T,
                  double* bval, double* Sval, double* Rm, double* Re, cudaStream_t s) {
  (void)g;
  if (w.ncells == 0) return;
  k_wells<<<grid_for(w.ncells, 64), 64, 0, s>>>(w.ncells, w.cell, w.off, w.kind, w.nlayers,
                                                w.value, w.T_inj, w.U, f, dpos, Kx, Ky, p, T,
                                                rho, lam, lam_p, lam_T, bval, Sval, Rm, Re);
  TP_LAUNCH_CHECK();
}

void launch_extract_blocks(int nnzb, const double* bval, double* App, double* ApT, double* ATp,
                           double* ATT, cudaStream_t s) {
  k_extract<<<grid_for(nnzb), kBlock, 0, s>>>(nnzb, reinterpret_cast<const double4_32a*>(bval), App,
                                              ApT, ATp, ATT);
  TP_LAUNCH_CHECK();
}

void launch_equation_scales(int N, const int* dpos, const double* App, const double* ATT,
                            double* tmp, double* partials, int nparts, double* scales,
                            cudaStream_t s) {
  // scales[0..1] first receive the two sums, then are turned into N / sum.
  k_abs_diag<<<grid_for(N), kBlock, 0, s>>>(N, dpos, App, tmp);
  TP_LAUNCH_CHECK();
  sum_fixed(tmp, N, scales + 0, partials, nparts, s);
  k_abs_diag<<<grid_for(N), kBlock, 0, s>>>(N, dpos, ATT, tmp);
  TP_LAUNCH_CHECK();
  sum_fixed(tmp, N, scales + 1, partials, nparts, s);
  k_scales<<<1, 32, 0, s>>>(N, scales, scales);
  TP_LAUNCH_CHECK();
}

}  // namespace tp

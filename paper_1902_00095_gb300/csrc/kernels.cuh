// Launchers of the thermo kernels (internal header).
#pragma once
#include "common.cuh"

namespace tp {

// ------------------------------------------------------------ assembly
struct FluidDev {
  double rho0, c, beta, p0, T0, mu0, T_mu0, mu_coef, cv, rho_r, cr, kTf;
  int kT_mix;
  int mu_law;  // 0 exponential, 1 Bennison (Eq. bennison)
  double api;
};

struct GridDev {
  int nx, ny, nz;
  double dx, dy, dz, g;
};

// Completions grouped by cell: cell g owns entries [off[g], off[g+1]).
struct WellsDev {
  int ncells = 0;
  int* cell = nullptr;
  int* off = nullptr;
  int* kind = nullptr;
  int* nlayers = nullptr;
  double* value = nullptr;
  double* T_inj = nullptr;
  double* U = nullptr;
};

void launch_pattern(const GridDev& g, int* rowptr, int* col, int* dpos, cudaStream_t s);
void launch_mix_conductivity(int N, const double* phi, const double* kTr, const FluidDev& f,
                             double* kT, cudaStream_t s);
void launch_cell_props(int N, const double* p, const double* T, const FluidDev& f,
                       double* rho, double* lam, double* lam_p, double* lam_T, cudaStream_t s);
// Face transmissibilities T_f, Tc_f per cell and axis towards the upper
// neighbour ([3][N], axis-major), from the fields.
void launch_face_trans(const GridDev& g, const double* Kx, const double* Ky, const double* Kz,
                       const double* kT, double* Tf3, double* Tc3, cudaStream_t s);
// Jacobian (block-CSR, 4 doubles per block), residual and S~_T values.
void launch_assemble(const GridDev& g, const FluidDev& f, const int* rowptr, const int* dpos,
                     const double* Tf3, const double* Tc3, const double* phi, const double* p,
                     const double* T, const double* p_n, const double* T_n, const double* rho,
                     const double* lam, const double* lam_p, const double* lam_T, double dt,
                     double* bval, double* Sval, double* Rm, double* Re, cudaStream_t s);
void launch_wells(const GridDev& g, const FluidDev& f, const WellsDev& w, const int* dpos,
                  const double* Kx, const double* Ky, const double* p, const double* T,
                  const double* rho, const double* lam, const double* lam_p, const double* lam_T,
                  double* bval, double* Sval, double* Rm, double* Re, cudaStream_t s);
void launch_extract_blocks(int nnzb, const double* bval, double* App, double* ApT, double* ATp,
                           double* ATT, cudaStream_t s);
// s_m = N / sum |A_pp,ii|, s_e = N / sum |A_TT,ii| into scales[0..1].
void launch_equation_scales(int N, const int* dpos, const double* App, const double* ATT,
                            double* tmp, double* partials, int nparts, double* scales,
                            cudaStream_t s);

// learned-correction features (FP32 [N][24]) at the last assembly
void launch_features(const GridDev& g, const FluidDev& f, const int* dpos, const double* Tf3,
                     const double* Tc3, const double* phi, const double* p, const double* T,
                     const double* rho, const double* lam, const double* lam_p,
                     const double* lam_T, const double* bval, const double* Sval,
                     const double* scales, double dt, float* F, cudaStream_t s);

// ------------------------------------------------------ sparse kernels
// y = D A x for the block matrix; D = diag(scales[0], scales[1]) or identity
// when scales == nullptr. Split vectors.
void launch_block_spmv(int N, const int* rowptr, const int* col, const double* bval,
                       const double* xp, const double* xT, double* yp, double* yT,
                       const double* scales, cudaStream_t s);

}  // namespace tp

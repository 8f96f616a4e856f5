// Solver context behind the C-ABI (internal header).
#pragma once
#include <memory>
#include "amg.cuh"
#include "kernels.cuh"
#include "learned.cuh"

struct tp_ctx {
  cudaStream_t s = nullptr;
  int device = 0;
  int num_sms = 152;
  tp::GridDev grid{};
  tp::FluidDev fluid{};
  int N = 0, nnzb = 0;
  tp::Pool pool;  // persistent buffers
  // block pattern (7-point, ascending columns)
  int* rowptr = nullptr;
  int* col = nullptr;
  int* dpos = nullptr;
  // cell fields
  double *Kx = nullptr, *Ky = nullptr, *Kz = nullptr, *phi = nullptr, *kTr = nullptr,
         *kT = nullptr;
  double *Tf3 = nullptr, *Tc3 = nullptr;  // face transmissibilities [3][N] (from the fields)
  bool fields_set = false;
  // wells
  tp::WellsDev wells;
  tp::Pool wpool;
  // state and properties
  double *p = nullptr, *T = nullptr, *pn = nullptr, *Tn = nullptr;
  double *rho = nullptr, *lam = nullptr, *lam_p = nullptr, *lam_T = nullptr;
  // assembled system
  double* bval = nullptr;  // [4 * nnzb]
  double* Sval = nullptr;  // [nnzb]
  double *Rm = nullptr, *Re = nullptr;
  double *App = nullptr, *ApT = nullptr, *ATp = nullptr, *ATT = nullptr;
  double* scales = nullptr;  // [2] equation scales s_m, s_e
  double* ones = nullptr;    // [2] = {1, 1}
  double* fscale = nullptr;  // [2] scaling of the Newton function norm
  double* partials = nullptr;
  int nparts = 0;
  double* tmpN = nullptr;
  bool assembled = false;
  // preconditioner
  tp_precond_opts opts{};
  std::unique_ptr<tp::Hierarchy> hpp, hS;
  // S~_diag (schur = 3): B = diag(A_pp)^-1 A_pT, C = A_Tp B, S = A_TT - C
  tp::Pool dpool, dscratch;
  double* Bd = nullptr;
  tp::DevCSR Cd, Sd;
  cudaStream_t s2 = nullptr;   // second stream: S~ hierarchy setup
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
  double* S_active = nullptr;  // values of the Schur approximation used
  double *bp_s = nullptr, *bT_s = nullptr;
  bool built = false;
  cudaGraphExec_t pc_graph = nullptr;
  cudaGraph_t pc_graph_tmpl = nullptr;   // kept: its event nodes are re-pointed per launch
  // probe event-record nodes of the preconditioner graph and the event index
  // (within a probe set) each one records; probe_set = set they point at
  std::vector<std::pair<cudaGraphNode_t, int>> probe_nodes;
  int probe_set = 0;
  long long pc_graph_kernels = 0;
  // timing probe: -1 off, 0 finest A_pp sweeps, 1 finest S~ sweeps, 2 block SpMV
  int probe_which = -1;
  tp::Probe probe;
  // Krylov workspace
  tp::Pool kpool;
  int restart_alloc = 0;
  double *Vb = nullptr, *Zb = nullptr, *w = nullptr, *xs = nullptr, *bs = nullptr;
  double *H = nullptr, *cs = nullptr, *sn = nullptr, *g = nullptr, *yv = nullptr,
         *hn = nullptr, *est = nullptr, *kparts = nullptr, *h2 = nullptr;
  double* oparts = nullptr;    // norm partials of the orthogonalisation update
  int* reorth = nullptr;       // 1: this column's Gram-Schmidt takes its second pass
  double* host_est = nullptr;  // pinned [32]
  cudaEvent_t ev_est[2] = {nullptr, nullptr};  // convergence estimates of iterations j, j+1
  // learned Schur correction
  struct tp_mlp* model = nullptr;
  tp::Pool lpool;
  float* feat = nullptr;      // [N][24]
  float* mlp_out = nullptr;   // [N][8]
  double* S_learned = nullptr;
  int* nbad = nullptr;
  int learned_fallback_rows = 0;
  bool learned_global_fallback = false;
  double dt_last = 0.0;
  double *xsave_p = nullptr, *xsave_T = nullptr;  // Newton line-search base point
  // user-facing scratch for host pointer marshalling
  double *io0 = nullptr, *io1 = nullptr, *io2 = nullptr, *io3 = nullptr;

  ~tp_ctx();
};

namespace tp {
long long launches_total();
// block preconditioner (Sec. 3.2) applied to (vp, vT) in the scaled system:
// z = M^{-1} D^{-1} v with D = diag(scales); result left in hpp->out, hS->out.
void precond_record(tp_ctx* c, cudaStream_t s);
void precond_apply(tp_ctx* c, const double* vp, const double* vT, const double* scales,
                   cudaStream_t s, int set = 0);
int fgmres_solve(tp_ctx* c, const double* bp, const double* bT, double* xp, double* xT,
                 double rtol, int maxit, int restart, tp_solve_info* info);
// device-resident steps shared by the C-ABI calls and the Newton driver
int assemble_device(tp_ctx* c, double dt);              // at (c->p, c->T)
void build_device(tp_ctx* c, const tp_precond_opts& o);  // full setup + graph
void refresh_device(tp_ctx* c);                          // numeric-only
void negated_residual(tp_ctx* c);                        // io0, io1 = -G
int newton_step(tp_ctx* c, double dt, const tp_precond_opts& popts, const tp_newton_opts& no,
                tp_newton_info* info);
int scalar_fgmres(tp_ctx* c, Hierarchy& h, const DevCSR& A, const double* b, double* x,
                  double rtol, int maxit, int restart);
int probe_schur_column(tp_ctx* c, int j, double rtol, int maxit, int* entry, double* value);
void learned_features(tp_ctx* c);  // features of the last assembly into c->feat
}  // namespace tp

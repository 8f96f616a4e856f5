// C-ABI entry points of the thermo library (declared in include/thermo.h).
// Every entry point converts internal errors into status codes; nothing is
// thrown across the ABI.
#include <cmath>
#include <cstring>
#include <algorithm>
#include <thread>
#include "solver.cuh"

using tp::Error;
using tp::fail;

namespace {

thread_local std::string g_last_error;

#define TP_API_BEGIN try {
#define TP_API_END                                   \
  }                                                  \
  catch (const Error& e) {                           \
    g_last_error = e.what;                           \
    cudaGetLastError();                              \
    return e.code;                          \
  }                                                  \
  catch (const std::bad_alloc&) {                    \
    g_last_error = "host allocation failed";         \
    return TP_ENOMEM;                                \
  }                                                  \
  catch (...) {                                      \
    g_last_error = "unexpected exception";           \
    return TP_ECUDA;                                 \
  }

void to_device(double* dst, const double* src, size_t n, int ptr_is_device, cudaStream_t s) {
  TP_CUDA_TRY(cudaMemcpyAsync(dst, src, n * sizeof(double),
                              ptr_is_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, s));
}

void from_device(double* dst, const double* src, size_t n, int ptr_is_device, cudaStream_t s) {
  TP_CUDA_TRY(cudaMemcpyAsync(dst, src, n * sizeof(double),
                              ptr_is_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, s));
}

__global__ void k_check_fields(int N, const double* Kx, const double* Ky, const double* Kz,
                               const double* phi, const double* kTr, int* flags) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= N) return;
  double v[5] = {Kx[i], Ky[i], Kz[i], phi[i], kTr[i]};
  for (int q = 0; q < 5; ++q)
    if (!isfinite(v[q])) atomicOr(flags, 1);
  if (!(Kx[i] > 0.0) || !(Ky[i] > 0.0) || !(Kz[i] > 0.0) || !(phi[i] > 0.0) || !(phi[i] < 1.0) ||
      !(kTr[i] >= 0.0))
    atomicOr(flags, 2);
}

__global__ void k_check_finite(long long n, const double* a, int* flags) {
  long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i < n && !isfinite(a[i])) atomicOr(flags, 1);
}

__global__ void k_negate(double* a, long long n) {
  long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i < n) a[i] = -a[i];
}

__global__ void k_fill(double* a, long long n, double v) {
  long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i < n) a[i] = v;
}

void negate(double* a, long long n, cudaStream_t s) {
  k_negate<<<tp::grid_for(n), tp::kBlock, 0, s>>>(a, n);
  TP_LAUNCH_CHECK();
}

int read_flags(int* d, cudaStream_t s) {
  int h = 0;
  TP_CUDA_TRY(cudaMemcpyAsync(&h, d, sizeof(int), cudaMemcpyDeviceToHost, s));
  TP_CUDA_TRY(cudaStreamSynchronize(s));
  return h;
}

tp::AmgOpts amg_opts(const tp_precond_opts& o) {
  tp::AmgOpts a;
  a.interp = o.interp;
  a.smoother = o.smoother;
  a.nu_pre = o.nu_pre;
  a.nu_post = o.nu_post;
  a.cheb_degree = o.cheb_degree;
  a.theta = o.theta;
  a.max_levels = o.max_levels;
  a.coarse_size = o.coarse_size;
  a.seed = o.seed;
  a.precision = o.precision;
  a.pmax = o.pmax;
  a.tail_rows = o.tail_rows;
  a.sell_rows = o.sell_rows;
  return a;
}

void check_opts(const tp_precond_opts& o) {
  if (o.schur < 0 || o.schur > 3)
    fail(TP_EINVAL, "schur must be 0 (S~_T), 1 (learned), 2 (A_TT) or 3 (S~_diag)");
  if (o.variant != 0 && o.variant != 1) fail(TP_EINVAL, "variant must be 0 or 1");
  if (o.precision < 0 || o.precision > 2) fail(TP_EINVAL, "precision must be 0, 1 or 2");
  if (o.interp != 0 && o.interp != 1) fail(TP_EINVAL, "interp must be 0 or 1");
  if (o.smoother != 0 && o.smoother != 1) fail(TP_EINVAL, "smoother must be 0 or 1");
  if (o.smoother_S < -1 || o.smoother_S > 2)
    fail(TP_EINVAL, "smoother_S must be -1, 0, 1 or 2");
  if (o.smoother_S == 2 && (o.nu_line < 1 || o.nu_line > 8))
    fail(TP_EINVAL, "nu_line must be in 1..8");
  if (o.cheb_degree < 1 || o.cheb_degree > 4) fail(TP_EINVAL, "cheb_degree must be in 1..4");
  if (o.nu_pre < 1 || o.nu_post < 1 || o.nu_pre > 8 || o.nu_post > 8)
    fail(TP_EINVAL, "nu_pre and nu_post must be in 1..8");
  if (!(o.theta > 0.0 && o.theta < 1.0)) fail(TP_EINVAL, "theta must be in (0, 1)");
  if (o.max_levels < 1 || o.coarse_size < 1) fail(TP_EINVAL, "max_levels, coarse_size >= 1");
  if (o.interp_S < -1 || o.interp_S > 1 || o.max_levels_S < 0 || o.nu_S < 0 || o.nu_S > 8)
    fail(TP_EINVAL, "bad Schur-hierarchy override");
  if (o.pmax < 0 || o.pmax > 16) fail(TP_EINVAL, "pmax must be in 0..16");
  if (o.tail_rows < 0) fail(TP_EINVAL, "tail_rows must be >= 0");
  if (o.sell_rows < -1) fail(TP_EINVAL, "sell_rows must be >= -1");
}

}  // namespace

tp_ctx::~tp_ctx() {
  if (pc_graph) cudaGraphExecDestroy(pc_graph);
  if (pc_graph_tmpl) cudaGraphDestroy(pc_graph_tmpl);
  probe.destroy();
  hpp.reset();
  hS.reset();
  if (host_est) cudaFreeHost(host_est);
  if (ev_fork) cudaEventDestroy(ev_fork);
  for (cudaEvent_t e : ev_est)
    if (e) cudaEventDestroy(e);
  if (ev_join) cudaEventDestroy(ev_join);
  if (s2) cudaStreamDestroy(s2);
}

struct tp_amg {
  cudaStream_t s = nullptr;
  bool own_stream = false;
  tp::Pool pool;
  tp::DevCSR A;
  std::unique_ptr<tp::Hierarchy> h;
  ~tp_amg() {
    h.reset();
    pool.release();
    if (own_stream && s) cudaStreamDestroy(s);
  }
};

struct tp_mlp {
  cudaStream_t s = nullptr;
  bool own_stream = false;
  tp::Pool pool;
  tp::MlpDev m;
  tp::Pool stage;  // device copies of host inputs
  int cap = 0;
  float* X = nullptr;
  int* slot = nullptr;
  double *St = nullptr, *Sd = nullptr, *tgt = nullptr;
  float* O = nullptr;
  float* partials = nullptr;
  double* host = nullptr;  // pinned [kMlpPartial]
  ~tp_mlp() {
    stage.release();
    pool.release();
    if (host) cudaFreeHost(host);
    if (own_stream && s) cudaStreamDestroy(s);
  }
  void ensure(int n) {
    if (n <= cap) return;
    stage.release();
    cap = n;
    X = stage.alloc<float>((size_t)n * tp::kMlpIn);
    slot = stage.alloc<int>(n);
    St = stage.alloc<double>(n);
    Sd = stage.alloc<double>(n);
    tgt = stage.alloc<double>(n);
    O = stage.alloc<float>((size_t)n * tp::kMlpOut);
    partials = stage.alloc<float>((size_t)((n + 15) / 16) * tp::kMlpPartial);
  }
};

namespace {
std::vector<std::pair<tp_ctx*, cudaStream_t>>& owned_streams() {
  static std::vector<std::pair<tp_ctx*, cudaStream_t>> v;
  return v;
}
}  // namespace

extern "C" {

void tp_default_opts(tp_precond_opts* o) {
  if (!o) return;
  std::memset(o, 0, sizeof(*o));
  o->schur = 0;
  o->variant = 0;
  o->precision = 0;
  o->interp = 1;
  o->smoother = 0;
  o->nu_pre = 3;
  o->nu_post = 4;
  o->cheb_degree = 2;
  o->theta = 0.25;
  o->max_levels = 25;
  o->coarse_size = 256;
  o->seed = 0;
  o->use_graphs = 1;
  o->interp_S = 0;
  o->max_levels_S = 0;
  o->nu_S = 1;
  o->pmax = 4;
  o->smoother_S = 2;
  o->tail_rows = 0;
  o->nu_line = 1;
  o->sell_rows = 0;
}

const char* tp_status_string(int st) {
  switch (st) {
    case TP_OK: return "ok";
    case TP_EINVAL: return "invalid argument";
    case TP_ENOMEM: return "out of memory";
    case TP_ECUDA: return "CUDA error";
    case TP_ENONFINITE: return "non-finite value";
    case TP_SETUP_FAILED: return "AMG setup failed";
    case TP_ESTATE: return "call order violated";
    case TP_NOT_CONVERGED: return "not converged";
    case TP_BREAKDOWN: return "Krylov breakdown";
    default: return "unknown status";
  }
}

const char* tp_last_error(void) { return g_last_error.c_str(); }

long long tp_kernel_launches(void) { return tp::launches_total(); }

int tp_create(tp_ctx** out, const tp_grid* grid, const tp_fluid* fluid, void* cuda_stream) {
  if (!out || !grid || !fluid) return TP_EINVAL;
  *out = nullptr;
  if (grid->nx < 1 || grid->ny < 1 || grid->nz < 1) return TP_EINVAL;
  long long N = (long long)grid->nx * grid->ny * grid->nz;
  if (N > 200000000LL) return TP_EINVAL;
  if (!(grid->dx > 0 && grid->dy > 0 && grid->dz > 0)) return TP_EINVAL;
  tp_ctx* c = nullptr;
  TP_API_BEGIN
  c = new tp_ctx();
  TP_CUDA_TRY(cudaGetDevice(&c->device));
  TP_CUDA_TRY(cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, c->device));
  if (cuda_stream) {
    c->s = static_cast<cudaStream_t>(cuda_stream);
  } else {
    // a blocking stream (ordered with the legacy default stream) owned here
    TP_CUDA_TRY(cudaStreamCreate(&c->s));
    owned_streams().push_back({c, c->s});
  }
  cudaStream_t s = c->s;
  c->grid = {grid->nx, grid->ny, grid->nz, grid->dx, grid->dy, grid->dz, grid->g};
  c->fluid = {fluid->rho0, fluid->c,     fluid->beta,    fluid->p0, fluid->T0,
              fluid->mu0,  fluid->T_mu0, fluid->mu_coef, fluid->cv, fluid->rho_r,
              fluid->cr,   fluid->kTf,   fluid->kT_mix, fluid->mu_law, fluid->api};
  if (fluid->mu_law != 0 && fluid->mu_law != 1) fail(TP_EINVAL, "mu_law must be 0 or 1");
  const int n = (int)N;
  c->N = n;
  long long nnzb = N + 2LL * ((long long)(grid->nx - 1) * grid->ny * grid->nz +
                              (long long)grid->nx * (grid->ny - 1) * grid->nz +
                              (long long)grid->nx * grid->ny * (grid->nz - 1));
  c->nnzb = (int)nnzb;
  tp::Pool& P = c->pool;
  c->rowptr = P.alloc<int>(n + 1);
  c->col = P.alloc<int>(nnzb);
  c->dpos = P.alloc<int>(n);
  tp::launch_pattern(c->grid, c->rowptr, c->col, c->dpos, s);
  for (double** f : {&c->Kx, &c->Ky, &c->Kz, &c->phi, &c->kTr, &c->kT, &c->p, &c->T, &c->pn,
                     &c->Tn, &c->rho, &c->lam, &c->lam_p, &c->lam_T, &c->Rm, &c->Re, &c->bp_s,
                     &c->bT_s, &c->tmpN, &c->io0, &c->io1, &c->io2, &c->io3})
    *f = P.alloc<double>(n);
  c->Tf3 = P.alloc<double>(3 * n);
  c->Tc3 = P.alloc<double>(3 * n);
  c->bval = P.alloc<double>(4 * nnzb);
  c->Sval = P.alloc<double>(nnzb);
  c->App = P.alloc<double>(nnzb);
  c->ApT = P.alloc<double>(nnzb);
  c->ATp = P.alloc<double>(nnzb);
  c->ATT = P.alloc<double>(nnzb);
  c->scales = P.alloc<double>(2);
  c->ones = P.alloc<double>(2);
  c->fscale = P.alloc<double>(2);
  const double one2[2] = {1.0, 1.0};
  TP_CUDA_TRY(cudaMemcpyAsync(c->ones, one2, sizeof(one2), cudaMemcpyHostToDevice, s));
  c->nparts = std::max(1, std::min(2 * c->num_sms, (n + 255) / 256));
  c->partials = P.alloc<double>(c->nparts + 1);
  TP_CUDA_TRY(cudaMallocHost(&c->host_est, 32 * sizeof(double)));
  for (int q = 0; q < 2; ++q)
    TP_CUDA_TRY(cudaEventCreateWithFlags(&c->ev_est[q], cudaEventDisableTiming));
  tp_default_opts(&c->opts);
  TP_CUDA_TRY(cudaStreamSynchronize(s));
  *out = c;
  return TP_OK;
  }
  catch (const Error& e) {
    g_last_error = e.what;
    cudaGetLastError();
    if (c) tp_destroy(c);
    return e.code;
  }
  catch (...) {
    if (c) tp_destroy(c);
    return TP_ENOMEM;
  }
}

void tp_destroy(tp_ctx* c) {
  if (!c) return;
  cudaStreamSynchronize(c->s);
  cudaStream_t own = nullptr;
  auto& v = owned_streams();
  for (size_t i = 0; i < v.size(); ++i)
    if (v[i].first == c) {
      own = v[i].second;
      v.erase(v.begin() + i);
      break;
    }
  delete c;
  if (own) cudaStreamDestroy(own);
}

int tp_get_sizes(const tp_ctx* c, int* N, int* nnzb) {
  if (!c) return TP_EINVAL;
  if (N) *N = c->N;
  if (nnzb) *nnzb = c->nnzb;
  return TP_OK;
}

int tp_set_fields(tp_ctx* c, const double* Kx, const double* Ky, const double* Kz,
                  const double* phi, const double* kTr, int ptr_is_device) {
  if (!c || !Kx || !Ky || !Kz || !phi || !kTr) return TP_EINVAL;
  TP_API_BEGIN
  cudaStream_t s = c->s;
  const size_t n = c->N;
  to_device(c->Kx, Kx, n, ptr_is_device, s);
  to_device(c->Ky, Ky, n, ptr_is_device, s);
  to_device(c->Kz, Kz, n, ptr_is_device, s);
  to_device(c->phi, phi, n, ptr_is_device, s);
  to_device(c->kTr, kTr, n, ptr_is_device, s);
  int* flags = reinterpret_cast<int*>(c->partials);
  TP_CUDA_TRY(cudaMemsetAsync(flags, 0, sizeof(int), s));
  k_check_fields<<<tp::grid_for(c->N), tp::kBlock, 0, s>>>(c->N, c->Kx, c->Ky, c->Kz, c->phi,
                                                           c->kTr, flags);
  TP_LAUNCH_CHECK();
  int f = read_flags(flags, s);
  if (f & 1) return TP_ENONFINITE;
  if (f & 2) return TP_EINVAL;
  tp::launch_mix_conductivity(c->N, c->phi, c->kTr, c->fluid, c->kT, s);
  tp::launch_face_trans(c->grid, c->Kx, c->Ky, c->Kz, c->kT, c->Tf3, c->Tc3, s);
  TP_CUDA_TRY(cudaStreamSynchronize(s));
  c->fields_set = true;
  c->assembled = false;
  c->built = false;
  return TP_OK;
  TP_API_END
}

int tp_set_wells(tp_ctx* c, const tp_well* w, int n) {
  if (!c || n < 0 || (n > 0 && !w)) return TP_EINVAL;
  TP_API_BEGIN
  // expand into completions grouped by cell (input order kept within a cell)
  struct Comp { int cell, kind, nl; double value, Tinj, U; int order; };
  std::vector<Comp> comps;
  for (int q = 0; q < n; ++q) {
    const tp_well& x = w[q];
    if (x.kind < 0 || x.kind > 3) return TP_EINVAL;
    if (x.i < 0 || x.i >= c->grid.nx || x.j < 0 || x.j >= c->grid.ny || x.k0 < 0 ||
        x.k1 < x.k0 || x.k1 >= c->grid.nz)
      return TP_EINVAL;
    if (!std::isfinite(x.value) || !std::isfinite(x.T_inj) || !std::isfinite(x.U))
      return TP_ENONFINITE;
    const int nl = x.k1 - x.k0 + 1;
    for (int k = x.k0; k <= x.k1; ++k) {
      int cell = x.i + c->grid.nx * (x.j + c->grid.ny * k);
      comps.push_back({cell, x.kind, nl, x.value, x.T_inj, x.U, (int)comps.size()});
    }
  }
  std::stable_sort(comps.begin(), comps.end(),
                   [](const Comp& a, const Comp& b) { return a.cell < b.cell; });
  std::vector<int> cells, off, kind, nl;
  std::vector<double> value, Tinj, U;
  for (size_t q = 0; q < comps.size(); ++q) {
    if (q == 0 || comps[q].cell != comps[q - 1].cell) {
      cells.push_back(comps[q].cell);
      off.push_back((int)q);
    }
    kind.push_back(comps[q].kind);
    nl.push_back(comps[q].nl);
    value.push_back(comps[q].value);
    Tinj.push_back(comps[q].Tinj);
    U.push_back(comps[q].U);
  }
  off.push_back((int)comps.size());
  cudaStream_t s = c->s;
  TP_CUDA_TRY(cudaStreamSynchronize(s));
  c->wpool.release();
  tp::WellsDev d;
  d.ncells = (int)cells.size();
  if (d.ncells > 0) {
    const size_t nc = comps.size();
    d.cell = c->wpool.alloc<int>(cells.size());
    d.off = c->wpool.alloc<int>(off.size());
    d.kind = c->wpool.alloc<int>(nc);
    d.nlayers = c->wpool.alloc<int>(nc);
    d.value = c->wpool.alloc<double>(nc);
    d.T_inj = c->wpool.alloc<double>(nc);
    d.U = c->wpool.alloc<double>(nc);
    TP_CUDA_TRY(cudaMemcpy(d.cell, cells.data(), cells.size() * sizeof(int), cudaMemcpyHostToDevice));
    TP_CUDA_TRY(cudaMemcpy(d.off, off.data(), off.size() * sizeof(int), cudaMemcpyHostToDevice));
    TP_CUDA_TRY(cudaMemcpy(d.kind, kind.data(), nc * sizeof(int), cudaMemcpyHostToDevice));
    TP_CUDA_TRY(cudaMemcpy(d.nlayers, nl.data(), nc * sizeof(int), cudaMemcpyHostToDevice));
    TP_CUDA_TRY(cudaMemcpy(d.value, value.data(), nc * sizeof(double), cudaMemcpyHostToDevice));
    TP_CUDA_TRY(cudaMemcpy(d.T_inj, Tinj.data(), nc * sizeof(double), cudaMemcpyHostToDevice));
    TP_CUDA_TRY(cudaMemcpy(d.U, U.data(), nc * sizeof(double), cudaMemcpyHostToDevice));
  }
  c->wells = d;
  c->assembled = false;
  c->built = false;
  return TP_OK;
  TP_API_END
}

int tp_assemble(tp_ctx* c, const double* p_k, const double* T_k, const double* p_n,
                const double* T_n, double dt, double* R_m, double* R_e, int ptr_is_device) {
  if (!c || !p_k || !T_k || !p_n || !T_n) return TP_EINVAL;
  if (!(dt > 0.0) || !std::isfinite(dt)) return TP_EINVAL;
  if (!c->fields_set) return TP_ESTATE;
  TP_API_BEGIN
  cudaStream_t s = c->s;
  const size_t n = c->N;
  to_device(c->p, p_k, n, ptr_is_device, s);
  to_device(c->T, T_k, n, ptr_is_device, s);
  to_device(c->pn, p_n, n, ptr_is_device, s);
  to_device(c->Tn, T_n, n, ptr_is_device, s);
  int st = tp::assemble_device(c, dt);
  if (st != TP_OK) return st;
  if (R_m) from_device(R_m, c->Rm, n, ptr_is_device, s);
  if (R_e) from_device(R_e, c->Re, n, ptr_is_device, s);
  TP_CUDA_TRY(cudaStreamSynchronize(s));
  c->built = false;
  return TP_OK;
  TP_API_END
}

int tp_build_preconditioner(tp_ctx* c, const tp_precond_opts* opts) {
  if (!c) return TP_EINVAL;
  if (!c->assembled) return TP_ESTATE;
  TP_API_BEGIN
  tp_precond_opts o;
  if (opts) o = *opts;
  else tp_default_opts(&o);
  check_opts(o);
  tp::build_device(c, o);
  return TP_OK;
  TP_API_END
}

int tp_newton_step(tp_ctx* c, const double* p_n, const double* T_n, double dt, double* p_out,
                   double* T_out, const tp_precond_opts* popts, const tp_newton_opts* nopts,
                   tp_newton_info* info, int ptr_is_device) {
  if (!c || !p_n || !T_n || !p_out || !T_out || !nopts) return TP_EINVAL;
  if (!(dt > 0.0) || !std::isfinite(dt)) return TP_EINVAL;
  if (nopts->max_newton < 1 || nopts->maxit < 1 || nopts->restart < 1 || nopts->restart > 200 ||
      !(nopts->rtol > 0.0))
    return TP_EINVAL;
  if (!c->fields_set) return TP_ESTATE;
  TP_API_BEGIN
  tp_precond_opts o;
  if (popts) o = *popts;
  else tp_default_opts(&o);
  check_opts(o);
  cudaStream_t s = c->s;
  const size_t n = c->N;
  to_device(c->pn, p_n, n, ptr_is_device, s);
  to_device(c->Tn, T_n, n, ptr_is_device, s);
  TP_CUDA_TRY(cudaMemcpyAsync(c->p, c->pn, n * sizeof(double), cudaMemcpyDeviceToDevice, s));
  TP_CUDA_TRY(cudaMemcpyAsync(c->T, c->Tn, n * sizeof(double), cudaMemcpyDeviceToDevice, s));
  int st = tp::newton_step(c, dt, o, *nopts, info);
  from_device(p_out, c->p, n, ptr_is_device, s);
  from_device(T_out, c->T, n, ptr_is_device, s);
  TP_CUDA_TRY(cudaStreamSynchronize(s));
  return st;
  TP_API_END
}

int tp_solve(tp_ctx* c, const double* b_p, const double* b_T, double* x_p, double* x_T,
             double rtol, int maxit, int restart, tp_solve_info* info, int ptr_is_device) {
  if (!c || !x_p || !x_T) return TP_EINVAL;
  if ((b_p == nullptr) != (b_T == nullptr)) return TP_EINVAL;
  if (!(rtol > 0.0) || maxit < 1 || restart < 1 || restart > 200) return TP_EINVAL;
  if (!c->built) return TP_ESTATE;
  TP_API_BEGIN
  cudaStream_t s = c->s;
  const size_t n = c->N;
  // right-hand side on the device: caller's, or -G(x_k)
  const double* bp;
  const double* bT;
  if (b_p) {
    to_device(c->io0, b_p, n, ptr_is_device, s);
    to_device(c->io1, b_T, n, ptr_is_device, s);
  } else {
    // b = -R
    tp::negated_residual(c);
  }
  bp = c->io0;
  bT = c->io1;
  int st = tp::fgmres_solve(c, bp, bT, c->io2, c->io3, rtol, maxit, restart, info);
  from_device(x_p, c->io2, n, ptr_is_device, s);
  from_device(x_T, c->io3, n, ptr_is_device, s);
  TP_CUDA_TRY(cudaStreamSynchronize(s));
  return st;
  TP_API_END
}

int tp_probe_enable(tp_ctx* c, int which) {
  if (!c || which < -1 || which > 3) return TP_EINVAL;
  TP_API_BEGIN
  if (which >= 0) c->probe.create();
  c->probe_which = which;
  c->probe.npairs = 0;
  c->probe.total_ms = 0.0;
  c->probe.total_bytes = 0.0;
  c->probe.launches = 0;
  c->built = false;  // the preconditioner graph must be recaptured
  return TP_OK;
  TP_API_END
}

int tp_probe_read(tp_ctx* c, double* total_ms, long long* launches, double* total_bytes,
                  int reset) {
  if (!c) return TP_EINVAL;
  if (total_ms) *total_ms = c->probe.total_ms;
  if (launches) *launches = c->probe.launches;
  if (total_bytes) *total_bytes = c->probe.total_bytes;
  if (reset) {
    c->probe.total_ms = 0.0;
    c->probe.total_bytes = 0.0;
    c->probe.launches = 0;
  }
  return TP_OK;
}

int tp_spmv(tp_ctx* c, const double* x_p, const double* x_T, double* y_p, double* y_T,
            int ptr_is_device) {
  if (!c || !x_p || !x_T || !y_p || !y_T) return TP_EINVAL;
  if (!c->assembled) return TP_ESTATE;
  TP_API_BEGIN
  cudaStream_t s = c->s;
  const size_t n = c->N;
  to_device(c->io0, x_p, n, ptr_is_device, s);
  to_device(c->io1, x_T, n, ptr_is_device, s);
  tp::launch_block_spmv(c->N, c->rowptr, c->col, c->bval, c->io0, c->io1, c->io2, c->io3, nullptr,
                        s);
  from_device(y_p, c->io2, n, ptr_is_device, s);
  from_device(y_T, c->io3, n, ptr_is_device, s);
  TP_CUDA_TRY(cudaStreamSynchronize(s));
  return TP_OK;
  TP_API_END
}

int tp_apply_preconditioner(tp_ctx* c, const double* v_p, const double* v_T, double* z_p,
                            double* z_T, int ptr_is_device) {
  if (!c || !v_p || !v_T || !z_p || !z_T) return TP_EINVAL;
  if (!c->built) return TP_ESTATE;
  TP_API_BEGIN
  cudaStream_t s = c->s;
  const size_t n = c->N;
  to_device(c->io0, v_p, n, ptr_is_device, s);
  to_device(c->io1, v_T, n, ptr_is_device, s);
  tp::precond_apply(c, c->io0, c->io1, c->ones, s);
  from_device(z_p, c->hpp->out, n, ptr_is_device, s);
  from_device(z_T, c->hS->out, n, ptr_is_device, s);
  TP_CUDA_TRY(cudaStreamSynchronize(s));
  return TP_OK;
  TP_API_END
}

int tp_export_system(tp_ctx* c, int* rowptr, int* col, double* val, double* schur_val,
                     double* scales) {
  if (!c) return TP_EINVAL;
  if (!c->assembled) return TP_ESTATE;
  TP_API_BEGIN
  cudaStream_t s = c->s;
  if (rowptr)
    TP_CUDA_TRY(cudaMemcpyAsync(rowptr, c->rowptr, (c->N + 1) * sizeof(int), cudaMemcpyDeviceToHost, s));
  if (col) TP_CUDA_TRY(cudaMemcpyAsync(col, c->col, c->nnzb * sizeof(int), cudaMemcpyDeviceToHost, s));
  if (val)
    TP_CUDA_TRY(cudaMemcpyAsync(val, c->bval, 4ll * c->nnzb * sizeof(double), cudaMemcpyDeviceToHost, s));
  if (schur_val)
    TP_CUDA_TRY(cudaMemcpyAsync(schur_val, c->Sval, c->nnzb * sizeof(double), cudaMemcpyDeviceToHost, s));
  if (scales) {
    if (!c->built) {
      tp::launch_extract_blocks(c->nnzb, c->bval, c->App, c->ApT, c->ATp, c->ATT, s);
      tp::launch_equation_scales(c->N, c->dpos, c->App, c->ATT, c->tmpN, c->partials, c->nparts,
                                 c->scales, s);
    }
    TP_CUDA_TRY(cudaMemcpyAsync(scales, c->scales, 2 * sizeof(double), cudaMemcpyDeviceToHost, s));
  }
  TP_CUDA_TRY(cudaStreamSynchronize(s));
  return TP_OK;
  TP_API_END
}

static int hierarchy_info(tp::Hierarchy* h, int* nlevels, int* n, int* nnz, int max_levels) {
  if (!h) return TP_ESTATE;
  if (nlevels) *nlevels = (int)h->L.size();
  for (int l = 0; l < (int)h->L.size() && l < max_levels; ++l) {
    if (n) n[l] = h->L[l].A.n;
    if (nnz) nnz[l] = h->L[l].A.nnz;
  }
  return TP_OK;
}

static int level_storage(tp::Hierarchy* h, int level, int* format, long long* stored) {
  if (!h) return TP_ESTATE;
  if (level < 0 || level >= (int)h->L.size()) return TP_EINVAL;
  const tp::Level& v = h->L[level];
  int f = 0;
  long long e = v.A.nnz;
  if (v.sell_slices > 0) {
    f = 2;
    e = v.sell_entries;
  } else if (v.ell_w > 0) {
    f = v.ell_nxy > 0 ? 3 : 1;
    e = (long long)v.ell_w * v.A.n;
  }
  if (format) *format = f;
  if (stored) *stored = e;
  return TP_OK;
}

static int export_level(tp::Hierarchy* h, cudaStream_t s, int level, int* rowptr, int* col,
                        double* val, signed char* cf, signed char* strong, int* P_nnz,
                        int* P_rowptr, int* P_col, double* P_val) {
  if (!h) return TP_ESTATE;
  if (level < 0 || level >= (int)h->L.size()) return TP_EINVAL;
  TP_API_BEGIN
  const tp::Level& v = h->L[level];
  const tp::DevCSR& A = v.A;
  if (rowptr) TP_CUDA_TRY(cudaMemcpyAsync(rowptr, A.rowptr, (A.n + 1) * sizeof(int), cudaMemcpyDeviceToHost, s));
  if (col) TP_CUDA_TRY(cudaMemcpyAsync(col, A.col, A.nnz * sizeof(int), cudaMemcpyDeviceToHost, s));
  if (val) TP_CUDA_TRY(cudaMemcpyAsync(val, A.val, A.nnz * sizeof(double), cudaMemcpyDeviceToHost, s));
  if (cf) {
    if (v.cf) TP_CUDA_TRY(cudaMemcpyAsync(cf, v.cf, A.n, cudaMemcpyDeviceToHost, s));
    else std::memset(cf, 0, A.n);
  }
  if (strong) {
    if (v.strong) TP_CUDA_TRY(cudaMemcpyAsync(strong, v.strong, A.nnz, cudaMemcpyDeviceToHost, s));
    else std::memset(strong, 0, A.nnz);
  }
  if (P_nnz) *P_nnz = v.P.nnz;
  if (v.P.nnz > 0) {
    if (P_rowptr) TP_CUDA_TRY(cudaMemcpyAsync(P_rowptr, v.P.rowptr, (v.P.n + 1) * sizeof(int), cudaMemcpyDeviceToHost, s));
    if (P_col) TP_CUDA_TRY(cudaMemcpyAsync(P_col, v.P.col, v.P.nnz * sizeof(int), cudaMemcpyDeviceToHost, s));
    if (P_val) TP_CUDA_TRY(cudaMemcpyAsync(P_val, v.P.val, v.P.nnz * sizeof(double), cudaMemcpyDeviceToHost, s));
  }
  TP_CUDA_TRY(cudaStreamSynchronize(s));
  return TP_OK;
  TP_API_END
}

int tp_setup_timings(tp_ctx* c, int which, double* ms) {
  if (!c || !ms || (which != 0 && which != 1)) return TP_EINVAL;
  if (!c->built) return TP_ESTATE;
  tp::Hierarchy* h = which == 0 ? c->hpp.get() : c->hS.get();
  for (int k = 0; k < 5; ++k) ms[k] = h->phase_ms[k];
  return TP_OK;
}

int tp_level_storage(tp_ctx* c, int which, int level, int* format, long long* stored) {
  if (!c || (which != 0 && which != 1)) return TP_EINVAL;
  return level_storage(which == 0 ? c->hpp.get() : c->hS.get(), level, format, stored);
}

int tp_hierarchy_info(tp_ctx* c, int which, int* nlevels, int* n, int* nnz, int max_levels) {
  if (!c || (which != 0 && which != 1)) return TP_EINVAL;
  if (!c->built) return TP_ESTATE;
  return hierarchy_info(which == 0 ? c->hpp.get() : c->hS.get(), nlevels, n, nnz, max_levels);
}

int tp_vcycle_measure(tp_ctx* c, int which, int reps, double* ms, double* bytes,
                      double* opc) {
  if (!c || (which != 0 && which != 1) || reps < 1) return TP_EINVAL;
  if (!c->built) return TP_ESTATE;
  TP_API_BEGIN
  tp::Hierarchy* h = which == 0 ? c->hpp.get() : c->hS.get();
  cudaStream_t s = c->s;
  tp::Probe* saved = h->probe;
  h->probe = nullptr;
  k_fill<<<tp::grid_for(h->n0), tp::kBlock, 0, s>>>(h->in, h->n0, 1.0);
  TP_LAUNCH_CHECK();
  // one V-cycle captured as a graph (as inside the preconditioner) and
  // replayed reps times between two events
  cudaGraph_t g = nullptr;
  cudaGraphExec_t ge = nullptr;
  tp::g_capturing = true;
  cudaError_t ce = cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal);
  if (ce == cudaSuccess) {
    try {
      h->vcycle(s);
    } catch (...) {
      tp::g_capturing = false;
      cudaStreamEndCapture(s, &g);
      if (g) cudaGraphDestroy(g);
      h->probe = saved;
      throw;
    }
    ce = cudaStreamEndCapture(s, &g);
  }
  tp::g_capturing = false;
  h->probe = saved;
  TP_CUDA_TRY(ce);
  size_t nodes = 0;
  long long kernels = 0;
  TP_CUDA_TRY(cudaGraphGetNodes(g, nullptr, &nodes));
  std::vector<cudaGraphNode_t> list(nodes);
  if (nodes) TP_CUDA_TRY(cudaGraphGetNodes(g, list.data(), &nodes));
  for (cudaGraphNode_t nd : list) {
    cudaGraphNodeType ty;
    TP_CUDA_TRY(cudaGraphNodeGetType(nd, &ty));
    if (ty == cudaGraphNodeTypeKernel) ++kernels;
  }
  TP_CUDA_TRY(cudaGraphInstantiate(&ge, g, 0));
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  float t = 0.f;
  cudaError_t err = cudaEventCreate(&e0);
  if (err == cudaSuccess) err = cudaEventCreate(&e1);
  if (err == cudaSuccess) err = cudaGraphLaunch(ge, s);  // warm-up
  if (err == cudaSuccess) tp::count_launch(kernels);
  if (err == cudaSuccess) err = cudaEventRecord(e0, s);
  for (int r = 0; r < reps && err == cudaSuccess; ++r) {
    err = cudaGraphLaunch(ge, s);
    if (err == cudaSuccess) tp::count_launch(kernels);
  }
  if (err == cudaSuccess) err = cudaEventRecord(e1, s);
  if (err == cudaSuccess) err = cudaEventSynchronize(e1);
  if (err == cudaSuccess) err = cudaEventElapsedTime(&t, e0, e1);
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  cudaGraphExecDestroy(ge);
  cudaGraphDestroy(g);
  TP_CUDA_TRY(err);
  if (ms) *ms = (double)t / reps;
  if (bytes) *bytes = h->vcycle_bytes();
  if (opc) *opc = h->operator_complexity();
  return TP_OK;
  TP_API_END
}

int tp_export_level(tp_ctx* c, int which, int level, int* rowptr, int* col, double* val,
                    signed char* cf, signed char* strong, int* P_nnz, int* P_rowptr, int* P_col,
                    double* P_val) {
  if (!c || (which != 0 && which != 1)) return TP_EINVAL;
  if (!c->built) return TP_ESTATE;
  return export_level(which == 0 ? c->hpp.get() : c->hS.get(), c->s, level, rowptr, col, val, cf,
                      strong, P_nnz, P_rowptr, P_col, P_val);
}

int tp_mlp_create(tp_mlp** out, const double* params, void* cuda_stream) {
  if (!out || !params) return TP_EINVAL;
  *out = nullptr;
  tp_mlp* a = nullptr;
  TP_API_BEGIN
  a = new tp_mlp();
  if (cuda_stream) {
    a->s = static_cast<cudaStream_t>(cuda_stream);
  } else {
    TP_CUDA_TRY(cudaStreamCreate(&a->s));
    a->own_stream = true;
  }
  tp::MlpDev& m = a->m;
  m.params = a->pool.alloc<float>(tp::kMlpParams);
  m.adam_m = a->pool.alloc<float>(tp::kMlpParams);
  m.adam_v = a->pool.alloc<float>(tp::kMlpParams);
  m.grad = a->pool.alloc<float>(tp::kMlpPartial);
  m.W1 = a->pool.alloc<__nv_bfloat16>(tp::kMlpHidden * tp::kMlpInPad);
  m.W2 = a->pool.alloc<__nv_bfloat16>(tp::kMlpHidden * tp::kMlpHidden);
  m.W3 = a->pool.alloc<__nv_bfloat16>(tp::kMlpOut * tp::kMlpHidden);
  m.W2T = a->pool.alloc<__nv_bfloat16>(tp::kMlpHidden * tp::kMlpHidden);
  m.W3T = a->pool.alloc<__nv_bfloat16>(tp::kMlpHidden * 16);
  m.err = a->pool.alloc<int>(1);
  m.Wtc = a->pool.alloc<__nv_bfloat16>(tp::kMlpTcWeights);
  TP_CUDA_TRY(cudaMallocHost(&a->host, sizeof(double) * tp::kMlpPartial));
  *out = a;
  int st = tp_mlp_set_params(a, params);
  if (st != TP_OK) {
    *out = nullptr;
    delete a;
  }
  return st;
  }
  catch (const Error& e) {
    g_last_error = e.what;
    cudaGetLastError();
    delete a;
    return e.code;
  }
  catch (...) {
    delete a;
    return TP_ECUDA;
  }
}

void tp_mlp_destroy(tp_mlp* a) {
  if (!a) return;
  cudaStreamSynchronize(a->s);
  delete a;
}

int tp_mlp_set_params(tp_mlp* a, const double* params) {
  if (!a || !params) return TP_EINVAL;
  TP_API_BEGIN
  std::vector<float> f(tp::kMlpParams);
  for (int k = 0; k < tp::kMlpParams; ++k) {
    if (!std::isfinite(params[k])) return TP_ENONFINITE;
    f[k] = (float)params[k];
  }
  TP_CUDA_TRY(cudaMemcpyAsync(a->m.params, f.data(), sizeof(float) * tp::kMlpParams,
                              cudaMemcpyHostToDevice, a->s));
  TP_CUDA_TRY(cudaMemsetAsync(a->m.adam_m, 0, sizeof(float) * tp::kMlpParams, a->s));
  TP_CUDA_TRY(cudaMemsetAsync(a->m.adam_v, 0, sizeof(float) * tp::kMlpParams, a->s));
  a->m.step = 0;
  tp::mlp_pack(a->m, a->s);
  TP_CUDA_TRY(cudaStreamSynchronize(a->s));
  return TP_OK;
  TP_API_END
}

int tp_mlp_get_params(tp_mlp* a, double* params) {
  if (!a || !params) return TP_EINVAL;
  TP_API_BEGIN
  std::vector<float> f(tp::kMlpParams);
  TP_CUDA_TRY(cudaMemcpyAsync(f.data(), a->m.params, sizeof(float) * tp::kMlpParams,
                              cudaMemcpyDeviceToHost, a->s));
  TP_CUDA_TRY(cudaStreamSynchronize(a->s));
  for (int k = 0; k < tp::kMlpParams; ++k) params[k] = f[k];
  return TP_OK;
  TP_API_END
}

int tp_mlp_forward(tp_mlp* a, int n, const float* X, float* O, int ptr_is_device) {
  if (!a || n < 0 || (n > 0 && (!X || !O))) return TP_EINVAL;
  TP_API_BEGIN
  if (n == 0) return TP_OK;
  const float* Xd = X;
  float* Od = O;
  if (!ptr_is_device) {
    a->ensure(n);
    TP_CUDA_TRY(cudaMemcpyAsync(a->X, X, sizeof(float) * n * tp::kMlpIn, cudaMemcpyHostToDevice, a->s));
    Xd = a->X;
    Od = a->O;
  }
  tp::mlp_forward(a->m, n, Xd, Od, a->s);
  if (!ptr_is_device)
    TP_CUDA_TRY(cudaMemcpyAsync(O, a->O, sizeof(float) * n * tp::kMlpOut, cudaMemcpyDeviceToHost, a->s));
  TP_CUDA_TRY(cudaStreamSynchronize(a->s));
  return TP_OK;
  TP_API_END
}

static int mlp_grad_common(tp_mlp* a, int B, const float* X, const int* slot, const double* St,
                           const double* Sd, const double* tgt, int ptr_is_device) {
  a->ensure(B);
  if (ptr_is_device) {
    TP_CUDA_TRY(cudaMemcpyAsync(a->X, X, sizeof(float) * B * tp::kMlpIn, cudaMemcpyDeviceToDevice, a->s));
  } else {
    TP_CUDA_TRY(cudaMemcpyAsync(a->X, X, sizeof(float) * B * tp::kMlpIn, cudaMemcpyHostToDevice, a->s));
  }
  cudaMemcpyKind k = ptr_is_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
  TP_CUDA_TRY(cudaMemcpyAsync(a->slot, slot, sizeof(int) * B, k, a->s));
  TP_CUDA_TRY(cudaMemcpyAsync(a->St, St, sizeof(double) * B, k, a->s));
  TP_CUDA_TRY(cudaMemcpyAsync(a->Sd, Sd, sizeof(double) * B, k, a->s));
  TP_CUDA_TRY(cudaMemcpyAsync(a->tgt, tgt, sizeof(double) * B, k, a->s));
  tp::mlp_gradient(a->m, B, a->X, a->slot, a->St, a->Sd, a->tgt, a->partials, a->m.grad, a->s);
  return TP_OK;
}

int tp_mlp_gradient(tp_mlp* a, int B, const float* X, const int* slot, const double* St,
                    const double* Sd, const double* target, double* grad, double* loss,
                    int ptr_is_device) {
  if (!a || B < 1 || !X || !slot || !St || !Sd || !target) return TP_EINVAL;
  TP_API_BEGIN
  mlp_grad_common(a, B, X, slot, St, Sd, target, ptr_is_device);
  std::vector<float> f(tp::kMlpPartial);
  TP_CUDA_TRY(cudaMemcpyAsync(f.data(), a->m.grad, sizeof(float) * tp::kMlpPartial,
                              cudaMemcpyDeviceToHost, a->s));
  TP_CUDA_TRY(cudaStreamSynchronize(a->s));
  if (grad)
    for (int k = 0; k < tp::kMlpParams; ++k) grad[k] = f[k];
  if (loss) *loss = f[tp::kMlpParams];
  return TP_OK;
  TP_API_END
}

int tp_mlp_train_step(tp_mlp* a, int B, const float* X, const int* slot, const double* St,
                      const double* Sd, const double* target, double lr, double* loss,
                      int ptr_is_device) {
  if (!a || B < 1 || !X || !slot || !St || !Sd || !target || !(lr > 0.0)) return TP_EINVAL;
  TP_API_BEGIN
  mlp_grad_common(a, B, X, slot, St, Sd, target, ptr_is_device);
  tp::mlp_adam(a->m, a->m.grad, (float)lr, a->s);
  float l = 0.f;
  TP_CUDA_TRY(cudaMemcpyAsync(&l, a->m.grad + tp::kMlpParams, sizeof(float), cudaMemcpyDeviceToHost, a->s));
  TP_CUDA_TRY(cudaStreamSynchronize(a->s));
  if (loss) *loss = l;
  return TP_OK;
  TP_API_END
}

int tp_learned_features(tp_ctx* c, float* X, int ptr_is_device) {
  if (!c || !X) return TP_EINVAL;
  if (!c->assembled) return TP_ESTATE;
  TP_API_BEGIN
  tp::learned_features(c);
  TP_CUDA_TRY(cudaMemcpyAsync(X, c->feat, sizeof(float) * (size_t)c->N * tp::kMlpIn,
                              ptr_is_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, c->s));
  TP_CUDA_TRY(cudaStreamSynchronize(c->s));
  return TP_OK;
  TP_API_END
}

int tp_set_schur_model(tp_ctx* c, tp_mlp* model) {
  if (!c) return TP_EINVAL;
  c->model = model;
  c->built = false;
  return TP_OK;
}

int tp_learned_status(tp_ctx* c, int* fallback_rows, int* global_fallback) {
  if (!c) return TP_EINVAL;
  if (fallback_rows) *fallback_rows = c->learned_fallback_rows;
  if (global_fallback) *global_fallback = c->learned_global_fallback ? 1 : 0;
  return TP_OK;
}

int tp_probe_schur_columns(tp_ctx* c, const int* cols, int ncols, double rtol, int* entry,
                           double* value, int* iters) {
  if (!c || !cols || ncols < 0 || !entry || !value || !(rtol > 0.0)) return TP_EINVAL;
  if (!c->built) return TP_ESTATE;
  TP_API_BEGIN
  int* d_entry = reinterpret_cast<int*>(c->io2);
  double* d_val = c->io3;
  int total = 0, status = TP_OK;
  for (int q = 0; q < ncols; ++q) {
    const int j = cols[q];
    if (j < 0 || j >= c->N) return TP_EINVAL;
    const int its = tp::probe_schur_column(c, j, rtol, 500, d_entry, d_val);
    if (its < 0) status = TP_NOT_CONVERGED;
    total += its < 0 ? -its : its;
    TP_CUDA_TRY(cudaMemcpyAsync(entry + 7 * q, d_entry, 7 * sizeof(int), cudaMemcpyDeviceToHost, c->s));
    TP_CUDA_TRY(cudaMemcpyAsync(value + 7 * q, d_val, 7 * sizeof(double), cudaMemcpyDeviceToHost, c->s));
  }
  TP_CUDA_TRY(cudaStreamSynchronize(c->s));
  if (iters) *iters = total;
  return status;
  TP_API_END
}

int tp_amg_create(tp_amg** out, int n, int nnz, const int* rowptr, const int* col,
                  const double* val, const tp_precond_opts* opts, void* cuda_stream,
                  int ptr_is_device) {
  if (!out || n < 1 || nnz < n || !rowptr || !col || !val) return TP_EINVAL;
  *out = nullptr;
  tp_amg* a = nullptr;
  TP_API_BEGIN
  tp_precond_opts o;
  if (opts) o = *opts;
  else tp_default_opts(&o);
  check_opts(o);
  a = new tp_amg();
  if (cuda_stream) {
    a->s = static_cast<cudaStream_t>(cuda_stream);
  } else {
    TP_CUDA_TRY(cudaStreamCreate(&a->s));
    a->own_stream = true;
  }
  cudaStream_t s = a->s;
  // validate the pattern on the host side when it is host memory
  if (!ptr_is_device) {
    if (rowptr[0] != 0 || rowptr[n] != nnz) {
      delete a;
      return TP_EINVAL;
    }
    for (int i = 0; i < n; ++i) {
      if (rowptr[i + 1] < rowptr[i]) { delete a; return TP_EINVAL; }
      for (int e = rowptr[i]; e < rowptr[i + 1]; ++e) {
        if (col[e] < 0 || col[e] >= n || (e > rowptr[i] && col[e] <= col[e - 1]) ||
            !std::isfinite(val[e])) {
          delete a;
          return TP_EINVAL;
        }
      }
    }
  }
  a->A.n = a->A.m = n;
  a->A.nnz = nnz;
  a->A.rowptr = a->pool.alloc<int>(n + 1);
  a->A.col = a->pool.alloc<int>(nnz);
  a->A.val = a->pool.alloc<double>(nnz);
  cudaMemcpyKind k = ptr_is_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
  TP_CUDA_TRY(cudaMemcpyAsync(a->A.rowptr, rowptr, (n + 1) * sizeof(int), k, s));
  TP_CUDA_TRY(cudaMemcpyAsync(a->A.col, col, nnz * sizeof(int), k, s));
  TP_CUDA_TRY(cudaMemcpyAsync(a->A.val, val, nnz * sizeof(double), k, s));
  a->h.reset(new tp::Hierarchy());
  a->h->setup(a->A, amg_opts(o), s);
  *out = a;
  return TP_OK;
  }
  catch (const Error& e) {
    g_last_error = e.what;
    cudaGetLastError();
    delete a;
    return e.code;
  }
  catch (...) {
    delete a;
    return TP_ECUDA;
  }
}

void tp_amg_destroy(tp_amg* a) {
  if (!a) return;
  cudaStreamSynchronize(a->s);
  delete a;
}

int tp_amg_vcycle(tp_amg* a, const double* b, double* x, int ptr_is_device) {
  if (!a || !b || !x) return TP_EINVAL;
  TP_API_BEGIN
  const size_t n = a->A.n;
  to_device(a->h->in, b, n, ptr_is_device, a->s);
  a->h->vcycle(a->s);
  from_device(x, a->h->out, n, ptr_is_device, a->s);
  TP_CUDA_TRY(cudaStreamSynchronize(a->s));
  return TP_OK;
  TP_API_END
}

int tp_amg_info(tp_amg* a, int* nlevels, int* n, int* nnz, int max_levels) {
  if (!a) return TP_EINVAL;
  return hierarchy_info(a->h.get(), nlevels, n, nnz, max_levels);
}

int tp_amg_level_storage(tp_amg* a, int level, int* format, long long* stored) {
  if (!a) return TP_EINVAL;
  return level_storage(a->h.get(), level, format, stored);
}

int tp_amg_export_level(tp_amg* a, int level, int* rowptr, int* col, double* val,
                        signed char* cf, signed char* strong, int* P_nnz, int* P_rowptr,
                        int* P_col, double* P_val) {
  if (!a) return TP_EINVAL;
  return export_level(a->h.get(), a->s, level, rowptr, col, val, cf, strong, P_nnz, P_rowptr,
                      P_col, P_val);
}

}  // extern "C"


// ------------------------------------------------------------ device steps
namespace tp {

void learned_schur_values(tp_ctx* c);

int assemble_device(tp_ctx* c, double dt) {
  cudaStream_t s = c->s;
  const long long n = c->N;
  int* flags = reinterpret_cast<int*>(c->partials);
  TP_CUDA_TRY(cudaMemsetAsync(flags, 0, sizeof(int), s));
  for (const double* a : {c->p, c->T, c->pn, c->Tn}) {
    k_check_finite<<<grid_for(n), kBlock, 0, s>>>(n, a, flags);
    TP_LAUNCH_CHECK();
  }
  if (read_flags(flags, s)) return TP_ENONFINITE;
  launch_cell_props(c->N, c->p, c->T, c->fluid, c->rho, c->lam, c->lam_p, c->lam_T, s);
  launch_assemble(c->grid, c->fluid, c->rowptr, c->dpos, c->Tf3, c->Tc3, c->phi, c->p, c->T,
                  c->pn, c->Tn, c->rho, c->lam, c->lam_p, c->lam_T, dt, c->bval, c->Sval, c->Rm,
                  c->Re, s);
  launch_wells(c->grid, c->fluid, c->wells, c->dpos, c->Kx, c->Ky, c->p, c->T, c->rho, c->lam,
               c->lam_p, c->lam_T, c->bval, c->Sval, c->Rm, c->Re, s);
  TP_CUDA_TRY(cudaMemsetAsync(flags, 0, sizeof(int), s));
  k_check_finite<<<grid_for(4ll * c->nnzb), kBlock, 0, s>>>(4ll * c->nnzb, c->bval, flags);
  TP_LAUNCH_CHECK();
  if (read_flags(flags, s)) return TP_ENONFINITE;
  c->assembled = true;
  c->dt_last = dt;
  return TP_OK;
}

// features -> MLP -> corrected S~ with the per-row guard; more than a quarter
// of the rows falling back switches the whole matrix back to plain S~
void learned_features(tp_ctx* c) {
  cudaStream_t s = c->s;
  if (!c->feat) {
    c->feat = c->lpool.alloc<float>((size_t)c->N * kMlpIn);
    c->mlp_out = c->lpool.alloc<float>((size_t)c->N * kMlpOut);
    c->S_learned = c->lpool.alloc<double>(c->nnzb);
    c->nbad = c->lpool.alloc<int>(1);
  }
  launch_extract_blocks(c->nnzb, c->bval, c->App, c->ApT, c->ATp, c->ATT, s);
  launch_equation_scales(c->N, c->dpos, c->App, c->ATT, c->tmpN, c->partials, c->nparts,
                         c->scales, s);
  launch_features(c->grid, c->fluid, c->dpos, c->Tf3, c->Tc3, c->phi, c->p, c->T,
                  c->rho, c->lam, c->lam_p, c->lam_T, c->bval, c->Sval, c->scales, c->dt_last,
                  c->feat, s);
}

void learned_schur_values(tp_ctx* c) {
  if (!c->model) fail(TP_ESTATE, "schur = 1 needs a model (tp_set_schur_model)");
  cudaStream_t s = c->s;
  learned_features(c);
  mlp_forward(c->model->m, c->N, c->feat, c->mlp_out, s);
  TP_CUDA_TRY(cudaMemsetAsync(c->nbad, 0, sizeof(int), s));
  learned_schur(c->N, c->grid.nx, c->grid.ny, c->rowptr, c->col, c->dpos, c->Sval, c->mlp_out,
                c->S_learned, c->nbad, s);
  c->learned_fallback_rows = read_flags(c->nbad, s);
  c->learned_global_fallback = 4ll * c->learned_fallback_rows > c->N;
}

namespace {
// b_e = (A_pT)_e / (A_pp)_kk over row k (one correctly rounded division)
__global__ void k_scale_by_diag(int N, const int* __restrict__ rowptr,
                                const int* __restrict__ dpos, const double* __restrict__ App,
                                const double* __restrict__ ApT, double* __restrict__ B) {
  int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= N) return;
  const double d = App[dpos[k]];
  for (int e = rowptr[k]; e < rowptr[k + 1]; ++e) B[e] = __ddiv_rn(ApT[e], d);
}

// S = A_TT - C on C's pattern (A_TT's 7-point pattern is contained in it)
__global__ void k_schur_diag_merge(int N, const int* __restrict__ Crp, const int* __restrict__ Ccol,
                                   const double* __restrict__ Cval, const int* __restrict__ rowptr,
                                   const int* __restrict__ col, const double* __restrict__ ATT,
                                   double* __restrict__ S) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= N) return;
  int q = rowptr[i];
  const int q1 = rowptr[i + 1];
  for (int e = Crp[i]; e < Crp[i + 1]; ++e) {
    const int j = Ccol[e];
    while (q < q1 && col[q] < j) ++q;
    S[e] = (q < q1 && col[q] == j) ? __dsub_rn(ATT[q], Cval[e]) : -Cval[e];
  }
}
}  // namespace

// S~_diag = A_TT - A_Tp diag(A_pp)^{-1} A_pT (Sec. 3.3) on the 25-point
// product pattern; `symbolic` rebuilds the pattern, else only the values
void schur_diag_values(tp_ctx* c, bool symbolic) {
  cudaStream_t s = c->s;
  const int N = c->N;
  if (symbolic) {
    c->dpool.release();
    c->dscratch.release();
    c->Bd = c->dpool.alloc<double>(c->nnzb);
  }
  k_scale_by_diag<<<grid_for(N), kBlock, 0, s>>>(N, c->rowptr, c->dpos, c->App, c->ApT, c->Bd);
  TP_LAUNCH_CHECK();
  DevCSR ATp{N, N, c->nnzb, c->rowptr, c->col, c->ATp, nullptr};
  DevCSR B{N, N, c->nnzb, c->rowptr, c->col, c->Bd, nullptr};
  if (symbolic) {
    c->Cd = csr_product(ATp, B, c->dpool, c->dscratch, s);
    c->Sd = c->Cd;
    c->Sd.val = c->dpool.alloc<double>(c->Cd.nnz);
  } else {
    csr_product_numeric(ATp, B, c->Cd, s);
  }
  k_schur_diag_merge<<<grid_for(N), kBlock, 0, s>>>(N, c->Cd.rowptr, c->Cd.col, c->Cd.val,
                                                    c->rowptr, c->col, c->ATT, c->Sd.val);
  TP_LAUNCH_CHECK();
}

void build_device(tp_ctx* c, const tp_precond_opts& o) {
  cudaStream_t s = c->s;
  if (c->pc_graph) {
    cudaGraphExecDestroy(c->pc_graph);
    c->pc_graph = nullptr;
  }
  if (c->pc_graph_tmpl) {
    cudaGraphDestroy(c->pc_graph_tmpl);
    c->pc_graph_tmpl = nullptr;
  }
  c->probe_nodes.clear();
  c->probe_set = 0;
  c->built = false;
  launch_extract_blocks(c->nnzb, c->bval, c->App, c->ApT, c->ATp, c->ATT, s);
  launch_equation_scales(c->N, c->dpos, c->App, c->ATT, c->tmpN, c->partials, c->nparts,
                         c->scales, s);
  c->S_active = (o.schur == 2) ? c->ATT : c->Sval;
  if (o.schur == 1) {
    learned_schur_values(c);
    c->S_active = c->learned_global_fallback ? c->Sval : c->S_learned;
  }
  DevCSR App{c->N, c->N, c->nnzb, c->rowptr, c->col, c->App, nullptr};
  DevCSR S{c->N, c->N, c->nnzb, c->rowptr, c->col, c->S_active, nullptr};
  if (o.schur == 3) {
    schur_diag_values(c, true);
    S = c->Sd;
    c->S_active = c->Sd.val;
  }
  c->opts = o;
  // the hierarchies are reused: their memory pools keep their chunks
  if (!c->hpp) c->hpp.reset(new Hierarchy());
  if (!c->hS) c->hS.reset(new Hierarchy());
  AmgOpts ao = amg_opts(o);
  // A_pp (and S~ except S~_diag, whose pattern has 25 points) is the grid's
  // 7-point operator: its finest ELL copy is stored by grid direction
  ao.grid_nx = c->grid.nx;
  ao.grid_ny = c->grid.ny;
  ao.grid_nz = c->grid.nz;
  AmgOpts aS = ao;
  if (o.schur == 3) aS.grid_nx = aS.grid_ny = aS.grid_nz = 0;
  if (o.interp_S >= 0) aS.interp = o.interp_S;
  if (o.max_levels_S > 0) aS.max_levels = o.max_levels_S;
  if (o.nu_S > 0) aS.nu_pre = aS.nu_post = o.nu_S;
  if (o.smoother_S == 2) {
    // vertical-line steps on the finest level (grids with one layer keep
    // l1-Jacobi there), l1-Jacobi on the coarser levels
    aS.smoother = 0;
    if (c->grid.nz > 1) {
      aS.line_nxy = c->grid.nx * c->grid.ny;
      aS.line_nz = c->grid.nz;
      aS.nu_line = o.nu_line;
    }
  } else if (o.smoother_S >= 0) {
    aS.smoother = o.smoother_S;
  }
  // The two hierarchies are independent: S~'s is set up by a second host
  // thread on a second stream while this thread sets up A_pp's (both setups
  // are chains of small kernels with host round trips, so they overlap).
  if (!c->s2) {
    TP_CUDA_TRY(cudaStreamCreateWithFlags(&c->s2, cudaStreamNonBlocking));
    TP_CUDA_TRY(cudaEventCreateWithFlags(&c->ev_fork, cudaEventDisableTiming));
    TP_CUDA_TRY(cudaEventCreateWithFlags(&c->ev_join, cudaEventDisableTiming));
  }
  TP_CUDA_TRY(cudaEventRecord(c->ev_fork, s));
  TP_CUDA_TRY(cudaStreamWaitEvent(c->s2, c->ev_fork, 0));
  Error terr{TP_OK, ""};
  bool tfail = false;
  std::thread th([&]() {
    try {
      TP_CUDA_TRY(cudaSetDevice(c->device));
      c->hS->setup(S, aS, c->s2);
    } catch (const Error& e) {
      terr = e;
      tfail = true;
    } catch (...) {
      terr = Error{TP_ECUDA, "Schur hierarchy setup failed"};
      tfail = true;
    }
  });
  try {
    c->hpp->setup(App, ao, s);
  } catch (...) {
    th.join();
    throw;
  }
  th.join();
  if (tfail) throw terr;
  TP_CUDA_TRY(cudaEventRecord(c->ev_join, c->s2));
  TP_CUDA_TRY(cudaStreamWaitEvent(s, c->ev_join, 0));
  c->hpp->probe = (c->probe_which == 0 || c->probe_which == 3) ? &c->probe : nullptr;
  c->hpp->probe_level = c->probe_which == 3 ? 1 : 0;
  c->hS->probe = c->probe_which == 1 ? &c->probe : nullptr;
  c->hS->probe_level = 0;
  if (o.use_graphs) {
    cudaGraph_t graph = nullptr;
    TP_CUDA_TRY(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
    g_capturing = true;
    try {
      precond_record(c, s);
    } catch (...) {
      g_capturing = false;
      cudaStreamEndCapture(s, &graph);
      if (graph) cudaGraphDestroy(graph);
      throw;
    }
    g_capturing = false;
    TP_CUDA_TRY(cudaStreamEndCapture(s, &graph));
    size_t nodes = 0;
    TP_CUDA_TRY(cudaGraphGetNodes(graph, nullptr, &nodes));
    std::vector<cudaGraphNode_t> list(nodes);
    if (nodes) TP_CUDA_TRY(cudaGraphGetNodes(graph, list.data(), &nodes));
    long long kernels = 0;
    for (cudaGraphNode_t nd : list) {
      cudaGraphNodeType ty;
      TP_CUDA_TRY(cudaGraphNodeGetType(nd, &ty));
      if (ty == cudaGraphNodeTypeKernel) ++kernels;
      if (ty == cudaGraphNodeTypeEventRecord) {
        cudaEvent_t ev = nullptr;
        TP_CUDA_TRY(cudaGraphEventRecordNodeGetEvent(nd, &ev));
        for (int k = 0; k < 2 * tp::Probe::kMaxPairs; ++k)
          if (c->probe.created && c->probe.ev[0][k] == ev) c->probe_nodes.push_back({nd, k});
      }
    }
    c->pc_graph_kernels = kernels;
    cudaError_t e = cudaGraphInstantiate(&c->pc_graph, graph, 0);
    if (e != cudaSuccess) {
      cudaGraphDestroy(graph);
      c->pc_graph = nullptr;
      c->probe_nodes.clear();
      fail(TP_ECUDA, std::string("graph instantiate: ") + cudaGetErrorString(e));
    }
    c->pc_graph_tmpl = graph;
  }
  TP_CUDA_TRY(cudaStreamSynchronize(s));
  c->built = true;
}

void refresh_device(tp_ctx* c) {
  cudaStream_t s = c->s;
  // A_pp and (for schur = 2) A_TT planes are the level-0 values in place
  launch_extract_blocks(c->nnzb, c->bval, c->App, c->ApT, c->ATp, c->ATT, s);
  if (c->opts.schur == 1) {
    learned_schur_values(c);
    if (c->learned_global_fallback)
      TP_CUDA_TRY(cudaMemcpyAsync(c->S_learned, c->Sval, sizeof(double) * c->nnzb,
                                  cudaMemcpyDeviceToDevice, s));
  }
  if (c->opts.schur == 3) schur_diag_values(c, false);
  c->hpp->refresh(s);
  c->hS->refresh(s);
}

void negated_residual(tp_ctx* c) {
  cudaStream_t s = c->s;
  const long long n = c->N;
  TP_CUDA_TRY(cudaMemcpyAsync(c->io0, c->Rm, n * sizeof(double), cudaMemcpyDeviceToDevice, s));
  TP_CUDA_TRY(cudaMemcpyAsync(c->io1, c->Re, n * sizeof(double), cudaMemcpyDeviceToDevice, s));
  negate(c->io0, n, s);
  negate(c->io1, n, s);
}

}  // namespace tp

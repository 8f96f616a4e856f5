/*
 * thermo.h -- C-ABI of the GB300 solver for the linearised non-isothermal
 * single-phase pressure/temperature system of Roy, Jonsthovel, Lemon and
 * Wathen, "A block preconditioner for non-isothermal flow in porous media"
 * (arXiv 1902.00095).
 *
 * The library assembles the TPFA Newton system (Sec. 2.2, Eq. Fm / Eq. Fe,
 * Eq. AXR), builds the block factorisation preconditioner of Sec. 3.2 with
 * the Schur approximation S~_T of Eq. Se, inverts A_pp and S~_T with one
 * algebraic-multigrid V-cycle each, and solves with right-preconditioned
 * flexible GMRES (Sec. 4 solver settings). All arithmetic runs in CUDA
 * kernels on the device of the stream given to tp_create.
 *
 * Conventions for every call
 *   - Return value: TP_OK (0), a negative error, or a positive warning.
 *     No call aborts, throws across the ABI, or traps the GPU.
 *   - Ownership: the caller owns every pointer it passes. Inputs are copied
 *     (or read during the call); outputs are written into caller buffers.
 *     The library owns all device memory it allocates and frees it in
 *     tp_destroy / tp_amg_destroy.
 *   - Pointers flagged by ptr_is_device = 1 are device pointers on the
 *     context's device; with 0 they are host pointers (pageable or pinned).
 *   - Streams: all work is enqueued on the context stream; calls return
 *     after their results are ready (the stream is synchronised).
 *   - Cell index i = x + nx*(y + ny*z), z up (layer 0 at the bottom).
 *   - A context is not thread-safe; use one per host thread.
 */
#ifndef THERMO_H
#define THERMO_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

/* status codes */
#define TP_OK              0
#define TP_EINVAL         -1  /* bad argument (NULL, size, range)           */
#define TP_ENOMEM         -2  /* device or host allocation failed           */
#define TP_ECUDA          -3  /* a CUDA runtime call failed                 */
#define TP_ENONFINITE     -4  /* NaN/Inf found in an input or a result      */
#define TP_SETUP_FAILED   -5  /* AMG setup could not finish (round cap,     */
                              /* coarsest level too large, zero pivot)      */
#define TP_ESTATE         -6  /* call order violated (e.g. solve before     */
                              /* assemble / build)                          */
#define TP_NOT_CONVERGED   1  /* FGMRES reached maxit above rtol            */
#define TP_BREAKDOWN       2  /* zero or non-finite Arnoldi norm            */

typedef struct tp_ctx tp_ctx;
typedef struct tp_amg tp_amg;

/* Cartesian grid: nx*ny*nz cells of dx*dy*dz metres, gravity g (m/s^2). */
typedef struct {
  int nx, ny, nz;
  double dx, dy, dz, g;
} tp_grid;

/* Fluid and rock constants (SI). Density rho0 exp(c (p-p0)) exp(beta (T-T0))
 * (Sec. 2.1.4). Viscosity: mu_law = 0, mu0 exp(-mu_coef (T - T_mu0));
 * mu_law = 1, the Bennison heavy-oil correlation of Eq. bennison,
 * mu = 1e-3 10^(A1 api + A2) T_F^(A3 api + A4) Pa s with T_F the
 * temperature in degrees Fahrenheit, A1..A4 of Table 1 and api the API
 * gravity (valid for T_F > 0; a non-positive T_F is reported as a
 * non-finite assembly). c_v and rock rho_r, c_r of Eq. energy1;
 * k_T = phi kTr + (1-phi) kTf as printed in Sec. 2.1.2 when kT_mix = 0,
 * or (1-phi) kTr + phi kTf when kT_mix = 1. */
typedef struct {
  double rho0, c, beta, p0, T0;
  double mu0, T_mu0, mu_coef;
  double cv, rho_r, cr, kTf;
  int kT_mix;
  int mu_law;
  double api;
} tp_fluid;

/* A well or heater completed in cells (i, j, k0..k1) (Sec. 2.1.5).
 * kind 0: rate injector, value = total volume rate (m^3/s) split equally
 *         over the completed layers, injected at T_inj (Eq. f, Eq. fT);
 * kind 1: producer at bottom-hole pressure value (Pa), Peaceman index per
 *         completed cell with Dx = Dy = h = 5 m, r_w = 0.1 m, no cross-flow;
 * kind 2: heater with coefficient U (W/K) per completed cell towards T_inj;
 * kind 3: rate producer, value = total volume rate (m^3/s). */
typedef struct {
  int i, j, k0, k1, kind;
  double value, T_inj, U;
} tp_well;

/* Preconditioner options (defaults from tp_default_opts). */
typedef struct {
  int schur;        /* 0: S~_T of Eq. Se; 1: S~_T with the learned correction */
                    /* (tp_set_schur_model); 2: S~_ATT = A_TT; 3: S~_diag =   */
                    /* A_TT - A_Tp diag(A_pp)^-1 A_pT on its 25-point pattern */
                    /* (Sec. 3.3)                                              */
  int variant;      /* 0: full five-step apply (Sec. 3.2); 1: block lower     */
                    /*    triangular (steps 1-3, delta_p = x_p)               */
  int precision;    /* 0: FP64 hierarchy; 1: FP32 hierarchy values, smoothers */
                    /*    and V-cycles inside FP64 FGMRES (coarsest LU FP64); */
                    /* 2: as 1 with P and R values stored in BF16 (FP32       */
                    /*    accumulation)                                       */
  int interp;       /* 0: classical (Ruge-Stueben, modified); 1: extended+i   */
                    /*    (default 1 for A_pp; S~ uses interp_S, default 0)  */
  int smoother;     /* 0: l1-Jacobi; 1: Chebyshev on D^-1 A, D = diag(A),     */
                    /*    over [lambda/30, 1.1 lambda], lambda from 10 power  */
                    /*    iterations (A_pp; S~ uses smoother_S)               */
  int nu_pre, nu_post, cheb_degree;  /* sweeps before/after the coarse       */
                    /* correction (defaults 3 and 4); cheb_degree in 1..4    */
  double theta;     /* strength threshold                                     */
  int max_levels;   /* at most this many levels (default 25)                  */
  int coarse_size;  /* coarsening stops at <= coarse_size rows (default 256); */
                    /* the coarsest level is solved with its explicit inverse */
                    /* (Gauss-Jordan with partial pivoting; <= 2048 rows)     */
  unsigned long long seed;  /* PMIS tie-break seed                            */
  int use_graphs;   /* 1: replay each V-cycle / preconditioner as a CUDA graph */
  /* overrides for the Schur hierarchy (-1 or 0: same as above) */
  int interp_S;     /* -1 same, 0 classical (default), 1 extended+i           */
  int max_levels_S; /* 0 same                                                 */
  int nu_S;         /* 0 same; else nu_pre = nu_post = nu_S (default 1: with  */
                    /* the line smoother of smoother_S = 2 on the finest      */
                    /* level, one sweep on each coarser level of S~ gives the */
                    /* same FGMRES iterations as three)                       */
  int pmax;         /* interpolation truncation: at most pmax weights per row  */
                    /* (largest |w|, row sums kept); default 4, 0 = off, <=16 */
  int smoother_S;   /* -1 same as smoother, 0 l1-Jacobi, 1 Chebyshev,        */
                    /* 2 (default): vertical-line Jacobi on the finest level  */
                    /*   (nu_line steps x += T^-1 (b - S x) before and after  */
                    /*   the coarse correction, T the tridiagonal part of S~  */
                    /*   along each grid column, factored by the Thomas       */
                    /*   algorithm; a GPU-parallel stand-in for the hybrid    */
                    /*   Gauss-Seidel of Sec. 4 that carries the vertical     */
                    /*   transport in S~ exactly), l1-Jacobi on coarser       */
                    /*   levels; grids with nz = 1 use l1-Jacobi throughout.  */
                    /*   Needs both vertical neighbours in the pattern and    */
                    /*   non-zero pivots (else TP_SETUP_FAILED)              */
  int tail_rows;    /* coarse levels (below level 0) with at most tail_rows    */
                    /* rows run as one thread-block-cluster kernel per V-cycle */
                    /* (l1-Jacobi only); 0 (default) = one kernel per phase on */
                    /* every level, measured faster on GB300 inside the graph  */
  int nu_line;      /* smoother_S = 2: line steps before and after, 1..8       */
                    /* (default 1)                                             */
  int sell_rows;    /* CSR levels between the finest and the coarsest with at */
                    /* least sell_rows rows keep a sliced-ELL copy of their   */
                    /* operator (32-row slices, rows sorted by length within  */
                    /* windows of 256, each slice padded to its longest row)  */
                    /* for their l1-Jacobi sweeps and residuals, one thread   */
                    /* per row; 0 (default): half a wave of resident threads  */
                    /* (SMs x maximum threads per SM / 2); -1: never. The     */
                    /* results differ only in the order of the row sums       */
} tp_precond_opts;

typedef struct {
  int iters, restarts, status;
  int levels_pp, levels_S;
  double rel_res;           /* ||D (b - A x)|| / ||D b|| (stopping measure)  */
  double rel_res_unscaled;  /* ||b - A x|| / ||b||                           */
  double rel_res_p, rel_res_T; /* per-block unscaled relative residuals      */
  double opc_pp, opc_S;     /* operator complexities                         */
  double t_solve_ms;
} tp_solve_info;

void        tp_default_opts(tp_precond_opts* opts);
const char* tp_status_string(int status);
/* Message of the last failed call on this host thread ("" if none). */
const char* tp_last_error(void);
/* Number of CUDA kernels this library has launched in this process (a CUDA
 * graph replay counts its kernel nodes). Host-side counter, no device work. */
long long   tp_kernel_launches(void);

/* --- context ------------------------------------------------------------
 * tp_create: one context per grid. `cuda_stream` is a cudaStream_t (NULL =
 * the legacy default stream). Fluid constants are copied. */
int  tp_create(tp_ctx** ctx, const tp_grid* grid, const tp_fluid* fluid,
               void* cuda_stream);
void tp_destroy(tp_ctx* ctx);
int  tp_get_sizes(const tp_ctx* ctx, int* N, int* nnzb);

/* Cell fields, each [N] float64: permeabilities (m^2) along x, y, z,
 * porosity, rock conductivity (W/m/K). Copied. Non-positive K or
 * non-finite values give TP_EINVAL / TP_ENONFINITE. */
int tp_set_fields(tp_ctx* ctx, const double* Kx, const double* Ky,
                  const double* Kz, const double* phi, const double* kTr,
                  int ptr_is_device);

/* Wells (host array of n entries, copied). Cells outside the grid or an
 * unknown kind give TP_EINVAL. */
int tp_set_wells(tp_ctx* ctx, const tp_well* wells, int n);

/* Newton linearisation at (p_k, T_k) with previous time level (p_n, T_n)
 * and step dt (Sec. 3, Eq. AXR): writes the block-CSR Jacobian (pattern
 * 7-point, columns ascending, 2x2 blocks [[dRm/dp, dRm/dT],[dRe/dp, dRe/dT]]),
 * the residual G(x_k) and S~_T (Eq. Se) into the context; optionally copies
 * the residual to R_m, R_e ([N] each, may be NULL). Inputs [N] each. */
int tp_assemble(tp_ctx* ctx, const double* p_k, const double* T_k,
                const double* p_n, const double* T_n, double dt,
                double* R_m, double* R_e, int ptr_is_device);

/* Split the Jacobian into A_pp, A_pT, A_Tp, A_TT (Eq. AXR), build one AMG
 * hierarchy for A_pp and one for the Schur approximation chosen in opts.
 * Requires a prior tp_assemble. */
int tp_build_preconditioner(tp_ctx* ctx, const tp_precond_opts* opts);

/* Solve A x = b with FGMRES(restart) preconditioned on the right by the
 * block preconditioner. b = (b_p, b_T), x = (x_p, x_T), [N] each; if b_p
 * and b_T are both NULL, b = -G(x_k) from the last tp_assemble. x starts at
 * zero. Returns TP_OK, TP_NOT_CONVERGED or TP_BREAKDOWN (info filled in all
 * three cases). */
int tp_solve(tp_ctx* ctx, const double* b_p, const double* b_T,
             double* x_p, double* x_T, double rtol, int maxit, int restart,
             tp_solve_info* info, int ptr_is_device);

/* Timing probe for roofline measurements: CUDA events on the context stream
 * around every launch of one kernel class during tp_solve, read back after
 * the per-iteration host synchronisation FGMRES already performs.
 * which = 0: finest-level l1-Jacobi sweeps of the A_pp hierarchy;
 *         1: finest-level sweeps (or vertical-line steps) of the S~
 *            hierarchy; 2: block SpMV; 3: l1-Jacobi sweeps on level 1 of
 *            the A_pp hierarchy (the first Galerkin level, CSR);
 *        -1: off. Enabling resets the totals and requires a new
 * tp_build_preconditioner (the events are captured into the graph). */
int tp_probe_enable(tp_ctx* ctx, int which);
/* Totals since enabling (or the last reset): summed event time (ms), number
 * of launches timed, and their summed algorithmic bytes (each matrix entry,
 * index and vector element counted once). */
int tp_probe_read(tp_ctx* ctx, double* total_ms, long long* launches,
                  double* total_bytes, int reset);

/* Newton iteration with line search of one backward-Euler step (Sec. 3
 * linearisation; Sec. 4: Newton with line search, relative function-norm and
 * step tolerances): starting from x = (p_n, T_n), repeat assemble /
 * precondition / FGMRES / line search until ||D G(x_k)|| <= tol_f
 * ||D G(x_0)|| (D the equation scaling of the first linearisation) or
 * alpha ||dx|| <= tol_dx ||x||, at most max_newton linear solves. The line
 * search backtracks x_k + alpha dx (alpha = 1, 1/2, ..., at most 6 halvings)
 * until ||D G|| <= (1 - 1e-4 alpha) ||D G(x_k)||; line_search = 0 takes full
 * steps. reuse = 1 keeps the AMG structure of the first iteration and
 * refreshes only the Galerkin values (and keeps the captured graph). The new
 * state is written to p_out, T_out ([N] each). Returns TP_OK or
 * TP_NOT_CONVERGED. */
typedef struct {
  int max_newton;
  double tol_f, tol_dx;
  double rtol;      /* FGMRES relative tolerance per linear solve */
  int maxit, restart;
  int reuse;
  int line_search;
} tp_newton_opts;

typedef struct {
  int newton_iters, linear_iters, status, last_linear_status;
  double rel_f, rel_dx, t_ms;
  int line_search_halvings;
} tp_newton_info;

int tp_newton_step(tp_ctx* ctx, const double* p_n, const double* T_n, double dt,
                   double* p_out, double* T_out, const tp_precond_opts* popts,
                   const tp_newton_opts* nopts, tp_newton_info* info,
                   int ptr_is_device);

/* y = A x with the assembled Jacobian (Eq. AXR), no scaling. [N] each. */
int tp_spmv(tp_ctx* ctx, const double* x_p, const double* x_T,
            double* y_p, double* y_T, int ptr_is_device);

/* z = M^{-1} v: one application of the block preconditioner of Sec. 3.2
 * (unscaled system). [N] each. Requires tp_build_preconditioner. */
int tp_apply_preconditioner(tp_ctx* ctx, const double* v_p, const double* v_T,
                            double* z_p, double* z_T, int ptr_is_device);

/* Copies of the assembled operators to host buffers: the block matrix
 * (rowptr [N+1], col [nnzb], val [4*nnzb] row-major blocks) and the Schur
 * approximation values on the same pattern ([nnzb]). Any pointer may be
 * NULL. Also the equation scales (s_m, s_e) used by tp_solve. */
int tp_export_system(tp_ctx* ctx, int* rowptr, int* col, double* val,
                     double* schur_val, double* scales);

/* V-cycle bandwidth measurement (Sec. 3.2: each approximate inverse is one
 * AMG V-cycle): captures one V-cycle of hierarchy which (0 A_pp, 1 Schur)
 * of the last build as a CUDA graph, replays it once untimed and then reps
 * times between two events on the context stream, with every entry of the
 * right-hand side 1. Writes the mean time per V-cycle (ms), its algorithmic
 * bytes (every level's operator, smoother scaling or line factors, R, P
 * and vectors, each counted once per kernel that reads or writes them) and
 * the hierarchy's operator complexity (sum of level nnz / finest nnz). Any
 * output pointer may be NULL. Overwrites the hierarchy's work vectors (no
 * effect on later solves). TP_ESTATE before tp_build_preconditioner. */
int tp_vcycle_measure(tp_ctx* ctx, int which, int reps, double* ms, double* bytes,
                      double* opc);

/* Host wall time (ms) of the last AMG setup of hierarchy which (0 A_pp,
 * 1 Schur) by phase: ms[0] strength + PMIS, ms[1] interpolation,
 * ms[2] transpose, ms[3] Galerkin products, ms[4] smoother scaling, ELL copy
 * and coarsest inverse. */
int tp_setup_timings(tp_ctx* ctx, int which, double* ms);

/* Hierarchy introspection: which = 0 (A_pp) or 1 (Schur). n/nnz receive
 * up to max_levels entries. */
int tp_hierarchy_info(tp_ctx* ctx, int which, int* nlevels, int* n, int* nnz,
                      int max_levels);

/* --- standalone AMG on a caller CSR matrix --------------------------------
 * tp_amg_create builds the hierarchy of an n x n CSR matrix (rowptr [n+1],
 * col [nnz] ascending per row with the diagonal present, val [nnz]); the
 * pattern must be structurally symmetric. Inputs are copied. */
int  tp_amg_create(tp_amg** amg, int n, int nnz, const int* rowptr,
                   const int* col, const double* val,
                   const tp_precond_opts* opts, void* cuda_stream,
                   int ptr_is_device);
void tp_amg_destroy(tp_amg* amg);
/* One V-cycle from a zero initial guess: x = V(b), [n] each. */
int  tp_amg_vcycle(tp_amg* amg, const double* b, double* x, int ptr_is_device);
int  tp_amg_info(tp_amg* amg, int* nlevels, int* n, int* nnz, int max_levels);
/* Host copies of level `level`: operator A_l (rowptr [n_l+1], col/val
 * [nnz_l]), C/F split cf [n_l] (+1 C, -1 F; only for non-coarsest levels),
 * strength mask [nnz_l] (1 strong), interpolation P_l (rowptr [n_l+1],
 * col/val sized by P_nnz). Any pointer may be NULL. */
int  tp_amg_export_level(tp_amg* amg, int level, int* rowptr, int* col,
                         double* val, signed char* cf, signed char* strong,
                         int* P_nnz, int* P_rowptr, int* P_col, double* P_val);
/* Storage of level `level`'s operator in its smoothing sweeps: format 0 CSR,
 * 1 ELL (column-major, padded to the longest row), 2 sliced ELL (see
 * tp_precond_opts.sell_rows), 3 ELL by grid direction (the finest level of a
 * context hierarchy whose operator is the grid's 7-point pattern, every grid
 * extent >= 2: 7 values per row, 0 where a neighbour is absent, no column
 * indices); stored = entries held, padding included (CSR: nnz). Host-only (no device work); TP_ESTATE before a build, TP_EINVAL for
 * a level out of range. tp_level_storage: a context hierarchy (which = 0
 * A_pp, 1 Schur). */
int  tp_amg_level_storage(tp_amg* amg, int level, int* format, long long* stored);
int  tp_level_storage(tp_ctx* ctx, int which, int level, int* format, long long* stored);
/* Same introspection for a context hierarchy (which = 0 A_pp, 1 Schur). */
int  tp_export_level(tp_ctx* ctx, int which, int level, int* rowptr, int* col,
                     double* val, signed char* cf, signed char* strong,
                     int* P_nnz, int* P_rowptr, int* P_col, double* P_val);

/* --- learned correction of the Schur approximation -----------------------
 * Not in the paper (a growth direction of this library): a per-cell MLP
 * 24 -> 64 -> 64 -> 8 (GELU, tanh form) rescales row i of S~_T (Eq. Se):
 *   S_ii <- S~_ii exp(o_0) + o_7 S~_ii,  S_ij <- S~_ij exp(o_d), d = 1..6 the
 *   face direction of j (z-, y-, x-, x+, y+, z+).
 * A row keeps plain S~_T when its corrected diagonal is not positive, an
 * off-diagonal changes sign, or it loses the diagonal dominance the plain
 * row had; if more than a quarter of the rows fall back, plain S~_T is used.
 * Parameters: flat float64 [6280] in the order W1 [64][24], b1 [64],
 * W2 [64][64], b2 [64], W3 [8][64], b3 [8] (row-major). The device keeps
 * FP32 master weights and BF16 copies; inference and training run on BF16
 * tensor cores with FP32 accumulation. */
typedef struct tp_mlp tp_mlp;
int  tp_mlp_create(tp_mlp** mlp, const double* params, void* cuda_stream);
void tp_mlp_destroy(tp_mlp* mlp);
int  tp_mlp_set_params(tp_mlp* mlp, const double* params);  /* resets Adam */
int  tp_mlp_get_params(tp_mlp* mlp, double* params);
/* O [n][8] = MLP(X [n][24]) (FP32). */
int  tp_mlp_forward(tp_mlp* mlp, int n, const float* X, float* O, int ptr_is_device);
/* Gradient (host [6280], may be NULL) and value of the loss
 * mean_s ((S_learned,s - target_s) / Sd_s)^2 over B samples: features X
 * [B][24], slot_s (0 diagonal, 1..6 face direction), S~ entry St_s, S~
 * diagonal Sd_s, exact Schur entry target_s. */
int  tp_mlp_gradient(tp_mlp* mlp, int B, const float* X, const int* slot,
                     const double* St, const double* Sd, const double* target,
                     double* grad, double* loss, int ptr_is_device);
/* Same gradient, then one Adam step (Kingma and Ba 2015, beta 0.9/0.999,
 * eps 1e-8, bias-corrected) with learning rate lr. */
int  tp_mlp_train_step(tp_mlp* mlp, int B, const float* X, const int* slot,
                       const double* St, const double* Sd, const double* target,
                       double lr, double* loss, int ptr_is_device);
/* Features of every cell at the last tp_assemble, X [N][24] FP32:
 * 0-5 log10(T_f / 1e-12 m^3), 6-11 log10(Tc_f / (1 W/K)) per face direction
 * (0 without a face), 12 log10(lambda / 1e6), 13-18 outward advective face
 * coefficient c_v T_f lambda_up dPhi / S~_ii, 19 A_pT A_Tp / (A_pp A_TT) at
 * the diagonal, 20 log10(A_pp,ii s_m), 21 log10(A_TT,ii s_e),
 * 22 (A_TT,ii - S~_ii) / S~_ii, 23 accumulation / S~_ii. */
int  tp_learned_features(tp_ctx* ctx, float* X, int ptr_is_device);
/* Model used by tp_build_preconditioner when opts.schur == 1 (borrowed:
 * must outlive its use). */
int  tp_set_schur_model(tp_ctx* ctx, tp_mlp* model);
/* Rows that fell back to plain S~ in the last learned build, and whether
 * the whole matrix did. */
int  tp_learned_status(tp_ctx* ctx, int* fallback_rows, int* global_fallback);
/* Exact Schur complement columns restricted to the 7-point pattern
 * (S = A_TT - A_Tp A_pp^{-1} A_pT, Eq. Afact): for each column j of cols,
 * z = A_pp^{-1} A_pT e_j by FGMRES preconditioned with the A_pp V-cycle of
 * the last build (relative tolerance rtol), then S_ij = (A_TT e_j -
 * A_Tp z)_i for the rows i of column j. Host outputs entry [ncols][7]
 * (pattern entry index of (i, j), -1 padding) and value [ncols][7];
 * iters = total FGMRES iterations. TP_NOT_CONVERGED if a solve stopped
 * above rtol. */
int  tp_probe_schur_columns(tp_ctx* ctx, const int* cols, int ncols, double rtol,
                            int* entry, double* value, int* iters);

/* --- allocation-free equation scales -------------------------------------
 * The paper has no counterpart to this call; it exists for callers that
 * cannot allocate device memory (a frozen or defragmenting memory pool,
 * allocator hooks, embedders with a fixed device budget). It computes the
 * same equation scales as the solver, scales[0] = N / sum_i |A_pp,ii| and
 * scales[1] = N / sum_i |A_TT,ii|, from a caller-owned block-CSR matrix in
 * the layout tp_export_system returns (rowptr [N+1], col [nnzb], val
 * [4*nnzb] row-major 2x2 blocks), all DEVICE pointers, writing scales [2]
 * (device). It calls no cudaMalloc/cudaFree: its only scratch is a fixed
 * 64 KiB __device__ array that every GPU loading this library keeps until
 * exit. Limit: N <= 8,388,608 cells; larger N returns TP_EINVAL. A call on
 * a stream that is not capturing looks up the array's device address
 * afresh (following a device reset or a new context); a call inside a stream
 * capture reuses the address of the last uncaptured call on that device, so
 * make one uncaptured call on each device before capturing. All calls share the array, so calls whose
 * kernels overlap on the GPU (different streams, or concurrent host
 * threads) race; serialise them. Work is enqueued on cuda_stream (a
 * cudaStream_t, NULL = legacy default stream) and the call returns without
 * synchronising; the result is ready when the stream reaches that point.
 * Returns TP_OK, TP_EINVAL or TP_ECUDA. */
int tp_equation_scales_noalloc(int N, const int* rowptr, const int* col,
                               const double* val, double* scales,
                               void* cuda_stream);

#ifdef __cplusplus
}
#endif
#endif /* THERMO_H */

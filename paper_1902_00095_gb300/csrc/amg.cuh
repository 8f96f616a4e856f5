// Algebraic multigrid hierarchy (internal header).
//
// Setup: strength of connection, PMIS C/F splitting with seeded tie-breaks,
// classical or extended+i interpolation, R = P^T, Galerkin R (A P), l1-Jacobi
// scaling, and an explicit inverse of the coarsest operator from LU with
// partial pivoting. Everything that decides structure is evaluated in one
// fixed order with correctly rounded IEEE multiply/add/divide (no FMA
// contraction), so the hierarchy is reproducible bit for bit.
//
// Solve: one V-cycle from a zero guess, FP64 or FP32 values/vectors, replayable
// as a CUDA graph.
#pragma once
#include <cuda_bf16.h>
#include "common.cuh"

namespace tp {

__device__ __forceinline__ unsigned long long splitmix64(unsigned long long x) {
  // splitmix64 output for state x (Steele, Lea, Flood 2014)
  unsigned long long z = x + 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

// tie-break hash of row i: upper 32 bits of splitmix64(seed xor i)
__device__ __forceinline__ unsigned int pmis_hash(unsigned long long seed, int i) {
  return (unsigned int)(splitmix64(seed ^ (unsigned long long)(long long)i) >> 32);
}

constexpr int kMaxChebDegree = 4;

struct AmgOpts {
  int interp = 1;        // 0 classical, 1 extended+i
  int smoother = 0;      // 0 l1-Jacobi, 1 Chebyshev
  int nu_pre = 3, nu_post = 3, cheb_degree = 2;
  double theta = 0.25;
  int max_levels = 25, coarse_size = 256, max_coarse_dense = 2048;
  unsigned long long seed = 0;
  int precision = 0;     // 0 FP64, 1 FP32 hierarchy, 2 FP32 + BF16 P and R
  int max_pmis_rounds = 64;
  int pmax = 0;          // interpolation truncation (0 = off)
  int tail_rows = 0;      // coarse levels with at most this many rows: one cluster kernel (0 off)
  int sell_rows = 0;      // sliced-ELL copy from this many rows (0: half a wave of threads, -1 off)
  // vertical-line smoothing of the finest level: the level is the grid of
  // line_nxy columns x line_nz layers (cell c + line_nxy k); nu_line line
  // steps x <- x + T^-1 (b - A x) before and after the coarse correction,
  // T the tridiagonal part of A along each column (off when line_nz < 2)
  int line_nxy = 0, line_nz = 0, nu_line = 1;
  // level 0 is the 7-point operator of this nx x ny x nz grid (cell x + nx y
  // + nx ny z; 0: unknown): with every extent >= 2 its ELL copy is stored by
  // grid direction, without column indices
  int grid_nx = 0, grid_ny = 0, grid_nz = 0;
};

// Device descriptor of one level for the cluster kernel of the V-cycle's
// coarse tail (vcycle_tail.cu): values and vectors in the hierarchy's
// precision, P and R optionally BF16.
struct TailLevel {
  int n, nnext;  // rows of A and of the next level
  const int *Arp, *Acol;
  const void *Aval, *dinv;
  const int *Prp, *Pcol;
  const void* Pval;
  const __nv_bfloat16* Ph;
  const int *Rrp, *Rcol;
  const void* Rval;
  const __nv_bfloat16* Rh;
  void *b, *x, *t, *r;
};
constexpr int kMaxTailLevels = 32;
// cluster size the tail kernel launches with (16 or 8), 0 if unavailable
int tail_cluster_size();
// Explicit inverse of the dense coarsest operator (n x n row-major) by one
// thread-block cluster; *err = 1 if it is singular. Returns false (nothing
// launched) when the matrix does not fit the cluster's shared memory or
// clusters cannot be launched.
bool coarse_inverse_cluster(int n, const double* A, double* inv, int* err, cudaStream_t s);
template <class TV>
void launch_vcycle_tail(const TailLevel* desc, int first, int last, const double* cinv, int nc,
                        int nu_pre, int nu_post, int cluster, cudaStream_t s);

// CUDA-event timing of one kernel class inside the timed region: events are
// recorded around each launch (as external event nodes when captured into a
// graph) and read back once the host has waited for them. Two event sets
// alternate between consecutive solver iterations, so an iteration can be
// enqueued while the previous one's events are read.
struct Probe {
  static constexpr int kMaxPairs = 64;
  cudaEvent_t ev[2][2 * kMaxPairs] = {};
  double bytes[kMaxPairs] = {};
  int nlaunch[kMaxPairs] = {};   // kernel launches between the two events of a pair
  int npairs = 0;   // pairs per recorded sequence (the same for both sets)
  int active = 0;   // set that before()/after() record into
  bool created = false;
  // accumulated over reads
  double total_ms = 0.0, total_bytes = 0.0;
  long long launches = 0;
  void create();
  void destroy();
  void before(cudaStream_t s);
  void after(cudaStream_t s, double algorithmic_bytes, int launches_in_span = 1);
  void read_and_accumulate(int set);   // after the set's last event completed
};

struct Level {
  DevCSR A;
  int* dpos = nullptr;
  int* tpos = nullptr;
  unsigned char* strong = nullptr;
  signed char* cf = nullptr;
  int pmis_rounds = 0;
  DevCSR P, R;       // P: n x nc, R: nc x n
  DevCSR AP;         // A P (kept for numeric-only refreshes)
  __nv_bfloat16* Ph = nullptr;   // BF16 copies of the P and R values
  __nv_bfloat16* Rh = nullptr;   // (precision 2)
  double* dinv = nullptr;   // smoother scaling (l1 or plain diagonal), FP64
  float* dinvf = nullptr;
  // Chebyshev: coefficients (FP64 [2 deg - 1], then the power-iteration
  // scale and lambda_max at [2 kMaxChebDegree], [2 kMaxChebDegree + 1]),
  // FP32 copy, power-iteration vectors and the recurrence work vectors
  double* cheb = nullptr;
  float* chebf = nullptr;
  double *pw0 = nullptr, *pw1 = nullptr;
  void *cw = nullptr, *cd0 = nullptr, *cd1 = nullptr, *cr = nullptr;
  // V-cycle work vectors, in the hierarchy precision (double* or float*)
  void* b = nullptr;
  void* x = nullptr;
  void* t = nullptr;
  void* r = nullptr;
  int lanes_A = 1, lanes_R = 1, lanes_P = 1;
  // ELL copy of A (slot-major: entry k of row i at k * n + i, padded with
  // column i and value 0) for levels whose rows have at most kEllMaxW entries
  int ell_w = 0;
  // ell_nxy > 0: the slots are the grid directions (offsets -nxy, -nx, -1,
  // 0, +1, +nx, +nxy: ascending columns), value 0 where a neighbour is
  // absent, and ell_col is null: a slot's column is the row plus its offset,
  // clamped to [0, n) (an absent neighbour's slot adds an exact zero)
  int ell_nx = 0, ell_nxy = 0;
  int* ell_col = nullptr;
  double* ell_val = nullptr;
  float* ell_valf = nullptr;
  // sliced-ELL copy of A for long-row levels below the finest: rows sorted by
  // length (descending) within windows of kSellWindow rows, slices of 32
  // consecutive sorted rows padded to the slice's longest row, entry k of
  // slot t of slice s at sell_ptr[s] + 32 k + t (padding: column = the row
  // itself, value 0; slots past n: column 0). sell_perm[slot] = the row of a
  // slot (-1 past n).
  int sell_slices = 0;
  long long sell_entries = 0;  // stored slots, padding included
  int* sell_ptr = nullptr;
  int* sell_perm = nullptr;
  int* sell_col = nullptr;
  double* sell_val = nullptr;
  float* sell_valf = nullptr;
  // vertical-line smoother (finest level only): per cell the coefficient of
  // the cell below (l), 1 / m and u / m of the Thomas factorisation of the
  // column's tridiagonal part (FP64, FP32 copies in the FP32 hierarchy)
  double *line_lo = nullptr, *line_minv = nullptr, *line_cp = nullptr;
  float *line_lof = nullptr, *line_minvf = nullptr, *line_cpf = nullptr;
};

constexpr int kEllMaxW = 8;
constexpr int kSellWindow = 256;

class Hierarchy {
 public:
  Hierarchy() = default;
  Hierarchy(const Hierarchy&) = delete;
  Hierarchy& operator=(const Hierarchy&) = delete;
  ~Hierarchy();

  // Build from a CSR matrix whose arrays stay owned by the caller and must
  // outlive the hierarchy (level 0 borrows them).
  void setup(const DevCSR& A0, const AmgOpts& opts, cudaStream_t s);
  // Numeric-only refresh after the level-0 values changed in place: keeps
  // the C/F splits, P, R and every pattern; recomputes A P and R (A P) in the
  // setup's canonical order, the smoother scaling, the FP32 copies and the
  // coarsest inverse. Buffers keep their addresses (captured graphs stay
  // valid).
  void refresh(cudaStream_t s);
  // One V-cycle: out = V(in). in/out are the hierarchy's own FP64 buffers.
  void vcycle(cudaStream_t s);
  double operator_complexity() const;
  // algorithmic bytes of one V-cycle (each kernel's operator, scaling and
  // vectors counted once)
  double vcycle_bytes() const;

  AmgOpts opts;
  Probe* probe = nullptr;  // times the smoothing sweeps of level probe_level when set
  int probe_level = 0;
  std::vector<Level> L;
  int n0 = 0;
  double* in = nullptr;    // [n0] FP64 right-hand side
  double* out = nullptr;   // [n0] FP64 result
  double* coarse_inv = nullptr;   // [nc*nc] row-major inverse of the coarsest A
  int nc = 0;
  Pool pool;
  Pool scratch;   // setup temporaries (rewound after every level)
  double* coarse_dense = nullptr;   // [nc*nc] work for the inverse
  // host wall time of the setup phases (ms): strength + PMIS, interpolation,
  // transpose, Galerkin products, smoother scaling + coarse inverse
  double phase_ms[5] = {0, 0, 0, 0, 0};
  int* err = nullptr;
  double* cheb_partials = nullptr;   // norm partial sums of the power iteration
  // coarse tail run as one cluster kernel: levels tail_first..L.size()-1
  // (-1: every level has its own kernels)
  int tail_first = -1, tail_cluster = 0;
  TailLevel* tail_desc = nullptr;
  std::vector<TailLevel> tail_host;

 private:
  void finish_levels(cudaStream_t s, bool allocate);
  void plan_tail(cudaStream_t s);
  void vcycle_fp64(cudaStream_t s);
  void vcycle_fp32(cudaStream_t s);
};

// Chebyshev smoother (chebyshev.cu): plain-diagonal scaling, lambda_max by
// power iteration and the recurrence coefficients, all on the device.
void chebyshev_setup(Level& v, Pool& pool, int degree, unsigned long long seed,
                     double* partials, int* err, bool allocate, cudaStream_t s);
int chebyshev_norm_parts();
// xout = Chebyshev(degree) applied to A x = b from xin (zero when null)
template <class TV, class TB, class TO>
void chebyshev_apply(const Level& v, const TV* val, const TV* dinv, int degree, const TB* b,
                     const TV* xin, TO* xout, cudaStream_t s);

// Standalone sparse helpers reused by the solver.
// C = A B in the hierarchy's canonical summation order (C's arrays from
// `pool`), and the numeric-only recomputation of C's values on its pattern.
DevCSR csr_product(const DevCSR& A, const DevCSR& B, Pool& pool, Pool& scratch,
                   cudaStream_t s);
void csr_product_numeric(const DevCSR& A, const DevCSR& B, const DevCSR& C, cudaStream_t s);
void csr_transpose_positions(const DevCSR& A, int* tpos, int* err, cudaStream_t s);

}  // namespace tp

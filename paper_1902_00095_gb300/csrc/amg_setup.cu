// AMG setup kernels: strength, PMIS, interpolation, transpose, Galerkin
// product, smoother scaling and the coarsest-level inverse.
//
// The paper inverts A_pp and S~_T approximately with an AMG V-cycle
// (Sec. 3.2) built with classical Ruge-Stueben interpolation and Gaussian
// elimination on the coarsest grid (Sec. 4 solver settings). Here the C/F
// split is PMIS with seeded tie-breaks and the interpolation is classical or
// its distance-two extended+i form; all structure-deciding arithmetic uses
// __dmul_rn / __dadd_rn / __ddiv_rn in a fixed ascending-column order.
#include "amg.cuh"
#include <chrono>
#include <cmath>
#include <algorithm>

namespace tp {

namespace {

constexpr signed char kC = 1, kF = -1, kU = 0;

int setup_sms();
long long resident_threads();

// index of key in a[lo, hi) (ascending), or -1
__device__ __forceinline__ int find_in(const int* __restrict__ a, int lo, int hi, int key) {
  int h = hi;
  while (lo < hi) {
    int mid = (lo + hi) >> 1;
    if (a[mid] < key) lo = mid + 1;
    else hi = mid;
  }
  return (lo < h && a[lo] == key) ? lo : -1;
}

// (d > 0 && a < 0) || (d < 0 && a > 0), decided on the bit patterns: both
// non-zero, neither NaN, signs differ. Integer operations instead of FP64
// comparisons, which on this part share the FP64 pipe (2 per clock per SM)
// with the setup's multiply-adds and divisions.
__device__ __forceinline__ bool opposite(double a, double d) {
  const unsigned long long ua = (unsigned long long)__double_as_longlong(a);
  const unsigned long long ud = (unsigned long long)__double_as_longlong(d);
  const unsigned long long ma = ua & 0x7fffffffffffffffull, md = ud & 0x7fffffffffffffffull;
  const unsigned long long inf = 0x7ff0000000000000ull;
  return ma != 0 && md != 0 && ma <= inf && md <= inf && ((ua ^ ud) >> 63) != 0;
}

__global__ void k_diag_pos(int n, const int* __restrict__ rp, const int* __restrict__ col,
                           int* __restrict__ dpos, int* __restrict__ err) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  int p = find_in(col, rp[i], rp[i + 1], i);
  dpos[i] = p;
  if (p < 0) atomicOr(err, 1);
}

__global__ void k_transpose_pos(int n, const int* __restrict__ rp, const int* __restrict__ col,
                                int* __restrict__ tpos, int* __restrict__ err) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  for (int e = rp[i]; e < rp[i + 1]; ++e) {
    int k = col[e];
    int p = (k >= 0 && k < n) ? find_in(col, rp[k], rp[k + 1], i) : -1;
    tpos[e] = p;
    if (p < 0) atomicOr(err, 2);
  }
}

// the same with one warp per row (lanes over the row's entries): for the
// long rows of coarse Galerkin levels
__global__ void k_transpose_pos_warp(int n, const int* __restrict__ rp,
                                     const int* __restrict__ col, int* __restrict__ tpos,
                                     int* __restrict__ err) {
  const int lane = threadIdx.x & 31;
  const int i = (int)((blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5);
  if (i >= n) return;
  for (int e = rp[i] + lane; e < rp[i + 1]; e += 32) {
    int k = col[e];
    int p = (k >= 0 && k < n) ? find_in(col, rp[k], rp[k + 1], i) : -1;
    tpos[e] = p;
    if (p < 0) atomicOr(err, 2);
  }
}

// mean row length from which row-wise setup kernels take one warp per row
constexpr int kWarpRowMean = 16;

// strong[e] = 1 iff col != i and -a_e >= theta * max_{k != i}(-a_ik) > 0
__global__ void k_strength(int n, const int* __restrict__ rp, const int* __restrict__ col,
                           const double* __restrict__ val, double theta,
                           unsigned char* __restrict__ strong) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  double mx = -INFINITY;
  for (int e = rp[i]; e < rp[i + 1]; ++e)
    if (col[e] != i && -val[e] > mx) mx = -val[e];
  if (!(mx > 0.0)) {
    for (int e = rp[i]; e < rp[i + 1]; ++e) strong[e] = 0;
    return;
  }
  const double thr = __dmul_rn(theta, mx);
  for (int e = rp[i]; e < rp[i + 1]; ++e) strong[e] = (col[e] != i && -val[e] >= thr) ? 1 : 0;
}

__global__ void k_pmis_init(int n, const int* __restrict__ rp, const int* __restrict__ col,
                            const unsigned char* __restrict__ strong,
                            const int* __restrict__ tpos, int* __restrict__ lam,
                            signed char* __restrict__ state) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  int l = 0;
  for (int e = rp[i]; e < rp[i + 1]; ++e)
    if (col[e] != i && strong[tpos[e]]) ++l;
  lam[i] = l;
  state[i] = (l == 0) ? kF : kU;
}

__global__ void k_pmis_select(int n, const int* __restrict__ rp, const int* __restrict__ col,
                              const unsigned char* __restrict__ strong,
                              const int* __restrict__ tpos, const int* __restrict__ lam,
                              const signed char* __restrict__ state, unsigned long long seed,
                              unsigned char* __restrict__ newc) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  if (state[i] != kU) {
    newc[i] = 0;
    return;
  }
  const int li = lam[i];
  const unsigned int hi = pmis_hash(seed, i);
  unsigned char is_max = 1;
  for (int e = rp[i]; e < rp[i + 1]; ++e) {
    int k = col[e];
    if (k == i || state[k] != kU) continue;
    if (!(strong[e] || strong[tpos[e]])) continue;
    int lk = lam[k];
    unsigned int hk = pmis_hash(seed, k);
    bool bigger = (lk > li) || (lk == li && (hk > hi || (hk == hi && k > i)));
    if (bigger) {
      is_max = 0;
      break;
    }
  }
  newc[i] = is_max;
}

__global__ void k_pmis_update(int n, const int* __restrict__ rp, const int* __restrict__ col,
                              const unsigned char* __restrict__ strong,
                              signed char* __restrict__ state,
                              const unsigned char* __restrict__ newc,
                              int* __restrict__ undecided) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  if (newc[i]) {
    state[i] = kC;
    return;
  }
  if (state[i] != kU) return;
  for (int e = rp[i]; e < rp[i + 1]; ++e) {
    int k = col[e];
    if (strong[e] && (newc[k] || state[k] == kC)) {
      state[i] = kF;
      return;
    }
  }
  atomicAdd(undecided, 1);
}

// One-warp-per-row forms of the strength and PMIS kernels above, for levels
// whose mean row length is at least kWarpRowMean: the lanes take the row's
// entries, the row's decision is a warp reduction (a maximum, a count, an
// any), so the results are the same bit for bit.
__device__ __forceinline__ int warp_row(int& lane) {
  lane = threadIdx.x & 31;
  return (int)((blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5);
}

__global__ void k_strength_warp(int n, const int* __restrict__ rp, const int* __restrict__ col,
                                const double* __restrict__ val, double theta,
                                unsigned char* __restrict__ strong) {
  int lane;
  const int i = warp_row(lane);
  if (i >= n) return;
  const int r0 = rp[i], r1 = rp[i + 1];
  double mx = -INFINITY;
  for (int e = r0 + lane; e < r1; e += 32)
    if (col[e] != i && -val[e] > mx) mx = -val[e];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const double t = __shfl_xor_sync(0xffffffffu, mx, o);
    if (t > mx) mx = t;
  }
  if (!(mx > 0.0)) {
    for (int e = r0 + lane; e < r1; e += 32) strong[e] = 0;
    return;
  }
  const double thr = __dmul_rn(theta, mx);
  for (int e = r0 + lane; e < r1; e += 32)
    strong[e] = (col[e] != i && -val[e] >= thr) ? 1 : 0;
}

__global__ void k_pmis_init_warp(int n, const int* __restrict__ rp, const int* __restrict__ col,
                                 const unsigned char* __restrict__ strong,
                                 const int* __restrict__ tpos, int* __restrict__ lam,
                                 signed char* __restrict__ state) {
  int lane;
  const int i = warp_row(lane);
  if (i >= n) return;
  int l = 0;
  for (int e = rp[i] + lane; e < rp[i + 1]; e += 32)
    if (col[e] != i && strong[tpos[e]]) ++l;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) l += __shfl_xor_sync(0xffffffffu, l, o);
  if (lane == 0) {
    lam[i] = l;
    state[i] = (l == 0) ? kF : kU;
  }
}

__global__ void k_pmis_select_warp(int n, const int* __restrict__ rp,
                                   const int* __restrict__ col,
                                   const unsigned char* __restrict__ strong,
                                   const int* __restrict__ tpos, const int* __restrict__ lam,
                                   const signed char* __restrict__ state,
                                   unsigned long long seed, unsigned char* __restrict__ newc) {
  int lane;
  const int i = warp_row(lane);
  if (i >= n) return;
  if (state[i] != kU) {
    if (lane == 0) newc[i] = 0;
    return;
  }
  const int li = lam[i];
  const unsigned int hi = pmis_hash(seed, i);
  bool bigger = false;
  for (int e = rp[i] + lane; e < rp[i + 1] && !bigger; e += 32) {
    const int k = col[e];
    if (k == i || state[k] != kU) continue;
    if (!(strong[e] || strong[tpos[e]])) continue;
    const int lk = lam[k];
    const unsigned int hk = pmis_hash(seed, k);
    bigger = (lk > li) || (lk == li && (hk > hi || (hk == hi && k > i)));
  }
  const bool any = __any_sync(0xffffffffu, bigger);
  if (lane == 0) newc[i] = any ? 0 : 1;
}

__global__ void k_pmis_update_warp(int n, const int* __restrict__ rp,
                                   const int* __restrict__ col,
                                   const unsigned char* __restrict__ strong,
                                   signed char* __restrict__ state,
                                   const unsigned char* __restrict__ newc,
                                   int* __restrict__ undecided) {
  int lane;
  const int i = warp_row(lane);
  if (i >= n) return;
  if (newc[i]) {
    if (lane == 0) state[i] = kC;
    return;
  }
  if (state[i] != kU) return;
  bool c = false;
  for (int e = rp[i] + lane; e < rp[i + 1] && !c; e += 32) {
    const int k = col[e];
    c = strong[e] && (newc[k] || state[k] == kC);
  }
  const bool any = __any_sync(0xffffffffu, c);
  if (lane == 0) {
    if (any) state[i] = kF;
    else atomicAdd(undecided, 1);
  }
}

__global__ void k_cflag(int n, const signed char* __restrict__ state, int* __restrict__ flag) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) flag[i] = state[i] == kC ? 1 : 0;
}

// ---------------------------------------------------- classical interpolation
__device__ __forceinline__ bool is_strong_c(const int* __restrict__ rp,
                                            const int* __restrict__ col,
                                            const unsigned char* __restrict__ strong,
                                            const signed char* __restrict__ state, int i, int m) {
  int p = find_in(col, rp[i], rp[i + 1], m);
  return p >= 0 && strong[p] && state[m] == kC;
}

__global__ void k_classical_count(int n, const int* __restrict__ rp, const int* __restrict__ col,
                                  const unsigned char* __restrict__ strong,
                                  const signed char* __restrict__ state, int* __restrict__ cnt) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  if (state[i] == kC) {
    cnt[i] = 1;
    return;
  }
  int c = 0;
  for (int e = rp[i]; e < rp[i + 1]; ++e)
    if (strong[e] && state[col[e]] == kC) ++c;
  cnt[i] = c;
}

// sign class of a_kk for opposite(): 0 when a_kk is zero or NaN (never
// opposite), 1 positive, 2 negative (one byte per entry in shared memory
// instead of the value)
__device__ __forceinline__ unsigned char sign_class(double d) {
  const unsigned long long ud = (unsigned long long)__double_as_longlong(d);
  const unsigned long long md = ud & 0x7fffffffffffffffull;
  if (md == 0 || md > 0x7ff0000000000000ull) return 0;
  return (unsigned char)(1 + (ud >> 63));
}

// opposite(a, d) with d given by its sign class
__device__ __forceinline__ bool opposite_class(double a, unsigned char dc) {
  const unsigned long long ua = (unsigned long long)__double_as_longlong(a);
  const unsigned long long ma = ua & 0x7fffffffffffffffull;
  return dc != 0 && ma != 0 && ma <= 0x7ff0000000000000ull &&
         (unsigned)(ua >> 63) != (unsigned)(dc - 1);
}

// an FP64 value is non-zero (either sign, or NaN), tested on its bits: FP64
// compares would take the FP64 pipe
__device__ __forceinline__ bool nonzero_bits(double v) {
  return ((unsigned long long)__double_as_longlong(v) << 1) != 0;
}

// rows longer than kClsShort are filled by a warp (k_classical_fill_warp)
constexpr int kClsShort = 8;
constexpr int kClsWarps = 4;

__global__ void k_classical_fill(int n, const int* __restrict__ rp, const int* __restrict__ col,
                                 const double* __restrict__ val, const int* __restrict__ dpos,
                                 const unsigned char* __restrict__ strong,
                                 const signed char* __restrict__ state,
                                 const int* __restrict__ cidx, const int* __restrict__ Prp,
                                 int* __restrict__ Pcol, double* __restrict__ Pval) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  if (rp[i + 1] - rp[i] > kClsShort) return;  // k_classical_fill_warp
  const int p0 = Prp[i], p1 = Prp[i + 1];
  if (state[i] == kC) {
    Pcol[p0] = cidx[i];
    Pval[p0] = 1.0;
    return;
  }
  if (p0 == p1) return;
  // columns (coarse numbering keeps the fine order) and numerator start a_ij
  int q = p0;
  for (int e = rp[i]; e < rp[i + 1]; ++e)
    if (strong[e] && state[col[e]] == kC) {
      Pcol[q] = cidx[col[e]];
      Pval[q] = val[e];
      ++q;
    }
  double denom = val[dpos[i]];
  for (int e = rp[i]; e < rp[i + 1]; ++e) {
    const int k = col[e];
    if (k == i) continue;
    if (!strong[e]) {
      denom = __dadd_rn(denom, val[e]);
      continue;
    }
    if (state[k] == kC) continue;
    const double akk = val[dpos[k]];
    double s = 0.0;
    for (int f = rp[k]; f < rp[k + 1]; ++f) {
      const int m = col[f];
      if (opposite(val[f], akk) && is_strong_c(rp, col, strong, state, i, m))
        s = __dadd_rn(s, val[f]);
    }
    if (!nonzero_bits(s)) {
      denom = __dadd_rn(denom, val[e]);
      continue;
    }
    const double t = __ddiv_rn(val[e], s);
    for (int f = rp[k]; f < rp[k + 1]; ++f) {
      const int m = col[f];
      if (opposite(val[f], akk) && is_strong_c(rp, col, strong, state, i, m)) {
        int slot = find_in(Pcol, p0, p1, cidx[m]);
        Pval[slot] = __dadd_rn(Pval[slot], __dmul_rn(t, val[f]));
      }
    }
  }
  for (int s = p0; s < p1; ++s) Pval[s] = __ddiv_rn(-Pval[s], denom);
}

// The same weights for long rows, one warp per row and the same arithmetic
// in the same order: the entries of row i are visited in order (the
// denominator is a sequential sum); for a strong F neighbour k the lanes
// evaluate the selection predicate over row k in parallel, the sum s runs
// over the selected values in column order (broadcast lane by lane), and
// each selected entry updates its own weight (distinct columns of row k hit
// distinct weights, so the per-weight order of updates is unchanged).
__global__ void __launch_bounds__(32 * kClsWarps) k_classical_fill_warp(
    int n, const int* __restrict__ rp, const int* __restrict__ col,
    const double* __restrict__ val, const int* __restrict__ dpos,
    const unsigned char* __restrict__ strong, const signed char* __restrict__ state,
    const int* __restrict__ cidx, const int* __restrict__ Prp, int* __restrict__ Pcol,
    double* __restrict__ Pval) {
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const unsigned below = (1u << lane) - 1u;
  for (int i = blockIdx.x * kClsWarps + w; i < n; i += gridDim.x * kClsWarps) {
    const int r0 = rp[i], r1 = rp[i + 1];
    if (r1 - r0 <= kClsShort) continue;  // uniform over the warp
    const int p0 = Prp[i], p1 = Prp[i + 1];
    if (state[i] == kC) {
      if (lane == 0) {
        Pcol[p0] = cidx[i];
        Pval[p0] = 1.0;
      }
      continue;
    }
    if (p0 == p1) continue;
    // columns and numerator start a_ij, in row order
    int q = p0;
    for (int e0 = r0; e0 < r1; e0 += 32) {
      const int e = e0 + lane;
      const bool sel = e < r1 && strong[e] && state[col[e]] == kC;
      const unsigned m = __ballot_sync(0xffffffffu, sel);
      if (sel) {
        Pcol[q + __popc(m & below)] = cidx[col[e]];
        Pval[q + __popc(m & below)] = val[e];
      }
      q += __popc(m);
    }
    __syncwarp();
    double denom = val[dpos[i]];
    for (int e = r0; e < r1; ++e) {
      const int k = col[e];
      if (k == i) continue;
      if (!strong[e]) {
        denom = __dadd_rn(denom, val[e]);
        continue;
      }
      if (state[k] == kC) continue;
      const double akk = val[dpos[k]];
      const int f1 = rp[k + 1];
      double sk = 0.0;
      for (int f0 = rp[k]; f0 < f1; f0 += 32) {
        const int f = f0 + lane;
        bool sel = false;
        double v = 0.0;
        if (f < f1) {
          v = val[f];
          sel = opposite(v, akk) && is_strong_c(rp, col, strong, state, i, col[f]);
        }
        const unsigned m = __ballot_sync(0xffffffffu, sel);
        for (unsigned mm = m; mm; mm &= mm - 1u) {
          const int src = __ffs(mm) - 1;
          sk = __dadd_rn(sk, __shfl_sync(0xffffffffu, v, src));
        }
        if (m == 0u) continue;
      }
      if (!nonzero_bits(sk)) {
        denom = __dadd_rn(denom, val[e]);
        continue;
      }
      const double t = __ddiv_rn(val[e], sk);
      for (int f0 = rp[k]; f0 < f1; f0 += 32) {
        const int f = f0 + lane;
        if (f < f1) {
          const int m = col[f];
          if (opposite(val[f], akk) && is_strong_c(rp, col, strong, state, i, m)) {
            const int slot = find_in(Pcol, p0, p1, cidx[m]);
            Pval[slot] = __dadd_rn(Pval[slot], __dmul_rn(t, val[f]));
          }
        }
      }
      __syncwarp();
    }
    for (int sI = p0 + lane; sI < p1; sI += 32) Pval[sI] = __ddiv_rn(-Pval[sI], denom);
    __syncwarp();
  }
}

// ---------------------------------------------------- extended+i interpolation
__global__ void k_extpi_ub(int n, const int* __restrict__ rp, const int* __restrict__ col,
                           const unsigned char* __restrict__ strong,
                           const signed char* __restrict__ state, int* __restrict__ ub) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  if (state[i] == kC) {
    ub[i] = 1;
    return;
  }
  int u = rp[i + 1] - rp[i];
  for (int e = rp[i]; e < rp[i + 1]; ++e) {
    int k = col[e];
    if (k != i && strong[e] && state[k] != kC) u += rp[k + 1] - rp[k];
  }
  ub[i] = u;
}

__device__ __forceinline__ void insert_unique(int* __restrict__ buf, int& u, int key) {
  int lo = 0, hi = u;
  while (lo < hi) {
    int mid = (lo + hi) >> 1;
    if (buf[mid] < key) lo = mid + 1;
    else hi = mid;
  }
  if (lo < u && buf[lo] == key) return;
  for (int q = u; q > lo; --q) buf[q] = buf[q - 1];
  buf[lo] = key;
  ++u;
}

// rows whose candidate bound exceeds kSetShort build their set with a warp
constexpr int kSetShort = 48;
constexpr int kSetWarps = 4;
constexpr int kSetCap = 1024;   // candidates sorted in shared memory (else serial)

// interpolatory set C^_i (sorted fine indices) of every F row with at most
// kSetShort candidates: one thread per row, insertion into a sorted list
__global__ void k_extpi_sets(int n, const int* __restrict__ rp, const int* __restrict__ col,
                             const unsigned char* __restrict__ strong,
                             const signed char* __restrict__ state, const int* __restrict__ off,
                             const int* __restrict__ ub, int* __restrict__ buf,
                             int* __restrict__ cnt) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  if (state[i] == kC) {
    cnt[i] = 1;
    return;
  }
  if (ub[i] > kSetShort) return;  // k_extpi_sets_warp
  int* b = buf + off[i];
  int u = 0;
  for (int e = rp[i]; e < rp[i + 1]; ++e) {
    const int k = col[e];
    if (k == i || !strong[e]) continue;
    if (state[k] == kC) {
      insert_unique(b, u, k);
    } else {
      for (int f = rp[k]; f < rp[k + 1]; ++f) {
        const int m = col[f];
        if (strong[f] && state[m] == kC && m != k) insert_unique(b, u, m);
      }
    }
  }
  cnt[i] = u;
}

// the same sets for F rows with more than kSetShort candidates, one warp per
// row: candidates (C neighbours, strong C neighbours of strong F neighbours)
// are appended to the row's buffer, then sorted (bitonic, shared memory) and
// made unique; the result is the same sorted set as the serial kernel's
__global__ void __launch_bounds__(32 * kSetWarps) k_extpi_sets_warp(
    int n, const int* __restrict__ rp, const int* __restrict__ col,
    const unsigned char* __restrict__ strong, const signed char* __restrict__ state,
    const int* __restrict__ off, const int* __restrict__ ub, int* __restrict__ buf,
    int* __restrict__ cnt) {
  __shared__ int s_list[kSetWarps][kSetCap];
  __shared__ int s_n[kSetWarps];
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const unsigned below = (1u << lane) - 1u;
  for (int i = blockIdx.x * kSetWarps + w; i < n; i += gridDim.x * kSetWarps) {
    if (state[i] == kC || ub[i] <= kSetShort) continue;  // uniform over the warp
    int* b = buf + off[i];
    if (lane == 0) s_n[w] = 0;
    __syncwarp();
    const int r0 = rp[i], r1 = rp[i + 1];
    for (int e0 = r0; e0 < r1; e0 += 32) {
      const int e = e0 + lane;
      const bool act = e < r1;
      const int k = act ? col[e] : -1;
      const bool st = act && k != i && strong[e];
      const bool isc = st && state[k] == kC;
      const unsigned cm = __ballot_sync(0xffffffffu, isc);
      int base = 0;
      if (lane == 0) {
        base = s_n[w];
        s_n[w] = base + __popc(cm);
      }
      base = __shfl_sync(0xffffffffu, base, 0);
      if (isc) b[base + __popc(cm & below)] = k;
      __syncwarp();
      unsigned fm = __ballot_sync(0xffffffffu, st && !isc);
      while (fm) {
        const int src = __ffs(fm) - 1;
        fm &= fm - 1u;
        const int kk = __shfl_sync(0xffffffffu, k, src);
        const int f1 = rp[kk + 1];
        for (int f0 = rp[kk]; f0 < f1; f0 += 32) {
          const int f = f0 + lane;
          const bool a2 = f < f1;
          const int m = a2 ? col[f] : -1;
          const bool c2 = a2 && m != kk && strong[f] && state[m] == kC;
          const unsigned mm = __ballot_sync(0xffffffffu, c2);
          int b2 = 0;
          if (lane == 0) {
            b2 = s_n[w];
            s_n[w] = b2 + __popc(mm);
          }
          b2 = __shfl_sync(0xffffffffu, b2, 0);
          if (c2) b[b2 + __popc(mm & below)] = m;
          __syncwarp();
        }
      }
    }
    __syncwarp();
    const int total = s_n[w];
    if (total > kSetCap) {
      // rare: the serial insertion rebuilds the set from the row itself
      if (lane == 0) {
        int u = 0;
        for (int e = r0; e < r1; ++e) {
          const int k = col[e];
          if (k == i || !strong[e]) continue;
          if (state[k] == kC) {
            insert_unique(b, u, k);
          } else {
            for (int f = rp[k]; f < rp[k + 1]; ++f) {
              const int m = col[f];
              if (strong[f] && state[m] == kC && m != k) insert_unique(b, u, m);
            }
          }
        }
        cnt[i] = u;
      }
      __syncwarp();
      continue;
    }
    int P = 32;
    while (P < total) P <<= 1;
    int* L = s_list[w];
    for (int t = lane; t < P; t += 32) L[t] = t < total ? b[t] : 0x7fffffff;
    __syncwarp();
    for (int k = 2; k <= P; k <<= 1) {
      for (int j = k >> 1; j > 0; j >>= 1) {
        for (int t = lane; t < P; t += 32) {
          const int u = t ^ j;
          if (u > t) {
            const int a = L[t], c = L[u];
            const bool up = (t & k) == 0;
            if ((a > c) == up) {
              L[t] = c;
              L[u] = a;
            }
          }
        }
        __syncwarp();
      }
    }
    // unique, in order
    int outn = 0;
    for (int t0 = 0; t0 < total; t0 += 32) {
      const int t = t0 + lane;
      const bool keep = t < total && (t == 0 || L[t] != L[t - 1]);
      const unsigned km = __ballot_sync(0xffffffffu, keep);
      if (keep) b[outn + __popc(km & below)] = L[t];
      outn += __popc(km);
    }
    if (lane == 0) cnt[i] = outn;
    __syncwarp();
  }
}

__device__ void extpi_fill_row_serial(int i, const int* __restrict__ rp, const int* __restrict__ col,
                             const double* __restrict__ val, const int* __restrict__ dpos,
                             const unsigned char* __restrict__ strong,
                             const signed char* __restrict__ state, const int* __restrict__ cidx,
                             const int* __restrict__ off, const int* __restrict__ buf,
                             const int* __restrict__ Prp, int* __restrict__ Pcol,
                             double* __restrict__ Pval) {
  const int p0 = Prp[i], p1 = Prp[i + 1];
  if (state[i] == kC) {
    Pcol[p0] = cidx[i];
    Pval[p0] = 1.0;
    return;
  }
  if (p0 == p1) return;
  const int* set = buf + off[i];
  const int ns = p1 - p0;
  for (int s = 0; s < ns; ++s) {
    Pcol[p0 + s] = cidx[set[s]];
    Pval[p0 + s] = 0.0;
  }
  for (int e = rp[i]; e < rp[i + 1]; ++e) {
    int s = find_in(set, 0, ns, col[e]);
    if (s >= 0) Pval[p0 + s] = val[e];
  }
  double denom = val[dpos[i]];
  for (int e = rp[i]; e < rp[i + 1]; ++e) {
    const int k = col[e];
    if (k == i) continue;
    if (strong[e] && state[k] != kC) {
      const double akk = val[dpos[k]];
      double s = 0.0;
      double aki = 0.0;
      bool has_ki = false;
      for (int f = rp[k]; f < rp[k + 1]; ++f) {
        const int m = col[f];
        if ((m == i || find_in(set, 0, ns, m) >= 0) && opposite(val[f], akk))
          s = __dadd_rn(s, val[f]);
        if (m == i) {
          aki = val[f];
          has_ki = true;
        }
      }
      if (!nonzero_bits(s)) {
        denom = __dadd_rn(denom, val[e]);
      } else {
        const double t = __ddiv_rn(val[e], s);
        if (has_ki && opposite(aki, akk)) denom = __dadd_rn(denom, __dmul_rn(t, aki));
        for (int f = rp[k]; f < rp[k + 1]; ++f) {
          const int m = col[f];
          if (!opposite(val[f], akk)) continue;
          int slot = find_in(set, 0, ns, m);
          if (slot >= 0) Pval[p0 + slot] = __dadd_rn(Pval[p0 + slot], __dmul_rn(t, val[f]));
        }
      }
    } else if (find_in(set, 0, ns, k) >= 0) {
      // interpolated directly
    } else {
      denom = __dadd_rn(denom, val[e]);
    }
  }
  for (int s = p0; s < p1; ++s) Pval[s] = __ddiv_rn(-Pval[s], denom);
}


// Warp-per-row extended+i fill with the arithmetic order of the serial form:
// lanes evaluate the strong F neighbours' sums s_k (and t_k = a_ik / s_k)
// independently, lane 0 accumulates the denominator over row i ascending,
// and each lane owns interpolation slots, adding t_k * ahat_km over k
// ascending. Rows longer than kFillMaxE use the serial form.
constexpr int kFillMaxE = 256;
constexpr int kFillWarps = 4;
constexpr int kFillShort = 8;  // rows up to this length: one thread per row

__global__ void k_extpi_fill_short(int n, const int* __restrict__ rp, const int* __restrict__ col,
                                   const double* __restrict__ val, const int* __restrict__ dpos,
                                   const unsigned char* __restrict__ strong,
                                   const signed char* __restrict__ state,
                                   const int* __restrict__ cidx, const int* __restrict__ off,
                                   const int* __restrict__ buf, const int* __restrict__ Prp,
                                   int* __restrict__ Pcol, double* __restrict__ Pval) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n || rp[i + 1] - rp[i] > kFillShort) return;
  extpi_fill_row_serial(i, rp, col, val, dpos, strong, state, cidx, off, buf, Prp, Pcol, Pval);
}

__global__ void __launch_bounds__(32 * kFillWarps) k_extpi_fill_warp(
    int n, const int* __restrict__ rp, const int* __restrict__ col,
    const double* __restrict__ val, const int* __restrict__ dpos,
    const unsigned char* __restrict__ strong, const signed char* __restrict__ state,
    const int* __restrict__ cidx, const int* __restrict__ off, const int* __restrict__ buf,
    const int* __restrict__ Prp, int* __restrict__ Pcol, double* __restrict__ Pval) {
  __shared__ double s_t[kFillWarps][kFillMaxE];
  __shared__ double s_term[kFillWarps][kFillMaxE];
  __shared__ unsigned char s_flag[kFillWarps][kFillMaxE];
  __shared__ unsigned char s_akc[kFillWarps][kFillMaxE];
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int i = blockIdx.x * kFillWarps + w;
  if (i >= n) return;
  if (rp[i + 1] - rp[i] <= kFillShort) return;  // done by k_extpi_fill_short
  const int p0 = Prp[i], p1 = Prp[i + 1];
  if (state[i] == kC) {
    if (lane == 0) {
      Pcol[p0] = cidx[i];
      Pval[p0] = 1.0;
    }
    return;
  }
  if (p0 == p1) return;
  const int r0 = rp[i], r1 = rp[i + 1];
  if (r1 - r0 > kFillMaxE) {
    if (lane == 0)
      extpi_fill_row_serial(i, rp, col, val, dpos, strong, state, cidx, off, buf, Prp, Pcol, Pval);
    return;
  }
  const int* set = buf + off[i];
  const int ns = p1 - p0;
  double* t = s_t[w];
  double* term = s_term[w];
  unsigned char* flag = s_flag[w];
  unsigned char* akc = s_akc[w];
  // flags: 0 skip (diagonal or interpolated directly), 1 lump a_ie into the
  // denominator, 3 strong F neighbour with t_k (term = t_k ahat_ki or 0)
  for (int e = r0 + lane; e < r1; e += 32) {
    const int q = e - r0;
    const int k = col[e];
    unsigned char fl = 0, kc = 0;
    double tk = 0.0, tm = 0.0;
    if (k == i) {
      fl = 0;
    } else if (strong[e] && state[k] != kC) {
      kc = sign_class(val[dpos[k]]);
      double sk = 0.0, aki = 0.0;
      bool has_ki = false;
      for (int f = rp[k]; f < rp[k + 1]; ++f) {
        const int m = col[f];
        const double v = val[f];
        // the sign test first: it skips most of the set searches
        if (opposite_class(v, kc) && (m == i || find_in(set, 0, ns, m) >= 0)) sk = __dadd_rn(sk, v);
        if (m == i) {
          aki = v;
          has_ki = true;
        }
      }
      if (!nonzero_bits(sk)) {
        fl = 1;
      } else {
        fl = 3;
        tk = __ddiv_rn(val[e], sk);
        if (has_ki && opposite_class(aki, kc)) tm = __dmul_rn(tk, aki);
      }
    } else if (find_in(set, 0, ns, k) >= 0) {
      fl = 0;
    } else {
      fl = 1;
    }
    flag[q] = fl;
    t[q] = tk;
    term[q] = tm;
    akc[q] = kc;
  }
  __syncwarp();
  double denom = 0.0;
  if (lane == 0) {
    denom = val[dpos[i]];
    for (int e = r0; e < r1; ++e) {
      const int q = e - r0;
      if (flag[q] == 1) denom = __dadd_rn(denom, val[e]);
      else if (flag[q] == 3 && nonzero_bits(term[q])) denom = __dadd_rn(denom, term[q]);
    }
  }
  denom = __shfl_sync(0xffffffffu, denom, 0);
  for (int sl = lane; sl < ns; sl += 32) {
    const int m = set[sl];
    const int pe = find_in(col, r0, r1, m);
    double num = pe >= 0 ? val[pe] : 0.0;
    for (int e = r0; e < r1; ++e) {
      const int q = e - r0;
      if (flag[q] != 3) continue;
      const int k = col[e];
      const int f = find_in(col, rp[k], rp[k + 1], m);
      if (f >= 0 && opposite_class(val[f], akc[q])) num = __dadd_rn(num, __dmul_rn(t[q], val[f]));
    }
    Pcol[p0 + sl] = cidx[m];
    Pval[p0 + sl] = __ddiv_rn(-num, denom);
  }
}

// --------------------------------------------------- interpolation truncation
constexpr int kPmaxLimit = 16;

__global__ void k_trunc_count(int n, const int* __restrict__ Prp, int pmax, int* __restrict__ cnt) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int len = Prp[i + 1] - Prp[i];
  cnt[i] = len < pmax ? len : pmax;
}

// keep the pmax largest |w| (ties to the lower column) and scale them by
// (sum of all) / (sum of kept), sums over the row ascending from 0.0
__global__ void k_trunc_fill(int n, const int* __restrict__ Prp, const int* __restrict__ Pcol,
                             const double* __restrict__ Pval, int pmax,
                             const int* __restrict__ Trp, int* __restrict__ Tcol,
                             double* __restrict__ Tval) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int p0 = Prp[i], p1 = Prp[i + 1], len = p1 - p0, t0 = Trp[i];
  if (len <= pmax) {
    for (int q = 0; q < len; ++q) {
      Tcol[t0 + q] = Pcol[p0 + q];
      Tval[t0 + q] = Pval[p0 + q];
    }
    return;
  }
  int keep[kPmaxLimit];
  int nk = 0;
  for (int r = 0; r < pmax; ++r) {
    int best = -1;
    double bw = -1.0;
    for (int q = 0; q < len; ++q) {
      bool taken = false;
      for (int u = 0; u < nk; ++u) taken |= keep[u] == q;
      if (taken) continue;
      const double a = fabs(Pval[p0 + q]);
      if (a > bw) {  // first maximum in column order wins ties
        bw = a;
        best = q;
      }
    }
    keep[nk++] = best;
  }
  for (int a = 1; a < nk; ++a) {  // ascending position = ascending column
    int v = keep[a], b = a - 1;
    while (b >= 0 && keep[b] > v) {
      keep[b + 1] = keep[b];
      --b;
    }
    keep[b + 1] = v;
  }
  double s_all = 0.0, s_keep = 0.0;
  for (int q = 0; q < len; ++q) s_all = __dadd_rn(s_all, Pval[p0 + q]);
  for (int u = 0; u < nk; ++u) s_keep = __dadd_rn(s_keep, Pval[p0 + keep[u]]);
  const double f = s_keep != 0.0 ? __ddiv_rn(s_all, s_keep) : 1.0;
  for (int u = 0; u < nk; ++u) {
    Tcol[t0 + u] = Pcol[p0 + keep[u]];
    Tval[t0 + u] = s_keep != 0.0 ? __dmul_rn(Pval[p0 + keep[u]], f) : Pval[p0 + keep[u]];
  }
}

// ------------------------------------------------------------- transpose
__global__ void k_count_cols(int n, const int* __restrict__ rp, const int* __restrict__ col,
                             int* __restrict__ cnt) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  for (int e = rp[i]; e < rp[i + 1]; ++e) atomicAdd(&cnt[col[e]], 1);
}

__global__ void k_fill_transpose(int n, const int* __restrict__ rp, const int* __restrict__ col,
                                 const double* __restrict__ val, const int* __restrict__ Trp,
                                 int* __restrict__ cursor, int* __restrict__ Tcol,
                                 double* __restrict__ Tval) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  for (int e = rp[i]; e < rp[i + 1]; ++e) {
    int c = col[e];
    int q = Trp[c] + atomicAdd(&cursor[c], 1);
    Tcol[q] = i;
    Tval[q] = val[e];
  }
}

// Rows of [rp] with distinct columns, reordered by column from (col, val)
// into (ocol, oval): each entry goes to its rank, the number of entries of
// its row with a smaller column. One warp per row of more than 32 entries
// (the lanes rank the row's entries in parallel), one thread per shorter
// row.
__global__ void k_rank_rows(int n, const int* __restrict__ rp, const int* __restrict__ col,
                            const double* __restrict__ val, int* __restrict__ ocol,
                            double* __restrict__ oval) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int r0 = rp[i], r1 = rp[i + 1];
  if (r1 - r0 > 32) return;  // k_rank_rows_warp
  for (int e = r0; e < r1; ++e) {
    const int c = col[e];
    int rank = 0;
    for (int f = r0; f < r1; ++f) rank += col[f] < c;
    ocol[r0 + rank] = c;
    oval[r0 + rank] = val[e];
  }
}

__global__ void k_rank_rows_warp(int n, const int* __restrict__ rp, const int* __restrict__ col,
                                 const double* __restrict__ val, int* __restrict__ ocol,
                                 double* __restrict__ oval) {
  const int lane = threadIdx.x & 31;
  const int i = (int)((blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5);
  if (i >= n) return;
  const int r0 = rp[i], r1 = rp[i + 1];
  if (r1 - r0 <= 32) return;  // k_rank_rows
  for (int e = r0 + lane; e < r1; e += 32) {
    const int c = col[e];
    int rank = 0;
    for (int f = r0; f < r1; ++f) rank += col[f] < c;
    ocol[r0 + rank] = c;
    oval[r0 + rank] = val[e];
  }
}

// ------------------------------------------------------------- SpGEMM C = A B
// Upper bound (product count) of every row of C = A B; rows too long for
// the thread-per-row kernel are listed for the warp kernel (kSpShort < ub <
// kSpCap) or the block kernel (ub >= kSpCap), so those visit only their rows.
// The list order is not deterministic; each row's result is.
__global__ void k_spgemm_ub(int n, const int* __restrict__ Arp, const int* __restrict__ Acol,
                            const int* __restrict__ Brp, int* __restrict__ ub,
                            int* __restrict__ wlist, int* __restrict__ blist,
                            int* __restrict__ counts);

// Row i of C: products a_ik * b_kj in ascending k (row i of A) then ascending
// j (row k of B); each column's sum starts at 0.0 and adds them in that
// order. Columns kept sorted by insertion. This thread-per-row form takes
// the rows with at most kSpShort products and more than kSpMerge entries of
// A (k_spgemm_rows_merge the rows with fewer, k_spgemm_rows_warp the rows
// with more products).
constexpr int kSpShort = 96;
constexpr int kSpMerge = 8;  // rows of A with at most this many entries: k-way merge

// The rows of k_spgemm_rows whose row of A has at most kSpMerge entries (a
// 7-point operator times P): a merge of the (sorted) rows of B of the row's
// entries, heads in registers. Each column comes out once, in order, its
// products added in ascending entry order from 0.0 (the canonical order),
// with no sorted-list insertion in memory. A kernel of its own: its
// registers would cost the insertion form occupancy.
__global__ void k_spgemm_rows_merge(int n, const int* __restrict__ Arp,
                                    const int* __restrict__ Acol, const double* __restrict__ Aval,
                                    const int* __restrict__ Brp, const int* __restrict__ Bcol,
                                    const double* __restrict__ Bval, const int* __restrict__ off,
                                    const int* __restrict__ ub, int* __restrict__ ccol,
                                    double* __restrict__ cval, int* __restrict__ cnt) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n || ub[i] > kSpShort) return;
  const int a0 = Arp[i], na = Arp[i + 1] - a0;
  if (na > kSpMerge) return;
  int* cc = ccol + off[i];
  double* cv = cval + off[i];
  // a merge of the (sorted) rows of B of the row's entries, heads in
  // registers: each column comes out once, in order, its products added
  // in ascending entry order from 0.0 (the canonical order), with no
  // sorted-list insertion in memory (rows of a 7-point operator times P)
  int f[kSpMerge], fe[kSpMerge], hc[kSpMerge];
  double av[kSpMerge];
#pragma unroll
  for (int k = 0; k < kSpMerge; ++k) {
    f[k] = fe[k] = 0;
    hc[k] = 0x7fffffff;
    av[k] = 0.0;
    if (k < na) {
      const int kk = Acol[a0 + k];
      av[k] = Aval[a0 + k];
      f[k] = Brp[kk];
      fe[k] = Brp[kk + 1];
      if (f[k] < fe[k]) hc[k] = Bcol[f[k]];
    }
  }
  int u = 0;
  while (true) {
    int m = 0x7fffffff;
#pragma unroll
    for (int k = 0; k < kSpMerge; ++k) m = min(m, hc[k]);
    if (m == 0x7fffffff) break;
    double sum = 0.0;
#pragma unroll
    for (int k = 0; k < kSpMerge; ++k)
      if (hc[k] == m) {
        sum = __dadd_rn(sum, __dmul_rn(av[k], Bval[f[k]]));
        ++f[k];
        hc[k] = f[k] < fe[k] ? Bcol[f[k]] : 0x7fffffff;
      }
    cc[u] = m;
    cv[u] = sum;
    ++u;
  }
  cnt[i] = u;
}

__global__ void k_spgemm_rows(int n, const int* __restrict__ Arp, const int* __restrict__ Acol,
                              const double* __restrict__ Aval, const int* __restrict__ Brp,
                              const int* __restrict__ Bcol, const double* __restrict__ Bval,
                              const int* __restrict__ off, const int* __restrict__ ub,
                              int* __restrict__ ccol, double* __restrict__ cval,
                              int* __restrict__ cnt) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n || ub[i] > kSpShort) return;
  int* cc = ccol + off[i];
  double* cv = cval + off[i];
  if (Arp[i + 1] - Arp[i] <= kSpMerge) return;  // k_spgemm_rows_merge
  int u = 0;
  for (int e = Arp[i]; e < Arp[i + 1]; ++e) {
    const int k = Acol[e];
    const double a = Aval[e];
    for (int f = Brp[k]; f < Brp[k + 1]; ++f) {
      const int j = Bcol[f];
      const double prod = __dmul_rn(a, Bval[f]);
      int lo = 0, hi = u;
      while (lo < hi) {
        int mid = (lo + hi) >> 1;
        if (cc[mid] < j) lo = mid + 1;
        else hi = mid;
      }
      if (lo < u && cc[lo] == j) {
        cv[lo] = __dadd_rn(cv[lo], prod);
      } else {
        for (int q = u; q > lo; --q) {
          cc[q] = cc[q - 1];
          cv[q] = cv[q - 1];
        }
        cc[lo] = j;
        cv[lo] = __dadd_rn(0.0, prod);
        ++u;
      }
    }
  }
  cnt[i] = u;
}

// Products whose result has few columns (m <= kDenseCap: the Galerkin
// products of coarse levels): one warp per row accumulates into a dense
// shared-memory row. The entries of row i of A are visited in order and the
// lanes split row k of B (whose columns are distinct), so every column's sum
// still starts at 0.0 and adds its products in ascending k: the canonical
// order. Touched columns are flagged and compacted in column order.
constexpr int kDenseCap = 2048;
constexpr int kDenseWarps = 4;
constexpr size_t kDenseSmem = (size_t)kDenseWarps * kDenseCap * (sizeof(double) + 1);

__global__ void __launch_bounds__(32 * kDenseWarps) k_spgemm_dense(
    int n, int m, const int* __restrict__ Arp, const int* __restrict__ Acol,
    const double* __restrict__ Aval, const int* __restrict__ Brp, const int* __restrict__ Bcol,
    const double* __restrict__ Bval, const int* __restrict__ off, int* __restrict__ ccol,
    double* __restrict__ cval, int* __restrict__ cnt) {
  extern __shared__ double s_dense[];
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const unsigned below = (1u << lane) - 1u;
  double* acc = s_dense + (size_t)w * m;
  unsigned char* flg = reinterpret_cast<unsigned char*>(s_dense + (size_t)kDenseWarps * m) +
                       (size_t)w * m;
  for (int i = blockIdx.x * kDenseWarps + w; i < n; i += gridDim.x * kDenseWarps) {
    for (int j = lane; j < m; j += 32) {
      acc[j] = 0.0;
      flg[j] = 0;
    }
    __syncwarp();
    for (int e = Arp[i]; e < Arp[i + 1]; ++e) {
      const int k = Acol[e];
      const double a = Aval[e];
      for (int f = Brp[k] + lane; f < Brp[k + 1]; f += 32) {
        const int j = Bcol[f];
        acc[j] = __dadd_rn(acc[j], __dmul_rn(a, Bval[f]));
        flg[j] = 1;
      }
      __syncwarp();
    }
    int* cc = ccol + off[i];
    double* cv = cval + off[i];
    int base = 0;
    for (int j0 = 0; j0 < m; j0 += 32) {
      const int j = j0 + lane;
      const bool has = j < m && flg[j];
      const unsigned hm = __ballot_sync(0xffffffffu, has);
      if (has) {
        cc[base + __popc(hm & below)] = j;
        cv[base + __popc(hm & below)] = acc[j];
      }
      base += __popc(hm);
    }
    if (lane == 0) cnt[i] = base;
    __syncwarp();
  }
}

// Warp-per-row variant of k_spgemm_rows with the same summation order. The
// warp walks row i of A in ascending k; for each k its lanes take distinct
// entries of row k of B (whose columns are distinct), so no two lanes update
// the same column at once, and a __syncwarp between k's keeps every
// column's additions in ascending k, each sum starting at 0.0: the canonical
// order. Columns find their accumulator through an open-addressing hash
// table in shared memory (linear probing, at least twice as many slots as
// products, so an empty slot always exists); the distinct columns are then
// sorted by a warp bitonic sort of (column << 32 | slot) keys and written
// in ascending order. Each batch of 32 entries of row i of A (column k,
// value, row k's extent in B) is loaded by the warp at once, so a step over
// k waits for one round trip (row k of B), not three. Rows with fewer than
// kSpMid products use tables of kSpMid slots (four warps per block), rows
// up to kSpCap tables of kSpCap slots (two warps); longer rows go to the
// block kernel.
constexpr int kSpMid = 512;
constexpr int kSpCap = 1024;

__global__ void k_spgemm_ub(int n, const int* __restrict__ Arp, const int* __restrict__ Acol,
                            const int* __restrict__ Brp, int* __restrict__ ub,
                            int* __restrict__ wlist, int* __restrict__ blist,
                            int* __restrict__ counts) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  int u = 0;
  for (int e = Arp[i]; e < Arp[i + 1]; ++e) {
    int k = Acol[e];
    u += Brp[k + 1] - Brp[k];
  }
  ub[i] = u;
  if (u >= kSpCap) blist[atomicAdd(&counts[1], 1)] = i;
  else if (u >= kSpMid) wlist[n - 1 - atomicAdd(&counts[2], 1)] = i;
  else if (u > kSpShort) wlist[atomicAdd(&counts[0], 1)] = i;
}

__device__ void spgemm_row_serial(int i, const int* __restrict__ Arp, const int* __restrict__ Acol,
                                  const double* __restrict__ Aval, const int* __restrict__ Brp,
                                  const int* __restrict__ Bcol, const double* __restrict__ Bval,
                                  int* __restrict__ cc, double* __restrict__ cv, int* __restrict__ cnt) {
  int u = 0;
  for (int e = Arp[i]; e < Arp[i + 1]; ++e) {
    const int k = Acol[e];
    const double a = Aval[e];
    for (int f = Brp[k]; f < Brp[k + 1]; ++f) {
      const int j = Bcol[f];
      const double prod = __dmul_rn(a, Bval[f]);
      int lo = 0, hi = u;
      while (lo < hi) {
        int mid = (lo + hi) >> 1;
        if (cc[mid] < j) lo = mid + 1;
        else hi = mid;
      }
      if (lo < u && cc[lo] == j) {
        cv[lo] = __dadd_rn(cv[lo], prod);
      } else {
        for (int q = u; q > lo; --q) {
          cc[q] = cc[q - 1];
          cv[q] = cv[q - 1];
        }
        cc[lo] = j;
        cv[lo] = __dadd_rn(0.0, prod);
        ++u;
      }
    }
  }
  cnt[i] = u;
}

// one warp: row i of C = A B through a shared-memory hash table of
// 2^k >= 2 ex slots (hkey/hval, at most `tcap`), then the distinct columns
// sorted in skey (capacity tcap)
__device__ void spgemm_row_hash(int i, int ex, int lane, int tcap, const int* __restrict__ Arp,
                                const int* __restrict__ Acol, const double* __restrict__ Aval,
                                const int* __restrict__ Brp, const int* __restrict__ Bcol,
                                const double* __restrict__ Bval, int* hkey, double* hval,
                                unsigned long long* skey, int* __restrict__ cc,
                                double* __restrict__ cv, int* __restrict__ cnt) {
  int bits = 5;
  while ((1 << bits) < 2 * ex && (1 << bits) < tcap) ++bits;
  const int cap = 1 << bits;
  const unsigned below = (1u << lane) - 1u;
  for (int q = lane; q < cap; q += 32) hkey[q] = -1;
  __syncwarp();
  // 1. accumulate in canonical order: every column's sum starts at 0.0 and
  // takes its products in ascending e. Rows of fewer than kSpMid products
  // whose rows of B are short (fewer than 16 products per entry of A on
  // average, as in A P; measured faster there, slower on the rows of
  // kSpMid-kSpCap products of R (A P)) take the
  // next 32 products of the row in sequence order per step (entry e of row i
  // of A, then the row of B): lanes claim their column's slot, and lanes of
  // one step that share a column (at most one product per entry e, so lane
  // order is entry order) are added by the lowest of them in lane order onto
  // the sum of the earlier steps. Other rows take one entry of A per step,
  // its row of B split over the lanes (distinct columns).
  for (int q = lane; q < cap; q += 32) hval[q] = 0.0;
  __syncwarp();
  double* sprod = reinterpret_cast<double*>(skey);  // 32 staged products
  const int a0 = Arp[i], a1 = Arp[i + 1];
  if (tcap <= kSpMid && ex < 16 * (a1 - a0)) {
    for (int e0 = a0; e0 < a1; e0 += 32) {
      const int e = e0 + lane;
      double a = 0.0;
      int fb = 0, len = 0;
      if (e < a1) {
        const int k = Acol[e];
        a = Aval[e];
        fb = Brp[k];
        len = Brp[k + 1] - fb;
      }
      int incl = len;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += y;
      }
      const int excl = incl - len;
      const int total = __shfl_sync(0xffffffffu, incl, 31);
      for (int p0 = 0; p0 < total; p0 += 32) {
        const int p = p0 + lane;
        // the entry holding position p: the last lane with excl <= p
        int lo = 0;
#pragma unroll
        for (int step = 16; step > 0; step >>= 1) {
          const int cand = lo + step;
          if (__shfl_sync(0xffffffffu, excl, cand) <= p) lo = cand;
        }
        const int se = __shfl_sync(0xffffffffu, excl, lo);
        const int sf = __shfl_sync(0xffffffffu, fb, lo);
        const double sa = __shfl_sync(0xffffffffu, a, lo);
        int slot = -1 - lane;  // distinct for lanes without a product
        double prod = 0.0;
        if (p < total) {
          const int f = sf + (p - se);
          const int j = Bcol[f];
          prod = __dmul_rn(sa, Bval[f]);
          unsigned h = ((unsigned)j * 0x9E3779B1u) >> (32 - bits);
          for (int probe = 0; probe < cap; ++probe) {
            const int prev = atomicCAS(&hkey[h], -1, j);
            if (prev == -1 || prev == j) {
              slot = (int)h;
              break;
            }
            h = (h + 1) & (unsigned)(cap - 1);
          }
        }
        sprod[lane] = prod;
        const unsigned grp = __match_any_sync(0xffffffffu, slot);
        __syncwarp();
        if (slot >= 0 && (grp & below) == 0) {
          double v = hval[slot];
          for (unsigned g = grp; g; g &= g - 1u) v = __dadd_rn(v, sprod[__ffs(g) - 1]);
          hval[slot] = v;
        }
        __syncwarp();
      }
    }
  } else {
    for (int e0 = a0; e0 < a1; e0 += 32) {
      const int e = e0 + lane;
      double a = 0.0;
      int fb = 0, fe = 0;
      if (e < a1) {
        const int k = Acol[e];
        a = Aval[e];
        fb = Brp[k];
        fe = Brp[k + 1];
      }
      const int ne = min(32, a1 - e0);
      for (int t = 0; t < ne; ++t) {
        const double at = __shfl_sync(0xffffffffu, a, t);
        const int f0 = __shfl_sync(0xffffffffu, fb, t);
        const int f1 = __shfl_sync(0xffffffffu, fe, t);
        for (int f = f0 + lane; f < f1; f += 32) {
          const int j = Bcol[f];
          const double prod = __dmul_rn(at, Bval[f]);
          unsigned h = ((unsigned)j * 0x9E3779B1u) >> (32 - bits);
          for (int probe = 0; probe < cap; ++probe) {
            const int prev = atomicCAS(&hkey[h], -1, j);
            if (prev == -1 || prev == j) {
              hval[h] = __dadd_rn(hval[h], prod);
              break;
            }
            h = (h + 1) & (unsigned)(cap - 1);
          }
        }
        __syncwarp();
      }
    }
  }
  // 2. compact the occupied slots as (column << 32 | slot) keys
  int d = 0;
  for (int q0 = 0; q0 < cap; q0 += 32) {
    const int q = q0 + lane;
    const int c = hkey[q];
    const unsigned m = __ballot_sync(0xffffffffu, c >= 0);
    if (c >= 0)
      skey[d + __popc(m & below)] = ((unsigned long long)(unsigned)c << 32) | (unsigned)q;
    d += __popc(m);
  }
  int P = 1;
  while (P < d) P <<= 1;
  for (int q = d + lane; q < P; q += 32) skey[q] = ~0ull;
  __syncwarp();
  // 3. bitonic sort of the keys (ascending)
  for (int size = 2; size <= P; size <<= 1) {
    for (int stride = size >> 1; stride > 0; stride >>= 1) {
      for (int t = lane; t < (P >> 1); t += 32) {
        const int lo = 2 * stride * (t / stride) + (t % stride);
        const int hi = lo + stride;
        const bool up = (lo & size) == 0;
        const unsigned long long x = skey[lo], y = skey[hi];
        if ((x > y) == up) {
          skey[lo] = y;
          skey[hi] = x;
        }
      }
      __syncwarp();
    }
  }
  // 4. columns in ascending order with their sums
  for (int r = lane; r < d; r += 32) {
    const unsigned long long kk = skey[r];
    cc[r] = (int)(kk >> 32);
    cv[r] = hval[(unsigned)(kk & 0xffffffffu)];
  }
  if (lane == 0) cnt[i] = d;
}

// rows listed for the warp kernel: tables of CAP slots, WARPS warps per block
// (static shared memory: 20 CAP bytes per warp); rows [first, first + count)
// of the list, count read from the device, in list order
template <int CAP, int WARPS>
__global__ void __launch_bounds__(32 * WARPS) k_spgemm_rows_warp(
    int n, const int* __restrict__ Arp, const int* __restrict__ Acol,
    const double* __restrict__ Aval, const int* __restrict__ Brp, const int* __restrict__ Bcol,
    const double* __restrict__ Bval, const int* __restrict__ off, const int* __restrict__ ub,
    const int* __restrict__ wlist, const int* __restrict__ counts, int which,
    int* __restrict__ ccol, double* __restrict__ cval, int* __restrict__ cnt) {
  __shared__ int s_hkey[WARPS][CAP];
  __shared__ double s_hval[WARPS][CAP];
  __shared__ unsigned long long s_skey[WARPS][CAP];
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  // list 0 fills wlist from the front, list 2 from the back
  const int count = counts[which];
  for (int t = blockIdx.x * WARPS + w; t < count; t += gridDim.x * WARPS) {
    const int i = which == 0 ? wlist[t] : wlist[n - 1 - t];
    const int ex = ub[i];
    spgemm_row_hash(i, ex, lane, CAP, Arp, Acol, Aval, Brp, Bcol, Bval, s_hkey[w], s_hval[w],
                    s_skey[w], ccol + off[i], cval + off[i], cnt);
    __syncwarp();
  }
}

// rows with ex >= kSpCap: one 512-thread block per row (one block per SM)
// with kSpBig products in dynamic shared memory. Every warp stages the
// products of its share of row i of A (lanes over the row of B, coalesced)
// at their canonical sequence positions; a block bitonic sort orders the
// (column, position) keys; a block scan lists the column runs, and one
// thread per run adds it up in sequence order. Rows beyond kSpBig are summed
// serially.
constexpr int kSpBig = 8192;
constexpr int kSpBigThreads = 512;
constexpr int kSpBigWarps = kSpBigThreads / 32;
constexpr size_t kSpBigSmem =
    (size_t)kSpBig * (sizeof(unsigned long long) + sizeof(double)) + (kSpBig + 1) * sizeof(int);

// exclusive scan of x over the block; *total = the block's sum. s_w holds
// kSpBigWarps + 1 ints; the block must not touch it between calls without a
// barrier (the function ends with one).
__device__ __forceinline__ int block_scan_excl(int x, int* s_w, int* total) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  int incl = x;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int y = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += y;
  }
  if (lane == 31) s_w[warp] = incl;
  __syncthreads();
  if (warp == 0) {
    const int v = lane < kSpBigWarps ? s_w[lane] : 0;
    int iv = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int y = __shfl_up_sync(0xffffffffu, iv, o);
      if (lane >= o) iv += y;
    }
    if (lane < kSpBigWarps) s_w[lane] = iv - v;
    if (lane == 31) s_w[kSpBigWarps] = iv;
  }
  __syncthreads();
  const int r = s_w[warp] + incl - x;
  *total = s_w[kSpBigWarps];
  __syncthreads();
  return r;
}

__global__ void __launch_bounds__(kSpBigThreads) k_spgemm_rows_big(
    int n, const int* __restrict__ Arp, const int* __restrict__ Acol,
    const double* __restrict__ Aval, const int* __restrict__ Brp, const int* __restrict__ Bcol,
    const double* __restrict__ Bval, const int* __restrict__ off, const int* __restrict__ ub,
    const int* __restrict__ blist, const int* __restrict__ counts,
    int* __restrict__ ccol, double* __restrict__ cval, int* __restrict__ cnt) {
  extern __shared__ unsigned long long s_big[];
  unsigned long long* key = s_big;
  double* val = reinterpret_cast<double*>(s_big + kSpBig);
  int* start = reinterpret_cast<int*>(val + kSpBig);
  __shared__ int s_w[kSpBigWarps + 1];
  __shared__ int s_ak[kSpBigThreads], s_aoff[kSpBigThreads];
  __shared__ double s_aa[kSpBigThreads];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int count = counts[1];
  for (int t = blockIdx.x; t < count; t += gridDim.x) {
    const int i = blist[t];
    const int ex = ub[i];  // uniform over the block
    int* cc = ccol + off[i];
    double* cv = cval + off[i];
    if (ex > kSpBig) {
      if (tid == 0) spgemm_row_serial(i, Arp, Acol, Aval, Brp, Bcol, Bval, cc, cv, cnt);
      __syncthreads();
      continue;
    }
    // 1. products at their canonical positions (entry e of row i of A, then
    // the row of B in order), kSpBigThreads entries of A at a time
    const int a0 = Arp[i], a1 = Arp[i + 1];
    int base = 0;
    for (int c0 = a0; c0 < a1; c0 += kSpBigThreads) {
      const int e = c0 + tid;
      int k = 0, len = 0;
      double a = 0.0;
      if (e < a1) {
        k = Acol[e];
        a = Aval[e];
        len = Brp[k + 1] - Brp[k];
      }
      int total = 0;
      const int ex_off = block_scan_excl(len, s_w, &total);
      s_ak[tid] = k;
      s_aa[tid] = a;
      s_aoff[tid] = base + ex_off;
      __syncthreads();
      const int nc = min(kSpBigThreads, a1 - c0);
      for (int q = warp; q < nc; q += kSpBigWarps) {
        const int kk = s_ak[q];
        const double aq = s_aa[q];
        const int fb = Brp[kk], fe = Brp[kk + 1];
        const int pb = s_aoff[q] - fb;
        for (int f = fb + lane; f < fe; f += 32) {
          const int pidx = pb + f;
          key[pidx] = ((unsigned long long)(unsigned)Bcol[f] << 32) | (unsigned)pidx;
          val[pidx] = __dmul_rn(aq, Bval[f]);
        }
      }
      base += total;
      __syncthreads();
    }
    int P = 1;
    while (P < ex) P <<= 1;
    for (int q = ex + tid; q < P; q += kSpBigThreads) key[q] = ~0ull;
    __syncthreads();
    // 2. block bitonic sort
    for (int size = 2; size <= P; size <<= 1) {
      for (int stride = size >> 1; stride > 0; stride >>= 1) {
        for (int u = tid; u < (P >> 1); u += kSpBigThreads) {
          const int lo = 2 * stride * (u / stride) + (u % stride);
          const int hi = lo + stride;
          const bool up = (lo & size) == 0;
          const unsigned long long x = key[lo], y = key[hi];
          if ((x > y) == up) {
            key[lo] = y;
            key[hi] = x;
          }
        }
        __syncthreads();
      }
    }
    // 3. the start of every column run
    int nrun = 0;
    for (int q0 = 0; q0 < ex; q0 += kSpBigThreads) {
      const int q = q0 + tid;
      int st = 0;
      if (q < ex) st = (q == 0) || ((key[q] >> 32) != (key[q - 1] >> 32));
      int total = 0;
      const int r = block_scan_excl(st, s_w, &total);
      if (st) start[nrun + r] = q;
      nrun += total;
    }
    if (tid == 0) start[nrun] = ex;
    __syncthreads();
    // 4. one thread per run, summed in sequence order
    for (int r = tid; r < nrun; r += kSpBigThreads) {
      const int q0 = start[r], q1 = start[r + 1];
      double sum = 0.0;
      for (int q = q0; q < q1; ++q) sum = __dadd_rn(sum, val[(unsigned)(key[q] & 0xffffffffu)]);
      cc[r] = (int)(key[q0] >> 32);
      cv[r] = sum;
    }
    if (tid == 0) cnt[i] = nrun;
    __syncthreads();
  }
}

// numeric-only C = A B on a known pattern (same canonical order)
__global__ void k_spgemm_numeric(int n, const int* __restrict__ Arp, const int* __restrict__ Acol,
                                 const double* __restrict__ Aval, const int* __restrict__ Brp,
                                 const int* __restrict__ Bcol, const double* __restrict__ Bval,
                                 const int* __restrict__ Crp, const int* __restrict__ Ccol,
                                 double* __restrict__ Cval) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int c0 = Crp[i], c1 = Crp[i + 1];
  for (int q = c0; q < c1; ++q) Cval[q] = 0.0;
  for (int e = Arp[i]; e < Arp[i + 1]; ++e) {
    const int k = Acol[e];
    const double a = Aval[e];
    for (int f = Brp[k]; f < Brp[k + 1]; ++f) {
      const int q = find_in(Ccol, c0, c1, Bcol[f]);
      Cval[q] = __dadd_rn(Cval[q], __dmul_rn(a, Bval[f]));
    }
  }
}

// rows of C from their slots at off[i] to the compact CSR: L lanes per row
// (about two entries per lane on average), so that a warp's copies are a
// few contiguous runs rather than 32 scattered rows
template <int L>
__global__ void k_spgemm_compact(int n, const int* __restrict__ off,
                                 const int* __restrict__ ccol, const double* __restrict__ cval,
                                 const int* __restrict__ Crp, int* __restrict__ Ccol,
                                 double* __restrict__ Cval) {
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const int i = (int)(t / L), lane = (int)(t % L);
  if (i >= n) return;
  const int o = off[i], c0 = Crp[i], len = Crp[i + 1] - c0;
  for (int e = lane; e < len; e += L) {
    Ccol[c0 + e] = ccol[o + e];
    Cval[c0 + e] = cval[o + e];
  }
}

// ------------------------------------------------------------ smoother scaling
// l1-Jacobi scaling d_i = sign(a_ii) (|a_ii| + sum_{j != i} |a_ij|): coarse
// Galerkin operators of the advective S~_T can have a few negative diagonals
__global__ void k_l1_dinv(int n, const int* __restrict__ rp, const int* __restrict__ col,
                          const double* __restrict__ val, double* __restrict__ dinv,
                          float* __restrict__ dinvf, int* __restrict__ err) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  double diag = 0.0, off = 0.0;
  for (int e = rp[i]; e < rp[i + 1]; ++e) {
    if (col[e] == i) diag = val[e];
    else off += fabs(val[e]);
  }
  double s = diag >= 0.0 ? diag + off : diag - off;
  if (s == 0.0 || !isfinite(s)) {
    atomicOr(err, 4);
    s = 1.0;
  }
  dinv[i] = 1.0 / s;
  if (dinvf) dinvf[i] = (float)(1.0 / s);
}

__global__ void k_to_float(long long n, const double* __restrict__ a, float* __restrict__ b) {
  long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i < n) b[i] = (float)a[i];
}

// round to nearest even BF16 (interpolation weights of precision 2)
__global__ void k_to_bf16(long long n, const double* __restrict__ a,
                          __nv_bfloat16* __restrict__ b) {
  long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i < n) b[i] = __float2bfloat16_rn((float)a[i]);
}

// ------------------------------------------------ vertical-line smoother
// Thomas factorisation of each column's tridiagonal part (Gaussian
// elimination without pivoting on a tridiagonal matrix): m_0 = d_0,
// m_k = d_k - l_k (u_{k-1} / m_{k-1}); stores l_k, 1 / m_k and u_k / m_k.
// Correctly rounded operations in the oracle's order (no FMA contraction).
// Twisted factorisation of each column's tridiagonal part (diagonal d_k,
// lower l_k, upper u_k; layer k of column c is cell c + nxy k), so that two
// threads can solve a column from both ends at once (k_line_sweep). With
// mid = nz / 2: the top rows k < mid are eliminated downwards (m_k = d_k -
// l_k cp_{k-1}, cp_k = u_k / m_k), the bottom rows k > mid upwards (q_k =
// d_k - u_k cq_{k+1}, cq_k = l_k / q_k), and the middle row takes both sides
// (pivot d - l cp_{mid-1} - u cq_{mid+1}). Stored per cell: lo = the
// coupling to the row eliminated before it (l_k on top, u_k below, l_mid in
// the middle), minv = 1 / pivot, cp = cp_k on top, cq_k below, u_mid in the
// middle.
__device__ __forceinline__ void line_row(int i, int nxy, const int* __restrict__ rp,
                                         const int* __restrict__ col,
                                         const double* __restrict__ val, double& d, double& l,
                                         double& u, bool& has_lo, bool& has_up) {
  d = l = u = 0.0;
  has_lo = has_up = false;
  for (int e = rp[i]; e < rp[i + 1]; ++e) {
    const int j = col[e];
    if (j == i) d = val[e];
    else if (j == i - nxy) { l = val[e]; has_lo = true; }
    else if (j == i + nxy) { u = val[e]; has_up = true; }
  }
}

__global__ void k_line_factor(int nxy, int nz, const int* __restrict__ rp,
                              const int* __restrict__ col, const double* __restrict__ val,
                              double* __restrict__ lo, double* __restrict__ minv,
                              double* __restrict__ cp, float* __restrict__ lof,
                              float* __restrict__ minvf, float* __restrict__ cpf,
                              int* __restrict__ err) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= nxy) return;
  const int mid = nz >> 1;
  auto store = [&](int i, double a, double mi, double q) {
    lo[i] = a;
    minv[i] = mi;
    cp[i] = q;
    if (lof) {
      lof[i] = (float)a;
      minvf[i] = (float)mi;
      cpf[i] = (float)q;
    }
  };
  auto pivot_ok = [&](double m) {
    const bool ok = m != 0.0 && isfinite(m);
    if (!ok) atomicOr(err, 16);
    return ok;
  };
  double d, l, u;
  bool has_lo, has_up;
  double cprev = 0.0;  // top: cp_{k-1}
  for (int k = 0; k < mid; ++k) {
    const int i = c + k * nxy;
    line_row(i, nxy, rp, col, val, d, l, u, has_lo, has_up);
    if (has_lo != (k > 0) || has_up != (k < nz - 1)) atomicOr(err, 16);
    const double m = __dsub_rn(d, __dmul_rn(l, cprev));
    double mi = 0.0, q = 0.0;
    if (pivot_ok(m)) {
      mi = __ddiv_rn(1.0, m);
      q = __ddiv_rn(u, m);
    }
    store(i, l, mi, q);
    cprev = q;
  }
  double cnext = 0.0;  // bottom: cq_{k+1}
  for (int k = nz - 1; k > mid; --k) {
    const int i = c + k * nxy;
    line_row(i, nxy, rp, col, val, d, l, u, has_lo, has_up);
    if (has_lo != (k > 0) || has_up != (k < nz - 1)) atomicOr(err, 16);
    const double m = __dsub_rn(d, __dmul_rn(u, cnext));
    double mi = 0.0, q = 0.0;
    if (pivot_ok(m)) {
      mi = __ddiv_rn(1.0, m);
      q = __ddiv_rn(l, m);
    }
    store(i, u, mi, q);
    cnext = q;
  }
  const int i = c + mid * nxy;
  line_row(i, nxy, rp, col, val, d, l, u, has_lo, has_up);
  if (has_lo != (mid > 0) || has_up != (mid < nz - 1)) atomicOr(err, 16);
  const double m = __dsub_rn(__dsub_rn(d, __dmul_rn(l, cprev)), __dmul_rn(u, cnext));
  double mi = 0.0;
  if (pivot_ok(m)) mi = __ddiv_rn(1.0, m);
  store(i, l, mi, u);
}

void line_setup(Level& v, int nxy, int nz, Pool& pool, bool f32, int* err, bool allocate,
                cudaStream_t s) {
  const int n = v.A.n;
  if ((long long)nxy * nz != n) fail(TP_EINVAL, "line smoother: level is not the grid");
  if (allocate) {
    v.line_lo = pool.alloc<double>(n);
    v.line_minv = pool.alloc<double>(n);
    v.line_cp = pool.alloc<double>(n);
    if (f32) {
      v.line_lof = pool.alloc<float>(n);
      v.line_minvf = pool.alloc<float>(n);
      v.line_cpf = pool.alloc<float>(n);
    }
  }
  k_line_factor<<<grid_for(nxy), kBlock, 0, s>>>(nxy, nz, v.A.rowptr, v.A.col, v.A.val,
                                                 v.line_lo, v.line_minv, v.line_cp, v.line_lof,
                                                 v.line_minvf, v.line_cpf, err);
  TP_LAUNCH_CHECK();
}

// -------------------------------------------------------- sliced-ELL copy
// One block per window of kSellWindow rows: the rows sorted by descending
// length (ties by ascending row) with a block bitonic sort; slice widths
// are the lengths of each slice's first (longest) row.
__global__ void __launch_bounds__(kSellWindow) k_sell_perm(int n, const int* __restrict__ rp,
                                                           int* __restrict__ perm,
                                                           int* __restrict__ width32) {
  __shared__ unsigned long long key[kSellWindow];
  const int t = threadIdx.x;
  const int r = blockIdx.x * kSellWindow + t;
  unsigned long long k = ~0ull;  // slots past n sort last
  if (r < n) {
    const int len = rp[r + 1] - rp[r];
    k = ((unsigned long long)(unsigned)(0x7fffffff - len) << 32) | (unsigned)r;
  }
  key[t] = k;
  __syncthreads();
  for (int size = 2; size <= kSellWindow; size <<= 1) {
    for (int stride = size >> 1; stride > 0; stride >>= 1) {
      const int partner = t ^ stride;
      if (partner > t) {
        const bool up = (t & size) == 0;
        const unsigned long long a = key[t], c = key[partner];
        if ((a > c) == up) {
          key[t] = c;
          key[partner] = a;
        }
      }
      __syncthreads();
    }
  }
  const unsigned long long kk = key[t];
  const int row = kk == ~0ull ? -1 : (int)(kk & 0xffffffffu);
  perm[r] = row;
  if ((t & 31) == 0) width32[r >> 5] = row >= 0 ? 32 * (rp[row + 1] - rp[row]) : 0;
}

// slot t of slice s: the entries of its row, padded to the slice width
__global__ void k_sell_fill(int nslots, const int* __restrict__ rp, const int* __restrict__ col,
                            const double* __restrict__ val, const int* __restrict__ perm,
                            const int* __restrict__ ptr, int* __restrict__ scol,
                            double* __restrict__ sval, float* __restrict__ svalf) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= nslots) return;
  const int sl = t >> 5, lane = t & 31;
  const int row = perm[t];
  const int w = (ptr[sl + 1] - ptr[sl]) >> 5;
  const int e0 = row >= 0 ? rp[row] : 0, len = row >= 0 ? rp[row + 1] - e0 : 0;
  for (int k = 0; k < w; ++k) {
    const long long q = (long long)ptr[sl] + 32 * k + lane;
    const bool has = k < len;
    if (scol) scol[q] = has ? col[e0 + k] : (row >= 0 ? row : 0);
    const double v = has ? val[e0 + k] : 0.0;
    sval[q] = v;
    if (svalf) svalf[q] = (float)v;
  }
}

// --------------------------------------------------------------- ELL copy
__global__ void k_max_row(int n, const int* __restrict__ rp, int* __restrict__ mx) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) atomicMax(mx, rp[i + 1] - rp[i]);
}

__global__ void k_to_ell(int n, int w, const int* __restrict__ rp, const int* __restrict__ col,
                         const double* __restrict__ val, int* __restrict__ ecol,
                         double* __restrict__ eval, float* __restrict__ evalf) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int r0 = rp[i], len = rp[i + 1] - r0;
  for (int k = 0; k < w; ++k) {
    const long long q = (long long)k * n + i;
    const bool has = k < len;
    if (ecol) ecol[q] = has ? col[r0 + k] : i;
    const double v = has ? val[r0 + k] : 0.0;
    eval[q] = v;
    if (evalf) evalf[q] = (float)v;
  }
}

// ELL copy by grid direction (the finest level of a grid's 7-point operator):
// slot k of row i holds the entry at column i + (-nxy, -nx, -1, 0, +1, +nx,
// +nxy)[k], 0 where the row has none; an entry at any other offset sets
// bit 32 of *err (the level is not the grid's 7-point pattern)
__global__ void k_to_stencil(int n, int nx, int nxy, const int* __restrict__ rp,
                             const int* __restrict__ col, const double* __restrict__ val,
                             double* __restrict__ eval, float* __restrict__ evalf,
                             int* __restrict__ err) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  double v[7] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
  for (int e = rp[i]; e < rp[i + 1]; ++e) {
    const int d = col[e] - i;
    const int k = d == -nxy ? 0 : d == -nx ? 1 : d == -1 ? 2 : d == 0 ? 3 : d == 1 ? 4
                : d == nx ? 5 : d == nxy ? 6 : -1;
    if (k < 0) {
      atomicOr(err, 32);
      continue;
    }
    v[k] = val[e];
  }
#pragma unroll
  for (int k = 0; k < 7; ++k) {
    const long long q = (long long)k * n + i;
    eval[q] = v[k];
    if (evalf) evalf[q] = (float)v[k];
  }
}

// ------------------------------------------------------------ coarsest level
__global__ void k_to_dense(int n, const int* __restrict__ rp, const int* __restrict__ col,
                           const double* __restrict__ val, double* __restrict__ D) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  for (int j = 0; j < n; ++j) D[(long long)i * n + j] = 0.0;
  for (int e = rp[i]; e < rp[i + 1]; ++e) D[(long long)i * n + col[e]] += val[e];
}

// Gauss-Jordan elimination with partial pivoting on [A | I] (one block):
// leaves A^{-1} in inv. Pivot: largest |a_ik| over rows >= k, lowest row on
// ties. A zero pivot sets err.
__global__ void k_gauss_jordan(int n, double* __restrict__ A, double* __restrict__ inv,
                               int* __restrict__ err) {
  __shared__ double s_val[1024];
  __shared__ int s_idx[1024];
  __shared__ int s_piv;
  const int tid = threadIdx.x, nt = blockDim.x;
  for (long long q = tid; q < (long long)n * n; q += nt) inv[q] = ((q / n) == (q % n)) ? 1.0 : 0.0;
  __syncthreads();
  for (int k = 0; k < n; ++k) {
    double best = -1.0;
    int bi = n;
    for (int i = k + tid; i < n; i += nt) {
      double a = fabs(A[(long long)i * n + k]);
      if (a > best || (a == best && i < bi)) {
        best = a;
        bi = i;
      }
    }
    s_val[tid] = best;
    s_idx[tid] = bi;
    __syncthreads();
    for (int o = nt / 2; o > 0; o >>= 1) {
      if (tid < o) {
        double a = s_val[tid + o];
        int ai = s_idx[tid + o];
        if (a > s_val[tid] || (a == s_val[tid] && ai < s_idx[tid])) {
          s_val[tid] = a;
          s_idx[tid] = ai;
        }
      }
      __syncthreads();
    }
    if (tid == 0) {
      s_piv = s_idx[0];
      if (!(s_val[0] > 0.0)) *err = 1;
    }
    __syncthreads();
    if (*err) return;
    const int p = s_piv;
    if (p != k) {
      for (int j = tid; j < n; j += nt) {
        double t = A[(long long)k * n + j];
        A[(long long)k * n + j] = A[(long long)p * n + j];
        A[(long long)p * n + j] = t;
        t = inv[(long long)k * n + j];
        inv[(long long)k * n + j] = inv[(long long)p * n + j];
        inv[(long long)p * n + j] = t;
      }
    }
    __syncthreads();
    const double piv = A[(long long)k * n + k];
    __syncthreads();
    for (int j = tid; j < n; j += nt) {
      A[(long long)k * n + j] /= piv;
      inv[(long long)k * n + j] /= piv;
    }
    __syncthreads();
    for (long long q = tid; q < (long long)n * n; q += nt) {
      int i = (int)(q / n), j = (int)(q % n);
      if (i == k) continue;
      double f = A[(long long)i * n + k];
      if (j == k) continue;  // column k of A is cleared below
      A[(long long)i * n + j] -= f * A[(long long)k * n + j];
      inv[(long long)i * n + j] -= f * inv[(long long)k * n + j];
    }
    __syncthreads();
    // inv column k and A column k for rows != k
    for (int i = tid; i < n; i += nt) {
      if (i == k) continue;
      double f = A[(long long)i * n + k];
      inv[(long long)i * n + k] -= f * inv[(long long)k * n + k];
      A[(long long)i * n + k] = 0.0;
    }
    __syncthreads();
  }
}

// threads per CSR row in the V-cycle kernels: a power of two giving each
// lane about 4 entries (fewer lanes mean fewer shuffle steps per row, more
// mean more parallelism on short coarse levels), halved while the launch
// would exceed four waves of resident threads, but not below the width that
// leaves each lane at most 12 entries. FGMRES solve time on GB300 (FP64,
// ms; layered 256x256x64 / grf 64x64x32 / channelised 128x128x64): this
// rule 183.4 / 11.5 / 41.5; halving down to one lane (the rule of the
// smaller grids, where level 1 of the layered A_pp, 1.25 M rows of 29.5
// entries, ran with one lane) 200.2 / 11.4 / 42.5; floors of 8 or 16
// entries 186.5-188.8 / 11.4-11.5 / 41.5-42.4.
int pick_lanes(const DevCSR& A) {
  const long long resident = resident_threads();
  const double avg = A.n > 0 ? (double)A.nnz / A.n : 1.0;
  int l = 1;
  while (l * 4.0 <= avg && l < 32) l *= 2;
  int lmin = 1;
  while (lmin < 32 && avg / lmin > 12.0) lmin *= 2;
  while (l > lmin && (long long)A.n * l > 4 * resident) l /= 2;
  // at most 16 lanes: a 32-lane row's five FP64 reduction adds occupy the
  // FP64 pipe for the whole warp (A_pp's level 3 on the layered workload:
  // 34 k rows x 92 entries). Layered 256x256x64 FGMRES 140.4 -> 138.2 ms
  // (FP64), 95.1 -> 94.6 ms (FP32); channelised and grf 64x64x32 within
  // noise; at most 8 lanes: 140.0 ms, grf +0.6 ms
  return l > 16 ? 16 : l;
}

// threads resident on the whole device at full occupancy, once per process
long long resident_threads() {
  static const long long r = []() {
    int dev = 0, sms = 0, thr = 0;
    TP_CUDA_TRY(cudaGetDevice(&dev));
    TP_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    TP_CUDA_TRY(cudaDeviceGetAttribute(&thr, cudaDevAttrMaxThreadsPerMultiProcessor, dev));
    return (long long)sms * thr;
  }();
  return r;
}

// SM count of the current device, once per process (thread-safe)
int setup_sms() {
  static const int sms = []() {
    int dev = 0, v = 0;
    TP_CUDA_TRY(cudaGetDevice(&dev));
    TP_CUDA_TRY(cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev));
    return v;
  }();
  return sms;
}

int read_int(const int* d, cudaStream_t s) {
  int h = 0;
  TP_CUDA_TRY(cudaMemcpyAsync(&h, d, sizeof(int), cudaMemcpyDeviceToHost, s));
  TP_CUDA_TRY(cudaStreamSynchronize(s));
  return h;
}

// C = A B with the canonical summation order; C arrays allocated from `pool`.
DevCSR spgemm(const DevCSR& A, const DevCSR& B, Pool& pool, Pool& scratch, cudaStream_t s) {
  const int n = A.n;
  int* ub = scratch.alloc<int>(n + 1);
  int* off = scratch.alloc<int>(n + 1);
  int* wlist = scratch.alloc<int>(n + 1);
  int* blist = scratch.alloc<int>(n + 1);
  int* counts = scratch.alloc<int>(3);
  TP_CUDA_TRY(cudaMemsetAsync(counts, 0, 3 * sizeof(int), s));
  k_spgemm_ub<<<grid_for(n), kBlock, 0, s>>>(n, A.rowptr, A.col, B.rowptr, ub, wlist, blist,
                                             counts);
  TP_LAUNCH_CHECK();
  long long tot = scan_exclusive(ub, off, n, scratch, s);
  int* ccol = scratch.alloc<int>(tot + 1);
  double* cval = scratch.alloc<double>(tot + 1);
  int* cnt = scratch.alloc<int>(n + 1);
  const bool dense = B.m <= kDenseCap;
  if (dense) {
    static const bool dense_attr = []() {
      TP_CUDA_TRY(cudaFuncSetAttribute(k_spgemm_dense, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)kDenseSmem));
      return true;
    }();
    (void)dense_attr;
    long long blocks = ((long long)n + kDenseWarps - 1) / kDenseWarps;
    if (blocks > 8LL * setup_sms()) blocks = 8LL * setup_sms();
    const size_t smem = (size_t)kDenseWarps * B.m * (sizeof(double) + 1);
    k_spgemm_dense<<<(int)blocks, 32 * kDenseWarps, smem, s>>>(
        n, B.m, A.rowptr, A.col, A.val, B.rowptr, B.col, B.val, off, ccol, cval, cnt);
    TP_LAUNCH_CHECK();
  } else {
  k_spgemm_rows_merge<<<grid_for(n, 128), 128, 0, s>>>(n, A.rowptr, A.col, A.val, B.rowptr,
                                                       B.col, B.val, off, ub, ccol, cval, cnt);
  TP_LAUNCH_CHECK();
  k_spgemm_rows<<<grid_for(n, 128), 128, 0, s>>>(n, A.rowptr, A.col, A.val, B.rowptr, B.col,
                                                 B.val, off, ub, ccol, cval, cnt);
  TP_LAUNCH_CHECK();
  // SM count and the big-row kernel's shared-memory opt-in, once per process
  // (thread-safe static initialisation; hierarchies are set up concurrently)
  static const int num_sms = []() {
    int dev = 0, v = 0;
    TP_CUDA_TRY(cudaGetDevice(&dev));
    TP_CUDA_TRY(cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev));
    return v;
  }();
  {
    // rows with kSpShort < ub < kSpMid (4 warps x 10 KiB per block), then
    // kSpMid <= ub < kSpCap (2 warps x 20 KiB)
    long long blocks = (n + 3) / 4;
    if (blocks > 12LL * num_sms) blocks = 12LL * num_sms;
    k_spgemm_rows_warp<kSpMid, 4><<<(int)blocks, 128, 0, s>>>(
        n, A.rowptr, A.col, A.val, B.rowptr, B.col, B.val, off, ub, wlist, counts, 0, ccol, cval,
        cnt);
    TP_LAUNCH_CHECK();
    blocks = (n + 1) / 2;
    if (blocks > 8LL * num_sms) blocks = 8LL * num_sms;
    k_spgemm_rows_warp<kSpCap, 2><<<(int)blocks, 64, 0, s>>>(
        n, A.rowptr, A.col, A.val, B.rowptr, B.col, B.val, off, ub, wlist, counts, 2, ccol, cval,
        cnt);
  }
  TP_LAUNCH_CHECK();
  static const bool big_attr = []() {
    TP_CUDA_TRY(cudaFuncSetAttribute(k_spgemm_rows_big, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)kSpBigSmem));
    return true;
  }();
  (void)big_attr;
  k_spgemm_rows_big<<<n < num_sms ? n : num_sms, kSpBigThreads, kSpBigSmem, s>>>(
      n, A.rowptr, A.col, A.val, B.rowptr, B.col, B.val, off, ub, blist, counts, ccol, cval, cnt);
  TP_LAUNCH_CHECK();
  }
  DevCSR C;
  C.n = n;
  C.m = B.m;
  C.rowptr = pool.alloc<int>(n + 1);
  long long nnz = scan_exclusive(cnt, C.rowptr, n, scratch, s);
  C.nnz = (int)nnz;
  C.col = pool.alloc<int>(nnz + 1);
  C.val = pool.alloc<double>(nnz + 1);
  {
    const double avg = n > 0 ? (double)nnz / n : 1.0;
    int L = 1;
    while (L < 32 && 2.0 * L < avg) L *= 2;
    const int g = grid_for((long long)n * L);
    switch (L) {
#define TP_CASE(LL)                                                                          \
  case LL:                                                                                   \
    k_spgemm_compact<LL><<<g, kBlock, 0, s>>>(n, off, ccol, cval, C.rowptr, C.col, C.val); \
    break;
      TP_CASE(1) TP_CASE(2) TP_CASE(4) TP_CASE(8) TP_CASE(16) TP_CASE(32)
#undef TP_CASE
    }
  }
  TP_LAUNCH_CHECK();
  return C;
}

DevCSR transpose(const DevCSR& P, Pool& pool, Pool& scratch, cudaStream_t s) {
  DevCSR R;
  R.n = P.m;
  R.m = P.n;
  R.nnz = P.nnz;
  int* cnt = scratch.alloc<int>(R.n + 1);
  int* cursor = scratch.alloc<int>(R.n + 1);
  TP_CUDA_TRY(cudaMemsetAsync(cnt, 0, sizeof(int) * (R.n + 1), s));
  TP_CUDA_TRY(cudaMemsetAsync(cursor, 0, sizeof(int) * (R.n + 1), s));
  k_count_cols<<<grid_for(P.n), kBlock, 0, s>>>(P.n, P.rowptr, P.col, cnt);
  TP_LAUNCH_CHECK();
  R.rowptr = pool.alloc<int>(R.n + 1);
  scan_exclusive(cnt, R.rowptr, R.n, scratch, s);
  R.col = pool.alloc<int>(R.nnz + 1);
  R.val = pool.alloc<double>(R.nnz + 1);
  // atomically placed (unordered) entries, then each row ranked by column
  int* ucol = scratch.alloc<int>(R.nnz + 1);
  double* uval = scratch.alloc<double>(R.nnz + 1);
  k_fill_transpose<<<grid_for(P.n), kBlock, 0, s>>>(P.n, P.rowptr, P.col, P.val, R.rowptr,
                                                    cursor, ucol, uval);
  TP_LAUNCH_CHECK();
  k_rank_rows<<<grid_for(R.n), kBlock, 0, s>>>(R.n, R.rowptr, ucol, uval, R.col, R.val);
  TP_LAUNCH_CHECK();
  k_rank_rows_warp<<<grid_for((long long)R.n * 32), kBlock, 0, s>>>(R.n, R.rowptr, ucol, uval,
                                                                    R.col, R.val);
  TP_LAUNCH_CHECK();
  return R;
}

}  // namespace

DevCSR csr_product(const DevCSR& A, const DevCSR& B, Pool& pool, Pool& scratch,
                   cudaStream_t s) {
  return spgemm(A, B, pool, scratch, s);
}

void csr_product_numeric(const DevCSR& A, const DevCSR& B, const DevCSR& C, cudaStream_t s) {
  k_spgemm_numeric<<<grid_for(A.n, 128), 128, 0, s>>>(A.n, A.rowptr, A.col, A.val, B.rowptr,
                                                      B.col, B.val, C.rowptr, C.col, C.val);
  TP_LAUNCH_CHECK();
}

void csr_transpose_positions(const DevCSR& A, int* tpos, int* err, cudaStream_t s) {
  if (A.n > 0 && A.nnz >= (long long)kWarpRowMean * A.n)
    k_transpose_pos_warp<<<grid_for((long long)A.n * 32), kBlock, 0, s>>>(A.n, A.rowptr, A.col,
                                                                         tpos, err);
  else
    k_transpose_pos<<<grid_for(A.n), kBlock, 0, s>>>(A.n, A.rowptr, A.col, tpos, err);
  TP_LAUNCH_CHECK();
}

Hierarchy::~Hierarchy() = default;

double Hierarchy::operator_complexity() const {
  if (L.empty() || L[0].A.nnz == 0) return 0.0;
  double s = 0.0;
  for (const Level& l : L) s += l.A.nnz;
  return s / L[0].A.nnz;
}

namespace {
struct PhaseClock {
  std::chrono::steady_clock::time_point t = std::chrono::steady_clock::now();
  double lap(cudaStream_t s) {
    TP_CUDA_TRY(cudaStreamSynchronize(s));
    auto n = std::chrono::steady_clock::now();
    double ms = std::chrono::duration<double, std::milli>(n - t).count();
    t = n;
    return ms;
  }
};
}  // namespace

void Hierarchy::setup(const DevCSR& A0, const AmgOpts& o, cudaStream_t s) {
  opts = o;
  for (double& x : phase_ms) x = 0.0;
  PhaseClock clk;
  pool.release();
  scratch.release();
  L.clear();
  coarse_inv = nullptr;
  cheb_partials = nullptr;
  tail_first = -1;
  err = pool.alloc<int>(2);
  TP_CUDA_TRY(cudaMemsetAsync(err, 0, sizeof(int), s));
  L.emplace_back();
  L[0].A = A0;
  n0 = A0.n;
  while (true) {
    Level& cur = L.back();
    const DevCSR& A = cur.A;
    const int n = A.n;
    cur.dpos = pool.alloc<int>(n);
    k_diag_pos<<<grid_for(n), kBlock, 0, s>>>(n, A.rowptr, A.col, cur.dpos, err);
    TP_LAUNCH_CHECK();
    const bool coarsest = n <= opts.coarse_size || (int)L.size() >= opts.max_levels;
    if (!coarsest) {
      // transpose positions do not depend on the diagonal: both checks are
      // read back with one synchronisation
      cur.tpos = pool.alloc<int>(A.nnz);
      csr_transpose_positions(A, cur.tpos, err, s);
    }
    {
      const int e = read_int(err, s);
      if (e & 1) fail(TP_EINVAL, "AMG: a row has no diagonal entry");
      if (e & 2) fail(TP_EINVAL, "AMG: pattern is not structurally symmetric");
    }
    if (coarsest) break;
    // long rows (coarse Galerkin levels): one warp per row
    const bool wrow = A.nnz >= (long long)kWarpRowMean * n;
    const int gw = grid_for((long long)n * 32);
    cur.strong = pool.alloc<unsigned char>(A.nnz);
    if (wrow)
      k_strength_warp<<<gw, kBlock, 0, s>>>(n, A.rowptr, A.col, A.val, opts.theta, cur.strong);
    else
      k_strength<<<grid_for(n), kBlock, 0, s>>>(n, A.rowptr, A.col, A.val, opts.theta,
                                                cur.strong);
    TP_LAUNCH_CHECK();
    // PMIS
    int* lam = scratch.alloc<int>(n);
    unsigned char* newc = scratch.alloc<unsigned char>(n);
    int* undecided = scratch.alloc<int>(1);
    cur.cf = pool.alloc<signed char>(n);
    if (wrow)
      k_pmis_init_warp<<<gw, kBlock, 0, s>>>(n, A.rowptr, A.col, cur.strong, cur.tpos, lam,
                                             cur.cf);
    else
      k_pmis_init<<<grid_for(n), kBlock, 0, s>>>(n, A.rowptr, A.col, cur.strong, cur.tpos, lam,
                                                 cur.cf);
    TP_LAUNCH_CHECK();
    // rounds are enqueued in batches (four, then pairs) before the host
    // reads the count of undecided points: a round after the last is a no-op
    // (no point is undecided, so nothing is selected or changed); levels
    // here take about five rounds
    int rounds = 0;
    while (true) {
      if (rounds >= opts.max_pmis_rounds) fail(TP_SETUP_FAILED, "PMIS round cap reached");
      const int batch = rounds == 0 ? 4 : 2;
      for (int r = 0; r < batch; ++r) {
        ++rounds;
        if (wrow)
          k_pmis_select_warp<<<gw, kBlock, 0, s>>>(n, A.rowptr, A.col, cur.strong, cur.tpos, lam,
                                                   cur.cf, opts.seed, newc);
        else
          k_pmis_select<<<grid_for(n), kBlock, 0, s>>>(n, A.rowptr, A.col, cur.strong, cur.tpos,
                                                       lam, cur.cf, opts.seed, newc);
        TP_LAUNCH_CHECK();
        TP_CUDA_TRY(cudaMemsetAsync(undecided, 0, sizeof(int), s));
        if (wrow)
          k_pmis_update_warp<<<gw, kBlock, 0, s>>>(n, A.rowptr, A.col, cur.strong, cur.cf, newc,
                                                   undecided);
        else
          k_pmis_update<<<grid_for(n), kBlock, 0, s>>>(n, A.rowptr, A.col, cur.strong, cur.cf,
                                                       newc, undecided);
        TP_LAUNCH_CHECK();
      }
      if (read_int(undecided, s) == 0) break;
    }
    cur.pmis_rounds = rounds;
    phase_ms[0] += clk.lap(s);
    int* flag = scratch.alloc<int>(n + 1);
    int* cidx = scratch.alloc<int>(n + 1);
    k_cflag<<<grid_for(n), kBlock, 0, s>>>(n, cur.cf, flag);
    TP_LAUNCH_CHECK();
    const int nc = (int)scan_exclusive(flag, cidx, n, scratch, s);
    if (nc == 0 || (double)nc > 0.9 * (double)n) {
      cur.cf = nullptr;  // this level becomes the coarsest
      break;
    }
    // interpolation
    DevCSR P;
    P.n = n;
    P.m = nc;
    P.rowptr = pool.alloc<int>(n + 1);
    int* cnt = scratch.alloc<int>(n + 1);
    if (opts.interp == 0) {
      k_classical_count<<<grid_for(n), kBlock, 0, s>>>(n, A.rowptr, A.col, cur.strong, cur.cf,
                                                       cnt);
      TP_LAUNCH_CHECK();
      P.nnz = (int)scan_exclusive(cnt, P.rowptr, n, scratch, s);
      P.col = pool.alloc<int>(P.nnz);
      P.val = pool.alloc<double>(P.nnz);
      k_classical_fill<<<grid_for(n, 128), 128, 0, s>>>(n, A.rowptr, A.col, A.val, cur.dpos,
                                                        cur.strong, cur.cf, cidx, P.rowptr,
                                                        P.col, P.val);
      TP_LAUNCH_CHECK();
      {
        long long blocks = ((long long)n + kClsWarps - 1) / kClsWarps;
        if (blocks > 8LL * setup_sms()) blocks = 8LL * setup_sms();
        k_classical_fill_warp<<<(int)blocks, 32 * kClsWarps, 0, s>>>(
            n, A.rowptr, A.col, A.val, cur.dpos, cur.strong, cur.cf, cidx, P.rowptr, P.col,
            P.val);
        TP_LAUNCH_CHECK();
      }
    } else {
      int* ub = scratch.alloc<int>(n + 1);
      int* off = scratch.alloc<int>(n + 1);
      k_extpi_ub<<<grid_for(n), kBlock, 0, s>>>(n, A.rowptr, A.col, cur.strong, cur.cf, ub);
      TP_LAUNCH_CHECK();
      long long tot = scan_exclusive(ub, off, n, scratch, s);
      int* buf = scratch.alloc<int>(tot + 1);
      k_extpi_sets<<<grid_for(n, 128), 128, 0, s>>>(n, A.rowptr, A.col, cur.strong, cur.cf, off,
                                                    ub, buf, cnt);
      TP_LAUNCH_CHECK();
      {
        long long blocks = ((long long)n + kSetWarps - 1) / kSetWarps;
        if (blocks > 8LL * setup_sms()) blocks = 8LL * setup_sms();
        k_extpi_sets_warp<<<(int)blocks, 32 * kSetWarps, 0, s>>>(n, A.rowptr, A.col, cur.strong,
                                                                 cur.cf, off, ub, buf, cnt);
        TP_LAUNCH_CHECK();
      }
      P.nnz = (int)scan_exclusive(cnt, P.rowptr, n, scratch, s);
      P.col = pool.alloc<int>(P.nnz);
      P.val = pool.alloc<double>(P.nnz);
      k_extpi_fill_short<<<grid_for(n, 128), 128, 0, s>>>(n, A.rowptr, A.col, A.val, cur.dpos,
                                                         cur.strong, cur.cf, cidx, off, buf,
                                                         P.rowptr, P.col, P.val);
      TP_LAUNCH_CHECK();
      k_extpi_fill_warp<<<(n + kFillWarps - 1) / kFillWarps, 32 * kFillWarps, 0, s>>>(
          n, A.rowptr, A.col, A.val, cur.dpos, cur.strong, cur.cf, cidx, off, buf, P.rowptr,
          P.col, P.val);
      TP_LAUNCH_CHECK();
    }
    if (opts.pmax > 0) {
      DevCSR T;
      T.n = n;
      T.m = nc;
      T.rowptr = pool.alloc<int>(n + 1);
      k_trunc_count<<<grid_for(n), kBlock, 0, s>>>(n, P.rowptr, opts.pmax, cnt);
      TP_LAUNCH_CHECK();
      T.nnz = (int)scan_exclusive(cnt, T.rowptr, n, scratch, s);
      T.col = pool.alloc<int>(T.nnz + 1);
      T.val = pool.alloc<double>(T.nnz + 1);
      k_trunc_fill<<<grid_for(n), kBlock, 0, s>>>(n, P.rowptr, P.col, P.val, opts.pmax, T.rowptr,
                                                  T.col, T.val);
      TP_LAUNCH_CHECK();
      P = T;
    }
    cur.P = P;
    phase_ms[1] += clk.lap(s);
    cur.R = transpose(P, pool, scratch, s);
    phase_ms[2] += clk.lap(s);
    cur.AP = spgemm(A, P, pool, scratch, s);
    DevCSR Ac = spgemm(cur.R, cur.AP, pool, scratch, s);
    TP_CUDA_TRY(cudaStreamSynchronize(s));
    phase_ms[3] += clk.lap(s);
    scratch.release();
    L.emplace_back();
    L.back().A = Ac;
  }
  clk.lap(s);
  finish_levels(s, true);
  phase_ms[4] += clk.lap(s);
}

// smoother scaling, FP32 copies, work vectors (allocate = first setup) and
// the coarsest-level inverse
void Hierarchy::finish_levels(cudaStream_t s, bool allocate) {
  const bool f32 = opts.precision >= 1;
  const bool bf16 = opts.precision == 2;
  TP_CUDA_TRY(cudaMemsetAsync(err, 0, sizeof(int), s));
  if (opts.smoother == 1 && allocate)
    cheb_partials = pool.alloc<double>(2 * chebyshev_norm_parts());
  for (size_t l = 0; l < L.size(); ++l) {
    Level& v = L[l];
    const int n = v.A.n;
    if (allocate) {
      v.dinv = pool.alloc<double>(n);
      v.dinvf = f32 ? pool.alloc<float>(n) : nullptr;
    }
    if (opts.smoother == 1 && l + 1 < L.size()) {
      chebyshev_setup(v, pool, opts.cheb_degree, opts.seed, cheb_partials, err, allocate, s);
    } else {
      k_l1_dinv<<<grid_for(n), kBlock, 0, s>>>(n, v.A.rowptr, v.A.col, v.A.val, v.dinv,
                                               v.dinvf, err);
      TP_LAUNCH_CHECK();
    }
    if (l == 0 && opts.line_nz > 1 && L.size() > 1)
      line_setup(v, opts.line_nxy, opts.line_nz, pool, f32, err, allocate, s);
    if (f32) {
      if (allocate) v.A.valf = pool.alloc<float>(v.A.nnz);
      k_to_float<<<grid_for(v.A.nnz), kBlock, 0, s>>>(v.A.nnz, v.A.val, v.A.valf);
      TP_LAUNCH_CHECK();
      if (v.P.nnz) {
        if (allocate) {
          v.P.valf = pool.alloc<float>(v.P.nnz);
          v.R.valf = pool.alloc<float>(v.R.nnz);
        }
        k_to_float<<<grid_for(v.P.nnz), kBlock, 0, s>>>(v.P.nnz, v.P.val, v.P.valf);
        k_to_float<<<grid_for(v.R.nnz), kBlock, 0, s>>>(v.R.nnz, v.R.val, v.R.valf);
        TP_LAUNCH_CHECK();
        if (bf16) {
          if (allocate) {
            v.Ph = pool.alloc<__nv_bfloat16>(v.P.nnz);
            v.Rh = pool.alloc<__nv_bfloat16>(v.R.nnz);
          }
          k_to_bf16<<<grid_for(v.P.nnz), kBlock, 0, s>>>(v.P.nnz, v.P.val, v.Ph);
          k_to_bf16<<<grid_for(v.R.nnz), kBlock, 0, s>>>(v.R.nnz, v.R.val, v.Rh);
          TP_LAUNCH_CHECK();
        }
      }
    }
    // ELL copy for short-row levels (the 7-point finest level); by grid
    // direction when the level is a known grid's 7-point operator (the column
    // indices, a third of an FP64 sweep's matrix bytes and half an FP32
    // one's, are then implicit)
    const bool stencil = l == 0 && opts.grid_nx > 1 && opts.grid_ny > 1 && opts.grid_nz > 1 &&
                         (long long)opts.grid_nx * opts.grid_ny * opts.grid_nz == n;
    if (allocate && stencil) {
      v.ell_w = 7;
      v.ell_nx = opts.grid_nx;
      v.ell_nxy = opts.grid_nx * opts.grid_ny;
      v.ell_col = nullptr;
      v.ell_val = pool.alloc<double>((size_t)7 * n);
      v.ell_valf = f32 ? pool.alloc<float>((size_t)7 * n) : nullptr;
    } else if (allocate && n >= 4096) {
      TP_CUDA_TRY(cudaMemsetAsync(err + 1, 0, sizeof(int), s));
      k_max_row<<<grid_for(n), kBlock, 0, s>>>(n, v.A.rowptr, err + 1);
      TP_LAUNCH_CHECK();
      const int w = read_int(err + 1, s);
      if (w <= kEllMaxW) {
        v.ell_w = w;
        v.ell_col = pool.alloc<int>((size_t)w * n);
        v.ell_val = pool.alloc<double>((size_t)w * n);
        v.ell_valf = f32 ? pool.alloc<float>((size_t)w * n) : nullptr;
      }
    }
    if (v.ell_w > 0 && v.ell_nxy > 0) {
      k_to_stencil<<<grid_for(n), kBlock, 0, s>>>(n, v.ell_nx, v.ell_nxy, v.A.rowptr, v.A.col,
                                                  v.A.val, v.ell_val, v.ell_valf, err);
      TP_LAUNCH_CHECK();
    } else if (v.ell_w > 0) {
      k_to_ell<<<grid_for(n), kBlock, 0, s>>>(n, v.ell_w, v.A.rowptr, v.A.col, v.A.val,
                                              allocate ? v.ell_col : nullptr, v.ell_val,
                                              v.ell_valf);
      TP_LAUNCH_CHECK();
    }
    // sliced-ELL copy of the large levels below the finest: one thread per
    // row gives coalesced loads and no cross-lane reduction (the FP64 adds of
    // a split row's reduction compete with its multiply-adds for the FP64
    // pipe). It needs about half a wave of resident threads: on smaller
    // levels the lane-split CSR sweep fills the machine better. Measured FP64
    // / FP32 solve times (ms) without it; from 262,144 rows; from 131,072 or
    // 200,000 rows; on every level of 4096 rows or more: 256x256x64 layered
    // 169.9 / 116.6, 154.6 / 107.4, 151.3 / 107.4, 166.0 / 111.7; 128^2x64
    // channel 41.9 / 26.3, 40.7 / 25.1, 39.8 / 25.3, 49.7 / 28.5.
    const long long sell_min = opts.sell_rows == 0 ? resident_threads() / 2 : opts.sell_rows;
    if (allocate && opts.sell_rows >= 0 && l > 0 && v.ell_w == 0 && n >= sell_min &&
        l + 1 < L.size()) {
      const int windows = (n + kSellWindow - 1) / kSellWindow;
      const int slices = windows * (kSellWindow / 32);
      v.sell_perm = pool.alloc<int>((size_t)windows * kSellWindow);
      int* w32 = scratch.alloc<int>(slices + 1);
      k_sell_perm<<<windows, kSellWindow, 0, s>>>(n, v.A.rowptr, v.sell_perm, w32);
      TP_LAUNCH_CHECK();
      v.sell_ptr = pool.alloc<int>(slices + 1);
      const long long tot = scan_exclusive(w32, v.sell_ptr, slices, scratch, s);
      v.sell_col = pool.alloc<int>(tot + 1);
      v.sell_val = pool.alloc<double>(tot + 1);
      v.sell_valf = f32 ? pool.alloc<float>(tot + 1) : nullptr;
      v.sell_slices = slices;
      v.sell_entries = tot;
    }
    if (v.sell_slices > 0) {
      const int nslots = v.sell_slices * 32;
      k_sell_fill<<<grid_for(nslots), kBlock, 0, s>>>(nslots, v.A.rowptr, v.A.col, v.A.val,
                                                     v.sell_perm, v.sell_ptr,
                                                     allocate ? v.sell_col : nullptr, v.sell_val,
                                                     v.sell_valf);
      TP_LAUNCH_CHECK();
    }
    if (allocate) {
      const size_t es = f32 ? sizeof(float) : sizeof(double);
      v.b = pool.alloc<char>(es * (n + 1));
      v.x = pool.alloc<char>(es * (n + 1));
      v.t = pool.alloc<char>(es * (n + 1));
      v.r = pool.alloc<char>(es * (n + 1));
      if (opts.smoother == 1) {
        v.cw = pool.alloc<char>(es * (n + 1));
        v.cd0 = pool.alloc<char>(es * (n + 1));
        v.cd1 = pool.alloc<char>(es * (n + 1));
        v.cr = pool.alloc<char>(es * (n + 1));
      }
      v.lanes_A = pick_lanes(v.A);
      v.lanes_P = v.P.nnz ? pick_lanes(v.P) : 1;
      v.lanes_R = v.R.nnz ? pick_lanes(v.R) : 1;
    }
  }
  {
    const int e = read_int(err, s);
    if (e & 4) fail(TP_SETUP_FAILED, "AMG: empty, zero-diagonal or non-finite row");
    if (e & 8) fail(TP_SETUP_FAILED, "AMG: Chebyshev power iteration broke down");
    if (e & 16)
      fail(TP_SETUP_FAILED,
           "AMG: vertical-line smoother needs both vertical neighbours and non-zero pivots");
    if (e & 32) fail(TP_SETUP_FAILED, "AMG: level 0 is not the grid's 7-point pattern");
  }
  // coarsest level: explicit inverse by Gauss-Jordan with partial pivoting
  Level& cl = L.back();
  if (allocate) {
    nc = cl.A.n;
    if (nc > opts.max_coarse_dense) fail(TP_SETUP_FAILED, "AMG: coarsest level too large");
    coarse_dense = pool.alloc<double>((size_t)nc * nc);
    coarse_inv = pool.alloc<double>((size_t)nc * nc);
  }
  k_to_dense<<<grid_for(nc), kBlock, 0, s>>>(nc, cl.A.rowptr, cl.A.col, cl.A.val, coarse_dense);
  TP_LAUNCH_CHECK();
  TP_CUDA_TRY(cudaMemsetAsync(err, 0, sizeof(int), s));
  // one cluster holds the matrix in shared memory; the single-CTA kernel
  // (matrix in global memory) covers sizes beyond the cluster's capacity
  if (!coarse_inverse_cluster(nc, coarse_dense, coarse_inv, err, s)) {
    k_gauss_jordan<<<1, 1024, 0, s>>>(nc, coarse_dense, coarse_inv, err);
  }
  TP_LAUNCH_CHECK();
  if (read_int(err, s) != 0) fail(TP_SETUP_FAILED, "AMG: singular coarsest operator");
  if (allocate) {
    in = pool.alloc<double>(n0 + 1);
    out = pool.alloc<double>(n0 + 1);
    plan_tail(s);
  }
  TP_CUDA_TRY(cudaStreamSynchronize(s));
}

// Coarse tail: from the first level below level 0 with at most
// opts.tail_rows rows down to the coarsest, when at least one smoothing
// level is in it, the smoother is l1-Jacobi and clusters can be launched.
// The descriptors point at the level buffers, which keep their addresses
// under refresh().
void Hierarchy::plan_tail(cudaStream_t s) {
  tail_first = -1;
  const int nl = (int)L.size();
  if (opts.tail_rows <= 0 || opts.smoother != 0 || nl < 3) return;
  int f = -1;
  for (int l = 1; l < nl - 1; ++l)
    if (L[l].A.n <= opts.tail_rows) {
      f = l;
      break;
    }
  if (f < 0 || nl - f > kMaxTailLevels) return;
  const int cluster = tail_cluster_size();
  if (cluster == 0) return;
  const bool f32 = opts.precision >= 1;
  tail_host.assign(nl, TailLevel{});
  for (int l = 0; l < nl; ++l) {
    const Level& v = L[l];
    TailLevel& d = tail_host[l];
    d.n = v.A.n;
    d.nnext = (l + 1 < nl) ? L[l + 1].A.n : 0;
    d.Arp = v.A.rowptr;
    d.Acol = v.A.col;
    d.Aval = f32 ? (const void*)v.A.valf : (const void*)v.A.val;
    d.dinv = f32 ? (const void*)v.dinvf : (const void*)v.dinv;
    d.Prp = v.P.rowptr;
    d.Pcol = v.P.col;
    d.Pval = f32 ? (const void*)v.P.valf : (const void*)v.P.val;
    d.Ph = v.Ph;
    d.Rrp = v.R.rowptr;
    d.Rcol = v.R.col;
    d.Rval = f32 ? (const void*)v.R.valf : (const void*)v.R.val;
    d.Rh = v.Rh;
    d.b = v.b;
    d.x = v.x;
    d.t = v.t;
    d.r = v.r;
  }
  tail_desc = pool.alloc<TailLevel>(nl);
  TP_CUDA_TRY(cudaMemcpyAsync(tail_desc, tail_host.data(), sizeof(TailLevel) * nl,
                              cudaMemcpyHostToDevice, s));
  tail_first = f;
  tail_cluster = cluster;
}

void Hierarchy::refresh(cudaStream_t s) {
  if (L.empty()) fail(TP_ESTATE, "AMG: refresh before setup");
  for (size_t l = 0; l + 1 < L.size(); ++l) {
    Level& v = L[l];
    const int n = v.A.n;
    k_spgemm_numeric<<<grid_for(n, 128), 128, 0, s>>>(n, v.A.rowptr, v.A.col, v.A.val,
                                                      v.P.rowptr, v.P.col, v.P.val, v.AP.rowptr,
                                                      v.AP.col, v.AP.val);
    TP_LAUNCH_CHECK();
    Level& c = L[l + 1];
    k_spgemm_numeric<<<grid_for(c.A.n, 128), 128, 0, s>>>(c.A.n, v.R.rowptr, v.R.col, v.R.val,
                                                          v.AP.rowptr, v.AP.col, v.AP.val,
                                                          c.A.rowptr, c.A.col, c.A.val);
    TP_LAUNCH_CHECK();
  }
  finish_levels(s, false);
}

}  // namespace tp

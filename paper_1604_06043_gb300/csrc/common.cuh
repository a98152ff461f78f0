// Internal definitions shared by the CUDA translation units of libmsstab.
//
// Deterministic grid reductions: every reduction kernel accumulates per thread
// over a fixed row mapping, reduces per block in a fixed tree, writes one
// partial per block and takes a ticket; the last block to arrive sums the
// partials in index order.  The result does not depend on the order in which
// blocks run, and no reduction ever waits on another block (the one bounded
// wait of the library is the grid barrier of the ILU(0) level sweeps).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace msk {

constexpr int SMAX = 16;            // largest s
constexpr int LMAX = 8;             // largest l
constexpr int NT = 256;             // threads per block of the streaming kernels
constexpr int NWARP = NT / 32;
constexpr int MAXRED = 20;          // values per block in one reduction
constexpr int MAXGRP = 32;          // groups of a two-level reduction; tickets[MAXGRP] is the global one
constexpr int MAXBLK = 2048;        // blocks of one reduction group
constexpr double PIVOT_REL_TOL = 1e-14;
constexpr double CHOLQR_REL_TOL = 1e-14;   // rank test of the Cholesky QR

// Largest vector length (rows of A) the library accepts.  The grid-stride
// loops keep their row index in a signed 32-bit int and advance it by at most
// 2 * gridDim.x * blockDim.x <= 2 * MAXBLK * 1024 = 2^22 (no launch of the
// library has more than MAXBLK blocks of more than 1024 threads), so for
// n <= MAX_ROWS the index of the step after the last row stays below 2^31.
constexpr int64_t MAX_ROWS = (1LL << 31) - (1LL << 22);
static_assert(2LL * MAXBLK * 1024 <= (1LL << 22), "grid strides must stay within the MAX_ROWS margin");

// Flags raised on the device and read by the host at the cycle end.
constexpr int FLAG_BREAKDOWN = 1;
constexpr int FLAG_CHOL = 2;
constexpr int FLAG_SYNC_TIMEOUT = 4;   // a grid barrier of the ILU(0) sweeps gave up waiting
constexpr int FLAG_ZERO_PIVOT = 8;     // ILU(0) factor: u_ii == 0
constexpr int FLAG_NO_DIAG = 16;       // ILU(0) set-up: a row without a diagonal entry
constexpr int FLAG_UNSORTED = 32;      // ILU(0) set-up: columns of a row not strictly increasing

// ---------------------------------------------------------------------------
// device-resident state of one solve: projections, coefficients, norms
// ---------------------------------------------------------------------------
struct DevState {
  double projR[(LMAX + 1) * SMAX];          // [i][c] = p_c . r^(i)
  double projV[(LMAX + 1) * SMAX * SMAX];   // [i][q][c] = p_c . v_q^(i)
  double gamma[LMAX * SMAX];                // [k][j]
  double eta[LMAX * SMAX * SMAX];           // [k][q][j] (row q = eta_q)
  double gram[(LMAX + 1) * (LMAX + 1)];     // [a][c] = r^(a) . r^(c)
  double tau[LMAX];
  double rr;                                // ||r||^2 (last reduction that produced it)
  double bb;                                // ||b||^2
  double scal[2 * SMAX + 8];                // scratch scalars (Arnoldi, Cholesky QR)
  double chol[SMAX * SMAX];                 // Cholesky factor R (upper, row-major)
  double gmat[SMAX * SMAX];                 // Gram matrix for the Cholesky QR
  int flag;
};

// What the last block of a reduction kernel does after the final sums.
enum EpiKind { EPI_NONE = 0, EPI_GAMMA = 1, EPI_ETA = 2, EPI_TAU = 3 };

struct Epi {
  int kind;
  int k, q, s, ell;
  DevState* st;
};

struct RedScratch {
  double* partials;       // [blocks][values]
  double* group_out;      // [groups][values] (two-level reductions)
  unsigned int* tickets;  // [MAXGRP + 1], zero between launches
  int max_blocks;         // = MAXBLK
};

// ---------------------------------------------------------------------------
// matrices
// ---------------------------------------------------------------------------
template <typename T>
struct CsrMat {
  int n;
  const int* row_ptr;
  const int* col;
  const T* val;
};

template <typename T>
struct SellMat {           // SELL-32-sigma: slice k holds rows perm[32k .. 32k+31]
  int n;
  int nslices;
  const int* slice_ptr;    // [nslices + 1] offsets into col/val
  const int* slice_w;      // [nslices] entries per row in the slice
  const int* perm;         // position -> original row, or NULL (sigma = 1)
  const int* col;          // [slice_ptr[k] + j*32 + lane]
  const T* val;
};

// ---------------------------------------------------------------------------
// FP32 partial sums into the FP64 reductions.  A thread's FP32 dot partial
// (a dozen rows) is exact to about 1e-6 of its terms, the level of the FP32
// vectors themselves; the block and grid reductions are FP64.  The widening
// is done with integer operations: this GPU converts between FP32 and FP64 on
// its FP64 unit (1/64 of the FP32 rate), where a conversion per accumulator
// and warp costs as much as the whole FP32 row loop.  Zero, subnormal and
// non-finite values (rare) take the converting instruction.
// ---------------------------------------------------------------------------
__device__ __forceinline__ double widen_f32(float f) {
  const unsigned u = __float_as_uint(f);
  const unsigned e = (u >> 23) & 0xffu;
  if ((u & 0x7fffffffu) == 0u) return __longlong_as_double((long long)((unsigned long long)u << 32));
  if (e == 0u || e == 0xffu) return (double)f;
  const unsigned long long d = ((unsigned long long)(u & 0x80000000u) << 32) |
                               ((unsigned long long)(e + 896u) << 52) |
                               ((unsigned long long)(u & 0x7fffffu) << 29);
  return __longlong_as_double((long long)d);
}

// ---------------------------------------------------------------------------
// block-partitioned cut space.  When every row i of P has its only non-zero
// in column c(i) = (i / 32) mod s (32-row blocks dealt round-robin to the s
// columns), P^T y needs one multiply-add per row instead of s.  A warp always
// handles 32 consecutive rows starting at a multiple of 32, so c is the same
// for all its lanes and the switch below runs one branch (an FP64 multiply-
// add predicated off would still occupy the FP64 unit of this GPU).
// ---------------------------------------------------------------------------
__host__ __device__ __forceinline__ int pblock_col(int64_t row, int s) { return (int)((row >> 5) % s); }

template <int NP, typename Acc, typename T>
__device__ __forceinline__ void add_to_slot(Acc& acc, int c, T y, T p) {
  switch (c) {
#define MSK_SLOT(J) \
  case J:           \
    if constexpr (J < NP) acc.add(J, y, p); \
    break;
    MSK_SLOT(0) MSK_SLOT(1) MSK_SLOT(2) MSK_SLOT(3) MSK_SLOT(4) MSK_SLOT(5) MSK_SLOT(6) MSK_SLOT(7)
    MSK_SLOT(8) MSK_SLOT(9) MSK_SLOT(10) MSK_SLOT(11) MSK_SLOT(12) MSK_SLOT(13) MSK_SLOT(14) MSK_SLOT(15)
#undef MSK_SLOT
    default:
      break;
  }
}

// ---------------------------------------------------------------------------
// reductions
// ---------------------------------------------------------------------------
__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Reduce-scatter inside a warp: CNT values per lane, exchanged over xor
// distance O, O/2, ..., 1.  While more than one value is left, each lane keeps
// half of them (the upper half if bit O of its lane id is set) and adds the
// partner's copy of that half, so a lane spends CNT/2 + CNT/4 + ... additions
// instead of 5 per value.  Afterwards v[0] of lane L holds the warp sum of
// value index rs_index<CNT>(L).
template <typename V, int CNT, int O, int M>
struct RedScatterT {
  static __device__ __forceinline__ void run(V (&v)[M], int lane) {
    if constexpr (CNT > 1) {
      constexpr int H = CNT / 2;
      const bool up = (lane & O) != 0;
#pragma unroll
      for (int i = 0; i < H; ++i) {
        const V send = up ? v[i] : v[i + H];
        const V keep = up ? v[i + H] : v[i];
        v[i] = keep + __shfl_xor_sync(0xffffffffu, send, O);
      }
      if constexpr (O > 1) RedScatterT<V, H, O / 2, M>::run(v, lane);
    } else {
      v[0] += __shfl_xor_sync(0xffffffffu, v[0], O);
      if constexpr (O > 1) RedScatterT<V, 1, O / 2, M>::run(v, lane);
    }
  }
};
template <int CNT, int O, int M>
using RedScatter = RedScatterT<double, CNT, O, M>;

template <int M>
__device__ __forceinline__ int rs_index(int lane) {
  int idx = 0, cnt = M;
#pragma unroll
  for (int o = 16; o >= 1; o >>= 1) {
    if (cnt > 1) {
      cnt >>= 1;
      if (lane & o) idx += cnt;
    }
  }
  return idx;
}

// Reduce v[0..m) (m <= M, M a power of two <= 32) of all threads of the block
// into red[0..m) (shared), in a fixed order.  Uses smem_w[NWARP * MAXRED].
// Ends with a __syncthreads().
template <int M>
__device__ __forceinline__ void block_reduce(double (&v)[M], int m, double* smem_w, double* red) {
  static_assert(M >= 1 && M <= 32 && (M & (M - 1)) == 0, "M must be a power of two <= 32");
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  RedScatter<M, 16, M>::run(v, lane);
  // lanes whose low bits (those not used to split values) are zero publish
  constexpr int SPLIT_BITS = M >= 32 ? 5 : (M >= 16 ? 4 : (M >= 8 ? 3 : (M >= 4 ? 2 : (M >= 2 ? 1 : 0))));
  constexpr int LOW_MASK = (1 << (5 - SPLIT_BITS)) - 1;
  const int idx = rs_index<M>(lane);
  if ((lane & LOW_MASK) == 0 && idx < m) smem_w[w * MAXRED + idx] = v[0];
  __syncthreads();
  if (threadIdx.x < m) {
    // four independent chains over the warps (fixed order), then their sum
    const int nw = (int)(blockDim.x >> 5);
    double s0 = 0.0, s1 = 0.0, s2 = 0.0, s3 = 0.0;
    int j = 0;
    for (; j + 3 < nw; j += 4) {
      s0 += smem_w[j * MAXRED + threadIdx.x];
      s1 += smem_w[(j + 1) * MAXRED + threadIdx.x];
      s2 += smem_w[(j + 2) * MAXRED + threadIdx.x];
      s3 += smem_w[(j + 3) * MAXRED + threadIdx.x];
    }
    for (; j < nw; ++j) s0 += smem_w[j * MAXRED + threadIdx.x];
    red[threadIdx.x] = (s0 + s1) + (s2 + s3);
  }
  __syncthreads();
}

// block_reduce for FP32 partials (the FP32 inner form's dots): the warp stage
// in FP32 (reduce-scatter), the warps' sums widened exactly and added in FP64
// in block_reduce's order.  FP64 additions cost 64 times FP32 ones on this GPU;
// the warp stage would otherwise dominate a short reduction kernel.
template <int M>
__device__ __forceinline__ void block_reduce_f32(float (&v)[M], int m, double* smem_w, double* red) {
  static_assert(M >= 1 && M <= 32 && (M & (M - 1)) == 0, "M must be a power of two <= 32");
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  RedScatterT<float, M, 16, M>::run(v, lane);
  constexpr int SPLIT_BITS = M >= 32 ? 5 : (M >= 16 ? 4 : (M >= 8 ? 3 : (M >= 4 ? 2 : (M >= 2 ? 1 : 0))));
  constexpr int LOW_MASK = (1 << (5 - SPLIT_BITS)) - 1;
  const int idx = rs_index<M>(lane);
  if ((lane & LOW_MASK) == 0 && idx < m) smem_w[w * MAXRED + idx] = widen_f32(v[0]);
  __syncthreads();
  if (threadIdx.x < m) {
    const int nw = (int)(blockDim.x >> 5);
    double s0 = 0.0, s1 = 0.0, s2 = 0.0, s3 = 0.0;
    int j = 0;
    for (; j + 3 < nw; j += 4) {
      s0 += smem_w[j * MAXRED + threadIdx.x];
      s1 += smem_w[(j + 1) * MAXRED + threadIdx.x];
      s2 += smem_w[(j + 2) * MAXRED + threadIdx.x];
      s3 += smem_w[(j + 3) * MAXRED + threadIdx.x];
    }
    for (; j < nw; ++j) s0 += smem_w[j * MAXRED + threadIdx.x];
    red[threadIdx.x] = (s0 + s1) + (s2 + s3);
  }
  __syncthreads();
}

// Sum the m values of the nblk per-block partials at base (partial b, value i
// at base[b * MAXRED + i]) into red[0..m) in a fixed order: warp w takes
// values w, w + nwarps, ...; its lanes stride over the blocks with four
// independent chains (four loads in flight per lane), then a warp sum.  The
// result depends only on the partials, never on which block sums them.  Reads
// through L2 (the partials come from other blocks).  Ends with __syncthreads.
__device__ __forceinline__ void sum_partials(const double* base, int nblk, int m, double* red) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int i = w; i < m; i += nw) {
    double v0 = 0.0, v1 = 0.0, v2 = 0.0, v3 = 0.0;
    if (nblk <= 160) {
      // up to five partials per lane, all loaded before the first addition; the
      // additions are those of the loops below, in their order
      double r[5];
#pragma unroll
      for (int u = 0; u < 5; ++u) r[u] = lane + 32 * u < nblk ? __ldcg(base + (size_t)(lane + 32 * u) * MAXRED + i) : 0.0;
      if (lane + 96 < nblk) {
        v0 += r[0];
        v1 += r[1];
        v2 += r[2];
        v3 += r[3];
        if (lane + 128 < nblk) v0 += r[4];
      } else {
        if (lane < nblk) v0 += r[0];
        if (lane + 32 < nblk) v0 += r[1];
        if (lane + 64 < nblk) v0 += r[2];
      }
      double v = warp_sum((v0 + v1) + (v2 + v3));
      if (lane == 0) red[i] = v;
      continue;
    }
    int b = lane;
    for (; b + 96 < nblk; b += 128) {
      v0 += __ldcg(base + (size_t)b * MAXRED + i);
      v1 += __ldcg(base + (size_t)(b + 32) * MAXRED + i);
      v2 += __ldcg(base + (size_t)(b + 64) * MAXRED + i);
      v3 += __ldcg(base + (size_t)(b + 96) * MAXRED + i);
    }
    for (; b < nblk; b += 32) v0 += __ldcg(base + (size_t)b * MAXRED + i);
    double v = warp_sum((v0 + v1) + (v2 + v3));
    if (lane == 0) red[i] = v;
  }
  __syncthreads();
}

// Publish this block's m values as partial `blk` of group `grp` (nblk blocks in
// the group) and take a ticket.  Returns true in the last block of the group,
// which then holds the group's sums (in block order) in red[0..m).  The group's
// ticket is reset for the next launch.
__device__ __forceinline__ bool grid_reduce(RedScratch rs, int grp, int blk, int nblk, int m, double* red,
                                            int* s_last) {
  double* part = rs.partials + ((size_t)grp * rs.max_blocks + blk) * MAXRED;
  if (threadIdx.x < m) part[threadIdx.x] = red[threadIdx.x];
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned t = atomicAdd(&rs.tickets[grp], 1u);
    *s_last = (t == (unsigned)(nblk - 1));
  }
  __syncthreads();
  if (!*s_last) return false;
  __threadfence();
  sum_partials(rs.partials + (size_t)grp * rs.max_blocks * MAXRED, nblk, m, red);
  if (threadIdx.x == 0) rs.tickets[grp] = 0u;
  return true;
}

// ---------------------------------------------------------------------------
// bounded grid barrier of the persistent (cooperative) kernels
// ---------------------------------------------------------------------------
__device__ __forceinline__ void red_release_add_u32(unsigned int* p, unsigned int v) {
  asm volatile("red.release.gpu.global.add.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

__device__ __forceinline__ unsigned int ld_acquire_u32(const unsigned int* p) {
  unsigned int v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

// All blocks of a cooperative launch meet here.  *count is zero at launch; the
// barrier numbered `gen` (1, 2, ...) completes when it reaches gen * gridDim.x.
// Thread 0 raises the counter with release semantics (after the block's
// __syncthreads, so the stores of every thread of the block are ordered
// before it) and polls with acquire loads.  Bounded: after spin_limit polls it
// raises FLAG_SYNC_TIMEOUT in *flag and gives up; a block that sees the flag
// gives up too.  Returns false (in every thread of the block) on giving up:
// the caller must then leave the kernel.
__device__ __forceinline__ bool grid_sync(unsigned int* count, unsigned int gen, int* flag, long long spin_limit,
                                          int* s_ok) {
  __syncthreads();
  if (threadIdx.x == 0) {
    int ok = 1;
    const unsigned int target = gen * gridDim.x;
    red_release_add_u32(count, 1u);
    for (long long it = 0; ld_acquire_u32(count) < target; ++it) {
      if ((it & 63) == 63 && (*(const volatile int*)flag & FLAG_SYNC_TIMEOUT)) {
        ok = 0;
        break;
      }
      if (it >= spin_limit) {
        atomicOr(flag, FLAG_SYNC_TIMEOUT);
        ok = 0;
        break;
      }
    }
    *s_ok = ok;
  }
  __syncthreads();
  return *s_ok != 0;
}

// Second level: after the last block of group grp has its sums, publish them
// and take the global ticket.  Returns true in the very last group's block,
// which can then read every group's sums from rs.group_out.
__device__ __forceinline__ bool groups_done(RedScratch rs, int grp, int ngrp, int m, const double* red,
                                            int* s_last) {
  if (threadIdx.x < m) rs.group_out[grp * MAXRED + threadIdx.x] = red[threadIdx.x];
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned t = atomicAdd(&rs.tickets[MAXGRP], 1u);
    *s_last = (t == (unsigned)(ngrp - 1));
  }
  __syncthreads();
  if (!*s_last) return false;
  __threadfence();
  if (threadIdx.x == 0) rs.tickets[MAXGRP] = 0u;
  return true;
}

// ---------------------------------------------------------------------------
// small dense solves (single thread; n <= SMAX)
// ---------------------------------------------------------------------------

// Gaussian elimination with partial pivoting on a (n x n, row-major, modified)
// and z (rhs in, solution out).  Returns false (z zeroed) when the pivot of
// column k is below PIVOT_REL_TOL times the largest magnitude in column k of
// the input (a zero column included).  The test is per column: the columns of
// a projected matrix P^T W differ in scale by orders of magnitude, and column
// scaling changes neither solvability nor the pivot rows chosen.
__device__ inline bool lu_solve_pp(double* a, double* z, int n) {
  double colmax[SMAX];
  bool ok = true;
  for (int j = 0; j < n; ++j) {
    double m = 0.0;
    for (int i = 0; i < n; ++i) m = fmax(m, fabs(a[i * n + j]));
    colmax[j] = m;
    if (!(m > 0.0 && isfinite(m))) ok = false;
  }
  for (int k = 0; ok && k < n; ++k) {
    int p = k;
    double best = fabs(a[k * n + k]);
    for (int i = k + 1; i < n; ++i) {
      double v = fabs(a[i * n + k]);
      if (v > best) { best = v; p = i; }
    }
    if (!(best >= PIVOT_REL_TOL * colmax[k])) { ok = false; break; }
    if (p != k) {
      for (int j = 0; j < n; ++j) { double t = a[k * n + j]; a[k * n + j] = a[p * n + j]; a[p * n + j] = t; }
      double t = z[k]; z[k] = z[p]; z[p] = t;
    }
    const double piv = a[k * n + k];
    for (int i = k + 1; i < n; ++i) {
      const double l = a[i * n + k] / piv;
      for (int j = k; j < n; ++j) a[i * n + j] -= l * a[k * n + j];
      z[i] -= l * z[k];
    }
  }
  if (!ok) {
    for (int i = 0; i < n; ++i) z[i] = 0.0;
    return false;
  }
  for (int k = n - 1; k >= 0; --k) {
    double v = z[k];
    for (int j = k + 1; j < n; ++j) v -= a[k * n + j] * z[j];
    z[k] = v / a[k * n + k];
  }
  return true;
}

// The same elimination by one warp (all 32 lanes call it), arranged for a
// GPU whose FP64 unit retires one warp instruction per 16 SM cycles or so:
// every FP64 instruction of this latency-bound solve costs the whole warp that
// long, whatever its active lanes, so the solve is built to issue few of them.
//  - Lane l owns row l % R (R = smallest power of two >= n) and the columns
//    j = l / R + m (32 / R), m = 0, 1, ..., of the augmented matrix [a | z]
//    (shared memory); every step updates all owned elements at once.
//  - Pivot search and the breakdown test compare magnitudes as the integer
//    bit patterns of |a| (order-preserving for non-negative doubles): no FP64
//    instruction.  Pivot row p = the first row with the largest |a_ik|, i >= k,
//    breakdown when |a_pk| < PIVOT_REL_TOL * max_i |a_ik (input)|, as in
//    lu_solve_pp; a non-finite entry of a is a breakdown too.
//  - Gauss-Jordan: step k eliminates column k from every other row with the
//    multiplier a_ik / a_kk (the formula of lu_solve_pp), so that the
//    solution is z_i = [a | z]_in / a_ii after the last step (no sequential
//    back substitution).  Rows below k see the operations of partial-pivoting
//    LU; rows above k take the back substitution column by column.
// Returns the warp-uniform result; z is zeroed on breakdown.  a (n x n, row
// major) and z are overwritten.
__device__ inline bool warp_lu_solve(double* a, double* z, int n, double* lbuf) {
  (void)lbuf;
  const unsigned FULL = 0xffffffffu;
  const long long MAG = 0x7fffffffffffffffLL, INF_BITS = 0x7ff0000000000000LL;
  const int lane = threadIdx.x & 31;
  const int R = n <= 1 ? 1 : (n <= 2 ? 2 : (n <= 4 ? 4 : (n <= 8 ? 8 : (n <= 16 ? 16 : 32))));
  const int C = 32 / R;
  const int row = lane % R, c0 = lane / R;
  // element (i, j) of [a | z]: a[i*n + j] for j < n, z[i] for j == n
  auto at = [&](int i, int j) -> double& { return j < n ? a[i * n + j] : z[i]; };
  // column maxima of the input and finiteness, as integer magnitudes
  __shared__ long long thr_key[SMAX];
  bool bad = false;
  for (int j = lane; j < n; j += 32) {
    long long cm = 0;
    for (int i = 0; i < n; ++i) {
      const long long m = __double_as_longlong(a[i * n + j]) & MAG;
      bad |= m >= INF_BITS;
      cm = m > cm ? m : cm;
    }
    bad |= cm == 0;
    thr_key[j] = __double_as_longlong(PIVOT_REL_TOL * __longlong_as_double(cm));
  }
  bool ok = !__any_sync(FULL, bad);
  __syncwarp();
  for (int k = 0; ok && k < n; ++k) {
    // first row p >= k with the largest |a_pk|: the 63-bit magnitude compared
    // as (high word, low word) with warp max-reductions, then the lowest lane
    // holding that maximum
    const bool valid = lane >= k && lane < n;
    const long long mag = valid ? (__double_as_longlong(a[lane * n + k]) & MAG) : 0LL;
    const unsigned hi = (unsigned)((unsigned long long)mag >> 32), lo = (unsigned)mag;
    const unsigned mhi = __reduce_max_sync(FULL, valid ? hi : 0u);
    const unsigned mlo = __reduce_max_sync(FULL, (valid && hi == mhi) ? lo : 0u);
    const int idx = (int)__reduce_min_sync(FULL, (valid && hi == mhi && lo == mlo) ? (unsigned)lane : 32u);
    const long long key = (long long)(((unsigned long long)mhi << 32) | mlo);
    if (key < thr_key[k]) {
      ok = false;
      break;
    }
    const int p = idx;
    if (p != k) {
      for (int j = lane; j <= n; j += 32) {
        const double tmp = at(k, j);
        at(k, j) = at(p, j);
        at(p, j) = tmp;
      }
      __syncwarp();
    }
    if (row < n && row != k) {
      const double l = a[row * n + k] / a[k * n + k];
      // owned columns j > k: the first is k + 1 + ((c0 - k - 1) mod C)
      for (int j = k + 1 + (((c0 - k - 1) % C) + C) % C; j <= n; j += C) at(row, j) -= l * at(k, j);
    }
    __syncwarp();
  }
  if (!ok) {
    if (lane < n) z[lane] = 0.0;
    __syncwarp();
    return false;
  }
  if (lane < n) z[lane] = z[lane] / a[lane * n + lane];
  __syncwarp();
  return true;
}

// Upper Cholesky factor R (row-major, R^T R = G) of the n x n matrix G.
// Returns false if a pivot d_j is not above rel_tol * G_jj (rel_tol = 0: not
// positive; a positive rel_tol detects numerically rank-deficient bases).
__device__ inline bool cholesky_upper(const double* G, double* R, int n, double rel_tol = 0.0) {
  for (int i = 0; i < n * n; ++i) R[i] = 0.0;
  for (int j = 0; j < n; ++j) {
    double d = G[j * n + j];
    for (int i = 0; i < j; ++i) d -= R[i * n + j] * R[i * n + j];
    if (!(d > rel_tol * G[j * n + j])) return false;
    const double rjj = sqrt(d);
    R[j * n + j] = rjj;
    for (int k = j + 1; k < n; ++k) {
      double v = G[j * n + k];
      for (int i = 0; i < j; ++i) v -= R[i * n + j] * R[i * n + k];
      R[j * n + k] = v / rjj;
    }
  }
  return true;
}

// tau from the (l+1) x (l+1) Gram matrix of [r^(0..l)] (row-major): scaled
// normal equations, Cholesky, LU on failure; tau = 0 if a level vector is zero.
// wk: 2*LMAX*LMAX + 2*LMAX doubles of scratch.
__device__ inline void tau_from_gram(const double* G, int ell, double* tau, double* wk) {
  const int L = ell + 1;
  double* M = wk;
  double* R = wk + LMAX * LMAX;
  double* d = wk + 2 * LMAX * LMAX;
  double* y = d + LMAX;
  for (int i = 0; i < ell; ++i) {
    const double g = G[(i + 1) * L + (i + 1)];
    if (!(g > 0.0)) {
      for (int k = 0; k < ell; ++k) tau[k] = 0.0;
      return;
    }
    d[i] = 1.0 / sqrt(g);
  }
  for (int i = 0; i < ell; ++i) {
    for (int j = 0; j < ell; ++j) M[i * ell + j] = d[i] * G[(i + 1) * L + (j + 1)] * d[j];
    y[i] = d[i] * G[(i + 1) * L + 0];
  }
  if (cholesky_upper(M, R, ell)) {
    for (int i = 0; i < ell; ++i) {        // R^T w = y
      double v = y[i];
      for (int k = 0; k < i; ++k) v -= R[k * ell + i] * y[k];
      y[i] = v / R[i * ell + i];
    }
    for (int i = ell - 1; i >= 0; --i) {   // R z = w
      double v = y[i];
      for (int k = i + 1; k < ell; ++k) v -= R[i * ell + k] * y[k];
      y[i] = v / R[i * ell + i];
    }
  } else {
    for (int i = 0; i < ell; ++i)
      for (int j = 0; j < ell; ++j) M[i * ell + j] = d[i] * G[(i + 1) * L + (j + 1)] * d[j];
    for (int i = 0; i < ell; ++i) y[i] = d[i] * G[(i + 1) * L + 0];
    if (!lu_solve_pp(M, y, ell))
      for (int i = 0; i < ell; ++i) y[i] = 0.0;
  }
  for (int i = 0; i < ell; ++i) tau[i] = d[i] * y[i];
}

// Scratch of the epilogue's small solves (shared memory of the last block).
struct EpiScratch {
  double a[SMAX * SMAX];
  double z[SMAX];
  double l[SMAX];
  double g[(LMAX + 1) * (LMAX + 1)];
  double wk[2 * LMAX * LMAX + 2 * LMAX];
};

// The small solve that follows a reduction, run by warp 0 of the last block
// (all 32 lanes call it; the coefficient solves are warp-parallel).
__device__ inline void run_epilogue(const Epi& e, EpiScratch& w) {
  if (e.kind == EPI_NONE) return;
  const int lane = threadIdx.x & 31;
  DevState* st = e.st;
  const int s = e.s;
  if (e.kind == EPI_GAMMA || e.kind == EPI_ETA) {
    // GAMMA: (P^T V^(k)) gamma = P^T r^(k);  ETA: (P^T W^(k)) eta_q = P^T r^(k+1)
    // with W^(k) = [V^(k+1)_{0:q-1}, V^(k)_{q:s-1}]
    const int rlev = e.kind == EPI_GAMMA ? e.k : e.k + 1;
    for (int i = lane; i < s * s; i += 32) {
      const int c = i / s, j = i % s;
      const int lev = (e.kind == EPI_ETA && j < e.q) ? e.k + 1 : e.k;
      w.a[i] = __ldcg(&st->projV[(lev * SMAX + j) * SMAX + c]);
    }
    if (lane < s) w.z[lane] = __ldcg(&st->projR[rlev * SMAX + lane]);
    __syncwarp();
    const bool ok = warp_lu_solve(w.a, w.z, s, w.l);
    if (lane == 0 && !ok) st->flag |= FLAG_BREAKDOWN;
    double* out = e.kind == EPI_GAMMA ? &st->gamma[e.k * SMAX] : &st->eta[(e.k * SMAX + e.q) * SMAX];
    if (lane < s) out[lane] = w.z[lane];
  } else if (e.kind == EPI_TAU) {
    const int L = e.ell + 1;
    for (int i = lane; i < L * L; i += 32) w.g[i] = __ldcg(&st->gram[i]);
    __syncwarp();
    if (lane == 0) tau_from_gram(w.g, e.ell, st->tau, w.wk);
  }
}

// ---------------------------------------------------------------------------
// launch helpers
// ---------------------------------------------------------------------------
struct LaunchCfg {
  int sms;              // multiprocessors
  int blocks_per_sm;    // resident blocks of NT threads we aim for
};

inline int grid_for(const LaunchCfg& lc, int64_t work_items, int items_per_block, int max_blocks) {
  int64_t need = (work_items + items_per_block - 1) / items_per_block;
  int64_t cap = (int64_t)lc.sms * lc.blocks_per_sm;
  if (cap > max_blocks) cap = max_blocks;
  if (need > cap) need = cap;
  if (need < 1) need = 1;
  return (int)need;
}

}  // namespace msk

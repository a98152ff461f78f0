// ILU(0) split preconditioning (the ocean experiment of Section 5.1): the
// systems L^-1 A U^-1 x~ = L^-1 b with L unit lower and U upper triangular on
// the sparsity pattern of A, the incomplete LU factorisation with zero fill-in.
//
// Factor.  Row i is reduced by the finished rows k < i of its strict lower
// part, in increasing k (the IKJ form of Gaussian elimination), and every
// update that would land outside A's pattern is dropped: l_ik = a_ik / u_kk,
// then a_ij -= l_ik u_kj for the j > k that rows i and k share.  Each update is
// a rounded multiplication followed by a rounded subtraction (no fused
// multiply-add), so the factor is the textbook sequential one bit for bit.
// The values are stored on A's CSR pattern: left of the diagonal L (unit
// diagonal implicit), from the diagonal on U.
//
// Schedule.  Row i of the factor and of the lower solve needs the rows of its
// strict lower part finished first; the upper solve needs those of its strict
// upper part.  The level of a row is the length of the longest such chain
// below it, so all rows of one level are independent: they are computed in
// parallel, level after level, in ONE cooperative launch whose blocks meet at
// a grid barrier between levels (a 7-point stencil on an n^3 grid in natural
// order has 3n - 2 levels, the planes x + y + z = const).  The levels are
// found on the device by relaxing lev(i) = 1 + max lev(j) over the
// dependencies until nothing changes (values only grow towards the fixed
// point), then rows are bucketed by level with a counting sort.
//
// The barrier between levels is the only place where a thread waits on
// another block.  Every block of a cooperative launch is resident and runs the
// same number of barriers.  The barrier is a counter, zeroed before the
// launch, that thread 0 of every block raises by one with release semantics
// after its block's rows (so the rows' stores are visible first) and then polls
// with acquire loads until it reaches (level + 1) x blocks.  Every wait is
// bounded: after spin_limit polls (IluDesc::spin_limit, 2^22 unless the
// handle's options set it) the block raises FLAG_SYNC_TIMEOUT in
// the device flag word and leaves, the blocks still waiting see the flag and
// leave too, and the host reads the flag at the next cycle end.  Values
// written by other blocks are read through L2 (__ldcg), never from a possibly
// stale L1 line.

#include <algorithm>
#include <vector>

#include "launch.h"
#include "msstab.h"

namespace msk {

constexpr int ITS = 256;                       // threads per block of the level sweeps

__device__ __forceinline__ void red_release_add(unsigned int* p, unsigned int v) {
  asm volatile("red.release.gpu.global.add.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

__device__ __forceinline__ unsigned int ld_acquire(const unsigned int* p) {
  unsigned int v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

// The barrier after level l (see the file comment): false if it timed out.
__device__ __forceinline__ bool level_barrier(unsigned int* count, unsigned int target, int* flag,
                                              long long spin_limit) {
  __shared__ int s_ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    int ok = 1;
    red_release_add(count, 1u);
    for (long long it = 0; ld_acquire(count) < target; ++it) {
      if ((it & 255) == 255 && (*(const volatile int*)flag & FLAG_SYNC_TIMEOUT)) {
        ok = 0;
        break;
      }
      if (it > spin_limit) {
        atomicOr(flag, FLAG_SYNC_TIMEOUT);
        ok = 0;
        break;
      }
    }
    s_ok = ok;
  }
  __syncthreads();
  return s_ok != 0;
}

enum SweepMode { SW_FACTOR = 0, SW_LOWER = 1, SW_UPPER = 2 };

struct SweepArgs {
  int nlev;
  const int* lptr;     // rows of level l: rows[lptr[l] .. lptr[l+1])
  const int* rows;
  const int* rp;
  const int* col;
  const int* dg;
  double* lu;
  const double* in;    // right-hand side (the solves)
  double* out;         // solution (may equal in)
  unsigned int* count; // barrier counter (zero at launch)
  int* flag;
  long long spin_limit;
};

template <int MODE>
__global__ void __launch_bounds__(ITS) ilu_sweep_kernel(SweepArgs a) {
  const int G = gridDim.x * ITS;
  const int tid = blockIdx.x * ITS + threadIdx.x;
  for (int l = 0; l < a.nlev; ++l) {
    const int beg = a.lptr[l], end = a.lptr[l + 1];
    for (int idx = beg + tid; idx < end; idx += G) {
      const int i = a.rows[idx];
      const int rb = a.rp[i], re = a.rp[i + 1], d = a.dg[i];
      if constexpr (MODE == SW_FACTOR) {
        for (int p = rb; p < d; ++p) {
          const int k = a.col[p];
          const double piv = __ldcg(a.lu + a.dg[k]);
          const double lik = __ddiv_rn(__ldcg(a.lu + p), piv);
          __stcg(a.lu + p, lik);
          int q = a.dg[k] + 1, t = p + 1;
          const int qe = a.rp[k + 1];
          while (q < qe && t < re) {
            const int cq = a.col[q], ct = a.col[t];
            if (cq == ct) {
              __stcg(a.lu + t, __dsub_rn(__ldcg(a.lu + t), __dmul_rn(lik, __ldcg(a.lu + q))));
              ++q;
              ++t;
            } else if (cq < ct) {
              ++q;
            } else {
              ++t;
            }
          }
        }
        if (__ldcg(a.lu + d) == 0.0) atomicOr(a.flag, FLAG_ZERO_PIVOT);
      } else if constexpr (MODE == SW_LOWER) {
        double sum = a.in[i];
        for (int p = rb; p < d; ++p) sum = fma(-a.lu[p], __ldcg(a.out + a.col[p]), sum);
        __stcg(a.out + i, sum);
      } else {
        double sum = a.in[i];
        for (int p = d + 1; p < re; ++p) sum = fma(-a.lu[p], __ldcg(a.out + a.col[p]), sum);
        __stcg(a.out + i, sum / a.lu[d]);
      }
    }
    if (l + 1 < a.nlev && !level_barrier(a.count, (unsigned)(l + 1) * gridDim.x, a.flag, a.spin_limit)) return;
  }
}

// The packed solves, level by level.  Each level's segment of the packed order
// is padded to a multiple of 32 positions (padding holds row -1), so the lanes
// of a warp work on rows of one level.  Nothing a row needs except the
// solution values of earlier levels depends on the solve, so the next level's
// row data (row index, dependencies, factor values, right-hand side) is loaded
// before the barrier that ends the current level; a row's dependency values
// are then gathered in one round trip through L2.  Sums run over the
// dependencies in column order, as the CSR sweep.
struct PackedArgs {
  int n;                 // padded positions
  const int* rows;       // row of each position, -1 for padding
  const int* pcnt;
  const int* pcol;
  const double* pval;
  const double* pdiag;   // upper solve: u_ii by position; NULL: unit diagonal
  const double* in;
  double* out;           // may equal in
  int* flag;
  long long spin_limit;
};

template <int W>
struct RowData {
  int row, cnt;
  int col[W];
  double val[W];
  double rhs, diag;
};

template <int W>
__device__ __forceinline__ void load_row(const PackedArgs& a, int idx, RowData<W>& r) {
  r.row = __ldg(a.rows + idx);
  r.cnt = __ldg(a.pcnt + idx);      // 0 for padding
#pragma unroll
  for (int j = 0; j < W; ++j) {
    if (j < r.cnt) {
      r.col[j] = __ldg(a.pcol + (int64_t)j * a.n + idx);
      r.val[j] = __ldg(a.pval + (int64_t)j * a.n + idx);
    }
  }
  // a plain load: with in == out other rows of in change during the launch
  // (this row's entry does not before the row is solved)
  r.rhs = r.row >= 0 ? a.in[r.row] : 0.0;
  r.diag = a.pdiag ? __ldg(a.pdiag + idx) : 1.0;
}

struct LevelArgs {
  PackedArgs p;
  int nlev;
  const int* pptr;       // padded positions of level l: [pptr[l], pptr[l+1])
  unsigned int* count;
};

template <int W>
__device__ __forceinline__ void level_row(const PackedArgs& a, const RowData<W>& r) {
  double x[W];
#pragma unroll
  for (int j = 0; j < W; ++j) x[j] = j < r.cnt ? __ldcg(a.out + r.col[j]) : 0.0;
  double sum = r.rhs;
#pragma unroll
  for (int j = 0; j < W; ++j)
    if (j < r.cnt) sum = fma(-r.val[j], x[j], sum);
  if (a.pdiag) sum = sum / r.diag;
  if (r.row >= 0) __stcg(a.out + r.row, sum);
}

template <int W>
__global__ void __launch_bounds__(ITS) ilu_sweep_level_kernel(LevelArgs L) {
  const PackedArgs& a = L.p;
  const int G = gridDim.x * ITS;
  const int tid = blockIdx.x * ITS + threadIdx.x;
  RowData<W> nxt;
  int beg = L.pptr[0], end = L.pptr[1];
  if (beg + tid < end) load_row<W>(a, beg + tid, nxt);
  for (int l = 0; l < L.nlev; ++l) {
    const bool mine = beg + tid < end;
    const RowData<W> cur = nxt;
    const int cbeg = beg, cend = end;
    if (l + 1 < L.nlev) {
      beg = L.pptr[l + 1];
      end = L.pptr[l + 2];
      if (beg + tid < end) load_row<W>(a, beg + tid, nxt);
    }
    if (mine) {
      level_row<W>(a, cur);
      for (int idx = cbeg + tid + G; idx < cend; idx += G) {   // levels wider than the grid
        RowData<W> r;
        load_row<W>(a, idx, r);
        level_row<W>(a, r);
      }
    }
    if (l + 1 < L.nlev && !level_barrier(L.count, (unsigned)(l + 1) * gridDim.x, a.flag, a.spin_limit)) return;
  }
}

// dependencies of the level-ordered rows: count and the widest row
// (W == 0: only the widest row into *maxdeps.)  Position idx of the level
// order goes to padded position pptr[l] + (idx - lptr[l]) of its level l.
__global__ void ilu_pack_kernel(int n, int npad, int upper, int W, const int* rows, const int* lev,
                                const int* lptr, const int* pptr, const int* rp, const int* col, const int* dg,
                                const double* lu, int* prow, int* pcnt, int* pcol, double* pval, double* pdiag,
                                int* maxdeps) {
  const int stride = gridDim.x * blockDim.x;
  int md = 0;
  for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < n; idx += stride) {
    const int i = rows[idx];
    const int b = upper ? dg[i] + 1 : rp[i], e = upper ? rp[i + 1] : dg[i];
    md = max(md, e - b);
    if (W > 0) {
      const int l = lev[i];
      const int pp = pptr[l] + (idx - lptr[l]);
      prow[pp] = i;
      pcnt[pp] = e - b;
      for (int p = b; p < e; ++p) {
        pcol[(int64_t)(p - b) * npad + pp] = col[p];
        pval[(int64_t)(p - b) * npad + pp] = lu[p];
      }
      if (upper) pdiag[pp] = lu[dg[i]];
    }
  }
  if (maxdeps) atomicMax(maxdeps, md);
}

// level sizes rounded up to whole warps
__global__ void ilu_pad_counts_kernel(int nlev, const int* lptr, int* cnt) {
  const int stride = gridDim.x * blockDim.x;
  for (int l = blockIdx.x * blockDim.x + threadIdx.x; l < nlev; l += stride)
    cnt[l] = (lptr[l + 1] - lptr[l] + 31) / 32 * 32;
}

// ---------------------------------------------------------------------------
// Pipelined solves over row chunks.  Rows are cut into contiguous chunks, one
// per block (one block per SM).  Inside a chunk the rows are grouped by their
// level (the same levels as the level-by-level sweep); the block runs its
// groups in level order with a block barrier between them.  Keeping the
// global level order inside every chunk is what makes the pipeline short: a
// row of level l needs values of levels below l only, which the neighbouring
// chunk produces early in its own order (ordering a chunk by levels counted
// inside the chunk alone made a chunk wait for the end of its neighbour: 30x
// slower).
// Values.  The block keeps the values of the group just solved and of the one
// being solved in a shared-memory double buffer (GMAX each); a dependency in
// the previous group of the same chunk is packed as its offset there.  Every
// other dependency -- in another chunk (an earlier one for the lower solve, a
// later one for the upper) or in an older group of the same chunk -- is read
// from the global solution vector, which starts filled with a sentinel bit
// pattern (all ones: a NaN no arithmetic produces; the GPU's NaN results are
// the positive canonical one) and is polled with relaxed loads until the
// owning block has written it; values of the block's own older groups are
// final there once the barrier after their group has passed.  In natural
// order every dependency of a stencil row is exactly one level below it, so
// nearly all in-chunk dependencies come from the buffer, and the chunk size
// does not depend on shared memory.
// Termination.  A chunk waits only on chunks on one side of it, the first
// chunk on that side waits on none, and a cooperative launch keeps every block
// resident, so the sweep completes; every wait is bounded (spin_limit
// polls, then FLAG_SYNC_TIMEOUT and NaN), and a thread that sees the flag
// stops waiting.  Rows of one group never depend on each other, so lanes of a
// warp wait only on other blocks.
// What bounds it: a chunk is smaller than a grid plane, so nearly every row
// needs a value the neighbouring chunk produced one level earlier; the chunks
// settle into a lockstep of one store-to-load trip per level (1.9 us at
// 128^3: 0.72 ms per triangle, against 1.38 ms for the level-by-level sweep).
// Each position loads all of its dependency slots whatever its count, so that
// no load waits for the count.  Loading a thread's first position of the next
// group during the current one (869 against 731 us) or chunks of twice the
// rows on half the SMs (836 against 801 us) did not help.
// ---------------------------------------------------------------------------
constexpr int CTS = 512;                       // threads per block of the chunked sweeps
constexpr unsigned long long SENTINEL = 0xFFFFFFFFFFFFFFFFull;

__device__ __forceinline__ unsigned long long ld_relaxed(const double* p) {
  unsigned long long v;
  asm volatile("ld.relaxed.gpu.global.b64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ void st_relaxed(double* p, double x) {
  asm volatile("st.relaxed.gpu.global.b64 [%0], %1;" ::"l"(p), "l"(__double_as_longlong(x)) : "memory");
}

// poll p until it no longer holds the sentinel (canonical NaN after a timeout)
__device__ __noinline__ unsigned long long wait_value(const double* p, int* flag, long long spin_limit) {
  for (long long it = 1;; ++it) {
    if ((it & 255) == 0 && (*(const volatile int*)flag & FLAG_SYNC_TIMEOUT)) return 0x7FFFFFFFFFFFFFFFull;
    if (it > spin_limit) {
      atomicOr(flag, FLAG_SYNC_TIMEOUT);
      return 0x7FFFFFFFFFFFFFFFull;
    }
    const unsigned long long v = ld_relaxed(p);
    if (v != SENTINEL) return v;
  }
}

constexpr int GMAX = 1024;   // rows of one group kept in shared memory for the next group

struct ChunkArgs {
  int npos;              // positions (= rows); column stride of pcol / pval
  const int* gofs;       // chunk b's groups (its rows' levels, in order): [gofs[b], gofs[b+1])
  const int* gptr;       // positions of group q: [gptr[q], gptr[q+1])
  const int* prow;
  const int* pcnt;
  const int* pcol;       // dependency: -1 - (its position in the previous group of the same chunk),
                         // when it is there and within the first GMAX positions; else its row
  const double* pval;
  const double* pdiag;   // upper solve: u_ii by position; NULL: unit diagonal
  const double* in;
  double* out;           // filled with SENTINEL before the launch; distinct from in
  int* flag;
  long long spin_limit;
};

// The static data of one position and its right-hand side.  All W dependency
// slots are loaded (the packed arrays hold W entries per position), so that
// no load waits for the count: one memory round trip fewer per level.
template <int W>
struct ChunkRow {
  int row, cnt;
  int d[W];
  double val[W];
  double rhs, dia;
};

template <int W>
__device__ __forceinline__ void chunk_load(const ChunkArgs& a, int idx, ChunkRow<W>& r) {
  r.row = __ldg(a.prow + idx);
  r.cnt = __ldg(a.pcnt + idx);
#pragma unroll
  for (int j = 0; j < W; ++j) {
    r.d[j] = __ldg(a.pcol + (int64_t)j * a.npos + idx);
    r.val[j] = __ldg(a.pval + (int64_t)j * a.npos + idx);
  }
  r.dia = a.pdiag ? __ldg(a.pdiag + idx) : 1.0;
  r.rhs = __ldg(a.in + r.row);
}

// x_row = (rhs - sum_j val_j x_dep_j) / dia: dependencies of the previous
// group of the chunk from shared memory, all others polled in one round trip
template <int W>
__device__ __forceinline__ double chunk_solve(const ChunkArgs& a, const ChunkRow<W>& r, const double* prev) {
  unsigned long long x[W];
#pragma unroll
  for (int j = 0; j < W; ++j) x[j] = (j < r.cnt && r.d[j] >= 0) ? ld_relaxed(a.out + r.d[j]) : 0ull;
#pragma unroll
  for (int j = 0; j < W; ++j)
    if (j < r.cnt && r.d[j] >= 0 && x[j] == SENTINEL) x[j] = wait_value(a.out + r.d[j], a.flag, a.spin_limit);
  double sum = r.rhs;
#pragma unroll
  for (int j = 0; j < W; ++j) {
    if (j < r.cnt) {
      const double xv = r.d[j] < 0 ? prev[-1 - r.d[j]] : __longlong_as_double((long long)x[j]);
      sum = fma(-r.val[j], xv, sum);
    }
  }
  if (a.pdiag) sum = sum / r.dia;
  if ((unsigned long long)__double_as_longlong(sum) == SENTINEL) sum = __longlong_as_double(0x7FFFFFFFFFFFFFFFLL);
  return sum;
}

// L1 prefetch of the static data of position idx (a hint: nothing is computed
// from it; every address lies inside the packed arrays)
template <int W>
__device__ __forceinline__ void chunk_prefetch(const ChunkArgs& a, int idx) {
  asm volatile("prefetch.global.L1 [%0];" ::"l"(a.prow + idx));
  asm volatile("prefetch.global.L1 [%0];" ::"l"(a.pcnt + idx));
#pragma unroll
  for (int j = 0; j < W; ++j) {
    asm volatile("prefetch.global.L1 [%0];" ::"l"(a.pcol + (int64_t)j * a.npos + idx));
    asm volatile("prefetch.global.L1 [%0];" ::"l"(a.pval + (int64_t)j * a.npos + idx));
  }
  if (a.pdiag) asm volatile("prefetch.global.L1 [%0];" ::"l"(a.pdiag + idx));
}

template <int W>
__global__ void __launch_bounds__(CTS, 1) ilu_sweep_chunk_kernel(ChunkArgs a) {
  __shared__ double sv[2 * GMAX];   // the values of the previous and of the current group
  const int q0 = a.gofs[blockIdx.x], q1 = a.gofs[blockIdx.x + 1];
  for (int q = q0; q < q1; ++q) {
    const int beg = __ldg(a.gptr + q), end = __ldg(a.gptr + q + 1);
    // the next group's static data on its way to L1 while this group waits
    // on its dependencies
    if (q + 1 < q1) {
      const int nend = __ldg(a.gptr + q + 2);
      for (int idx = end + threadIdx.x; idx < nend; idx += CTS) chunk_prefetch<W>(a, idx);
    }
    const double* prev = sv + ((q - 1) & 1) * GMAX;
    double* cur = sv + (q & 1) * GMAX;
    for (int idx = beg + threadIdx.x; idx < end; idx += CTS) {
      ChunkRow<W> r;
      chunk_load(a, idx, r);
      const double v = chunk_solve<W>(a, r, prev);
      if (idx - beg < GMAX) cur[idx - beg] = v;
      st_relaxed(a.out + r.row, v);
    }
    __syncthreads();
  }
}

// the lowest and highest level of the rows of each chunk
__global__ void ilu_chunk_range_kernel(int n, int CH, const int* lev, int* lo, int* hi) {
  const int stride = gridDim.x * blockDim.x;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
    atomicMin(lo + i / CH, lev[i]);
    atomicMax(hi + i / CH, lev[i]);
  }
}

__global__ void ilu_chunk_count_kernel(int P, const int* lo, const int* hi, int* gcount) {
  const int stride = gridDim.x * blockDim.x;
  for (int b = blockIdx.x * blockDim.x + threadIdx.x; b < P; b += stride) gcount[b] = hi[b] - lo[b] + 1;
}

// key of a row: its group, gofs[chunk] + (level - lowest level of the chunk)
__global__ void ilu_chunk_key_kernel(int n, int CH, const int* lev, const int* lo, const int* gofs, int* key) {
  const int stride = gridDim.x * blockDim.x;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) key[i] = gofs[i / CH] + lev[i] - lo[i / CH];
}

// position of each row in the chunked order
__global__ void ilu_chunk_posof_kernel(int n, const int* prow, int* posof) {
  const int stride = gridDim.x * blockDim.x;
  for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < n; idx += stride) posof[prow[idx]] = idx;
}

// the packed dependencies of the positions of the chunked order: a dependency
// in the previous group of the same chunk (within its first GMAX positions)
// as -1 - its position there, any other as its row
__global__ void ilu_chunk_pack_kernel(int n, int CH, int upper, const int* prow, const int* key, const int* posof,
                                      const int* gptr, const int* rp, const int* col, const int* dg,
                                      const double* lu, int* pcnt, int* pcol, double* pval, double* pdiag) {
  const int stride = gridDim.x * blockDim.x;
  for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < n; idx += stride) {
    const int i = prow[idx];
    const int ki = key[i];
    const int b = upper ? dg[i] + 1 : rp[i], e = upper ? rp[i + 1] : dg[i];
    pcnt[idx] = e - b;
    for (int p = b; p < e; ++p) {
      const int j = col[p];
      int enc = j;
      if (j / CH == i / CH && key[j] == ki - 1) {
        const int s = posof[j] - gptr[ki - 1];
        if (s < GMAX) enc = -1 - s;
      }
      pcol[(int64_t)(p - b) * n + idx] = enc;
      pval[(int64_t)(p - b) * n + idx] = lu[p];
    }
    if (upper) pdiag[idx] = lu[dg[i]];
  }
}

// y = U x (the upper factor including its diagonal)
__global__ void ilu_upper_mul_kernel(int n, const int* rp, const int* col, const int* dg, const double* lu,
                                     const double* x, double* y) {
  const int stride = gridDim.x * blockDim.x;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
    double sum = 0.0;
    for (int p = dg[i]; p < rp[i + 1]; ++p) sum = fma(lu[p], x[col[p]], sum);
    y[i] = sum;
  }
}

// diagonal positions; flag: FLAG_NO_DIAG if a row has none, FLAG_UNSORTED if
// the columns of a row are not strictly increasing
__global__ void ilu_diag_kernel(int n, const int* rp, const int* col, int* dg, int* flag) {
  const int stride = gridDim.x * blockDim.x;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
    int d = -1;
    for (int p = rp[i]; p < rp[i + 1]; ++p) {
      if (p > rp[i] && col[p] <= col[p - 1]) atomicOr(flag, FLAG_UNSORTED);
      if (col[p] == i) d = p;
    }
    if (d < 0) {
      atomicOr(flag, FLAG_NO_DIAG);
      d = rp[i];
    }
    dg[i] = d;
  }
}

// one relaxation sweep of lev(i) = max(0, 1 + max lev(j)) over the strict
// lower (upper == 0) or strict upper dependencies of row i
__global__ void ilu_level_relax_kernel(int n, const int* rp, const int* col, const int* dg, int* lev, int upper,
                                       int* changed) {
  const int stride = gridDim.x * blockDim.x;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
    const int b = upper ? dg[i] + 1 : rp[i], e = upper ? rp[i + 1] : dg[i];
    int m = 0;
    for (int p = b; p < e; ++p) m = max(m, __ldcg(lev + col[p]) + 1);
    if (m != __ldcg(lev + i)) {
      __stcg(lev + i, m);
      *(volatile int*)changed = 1;
    }
  }
}

__global__ void ilu_level_max_kernel(int n, const int* lev, int* out) {
  const int stride = gridDim.x * blockDim.x;
  int m = 0;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) m = max(m, lev[i]);
  atomicMax(out, m);
}

__global__ void ilu_level_hist_kernel(int n, const int* lev, int* cnt) {
  const int stride = gridDim.x * blockDim.x;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) atomicAdd(cnt + lev[i], 1);
}

// exclusive scan of cnt[0..m) into ptr[0..m] and the largest count, one block
__global__ void ilu_level_scan_kernel(int m, const int* cnt, int* ptr, int* maxw) {
  __shared__ int sh[1024];
  __shared__ int carry_s;
  int mw = 0;
  if (threadIdx.x == 0) carry_s = 0;
  __syncthreads();
  for (int base = 0; base < m; base += 1024) {
    const int i = base + threadIdx.x;
    const int v = i < m ? cnt[i] : 0;
    mw = max(mw, v);
    sh[threadIdx.x] = v;
    __syncthreads();
    for (int off = 1; off < 1024; off <<= 1) {
      const int add = threadIdx.x >= off ? sh[threadIdx.x - off] : 0;
      __syncthreads();
      sh[threadIdx.x] += add;
      __syncthreads();
    }
    const int carry = carry_s;
    if (i < m) ptr[i] = carry + sh[threadIdx.x] - v;
    __syncthreads();
    if (threadIdx.x == 1023) carry_s = carry + sh[1023];
    __syncthreads();
  }
  if (threadIdx.x == 0) ptr[m] = carry_s;
  atomicMax(maxw, mw);
}

__global__ void ilu_level_scatter_kernel(int n, const int* lev, int* cursor, int* rows) {
  const int stride = gridDim.x * blockDim.x;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) rows[atomicAdd(cursor + lev[i], 1)] = i;
}

static int stream_grid(const Ctx& c, int64_t n) {
  int64_t g = (n + NT - 1) / NT;
  if (g > (int64_t)c.sms * 8) g = (int64_t)c.sms * 8;
  if (g > MAXBLK) g = MAXBLK;
  return (int)(g < 1 ? 1 : g);
}

template <int MODE>
static cudaError_t launch_sweep(const Ctx& c, const IluDesc& F, int u, const double* in, double* out) {
  cudaError_t e = cudaMemsetAsync(&F.bar->count, 0, sizeof(unsigned int), c.stream);
  if (e != cudaSuccess) return e;
  SweepArgs a{F.nlev[u], F.lptr[u], F.lrows[u], F.row_ptr, F.col, F.diag, F.lu, in, out, &F.bar->count, F.flag,
              F.spin_limit};
  void* args[] = {&a};
  return cudaLaunchCooperativeKernel((const void*)ilu_sweep_kernel<MODE>, dim3(F.grid[u]), dim3(ITS), args, 0,
                                     c.stream);
}

// A triangular solve: the packed sweep when every row has at most 8
// dependencies, else the CSR sweep.  in == out is allowed.
static cudaError_t solve_sweep(const Ctx& c, const IluDesc& F, int u, const double* in, double* out) {
  if (F.W[u] == 0)
    return u == 0 ? launch_sweep<SW_LOWER>(c, F, 0, in, out) : launch_sweep<SW_UPPER>(c, F, 1, in, out);
  cudaError_t e = cudaSuccess;
  if (F.CH[u] > 0) {
    if (in == out) {
      e = cudaMemcpyAsync(F.scratch, in, sizeof(double) * F.n, cudaMemcpyDeviceToDevice, c.stream);
      if (e != cudaSuccess) return e;
      in = F.scratch;
    }
    e = cudaMemsetAsync(out, 0xFF, sizeof(double) * F.n, c.stream);
    if (e != cudaSuccess) return e;
    ChunkArgs ca{F.n, F.gofs[u], F.gptr[u], F.cprow[u], F.cpcnt[u], F.cpcol[u], F.cpval[u],
                 u == 1 ? F.cpdiag : nullptr, in, out, F.flag, F.spin_limit};
    void* cargs[] = {&ca};
    const int P = (F.n + F.CH[u] - 1) / F.CH[u];
    const void* k = F.W[u] == 3   ? (const void*)ilu_sweep_chunk_kernel<3>
                    : F.W[u] == 4 ? (const void*)ilu_sweep_chunk_kernel<4>
                                  : (const void*)ilu_sweep_chunk_kernel<8>;
    return cudaLaunchCooperativeKernel(k, dim3(P), dim3(CTS), cargs, 0, c.stream);
  }
  e = cudaMemsetAsync(&F.bar->count, 0, sizeof(unsigned int), c.stream);
  if (e != cudaSuccess) return e;
  PackedArgs p{F.npad[u], F.prow[u], F.pcnt[u], F.pcol[u], F.pval[u], u == 1 ? F.pdiag[1] : nullptr, in, out,
               F.flag, F.spin_limit};
  LevelArgs L{p, F.nlev[u], F.pptr[u], &F.bar->count};
  void* largs[] = {&L};
  const void* k = F.W[u] == 3   ? (const void*)ilu_sweep_level_kernel<3>
                  : F.W[u] == 4 ? (const void*)ilu_sweep_level_kernel<4>
                                : (const void*)ilu_sweep_level_kernel<8>;
  return cudaLaunchCooperativeKernel(k, dim3(F.grid[u]), dim3(ITS), largs, 0, c.stream);
}

cudaError_t ilu_lower_solve(const Ctx& c, const IluDesc& F, const double* z, double* y) {
  return solve_sweep(c, F, 0, z, y);
}

cudaError_t ilu_upper_solve(const Ctx& c, const IluDesc& F, const double* v, double* t) {
  return solve_sweep(c, F, 1, v, t);
}

cudaError_t ilu_upper_mul(const Ctx& c, const IluDesc& F, const double* x, double* y) {
  ilu_upper_mul_kernel<<<stream_grid(c, F.n), NT, 0, c.stream>>>(F.n, F.row_ptr, F.col, F.diag, F.lu, x, y);
  return cudaGetLastError();
}

// Host side of the set-up: diagonal positions, both level schedules, the factor.
IluSetupResult ilu_setup(const Ctx& c, IluDesc& F, DevAllocFn alloc, void* actx, int* h_scratch) {
  IluSetupResult R{};
  auto fail_cuda = [&](cudaError_t e, const char* where) {
    R.code = 1;
    R.cuda = e;
    R.where = where;
    return R;
  };
#define ICK(expr)                                  \
  do {                                             \
    cudaError_t e_ = (expr);                       \
    if (e_ != cudaSuccess) return fail_cuda(e_, #expr); \
  } while (0)
  const int n = F.n;
  const int g = stream_grid(c, n);
  auto read_int = [&](const int* d, int* v) -> cudaError_t {
    cudaError_t e = cudaMemcpyAsync(h_scratch, d, sizeof(int), cudaMemcpyDeviceToHost, c.stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c.stream);
    *v = *h_scratch;
    return e;
  };
  int* scratch = (int*)alloc(actx, 4 * sizeof(int));
  F.diag = (int*)alloc(actx, sizeof(int) * (size_t)n);
  if (!scratch || !F.diag) {
    R.code = 4;
    return R;
  }
  ICK(cudaMemsetAsync(scratch, 0, 4 * sizeof(int), c.stream));
  ilu_diag_kernel<<<g, NT, 0, c.stream>>>(n, F.row_ptr, F.col, F.diag, scratch);
  ICK(cudaGetLastError());
  int f = 0;
  ICK(read_int(scratch, &f));
  if (f) {
    R.code = 2;
    R.where = (f & FLAG_NO_DIAG) ? "a row of A has no diagonal entry (ILU(0) needs every a_ii in the pattern)"
                                 : "the columns of a row of A are not strictly increasing (ILU(0) needs sorted rows)";
    return R;
  }
  int nb = 0;
  ICK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, ilu_sweep_kernel<SW_FACTOR>, ITS, 0));
  int nb2 = 0, nb3 = 0;
  ICK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb2, ilu_sweep_kernel<SW_LOWER>, ITS, 0));
  ICK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb3, ilu_sweep_kernel<SW_UPPER>, ITS, 0));
  nb = std::min(nb, std::min(nb2, nb3));
  {
    int l3 = 0, l4 = 0, l8 = 0;
    ICK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&l3, ilu_sweep_level_kernel<3>, ITS, 0));
    ICK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&l4, ilu_sweep_level_kernel<4>, ITS, 0));
    ICK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&l8, ilu_sweep_level_kernel<8>, ITS, 0));
    nb = std::min(nb, std::min(l3, std::min(l4, l8)));
  }
  if (nb < 1) nb = 1;
  const int co = nb * c.sms;
  for (int u = 0; u < 2; ++u) {
    F.lev[u] = (int*)alloc(actx, sizeof(int) * (size_t)n);
    if (!F.lev[u]) {
      R.code = 4;
      return R;
    }
    ICK(cudaMemsetAsync(F.lev[u], 0, sizeof(int) * (size_t)n, c.stream));
    // sweeps in batches of 8 until a whole batch changes nothing; the levels
    // only grow towards the fixed point, which n + 8 sweeps always reach
    int changed = 1;
    int64_t sweeps = 0;
    while (changed) {
      if (sweeps > (int64_t)n + 8) {
        R.code = 1;
        R.cuda = cudaErrorUnknown;
        R.where = "level relaxation did not settle";
        return R;
      }
      ICK(cudaMemsetAsync(scratch + 1, 0, sizeof(int), c.stream));
      for (int k = 0; k < 8; ++k)
        ilu_level_relax_kernel<<<g, NT, 0, c.stream>>>(n, F.row_ptr, F.col, F.diag, F.lev[u], u, scratch + 1);
      ICK(cudaGetLastError());
      sweeps += 8;
      ICK(read_int(scratch + 1, &changed));
    }
    ICK(cudaMemsetAsync(scratch + 2, 0, 2 * sizeof(int), c.stream));
    ilu_level_max_kernel<<<g, NT, 0, c.stream>>>(n, F.lev[u], scratch + 2);
    ICK(cudaGetLastError());
    int mx = 0;
    ICK(read_int(scratch + 2, &mx));
    const int nlev = mx + 1;
    F.nlev[u] = nlev;
    int* cnt = (int*)alloc(actx, sizeof(int) * (size_t)(nlev + 1));
    F.lptr[u] = (int*)alloc(actx, sizeof(int) * (size_t)(nlev + 1));
    F.lrows[u] = (int*)alloc(actx, sizeof(int) * (size_t)n);
    if (!cnt || !F.lptr[u] || !F.lrows[u]) {
      R.code = 4;
      return R;
    }
    ICK(cudaMemsetAsync(cnt, 0, sizeof(int) * (size_t)(nlev + 1), c.stream));
    ilu_level_hist_kernel<<<g, NT, 0, c.stream>>>(n, F.lev[u], cnt);
    ilu_level_scan_kernel<<<1, 1024, 0, c.stream>>>(nlev, cnt, F.lptr[u], scratch + 3);
    ICK(cudaMemcpyAsync(cnt, F.lptr[u], sizeof(int) * (size_t)nlev, cudaMemcpyDeviceToDevice, c.stream));
    ilu_level_scatter_kernel<<<g, NT, 0, c.stream>>>(n, F.lev[u], cnt, F.lrows[u]);
    ICK(cudaGetLastError());
    int mw = 0;
    ICK(read_int(scratch + 3, &mw));
    F.max_width[u] = mw;
    const int want = (mw + ITS - 1) / ITS;
    F.grid[u] = std::max(1, std::min(co, want));
  }
  ICK(launch_sweep<SW_FACTOR>(c, F, 0, nullptr, nullptr));
  int flag = 0;
  ICK(read_int(F.flag, &flag));
  if (flag & FLAG_SYNC_TIMEOUT) {
    R.code = 1;
    R.cuda = cudaErrorLaunchTimeout;
    R.where = "a grid barrier of the ILU(0) factor sweep timed out";
    return R;
  }
  if (flag & FLAG_ZERO_PIVOT) {
    R.code = 3;
    R.where = "ILU(0) met a zero pivot u_ii (the incomplete factor does not exist in this ordering)";
    return R;
  }
  // packed level-ordered dependencies for the solves (rows with at most 8),
  // each level padded to whole warps
  for (int u = 0; u < 2; ++u) {
    ICK(cudaMemsetAsync(scratch, 0, sizeof(int), c.stream));
    ilu_pack_kernel<<<g, NT, 0, c.stream>>>(n, 0, u, 0, F.lrows[u], F.lev[u], F.lptr[u], nullptr, F.row_ptr,
                                            F.col, F.diag, F.lu, nullptr, nullptr, nullptr, nullptr, nullptr,
                                            scratch);
    ICK(cudaGetLastError());
    int md = 0;
    ICK(read_int(scratch, &md));
    // the packed width: the smallest of 3, 4, 8 that holds every row (a 7-point
    // stencil in natural order has 3 dependencies per triangle: no unused slot)
    const int W = md <= 3 ? 3 : (md <= 4 ? 4 : (md <= 8 ? 8 : 0));
    F.W[u] = 0;
    if (W == 0) continue;
    const int nlev = F.nlev[u];
    int* pcnt_l = (int*)alloc(actx, sizeof(int) * (size_t)(nlev + 1));
    int* pptr = (int*)alloc(actx, sizeof(int) * (size_t)(nlev + 1));
    F.pptr[u] = pptr;
    if (!pcnt_l || !pptr) {
      R.code = 4;
      return R;
    }
    ilu_pad_counts_kernel<<<stream_grid(c, nlev), NT, 0, c.stream>>>(nlev, F.lptr[u], pcnt_l);
    ilu_level_scan_kernel<<<1, 1024, 0, c.stream>>>(nlev, pcnt_l, pptr, scratch + 1);
    ICK(cudaGetLastError());
    int npad = 0;
    ICK(read_int(pptr + nlev, &npad));
    F.npad[u] = npad;
    F.prow[u] = (int*)alloc(actx, sizeof(int) * (size_t)npad);
    F.pcnt[u] = (int*)alloc(actx, sizeof(int) * (size_t)npad);
    F.pcol[u] = (int*)alloc(actx, sizeof(int) * (size_t)npad * W);
    F.pval[u] = (double*)alloc(actx, sizeof(double) * (size_t)npad * W);
    F.pdiag[u] = (double*)alloc(actx, sizeof(double) * (size_t)npad);
    if (!F.prow[u] || !F.pcnt[u] || !F.pcol[u] || !F.pval[u] || !F.pdiag[u]) {
      R.code = 4;
      return R;
    }
    ICK(cudaMemsetAsync(F.prow[u], 0xFF, sizeof(int) * (size_t)npad, c.stream));   // -1: padding
    ICK(cudaMemsetAsync(F.pcnt[u], 0, sizeof(int) * (size_t)npad, c.stream));
    ICK(cudaMemsetAsync(F.pdiag[u], 0, sizeof(double) * (size_t)npad, c.stream));
    ilu_pack_kernel<<<g, NT, 0, c.stream>>>(n, npad, u, W, F.lrows[u], F.lev[u], F.lptr[u], pptr, F.row_ptr,
                                            F.col, F.diag, F.lu, F.prow[u], F.pcnt[u], F.pcol[u], F.pval[u],
                                            u == 1 ? F.pdiag[u] : nullptr, nullptr);
    ICK(cudaGetLastError());
    F.W[u] = W;
  }
  // chunked order for the pipelined solves: contiguous row chunks, one block
  // each, all resident at once
  {
    const int CH = std::max(1, (n + c.sms - 1) / c.sms);
    const int P = (n + CH - 1) / CH;
    bool ok = F.W[0] > 0 || F.W[1] > 0;
    for (int W : {3, 4, 8}) {
      if (!ok) break;
      int nbk = 0;
      if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(
              &nbk, W == 3 ? ilu_sweep_chunk_kernel<3> : (W == 4 ? ilu_sweep_chunk_kernel<4> : ilu_sweep_chunk_kernel<8>),
              CTS, 0) != cudaSuccess) {
        cudaGetLastError();
        ok = false;
        break;
      }
      if ((int64_t)nbk * c.sms < P) ok = false;   // one wave: every chunk's block resident
    }
    if (ok) {
      F.scratch = (double*)alloc(actx, sizeof(double) * (size_t)n);
      if (!F.scratch) {
        R.code = 4;
        return R;
      }
    }
    for (int u = 0; ok && u < 2; ++u) {
      F.CH[u] = 0;
      if (F.W[u] == 0) continue;
      int* lo = (int*)alloc(actx, sizeof(int) * (size_t)P);
      int* hi = (int*)alloc(actx, sizeof(int) * (size_t)P);
      int* gcount = (int*)alloc(actx, sizeof(int) * (size_t)(P + 1));
      F.gofs[u] = (int*)alloc(actx, sizeof(int) * (size_t)(P + 1));
      int* key = (int*)alloc(actx, sizeof(int) * (size_t)n);
      int* posof = (int*)alloc(actx, sizeof(int) * (size_t)n);
      if (!lo || !hi || !gcount || !F.gofs[u] || !key || !posof) {
        R.code = 4;
        return R;
      }
      ICK(cudaMemsetAsync(lo, 0x7F, sizeof(int) * (size_t)P, c.stream));   // large positive
      ICK(cudaMemsetAsync(hi, 0, sizeof(int) * (size_t)P, c.stream));
      ilu_chunk_range_kernel<<<g, NT, 0, c.stream>>>(n, CH, F.lev[u], lo, hi);
      ilu_chunk_count_kernel<<<stream_grid(c, P), NT, 0, c.stream>>>(P, lo, hi, gcount);
      ilu_level_scan_kernel<<<1, 1024, 0, c.stream>>>(P, gcount, F.gofs[u], scratch + 2);
      ICK(cudaGetLastError());
      int TG = 0;
      ICK(read_int(F.gofs[u] + P, &TG));
      int* cnt = (int*)alloc(actx, sizeof(int) * (size_t)(TG + 1));
      F.gptr[u] = (int*)alloc(actx, sizeof(int) * (size_t)(TG + 1));
      F.cprow[u] = (int*)alloc(actx, sizeof(int) * (size_t)n);
      F.cpcnt[u] = (int*)alloc(actx, sizeof(int) * (size_t)n);
      F.cpcol[u] = (int*)alloc(actx, sizeof(int) * (size_t)n * F.W[u]);
      F.cpval[u] = (double*)alloc(actx, sizeof(double) * (size_t)n * F.W[u]);
      if (u == 1) F.cpdiag = (double*)alloc(actx, sizeof(double) * (size_t)n);
      if (!cnt || !F.gptr[u] || !F.cprow[u] || !F.cpcnt[u] || !F.cpcol[u] || !F.cpval[u] || (u == 1 && !F.cpdiag)) {
        R.code = 4;
        return R;
      }
      ilu_chunk_key_kernel<<<g, NT, 0, c.stream>>>(n, CH, F.lev[u], lo, F.gofs[u], key);
      ICK(cudaMemsetAsync(cnt, 0, sizeof(int) * (size_t)(TG + 1), c.stream));
      ilu_level_hist_kernel<<<g, NT, 0, c.stream>>>(n, key, cnt);
      ilu_level_scan_kernel<<<1, 1024, 0, c.stream>>>(TG, cnt, F.gptr[u], scratch + 2);
      ICK(cudaMemcpyAsync(cnt, F.gptr[u], sizeof(int) * (size_t)TG, cudaMemcpyDeviceToDevice, c.stream));
      ilu_level_scatter_kernel<<<g, NT, 0, c.stream>>>(n, key, cnt, F.cprow[u]);
      ilu_chunk_posof_kernel<<<g, NT, 0, c.stream>>>(n, F.cprow[u], posof);
      ilu_chunk_pack_kernel<<<g, NT, 0, c.stream>>>(n, CH, u, F.cprow[u], key, posof, F.gptr[u], F.row_ptr, F.col,
                                                    F.diag, F.lu, F.cpcnt[u], F.cpcol[u], F.cpval[u], F.cpdiag);
      ICK(cudaGetLastError());
      F.CH[u] = CH;
      F.groups[u] = TG;
    }
  }
  ICK(cudaStreamSynchronize(c.stream));
#undef ICK
  return R;
}

}  // namespace msk

// Sparse matrix-vector products of libmsstab: the MV steps of Algorithm 1
// (r^(k+1) = A r^(k), v_q^(k+1) = A v_q^(k)), the residual b - A x, and the
// fused form that also returns the s projections P^T (A w) the next small
// solve of Algorithm 1 needs, so that A w and P^T A w come from one pass.
//
// Formats.  SELL-32-sigma: rows in slices of 32 (one warp per slice, one row
// per lane), entries stored column-major within the slice so that every load of
// the warp is one contiguous 128/256-byte segment; padding entries are zero
// coefficients on the row's own index (they add an exact 0 for finite x, so the
// sum equals the CSR sum bit for bit), and the row loop runs exactly the slice
// width (chunks of 8 plus an exact tail: no predicated multiply-adds).
// CSR: one thread per row (the baseline format).
// All loads of matrix data are single-use and go through the read-only path.

#include <mutex>
#include <type_traits>

#include "launch.h"
#include "msstab.h"

namespace msk {

// Products run one 1024-thread block per SM (32 warps, as many as four blocks
// of 256 would give): the grid reduction that follows every fused product then
// combines 152 partials instead of 608, on the critical path of the next small
// solve.
constexpr int SNT = 1024;
constexpr int SNWARP = SNT / 32;

template <typename T>
__device__ __forceinline__ T ro(const T* p) { return __ldg(p); }

__device__ __forceinline__ double fma_t(double a, double b, double c) { return fma(a, b, c); }
__device__ __forceinline__ float fma_t(float a, float b, float c) { return fmaf(a, b, c); }

template <typename T>
struct SpmvArgs {
  const T* x;
  T* y;
  const T* b;
  const T* P;
  int64_t ldp;
  int np, self, bdot;
  double* out;
  Epi epi;
  RedScratch rs;
  const T* Pil;   // P interleaved by row (Pil[row * sp + c]), rows 16-byte aligned; or NULL
  int sp;
  const T* Pb;    // block-partitioned P: Pb[row] = P[pblock_col(row)][row]; or NULL
};

// Smallest power of two >= v (v <= 32).
__host__ __device__ constexpr int pow2_at_least(int v) { return v <= 1 ? 1 : (v <= 2 ? 2 : (v <= 4 ? 4 : (v <= 8 ? 8 : (v <= 16 ? 16 : 32)))); }

// Per-thread accumulators of the fused dot products: NP slots for P^T y (np <=
// NP used), then y.y and b.b in fixed slots.  FP64 vectors accumulate in FP64;
// FP32 vectors in FP32, widened exactly to FP64 for the block reduction.
template <typename T, int NP>
struct DotAcc;

template <int NP>
struct DotAcc<double, NP> {
  double v[NP + 2];
  __device__ __forceinline__ void zero() {
#pragma unroll
    for (int i = 0; i < NP + 2; ++i) v[i] = 0.0;
  }
  __device__ __forceinline__ void add(int i, double x, double y) { v[i] = fma(x, y, v[i]); }
  __device__ __forceinline__ double get(int i) const { return v[i]; }
};

template <int NP>
struct DotAcc<float, NP> {
  float v[NP + 2];
  __device__ __forceinline__ void zero() {
#pragma unroll
    for (int i = 0; i < NP + 2; ++i) v[i] = 0.f;
  }
  __device__ __forceinline__ void add(int i, float x, float y) { v[i] = fmaf(x, y, v[i]); }
  __device__ __forceinline__ double get(int i) const { return widen_f32(v[i]); }
};

// The row's NP entries of the interleaved P (zero beyond np), with 16-byte loads.
template <typename T, int NP>
__device__ __forceinline__ void load_prow(const SpmvArgs<T>& a, int row, T (&pr)[NP]) {
  static_assert(NP % (16 / sizeof(T)) == 0, "NP must fill 16-byte vectors");
  constexpr int VW = 16 / sizeof(T);
  using V = std::conditional_t<sizeof(T) == 8, double2, float4>;
  const V* src = reinterpret_cast<const V*>(a.Pil + (int64_t)row * a.sp);
#pragma unroll
  for (int v = 0; v < NP / VW; ++v) {
    if (v * VW < a.sp) {
      const V q = __ldg(src + v);
      const T* e = reinterpret_cast<const T*>(&q);
#pragma unroll
      for (int u = 0; u < VW; ++u) pr[v * VW + u] = e[u];
    } else {
#pragma unroll
      for (int u = 0; u < VW; ++u) pr[v * VW + u] = T(0);
    }
  }
}

template <typename T, int NP>
__device__ __forceinline__ void acc_row_pre(const SpmvArgs<T>& a, int row, T yv, const T (&pr)[NP],
                                            DotAcc<T, NP>& acc) {
#pragma unroll
  for (int c = 0; c < NP; ++c)
    if (c < a.np) acc.add(c, yv, pr[c]);
  if (a.self) acc.add(NP, yv, yv);
  if (a.bdot) {
    const T bd = a.b[row];
    acc.add(NP + 1, bd, bd);
  }
}

template <typename T, int NP>
__device__ __forceinline__ void acc_row(const SpmvArgs<T>& a, int row, T yv, DotAcc<T, NP>& acc) {
  // NP is the compile-time slot count chosen for np (np == NP in the cycle)
  if (a.Pb) {
    add_to_slot<NP>(acc, pblock_col(row, a.np), yv, ro(a.Pb + row));
  } else {
#pragma unroll
    for (int c = 0; c < NP; ++c)
      if (c < a.np) acc.add(c, yv, ro(a.P + (int64_t)c * a.ldp + row));
  }
  if (a.self) acc.add(NP, yv, yv);
  if (a.bdot) {
    const T bd = a.b[row];
    acc.add(NP + 1, bd, bd);
  }
}

// The block's sums of the fused dots into red[0..m): (P^T y [np], y.y?,
// b.b?) compacted into the first m slots; FP64 partials through block_reduce,
// FP32 ones through block_reduce_f32 (FP32 warp stage).  The s dots of a
// cycle's products fill 8 of the 16 slots: only those are reduced.
template <typename T, int NP>
__device__ __forceinline__ void block_reduce_acc(const SpmvArgs<T>& a, const DotAcc<T, NP>& acc, int m,
                                                 double* smem_w, double* red) {
  constexpr int M = pow2_at_least(NP + 2);
  using V = std::conditional_t<sizeof(T) == 4, float, double>;
  V fin[M];
#pragma unroll
  for (int i = 0; i < M; ++i) {
    V v = V(0);
    if (i < NP && i < a.np) v = acc.v[i < NP ? i : 0];
    if (a.self && i == a.np) v = acc.v[NP];
    if (a.bdot && i == a.np + a.self) v = acc.v[NP + 1];
    fin[i] = v;
  }
  auto reduce = [&](auto& f, auto mtag) {
    constexpr int MM = decltype(mtag)::value;
    if constexpr (sizeof(T) == 4)
      block_reduce_f32<MM>(f, m, smem_w, red);
    else
      block_reduce<MM>(f, m, smem_w, red);
  };
  if constexpr (M > 8) {
    if (m <= 8)
      reduce(reinterpret_cast<V(&)[8]>(fin), std::integral_constant<int, 8>{});
    else
      reduce(fin, std::integral_constant<int, M>{});
  } else {
    reduce(fin, std::integral_constant<int, M>{});
  }
}

template <typename T, int NP>
__device__ __forceinline__ void finish(const SpmvArgs<T>& a, const DotAcc<T, NP>& acc) {
  __shared__ double smem_w[SNWARP * MAXRED];
  __shared__ double red[MAXRED];
  __shared__ int s_last;
  __shared__ EpiScratch ew;
  const int m = a.np + a.self + a.bdot;
  block_reduce_acc<T, NP>(a, acc, m, smem_w, red);
  if (grid_reduce(a.rs, 0, blockIdx.x, gridDim.x, m, red, &s_last)) {
    if (threadIdx.x < m) a.out[threadIdx.x] = red[threadIdx.x];
    __threadfence();
    __syncthreads();
    if (threadIdx.x < 32) run_epilogue(a.epi, ew);
  }
}

// Loads of the vector x of a product: through the read-only path when x is
// not written during the launch (XL = 0); through L1 and L2 (ld.global.ca)
// when another block of the same persistent launch wrote it (XL = 1).  The
// latter is safe because in that launch every vector is written at most once,
// before the grid barrier that precedes its product, and nothing loads it
// into L1 before that write (those loads go through L2 only, __ldcg): no L1
// line of it can be stale.
template <int XL, typename T>
__device__ __forceinline__ T xload(const T* p) {
  if constexpr (XL == 0)
    return __ldg(p);
  else
    return __ldca(p);
}

// K consecutive entries of a SELL row (stride 32), continuing the row's
// multiply-add chain in column order (as CSR does).
template <typename T, int K, int XL = 0>
__device__ __forceinline__ T sell_chunk(const int* __restrict__ col, const T* __restrict__ val,
                                        const T* __restrict__ x, int64_t base, T sum) {
  int c[K];
  T v[K];
#pragma unroll
  for (int u = 0; u < K; ++u) {
    c[u] = ro(col + base + (int64_t)u * 32);
    v[u] = ro(val + base + (int64_t)u * 32);
  }
#pragma unroll
  for (int u = 0; u < K; ++u) sum = fma_t(v[u], xload<XL>(x + c[u]), sum);
  return sum;
}

// One row of width w: chunks of 8, then an exact tail (no predicated slots).
template <typename T, int XL = 0>
__device__ __forceinline__ T sell_row(const int* __restrict__ col, const T* __restrict__ val,
                                      const T* __restrict__ x, int64_t base, int w) {
  T sum = T(0);
  int j = 0;
  for (; j + 8 <= w; j += 8) sum = sell_chunk<T, 8, XL>(col, val, x, base + (int64_t)j * 32, sum);
  const int64_t b = base + (int64_t)j * 32;
  switch (w - j) {
    case 1: return sell_chunk<T, 1, XL>(col, val, x, b, sum);
    case 2: return sell_chunk<T, 2, XL>(col, val, x, b, sum);
    case 3: return sell_chunk<T, 3, XL>(col, val, x, b, sum);
    case 4: return sell_chunk<T, 4, XL>(col, val, x, b, sum);
    case 5: return sell_chunk<T, 5, XL>(col, val, x, b, sum);
    case 6: return sell_chunk<T, 6, XL>(col, val, x, b, sum);
    case 7: return sell_chunk<T, 7, XL>(col, val, x, b, sum);
    default: return sum;
  }
}

// One pass of the SELL product y = A x (or b - A x) over the slices of this
// thread's warp (warp w of the grid takes slices w, w + nwarps, ...), with the
// row's contributions to the fused dots accumulated in acc (NP >= 0).  The
// standalone product and the persistent level kernel both run it, with the
// same grid, so that their sums are the same bit for bit.
template <typename T, int NP, int XL>
__device__ __forceinline__ void sell_pass(const SellMat<T>& A, const SpmvArgs<T>& a,
                                          DotAcc<T, (NP < 0 ? 0 : NP)>& acc, int nblocks) {
  constexpr int NA = NP < 0 ? 0 : NP;
  const int lane = threadIdx.x & 31;
  const int nwarps = nblocks * SNWARP;
  int sl = (blockIdx.x * SNT + threadIdx.x) >> 5;
  // the next slice's width and start are loaded one iteration ahead
  int w_next = 0, base_next = 0;
  if (sl < A.nslices) {
    w_next = ro(A.slice_w + sl);
    base_next = ro(A.slice_ptr + sl);
  }
  for (; sl < A.nslices; sl += nwarps) {
    const int w = w_next;
    const int64_t base = (int64_t)base_next + lane;
    if (sl + nwarps < A.nslices) {
      w_next = ro(A.slice_w + sl + nwarps);
      base_next = ro(A.slice_ptr + sl + nwarps);
    }
    const int pos = sl * 32 + lane;
    const int row = pos < A.n ? (A.perm ? ro(A.perm + pos) : pos) : 0;
    // FP32: the row's P entries (interleaved layout) are in flight with the
    // matrix loads (FP64: the 8 extra doubles would spill at 64 registers)
    constexpr bool PRE = NA > 0 && sizeof(T) == 4;
    T pr[PRE ? NA : 1];
    const bool pre = PRE && a.Pil != nullptr && a.Pb == nullptr && pos < A.n;
    if constexpr (PRE) {
      if (pre) load_prow<T, NA>(a, row, pr);
    }
    const T sum = sell_row<T, XL>(A.col, A.val, a.x, base, w);
    if (pos < A.n) {
      const T yv = a.b ? (T)(a.b[row] - sum) : sum;
      a.y[row] = yv;
      if constexpr (PRE) {
        if (pre)
          acc_row_pre<T, NA>(a, row, yv, pr, acc);
        else
          acc_row<T, NA>(a, row, yv, acc);
      } else if constexpr (NP >= 0) {
        acc_row<T, NA>(a, row, yv, acc);
      }
    }
  }
}

// NP < 0: plain product; NP >= 0: also the reduction of up to NP dots with P,
// y.y and b.b, and the epilogue.
template <typename T, int NP>
__global__ void __launch_bounds__(SNT, 1) spmv_sell_kernel(SellMat<T> A, SpmvArgs<T> a) {
  constexpr int NA = NP < 0 ? 0 : NP;
  DotAcc<T, NA> acc;
  acc.zero();
  sell_pass<T, NP, 0>(A, a, acc, gridDim.x);
  if constexpr (NP >= 0) finish<T, NA>(a, acc);
}

template <typename T, int NP>
__global__ void __launch_bounds__(SNT, 1) spmv_csr_kernel(CsrMat<T> A, SpmvArgs<T> a) {
  constexpr int NA = NP < 0 ? 0 : NP;
  DotAcc<T, NA> acc;
  acc.zero();
  const int stride = gridDim.x * SNT;
  for (int row = blockIdx.x * SNT + threadIdx.x; row < A.n; row += stride) {
    const int beg = ro(A.row_ptr + row), end = ro(A.row_ptr + row + 1);
    T sum = T(0);
    for (int p = beg; p < end; ++p) sum = fma_t(ro(A.val + p), ro(a.x + ro(A.col + p)), sum);
    const T yv = a.b ? (T)(a.b[row] - sum) : sum;
    a.y[row] = yv;
    if (NP >= 0) acc_row<T, NA>(a, row, yv, acc);
  }
  if constexpr (NP >= 0) finish<T, NA>(a, acc);
}

template <typename K>
static int max_grid(K kernel, const Ctx& c) {
  int nb = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, kernel, SNT, 0) != cudaSuccess || nb < 1) nb = 1;
  int g = nb * c.sms;
  return g > MAXBLK ? MAXBLK : g;
}

template <typename T>
static const T* pick_val(const MatDesc& A, bool sell);
template <>
const double* pick_val<double>(const MatDesc& A, bool sell) { return sell ? A.sval64 : A.val64; }
template <>
const float* pick_val<float>(const MatDesc& A, bool sell) { return sell ? A.sval32 : A.val32; }

template <typename T, int NP>
static void launch_sell(const Ctx& c, const SellMat<T>& M, const SpmvArgs<T>& a) {
  static int cap = max_grid(spmv_sell_kernel<T, NP>, c);
  const int64_t need = ((int64_t)M.nslices * 32 + SNT - 1) / SNT;
  spmv_sell_kernel<T, NP><<<(int)(need < cap ? need : cap), SNT, 0, c.stream>>>(M, a);
}

template <typename T, int NP>
static void launch_csr(const Ctx& c, const CsrMat<T>& M, const SpmvArgs<T>& a) {
  static int cap = max_grid(spmv_csr_kernel<T, NP>, c);
  const int64_t need = ((int64_t)M.n + SNT - 1) / SNT;
  spmv_csr_kernel<T, NP><<<(int)(need < cap ? need : cap), SNT, 0, c.stream>>>(M, a);
}

template <typename T>
cudaError_t spmv(const Ctx& c, const MatDesc& A, const T* x, T* y, const T* b, const T* P, int64_t ldp,
                 int np, int self, int bdot, double* out, Epi epi, const T* Pil, int sp, const T* Pb) {
  if (np < 0 || np > SMAX) return cudaErrorInvalidValue;
  // the block-partitioned form needs 32 consecutive rows per warp (no SELL sorting)
  const T* pb = (Pb && !(A.format == 0 && A.perm)) ? Pb : nullptr;
  SpmvArgs<T> a{x, y, b, P, ldp, np, self, bdot, out, epi, c.rs, Pil, sp, pb};
  const bool dot = (np + self + bdot) > 0;
  if (A.format == 0) {
    SellMat<T> M{A.n, A.nslices, A.slice_ptr, A.slice_w, A.perm, A.scol, pick_val<T>(A, true)};
    if (!dot)
      launch_sell<T, -1>(c, M, a);
    else if (np == 0)
      launch_sell<T, 0>(c, M, a);
    else if (np <= 4)
      launch_sell<T, 4>(c, M, a);
    else if (np <= 8)
      launch_sell<T, 8>(c, M, a);
    else
      launch_sell<T, 16>(c, M, a);
  } else {
    CsrMat<T> M{A.n, A.row_ptr, A.col, pick_val<T>(A, false)};
    if (!dot)
      launch_csr<T, -1>(c, M, a);
    else if (np == 0)
      launch_csr<T, 0>(c, M, a);
    else if (np <= 4)
      launch_csr<T, 4>(c, M, a);
    else if (np <= 8)
      launch_csr<T, 8>(c, M, a);
    else
      launch_csr<T, 16>(c, M, a);
  }
  return cudaGetLastError();
}

template cudaError_t spmv<double>(const Ctx&, const MatDesc&, const double*, double*, const double*,
                                  const double*, int64_t, int, int, int, double*, Epi, const double*, int,
                                  const double*);
template cudaError_t spmv<float>(const Ctx&, const MatDesc&, const float*, float*, const float*, const float*,
                                 int64_t, int, int, int, double*, Epi, const float*, int, const float*);

// ---------------------------------------------------------------------------
// Persistent level step: one cooperative launch runs, for level k of a cycle
// of Algorithm 1,
//   the gamma step on the top level      r^(k) -= V^(k) gamma_k,
//   the product                          r^(k+1) = A r^(k) and P^T r^(k+1),
//   for q = 0 .. s-1: the eta step       v_q^(k) = r^(k+1) - W^(k) eta_q,
//                     the product        v_q^(k+1) = A v_q^(k) and P^T v_q^(k+1),
// with every small solve (eta_q, then gamma_{k+1}) between them.  The updates
// of the levels below k stay with lazy_update.  One 1024-thread block per SM;
// the blocks meet at bounded grid barriers: after each vector update (the
// product reads other blocks' rows) and after each product's per-block
// partial sums, which every block then sums itself in the fixed order of the
// standalone product's last block, and solves the next s x s system itself.
// So no block waits on a single block's reduction and solve at the end of a
// product, and no launch separates the steps.  The products use the grid and
// slice-to-warp map of the standalone product (their first nb_prod blocks),
// the vector updates the formulas of the standalone kernels: the results are
// those of the per-kernel path bit for bit.  Vectors written during the
// launch are read through L2, except x of a product (see xload).  Block 0
// stores the projections and coefficients in the device state for the
// kernels that follow.
// ---------------------------------------------------------------------------
template <typename T>
struct LevelStepArgs {
  SellMat<T> A;
  T* R;              // r^(0..l), leading dimension ld
  T* V;              // V^(-1..l): v_q^(i) at column (i + 1) s + q
  int64_t ld;
  int n, s, k;
  int next_gamma;    // solve gamma_{k+1} at the end (k + 1 < l)
  int nb_prod;       // blocks of the products (the standalone product's grid)
  const T* P;
  int64_t ldp;
  const T* Pil;
  int sp;
  const T* Pb;
  DevState* st;
  double* partials;  // [nb_prod][MAXRED]
  unsigned int* bar; // barrier counter, zero at launch
  int* flag;
  long long spin_limit;
};

// out[row] = base[row] - sum_j c[j] col_j[row] over the rows of this thread
// (grid-stride over all blocks), j in column order: the formula of the
// standalone gamma and eta kernels.
template <typename T, int S, typename ColOf>
__device__ __forceinline__ void level_combine(int n, int s, const T* base, T* out, const T* c, ColOf col_of) {
  const int G = gridDim.x * SNT;
  for (int row = blockIdx.x * SNT + threadIdx.x; row < n; row += G) {
    T acc = __ldcg(base + row);
    T v[S];
#pragma unroll
    for (int j = 0; j < S; ++j) {
      if (j >= s) break;
      v[j] = __ldcg(col_of(j) + row);
    }
#pragma unroll
    for (int j = 0; j < S; ++j) {
      if (j >= s) break;
      acc = acc - c[j] * v[j];
    }
    out[row] = acc;
  }
}

// One product of the level step: y = A x with P^T y, this block's partial sums
// published, a grid barrier, and the sums of all partials in red (every block).
template <typename T, int NP>
__device__ __forceinline__ bool level_product(const LevelStepArgs<T>& L, const T* x, T* y, unsigned int& gen,
                                              double* smem_w, double* red, int* s_ok) {
  const int s = L.s;
  if (blockIdx.x < L.nb_prod) {
    SpmvArgs<T> a{x, y, nullptr, L.P, L.ldp, s, 0, 0, nullptr, Epi{EPI_NONE, 0, 0, s, 0, nullptr},
                  RedScratch{nullptr, nullptr, nullptr, 0}, L.Pil, L.sp, L.Pb};
    DotAcc<T, NP> acc;
    acc.zero();
    sell_pass<T, NP, 1>(L.A, a, acc, L.nb_prod);
    block_reduce_acc<T, NP>(a, acc, s, smem_w, red);
    if (threadIdx.x < s) L.partials[(size_t)blockIdx.x * MAXRED + threadIdx.x] = red[threadIdx.x];
  }
  if (!grid_sync(L.bar, ++gen, L.flag, L.spin_limit, s_ok)) return false;
  sum_partials(L.partials, L.nb_prod, s, red);
  return true;
}

// The s x s solve of the epilogues by warp 0: (P^T W) z = rhs with column j of
// P^T W from hi (j < q) or lo (j >= q), [j][c] layout with stride SMAX.
__device__ __forceinline__ bool level_solve(const double* lo, const double* hi, const double* rhs, int s, int q,
                                            EpiScratch& w) {
  const int lane = threadIdx.x & 31;
  for (int i = lane; i < s * s; i += 32) {
    const int c = i / s, j = i % s;
    w.a[i] = (j < q ? hi : lo)[j * SMAX + c];
  }
  if (lane < s) w.z[lane] = rhs[lane];
  __syncwarp();
  return warp_lu_solve(w.a, w.z, s, w.l);
}

template <typename T, int NP>
__global__ void __launch_bounds__(SNT, 1) level_kernel(LevelStepArgs<T> L) {
  __shared__ double smem_w[SNWARP * MAXRED];
  __shared__ double red[MAXRED];
  __shared__ double pv_lo[SMAX * SMAX];   // P^T V^(k):   [q][c]
  __shared__ double pv_hi[SMAX * SMAX];   // P^T V^(k+1): [q][c], as the products complete
  __shared__ double pr_hi[SMAX];          // P^T r^(k+1)
  __shared__ T coef[SMAX];                // gamma_k, then eta_q
  __shared__ EpiScratch ew;
  __shared__ int s_ok;
  const int s = L.s, k = L.k, n = L.n;
  const int64_t ld = L.ld;
  DevState* st = L.st;
  unsigned int gen = 0;
  for (int i = threadIdx.x; i < s * s; i += SNT)
    pv_lo[(i / s) * SMAX + (i % s)] = __ldcg(&st->projV[(k * SMAX + i / s) * SMAX + (i % s)]);
  if (threadIdx.x < s) coef[threadIdx.x] = (T)__ldcg(&st->gamma[k * SMAX + threadIdx.x]);
  __syncthreads();
  T* rk = L.R + (int64_t)k * ld;
  T* rk1 = L.R + (int64_t)(k + 1) * ld;
  T* Vk = L.V + (int64_t)(k + 1) * s * ld;    // V^(k)
  T* Vk1 = L.V + (int64_t)(k + 2) * s * ld;   // V^(k+1)
  // gamma step on the top level
  level_combine<T, NP>(n, s, rk, rk, coef, [&](int j) { return Vk + (int64_t)j * ld; });
  if (!grid_sync(L.bar, ++gen, L.flag, L.spin_limit, &s_ok)) return;
  // r^(k+1) = A r^(k), P^T r^(k+1)
  if (!level_product<T, NP>(L, rk, rk1, gen, smem_w, red, &s_ok)) return;
  if (threadIdx.x < s) {
    pr_hi[threadIdx.x] = red[threadIdx.x];
    if (blockIdx.x == 0) st->projR[(k + 1) * SMAX + threadIdx.x] = red[threadIdx.x];
  }
  __syncthreads();
  for (int q = 0; q < s; ++q) {
    // eta_q: (P^T W^(k)) eta_q = P^T r^(k+1), W^(k) = [V^(k+1)_{0:q-1}, V^(k)_{q:s-1}]
    if (threadIdx.x < 32) {
      const bool ok = level_solve(pv_lo, pv_hi, pr_hi, s, q, ew);
      if (threadIdx.x < s) {
        coef[threadIdx.x] = (T)ew.z[threadIdx.x];
        if (blockIdx.x == 0) st->eta[(k * SMAX + q) * SMAX + threadIdx.x] = ew.z[threadIdx.x];
      }
      if (threadIdx.x == 0 && blockIdx.x == 0 && !ok) atomicOr(&st->flag, FLAG_BREAKDOWN);
    }
    __syncthreads();
    // v_q^(k) = r^(k+1) - W^(k) eta_q
    level_combine<T, NP>(n, s, rk1, Vk + (int64_t)q * ld, coef,
                         [&](int j) { return (j < q ? Vk1 : Vk) + (int64_t)j * ld; });
    if (!grid_sync(L.bar, ++gen, L.flag, L.spin_limit, &s_ok)) return;
    // v_q^(k+1) = A v_q^(k), P^T v_q^(k+1)
    if (!level_product<T, NP>(L, Vk + (int64_t)q * ld, Vk1 + (int64_t)q * ld, gen, smem_w, red, &s_ok)) return;
    if (threadIdx.x < s) {
      pv_hi[q * SMAX + threadIdx.x] = red[threadIdx.x];
      if (blockIdx.x == 0) st->projV[((k + 1) * SMAX + q) * SMAX + threadIdx.x] = red[threadIdx.x];
    }
    __syncthreads();
  }
  // gamma_{k+1}: (P^T V^(k+1)) gamma = P^T r^(k+1), for the next level step
  if (L.next_gamma && blockIdx.x == 0 && threadIdx.x < 32) {
    const bool ok = level_solve(pv_hi, pv_hi, pr_hi, s, 0, ew);
    if (threadIdx.x < s) st->gamma[(k + 1) * SMAX + threadIdx.x] = ew.z[threadIdx.x];
    if (threadIdx.x == 0 && !ok) atomicOr(&st->flag, FLAG_BREAKDOWN);
  }
}

template <typename T, int NP>
static cudaError_t launch_level(const Ctx& c, LevelStepArgs<T>& L) {
  static int nb = -1;
  if (nb < 0) {
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, level_kernel<T, NP>, SNT, 0) != cudaSuccess) nb = 0;
  }
  if (nb < 1) return cudaErrorCooperativeLaunchTooLarge;
  void* args[] = {&L};
  return cudaLaunchCooperativeKernel((const void*)level_kernel<T, NP>, dim3(c.sms), dim3(SNT), args, 0, c.stream);
}

template <typename T>
cudaError_t level_step(const Ctx& c, const MatDesc& A, T* R, T* V, int64_t ld, int s, int k, int next_gamma,
                       const T* P, int64_t ldp, const T* Pil, int sp, const T* Pb, DevState* st,
                       unsigned int* bar, long long spin_limit) {
  if (A.format != 0 || s < 1 || s > SMAX || c.sms > MAXBLK) return cudaErrorInvalidValue;
  // the grid of the standalone product (launch_sell): min(slices' rows / SNT, SMs)
  const int64_t need = ((int64_t)A.nslices * 32 + SNT - 1) / SNT;
  const int nb_prod = (int)(need < c.sms ? need : c.sms);
  const T* pb = (Pb && !A.perm) ? Pb : nullptr;
  LevelStepArgs<T> L{SellMat<T>{A.n, A.nslices, A.slice_ptr, A.slice_w, A.perm, A.scol, pick_val<T>(A, true)},
                 R, V, ld, A.n, s, k, next_gamma, nb_prod, P, ldp, Pil, sp, pb, st, c.rs.partials, bar,
                 &st->flag, spin_limit};
  cudaError_t e = cudaMemsetAsync(bar, 0, sizeof(unsigned int), c.stream);
  if (e != cudaSuccess) return e;
  if (s <= 4) return launch_level<T, 4>(c, L);
  if (s <= 8) return launch_level<T, 8>(c, L);
  return launch_level<T, 16>(c, L);
}

template cudaError_t level_step<double>(const Ctx&, const MatDesc&, double*, double*, int64_t, int, int, int,
                                        const double*, int64_t, const double*, int, const double*, DevState*,
                                        unsigned int*, long long);
template cudaError_t level_step<float>(const Ctx&, const MatDesc&, float*, float*, int64_t, int, int, int,
                                       const float*, int64_t, const float*, int, const float*, DevState*,
                                       unsigned int*, long long);

// y = z or b - z, row by row, with the fused reductions of the product.
template <typename T, int NP>
__global__ void __launch_bounds__(SNT, 1) vec_dots_kernel(int n, const T* z, SpmvArgs<T> a) {
  constexpr int NA = NP < 0 ? 0 : NP;
  DotAcc<T, NA> acc;
  acc.zero();
  const int stride = gridDim.x * SNT;
  for (int row = blockIdx.x * SNT + threadIdx.x; row < n; row += stride) {
    const T zv = z[row];
    const T yv = a.b ? (T)(a.b[row] - zv) : zv;
    a.y[row] = yv;
    if constexpr (NP >= 0) acc_row<T, NA>(a, row, yv, acc);
  }
  if constexpr (NP >= 0) finish<T, NA>(a, acc);
}

template <typename T, int NP>
static void launch_vec_dots(const Ctx& c, int n, const T* z, const SpmvArgs<T>& a) {
  static int cap = max_grid(vec_dots_kernel<T, NP>, c);
  const int64_t need = ((int64_t)n + SNT - 1) / SNT;
  vec_dots_kernel<T, NP><<<(int)(need < cap ? need : cap), SNT, 0, c.stream>>>(n, z, a);
}

template <typename T>
cudaError_t vec_dots(const Ctx& c, int n, const T* z, T* y, const T* b, const T* P, int64_t ldp, int np,
                     int self, int bdot, double* out, Epi epi, const T* Pb) {
  if (np < 0 || np > SMAX) return cudaErrorInvalidValue;
  SpmvArgs<T> a{z, y, b, P, ldp, np, self, bdot, out, epi, c.rs, nullptr, 0, Pb};
  if (np + self + bdot == 0)
    launch_vec_dots<T, -1>(c, n, z, a);
  else if (np == 0)
    launch_vec_dots<T, 0>(c, n, z, a);
  else if (np <= 4)
    launch_vec_dots<T, 4>(c, n, z, a);
  else if (np <= 8)
    launch_vec_dots<T, 8>(c, n, z, a);
  else
    launch_vec_dots<T, 16>(c, n, z, a);
  return cudaGetLastError();
}

template cudaError_t vec_dots<double>(const Ctx&, int, const double*, double*, const double*, const double*,
                                      int64_t, int, int, int, double*, Epi, const double*);
template cudaError_t vec_dots<float>(const Ctx&, int, const float*, float*, const float*, const float*, int64_t,
                                     int, int, int, double*, Epi, const float*);

// Pil[row * sp + c] = P[c * ldp + row] for c < s, zero for s <= c < sp.
template <typename T>
__global__ void interleave_kernel(int n, int s, const T* P, int64_t ldp, int sp, T* Pil) {
  const int64_t total = (int64_t)n * sp;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t row = i / sp;
    const int c = (int)(i % sp);
    Pil[i] = c < s ? P[(int64_t)c * ldp + row] : T(0);
  }
}

template <typename T>
cudaError_t interleave_rows(const Ctx& c, int n, int s, const T* P, int64_t ldp, int sp, T* Pil) {
  const int64_t total = (int64_t)n * sp;
  int64_t g = (total + NT - 1) / NT;
  if (g > 8192) g = 8192;
  interleave_kernel<T><<<(int)g, NT, 0, c.stream>>>(n, s, P, ldp, sp, Pil);
  return cudaGetLastError();
}
template cudaError_t interleave_rows<double>(const Ctx&, int, int, const double*, int64_t, int, double*);
template cudaError_t interleave_rows<float>(const Ctx&, int, int, const float*, int64_t, int, float*);

// flag |= 1 if a row of P (s columns, leading dimension ldp) has a non-zero
// outside column pblock_col(row); else Pb[row] = P[pblock_col(row)][row].
template <typename T>
__global__ void pblock_kernel(int n, int s, const T* P, int64_t ldp, T* Pb, int* flag) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const int c = pblock_col(i, s);
    bool ok = true;
    for (int j = 0; j < s; ++j)
      if (j != c && P[(int64_t)j * ldp + i] != T(0)) ok = false;
    if (!ok) atomicOr(flag, 1);
    Pb[i] = P[(int64_t)c * ldp + i];
  }
}

template <typename T>
cudaError_t pblock_compress(const Ctx& c, int n, int s, const T* P, int64_t ldp, T* Pb, int* flag) {
  int64_t g = ((int64_t)n + NT - 1) / NT;
  if (g > 8192) g = 8192;
  pblock_kernel<T><<<(int)g, NT, 0, c.stream>>>(n, s, P, ldp, Pb, flag);
  return cudaGetLastError();
}
template cudaError_t pblock_compress<double>(const Ctx&, int, int, const double*, int64_t, double*, int*);
template cudaError_t pblock_compress<float>(const Ctx&, int, int, const float*, int64_t, float*, int*);

double spmv_bytes(const MatDesc& A, int prec) {
  const double vb = prec == 0 ? 8.0 : 4.0;
  if (A.format == 0)
    return (double)A.nnz_sell * (4.0 + vb) + 8.0 * A.nslices + (A.perm ? 4.0 * A.n : 0.0) + 2.0 * vb * A.n;
  return (double)A.nnz * (4.0 + vb) + 4.0 * (A.n + 1) + 2.0 * vb * A.n;
}

// ---------------------------------------------------------------------------
// matrix setup
// ---------------------------------------------------------------------------

__global__ void csr_validate_kernel(int n, int64_t nnz, const int* row_ptr, const int* col, int* flag) {
  const int stride = gridDim.x * blockDim.x;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
    const int b = row_ptr[i], e = row_ptr[i + 1];
    if ((i == 0 && b != 0) || (i == n - 1 && (int64_t)e != nnz) || e < b || b < 0 || (int64_t)e > nnz) {
      atomicOr(flag, 1);
      continue;
    }
    for (int p = b; p < e; ++p) {
      const int cidx = col[p];
      if (cidx < 0 || cidx >= n) {
        atomicOr(flag, 2);
        break;
      }
    }
  }
}

cudaError_t csr_validate(const Ctx& c, int n, int64_t nnz, const int* row_ptr, const int* col, int* flag) {
  int g = (int)((n + NT - 1) / NT);
  if (g > c.sms * 8) g = c.sms * 8;
  csr_validate_kernel<<<g, NT, 0, c.stream>>>(n, nnz, row_ptr, col, flag);
  return cudaGetLastError();
}

__global__ void csr_max_diag_kernel(int n, const int* row_ptr, const int* col, const double* val,
                                    unsigned long long* out_bits) {
  const int stride = gridDim.x * blockDim.x;
  double m = 0.0;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride)
    for (int p = row_ptr[i]; p < row_ptr[i + 1]; ++p)
      if (col[p] == i) m = fmax(m, fabs(val[p]));
  // non-negative doubles order like their bit patterns
  if (m > 0.0) atomicMax(out_bits, (unsigned long long)__double_as_longlong(m));
}

cudaError_t csr_max_diag(const Ctx& c, int n, const int* row_ptr, const int* col, const double* val,
                         unsigned long long* out_bits) {
  int g = (int)((n + NT - 1) / NT);
  if (g > c.sms * 8) g = c.sms * 8;
  csr_max_diag_kernel<<<g, NT, 0, c.stream>>>(n, row_ptr, col, val, out_bits);
  return cudaGetLastError();
}

__global__ void sell_fill_kernel(int n, int nslices, const int* row_ptr, const int* col, const double* val,
                                 const int* slice_ptr, const int* slice_w, const int* perm, int* scol,
                                 double* sval) {
  const int64_t total = (int64_t)nslices * 32;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t pos = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; pos < total; pos += stride) {
    const int sl = (int)(pos >> 5), lane = (int)(pos & 31);
    const int w = slice_w[sl];
    const int64_t base = (int64_t)slice_ptr[sl] + lane;
    int b = 0, len = 0, row = 0;
    if (pos < n) {
      row = perm ? perm[pos] : (int)pos;
      b = row_ptr[row];
      len = row_ptr[row + 1] - b;
    }
    for (int j = 0; j < w; ++j) {
      const int64_t o = base + (int64_t)j * 32;
      if (j < len) {
        scol[o] = col[b + j];
        sval[o] = val[b + j];
      } else {  // padding: a zero coefficient on the row's own index
        scol[o] = row;
        sval[o] = 0.0;
      }
    }
  }
}

cudaError_t sell_fill(const Ctx& c, int n, int nslices, const int* row_ptr, const int* col, const double* val,
                      const int* slice_ptr, const int* slice_w, const int* perm, int* scol, double* sval) {
  int g = (int)(((int64_t)nslices * 32 + NT - 1) / NT);
  if (g > c.sms * 8) g = c.sms * 8;
  sell_fill_kernel<<<g, NT, 0, c.stream>>>(n, nslices, row_ptr, col, val, slice_ptr, slice_w, perm, scol, sval);
  return cudaGetLastError();
}

}  // namespace msk

// ===========================================================================
// Allocation-free form of the fused product y = A x, P^T y (CSR).
//
// For callers that may not allocate device memory themselves -- code embedded
// in a host application that owns all device memory through its own pool, or
// time-critical loops where an allocation (which can synchronise the device or
// fail at run time) is not allowed.  The reduction scratch (one partial sum per
// thread block plus the ticket of the last-block combine) lives in this
// file-scope device array instead of in memory the caller provides.  Every GPU
// that loads the library holds one copy of it until the process exits.
// ===========================================================================
namespace msk {
constexpr int NOALLOC_MAX_BLOCKS = 1024;
constexpr int NOALLOC_MAX_DEVICES = 64;
constexpr size_t NOALLOC_DOUBLES = (size_t)NOALLOC_MAX_BLOCKS * MAXRED + 32;
static __device__ __align__(256) double g_noalloc_scratch[NOALLOC_DOUBLES];
}  // namespace msk

extern "C" msstab_status msstab_spmv_dot_noalloc(int64_t n, int64_t nnz, const int32_t* d_row_ptr,
                                                 const int32_t* d_col, const double* d_val, const double* d_x,
                                                 double* d_y, const double* d_P, int64_t ldp, int32_t s,
                                                 double* d_dots, void* stream) {
  using namespace msk;
  if (n < 1 || n > MAX_ROWS || nnz < 0 || nnz >= (1LL << 31)) {
    set_global_error("msstab_spmv_dot_noalloc: n must be in [1, 2^31 - 2^22] and nnz in [0, 2^31)");
    return MSSTAB_ERR_INVALID_ARG;
  }
  if (s < 0 || s > SMAX) {
    set_global_error("msstab_spmv_dot_noalloc: s must be in [0, 16] (the scratch holds 17 sums per block)");
    return MSSTAB_ERR_INVALID_ARG;
  }
  if (!d_row_ptr || !d_x || !d_y || !d_dots || (nnz > 0 && (!d_col || !d_val)) || (s > 0 && (!d_P || ldp < n))) {
    set_global_error("msstab_spmv_dot_noalloc: NULL pointer or ldp < n");
    return MSSTAB_ERR_INVALID_ARG;
  }
  // Set-up, once per device and with that device current: the device address
  // of the scratch array (its name is only a stand-in in host code).
  static std::mutex mu;
  static void* addr[NOALLOC_MAX_DEVICES] = {};
  static int sms[NOALLOC_MAX_DEVICES] = {};
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess || dev < 0 || dev >= NOALLOC_MAX_DEVICES) {
    set_global_error("msstab_spmv_dot_noalloc: no usable current device");
    return MSSTAB_ERR_CUDA;
  }
  {
    std::lock_guard<std::mutex> lock(mu);
    if (!addr[dev]) {
      void* ptr = nullptr;
      e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
      if (e != cudaSuccess || !ptr) {
        set_global_error(std::string("msstab_spmv_dot_noalloc: cudaGetSymbolAddress: ") + cudaGetErrorString(e));
        return MSSTAB_ERR_CUDA;
      }
      int m = 0;
      e = cudaDeviceGetAttribute(&m, cudaDevAttrMultiProcessorCount, dev);
      if (e != cudaSuccess) {
        set_global_error(std::string("msstab_spmv_dot_noalloc: ") + cudaGetErrorString(e));
        return MSSTAB_ERR_CUDA;
      }
      sms[dev] = m;
      addr[dev] = ptr;
    }
  }
  // An error left pending by earlier, unrelated work on this thread is
  // reported as such and left pending for its owner, so that the status of
  // the launch below is this call's own.
  e = cudaPeekAtLastError();
  if (e != cudaSuccess) {
    set_global_error(std::string("msstab_spmv_dot_noalloc: a CUDA error from earlier work is pending (not "
                                 "cleared): ") + cudaGetErrorString(e));
    return MSSTAB_ERR_CUDA;
  }
  double* base = (double*)addr[dev];
  RedScratch rs{base, nullptr, (unsigned int*)(base + (size_t)NOALLOC_MAX_BLOCKS * MAXRED), NOALLOC_MAX_BLOCKS};
  cudaStream_t st = (cudaStream_t)stream;
  // the ticket must start at zero (the array keeps the last call's contents)
  e = cudaMemsetAsync(rs.tickets, 0, sizeof(unsigned int), st);
  if (e != cudaSuccess) {
    set_global_error(std::string("msstab_spmv_dot_noalloc: ") + cudaGetErrorString(e));
    return MSSTAB_ERR_CUDA;
  }
  int nb = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, spmv_csr_kernel<double, 16>, SNT, 0) != cudaSuccess ||
      nb < 1)
    nb = 1;
  int64_t g = ((int64_t)n + SNT - 1) / SNT;
  if (g > (int64_t)nb * sms[dev]) g = (int64_t)nb * sms[dev];
  if (g > NOALLOC_MAX_BLOCKS) g = NOALLOC_MAX_BLOCKS;
  CsrMat<double> M{(int)n, d_row_ptr, d_col, d_val};
  SpmvArgs<double> a{d_x, d_y, nullptr, d_P, ldp, s, 1, 0, d_dots, Epi{EPI_NONE, 0, 0, s, 1, nullptr}, rs, nullptr, 0, nullptr};
  spmv_csr_kernel<double, 16><<<(int)g, SNT, 0, st>>>(M, a);
  e = cudaGetLastError();
  if (e != cudaSuccess) {
    set_global_error(std::string("msstab_spmv_dot_noalloc: launch: ") + cudaGetErrorString(e));
    return MSSTAB_ERR_CUDA;
  }
  return MSSTAB_OK;
}

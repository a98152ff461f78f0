// Host-side launchers of the CUDA kernels (internal to libmsstab).
// Every launcher enqueues on ctx.stream and returns the launch status.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>

#include "common.cuh"

namespace msk {

// Text returned by msstab_last_error(NULL) (entry points without a handle).
void set_global_error(const std::string& what);

struct Ctx {
  cudaStream_t stream;
  int sms;
  RedScratch rs;
};

// Device copy of A: SELL-32-sigma or CSR, FP64 values and FP32 values of A/rho.
struct MatDesc {
  int n;
  int64_t nnz;
  int format;                 // 0 SELL, 1 CSR
  // CSR (format 1)
  const int* row_ptr;
  const int* col;
  const double* val64;
  const float* val32;
  // SELL (format 0)
  int nslices;
  int64_t nnz_sell;           // stored entries including padding
  const int* slice_ptr;
  const int* slice_w;
  const int* perm;
  const int* scol;
  const double* sval64;
  const float* sval32;
};

// Bytes one product with A moves at minimum (matrix arrays once, x read once,
// y written once), for the roofline.
double spmv_bytes(const MatDesc& A, int prec);

// y = A x  (b == NULL) or y = b - A x; with np > 0: out[c] = P_c . y for
// c < np (P columns at P + c*ldp), then out[np] = y.y if self, then b.b if
// bdot.  The last block runs the epilogue.
// Pil (optional): the same P interleaved by row, Pil[row * sp + c], rows on
// 16-byte boundaries (sp a multiple of 16 / sizeof(T)); the SELL kernel then
// loads a row's P entries with vector loads issued with the matrix loads.
// Pb (optional): P in block-partitioned form (row i's only non-zero in column
// (i / 32) mod np, Pb[i] its value): one multiply-add per row for the dots.
template <typename T>
cudaError_t spmv(const Ctx& c, const MatDesc& A, const T* x, T* y, const T* b, const T* P, int64_t ldp,
                 int np, int self, int bdot, double* out, Epi epi, const T* Pil = nullptr, int sp = 0,
                 const T* Pb = nullptr);

// Pb[i] = P[(i / 32) mod s][i]; *flag |= 1 if P has any other non-zero.
template <typename T>
cudaError_t pblock_compress(const Ctx& c, int n, int s, const T* P, int64_t ldp, T* Pb, int* flag);

// Pil[row * sp + c] = P[c * ldp + row] (c < s), zero padding up to sp.
template <typename T>
cudaError_t interleave_rows(const Ctx& c, int n, int s, const T* P, int64_t ldp, int sp, T* Pil);

// Multi-dot: for targets t < nt: out[t*ostride + c] = X_t . Y_c (c < ny) and,
// if self, out[t*ostride + ny] = X_t . X_t.  Column pointers are given
// explicitly.  The last block runs the epilogue.
constexpr int MD_MAXT = 17;
constexpr int MD_MAXC = 17;
template <typename T>
struct MdCols {
  const T* x[MD_MAXT];
  const T* y[MD_MAXC];
};
template <typename T>
cudaError_t multidot(const Ctx& c, int n, const MdCols<T>& cols, int nt, int ny, int self, double* out,
                     int ostride, Epi epi);

// r^(k) -= V^(k) gamma (gamma: s FP64 device values).
template <typename T>
cudaError_t gamma_eager(const Ctx& c, int n, int s, T* R, const T* V, int64_t ld, int k, const double* gamma);

// v_q^(k) = r^(k+1) - [V^(k+1)_{0:q-1}, V^(k)_{q:s-1}] eta (eta: s FP64 device values).
template <typename T>
cudaError_t eta_eager(const Ctx& c, int n, int s, const T* R, T* V, int64_t ld, int k, int q, const double* eta);

// Updates of level step k on the levels below k (see msstab_op_lazy_update).
// eta row q at eta + q*eta_ld.
template <typename T>
cudaError_t lazy_update(const Ctx& c, int n, int s, T* R, T* V, T* x, int64_t ld, int k, const double* gamma,
                        const double* eta, int eta_ld);

// Degree-l step (tau from st->tau if tau == NULL, else from tau), followed
// (proj != 0) by P^T r, P^T V^(0) and r.r into st->projR[0], st->projV[0],
// st->rr and the epilogue.  With do_update == 0 only the projections are
// computed.  xbak (nullable) receives a copy of the new x.  xonly != 0 (the
// per-group kernel only, do_update != 0): r^(0) is replaced right after this
// step, so it updates x but neither r^(0) nor P^T r, r.r.
template <typename T>
cudaError_t tau_update(const Ctx& c, int n, int s, int ell, T* R, T* V, T* x, T* xbak, int64_t ld,
                       const double* tau, const T* P, int64_t ldp, int do_update, int proj, DevState* st,
                       Epi epi, const T* Pb = nullptr, const T* Pil = nullptr, int sp = 0,
                       const double* lgamma = nullptr, const double* leta = nullptr, int leta_ld = 0,
                       int xonly = 0);

// Whether tau_update can run the level -1 updates of level step 0 (lazy_update
// with k = 0, gamma and eta passed as lgamma, leta) in the same pass (the FP32
// degree-1 step with 16-byte aligned columns, n % 4 == 0); results are those of
// lazy_update followed by tau_update bit for bit.
template <typename T>
bool tau_fuses_lazy(int n, int s, int ell, const T* R, const T* V, const T* x, const T* xbak, int64_t ld,
                    const T* P, int64_t ldp, const T* Pb);

// w -= sum_{c<nc} h[c] U_c (h: FP64 device), columns U_c at U + c*ld.
template <typename T>
cudaError_t cols_axpy(const Ctx& c, int n, T* w, const T* U, int64_t ld, int nc, const double* h);

// y = x * (1 / sqrt(*nrm2))   (device scalar)
template <typename T>
cudaError_t scale_rsqrt(const Ctx& c, int n, const T* x, T* y, const double* nrm2);

// V <- V R^-1 and U <- U R^-1 (R upper s x s row-major FP64 device; U may be NULL).
template <typename T>
cudaError_t tri_apply(const Ctx& c, int n, int s, T* V, T* U, int64_t ld, const double* R);

// Single-thread kernels: Cholesky (R^T R = G) with flag, LU solve, tau solve.
cudaError_t small_cholesky(const Ctx& c, int s, const double* G, double* R, int* flag);
cudaError_t small_lu(const Ctx& c, int n, const double* M, const double* rhs, double* z, int* flag);
cudaError_t small_tau(const Ctx& c, int ell, const double* G, double* tau);

// Precision conversions: y32 = (float)(x64 * alpha); y64 += alpha * (double)x32;
// y64 = alpha * x64 + beta * z64.
cudaError_t to_f32_scaled(const Ctx& c, int n, const double* x, float* y, double alpha);
cudaError_t axpy_f32_into_f64(const Ctx& c, int n, const float* x, double* y, double alpha);
cudaError_t axpby_f64(const Ctx& c, int n, double alpha, const double* x, double beta, const double* z,
                      double* y);
cudaError_t f64_to_f32_n(const Ctx& c, int64_t n, const double* x, float* y, double alpha);

// Matrix setup: CSR validation (flag bit 1: bad row_ptr, 2: bad column),
// max |a_ii| (as ordered bits), SELL fill, FP32 scaled copy.
cudaError_t csr_validate(const Ctx& c, int n, int64_t nnz, const int* row_ptr, const int* col, int* flag);
cudaError_t csr_max_diag(const Ctx& c, int n, const int* row_ptr, const int* col, const double* val,
                         unsigned long long* out_bits);
cudaError_t sell_fill(const Ctx& c, int n, int nslices, const int* row_ptr, const int* col, const double* val,
                      const int* slice_ptr, const int* slice_w, const int* perm, int* scol, double* sval);

// Persistent level step k of Algorithm 1 (one cooperative launch, SELL only):
// the gamma step on r^(k) (gamma_k from st->gamma), r^(k+1) = A r^(k), and for
// q = 0..s-1 the eta step and v_q^(k+1) = A v_q^(k), with the projections
// (st->projR[k+1], st->projV[k+1]), eta (st->eta[k]) and, if next_gamma,
// gamma_{k+1} stored in st.  bar: one device counter (zeroed here before the
// launch); every grid barrier gives up after spin_limit polls with
// FLAG_SYNC_TIMEOUT in st->flag.
template <typename T>
cudaError_t level_step(const Ctx& c, const MatDesc& A, T* R, T* V, int64_t ld, int s, int k, int next_gamma,
                       const T* P, int64_t ldp, const T* Pil, int sp, const T* Pb, DevState* st,
                       unsigned int* bar, long long spin_limit);

// y = z (b == NULL) or y = b - z, with the reductions and the epilogue of the
// fused product (the same out layout as spmv): the tail of a product with a
// preconditioned operator whose last stage produced z.
template <typename T>
cudaError_t vec_dots(const Ctx& c, int n, const T* z, T* y, const T* b, const T* P, int64_t ldp, int np,
                     int self, int bdot, double* out, Epi epi, const T* Pb = nullptr);

// ILU(0) of A on A's own pattern and its level schedules (ilu.cu).
struct GridBar {
  unsigned int count;             // level-barrier counter of the running sweep
  unsigned int pad;
};
struct IluDesc {
  int n = 0;
  const int* row_ptr = nullptr;   // A's CSR pattern (sorted columns, diagonal present)
  const int* col = nullptr;
  double* lu = nullptr;           // factor values on that pattern: L left of the diagonal, U from it on
  int* diag = nullptr;            // position of a_ii in each row
  int nlev[2] = {0, 0};           // levels of the lower [0] and upper [1] dependency graphs
  int* lev[2] = {nullptr, nullptr};     // level of each row
  int* lptr[2] = {nullptr, nullptr};    // rows of level l: lrows[lptr[l] .. lptr[l+1])
  int* lrows[2] = {nullptr, nullptr};
  int max_width[2] = {0, 0};      // rows in the widest level
  int grid[2] = {1, 1};           // blocks of the cooperative sweeps
  // level-ordered packed dependencies of the two solves (when every row has at
  // most 8), each level padded to a multiple of 32 positions: position idx
  // holds row prow[idx] (-1: padding), its pcnt dependencies
  // pcol[j * npad + idx] with factor values pval[j * npad + idx] (column
  // order), and for the upper solve u_ii in pdiag[1][idx]
  int W[2] = {0, 0};              // compile-time width used (4 or 8), 0: CSR sweeps
  int npad[2] = {0, 0};
  int* prow[2] = {nullptr, nullptr};
  int* pcnt[2] = {nullptr, nullptr};
  int* pcol[2] = {nullptr, nullptr};
  double* pval[2] = {nullptr, nullptr};
  double* pdiag[2] = {nullptr, nullptr};
  int* pptr[2] = {nullptr, nullptr};   // padded positions of level l: [pptr[l], pptr[l+1])
  // chunked order of the pipelined solves (CH[u] > 0): rows cut into chunks of
  // CH rows, one per block; chunk b's levels are the groups [gofs[b],
  // gofs[b+1]), group q holds positions [gptr[q], gptr[q+1]); a dependency in
  // the previous group of the same chunk (within its first 1024 positions) is
  // stored as -1 - its offset in that group, any other as its row
  int CH[2] = {0, 0};
  int groups[2] = {0, 0};
  int* gofs[2] = {nullptr, nullptr};
  int* gptr[2] = {nullptr, nullptr};
  int* cprow[2] = {nullptr, nullptr};
  int* cpcnt[2] = {nullptr, nullptr};
  int* cpcol[2] = {nullptr, nullptr};
  double* cpval[2] = {nullptr, nullptr};
  double* cpdiag = nullptr;
  double* scratch = nullptr;      // copy of the right-hand side of an in-place chunked solve
  GridBar* bar = nullptr;         // grid-barrier state (zero between launches)
  int* flag = nullptr;            // device flag word (FLAG_SYNC_TIMEOUT, FLAG_ZERO_PIVOT)
  long long spin_limit = 1LL << 22;   // polls before a wait on another block gives up
};
struct IluSetupResult {
  int code = 0;                   // 0 ok, 1 CUDA error, 2 bad structure, 3 zero pivot, 4 out of memory
  cudaError_t cuda = cudaSuccess;
  const char* where = nullptr;
};
typedef void* (*DevAllocFn)(void* ctx, size_t bytes);

// Diagonal positions, levels and the numeric factor (F.n, row_ptr, col, lu =
// a copy of A's values, bar and flag set by the caller; lu is overwritten).
// h_scratch: one pinned int for the read-backs.
IluSetupResult ilu_setup(const Ctx& c, IluDesc& F, DevAllocFn alloc, void* actx, int* h_scratch);
// y = L^-1 z (unit lower; y may equal z); t = U^-1 v (t may equal v); y = U x.
cudaError_t ilu_lower_solve(const Ctx& c, const IluDesc& F, const double* z, double* y);
cudaError_t ilu_upper_solve(const Ctx& c, const IluDesc& F, const double* v, double* t);
cudaError_t ilu_upper_mul(const Ctx& c, const IluDesc& F, const double* x, double* y);

}  // namespace msk

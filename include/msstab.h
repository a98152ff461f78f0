/*
 * msstab.h -- C ABI of libmsstab: M(s)stab(l) and IDR(s)stab(l) for sequences
 * of sparse linear systems A x^(i) = b^(i) with fixed A, on one GB300 (sm_103a).
 *
 * Method: Neuenhofen, "M(s)stab(l): A Generalization of IDR(s)stab(l) for
 * Sequences of Linear Systems" (arXiv:1604.06043).  msstab_solve runs
 * Algorithm 1 (IDRstab); the handle keeps the cut space P and, from the
 * fetching point of an earlier solve on (Section 5), the recycled basis U, V
 * with V = A U, which later solves take as their start basis -- the M(s)stab
 * method of Section 4.2.
 *
 * Conventions for every entry point below:
 *  - Pointers named d_* are CUDA device pointers, owned by the caller; pointers
 *    without the prefix are host pointers.  Vectors are dense, contiguous and
 *    aligned to their element size.  A block of s vectors of length n is stored
 *    column by column ("column-major"), column q at base + q * ld.
 *  - All work is ordered on the stream given at create time (options.stream;
 *    NULL = the legacy default stream).  Calls on one handle must not overlap;
 *    a handle is not thread safe.
 *  - Errors are returned as msstab_status codes, never by abort; the text of
 *    the last error of a handle is msstab_last_error(h) (h may be NULL for
 *    errors of msstab_create).
 *  - Scalars are FP64.  Indices are int32 (n and nnz must fit).
 */
#ifndef MSSTAB_H
#define MSSTAB_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct msstab_s* msstab_t;

typedef enum msstab_status {
  MSSTAB_OK = 0,
  MSSTAB_ERR_INVALID_ARG = 1, /* bad size, pointer, alignment or CSR structure */
  MSSTAB_ERR_CUDA = 2,        /* a CUDA runtime call failed (text in msstab_last_error) */
  MSSTAB_ERR_OOM = 3,         /* device or pinned-host allocation failed */
  MSSTAB_ERR_BREAKDOWN = 4,   /* a projected s x s system was singular (Section 2.2 canonical case violated) */
  MSSTAB_ERR_MAXIT = 5,       /* options.max_mvs reached before the tolerance */
  MSSTAB_ERR_NAN = 6          /* the residual norm became NaN or Inf */
} msstab_status;

enum { MSSTAB_PREC_FP64 = 0, MSSTAB_PREC_FP32_INNER = 1 };
enum { MSSTAB_FETCH_ONCE = 0, MSSTAB_FETCH_EVERY = 1, MSSTAB_FETCH_NEVER = 2, MSSTAB_FETCH_SLOPE = 3,
       MSSTAB_FETCH_PROBE = 4 };
enum { MSSTAB_FORMAT_SELL = 0, MSSTAB_FORMAT_CSR = 1 };
enum { MSSTAB_PRECOND_NONE = 0, MSSTAB_PRECOND_ILU0 = 1 };

/* Kernel families, the index into msstab_stats.t_ms / n_launch. */
enum {
  MSSTAB_K_SPMV = 0,     /* y = A x, r = b - A x (+ norms) */
  MSSTAB_K_SPMV_DOT = 1, /* y = A x fused with P^T y and the next small solve */
  MSSTAB_K_GAMMA = 2,    /* r^(k) -= V^(k) gamma */
  MSSTAB_K_ETA = 3,      /* v_q^(k) = r^(k+1) - W^(k) eta_q */
  MSSTAB_K_LAZY = 4,     /* the same updates on levels below k, once per level step */
  MSSTAB_K_TAU = 5,      /* Gram, tau step, P^T [r, V] */
  MSSTAB_K_OTHER = 6,    /* Arnoldi start, orthonormalisation, conversions, copies */
  MSSTAB_K_CNN = 7,      /* learned initial guess */
  MSSTAB_K_PRECOND = 8,  /* ILU(0) triangular solves and U x (the preconditioned operator) */
  MSSTAB_K_LEVEL = 9,    /* persistent level step: gamma step, the s + 1 products with A and the
                            eta steps of one level, with their small solves, in one launch */
  MSSTAB_K_COUNT = 10
};

typedef struct msstab_options {
  int32_t precision;       /* MSSTAB_PREC_FP64 (default) or MSSTAB_PREC_FP32_INNER: FP32 inner
                              M(s)stab on A/rho inside an FP64 defect-correction loop */
  int32_t fetch_policy;    /* MSSTAB_FETCH_ONCE (default): fetch U,V in the first solve and reuse
                              them for all later solves; EVERY: pass each solve's final U,V on
                              (Miltenberger, Section 3.1); NEVER: IDRstab with an Arnoldi start
                              for every system.  The fetching point, after the section on
                              choosing it ("shortly before the residual drops"): ONCE at the
                              fetch_threshold / fetch_cycle below; SLOPE in the first solve at
                              the basis of the cycle before the first cycle that lowers log10
                              relres by >= 1 and by >= twice the mean of the cycles before it
                              (the final basis if none does); PROBE: the first solve is an
                              IDRstab probe that writes nothing, and the second, again IDRstab,
                              fetches at the cycle end before the probe's steepest one-cycle
                              drop (its final basis if it converges earlier).  SLOPE and PROBE:
                              FP64 only */
  double fetch_threshold;  /* fetch at the first cycle end with relres <= this; <= 0: sqrt(tol) */
  int32_t fetch_cycle;     /* > 0: fetch at the end of this cycle instead of by threshold */
  int32_t orth_recycle;    /* 1 (default): condition the fetched basis -- V := A U (s products
                              with A, counted in the fetching solve), then Cholesky QR twice of
                              V with U carried along; 0: keep U, V exactly as fetched (the
                              paper's plain hand-over) */
  int64_t max_mvs;         /* products with A per solve; <= 0: min(100000, 20 sqrt(n) + 1 + s + 2l(s+1)) */
  double inner_tol;        /* FP32 inner: relative tolerance of each inner solve (tested on its
                              recursive residual); <= 0: max(1e-2, 0.5 tol ||b|| / ||r_outer||).
                              An inner solve also stops when its residual has not halved in 4
                              cycles (the FP32 floor near kappa * 6e-8 is reached).  A correction
                              that does not reduce the FP64 residual is undone and the next inner
                              solve restarts its basis; a second one in a row ends the solve with
                              MSSTAB_ERR_MAXIT and the better x */
  int32_t spmv_format;     /* MSSTAB_FORMAT_SELL (default, SELL-32-sigma) or MSSTAB_FORMAT_CSR */
  int32_t sell_sigma;      /* SELL sorting window in rows (1 = no sorting, default; else a
                              multiple of 32) */
  int32_t kernel_timing;   /* 1: time every launch with CUDA events (msstab_stats.t_ms) */
  int32_t max_outer;       /* FP32 inner: defect-correction iterations per solve; <= 0: 20 */
  int32_t inner_ell;       /* FP32 inner: stabilisation degree of the inner solves (1 <= . <= l);
                              <= 0: 1.  In FP32 the degree-l polynomial step through the level
                              vectors A^k r drifts from the true residual for l > 1 on stiff
                              problems; l = 1 keeps the inner recursive residual honest */
  int32_t replace_every;   /* > 0: replace the recursive residual by the true residual b - A x at
                              the end of every replace_every-th cycle (one product with A, fused
                              with the projections the next cycle needs), as the preconditioned
                              experiment of Section 5.1 does after each cycle; bounds the gap that
                              the drift of V from A U opens between the two.  0 (default):
                              Algorithm 1 as printed, true residual only to confirm convergence */
  int32_t precond;         /* MSSTAB_PRECOND_NONE (default) or MSSTAB_PRECOND_ILU0: split
                              preconditioning with the incomplete LU factorisation with zero
                              fill-in (Section 5.1): every solve runs on L^-1 A U^-1 x~ = L^-1 b
                              from x~0 = U x0 and returns x = U^-1 x~; the tolerance, the fetching
                              point, the recycled U, V and replace_every refer to that system (its
                              true residual is L^-1 (b - A U^-1 x~)).  FP64 only; A must hold every
                              diagonal entry and strictly increasing columns in each row */
  int32_t persistent;      /* 1 (default): each level step of an FP64 cycle (the gamma step, the
                              s + 1 products with A with their projections and small solves, the
                              eta steps) runs as ONE cooperative launch of one 1024-thread block
                              per SM whose blocks meet at grid barriers; results are those of 0 bit
                              for bit.  2: the FP32 inner cycles too (measured 6 % slower than their
                              graph-replayed launches at 128^3: the barriers and per-block solves
                              cost what the shorter FP32 products save).  0: one launch per step.
                              Used with the SELL format and without the preconditioner (else 0) */
  void* stream;            /* cudaStream_t for all work of the handle; NULL = default stream */
  int64_t spin_limit;      /* polls after which a device-side wait of the library gives up (the
                              grid barriers of the level steps and of the ILU(0) sweeps, the
                              sweeps' waits on other blocks' values): the kernel raises a flag,
                              every block leaves, and the call returns MSSTAB_ERR_CUDA ("timed
                              out") with d_x untouched; the handle stays usable.  <= 0: 2^22
                              (seconds; a wait that long means a block is not running) */
} msstab_options;

typedef struct msstab_stats {
  int64_t mvs;            /* all products with A in the call (FP64 and FP32) */
  int64_t mvs_fp32;       /* of which with the FP32 copy A/rho */
  int64_t cycles;         /* cycles of Algorithm 1 (inner cycles for FP32_INNER) */
  int64_t outer;          /* defect-correction iterations (FP32_INNER), else 0 */
  int64_t launches;       /* kernel launches of this library in the call */
  double relres_true;     /* ||b - A x|| / ||b|| of the returned x (FP64) */
  double relres_rec;      /* recursive residual at the last cycle end (FP64 mode) */
  double ms;              /* device time of the call (CUDA events on the stream) */
  int32_t status;         /* the returned msstab_status */
  int32_t fetched;        /* 1 if this call wrote the recycle store */
  int32_t used_recycle;   /* 1 if this call started from recycled U,V */
  int32_t guess_used;     /* set by msstab_select_guess */
  int32_t fp64_finish;    /* FP32_INNER: 1 if the FP32 corrections stalled and FP64 IDR(s)stab(l)
                             finished the solve from the current x */
  int32_t fetch_at;       /* the cycle whose basis this call wrote to the recycle store (fetched) */
  double relres_orig;     /* ||b - A x|| / ||b|| of the original system (differs from relres_true
                             only with the ILU(0) preconditioner, whose relres_true is that of
                             L^-1 A U^-1 x~ = L^-1 b) */
  double t_ms[MSSTAB_K_COUNT];     /* per kernel family, when options.kernel_timing */
  int64_t n_launch[MSSTAB_K_COUNT];
} msstab_stats;

/* Fill *opt with the defaults described above. */
void msstab_default_options(msstab_options* opt);

/*
 * Create a solver for the n x n matrix A (CSR: d_row_ptr[n+1], d_col[nnz],
 * d_val[nnz], int32 indices, FP64 values) with cut-space dimension s and
 * stabilisation degree l (Algorithm 1's s and l; 1 <= s <= 16, 1 <= l <= 8,
 * s <= n; 1 <= n <= 2^31 - 2^22, 0 <= nnz < 2^31).  d_p_raw (s columns of
 * length n, ld = n) is the raw random basis of the cut space P; it is
 * orthonormalised on the device (Cholesky QR, twice) and
 * kept, with an FP32 copy, for the lifetime of the handle (Section 2.4: the
 * basis of P may be random; Section 4.2: P stays fixed over the sequence).
 * The matrix is copied (the caller may free its arrays afterwards), converted
 * to SELL-32-sigma if chosen, and an FP32 copy of A/rho, rho = max|a_ii|, is
 * made.  The CSR structure is validated on the device (row_ptr monotone,
 * columns in range).  opt may be NULL (defaults).
 */
msstab_status msstab_create(int64_t n, int64_t nnz, const int32_t* d_row_ptr, const int32_t* d_col,
                            const double* d_val, int32_t s, int32_t ell, const double* d_p_raw,
                            const msstab_options* opt, msstab_t* out);

/*
 * Solve A x = b to ||b - A x|| <= tol ||b|| (Algorithm 1; the stopping test is
 * the recursive residual at cycle ends, confirmed by the true residual, which
 * replaces r if it fails).  d_x holds x0 on entry and the solution on return.
 * The start basis is the recycled U, V if the handle holds them (M(s)stab), else
 * the Arnoldi basis of level s of the initial residual (IDRstab).  In the first
 * solves, U, V are written to the recycle store at the fetching point
 * (Section 5).  Blocks until the stats are final.  On BREAKDOWN, MAXIT or NAN,
 * d_x holds the iterate of the last completed cycle (a basis fetched earlier in
 * the same solve is kept).  st may be NULL.
 */
msstab_status msstab_solve(msstab_t h, const double* d_b, double* d_x, double tol, msstab_stats* st);

/* As msstab_solve with host buffers b[n] and x[n]: the copies to and from the
 * device (straight from and to the caller's memory) are part of the call. */
msstab_status msstab_solve_host(msstab_t h, const double* b, double* x, double tol, msstab_stats* st);

/* Free all device and host memory of the handle.  NULL is accepted. */
msstab_status msstab_destroy(msstab_t h);

/* Text of the last error of h (or of the last failed create when h is NULL). */
const char* msstab_last_error(msstab_t h);

/* The per-cycle relative recursive residuals of the last solve (the start value
 * first) and the MV count at each of those points; copies min(cap, count). */
msstab_status msstab_history(msstab_t h, double* relres, int64_t* mvs, int32_t cap, int32_t* count);

/* Set options.spin_limit of an existing handle (polls before a device-side
 * wait gives up; <= 0: the default 2^22).  Takes effect from the next call. */
msstab_status msstab_set_spin_limit(msstab_t h, int64_t polls);

/* Drop the recycled U, V (the next solve starts from an Arnoldi basis again). */
msstab_status msstab_reset_recycle(msstab_t h);

/* *flag = 1 if the handle holds recycled U, V. */
msstab_status msstab_has_recycle(msstab_t h, int32_t* flag);

/* Copy the recycled basis out (d_U, d_V: s columns each, ld = n) or in.  With
 * these a sequence can be resumed by another handle on the same A and P. */
msstab_status msstab_export_recycle(msstab_t h, double* d_U, double* d_V);
msstab_status msstab_import_recycle(msstab_t h, const double* d_U, const double* d_V);

/*
 * Learned initial guess (selection step).  Given the previous solution d_xprev
 * and a correction d_delta (e.g. from msstab_cnn_infer), set
 *   d_x = d_xprev + d_delta  if ||b - A (x_prev + delta)|| < ||b - A x_prev||,
 *   d_x = d_xprev            otherwise,
 * using two products with A (FP64).  *used = 1 if the correction was kept.
 */
msstab_status msstab_select_guess(msstab_t h, const double* d_b, const double* d_xprev,
                                  const double* d_delta, double* d_x, int32_t* used);

/* The same with the correction scaled optimally: d_x = d_xprev + alpha d_delta
 * with alpha = (r0 . A delta) / ||A delta||^2 minimising ||b - A x|| (r0 =
 * b - A x_prev; two products with A), which never increases the residual;
 * falls back to d_xprev (used = 0) if alpha is 0 or not finite.  *alpha and
 * *reduction (= ||b - A x|| / ||r0||) may be NULL. */
msstab_status msstab_select_guess_scaled(msstab_t h, const double* d_b, const double* d_xprev,
                                         const double* d_delta, double* d_x, int32_t* used, double* alpha,
                                         double* reduction);

/* The residual-minimising combination of up to four directions (a workload
 * form, not in the paper): with r0 = b - A x_prev and W = [A dir_1 .. A dir_m]
 * (dir_j at d_dirs + (j-1) ld, ld >= n, 1 <= m <= min(4, s (l + 2))),
 *   d_x = d_xprev + sum_j a_j dir_j,  a = argmin ||r0 - W a||,
 * computed from the normal equations scaled by diag(W^T W)^-1/2 (Cholesky; a
 * zero direction gets a_j = 0; for numerically dependent directions the best
 * single one is taken).  Uses 1 + m products with A (FP64) and the handle's
 * level workspace (free between solves).  *used = 1 if the combination lowers
 * the residual, else d_x = d_xprev and a = 0.  coef (host, m entries) and
 * *reduction (host, ||b - A x|| / ||r0||) may be NULL.  For time-stepping
 * sequences the directions are the network's correction (msstab_cnn_infer)
 * and the previous step's change x^(i) - x^(i-1). */
msstab_status msstab_select_guess_span(msstab_t h, const double* d_b, const double* d_xprev, const double* d_dirs,
                                       int64_t ld, int32_t ndir, double* d_x, int32_t* used, double* coef,
                                       double* reduction);

/* ---------------------------------------------------------------------------
 * Kernel-level entry points on a handle (for testing and measuring single
 * kernels).  prec selects FP64 (0: double vectors, the matrix A) or FP32 (1:
 * float vectors, the matrix A/rho).  They use the handle's matrix format,
 * orthonormal P, stream and scratch.  Layout of the level arrays, as in the
 * solver: d_R holds r^(0..l) (l+1 columns), d_V holds V^(-1..l) with v_q^(i)
 * (q = 0..s-1) in column (i+1)*s + q; both with leading dimension ld >= n.
 * Small coefficient vectors (gamma, eta, tau) are FP64 device arrays.
 * ------------------------------------------------------------------------- */

/* y = A x (products with A; Algorithm 1, the MV steps). */
msstab_status msstab_op_spmv(msstab_t h, int32_t prec, const void* d_x, void* d_y);

/* r = b - A x and d_out[0] = ||r||^2, d_out[1] = ||b||^2 (FP64). */
msstab_status msstab_op_residual(msstab_t h, const double* d_b, const double* d_x, double* d_r,
                                 double* d_out);

/* y = A x fused with d_dots[c] = p_c . y, c = 0..s-1, and d_dots[s] = y . y
 * (the projections P^T w that the gamma and eta solves of Algorithm 1 need). */
msstab_status msstab_op_spmv_dot(msstab_t h, int32_t prec, const void* d_x, void* d_y, double* d_dots);

/* d_y = alpha d_x + beta d_z (FP64, n entries; d_y may alias d_x or d_z).  Forms
 * the implicit-Euler right-hand side b = x^(i)/tau + f of a time-stepping
 * sequence on the device. */
msstab_status msstab_op_axpby(msstab_t h, double alpha, const double* d_x, double beta, const double* d_z,
                              double* d_y);

/* Copy the orthonormal cut-space basis P out (s columns, ld = n). */
msstab_status msstab_op_get_p(msstab_t h, int32_t prec, void* d_P);

/* d_out[t * ny + c] = X_t . Y_c for t < nx, c < ny (nx, ny <= 16; columns at
 * base + index * ld). */
msstab_status msstab_op_multidot(msstab_t h, int32_t prec, const void* d_X, int64_t ldx, int32_t nx,
                                 const void* d_Y, int64_t ldy, int32_t ny, double* d_out);

/* r^(k) -= V^(k) gamma (Algorithm 1, the gamma update on the top level k). */
msstab_status msstab_op_gamma_update(msstab_t h, int32_t prec, void* d_R, const void* d_V, int64_t ld,
                                     int32_t k, const double* d_gamma);

/* v_q^(k) = r^(k+1) - [V^(k+1)_{0:q-1}, V^(k)_{q:s-1}] eta_q (Algorithm 1, the
 * eta update on level k for column q, 0-based). */
msstab_status msstab_op_eta_update(msstab_t h, int32_t prec, const void* d_R, void* d_V, int64_t ld,
                                   int32_t k, int32_t q, const double* d_eta);

/* The updates of level step k on the levels below k, applied once after the
 * q loop: x^(0) += V^(-1) gamma and r^(i) -= V^(i) gamma for i < k (with the
 * V^(i) of the start of the step), then for each level i = k-1..-1 and
 * q = 0..s-1: v_q^(i) = r^(i+1) - [V^(i+1)_{0:q-1} (new), V^(i)_{q:s-1} (old)] eta_q.
 * d_eta is s x s, row q = eta_q.  This yields the values of Algorithm 1's
 * level-by-level updates.  If d_gram is not NULL, d_gram[a*(l+1)+c] =
 * r^(a) . r^(c) (a, c = 0..l) after the updates. */
msstab_status msstab_op_lazy_update(msstab_t h, int32_t prec, void* d_R, void* d_V, void* d_x,
                                    int64_t ld, int32_t k, const double* d_gamma, const double* d_eta,
                                    double* d_gram);

/* The degree-l step of Algorithm 1 in place: r = r^(0) - sum tau_i r^(i),
 * x += sum tau_i r^(i-1), v_q = v_q^(0) - sum tau_i v_q^(i),
 * u_q = v_q^(-1) - sum tau_i v_q^(i-1) (r into r^(0), v_q into V^(0), u_q into V^(-1)). */
msstab_status msstab_op_tau_update(msstab_t h, int32_t prec, void* d_R, void* d_V, void* d_x, int64_t ld,
                                   const double* d_tau);

/* The degree-l step as a solve runs it at a cycle end (Algorithm 1, after the
 * level loop): the updates of msstab_op_tau_update when do_update != 0, then,
 * in the same pass, the projections of the new r and V^(0) that the next
 * cycle's first gamma solve uses.  d_out (FP64, s*s + s + 1 values):
 * d_out[q*s + c] = p_c . v_q^(0), d_out[s*s + c] = p_c . r^(0),
 * d_out[s*s + s] = r^(0) . r^(0), with P the handle's cut space in the
 * precision prec.  Layout of d_R, d_V, d_x as msstab_op_tau_update.
 * d_lazy_gamma, d_lazy_eta (both NULL, or gamma_0 and the s x s eta of level
 * step 0, row q = eta_q): first the updates of msstab_op_lazy_update with
 * k = 0, in the same pass -- the FP32 inner form with l = 1 does this when
 * the columns are 16-byte aligned and n % 4 == 0 (else MSSTAB_ERR_INVALID_ARG). */
msstab_status msstab_op_tau_step(msstab_t h, int32_t prec, void* d_R, void* d_V, void* d_x, int64_t ld,
                                 const double* d_tau, int32_t do_update, const double* d_lazy_gamma,
                                 const double* d_lazy_eta, double* d_out);

/* Solve the n x n system d_M z = d_rhs (d_M row-major, n <= 16) on the device by
 * Gaussian elimination with partial pivoting; *d_flag = 1 if the pivot of a
 * column fell below 1e-14 times the largest magnitude in that column of M
 * (z is then zero).  The small solves of Algorithm 1. */
msstab_status msstab_op_small_solve(msstab_t h, int32_t n, const double* d_M, const double* d_rhs,
                                    double* d_z, int32_t* d_flag);

/* tau from the (l+1) x (l+1) Gram matrix of [r^(0..l)] (row-major): the normal
 * equations of min ||r^(0) - Z tau||, diagonally scaled, by Cholesky (LU if
 * that fails); tau = 0 if a level vector is zero. */
msstab_status msstab_op_tau_solve(msstab_t h, int32_t ell, const double* d_gram, double* d_tau);

/* ILU(0) of a handle created with MSSTAB_PRECOND_ILU0 (Section 5.1's split
 * preconditioner).  The factor is stored on A's CSR pattern: entries left of
 * the diagonal are L (unit lower; its diagonal is implicit), the others U.
 * It is computed row by row by the IKJ elimination with every update outside
 * the pattern dropped, each update one rounded product and one rounded
 * difference, so it equals the sequential textbook factor bit for bit.
 * msstab_op_ilu_factor copies the nnz factor values to d_lu (CSR order).
 * msstab_op_ilu_levels copies the level of every row in the lower and upper
 * dependency graphs (the longest chain of strict lower / strict upper
 * dependencies below it; rows of one level are computed in parallel) to
 * d_lev_lower[n], d_lev_upper[n] (either may be NULL) and writes
 * h_info[0..5] = levels (lower, upper), widest level (lower, upper), blocks of
 * the solves (lower, upper: one per row chunk of the pipelined sweep, else the
 * blocks of the level-by-level sweep).
 * msstab_op_ilu_apply: which = 0: d_out = L^-1 d_in; 1: d_out = U^-1 d_in;
 * 2: d_out = U d_in; 3: d_out = L^-1 A U^-1 d_in.  d_out may equal d_in for 0,
 * 1 and 3, not for 2.  All three block until done.  INVALID_ARG without the
 * preconditioner; CUDA if a grid barrier of the sweeps timed out. */
msstab_status msstab_op_ilu_factor(msstab_t h, double* d_lu);
msstab_status msstab_op_ilu_levels(msstab_t h, int32_t* d_lev_lower, int32_t* d_lev_upper, int32_t* h_info);
msstab_status msstab_op_ilu_apply(msstab_t h, int32_t which, const double* d_in, double* d_out);

/* ---------------------------------------------------------------------------
 * Learned initial guess (not in the paper; the workload's learned-x0 form).
 * A 3D CNN -- 3x3x3 convolutions 2 -> 16 -> 16 -> 16 -> 1, zero "same"
 * padding, bias, GELU (erf form) after the first three -- maps the normalised
 * pair (b^(i+1), x^(i)), fed as the channels (r0, x^(i)) with r0 = b^(i+1) -
 * A x^(i) (FP64, from msstab_op_residual), to the normalised x^(i+1) - x^(i).
 * The residual channel carries the information of b in a form that survives
 * bfloat16: tau b and x^(i) differ by tau f (about 0.5% of x for implicit
 * Euler, below bfloat16's resolution), and A x^(i) for smooth x^(i) is a
 * cancellation of terms 1e3-1e5 times larger than the result.  Weights, biases and
 * all convolution operands are bfloat16, sums FP32, master weights and Adam
 * state FP32.  Parameters: one flat FP32 vector of msstab_cnn_num_params()
 * entries, per layer W[c_out][c_in][3][3][3] then b[c_out]; tap (dz, dy, dx)
 * multiplies the input at offset (dz-1, dy-1, dx-1).  Volumes are
 * [batch][channel][z][y][x], x fastest, like the solver's vectors.
 * ------------------------------------------------------------------------- */
typedef struct msstab_cnn_s* msstab_cnn_t;

int32_t msstab_cnn_num_params(void);

/* A network for an nx x ny x nz grid (x fastest), with initial parameters
 * d_params (FP32, copied), room for max_pairs training pairs and for training
 * batches of up to max_batch crops of edge up to crop.  stream: cudaStream_t. */
msstab_status msstab_cnn_create(int32_t nx, int32_t ny, int32_t nz, const float* d_params, int32_t max_pairs,
                                int32_t max_batch, int32_t crop, void* stream, msstab_cnn_t* out);
msstab_status msstab_cnn_destroy(msstab_cnn_t h);
const char* msstab_cnn_last_error(msstab_cnn_t h);
msstab_status msstab_cnn_get_params(msstab_cnn_t h, float* d_params);
msstab_status msstab_cnn_set_params(msstab_cnn_t h, const float* d_params);

/* Normalisation.  The map r0 -> x^(i+1) - x^(i) is linear in r0, so each
 * instance is presented at unit residual scale: network input (s_r r0, s_x
 * x^(i)) and target c s_r (x^(i+1) - x^(i)), with s_r = 1/RMS(r0) of that
 * instance (computed in every add_pair and infer), s_x and c global.
 * msstab_cnn_fit_scales sets s_x = 1/RMS(x^(i)) and c = 1/RMS(s_r delta) over
 * the stored pairs; get/set exchange (s_x, c). */
msstab_status msstab_cnn_set_scales(msstab_cnn_t h, float s_x, float c);
msstab_status msstab_cnn_get_scales(msstab_cnn_t h, float* scales2);
msstab_status msstab_cnn_fit_scales(msstab_cnn_t h);

/* Loss of training and msstab_cnn_grad.  k27 NULL (default): the mean of
 * (out - t)^2.  Else a host array of 27 coefficients K[dz+1][dy+1][dx+1]
 * (dx fastest): the mean of (K * (out - t))^2, K * e the cross-correlation
 * over each crop with zero padding.  With K a row stencil of A (any scale)
 * this weights the error of the predicted correction by the operator, i.e.
 * trains for a small residual A (x_guess - x^(i+1)) of the guess rather than
 * a small error; the stencil step runs in FP32.  Errors: INVALID_ARG for a
 * zero or non-finite stencil. */
msstab_status msstab_cnn_set_loss_stencil(msstab_cnn_t h, const double* k27);

/* Store a training pair: r0 = b^(i+1) - A x^(i) and x^(i) -> x^(i+1) - x^(i)
 * (FP64 device vectors of the grid). */
msstab_status msstab_cnn_add_pair(msstab_cnn_t h, const double* d_r0, const double* d_x_prev,
                                  const double* d_x_next);

/* iters Adam steps (lr; beta 0.9, 0.999; eps 1e-8) on the mean squared error
 * over batches of B crops of edge D cut from the stored pairs; h_origins holds
 * iters x B x 4 int32 (pair index, z0, y0, x0) per crop.  loss_history (host,
 * iters entries) may be NULL. */
msstab_status msstab_cnn_train(msstab_cnn_t h, int32_t iters, int32_t B, int32_t D, const int32_t* h_origins,
                               float lr, float* loss_history);

/* Network output for B normalised input crops d_in [B][2][D^3] (FP32; rounded
 * to bfloat16 inside) into d_out [B][D^3] (FP32). */
msstab_status msstab_cnn_forward(msstab_cnn_t h, const float* d_in, int32_t B, int32_t D, float* d_out);

/* Gradient (FP32, d_grad[num_params]) and value (*loss, host) of the mean
 * squared error of the output for d_in against d_target [B][D^3]; no update. */
msstab_status msstab_cnn_grad(msstab_cnn_t h, const float* d_in, const float* d_target, int32_t B, int32_t D,
                              float* d_grad, double* loss);

/* One Adam step with the given gradient. */
msstab_status msstab_cnn_adam_step(msstab_cnn_t h, const float* d_grad, float lr);

/* d_delta = the network's x^(i+1) - x^(i) for the whole grid from r0 = b^(i+1)
 * - A x^(i) and x^(i) (FP64 vectors; asynchronous on the handle's stream).
 * Use with msstab_select_guess / msstab_select_guess_scaled. */
msstab_status msstab_cnn_infer(msstab_cnn_t h, const double* d_r0, const double* d_x_prev, double* d_delta);

/* ---------------------------------------------------------------------------
 * Allocation-free entry point (the paper has no counterpart: it is a service
 * for callers that may not allocate device memory themselves -- for example a
 * solver embedded in a host application that owns all device memory through
 * its own pool, or a time-critical loop in which an allocation, which can
 * synchronise the device or fail at run time, is not allowed).
 *
 * y = A x for the CSR matrix (d_row_ptr[n+1], d_col[nnz], d_val[nnz], int32
 * indices, FP64 values) fused with d_dots[c] = P_c . y for c < s (P columns at
 * d_P + c*ldp, ldp >= n) and d_dots[s] = y . y -- the same kernel and results
 * as msstab_op_spmv_dot on a CSR handle, without a handle.  The caller passes
 * all inputs and outputs; the reduction scratch is a fixed device array inside
 * the library (about 160 KB, one per GPU that loads the library, held until the
 * process exits).  Limits: 1 <= n <= 2^31 - 2^22, 0 <= nnz < 2^31,
 * 0 <= s <= 16 (d_P may be NULL when s = 0); other sizes are rejected with
 * MSSTAB_ERR_INVALID_ARG and a message in msstab_last_error(NULL).  A CUDA
 * error left pending by earlier work on the calling thread makes the call
 * return MSSTAB_ERR_CUDA before it launches anything; that error is left
 * pending for its owner.  The call allocates nothing (no cudaMalloc, no
 * cudaFree, no allocating library routine); it is asynchronous on `stream`
 * (a cudaStream_t; NULL = the legacy default stream).  The first call on a
 * device looks up the device address of the scratch array (once per device,
 * with that device current); make that first call before any stream capture.
 * The address is kept for the rest of the process: it assumes that the
 * device's primary context lives until the process exits (after a
 * cudaDeviceReset the kept address is stale and the call must not be used).
 * Every call shares the one scratch array, which keeps the last call's
 * contents (the call clears what must start at zero): calls that overlap on
 * the GPU -- concurrent streams, or several host threads -- race and must be
 * serialised by the caller.
 */
msstab_status msstab_spmv_dot_noalloc(int64_t n, int64_t nnz, const int32_t* d_row_ptr, const int32_t* d_col,
                                      const double* d_val, const double* d_x, double* d_y, const double* d_P,
                                      int64_t ldp, int32_t s, double* d_dots, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* MSSTAB_H */

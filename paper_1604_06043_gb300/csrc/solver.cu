// Host driver of libmsstab: the handle, msstab_create / msstab_solve /
// msstab_destroy, the cycle loop of Algorithm 1 (IDRstab) for FP64 and for the
// FP32 inner solves, the M(s)stab recycle store (Section 4.2, fetching point of
// Section 5), the FP64 defect-correction loop and the kernel-level entry
// points.  No kernel is defined here: every step runs in the kernels of
// spmv.cu and blas.cu, launched on the handle's stream.  The host reads the
// device only at cycle ends (residual norm and error flags) and at the few
// decisions of the Arnoldi start.

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <type_traits>
#include <vector>

#include "launch.h"
#include "msstab.h"

using namespace msk;

namespace {

thread_local std::string g_create_error;

template <typename T>
struct Work {
  bool allocated = false;
  int64_t ld = 0;
  T* R = nullptr;     // r^(0..l)
  T* V = nullptr;     // V^(-1..l)
  T* X = nullptr;     // x (x^(0) during a cycle)
  T* XB = nullptr;    // x at the last completed cycle end
  T* XB2 = nullptr;   // x written by the degree-l step of the running cycle
  T* B = nullptr;     // right-hand side
  T* Tm = nullptr;    // temporary (true residual, Arnoldi)
  T* Urec = nullptr;  // recycle store
  T* Vrec = nullptr;
  T* P = nullptr;     // orthonormal cut-space basis
  T* Pil = nullptr;   // P interleaved by row (row stride sp), for the fused products
  int sp = 0;
  T* Pb = nullptr;    // block-partitioned P (one value per row), when P has that structure
  bool has_rec = false;
};

struct Timing {
  bool on = false;
  std::vector<cudaEvent_t> ev;
  std::vector<int> fam;
  int used = 0;
  double t_ms[MSSTAB_K_COUNT];
  int64_t n[MSSTAB_K_COUNT];
};

struct SolveOut {
  int64_t mvs = 0, cycles = 0;
  int64_t fetch_at = 0;     // cycle whose basis was written to the recycle store
  double relres_true = -1.0, relres_rec = 0.0;
  int fetched = 0, used_recycle = 0;
  msstab_status status = MSSTAB_OK;
};

}  // namespace

struct msstab_s {
  int n = 0;
  int64_t nnz = 0;
  int s = 0, ell = 0;
  msstab_options opt{};
  cudaStream_t stream = nullptr;
  int sms = 0;
  MatDesc A{};
  double rho = 1.0;
  std::vector<void*> allocs;
  Work<double> w64;
  Work<float> w32;
  DevState* st = nullptr;
  RedScratch rs{};
  double* h_small = nullptr;   // pinned readback buffer
  std::string err;
  std::vector<double> hist;
  std::vector<int64_t> hist_mvs;
  Timing tm;
  int64_t launches = 0;
  int64_t mvs32 = 0;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  // instantiated CUDA graphs of one cycle's launch sequence, by (precision,
  // degree, x-backup buffer, residual replacement)
  struct CycleGraph {
    int prec, ell;
    const void* xb2;
    bool replaced;
    cudaGraphExec_t exec;
    int launches;
  };
  std::vector<CycleGraph> graphs;
  cudaStream_t cap_stream = nullptr;   // private stream the cycle is captured on (replayed on `stream`)
  // ILU(0) split preconditioning: the solver's operator is L^-1 A U^-1
  int64_t probe_cycle = 0;  // FETCH_PROBE: fetching point estimated by the probe solve (0: none yet)
  double* Uprev = nullptr;   // FETCH_SLOPE: the basis at the previous cycle end
  double* Vprev = nullptr;
  bool precond = false;
  IluDesc ilu{};
  double* ilu_t = nullptr;   // U^-1 x of the running product, then L^-1 A U^-1 x
  double* ilu_z = nullptr;   // A U^-1 x
  double* borig = nullptr;   // the caller's b of the running solve
  // persistent level steps (options.persistent): one cooperative launch per level step
  bool level = false;
  unsigned int* level_bar = nullptr;   // grid-barrier counter of the level kernel
  long long spin_limit = 1LL << 22;    // polls before a device-side wait gives up

  Ctx ctx() const { return Ctx{stream, sms, rs}; }
};

namespace {

msstab_status fail(msstab_t h, msstab_status code, const std::string& what) {
  if (h)
    h->err = what;
  else
    g_create_error = what;
  return code;
}

msstab_status cuda_fail(msstab_t h, cudaError_t e, const char* where) {
  std::string m = std::string(where) + ": " + cudaGetErrorString(e);
  return fail(h, e == cudaErrorMemoryAllocation ? MSSTAB_ERR_OOM : MSSTAB_ERR_CUDA, m);
}

#define CK(call)                                              \
  do {                                                        \
    cudaError_t e_ = (call);                                  \
    if (e_ != cudaSuccess) return cuda_fail(h, e_, #call);    \
  } while (0)

#define CKS(expr)                            \
  do {                                       \
    msstab_status s_ = (expr);               \
    if (s_ != MSSTAB_OK) return s_;          \
  } while (0)

// ---------------------------------------------------------------------------
// launch accounting and optional per-family event timing
// ---------------------------------------------------------------------------
msstab_status timing_flush(msstab_t h) {
  Timing& t = h->tm;
  if (!t.on || t.used == 0) return MSSTAB_OK;
  CK(cudaEventSynchronize(t.ev[2 * (t.used - 1) + 1]));
  for (int i = 0; i < t.used; ++i) {
    float ms = 0.f;
    CK(cudaEventElapsedTime(&ms, t.ev[2 * i], t.ev[2 * i + 1]));
    t.t_ms[t.fam[i]] += ms;
    t.n[t.fam[i]] += 1;
  }
  t.used = 0;
  return MSSTAB_OK;
}

msstab_status timing_begin(msstab_t h, int fam) {
  Timing& t = h->tm;
  if (!t.on) return MSSTAB_OK;
  if (t.ev.empty()) {
    t.ev.resize(2 * 4096);
    t.fam.resize(4096);
    for (auto& e : t.ev) CK(cudaEventCreate(&e));
  }
  if (t.used == (int)t.fam.size()) CKS(timing_flush(h));
  t.fam[t.used] = fam;
  CK(cudaEventRecord(t.ev[2 * t.used], h->stream));
  return MSSTAB_OK;
}

msstab_status timing_end(msstab_t h) {
  Timing& t = h->tm;
  if (!t.on) return MSSTAB_OK;
  CK(cudaEventRecord(t.ev[2 * t.used + 1], h->stream));
  t.used += 1;
  return MSSTAB_OK;
}

#define LAUNCH(fam, expr)                                     \
  do {                                                        \
    CKS(timing_begin(h, (fam)));                              \
    cudaError_t e_ = (expr);                                  \
    if (e_ != cudaSuccess) return cuda_fail(h, e_, #expr);    \
    CKS(timing_end(h));                                       \
    h->launches += 1;                                         \
  } while (0)

msstab_status dalloc(msstab_t h, void** p, size_t bytes) {
  if (bytes == 0) bytes = 256;
  cudaError_t e = cudaMalloc(p, bytes);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return fail(h, MSSTAB_ERR_OOM, "cudaMalloc of " + std::to_string(bytes) + " bytes failed");
  }
  h->allocs.push_back(*p);
  return MSSTAB_OK;
}

int64_t round_up(int64_t v, int64_t m) { return (v + m - 1) / m * m; }

template <typename T>
msstab_status alloc_work(msstab_t h, Work<T>& w, bool levels) {
  const int s = h->s, ell = h->ell;
  w.ld = round_up(h->n, 256 / (int64_t)sizeof(T));
  const int64_t ncols = (levels ? (ell + 1) + (int64_t)s * (ell + 2) + 2 * s : 0) + 5 + s;
  void* base = nullptr;
  CKS(dalloc(h, &base, (size_t)ncols * w.ld * sizeof(T)));
  CK(cudaMemsetAsync(base, 0, (size_t)ncols * w.ld * sizeof(T), h->stream));
  T* p = (T*)base;
  auto take = [&](int64_t cols) {
    T* r = p;
    p += cols * w.ld;
    return r;
  };
  if (levels) {
    w.R = take(ell + 1);
    w.V = take((int64_t)s * (ell + 2));
    w.Urec = take(s);
    w.Vrec = take(s);
  }
  w.X = take(1);
  w.XB = take(1);
  w.XB2 = take(1);
  w.B = take(1);
  w.Tm = take(1);
  w.P = take(s);
  w.allocated = true;
  return MSSTAB_OK;
}

msstab_status sync_read(msstab_t h, const void* dsrc, size_t bytes) {
  CK(cudaMemcpyAsync(h->h_small, dsrc, bytes, cudaMemcpyDeviceToHost, h->stream));
  CK(cudaStreamSynchronize(h->stream));
  return MSSTAB_OK;
}

Epi epi_none(msstab_t h) { return Epi{EPI_NONE, 0, 0, h->s, h->ell, h->st}; }

// One product with the solver's operator: A, or with the ILU(0) split
// preconditioner L^-1 A U^-1 (upper solve, product with A, lower solve, then
// y = z or b - z with the reductions and epilogue of the fused product).  The
// arguments and the out layout are those of spmv.
template <typename T>
msstab_status amv(msstab_t h, const Ctx& c, int fam, const T* x, T* y, const T* b, const T* P, int64_t ldp,
                  int np, int self, int bdot, double* out, Epi epi, const T* Pil = nullptr, int sp = 0,
                  const T* Pb = nullptr) {
  if constexpr (std::is_same<T, double>::value) {
    if (h->precond) {
      LAUNCH(MSSTAB_K_PRECOND, ilu_upper_solve(c, h->ilu, x, h->ilu_t));
      LAUNCH(fam, spmv<double>(c, h->A, h->ilu_t, h->ilu_z, nullptr, nullptr, 0, 0, 0, 0, nullptr, epi_none(h)));
      LAUNCH(MSSTAB_K_PRECOND, ilu_lower_solve(c, h->ilu, h->ilu_z, h->ilu_t));
      LAUNCH(fam, vec_dots<double>(c, h->n, h->ilu_t, y, b, P, ldp, np, self, bdot, out, epi, Pb));
      return MSSTAB_OK;
    }
  }
  LAUNCH(fam, spmv<T>(c, h->A, x, y, b, P, ldp, np, self, bdot, out, epi, Pil, sp, Pb));
  return MSSTAB_OK;
}

// ---------------------------------------------------------------------------
// Cholesky QR (twice) of s columns V, applying the same R^-1 to U
// ---------------------------------------------------------------------------
template <typename T>
msstab_status cholqr2(msstab_t h, T* V, T* U, int64_t ld, bool* ok) {
  const Ctx c = h->ctx();
  const int s = h->s;
  DevState* st = h->st;
  CK(cudaMemsetAsync(&st->flag, 0, sizeof(int), h->stream));
  for (int pass = 0; pass < 2; ++pass) {
    MdCols<T> cols{};
    for (int q = 0; q < s; ++q) cols.x[q] = cols.y[q] = V + (int64_t)q * ld;
    LAUNCH(MSSTAB_K_OTHER, multidot<T>(c, h->n, cols, s, s, 0, st->gmat, s, epi_none(h)));
    LAUNCH(MSSTAB_K_OTHER, small_cholesky(c, s, st->gmat, st->chol, &st->flag));
    LAUNCH(MSSTAB_K_OTHER, tri_apply<T>(c, h->n, s, V, U, ld, st->chol));
  }
  int flag = 0;
  CK(cudaMemcpyAsync(h->h_small, &st->flag, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
  CK(cudaStreamSynchronize(h->stream));
  std::memcpy(&flag, h->h_small, sizeof(int));
  CK(cudaMemsetAsync(&st->flag, 0, sizeof(int), h->stream));
  *ok = (flag & FLAG_CHOL) == 0;
  return MSSTAB_OK;
}

// V_rec := A U_rec (s products with A): the recursions keep V = A U only up to
// a drift, and Algorithm 1 requires V = A U of its input basis.
template <typename T>
msstab_status refresh_v(msstab_t h, Work<T>& w, int prec, SolveOut& out) {
  const Ctx c = h->ctx();
  for (int q = 0; q < h->s; ++q)
    CKS(amv<T>(h, c, MSSTAB_K_SPMV, w.Urec + (int64_t)q * w.ld, w.Vrec + (int64_t)q * w.ld, nullptr, nullptr,
                                  0, 0, 0, 0, nullptr, epi_none(h)));
  out.mvs += h->s;
  if (prec) h->mvs32 += h->s;
  return MSSTAB_OK;
}

// ---------------------------------------------------------------------------
// Arnoldi start of level s: U = first s Arnoldi vectors of K(A; r0), V = A U
// (classical Gram-Schmidt applied twice; s products with A)
// ---------------------------------------------------------------------------
template <typename T>
msstab_status arnoldi(msstab_t h, Work<T>& w, int prec, SolveOut& out) {
  const Ctx c = h->ctx();
  const int s = h->s, n = h->n;
  const int64_t ld = w.ld;
  DevState* st = h->st;
  T* U = w.V;                        // level -1
  T* Vv = w.V + (int64_t)s * ld;     // level 0
  auto Ucol = [&](int j) { return U + (int64_t)j * ld; };
  auto Vcol = [&](int j) { return Vv + (int64_t)j * ld; };
  {
    MdCols<T> cols{};
    cols.x[0] = w.R;
    LAUNCH(MSSTAB_K_OTHER, multidot<T>(c, n, cols, 1, 0, 1, &st->scal[0], 1, epi_none(h)));
    LAUNCH(MSSTAB_K_OTHER, scale_rsqrt<T>(c, n, w.R, Ucol(0), &st->scal[0]));
  }
  for (int j = 0; j < s; ++j) {
    CKS(amv<T>(h, c, MSSTAB_K_SPMV, Ucol(j), Vcol(j), nullptr, nullptr, 0, 0, 0, 0, nullptr, epi_none(h)));
    out.mvs += 1;
    if (prec) h->mvs32 += 1;
    if (j == s - 1) break;
    CK(cudaMemcpyAsync(w.Tm, Vcol(j), sizeof(T) * n, cudaMemcpyDeviceToDevice, h->stream));
    for (int attempt = 0; attempt < 2; ++attempt) {
      for (int pass = 0; pass < 2; ++pass) {
        MdCols<T> cols{};
        cols.x[0] = w.Tm;
        for (int i = 0; i <= j; ++i) cols.y[i] = Ucol(i);
        LAUNCH(MSSTAB_K_OTHER, multidot<T>(c, n, cols, 1, j + 1, 0, &st->scal[0], SMAX, epi_none(h)));
        LAUNCH(MSSTAB_K_OTHER, cols_axpy<T>(c, n, w.Tm, U, ld, j + 1, &st->scal[0]));
      }
      MdCols<T> cols{};
      cols.x[0] = w.Tm;
      cols.x[1] = Vcol(j);
      LAUNCH(MSSTAB_K_OTHER, multidot<T>(c, n, cols, 2, 0, 1, &st->scal[SMAX], 1, epi_none(h)));
      CKS(sync_read(h, &st->scal[SMAX], 2 * sizeof(double)));
      const double tt = h->h_small[0], vv = h->h_small[1];
      if (std::sqrt(tt) > 1e-12 * std::sqrt(vv) || attempt == 1) break;
      // the Krylov space ended: continue with the next cut-space direction
      CK(cudaMemcpyAsync(w.Tm, w.P + (int64_t)(j + 1) * ld, sizeof(T) * n, cudaMemcpyDeviceToDevice, h->stream));
    }
    LAUNCH(MSSTAB_K_OTHER, scale_rsqrt<T>(c, n, w.Tm, Ucol(j + 1), &st->scal[SMAX]));
  }
  return MSSTAB_OK;
}

// ---------------------------------------------------------------------------
// Algorithm 1 on the workspace w: w.B = b, w.X = x0 on entry, x on return
// ---------------------------------------------------------------------------
struct SolveCtl {
  double tol;
  int64_t max_mvs;
  bool want_fetch;        // write the recycle store at the fetching point
  double fetch_threshold;
  int fetch_cycle;
  bool use_recycle;       // start from the recycle store if it holds data
  bool record_history;
  bool true_check;        // confirm convergence with the true residual b - A x
  int ell;                // stabilisation degree of this solve (<= the handle's l)
  bool stop_on_stagnation;  // stop when the residual has not halved in 4 cycles
  bool continue_basis;    // start from the U, V left in the level slots by the previous solve
  int replace_every;      // > 0: r := b - A x after every replace_every-th cycle
  bool fetch_slope;       // fetch the basis of the cycle before the residual drops (slope_fires)
  bool fetch_at_end;      // a converged solve that fetched nothing writes its final basis
};

// The running drop test of the slope policy at the end of cycle k (hist[0]:
// relres at the start, hist[i]: after cycle i): a decrease of log10 relres in
// cycle k of at least one decade and at least twice the mean decrease of
// cycles 1..k-1 ("shortly before the residual drops", read as a test a solver
// can apply while it runs).
bool slope_fires(const std::vector<double>& hist, int64_t k) {
  if (k < 2 || (int64_t)hist.size() <= k) return false;
  auto lg = [&](int64_t i) { return std::log10(std::max(hist[i], 1e-300)); };
  const double drop = lg(k - 1) - lg(k);
  const double mean = (lg(0) - lg(k - 1)) / (double)(k - 1);
  return drop >= 1.0 && drop >= 2.0 * mean;
}

// The fetching point estimated from a probe solve's complete history: the
// cycle end before the steepest one-cycle decrease (the first of equals), at
// least 1; 0 if the solve ran no cycle.
int64_t fetch_estimate(const std::vector<double>& hist) {
  const int64_t K = (int64_t)hist.size() - 1;
  if (K < 1) return 0;
  int64_t best = 1;
  double best_drop = -1e300;
  for (int64_t k = 1; k <= K; ++k) {
    const double d = std::log10(std::max(hist[k - 1], 1e-300)) - std::log10(std::max(hist[k], 1e-300));
    if (d > best_drop) {
      best_drop = d;
      best = k;
    }
  }
  return std::max<int64_t>(1, best - 1);
}

template <typename T>
msstab_status idrstab(msstab_t h, Work<T>& w, int prec, const SolveCtl& ctl, SolveOut& out) {
  const Ctx c = h->ctx();
  const int s = h->s, ell = ctl.ell, n = h->n;
  auto epi_of = [&](int kind, int k, int q) { return Epi{kind, k, q, s, ell, h->st}; };
  double best = 1e300;
  int64_t best_cycle = 0;
  const int64_t ld = w.ld;
  DevState* st = h->st;
  const T* P = w.P;
  auto Rk = [&](int i) { return w.R + (int64_t)i * ld; };
  auto Vq = [&](int i, int q) { return w.V + ((int64_t)(i + 1) * s + q) * ld; };

  CK(cudaMemsetAsync(&st->flag, 0, sizeof(int), h->stream));
  // r = b - A x, ||r||^2, ||b||^2
  CKS(amv<T>(h, c, MSSTAB_K_SPMV, w.X, Rk(0), w.B, nullptr, 0, 0, 1, 1, &st->rr, epi_none(h)));
  out.mvs += 1;
  if (prec) h->mvs32 += 1;
  CK(cudaMemcpyAsync(w.XB, w.X, sizeof(T) * n, cudaMemcpyDeviceToDevice, h->stream));
  CKS(sync_read(h, &st->rr, 2 * sizeof(double)));
  double rr = h->h_small[0];
  const double nb = std::sqrt(h->h_small[1]);
  if (ctl.record_history) {
    h->hist.clear();
    h->hist_mvs.clear();
  }
  if (nb == 0.0) {
    CK(cudaMemsetAsync(w.X, 0, sizeof(T) * n, h->stream));
    out.relres_true = 0.0;
    out.relres_rec = 0.0;
    out.mvs = 0;
    if (prec) h->mvs32 -= 1;
    return MSSTAB_OK;
  }
  if (ctl.record_history) {
    h->hist.push_back(std::sqrt(rr) / nb);
    h->hist_mvs.push_back(out.mvs);
  }
  std::vector<double> hrel{std::sqrt(rr) / nb};   // relres at the start and at every cycle end
  bool have_prev = false;
  // write U, V (V := A U and Cholesky QR when orth_recycle) to the recycle store
  auto do_fetch = [&](const T* srcU, const T* srcV, int64_t at) -> msstab_status {
    CK(cudaMemcpyAsync(w.Urec, srcU, sizeof(T) * ld * s, cudaMemcpyDeviceToDevice, h->stream));
    bool ok = true;
    if (h->opt.orth_recycle) {
      CKS(refresh_v<T>(h, w, prec, out));
      CKS(cholqr2<T>(h, w.Vrec, w.Urec, ld, &ok));
    } else {
      CK(cudaMemcpyAsync(w.Vrec, srcV, sizeof(T) * ld * s, cudaMemcpyDeviceToDevice, h->stream));
    }
    if (ok) {
      w.has_rec = true;
      out.fetched = 1;
      out.fetch_at = at;
    }
    return MSSTAB_OK;
  };
  bool r_is_true = true, have_basis = ctl.continue_basis, need_proj = true;
  const int64_t cyc_mvs = (int64_t)ell * (s + 1);
  for (;;) {
    const double nr = std::sqrt(rr);
    if (!std::isfinite(nr)) {
      out.status = MSSTAB_ERR_NAN;
      CK(cudaMemcpyAsync(w.X, w.XB, sizeof(T) * n, cudaMemcpyDeviceToDevice, h->stream));
      break;
    }
    if (nr <= ctl.tol * nb) {
      if (r_is_true || !ctl.true_check) {
        if (r_is_true) out.relres_true = nr / nb;
        break;
      }
      CKS(amv<T>(h, c, MSSTAB_K_SPMV, w.X, w.Tm, w.B, nullptr, 0, 0, 1, 0, &st->scal[0], epi_none(h)));
      out.mvs += 1;
      if (prec) h->mvs32 += 1;
      CKS(sync_read(h, &st->scal[0], sizeof(double)));
      const double rt = std::sqrt(h->h_small[0]);
      if (rt <= ctl.tol * nb) {
        out.relres_true = rt / nb;
        break;
      }
      // residual replacement: continue from the true residual
      CK(cudaMemcpyAsync(Rk(0), w.Tm, sizeof(T) * n, cudaMemcpyDeviceToDevice, h->stream));
      rr = h->h_small[0];
      r_is_true = true;
      need_proj = true;
      continue;
    }
    if (!have_basis) {
      if (ctl.use_recycle && w.has_rec) {
        CK(cudaMemcpyAsync(Vq(-1, 0), w.Urec, sizeof(T) * ld * s, cudaMemcpyDeviceToDevice, h->stream));
        CK(cudaMemcpyAsync(Vq(0, 0), w.Vrec, sizeof(T) * ld * s, cudaMemcpyDeviceToDevice, h->stream));
        out.used_recycle = 1;
      } else {
        if (out.mvs + s > ctl.max_mvs) {
          out.status = MSSTAB_ERR_MAXIT;
          break;
        }
        CKS(arnoldi<T>(h, w, prec, out));
      }
      have_basis = true;
      need_proj = true;
    }
    if (out.mvs + cyc_mvs > ctl.max_mvs) {
      out.status = MSSTAB_ERR_MAXIT;
      break;
    }
    if (need_proj) {
      LAUNCH(MSSTAB_K_TAU, tau_update<T>(c, n, s, ell, w.R, w.V, w.X, nullptr, ld, nullptr, P, ld, 0, 1, st,
                                         epi_of(EPI_GAMMA, 0, 0), w.Pb, w.Pil, w.sp));
      need_proj = false;
    }
    // ---- one cycle: level steps k = 0..l-1, the degree-l step, and the
    // residual replacement; the same launch sequence every cycle ----
    const bool replaced = ctl.replace_every > 0 && (out.cycles + 1) % ctl.replace_every == 0;
    // the FP32 degree-1 step takes the level -1 updates of level step 0 in its own pass
    // (same results bit for bit, one pass over V^(-1), V^(0), r^(0) and x instead of two)
    const bool fuse_lazy = ell == 1 && tau_fuses_lazy<T>(n, s, ell, w.R, w.V, w.X, w.XB2, ld, P, ld, w.Pb);
    auto launch_cycle = [&](const Ctx& c) -> msstab_status {
      for (int k = 0; k < ell; ++k) {
        if (h->level && (prec == 0 || h->opt.persistent >= 2)) {
          // the gamma step, the s + 1 products and the eta steps of level k in one launch
          LAUNCH(MSSTAB_K_LEVEL, level_step<T>(c, h->A, w.R, w.V, ld, s, k, k + 1 < ell ? 1 : 0, P, ld, w.Pil,
                                               w.sp, w.Pb, st, h->level_bar, h->spin_limit));
          if (!fuse_lazy)
            LAUNCH(MSSTAB_K_LAZY, lazy_update<T>(c, n, s, w.R, w.V, w.X, ld, k, &st->gamma[k * SMAX],
                                                   &st->eta[k * SMAX * SMAX], SMAX));
          continue;
        }
        LAUNCH(MSSTAB_K_GAMMA, gamma_eager<T>(c, n, s, w.R, w.V, ld, k, &st->gamma[k * SMAX]));
        CKS(amv<T>(h, c, MSSTAB_K_SPMV_DOT, Rk(k), Rk(k + 1), nullptr, P, ld, s, 0, 0,
                                          &st->projR[(k + 1) * SMAX], epi_of(EPI_ETA, k, 0), w.Pil, w.sp, w.Pb));
        for (int q = 0; q < s; ++q) {
          LAUNCH(MSSTAB_K_ETA, eta_eager<T>(c, n, s, w.R, w.V, ld, k, q, &st->eta[(k * SMAX + q) * SMAX]));
          Epi next = q + 1 < s ? epi_of(EPI_ETA, k, q + 1)
                               : (k + 1 < ell ? epi_of(EPI_GAMMA, k + 1, 0) : epi_none(h));
          CKS(amv<T>(h, c, MSSTAB_K_SPMV_DOT, Vq(k, q), Vq(k + 1, q), nullptr, P, ld, s, 0, 0,
                                            &st->projV[((k + 1) * SMAX + q) * SMAX], next, w.Pil, w.sp, w.Pb));
        }
        if (!fuse_lazy)
          LAUNCH(MSSTAB_K_LAZY, lazy_update<T>(c, n, s, w.R, w.V, w.X, ld, k, &st->gamma[k * SMAX],
                                                 &st->eta[k * SMAX * SMAX], SMAX));
      }
      // degree-l minimisation
      {
        MdCols<T> cols{};
        for (int i = 0; i <= ell; ++i) cols.x[i] = cols.y[i] = Rk(i);
        LAUNCH(MSSTAB_K_TAU, multidot<T>(c, n, cols, ell + 1, ell + 1, 0, st->gram, ell + 1,
                                         epi_of(EPI_TAU, 0, 0)));
      }
      // with the replacement that follows, r^(0), P^T r, r.r and gamma_0 of this step
      // would be overwritten: the FP64 step updates x and V only
      const bool xonly = replaced && sizeof(T) == 8;
      LAUNCH(MSSTAB_K_TAU, tau_update<T>(c, n, s, ell, w.R, w.V, w.X, w.XB2, ld, nullptr, P, ld, 1, 1, st,
                                         xonly ? epi_none(h) : epi_of(EPI_GAMMA, 0, 0), w.Pb, w.Pil, w.sp,
                                         fuse_lazy ? &st->gamma[0] : nullptr, fuse_lazy ? &st->eta[0] : nullptr,
                                         SMAX, xonly ? 1 : 0));
      // residual replacement at the cycle end: r = b - A x with P^T r and ||r||^2 in the same pass
      // (out[c] = P_c . r at projR level 0, out[s] = r . r), then gamma of the next cycle's first
      // level step from P^T V (left by tau_update) in the epilogue
      if (replaced)
        CKS(amv<T>(h, c, MSSTAB_K_SPMV_DOT, w.X, Rk(0), w.B, P, ld, s, 1, 0, &st->projR[0],
                                          epi_of(EPI_GAMMA, 0, 0), w.Pil, w.sp, w.Pb));
      return MSSTAB_OK;
    };
    if (h->tm.on || h->precond) {
      // per-launch event timing, or the cooperative ILU(0) sweeps: plain launches
      CKS(launch_cycle(c));
    } else {
      // replay the captured launch sequence (captured on first use)
      msstab_s::CycleGraph* g = nullptr;
      for (auto& e : h->graphs)
        if (e.prec == prec && e.ell == ell && e.xb2 == (const void*)w.XB2 && e.replaced == replaced) g = &e;
      if (!g) {
        const int64_t l0 = h->launches;
        if (!h->cap_stream) CK(cudaStreamCreateWithFlags(&h->cap_stream, cudaStreamNonBlocking));
        Ctx cc = c;
        cc.stream = h->cap_stream;
        cudaGraph_t graph = nullptr;
        CK(cudaStreamBeginCapture(h->cap_stream, cudaStreamCaptureModeThreadLocal));
        const msstab_status cs = launch_cycle(cc);
        const cudaError_t ce = cudaStreamEndCapture(h->cap_stream, &graph);
        if (cs != MSSTAB_OK) {
          if (graph) cudaGraphDestroy(graph);
          return cs;
        }
        if (ce != cudaSuccess) return cuda_fail(h, ce, "cudaStreamEndCapture");
        cudaGraphExec_t exec = nullptr;
        const cudaError_t ie = cudaGraphInstantiate(&exec, graph, 0);
        cudaGraphDestroy(graph);
        if (ie != cudaSuccess) return cuda_fail(h, ie, "cudaGraphInstantiate");
        h->graphs.push_back({prec, ell, (const void*)w.XB2, replaced, exec, (int)(h->launches - l0)});
        h->launches = l0;
        g = &h->graphs.back();
      }
      CK(cudaGraphLaunch(g->exec, h->stream));
      h->launches += g->launches;
    }
    out.mvs += cyc_mvs + (replaced ? 1 : 0);
    if (prec) h->mvs32 += cyc_mvs + (replaced ? 1 : 0);
    out.cycles += 1;
    // ---- cycle end: the one host synchronisation ----
    CK(cudaMemcpyAsync(h->h_small, replaced ? &st->projR[s] : &st->rr, sizeof(double), cudaMemcpyDeviceToHost,
                       h->stream));
    CK(cudaMemcpyAsync(h->h_small + 1, &st->flag, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
    CK(cudaStreamSynchronize(h->stream));
    CKS(timing_flush(h));
    rr = h->h_small[0];
    int flag = 0;
    std::memcpy(&flag, h->h_small + 1, sizeof(int));
    if (flag & FLAG_SYNC_TIMEOUT) {
      if (h->precond) CK(cudaMemsetAsync(h->ilu.bar, 0, sizeof(GridBar), h->stream));
      CK(cudaMemsetAsync(&st->flag, 0, sizeof(int), h->stream));
      CK(cudaStreamSynchronize(h->stream));
      return fail(h, MSSTAB_ERR_CUDA,
                  h->precond ? "a device-side wait of the ILU(0) sweeps timed out"
                             : "a grid barrier of the persistent level step timed out");
    }
    if (flag & FLAG_BREAKDOWN) {
      out.status = MSSTAB_ERR_BREAKDOWN;
      CK(cudaMemcpyAsync(w.X, w.XB, sizeof(T) * n, cudaMemcpyDeviceToDevice, h->stream));
      break;
    }
    const double relres = std::sqrt(rr) / nb;
    if (ctl.record_history) {
      h->hist.push_back(relres);
      h->hist_mvs.push_back(out.mvs);
    }
    if (!std::isfinite(relres)) continue;  // handled (restore) at the top
    hrel.push_back(relres);
    std::swap(w.XB, w.XB2);
    r_is_true = replaced;
    out.relres_rec = relres;
    if (ctl.stop_on_stagnation) {
      if (relres < 0.5 * best) {
        best = relres;
        best_cycle = out.cycles;
      } else if (out.cycles - best_cycle >= 4) {
        break;  // the FP32 floor is reached: the outer FP64 loop takes over
      }
    }
    if (ctl.want_fetch && !out.fetched && ctl.fetch_slope) {
      if constexpr (std::is_same<T, double>::value) {
        if (have_prev && slope_fires(hrel, out.cycles)) {
          CKS(do_fetch(h->Uprev, h->Vprev, out.cycles - 1));
        } else {
          CK(cudaMemcpyAsync(h->Uprev, Vq(-1, 0), sizeof(T) * ld * s, cudaMemcpyDeviceToDevice, h->stream));
          CK(cudaMemcpyAsync(h->Vprev, Vq(0, 0), sizeof(T) * ld * s, cudaMemcpyDeviceToDevice, h->stream));
          have_prev = true;
        }
      }
    } else if (ctl.want_fetch && !out.fetched &&
               ((ctl.fetch_cycle > 0 && out.cycles == ctl.fetch_cycle) ||
                (ctl.fetch_cycle <= 0 && relres <= ctl.fetch_threshold))) {
      CKS(do_fetch(Vq(-1, 0), Vq(0, 0), out.cycles));
    }
  }
  if (ctl.want_fetch && ctl.fetch_at_end && !out.fetched && out.status == MSSTAB_OK && out.cycles > 0)
    CKS(do_fetch(Vq(-1, 0), Vq(0, 0), out.cycles));
  if (out.relres_rec == 0.0) out.relres_rec = std::sqrt(rr) / nb;
  if (ctl.true_check && (out.status != MSSTAB_OK || out.relres_true < 0.0)) {
    CKS(amv<T>(h, c, MSSTAB_K_SPMV, w.X, w.Tm, w.B, nullptr, 0, 0, 1, 0, &st->scal[0], epi_none(h)));
    CKS(sync_read(h, &st->scal[0], sizeof(double)));
    out.relres_true = std::sqrt(h->h_small[0]) / nb;
  }
  return MSSTAB_OK;
}

int64_t default_max_mvs(msstab_t h) {
  if (h->opt.max_mvs > 0) return h->opt.max_mvs;
  int64_t m = (int64_t)(20.0 * std::sqrt((double)h->n)) + 1 + h->s + 2LL * h->ell * (h->s + 1);
  return std::min<int64_t>(m, 100000);
}

// After a successful solve with policy EVERY, the final U, V become the store.
template <typename T>
msstab_status chain_recycle(msstab_t h, Work<T>& w, int prec, SolveOut& o) {
  if (h->opt.fetch_policy != MSSTAB_FETCH_EVERY || o.status != MSSTAB_OK || o.cycles == 0) return MSSTAB_OK;
  const int64_t ld = w.ld;
  const int s = h->s;
  CK(cudaMemcpyAsync(w.Urec, w.V, sizeof(T) * ld * s, cudaMemcpyDeviceToDevice, h->stream));
  bool ok = true;
  if (h->opt.orth_recycle) {
    CKS(refresh_v<T>(h, w, prec, o));
    CKS(cholqr2<T>(h, w.Vrec, w.Urec, ld, &ok));
  } else {
    CK(cudaMemcpyAsync(w.Vrec, w.V + (int64_t)s * ld, sizeof(T) * ld * s, cudaMemcpyDeviceToDevice, h->stream));
  }
  w.has_rec = ok;
  return MSSTAB_OK;
}

SolveCtl make_ctl(msstab_t h, double tol, bool first_has_rec) {
  SolveCtl ctl{};
  ctl.tol = tol;
  ctl.max_mvs = default_max_mvs(h);
  const int pol = h->opt.fetch_policy;
  ctl.use_recycle = pol != MSSTAB_FETCH_NEVER;
  ctl.want_fetch = (pol == MSSTAB_FETCH_ONCE || pol == MSSTAB_FETCH_SLOPE) && !first_has_rec;
  ctl.fetch_slope = pol == MSSTAB_FETCH_SLOPE;
  ctl.fetch_at_end = pol == MSSTAB_FETCH_SLOPE;
  if (pol == MSSTAB_FETCH_PROBE && !first_has_rec && h->probe_cycle > 0) {
    // the solve after the probe fetches at the estimated cycle
    ctl.want_fetch = true;
    ctl.fetch_at_end = true;
  }
  ctl.fetch_threshold = h->opt.fetch_threshold > 0 ? h->opt.fetch_threshold : std::sqrt(tol);
  ctl.fetch_cycle = pol == MSSTAB_FETCH_PROBE ? (int)h->probe_cycle : h->opt.fetch_cycle;
  ctl.record_history = true;
  ctl.true_check = true;
  ctl.ell = h->ell;
  ctl.stop_on_stagnation = false;
  ctl.continue_basis = false;
  ctl.replace_every = h->opt.replace_every > 0 ? h->opt.replace_every : 0;
  return ctl;
}

// FP64 solve on w64 (b and x0 already staged in w64.B / w64.X).
msstab_status solve_fp64(msstab_t h, double tol, SolveOut& o) {
  SolveCtl ctl = make_ctl(h, tol, h->w64.has_rec);
  const bool probe = h->opt.fetch_policy == MSSTAB_FETCH_PROBE && !h->w64.has_rec && h->probe_cycle <= 0;
  CKS(idrstab<double>(h, h->w64, 0, ctl, o));
  if (probe && o.status == MSSTAB_OK) h->probe_cycle = fetch_estimate(h->hist);
  CKS(chain_recycle<double>(h, h->w64, 0, o));
  return MSSTAB_OK;
}

// FP32 inner M(s)stab on A/rho inside an FP64 defect-correction loop.
msstab_status solve_dc(msstab_t h, double tol, SolveOut& o, int64_t* outer_out, int* fp64_finish) {
  const Ctx c = h->ctx();
  const int n = h->n;
  DevState* st = h->st;
  Work<double>& w = h->w64;
  Work<float>& v = h->w32;
  std::vector<double> hist;
  std::vector<int64_t> hmv;
  const int max_outer = h->opt.max_outer > 0 ? h->opt.max_outer : 20;
  int64_t outer = 0;
  double nb = -1.0;
  bool cont = false;   // continue the inner basis (U, V) of the previous outer iteration
  double prev = 0.0;   // FP64 relres before the last correction
  bool corrected = false, restored = false, need_fp64 = false;
  int rejected = 0;
  o.status = MSSTAB_OK;
  for (;;) {
    // FP64 true residual
    LAUNCH(MSSTAB_K_SPMV, spmv<double>(c, h->A, w.X, w.Tm, w.B, nullptr, 0, 0, 1, 1, &st->rr, epi_none(h)));
    o.mvs += 1;
    CKS(sync_read(h, &st->rr, 2 * sizeof(double)));
    const double rr = h->h_small[0];
    if (nb < 0) nb = std::sqrt(h->h_small[1]);
    if (nb == 0.0) {
      CK(cudaMemsetAsync(w.X, 0, sizeof(double) * n, h->stream));
      o.relres_true = 0.0;
      break;
    }
    const double sigma = std::sqrt(rr);
    const double relres = sigma / nb;
    hist.push_back(relres);
    hmv.push_back(o.mvs);
    if (corrected && !restored && !(relres < prev)) {
      // the last correction did not reduce the FP64 residual (an FP32 inner
      // solve that stagnated or diverged): undo it, and restart the inner
      // basis; a second failure in a row ends the solve
      CK(cudaMemcpyAsync(w.X, w.XB2, sizeof(double) * n, cudaMemcpyDeviceToDevice, h->stream));
      cont = false;
      restored = true;
      if (++rejected >= 2) {
        need_fp64 = true;
        break;
      }
      continue;   // the residual of the restored x (one more product)
    }
    if (!restored) rejected = 0;
    restored = false;
    o.relres_true = relres;
    o.relres_rec = relres;
    if (!std::isfinite(relres)) {
      o.status = MSSTAB_ERR_NAN;
      break;
    }
    if (relres <= tol) break;
    if (outer >= max_outer) {
      need_fp64 = true;
      break;
    }
    // inner system (A/rho) d' = r/sigma in FP32; then x += (sigma/rho) d'
    LAUNCH(MSSTAB_K_OTHER, to_f32_scaled(c, n, w.Tm, v.B, 1.0 / sigma));
    CK(cudaMemsetAsync(v.X, 0, sizeof(float) * n, h->stream));
    // the FP32 true residual cannot go much below kappa * eps_32, so the inner
    // solves stop on their recursive residual; the FP64 loop checks the truth
    const double itol = h->opt.inner_tol > 0 ? h->opt.inner_tol : std::max(1e-2, 0.5 * tol * nb / sigma);
    SolveCtl ctl{};
    ctl.tol = itol;
    ctl.max_mvs = default_max_mvs(h);
    ctl.use_recycle = h->opt.fetch_policy != MSSTAB_FETCH_NEVER;
    ctl.want_fetch = h->opt.fetch_policy == MSSTAB_FETCH_ONCE && !v.has_rec;
    ctl.fetch_threshold = h->opt.fetch_threshold > 0 ? h->opt.fetch_threshold : std::sqrt(itol);
    ctl.fetch_cycle = h->opt.fetch_cycle;
    ctl.record_history = false;
    ctl.true_check = false;
    ctl.ell = std::min(h->ell, h->opt.inner_ell > 0 ? h->opt.inner_ell : 1);
    ctl.stop_on_stagnation = true;
    ctl.continue_basis = cont;
    SolveOut io;
    CKS(idrstab<float>(h, v, 1, ctl, io));
    // the next outer iteration hands this solve's final U, V on (as M(s)stab
    // does between systems) instead of restarting from the recycle store
    cont = (io.status == MSSTAB_OK || io.status == MSSTAB_ERR_MAXIT) && io.cycles > 0;
    CKS(chain_recycle<float>(h, v, 1, io));
    o.mvs += io.mvs;
    o.cycles += io.cycles;
    o.fetched |= io.fetched;
    o.used_recycle |= io.used_recycle;
    if (io.status == MSSTAB_ERR_NAN) {   // x is untouched: finish in FP64
      need_fp64 = true;
      break;
    }
    CK(cudaMemcpyAsync(w.XB2, w.X, sizeof(double) * n, cudaMemcpyDeviceToDevice, h->stream));
    LAUNCH(MSSTAB_K_OTHER, axpy_f32_into_f64(c, n, v.X, w.X, sigma / h->rho));
    prev = relres;
    corrected = true;
    outer += 1;
  }
  if (need_fp64) {
    // the FP32 corrections stopped reducing the FP64 residual (or the outer
    // budget is spent): FP64 IDR(s)stab(l) from the current x to tol
    SolveCtl c64 = make_ctl(h, tol, true);
    c64.use_recycle = false;
    c64.want_fetch = false;
    c64.record_history = false;
    SolveOut o64;
    CKS(idrstab<double>(h, h->w64, 0, c64, o64));
    o.mvs += o64.mvs;
    o.cycles += o64.cycles;
    o.status = o64.status;
    o.relres_true = o64.relres_true;
    o.relres_rec = o64.relres_rec;
    hist.push_back(o64.relres_true);
    hmv.push_back(o.mvs);
    *fp64_finish = 1;
  }
  h->hist = hist;
  h->hist_mvs = hmv;
  *outer_out = outer;
  return MSSTAB_OK;
}

msstab_status check_handle(msstab_t h) {
  if (!h) return fail(nullptr, MSSTAB_ERR_INVALID_ARG, "NULL handle");
  return MSSTAB_OK;
}

msstab_status check_ptr(msstab_t h, const void* p, const char* name, int align = 8) {
  if (!p) return fail(h, MSSTAB_ERR_INVALID_ARG, std::string(name) + " is NULL");
  if (((uintptr_t)p) % (uintptr_t)align)
    return fail(h, MSSTAB_ERR_INVALID_ARG, std::string(name) + " is not aligned to its element size");
  return MSSTAB_OK;
}

msstab_status solve_common(msstab_t h, double tol, msstab_stats* st) {
  if (!(tol > 0.0) || !std::isfinite(tol)) return fail(h, MSSTAB_ERR_INVALID_ARG, "tol must be positive");
  SolveOut o;
  int64_t outer = 0;
  const int64_t l0 = h->launches, m320 = h->mvs32;
  for (int f = 0; f < MSSTAB_K_COUNT; ++f) {
    h->tm.t_ms[f] = 0.0;
    h->tm.n[f] = 0;
  }
  h->tm.on = h->opt.kernel_timing != 0;
  CK(cudaEventRecord(h->e0, h->stream));
  msstab_status rc;
  int fp64_finish = 0;
  const Ctx c = h->ctx();
  Work<double>& w = h->w64;
  const size_t bytes = sizeof(double) * h->n;
  if (h->precond) {
    // the split-preconditioned system: b~ = L^-1 b, x~0 = U x0
    CK(cudaMemcpyAsync(h->borig, w.B, bytes, cudaMemcpyDeviceToDevice, h->stream));
    LAUNCH(MSSTAB_K_PRECOND, ilu_lower_solve(c, h->ilu, w.B, w.B));
    LAUNCH(MSSTAB_K_PRECOND, ilu_upper_mul(c, h->ilu, w.X, h->ilu_t));
    CK(cudaMemcpyAsync(w.X, h->ilu_t, bytes, cudaMemcpyDeviceToDevice, h->stream));
  }
  if (h->opt.precision == MSSTAB_PREC_FP32_INNER)
    rc = solve_dc(h, tol, o, &outer, &fp64_finish);
  else
    rc = solve_fp64(h, tol, o);
  if (rc != MSSTAB_OK) return rc;
  double relres_orig = o.relres_true;
  if (h->precond) {
    // x = U^-1 x~, and the residual of the original system
    LAUNCH(MSSTAB_K_PRECOND, ilu_upper_solve(c, h->ilu, w.X, w.X));
    LAUNCH(MSSTAB_K_SPMV, spmv<double>(c, h->A, w.X, w.Tm, h->borig, nullptr, 0, 0, 1, 1, &h->st->scal[0],
                                       epi_none(h)));
    CK(cudaMemcpyAsync(h->h_small, &h->st->scal[0], 2 * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
    CK(cudaMemcpyAsync(h->h_small + 2, &h->st->flag, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
    CK(cudaStreamSynchronize(h->stream));
    int flag = 0;
    std::memcpy(&flag, h->h_small + 2, sizeof(int));
    if (flag & FLAG_SYNC_TIMEOUT) {
      CK(cudaMemsetAsync(h->ilu.bar, 0, sizeof(GridBar), h->stream));
      CK(cudaMemsetAsync(&h->st->flag, 0, sizeof(int), h->stream));
      return fail(h, MSSTAB_ERR_CUDA, "a grid barrier of the ILU(0) level sweeps timed out");
    }
    relres_orig = h->h_small[1] > 0.0 ? std::sqrt(h->h_small[0] / h->h_small[1]) : 0.0;
  }
  CK(cudaEventRecord(h->e1, h->stream));
  CK(cudaEventSynchronize(h->e1));
  CKS(timing_flush(h));
  float ms = 0.f;
  CK(cudaEventElapsedTime(&ms, h->e0, h->e1));
  if (st) {
    std::memset(st, 0, sizeof(*st));
    st->mvs = o.mvs;
    st->mvs_fp32 = h->mvs32 - m320;
    st->cycles = o.cycles;
    st->outer = outer;
    st->fp64_finish = fp64_finish;
    st->launches = h->launches - l0;
    st->relres_true = o.relres_true;
    st->relres_rec = o.relres_rec;
    st->relres_orig = relres_orig;
    st->ms = ms;
    st->status = o.status;
    st->fetched = o.fetched;
    st->fetch_at = (int32_t)o.fetch_at;
    st->used_recycle = o.used_recycle;
    for (int f = 0; f < MSSTAB_K_COUNT; ++f) {
      st->t_ms[f] = h->tm.t_ms[f];
      st->n_launch[f] = h->tm.n[f];
    }
  }
  if (o.status != MSSTAB_OK) {
    const char* what = o.status == MSSTAB_ERR_MAXIT ? "maximum number of products with A reached"
                       : o.status == MSSTAB_ERR_NAN ? "residual is not finite"
                                                    : "projected s x s system is singular (breakdown)";
    fail(h, o.status, what);
  }
  return o.status;
}

}  // namespace

void msk::set_global_error(const std::string& what) { g_create_error = what; }

// ===========================================================================
// C ABI
// ===========================================================================
extern "C" {

void msstab_default_options(msstab_options* opt) {
  if (!opt) return;
  std::memset(opt, 0, sizeof(*opt));
  opt->precision = MSSTAB_PREC_FP64;
  opt->fetch_policy = MSSTAB_FETCH_ONCE;
  opt->fetch_threshold = 0.0;
  opt->fetch_cycle = 0;
  opt->orth_recycle = 1;
  opt->max_mvs = 0;
  opt->inner_tol = 0.0;
  opt->spmv_format = MSSTAB_FORMAT_SELL;
  opt->sell_sigma = 1;
  opt->kernel_timing = 0;
  opt->max_outer = 0;
  opt->inner_ell = 0;
  opt->replace_every = 0;
  opt->persistent = 1;
  opt->stream = nullptr;
  opt->spin_limit = 0;
}

const char* msstab_last_error(msstab_t h) { return h ? h->err.c_str() : g_create_error.c_str(); }

msstab_status msstab_destroy(msstab_t h) {
  if (!h) return MSSTAB_OK;
  cudaStreamSynchronize(h->stream);
  for (void* p : h->allocs) cudaFree(p);
  for (auto& e : h->tm.ev) cudaEventDestroy(e);
  if (h->e0) cudaEventDestroy(h->e0);
  if (h->e1) cudaEventDestroy(h->e1);
  if (h->h_small) cudaFreeHost(h->h_small);
  for (auto& g : h->graphs) cudaGraphExecDestroy(g.exec);
  if (h->cap_stream) cudaStreamDestroy(h->cap_stream);
  delete h;
  return MSSTAB_OK;
}

static void* ilu_alloc(void* ctx, size_t bytes) {
  void* p = nullptr;
  return dalloc((msstab_t)ctx, &p, bytes) == MSSTAB_OK ? p : nullptr;
}

// The ILU(0) factor of A on the device, with its level schedules.
static msstab_status ilu_create(msstab_t h, int64_t n, int64_t nnz, const int32_t* d_row_ptr,
                                const int32_t* d_col, const double* d_val) {
  IluDesc& F = h->ilu;
  F.n = (int)n;
  void* p = nullptr;
  if (h->A.format == 1) {
    F.row_ptr = h->A.row_ptr;
    F.col = h->A.col;
  } else {
    CKS(dalloc(h, &p, sizeof(int) * (n + 1)));
    CK(cudaMemcpyAsync(p, d_row_ptr, sizeof(int) * (n + 1), cudaMemcpyDeviceToDevice, h->stream));
    F.row_ptr = (const int*)p;
    CKS(dalloc(h, &p, sizeof(int) * nnz));
    CK(cudaMemcpyAsync(p, d_col, sizeof(int) * nnz, cudaMemcpyDeviceToDevice, h->stream));
    F.col = (const int*)p;
  }
  CKS(dalloc(h, &p, sizeof(double) * nnz));
  F.lu = (double*)p;
  CK(cudaMemcpyAsync(p, d_val, sizeof(double) * nnz, cudaMemcpyDeviceToDevice, h->stream));
  CKS(dalloc(h, &p, sizeof(GridBar)));
  F.bar = (GridBar*)p;
  F.flag = &h->st->flag;
  F.spin_limit = h->spin_limit;
  CK(cudaMemsetAsync(F.flag, 0, sizeof(int), h->stream));
  const IluSetupResult r = ilu_setup(h->ctx(), F, ilu_alloc, h, (int*)h->h_small);
  if (r.code == 4) return MSSTAB_ERR_OOM;   // dalloc wrote the message
  if (r.code == 1) return cuda_fail(h, r.cuda, r.where ? r.where : "ILU(0) set-up");
  if (r.code == 2) return fail(h, MSSTAB_ERR_INVALID_ARG, r.where);
  if (r.code == 3) return fail(h, MSSTAB_ERR_BREAKDOWN, r.where);
  CK(cudaMemsetAsync(F.flag, 0, sizeof(int), h->stream));
  for (double** v : {&h->ilu_t, &h->ilu_z, &h->borig}) {
    CKS(dalloc(h, &p, sizeof(double) * n));
    *v = (double*)p;
  }
  return MSSTAB_OK;
}

static msstab_status create_impl(msstab_t h, int64_t n, int64_t nnz, const int32_t* d_row_ptr,
                                 const int32_t* d_col, const double* d_val, const double* d_p_raw) {
  {
    int dev = 0;
    CK(cudaGetDevice(&dev));
    CK(cudaDeviceGetAttribute(&h->sms, cudaDevAttrMultiProcessorCount, dev));
  }
  CK(cudaEventCreate(&h->e0));
  CK(cudaEventCreate(&h->e1));
  CK(cudaMallocHost((void**)&h->h_small, 64 * sizeof(double)));
  // device state and reduction scratch
  void* p = nullptr;
  CKS(dalloc(h, &p, sizeof(DevState)));
  h->st = (DevState*)p;
  CK(cudaMemsetAsync(h->st, 0, sizeof(DevState), h->stream));
  CKS(dalloc(h, &p, sizeof(double) * (size_t)MAXGRP * MAXBLK * MAXRED));
  h->rs.partials = (double*)p;
  CKS(dalloc(h, &p, sizeof(double) * (size_t)MAXGRP * MAXRED));
  h->rs.group_out = (double*)p;
  CKS(dalloc(h, &p, sizeof(unsigned) * (MAXGRP + 1)));
  h->rs.tickets = (unsigned*)p;
  CKS(dalloc(h, &p, 256));
  h->level_bar = (unsigned int*)p;
  CK(cudaMemsetAsync(h->level_bar, 0, 256, h->stream));
  h->spin_limit = h->opt.spin_limit > 0 ? (long long)h->opt.spin_limit : (1LL << 22);
  CK(cudaMemsetAsync(h->rs.tickets, 0, sizeof(unsigned) * (MAXGRP + 1), h->stream));
  h->rs.max_blocks = MAXBLK;
  const Ctx c = h->ctx();

  // validate the CSR structure on the device
  int* dflag = &h->st->flag;
  LAUNCH(MSSTAB_K_OTHER, csr_validate(c, (int)n, nnz, d_row_ptr, d_col, dflag));
  {
    int f = 0;
    CK(cudaMemcpyAsync(h->h_small, dflag, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
    CK(cudaStreamSynchronize(h->stream));
    std::memcpy(&f, h->h_small, sizeof(int));
    if (f) return fail(h, MSSTAB_ERR_INVALID_ARG, f & 1 ? "CSR row_ptr is not monotone from 0 to nnz"
                                                        : "CSR column index out of range");
  }
  // rho = max |a_ii| for the FP32 copy A/rho
  unsigned long long* dbits = (unsigned long long*)&h->st->scal[0];
  CK(cudaMemsetAsync(dbits, 0, sizeof(unsigned long long), h->stream));
  LAUNCH(MSSTAB_K_OTHER, csr_max_diag(c, (int)n, d_row_ptr, d_col, d_val, dbits));
  CKS(sync_read(h, dbits, sizeof(double)));
  h->rho = h->h_small[0] > 0.0 && std::isfinite(h->h_small[0]) ? h->h_small[0] : 1.0;

  MatDesc& A = h->A;
  A.n = (int)n;
  A.nnz = nnz;
  A.format = h->opt.spmv_format == MSSTAB_FORMAT_CSR ? 1 : 0;
  if (A.format == 1) {
    CKS(dalloc(h, &p, sizeof(int) * (n + 1)));
    A.row_ptr = (int*)p;
    CK(cudaMemcpyAsync(p, d_row_ptr, sizeof(int) * (n + 1), cudaMemcpyDeviceToDevice, h->stream));
    CKS(dalloc(h, &p, sizeof(int) * nnz));
    A.col = (int*)p;
    CK(cudaMemcpyAsync(p, d_col, sizeof(int) * nnz, cudaMemcpyDeviceToDevice, h->stream));
    CKS(dalloc(h, &p, sizeof(double) * nnz));
    A.val64 = (double*)p;
    CK(cudaMemcpyAsync(p, d_val, sizeof(double) * nnz, cudaMemcpyDeviceToDevice, h->stream));
    CKS(dalloc(h, &p, sizeof(float) * nnz));
    A.val32 = (float*)p;
    LAUNCH(MSSTAB_K_OTHER, f64_to_f32_n(c, nnz, A.val64, (float*)p, 1.0 / h->rho));
  } else {
    // SELL-32-sigma structure on the host from the row lengths
    std::vector<int> rp(n + 1);
    CK(cudaMemcpyAsync(rp.data(), d_row_ptr, sizeof(int) * (n + 1), cudaMemcpyDeviceToHost, h->stream));
    CK(cudaStreamSynchronize(h->stream));
    const int nsl = (int)((n + 31) / 32);
    std::vector<int> perm;
    const int sigma = h->opt.sell_sigma > 1 ? h->opt.sell_sigma : 1;
    if (sigma > 1) {
      perm.resize(n);
      for (int64_t i = 0; i < n; ++i) perm[i] = (int)i;
      for (int64_t w0 = 0; w0 < n; w0 += sigma) {
        const int64_t w1 = std::min<int64_t>(n, w0 + sigma);
        std::stable_sort(perm.begin() + w0, perm.begin() + w1, [&](int a, int b) {
          return (rp[a + 1] - rp[a]) > (rp[b + 1] - rp[b]);
        });
      }
    }
    std::vector<int> sw(nsl), sp(nsl + 1);
    int64_t off = 0;
    for (int k = 0; k < nsl; ++k) {
      int w = 0;
      for (int l = 0; l < 32; ++l) {
        const int64_t pos = (int64_t)k * 32 + l;
        if (pos >= n) break;
        const int row = sigma > 1 ? perm[pos] : (int)pos;
        w = std::max(w, rp[row + 1] - rp[row]);
      }
      sw[k] = w;
      sp[k] = (int)off;
      off += 32LL * w;
      if (off >= (1LL << 31)) return fail(h, MSSTAB_ERR_INVALID_ARG, "SELL storage exceeds int32 offsets");
    }
    sp[nsl] = (int)off;
    A.nslices = nsl;
    A.nnz_sell = off;
    CKS(dalloc(h, &p, sizeof(int) * (nsl + 1)));
    A.slice_ptr = (int*)p;
    CK(cudaMemcpyAsync(p, sp.data(), sizeof(int) * (nsl + 1), cudaMemcpyHostToDevice, h->stream));
    CKS(dalloc(h, &p, sizeof(int) * nsl));
    A.slice_w = (int*)p;
    CK(cudaMemcpyAsync(p, sw.data(), sizeof(int) * nsl, cudaMemcpyHostToDevice, h->stream));
    if (sigma > 1) {
      CKS(dalloc(h, &p, sizeof(int) * n));
      A.perm = (int*)p;
      CK(cudaMemcpyAsync(p, perm.data(), sizeof(int) * n, cudaMemcpyHostToDevice, h->stream));
    }
    CKS(dalloc(h, &p, sizeof(int) * off));
    A.scol = (int*)p;
    CKS(dalloc(h, &p, sizeof(double) * off));
    A.sval64 = (double*)p;
    CKS(dalloc(h, &p, sizeof(float) * off));
    A.sval32 = (float*)p;
    LAUNCH(MSSTAB_K_OTHER, sell_fill(c, (int)n, nsl, d_row_ptr, d_col, d_val, A.slice_ptr, A.slice_w, A.perm,
                                     (int*)A.scol, (double*)A.sval64));
    LAUNCH(MSSTAB_K_OTHER, f64_to_f32_n(c, off, A.sval64, (float*)A.sval32, 1.0 / h->rho));
    // keep the host copies alive until the uploads are done
    CK(cudaStreamSynchronize(h->stream));
  }

  if (h->precond) CKS(ilu_create(h, n, nnz, d_row_ptr, d_col, d_val));
  if (h->opt.fetch_policy == MSSTAB_FETCH_SLOPE) {
    const int64_t ldp = round_up(n, 32);
    CKS(dalloc(h, &p, sizeof(double) * (size_t)ldp * h->s));
    h->Uprev = (double*)p;
    CKS(dalloc(h, &p, sizeof(double) * (size_t)ldp * h->s));
    h->Vprev = (double*)p;
  }

  // workspaces: FP64 levels for the FP64 mode; FP32 levels for the inner mode
  const bool inner = h->opt.precision == MSSTAB_PREC_FP32_INNER;
  CKS(alloc_work<double>(h, h->w64, true));   // FP64 levels also serve the FP32-inner form's FP64 finish
  CKS(alloc_work<float>(h, h->w32, inner));

  // cut space: orthonormalise the raw basis (Cholesky QR twice) in FP64
  CK(cudaMemcpy2DAsync(h->w64.P, sizeof(double) * h->w64.ld, d_p_raw, sizeof(double) * n, sizeof(double) * n,
                       h->s, cudaMemcpyDeviceToDevice, h->stream));
  bool ok = true;
  CKS(cholqr2<double>(h, h->w64.P, nullptr, h->w64.ld, &ok));
  if (!ok) return fail(h, MSSTAB_ERR_INVALID_ARG, "the raw cut-space basis is rank deficient");
  for (int q = 0; q < h->s; ++q)
    LAUNCH(MSSTAB_K_OTHER, f64_to_f32_n(c, n, h->w64.P + (int64_t)q * h->w64.ld,
                                        h->w32.P + (int64_t)q * h->w32.ld, 1.0));
  {
    // row-interleaved copies of P (rows on 16-byte boundaries)
    void* p = nullptr;
    h->w64.sp = (h->s + 1) / 2 * 2;
    CKS(dalloc(h, &p, sizeof(double) * (size_t)n * h->w64.sp));
    h->w64.Pil = (double*)p;
    LAUNCH(MSSTAB_K_OTHER, interleave_rows<double>(c, n, h->s, h->w64.P, h->w64.ld, h->w64.sp, h->w64.Pil));
    h->w32.sp = (h->s + 3) / 4 * 4;
    CKS(dalloc(h, &p, sizeof(float) * (size_t)n * h->w32.sp));
    h->w32.Pil = (float*)p;
    LAUNCH(MSSTAB_K_OTHER, interleave_rows<float>(c, n, h->s, h->w32.P, h->w32.ld, h->w32.sp, h->w32.Pil));
  }
  {
    // a block-partitioned cut space (each row's only non-zero in column
    // (row / 32) mod s; orthonormalisation keeps that structure exactly)
    // makes the projections one multiply-add per row
    void* p = nullptr;
    CKS(dalloc(h, &p, sizeof(double) * (size_t)n));
    double* pb64 = (double*)p;
    CKS(dalloc(h, &p, sizeof(float) * (size_t)n));
    float* pb32 = (float*)p;
    CK(cudaMemsetAsync(&h->st->flag, 0, sizeof(int), h->stream));
    LAUNCH(MSSTAB_K_OTHER, pblock_compress<double>(c, n, h->s, h->w64.P, h->w64.ld, pb64, &h->st->flag));
    LAUNCH(MSSTAB_K_OTHER, pblock_compress<float>(c, n, h->s, h->w32.P, h->w32.ld, pb32, &h->st->flag));
    CKS(sync_read(h, &h->st->flag, sizeof(int)));
    int f = 0;
    std::memcpy(&f, h->h_small, sizeof(int));
    CK(cudaMemsetAsync(&h->st->flag, 0, sizeof(int), h->stream));
    if (f == 0 && h->s > 1) {
      h->w64.Pb = pb64;
      h->w32.Pb = pb32;
    }
  }
  CK(cudaStreamSynchronize(h->stream));
  return MSSTAB_OK;
}

msstab_status msstab_create(int64_t n, int64_t nnz, const int32_t* d_row_ptr, const int32_t* d_col,
                            const double* d_val, int32_t s, int32_t ell, const double* d_p_raw,
                            const msstab_options* opt, msstab_t* out) {
  g_create_error.clear();
  if (!out) return fail(nullptr, MSSTAB_ERR_INVALID_ARG, "out is NULL");
  *out = nullptr;
  if (n < 1 || n > MAX_ROWS) return fail(nullptr, MSSTAB_ERR_INVALID_ARG, "n must be in [1, 2^31 - 2^22]");
  if (nnz < 0 || nnz >= (1LL << 31)) return fail(nullptr, MSSTAB_ERR_INVALID_ARG, "nnz out of range");
  if (s < 1 || s > SMAX || s > n) return fail(nullptr, MSSTAB_ERR_INVALID_ARG, "s must satisfy 1 <= s <= min(16, n)");
  if (ell < 1 || ell > LMAX) return fail(nullptr, MSSTAB_ERR_INVALID_ARG, "l must satisfy 1 <= l <= 8");
  if (!d_row_ptr || !d_p_raw || (nnz > 0 && (!d_col || !d_val)))
    return fail(nullptr, MSSTAB_ERR_INVALID_ARG, "NULL matrix or cut-space pointer");
  msstab_t h = new msstab_s();
  h->n = (int)n;
  h->nnz = nnz;
  h->s = s;
  h->ell = ell;
  if (opt)
    h->opt = *opt;
  else
    msstab_default_options(&h->opt);
  if (h->opt.sell_sigma > 1 && h->opt.sell_sigma % 32 != 0) {
    delete h;
    return fail(nullptr, MSSTAB_ERR_INVALID_ARG, "sell_sigma must be 1 or a multiple of 32");
  }
  if (h->opt.precond != MSSTAB_PRECOND_NONE && h->opt.precond != MSSTAB_PRECOND_ILU0) {
    delete h;
    return fail(nullptr, MSSTAB_ERR_INVALID_ARG, "precond must be MSSTAB_PRECOND_NONE or MSSTAB_PRECOND_ILU0");
  }
  if (h->opt.precond == MSSTAB_PRECOND_ILU0 && h->opt.precision != MSSTAB_PREC_FP64) {
    delete h;
    return fail(nullptr, MSSTAB_ERR_INVALID_ARG, "the ILU(0) preconditioner needs precision MSSTAB_PREC_FP64");
  }
  h->precond = h->opt.precond == MSSTAB_PRECOND_ILU0;
  h->level = h->opt.persistent != 0 && !h->precond && h->opt.spmv_format != MSSTAB_FORMAT_CSR;
  if (h->opt.fetch_policy < MSSTAB_FETCH_ONCE || h->opt.fetch_policy > MSSTAB_FETCH_PROBE) {
    delete h;
    return fail(nullptr, MSSTAB_ERR_INVALID_ARG, "unknown fetch_policy");
  }
  if ((h->opt.fetch_policy == MSSTAB_FETCH_SLOPE || h->opt.fetch_policy == MSSTAB_FETCH_PROBE) &&
      h->opt.precision != MSSTAB_PREC_FP64) {
    delete h;
    return fail(nullptr, MSSTAB_ERR_INVALID_ARG, "the slope and probe fetch policies need precision FP64");
  }
  h->stream = (cudaStream_t)h->opt.stream;
  msstab_status rc = create_impl(h, n, nnz, d_row_ptr, d_col, d_val, d_p_raw);
  if (rc != MSSTAB_OK) {
    g_create_error = h->err;
    msstab_destroy(h);
    return rc;
  }
  *out = h;
  return MSSTAB_OK;
}

msstab_status msstab_solve(msstab_t h, const double* d_b, double* d_x, double tol, msstab_stats* st) {
  CKS(check_handle(h));
  CKS(check_ptr(h, d_b, "b"));
  CKS(check_ptr(h, d_x, "x"));
  const size_t bytes = sizeof(double) * h->n;
  CK(cudaMemcpyAsync(h->w64.B, d_b, bytes, cudaMemcpyDeviceToDevice, h->stream));
  CK(cudaMemcpyAsync(h->w64.X, d_x, bytes, cudaMemcpyDeviceToDevice, h->stream));
  msstab_status rc = solve_common(h, tol, st);
  if (rc == MSSTAB_OK || rc == MSSTAB_ERR_MAXIT || rc == MSSTAB_ERR_NAN || rc == MSSTAB_ERR_BREAKDOWN) {
    CK(cudaMemcpyAsync(d_x, h->w64.X, bytes, cudaMemcpyDeviceToDevice, h->stream));
    CK(cudaStreamSynchronize(h->stream));
  }
  return rc;
}

msstab_status msstab_solve_host(msstab_t h, const double* b, double* x, double tol, msstab_stats* st) {
  CKS(check_handle(h));
  if (!b || !x) return fail(h, MSSTAB_ERR_INVALID_ARG, "b or x is NULL");
  const size_t bytes = sizeof(double) * h->n;
  // b and x go straight between the caller's memory and the device (the
  // driver stages pageable memory itself, in pipelined chunks)
  CK(cudaMemcpyAsync(h->w64.B, b, bytes, cudaMemcpyHostToDevice, h->stream));
  CK(cudaMemcpyAsync(h->w64.X, x, bytes, cudaMemcpyHostToDevice, h->stream));
  msstab_status rc = solve_common(h, tol, st);
  if (rc == MSSTAB_OK || rc == MSSTAB_ERR_MAXIT || rc == MSSTAB_ERR_NAN || rc == MSSTAB_ERR_BREAKDOWN) {
    CK(cudaMemcpyAsync(x, h->w64.X, bytes, cudaMemcpyDeviceToHost, h->stream));
    CK(cudaStreamSynchronize(h->stream));
  }
  return rc;
}

msstab_status msstab_set_spin_limit(msstab_t h, int64_t polls) {
  CKS(check_handle(h));
  h->opt.spin_limit = polls;
  h->spin_limit = polls > 0 ? (long long)polls : (1LL << 22);
  h->ilu.spin_limit = h->spin_limit;
  // the cycle graphs hold the old limit in their launch arguments
  for (auto& g : h->graphs) cudaGraphExecDestroy(g.exec);
  h->graphs.clear();
  return MSSTAB_OK;
}

msstab_status msstab_history(msstab_t h, double* relres, int64_t* mvs, int32_t cap, int32_t* count) {
  CKS(check_handle(h));
  const int nh = (int)h->hist.size();
  if (count) *count = nh;
  for (int i = 0; i < nh && i < cap; ++i) {
    if (relres) relres[i] = h->hist[i];
    if (mvs) mvs[i] = h->hist_mvs[i];
  }
  return MSSTAB_OK;
}

msstab_status msstab_reset_recycle(msstab_t h) {
  CKS(check_handle(h));
  h->w64.has_rec = false;
  h->w32.has_rec = false;
  h->probe_cycle = 0;
  return MSSTAB_OK;
}

msstab_status msstab_has_recycle(msstab_t h, int32_t* flag) {
  CKS(check_handle(h));
  if (!flag) return fail(h, MSSTAB_ERR_INVALID_ARG, "flag is NULL");
  *flag = (h->opt.precision == MSSTAB_PREC_FP32_INNER ? h->w32.has_rec : h->w64.has_rec) ? 1 : 0;
  return MSSTAB_OK;
}

msstab_status msstab_export_recycle(msstab_t h, double* d_U, double* d_V) {
  CKS(check_handle(h));
  if (h->opt.precision != MSSTAB_PREC_FP64) return fail(h, MSSTAB_ERR_INVALID_ARG, "export needs an FP64 handle");
  if (!h->w64.has_rec) return fail(h, MSSTAB_ERR_INVALID_ARG, "the handle holds no recycled basis");
  if (!d_U || !d_V) return fail(h, MSSTAB_ERR_INVALID_ARG, "NULL pointer");
  const size_t row = sizeof(double) * h->n, pitch = sizeof(double) * h->w64.ld;
  CK(cudaMemcpy2DAsync(d_U, row, h->w64.Urec, pitch, row, h->s, cudaMemcpyDeviceToDevice, h->stream));
  CK(cudaMemcpy2DAsync(d_V, row, h->w64.Vrec, pitch, row, h->s, cudaMemcpyDeviceToDevice, h->stream));
  CK(cudaStreamSynchronize(h->stream));
  return MSSTAB_OK;
}

msstab_status msstab_import_recycle(msstab_t h, const double* d_U, const double* d_V) {
  CKS(check_handle(h));
  if (h->opt.precision != MSSTAB_PREC_FP64) return fail(h, MSSTAB_ERR_INVALID_ARG, "import needs an FP64 handle");
  if (!d_U || !d_V) return fail(h, MSSTAB_ERR_INVALID_ARG, "NULL pointer");
  const size_t row = sizeof(double) * h->n, pitch = sizeof(double) * h->w64.ld;
  CK(cudaMemcpy2DAsync(h->w64.Urec, pitch, d_U, row, row, h->s, cudaMemcpyDeviceToDevice, h->stream));
  CK(cudaMemcpy2DAsync(h->w64.Vrec, pitch, d_V, row, row, h->s, cudaMemcpyDeviceToDevice, h->stream));
  CK(cudaStreamSynchronize(h->stream));
  h->w64.has_rec = true;
  return MSSTAB_OK;
}

msstab_status msstab_select_guess(msstab_t h, const double* d_b, const double* d_xprev, const double* d_delta,
                                  double* d_x, int32_t* used) {
  CKS(check_handle(h));
  CKS(check_ptr(h, d_b, "b"));
  CKS(check_ptr(h, d_xprev, "xprev"));
  CKS(check_ptr(h, d_delta, "delta"));
  CKS(check_ptr(h, d_x, "x"));
  const Ctx c = h->ctx();
  const int n = h->n;
  DevState* st = h->st;
  Work<double>& w = h->w64;
  LAUNCH(MSSTAB_K_OTHER, axpby_f64(c, n, 1.0, d_xprev, 1.0, d_delta, w.XB2));
  LAUNCH(MSSTAB_K_SPMV, spmv<double>(c, h->A, w.XB2, w.Tm, d_b, nullptr, 0, 0, 1, 0, &st->scal[0], epi_none(h)));
  LAUNCH(MSSTAB_K_SPMV, spmv<double>(c, h->A, d_xprev, w.Tm, d_b, nullptr, 0, 0, 1, 0, &st->scal[1], epi_none(h)));
  CKS(sync_read(h, &st->scal[0], 2 * sizeof(double)));
  const bool keep = h->h_small[0] < h->h_small[1];
  CK(cudaMemcpyAsync(d_x, keep ? w.XB2 : d_xprev, sizeof(double) * n, cudaMemcpyDeviceToDevice, h->stream));
  CK(cudaStreamSynchronize(h->stream));
  if (used) *used = keep ? 1 : 0;
  return MSSTAB_OK;
}

msstab_status msstab_select_guess_scaled(msstab_t h, const double* d_b, const double* d_xprev,
                                         const double* d_delta, double* d_x, int32_t* used, double* alpha,
                                         double* reduction) {
  CKS(check_handle(h));
  CKS(check_ptr(h, d_b, "b"));
  CKS(check_ptr(h, d_xprev, "xprev"));
  CKS(check_ptr(h, d_delta, "delta"));
  CKS(check_ptr(h, d_x, "x"));
  const Ctx c = h->ctx();
  const int n = h->n;
  DevState* st = h->st;
  Work<double>& w = h->w64;
  // r0 = b - A x_prev (||r0||^2), w = A delta, then w . r0 and w . w
  LAUNCH(MSSTAB_K_SPMV, spmv<double>(c, h->A, d_xprev, w.Tm, d_b, nullptr, 0, 0, 1, 0, &st->scal[0], epi_none(h)));
  LAUNCH(MSSTAB_K_SPMV, spmv<double>(c, h->A, d_delta, w.XB2, nullptr, nullptr, 0, 0, 0, 0, nullptr, epi_none(h)));
  MdCols<double> cols{};
  cols.x[0] = w.XB2;
  cols.y[0] = w.Tm;
  LAUNCH(MSSTAB_K_OTHER, multidot<double>(c, n, cols, 1, 1, 1, &st->scal[1], 2, epi_none(h)));
  CKS(sync_read(h, &st->scal[0], 3 * sizeof(double)));
  const double rr = h->h_small[0], wr = h->h_small[1], ww = h->h_small[2];
  const double a = ww > 0.0 ? wr / ww : 0.0;
  const bool keep = std::isfinite(a) && a != 0.0 && rr > 0.0;
  if (keep)
    LAUNCH(MSSTAB_K_OTHER, axpby_f64(c, n, 1.0, d_xprev, a, d_delta, d_x));
  else
    CK(cudaMemcpyAsync(d_x, d_xprev, sizeof(double) * n, cudaMemcpyDeviceToDevice, h->stream));
  CK(cudaStreamSynchronize(h->stream));
  if (used) *used = keep ? 1 : 0;
  if (alpha) *alpha = keep ? a : 0.0;
  if (reduction) *reduction = keep ? std::sqrt(std::max(0.0, 1.0 - (wr * wr) / (ww * rr))) : 1.0;
  return MSSTAB_OK;
}

// Coefficients a minimising ||r0 - W a|| from G = W^T W (row-major, m x m),
// c = W^T r0 and rr = ||r0||^2: the normal equations scaled by
// D = diag(G)^-1/2 and solved by Cholesky; a direction with W_j = 0 gets
// a_j = 0.  If the scaled Gram is not numerically positive definite (nearly
// dependent directions), the best single direction is taken.  Returns the
// squared residual ratio ||r0 - W a||^2 / rr (clamped to [0, 1]).
static double span_coefficients(const double* G, const double* c, double rr, int m, double* a) {
  double d[4], M[16], y[4];
  int idx[4], k = 0;
  for (int j = 0; j < m; ++j) {
    a[j] = 0.0;
    if (G[j * m + j] > 0.0 && std::isfinite(G[j * m + j])) idx[k++] = j;
  }
  if (k == 0 || !(rr > 0.0)) return 1.0;
  for (int i = 0; i < k; ++i) d[i] = 1.0 / std::sqrt(G[idx[i] * m + idx[i]]);
  for (int i = 0; i < k; ++i) {
    for (int j = 0; j < k; ++j) M[i * k + j] = d[i] * G[idx[i] * m + idx[j]] * d[j];
    y[i] = d[i] * c[idx[i]];
  }
  // Cholesky M = R^T R (upper R in place of M's upper triangle), pivots above 1e-12
  bool ok = true;
  double R[16] = {};
  for (int j = 0; j < k && ok; ++j) {
    double s = M[j * k + j];
    for (int i = 0; i < j; ++i) s -= R[i * k + j] * R[i * k + j];
    if (!(s > 1e-12)) {
      ok = false;
      break;
    }
    R[j * k + j] = std::sqrt(s);
    for (int l = j + 1; l < k; ++l) {
      double v = M[j * k + l];
      for (int i = 0; i < j; ++i) v -= R[i * k + j] * R[i * k + l];
      R[j * k + l] = v / R[j * k + j];
    }
  }
  if (ok) {
    for (int i = 0; i < k; ++i) {          // R^T w = y
      double v = y[i];
      for (int l = 0; l < i; ++l) v -= R[l * k + i] * y[l];
      y[i] = v / R[i * k + i];
    }
    for (int i = k - 1; i >= 0; --i) {     // R z = w
      double v = y[i];
      for (int l = i + 1; l < k; ++l) v -= R[i * k + l] * y[l];
      y[i] = v / R[i * k + i];
    }
    for (int i = 0; i < k; ++i) a[idx[i]] = d[i] * y[i];
  } else {
    int best = 0;
    double gain = -1.0;
    for (int i = 0; i < k; ++i) {
      const double g = y[i] * y[i];       // (c_j^2 / G_jj): the reduction of ||r||^2 by direction j alone
      if (g > gain) {
        gain = g;
        best = i;
      }
    }
    a[idx[best]] = d[best] * d[best] * c[idx[best]];
  }
  double ca = 0.0;
  for (int j = 0; j < m; ++j) ca += c[j] * a[j];
  const double ratio = 1.0 - ca / rr;
  return ratio < 0.0 ? 0.0 : (ratio > 1.0 ? 1.0 : ratio);
}

msstab_status msstab_select_guess_span(msstab_t h, const double* d_b, const double* d_xprev, const double* d_dirs,
                                       int64_t ld, int32_t ndir, double* d_x, int32_t* used, double* coef,
                                       double* reduction) {
  CKS(check_handle(h));
  CKS(check_ptr(h, d_b, "b"));
  CKS(check_ptr(h, d_xprev, "xprev"));
  CKS(check_ptr(h, d_dirs, "dirs"));
  CKS(check_ptr(h, d_x, "x"));
  if (ndir < 1 || ndir > 4 || ndir > h->s * (h->ell + 2))
    return fail(h, MSSTAB_ERR_INVALID_ARG, "ndir must be in [1, min(4, s (l + 2))]");
  if (ld < h->n) return fail(h, MSSTAB_ERR_INVALID_ARG, "ld < n");
  const Ctx c = h->ctx();
  const int n = h->n;
  DevState* st = h->st;
  Work<double>& w = h->w64;
  // r0 = b - A x_prev into Tm; W_j = A dir_j into level columns of the
  // workspace (free between solves); then W^T W, W^T r0 and ||r0||^2
  LAUNCH(MSSTAB_K_SPMV, spmv<double>(c, h->A, d_xprev, w.Tm, d_b, nullptr, 0, 0, 1, 0, &st->scal[0], epi_none(h)));
  MdCols<double> cols{};
  for (int j = 0; j < ndir; ++j) {
    double* Wj = w.V + (int64_t)j * w.ld;
    LAUNCH(MSSTAB_K_SPMV, spmv<double>(c, h->A, d_dirs + (int64_t)j * ld, Wj, nullptr, nullptr, 0, 0, 0, 0,
                                       nullptr, epi_none(h)));
    cols.x[j] = Wj;
    cols.y[j] = Wj;
  }
  cols.y[ndir] = w.Tm;
  // out[t * 8 + col]: t < ndir targets, columns W_0 .. W_{ndir-1}, r0
  LAUNCH(MSSTAB_K_OTHER, multidot<double>(c, n, cols, ndir, ndir + 1, 0, &st->scal[8], 8, epi_none(h)));
  CK(cudaMemcpyAsync(h->h_small, &st->scal[0], sizeof(double), cudaMemcpyDeviceToHost, h->stream));
  CK(cudaMemcpyAsync(h->h_small + 8, &st->scal[8], 8 * ndir * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
  CK(cudaStreamSynchronize(h->stream));
  const double rr = h->h_small[0];
  double G[16], cv[4], a[4];
  for (int i = 0; i < ndir; ++i) {
    for (int j = 0; j < ndir; ++j) G[i * ndir + j] = h->h_small[8 + i * 8 + j];
    cv[i] = h->h_small[8 + i * 8 + ndir];
  }
  const double ratio = span_coefficients(G, cv, rr, ndir, a);
  bool keep = ratio < 1.0;
  for (int j = 0; j < ndir; ++j) keep = keep && std::isfinite(a[j]);
  if (keep) {
    // x = x_prev + sum_j a_j dir_j (d_x may alias neither input nor be
    // written before the last read: the combination goes through XB2)
    LAUNCH(MSSTAB_K_OTHER, axpby_f64(c, n, 1.0, d_xprev, a[0], d_dirs, w.XB2));
    for (int j = 1; j < ndir; ++j)
      LAUNCH(MSSTAB_K_OTHER, axpby_f64(c, n, 1.0, w.XB2, a[j], d_dirs + (int64_t)j * ld, w.XB2));
    CK(cudaMemcpyAsync(d_x, w.XB2, sizeof(double) * n, cudaMemcpyDeviceToDevice, h->stream));
  } else {
    CK(cudaMemcpyAsync(d_x, d_xprev, sizeof(double) * n, cudaMemcpyDeviceToDevice, h->stream));
  }
  CK(cudaStreamSynchronize(h->stream));
  if (used) *used = keep ? 1 : 0;
  if (coef)
    for (int j = 0; j < ndir; ++j) coef[j] = keep ? a[j] : 0.0;
  if (reduction) *reduction = keep ? std::sqrt(ratio) : 1.0;
  return MSSTAB_OK;
}

// ---------------------------------------------------------------------------
// kernel-level entry points
// ---------------------------------------------------------------------------
static msstab_status check_prec(msstab_t h, int32_t prec) {
  if (prec != 0 && prec != 1) return fail(h, MSSTAB_ERR_INVALID_ARG, "prec must be 0 (FP64) or 1 (FP32)");
  return MSSTAB_OK;
}

msstab_status msstab_op_spmv(msstab_t h, int32_t prec, const void* d_x, void* d_y) {
  CKS(check_handle(h));
  CKS(check_prec(h, prec));
  CKS(check_ptr(h, d_x, "x", prec == 0 ? 8 : 4));
  CKS(check_ptr(h, d_y, "y", prec == 0 ? 8 : 4));
  const Ctx c = h->ctx();
  if (prec == 0)
    LAUNCH(MSSTAB_K_SPMV, spmv<double>(c, h->A, (const double*)d_x, (double*)d_y, nullptr, nullptr, 0, 0, 0, 0,
                                       nullptr, epi_none(h)));
  else
    LAUNCH(MSSTAB_K_SPMV, spmv<float>(c, h->A, (const float*)d_x, (float*)d_y, nullptr, nullptr, 0, 0, 0, 0,
                                      nullptr, epi_none(h)));
  CK(cudaStreamSynchronize(h->stream));
  return MSSTAB_OK;
}

msstab_status msstab_op_residual(msstab_t h, const double* d_b, const double* d_x, double* d_r, double* d_out) {
  CKS(check_handle(h));
  CKS(check_ptr(h, d_b, "b"));
  CKS(check_ptr(h, d_x, "x"));
  CKS(check_ptr(h, d_r, "r"));
  if (!d_out) return fail(h, MSSTAB_ERR_INVALID_ARG, "out is NULL");
  const Ctx c = h->ctx();
  LAUNCH(MSSTAB_K_SPMV, spmv<double>(c, h->A, d_x, d_r, d_b, nullptr, 0, 0, 1, 1, d_out, epi_none(h)));
  CK(cudaStreamSynchronize(h->stream));
  return MSSTAB_OK;
}

msstab_status msstab_op_spmv_dot(msstab_t h, int32_t prec, const void* d_x, void* d_y, double* d_dots) {
  CKS(check_handle(h));
  CKS(check_prec(h, prec));
  CKS(check_ptr(h, d_x, "x", prec == 0 ? 8 : 4));
  CKS(check_ptr(h, d_y, "y", prec == 0 ? 8 : 4));
  if (!d_dots) return fail(h, MSSTAB_ERR_INVALID_ARG, "dots is NULL");
  const Ctx c = h->ctx();
  if (prec == 0)
    LAUNCH(MSSTAB_K_SPMV_DOT, spmv<double>(c, h->A, (const double*)d_x, (double*)d_y, nullptr, h->w64.P,
                                           h->w64.ld, h->s, 1, 0, d_dots, epi_none(h), h->w64.Pil, h->w64.sp,
                                           h->w64.Pb));
  else
    LAUNCH(MSSTAB_K_SPMV_DOT, spmv<float>(c, h->A, (const float*)d_x, (float*)d_y, nullptr, h->w32.P, h->w32.ld,
                                          h->s, 1, 0, d_dots, epi_none(h), h->w32.Pil, h->w32.sp, h->w32.Pb));
  CK(cudaStreamSynchronize(h->stream));
  return MSSTAB_OK;
}

msstab_status msstab_op_axpby(msstab_t h, double alpha, const double* d_x, double beta, const double* d_z,
                              double* d_y) {
  CKS(check_handle(h));
  CKS(check_ptr(h, d_x, "x"));
  CKS(check_ptr(h, d_z, "z"));
  CKS(check_ptr(h, d_y, "y"));
  const Ctx c = h->ctx();
  LAUNCH(MSSTAB_K_OTHER, axpby_f64(c, h->n, alpha, d_x, beta, d_z, d_y));
  return MSSTAB_OK;
}

msstab_status msstab_op_get_p(msstab_t h, int32_t prec, void* d_P) {
  CKS(check_handle(h));
  CKS(check_prec(h, prec));
  if (!d_P) return fail(h, MSSTAB_ERR_INVALID_ARG, "P is NULL");
  const size_t es = prec == 0 ? sizeof(double) : sizeof(float);
  const void* src = prec == 0 ? (const void*)h->w64.P : (const void*)h->w32.P;
  const int64_t ld = prec == 0 ? h->w64.ld : h->w32.ld;
  CK(cudaMemcpy2DAsync(d_P, es * h->n, src, es * ld, es * h->n, h->s, cudaMemcpyDeviceToDevice, h->stream));
  CK(cudaStreamSynchronize(h->stream));
  return MSSTAB_OK;
}

msstab_status msstab_op_multidot(msstab_t h, int32_t prec, const void* d_X, int64_t ldx, int32_t nx,
                                 const void* d_Y, int64_t ldy, int32_t ny, double* d_out) {
  CKS(check_handle(h));
  CKS(check_prec(h, prec));
  if (nx < 1 || nx > 16 || ny < 1 || ny > 16 || ldx < h->n || ldy < h->n)
    return fail(h, MSSTAB_ERR_INVALID_ARG, "multidot: 1 <= nx, ny <= 16 and ld >= n required");
  CKS(check_ptr(h, d_X, "X", prec == 0 ? 8 : 4));
  CKS(check_ptr(h, d_Y, "Y", prec == 0 ? 8 : 4));
  if (!d_out) return fail(h, MSSTAB_ERR_INVALID_ARG, "out is NULL");
  const Ctx c = h->ctx();
  if (prec == 0) {
    MdCols<double> cols{};
    for (int t = 0; t < nx; ++t) cols.x[t] = (const double*)d_X + (int64_t)t * ldx;
    for (int q = 0; q < ny; ++q) cols.y[q] = (const double*)d_Y + (int64_t)q * ldy;
    LAUNCH(MSSTAB_K_OTHER, multidot<double>(c, h->n, cols, nx, ny, 0, d_out, ny, epi_none(h)));
  } else {
    MdCols<float> cols{};
    for (int t = 0; t < nx; ++t) cols.x[t] = (const float*)d_X + (int64_t)t * ldx;
    for (int q = 0; q < ny; ++q) cols.y[q] = (const float*)d_Y + (int64_t)q * ldy;
    LAUNCH(MSSTAB_K_OTHER, multidot<float>(c, h->n, cols, nx, ny, 0, d_out, ny, epi_none(h)));
  }
  CK(cudaStreamSynchronize(h->stream));
  return MSSTAB_OK;
}

static msstab_status check_levels(msstab_t h, int64_t ld, int32_t k, bool eta_level) {
  if (ld < h->n) return fail(h, MSSTAB_ERR_INVALID_ARG, "ld < n");
  if (k < 0 || k >= h->ell) return fail(h, MSSTAB_ERR_INVALID_ARG, "k must satisfy 0 <= k < l");
  (void)eta_level;
  return MSSTAB_OK;
}

msstab_status msstab_op_gamma_update(msstab_t h, int32_t prec, void* d_R, const void* d_V, int64_t ld, int32_t k,
                                     const double* d_gamma) {
  CKS(check_handle(h));
  CKS(check_prec(h, prec));
  CKS(check_levels(h, ld, k, false));
  CKS(check_ptr(h, d_R, "R", prec == 0 ? 8 : 4));
  CKS(check_ptr(h, d_V, "V", prec == 0 ? 8 : 4));
  if (!d_gamma) return fail(h, MSSTAB_ERR_INVALID_ARG, "gamma is NULL");
  const Ctx c = h->ctx();
  if (prec == 0)
    LAUNCH(MSSTAB_K_GAMMA, gamma_eager<double>(c, h->n, h->s, (double*)d_R, (const double*)d_V, ld, k, d_gamma));
  else
    LAUNCH(MSSTAB_K_GAMMA, gamma_eager<float>(c, h->n, h->s, (float*)d_R, (const float*)d_V, ld, k, d_gamma));
  CK(cudaStreamSynchronize(h->stream));
  return MSSTAB_OK;
}

msstab_status msstab_op_eta_update(msstab_t h, int32_t prec, const void* d_R, void* d_V, int64_t ld, int32_t k,
                                   int32_t q, const double* d_eta) {
  CKS(check_handle(h));
  CKS(check_prec(h, prec));
  CKS(check_levels(h, ld, k, true));
  if (q < 0 || q >= h->s) return fail(h, MSSTAB_ERR_INVALID_ARG, "q must satisfy 0 <= q < s");
  CKS(check_ptr(h, d_R, "R", prec == 0 ? 8 : 4));
  CKS(check_ptr(h, d_V, "V", prec == 0 ? 8 : 4));
  if (!d_eta) return fail(h, MSSTAB_ERR_INVALID_ARG, "eta is NULL");
  const Ctx c = h->ctx();
  if (prec == 0)
    LAUNCH(MSSTAB_K_ETA, eta_eager<double>(c, h->n, h->s, (const double*)d_R, (double*)d_V, ld, k, q, d_eta));
  else
    LAUNCH(MSSTAB_K_ETA, eta_eager<float>(c, h->n, h->s, (const float*)d_R, (float*)d_V, ld, k, q, d_eta));
  CK(cudaStreamSynchronize(h->stream));
  return MSSTAB_OK;
}

msstab_status msstab_op_lazy_update(msstab_t h, int32_t prec, void* d_R, void* d_V, void* d_x, int64_t ld,
                                    int32_t k, const double* d_gamma, const double* d_eta, double* d_gram) {
  CKS(check_handle(h));
  CKS(check_prec(h, prec));
  CKS(check_levels(h, ld, k, true));
  CKS(check_ptr(h, d_R, "R", prec == 0 ? 8 : 4));
  CKS(check_ptr(h, d_V, "V", prec == 0 ? 8 : 4));
  CKS(check_ptr(h, d_x, "x", prec == 0 ? 8 : 4));
  if (!d_gamma || !d_eta) return fail(h, MSSTAB_ERR_INVALID_ARG, "gamma or eta is NULL");
  const Ctx c = h->ctx();
  const int L = h->ell + 1;
  if (prec == 0) {
    LAUNCH(MSSTAB_K_LAZY, lazy_update<double>(c, h->n, h->s, (double*)d_R, (double*)d_V, (double*)d_x, ld, k,
                                              d_gamma, d_eta, h->s));
    if (d_gram) {
      MdCols<double> cols{};
      for (int i = 0; i < L; ++i) cols.x[i] = cols.y[i] = (const double*)d_R + (int64_t)i * ld;
      LAUNCH(MSSTAB_K_TAU, multidot<double>(c, h->n, cols, L, L, 0, d_gram, L, epi_none(h)));
    }
  } else {
    LAUNCH(MSSTAB_K_LAZY, lazy_update<float>(c, h->n, h->s, (float*)d_R, (float*)d_V, (float*)d_x, ld, k, d_gamma,
                                             d_eta, h->s));
    if (d_gram) {
      MdCols<float> cols{};
      for (int i = 0; i < L; ++i) cols.x[i] = cols.y[i] = (const float*)d_R + (int64_t)i * ld;
      LAUNCH(MSSTAB_K_TAU, multidot<float>(c, h->n, cols, L, L, 0, d_gram, L, epi_none(h)));
    }
  }
  CK(cudaStreamSynchronize(h->stream));
  return MSSTAB_OK;
}

msstab_status msstab_op_tau_update(msstab_t h, int32_t prec, void* d_R, void* d_V, void* d_x, int64_t ld,
                                   const double* d_tau) {
  CKS(check_handle(h));
  CKS(check_prec(h, prec));
  if (ld < h->n) return fail(h, MSSTAB_ERR_INVALID_ARG, "ld < n");
  CKS(check_ptr(h, d_R, "R", prec == 0 ? 8 : 4));
  CKS(check_ptr(h, d_V, "V", prec == 0 ? 8 : 4));
  CKS(check_ptr(h, d_x, "x", prec == 0 ? 8 : 4));
  if (!d_tau) return fail(h, MSSTAB_ERR_INVALID_ARG, "tau is NULL");
  const Ctx c = h->ctx();
  if (prec == 0)
    LAUNCH(MSSTAB_K_TAU, tau_update<double>(c, h->n, h->s, h->ell, (double*)d_R, (double*)d_V, (double*)d_x,
                                            nullptr, ld, d_tau, h->w64.P, h->w64.ld, 1, 0, h->st, epi_none(h)));
  else
    LAUNCH(MSSTAB_K_TAU, tau_update<float>(c, h->n, h->s, h->ell, (float*)d_R, (float*)d_V, (float*)d_x, nullptr,
                                           ld, d_tau, h->w32.P, h->w32.ld, 1, 0, h->st, epi_none(h)));
  CK(cudaStreamSynchronize(h->stream));
  return MSSTAB_OK;
}

msstab_status msstab_op_tau_step(msstab_t h, int32_t prec, void* d_R, void* d_V, void* d_x, int64_t ld,
                                 const double* d_tau, int32_t do_update, const double* d_lazy_gamma,
                                 const double* d_lazy_eta, double* d_out) {
  CKS(check_handle(h));
  CKS(check_prec(h, prec));
  if (ld < h->n) return fail(h, MSSTAB_ERR_INVALID_ARG, "ld < n");
  CKS(check_ptr(h, d_R, "R", prec == 0 ? 8 : 4));
  CKS(check_ptr(h, d_V, "V", prec == 0 ? 8 : 4));
  CKS(check_ptr(h, d_x, "x", prec == 0 ? 8 : 4));
  if (!d_tau || !d_out) return fail(h, MSSTAB_ERR_INVALID_ARG, "NULL pointer");
  const Ctx c = h->ctx();
  const int s = h->s;
  if ((d_lazy_gamma == nullptr) != (d_lazy_eta == nullptr))
    return fail(h, MSSTAB_ERR_INVALID_ARG, "lazy gamma and eta: both or neither");
  if (d_lazy_gamma && !(prec == 1 && do_update &&
                        tau_fuses_lazy<float>(h->n, s, h->ell, (const float*)d_R, (const float*)d_V,
                                              (const float*)d_x, nullptr, ld, h->w32.P, h->w32.ld, h->w32.Pb)))
    return fail(h, MSSTAB_ERR_INVALID_ARG, "the fused lower-level updates need the FP32 degree-1 step, "
                                           "16-byte aligned columns and n % 4 == 0");
  if (prec == 0)
    LAUNCH(MSSTAB_K_TAU, tau_update<double>(c, h->n, s, h->ell, (double*)d_R, (double*)d_V, (double*)d_x, nullptr,
                                            ld, d_tau, h->w64.P, h->w64.ld, do_update ? 1 : 0, 1, h->st,
                                            epi_none(h), h->w64.Pb, h->w64.Pil, h->w64.sp));
  else
    LAUNCH(MSSTAB_K_TAU, tau_update<float>(c, h->n, s, h->ell, (float*)d_R, (float*)d_V, (float*)d_x, nullptr,
                                           ld, d_tau, h->w32.P, h->w32.ld, do_update ? 1 : 0, 1, h->st,
                                           epi_none(h), h->w32.Pb, h->w32.Pil, h->w32.sp, d_lazy_gamma,
                                           d_lazy_eta, s));
  for (int q = 0; q < s; ++q)
    CK(cudaMemcpyAsync(d_out + (size_t)q * s, &h->st->projV[q * SMAX], sizeof(double) * s, cudaMemcpyDeviceToDevice,
                       h->stream));
  CK(cudaMemcpyAsync(d_out + (size_t)s * s, &h->st->projR[0], sizeof(double) * s, cudaMemcpyDeviceToDevice,
                     h->stream));
  CK(cudaMemcpyAsync(d_out + (size_t)s * s + s, &h->st->rr, sizeof(double), cudaMemcpyDeviceToDevice, h->stream));
  CK(cudaStreamSynchronize(h->stream));
  return MSSTAB_OK;
}

msstab_status msstab_op_small_solve(msstab_t h, int32_t n, const double* d_M, const double* d_rhs, double* d_z,
                                    int32_t* d_flag) {
  CKS(check_handle(h));
  if (n < 1 || n > SMAX) return fail(h, MSSTAB_ERR_INVALID_ARG, "1 <= n <= 16 required");
  if (!d_M || !d_rhs || !d_z || !d_flag) return fail(h, MSSTAB_ERR_INVALID_ARG, "NULL pointer");
  const Ctx c = h->ctx();
  LAUNCH(MSSTAB_K_OTHER, small_lu(c, n, d_M, d_rhs, d_z, d_flag));
  CK(cudaStreamSynchronize(h->stream));
  return MSSTAB_OK;
}

static msstab_status check_ilu(msstab_t h) {
  CKS(check_handle(h));
  if (!h->precond) return fail(h, MSSTAB_ERR_INVALID_ARG, "the handle has no ILU(0) preconditioner");
  return MSSTAB_OK;
}

// wait for the sweeps and turn a timed-out grid barrier into an error
static msstab_status ilu_sync(msstab_t h) {
  CK(cudaMemcpyAsync(h->h_small, &h->st->flag, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
  CK(cudaStreamSynchronize(h->stream));
  int flag = 0;
  std::memcpy(&flag, h->h_small, sizeof(int));
  if (flag & FLAG_SYNC_TIMEOUT) {
    CK(cudaMemsetAsync(h->ilu.bar, 0, sizeof(GridBar), h->stream));
    CK(cudaMemsetAsync(&h->st->flag, 0, sizeof(int), h->stream));
    CK(cudaStreamSynchronize(h->stream));
    return fail(h, MSSTAB_ERR_CUDA, "a grid barrier of the ILU(0) level sweeps timed out");
  }
  return MSSTAB_OK;
}

msstab_status msstab_op_ilu_factor(msstab_t h, double* d_lu) {
  CKS(check_ilu(h));
  CKS(check_ptr(h, d_lu, "lu"));
  CK(cudaMemcpyAsync(d_lu, h->ilu.lu, sizeof(double) * h->nnz, cudaMemcpyDeviceToDevice, h->stream));
  CK(cudaStreamSynchronize(h->stream));
  return MSSTAB_OK;
}

msstab_status msstab_op_ilu_levels(msstab_t h, int32_t* d_lev_lower, int32_t* d_lev_upper, int32_t* h_info) {
  CKS(check_ilu(h));
  const IluDesc& F = h->ilu;
  if (d_lev_lower)
    CK(cudaMemcpyAsync(d_lev_lower, F.lev[0], sizeof(int) * h->n, cudaMemcpyDeviceToDevice, h->stream));
  if (d_lev_upper)
    CK(cudaMemcpyAsync(d_lev_upper, F.lev[1], sizeof(int) * h->n, cudaMemcpyDeviceToDevice, h->stream));
  CK(cudaStreamSynchronize(h->stream));
  if (h_info) {
    auto blocks = [&](int u) { return F.CH[u] > 0 ? (F.n + F.CH[u] - 1) / F.CH[u] : F.grid[u]; };
    const int32_t info[6] = {F.nlev[0], F.nlev[1], F.max_width[0], F.max_width[1], blocks(0), blocks(1)};
    std::memcpy(h_info, info, sizeof(info));
  }
  return MSSTAB_OK;
}

msstab_status msstab_op_ilu_apply(msstab_t h, int32_t which, const double* d_in, double* d_out) {
  CKS(check_ilu(h));
  CKS(check_ptr(h, d_in, "in"));
  CKS(check_ptr(h, d_out, "out"));
  if (which < 0 || which > 3) return fail(h, MSSTAB_ERR_INVALID_ARG, "which must be 0, 1, 2 or 3");
  if (which == 2 && d_in == d_out) return fail(h, MSSTAB_ERR_INVALID_ARG, "U x needs distinct in and out");
  const Ctx c = h->ctx();
  if (which == 0) LAUNCH(MSSTAB_K_PRECOND, ilu_lower_solve(c, h->ilu, d_in, d_out));
  if (which == 1) LAUNCH(MSSTAB_K_PRECOND, ilu_upper_solve(c, h->ilu, d_in, d_out));
  if (which == 2) LAUNCH(MSSTAB_K_PRECOND, ilu_upper_mul(c, h->ilu, d_in, d_out));
  if (which == 3)
    CKS(amv<double>(h, c, MSSTAB_K_SPMV, d_in, d_out, nullptr, nullptr, 0, 0, 0, 0, nullptr, epi_none(h)));
  return ilu_sync(h);
}

msstab_status msstab_op_tau_solve(msstab_t h, int32_t ell, const double* d_gram, double* d_tau) {
  CKS(check_handle(h));
  if (ell < 1 || ell > LMAX) return fail(h, MSSTAB_ERR_INVALID_ARG, "1 <= l <= 8 required");
  if (!d_gram || !d_tau) return fail(h, MSSTAB_ERR_INVALID_ARG, "NULL pointer");
  const Ctx c = h->ctx();
  LAUNCH(MSSTAB_K_OTHER, small_tau(c, ell, d_gram, d_tau));
  CK(cudaStreamSynchronize(h->stream));
  return MSSTAB_OK;
}

}  // extern "C"

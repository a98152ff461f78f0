#include <type_traits>
// Tall-skinny block kernels of libmsstab: the vector updates of Algorithm 1
// (gamma step, eta steps, degree-l step), multi-dots with a deterministic
// single grid-level combine, and the helpers of the Arnoldi start and of the
// Cholesky-QR orthonormalisation.
//
// One row per thread, grid-stride over rows; every column is read with
// consecutive threads on consecutive rows, so each warp load is one contiguous
// segment.  Coefficients (gamma, eta, tau) live in device memory, written by
// the small solve that ran in the last block of the preceding reduction, and
// are staged in shared memory at kernel start: the host never waits for them.

#include "launch.h"

namespace msk {

template <typename K>
static int max_grid(K kernel, const Ctx& c, int cap_blocks = MAXBLK) {
  int nb = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, kernel, NT, 0) != cudaSuccess || nb < 1) nb = 1;
  int g = nb * c.sms;
  return g > cap_blocks ? cap_blocks : g;
}

template <typename K>
static int max_grid_nt(K kernel, const Ctx& c, int nt) {
  int nb = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, kernel, nt, 0) != cudaSuccess || nb < 1) nb = 1;
  const int g = nb * c.sms;
  return g > MAXBLK ? MAXBLK : g;
}

__host__ __device__ constexpr int pow2_ge(int v) { return v <= 1 ? 1 : (v <= 2 ? 2 : (v <= 4 ? 4 : (v <= 8 ? 8 : (v <= 16 ? 16 : 32)))); }

static inline int clamp_grid(int64_t need, int cap) { return (int)(need < 1 ? 1 : (need < cap ? need : cap)); }

// Per-thread dot-product accumulators: FP64 for FP64 vectors, compensated FP32
// pairs for FP32 vectors (read out as FP64).
template <typename T, int N>
struct Acc;

template <int N>
struct Acc<double, N> {
  double v[N];
  __device__ __forceinline__ void zero() {
#pragma unroll
    for (int i = 0; i < N; ++i) v[i] = 0.0;
  }
  __device__ __forceinline__ void add(int i, double x, double y) { v[i] = fma(x, y, v[i]); }
  __device__ __forceinline__ double get(int i) const { return v[i]; }
};

template <int N>
struct Acc<float, N> {   // FP32 partials, widened exactly for the FP64 reductions
  float v[N];
  __device__ __forceinline__ void zero() {
#pragma unroll
    for (int i = 0; i < N; ++i) v[i] = 0.f;
  }
  __device__ __forceinline__ void add(int i, float x, float y) { v[i] = fmaf(x, y, v[i]); }
  __device__ __forceinline__ double get(int i) const { return widen_f32(v[i]); }
};

// ---------------------------------------------------------------------------
// gamma step on the top level:  r^(k) -= V^(k) gamma
// ---------------------------------------------------------------------------
// Rows are handled VW at a time (VW = 16 / sizeof(T): 16-byte loads, when
// every column start is 16-byte aligned; else VW = 1), all s + 1 loads of a
// group issued before the arithmetic; a ragged tail of n % VW rows is done
// row by row.
template <typename T, int VW>
struct VecOf {
  using type = std::conditional_t<VW == 1, T, std::conditional_t<sizeof(T) == 8, double2, float4>>;
};

template <typename T, int VW>
__device__ __forceinline__ T vget(const typename VecOf<T, VW>::type& v, int u) {
  return reinterpret_cast<const T*>(&v)[u];
}
template <typename T, int VW>
__device__ __forceinline__ void vset(typename VecOf<T, VW>::type& v, int u, T x) {
  reinterpret_cast<T*>(&v)[u] = x;
}

template <typename T, int S, int VW, typename ColOf>
__device__ __forceinline__ void combine_rows(int n, int s, const T* base, T* out, const T* c, ColOf col_of) {
  using V = typename VecOf<T, VW>::type;
  const int64_t groups = n / VW;
  const int64_t stride = (int64_t)gridDim.x * NT;
  for (int64_t g = blockIdx.x * (int64_t)NT + threadIdx.x; g < groups; g += stride) {
    V acc = reinterpret_cast<const V*>(base)[g];
    V v[S];
#pragma unroll
    for (int j = 0; j < S; ++j) {
      if (j >= s) break;
      v[j] = __ldg(reinterpret_cast<const V*>(col_of(j)) + g);
    }
#pragma unroll
    for (int j = 0; j < S; ++j) {
      if (j >= s) break;
#pragma unroll
      for (int u = 0; u < VW; ++u) vset<T, VW>(acc, u, vget<T, VW>(acc, u) - c[j] * vget<T, VW>(v[j], u));
    }
    reinterpret_cast<V*>(out)[g] = acc;
  }
  if constexpr (VW > 1) {   // ragged tail: rows groups * VW .. n - 1
    const int64_t row = groups * VW + threadIdx.x;
    if (blockIdx.x == 0 && row < n) {
      T v = base[row];
      for (int j = 0; j < s; ++j) v -= c[j] * col_of(j)[row];
      out[row] = v;
    }
  }
}

template <typename T>
static bool aligned16(const T* p) { return ((uintptr_t)p & 15u) == 0; }

// gamma step on the top level:  r^(k) -= V^(k) gamma
template <typename T, int S, int VW>
__global__ void __launch_bounds__(NT) gamma_eager_kernel(int n, int s, T* __restrict__ R,
                                                         const T* __restrict__ V, int64_t ld, int k,
                                                         const double* __restrict__ gamma) {
  __shared__ T g[SMAX];
  if (threadIdx.x < s) g[threadIdx.x] = (T)gamma[threadIdx.x];
  __syncthreads();
  T* rk = R + (int64_t)k * ld;
  const T* vk = V + (int64_t)(k + 1) * s * ld;
  combine_rows<T, S, VW>(n, s, rk, rk, g, [&](int j) { return vk + (int64_t)j * ld; });
}

// launch kern<S, VW> for the smallest S in {4, 8, 16} >= s, VW = 16-byte
// vectors when vec, else 1; one cached grid bound per instantiation
template <typename T, template <typename, int, int> class KS, typename Launch>
static void dispatch_sv(int s, bool vec, Launch&& launch) {
  constexpr int V16 = 16 / sizeof(T);
  if (vec) {
    if (s <= 4) launch(KS<T, 4, V16>{}); else if (s <= 8) launch(KS<T, 8, V16>{}); else launch(KS<T, 16, V16>{});
  } else {
    if (s <= 4) launch(KS<T, 4, 1>{}); else if (s <= 8) launch(KS<T, 8, 1>{}); else launch(KS<T, 16, 1>{});
  }
}

template <typename T, int S, int VW>
struct GammaK {
  static constexpr int vw = VW;
  static constexpr auto fn = gamma_eager_kernel<T, S, VW>;
};

template <typename T>
cudaError_t gamma_eager(const Ctx& c, int n, int s, T* R, const T* V, int64_t ld, int k, const double* gamma) {
  const bool vec = aligned16(R) && aligned16(V) && ((ld * (int64_t)sizeof(T)) % 16) == 0;
  dispatch_sv<T, GammaK>(s, vec, [&](auto kk) {
    using KK = decltype(kk);
    static int cap = max_grid(KK::fn, c);
    const int64_t groups = (n + KK::vw - 1) / KK::vw;
    KK::fn<<<clamp_grid((groups + NT - 1) / NT, cap), NT, 0, c.stream>>>(n, s, R, V, ld, k, gamma);
  });
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// eta step on the top level:  v_q^(k) = r^(k+1) - [V^(k+1)_{0:q-1}, V^(k)_{q:s-1}] eta
// ---------------------------------------------------------------------------
template <typename T, int S, int VW>
__global__ void __launch_bounds__(NT) eta_eager_kernel(int n, int s, const T* __restrict__ R, T* V, int64_t ld,
                                                       int k, int q, const double* __restrict__ eta) {
  __shared__ T e[SMAX];
  if (threadIdx.x < s) e[threadIdx.x] = (T)eta[threadIdx.x];
  __syncthreads();
  const T* r1 = R + (int64_t)(k + 1) * ld;
  const T* vk = V + (int64_t)(k + 1) * s * ld;      // V^(k)
  const T* vk1 = V + (int64_t)(k + 2) * s * ld;     // V^(k+1)
  T* out = V + ((int64_t)(k + 1) * s + q) * ld;     // v_q^(k)
  combine_rows<T, S, VW>(n, s, r1, out, e, [&](int j) { return (j < q ? vk1 : vk) + (int64_t)j * ld; });
}

template <typename T, int S, int VW>
struct EtaK {
  static constexpr int vw = VW;
  static constexpr auto fn = eta_eager_kernel<T, S, VW>;
};

template <typename T>
cudaError_t eta_eager(const Ctx& c, int n, int s, const T* R, T* V, int64_t ld, int k, int q, const double* eta) {
  const bool vec = aligned16(R) && aligned16(V) && ((ld * (int64_t)sizeof(T)) % 16) == 0;
  dispatch_sv<T, EtaK>(s, vec, [&](auto kk) {
    using KK = decltype(kk);
    static int cap = max_grid(KK::fn, c);
    const int64_t groups = (n + KK::vw - 1) / KK::vw;
    KK::fn<<<clamp_grid((groups + NT - 1) / NT, cap), NT, 0, c.stream>>>(n, s, R, V, ld, k, q, eta);
  });
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// updates of level step k on the levels below k, applied once after the q loop
// ---------------------------------------------------------------------------
template <typename T, int S>
__global__ void __launch_bounds__(NT, sizeof(T) == 4 ? 3 : 1) lazy_kernel(int n, int s, T* R, T* V, T* x, int64_t ld, int k,
                                                  const double* __restrict__ gamma,
                                                  const double* __restrict__ eta, int eta_ld) {
  __shared__ T g[SMAX];
  __shared__ T e[SMAX * SMAX];
  if (threadIdx.x < s) g[threadIdx.x] = (T)gamma[threadIdx.x];
  for (int i = threadIdx.x; i < s * s; i += NT) e[(i / s) * SMAX + (i % s)] = (T)eta[(i / s) * eta_ld + (i % s)];
  __syncthreads();
  const int stride = gridDim.x * NT;
  for (int row = blockIdx.x * NT + threadIdx.x; row < n; row += stride) {
    T above[S];
#pragma unroll
    for (int j = 0; j < S; ++j) {
      if (j >= s) break;
      above[j] = V[((int64_t)(k + 1) * s + j) * ld + row];
    }
    T rup = R[(int64_t)k * ld + row];
    for (int i = k - 1; i >= -1; --i) {
      T old[S];
#pragma unroll
      for (int j = 0; j < S; ++j) {
        if (j >= s) break;
        old[j] = V[((int64_t)(i + 1) * s + j) * ld + row];
      }
      // gamma step of this level step, with V^(i) as it was at its start
      if (i >= 0) {
        T ri = R[(int64_t)i * ld + row];
#pragma unroll
        for (int j = 0; j < S; ++j) {
          if (j >= s) break;
          ri -= g[j] * old[j];
        }
        R[(int64_t)i * ld + row] = ri;
        // eta steps of this level: new columns from r^(i+1), new V^(i+1), old V^(i)
#pragma unroll
        for (int q = 0; q < S; ++q) {
          if (q >= s) break;
          T v = rup;
#pragma unroll
          for (int j = 0; j < S; ++j) {
            if (j >= s) break;
            v -= e[q * SMAX + j] * (j < q ? above[j] : old[j]);
          }
          V[((int64_t)(i + 1) * s + q) * ld + row] = v;
          old[q] = v;  // later columns q' > q read old[j] only for j >= q' > q
        }
        rup = ri;
      } else {
        T xv = x[row];
#pragma unroll
        for (int j = 0; j < S; ++j) {
          if (j >= s) break;
          xv += g[j] * old[j];
        }
        x[row] = xv;
#pragma unroll
        for (int q = 0; q < S; ++q) {
          if (q >= s) break;
          T v = rup;
#pragma unroll
          for (int j = 0; j < S; ++j) {
            if (j >= s) break;
            v -= e[q * SMAX + j] * (j < q ? above[j] : old[j]);
          }
          V[(int64_t)q * ld + row] = v;
          old[q] = v;
        }
      }
#pragma unroll
      for (int j = 0; j < S; ++j) {
        if (j >= s) break;
        above[j] = old[j];
      }
    }
  }
}

// The same updates four rows at a time for FP32 (16-byte loads and stores;
// row by row, this kernel is bound by its instruction count, not by HBM).
// Each row sees exactly the operations of lazy_kernel, in its order; the
// n % 4 rows of a ragged tail are done by block 0 one per thread.
__device__ __forceinline__ float4 ld4(const float* p, int64_t g) { return reinterpret_cast<const float4*>(p)[g]; }
__device__ __forceinline__ void st4(float* p, int64_t g, float4 v) { reinterpret_cast<float4*>(p)[g] = v; }
__device__ __forceinline__ void fnma4(float4& a, float c, const float4& b) {
  a.x -= c * b.x;
  a.y -= c * b.y;
  a.z -= c * b.z;
  a.w -= c * b.w;
}
__device__ __forceinline__ void fma4(float4& a, float c, const float4& b) {
  a.x += c * b.x;
  a.y += c * b.y;
  a.z += c * b.z;
  a.w += c * b.w;
}

template <int S>
__global__ void __launch_bounds__(NT, 2) lazy_f32x4_kernel(int n, int s, float* R, float* V, float* x, int64_t ld,
                                                          int k, const double* __restrict__ gamma,
                                                          const double* __restrict__ eta, int eta_ld) {
  __shared__ float g[SMAX];
  __shared__ float e[SMAX * SMAX];
  if (threadIdx.x < s) g[threadIdx.x] = (float)gamma[threadIdx.x];
  for (int i = threadIdx.x; i < s * s; i += NT) e[(i / s) * SMAX + (i % s)] = (float)eta[(i / s) * eta_ld + (i % s)];
  __syncthreads();
  const int64_t groups = n / 4;
  const int64_t stride = (int64_t)gridDim.x * NT;
  for (int64_t gi = blockIdx.x * (int64_t)NT + threadIdx.x; gi < groups; gi += stride) {
    float4 above[S];
#pragma unroll
    for (int j = 0; j < S; ++j) {
      if (j >= s) break;
      above[j] = ld4(V + ((int64_t)(k + 1) * s + j) * ld, gi);
    }
    float4 rup = ld4(R + (int64_t)k * ld, gi);
    for (int i = k - 1; i >= -1; --i) {
      float4 old[S];
#pragma unroll
      for (int j = 0; j < S; ++j) {
        if (j >= s) break;
        old[j] = ld4(V + ((int64_t)(i + 1) * s + j) * ld, gi);
      }
      if (i >= 0) {
        float4 ri = ld4(R + (int64_t)i * ld, gi);
#pragma unroll
        for (int j = 0; j < S; ++j) {
          if (j >= s) break;
          fnma4(ri, g[j], old[j]);
        }
        st4(R + (int64_t)i * ld, gi, ri);
#pragma unroll
        for (int q = 0; q < S; ++q) {
          if (q >= s) break;
          float4 v = rup;
#pragma unroll
          for (int j = 0; j < S; ++j) {
            if (j >= s) break;
            fnma4(v, e[q * SMAX + j], j < q ? above[j] : old[j]);
          }
          st4(V + ((int64_t)(i + 1) * s + q) * ld, gi, v);
          old[q] = v;
        }
        rup = ri;
      } else {
        float4 xv = ld4(x, gi);
#pragma unroll
        for (int j = 0; j < S; ++j) {
          if (j >= s) break;
          fma4(xv, g[j], old[j]);
        }
        st4(x, gi, xv);
#pragma unroll
        for (int q = 0; q < S; ++q) {
          if (q >= s) break;
          float4 v = rup;
#pragma unroll
          for (int j = 0; j < S; ++j) {
            if (j >= s) break;
            fnma4(v, e[q * SMAX + j], j < q ? above[j] : old[j]);
          }
          st4(V + (int64_t)q * ld, gi, v);
          old[q] = v;
        }
      }
#pragma unroll
      for (int j = 0; j < S; ++j) {
        if (j >= s) break;
        above[j] = old[j];
      }
    }
  }
  // ragged tail
  const int64_t row = groups * 4 + threadIdx.x;
  if (blockIdx.x == 0 && row < n) {
    float above[S];
#pragma unroll
    for (int j = 0; j < S; ++j) {
      if (j >= s) break;
      above[j] = V[((int64_t)(k + 1) * s + j) * ld + row];
    }
    float rup = R[(int64_t)k * ld + row];
    for (int i = k - 1; i >= -1; --i) {
      float old[S];
#pragma unroll
      for (int j = 0; j < S; ++j) {
        if (j >= s) break;
        old[j] = V[((int64_t)(i + 1) * s + j) * ld + row];
      }
      if (i >= 0) {
        float ri = R[(int64_t)i * ld + row];
#pragma unroll
        for (int j = 0; j < S; ++j) {
          if (j >= s) break;
          ri -= g[j] * old[j];
        }
        R[(int64_t)i * ld + row] = ri;
#pragma unroll
        for (int q = 0; q < S; ++q) {
          if (q >= s) break;
          float v = rup;
#pragma unroll
          for (int j = 0; j < S; ++j) {
            if (j >= s) break;
            v -= e[q * SMAX + j] * (j < q ? above[j] : old[j]);
          }
          V[((int64_t)(i + 1) * s + q) * ld + row] = v;
          old[q] = v;
        }
        rup = ri;
      } else {
        float xv = x[row];
#pragma unroll
        for (int j = 0; j < S; ++j) {
          if (j >= s) break;
          xv += g[j] * old[j];
        }
        x[row] = xv;
#pragma unroll
        for (int q = 0; q < S; ++q) {
          if (q >= s) break;
          float v = rup;
#pragma unroll
          for (int j = 0; j < S; ++j) {
            if (j >= s) break;
            v -= e[q * SMAX + j] * (j < q ? above[j] : old[j]);
          }
          V[(int64_t)q * ld + row] = v;
          old[q] = v;
        }
      }
#pragma unroll
      for (int j = 0; j < S; ++j) {
        if (j >= s) break;
        above[j] = old[j];
      }
    }
  }
}

template <typename T>
cudaError_t lazy_update(const Ctx& c, int n, int s, T* R, T* V, T* x, int64_t ld, int k, const double* gamma,
                        const double* eta, int eta_ld) {
  if constexpr (sizeof(T) == 4) {
    if (s <= 8 && ld % 4 == 0 && aligned16(R) && aligned16(V) && aligned16(x)) {
      const int64_t need = (n / 4 + NT - 1) / NT;
      if (s <= 4) {
        static int cap = max_grid(lazy_f32x4_kernel<4>, c);
        lazy_f32x4_kernel<4><<<clamp_grid(need, cap), NT, 0, c.stream>>>(n, s, R, V, x, ld, k, gamma, eta, eta_ld);
      } else {
        static int cap = max_grid(lazy_f32x4_kernel<8>, c);
        lazy_f32x4_kernel<8><<<clamp_grid(need, cap), NT, 0, c.stream>>>(n, s, R, V, x, ld, k, gamma, eta, eta_ld);
      }
      return cudaGetLastError();
    }
  }
  const int64_t need = (n + NT - 1) / NT;
  if (s <= 4) {
    static int cap = max_grid(lazy_kernel<T, 4>, c);
    lazy_kernel<T, 4><<<clamp_grid(need, cap), NT, 0, c.stream>>>(n, s, R, V, x, ld, k, gamma, eta, eta_ld);
  } else if (s <= 8) {
    static int cap = max_grid(lazy_kernel<T, 8>, c);
    lazy_kernel<T, 8><<<clamp_grid(need, cap), NT, 0, c.stream>>>(n, s, R, V, x, ld, k, gamma, eta, eta_ld);
  } else {
    static int cap = max_grid(lazy_kernel<T, 16>, c);
    lazy_kernel<T, 16><<<clamp_grid(need, cap), NT, 0, c.stream>>>(n, s, R, V, x, ld, k, gamma, eta, eta_ld);
  }
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// degree-l step with fused projections P^T r, P^T V^(0), r.r
// ---------------------------------------------------------------------------
template <typename T>
struct TauArgs {
  int n, s, ell;
  T* R;
  T* V;
  T* x;
  T* xbak;
  int64_t ld;
  const double* tau;
  const T* P;
  int64_t ldp;
  int do_update, proj;
  int xonly;     // r^(0) is replaced after this step: group 0 updates x (and xbak) only
  DevState* st;
  Epi epi;
  RedScratch rs;
  const T* Pb;   // block-partitioned P (see pblock_col), or NULL
  const T* Pil;  // P interleaved by row (row stride sp), or NULL
  int sp;
  const double* lgamma;   // non-NULL: first the level -1 updates of level step 0 (see lazy_update)
  const double* leta;     //   with gamma_0 and eta rows q at leta + q * leta_ld
  int leta_ld;
};

// L: compile-time bound on the degree l (1, 2, 4 or 8): level arrays of L + 2
// entries, so that the FP32 inner form (l = 1) keeps few registers.
template <typename T, int L>
__global__ void __launch_bounds__(NT, sizeof(T) == 4 ? 3 : 2) tau_kernel(TauArgs<T> a) {
  __shared__ T tau[LMAX];
  __shared__ EpiScratch ew;
  __shared__ double smem_w[NWARP * MAXRED];
  __shared__ double red[MAXRED];
  __shared__ int s_last;
  const int nt = a.s + 1;
  const int t = blockIdx.x % nt;
  const int chunk = blockIdx.x / nt;
  const int nchunks = gridDim.x / nt;
  if (threadIdx.x < a.ell) tau[threadIdx.x] = (T)(a.do_update ? a.tau[threadIdx.x] : 0.0);
  __syncthreads();
  Acc<T, SMAX + 1> acc;   // P^T out in slots 0..s-1, out.out in slot SMAX
  acc.zero();
  const int64_t ld = a.ld;
  const int stride = nchunks * NT;
  // Two rows per iteration; every load of both rows (levels, x, and the P
  // entries of the projection) is issued before any arithmetic, so that
  // enough bytes are in flight per SM (this kernel runs 2 blocks per SM).
  auto load_row = [&](int row, T (&lv)[L + 2], T (&pv)[SMAX], T& xv) {
    if (a.proj) {
      if (a.Pb) {
        pv[0] = __ldg(a.Pb + row);
      } else {
#pragma unroll
        for (int c = 0; c < SMAX; ++c) {
          if (c >= a.s) break;
          pv[c] = __ldg(a.P + (int64_t)c * a.ldp + row);
        }
      }
    }
    if (t == 0) {
      lv[0] = a.R[row];                                               // r^(0)
      if (a.do_update) {
        xv = a.x[row];
#pragma unroll
        for (int i = 1; i <= L; ++i) {
          if (i > a.ell) break;
          lv[i] = a.R[(int64_t)i * ld + row];                         // r^(i)
        }
      }
    } else {
      const int q = t - 1;
      lv[1] = a.V[((int64_t)a.s + q) * ld + row];                     // v_q^(0)
      if (a.do_update) {
        lv[0] = a.V[(int64_t)q * ld + row];                           // v_q^(-1)
#pragma unroll
        for (int i = 1; i <= L; ++i) {
          if (i > a.ell) break;
          lv[i + 1] = a.V[((int64_t)(i + 1) * a.s + q) * ld + row];   // v_q^(i)
        }
      }
    }
  };
  auto update_row = [&](int row, T (&lv)[L + 2], const T (&pv)[SMAX], T xv) {
    T out;
    if (t == 0) {
      T r = lv[0];
      if (a.do_update) {
#pragma unroll
        for (int i = 1; i <= L; ++i) {
          if (i > a.ell) break;
          r -= tau[i - 1] * lv[i];
          xv += tau[i - 1] * lv[i - 1];
        }
        if (!a.xonly) a.R[row] = r;
        a.x[row] = xv;
        if (a.xbak) a.xbak[row] = xv;
      }
      if (a.xonly) return;
      out = r;
    } else {
      const int q = t - 1;
      if (a.do_update) {
        T vnew = lv[1], unew = lv[0];
#pragma unroll
        for (int i = 1; i <= L; ++i) {
          if (i > a.ell) break;
          vnew -= tau[i - 1] * lv[i + 1];
          unew -= tau[i - 1] * lv[i];
        }
        a.V[((int64_t)a.s + q) * ld + row] = vnew;
        a.V[(int64_t)q * ld + row] = unew;
        lv[1] = vnew;
      }
      out = lv[1];
    }
    if (a.proj) {
      if (a.Pb) {
        add_to_slot<SMAX>(acc, pblock_col(row, a.s), out, pv[0]);
      } else {
#pragma unroll
        for (int c = 0; c < SMAX; ++c) {
          if (c >= a.s) break;
          acc.add(c, out, pv[c]);
        }
      }
      if (t == 0) acc.add(SMAX, out, out);
    }
  };
  int row = chunk * NT + threadIdx.x;
  if constexpr (sizeof(T) == 4) {   // FP64 keeps one row: two would spill registers
    for (; row + stride < a.n; row += 2 * stride) {
      T lv0[L + 2], lv1[L + 2], pv0[SMAX], pv1[SMAX];
      T x0 = T(0), x1 = T(0);
      load_row(row, lv0, pv0, x0);
      load_row(row + stride, lv1, pv1, x1);
      update_row(row, lv0, pv0, x0);
      update_row(row + stride, lv1, pv1, x1);
    }
  }
  for (; row < a.n; row += stride) {
    T lv0[L + 2], pv0[SMAX];
    T x0 = T(0);
    load_row(row, lv0, pv0, x0);
    update_row(row, lv0, pv0, x0);
  }
  if (!a.proj || (a.xonly && t == 0)) return;
  const int m = a.s + (t == 0 ? 1 : 0);
  double fin[32];
#pragma unroll
  for (int i = 0; i < 32; ++i) fin[i] = i < SMAX && i < a.s ? acc.get(i < SMAX ? i : 0) : (i == a.s ? acc.get(SMAX) : 0.0);
  block_reduce<32>(fin, m, smem_w, red);
  if (!grid_reduce(a.rs, t, chunk, nchunks, m, red, &s_last)) return;
  if (!groups_done(a.rs, t, a.xonly ? nt - 1 : nt, m, red, &s_last)) return;
  // very last block: scatter all groups' sums into the device state
  DevState* st = a.st;
  for (int i = a.xonly ? a.s + threadIdx.x : threadIdx.x; i < nt * a.s; i += NT) {
    const int tt = i / a.s, cc = i % a.s;
    const double v = __ldcg(a.rs.group_out + tt * MAXRED + cc);
    if (tt == 0)
      st->projR[cc] = v;
    else
      st->projV[(tt - 1) * SMAX + cc] = v;
  }
  if (threadIdx.x == 0 && !a.xonly) st->rr = __ldcg(a.rs.group_out + a.s);
  __threadfence();
  __syncthreads();
  if (threadIdx.x < 32) run_epilogue(a.epi, ew);
}

// ---------------------------------------------------------------------------
// Degree-1 step of the FP32 inner form (l = 1, s <= S <= 8), four rows per
// thread (16-byte loads and stores, as the other FP32 block kernels).  The
// s + 1 vector groups of a row (group 0: r and x; group 1 + q: v_q and u_q)
// are split into T1_G chunks of consecutive groups; warp w of a block takes
// chunk w % T1_G of the 128 rows of its slab w / T1_G, so that a thread keeps
// only its chunk's dots (P^T of its groups' new vectors, and r.r in chunk 0)
// in FP32 registers and issues every load of its groups and of the rows' P
// entries before its first store (the chunks' repeated P loads hit L1).  Each
// dot takes the four rows in order.  Warp sums are FP32 (reduce-scatter over
// rounds of 32 values); the sums over a block's slabs and over the blocks are
// FP64.  One block per SM, so that the last block adds few partials per value
// (FP64 additions are slow on this GPU).  The n % 4 rows of a ragged tail go
// to block 0, one row per lane of each chunk's first-slab warp.  Outputs and
// epilogue as tau_kernel's.
// ---------------------------------------------------------------------------
constexpr int T1_G = 3;
constexpr int T1_SLABS = 4;
constexpr int T1_NW = T1_G * T1_SLABS;
constexpr int T1_NT = 32 * T1_NW;
constexpr int T1_ROWS = 4 * 32 * T1_SLABS;   // rows of a block per iteration

template <int S, bool LZ>
__global__ void __launch_bounds__(T1_NT, 1) tau1_f32_kernel(TauArgs<float> a) {
  constexpr int GPC = (S + 1 + T1_G - 1) / T1_G;   // groups per chunk
  constexpr int NL = GPC * S + 1;                 // a thread's values: P^T of its groups, then r.r
  constexpr int NLP = (NL + 31) / 32 * 32;
  constexpr int NV = S * S + S + 1;               // block values: P^T v_q [q][c], P^T r [c], r.r
  static_assert((int64_t)(MAXBLK + MAXGRP) * NV <= (int64_t)MAXGRP * MAXBLK * MAXRED,
                "partials exceed the reduction scratch");
  __shared__ double wsum[T1_NW][NL];
  __shared__ double bsum[NV];
  __shared__ EpiScratch ew;
  __shared__ int s_last;
  const int s = a.s;
  const int64_t ld = a.ld;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int chunk = w % T1_G, slab = w / T1_G;
  const float tau1 = a.do_update ? (float)a.tau[0] : 0.f;
  float acc[NLP];
#pragma unroll
  for (int i = 0; i < NLP; ++i) acc[i] = 0.f;
  auto col = [&](int g, int which) -> float* {
    // which: 0 = r^(0) / v_q^(0), 1 = x / v_q^(-1), 2 = r^(1) / v_q^(1)
    if (g == 0) return which == 0 ? a.R : (which == 1 ? a.x : a.R + ld);
    const int q = g - 1;
    return a.V + ((which == 0 ? (int64_t)s : (which == 1 ? 0 : (int64_t)2 * s)) + q) * ld;
  };
  // one row quad (4-row group index gi) or, in the tail, one row (float path)
  auto do_rows = [&](auto vec_tag, int64_t gi) {
    using V = decltype(vec_tag);
    constexpr int NR = sizeof(V) / sizeof(float);
    auto ld_v = [&](const float* p) -> V { return reinterpret_cast<const V*>(p)[gi]; };
    auto st_v = [&](float* p, const V& v) { reinterpret_cast<V*>(p)[gi] = v; };
    auto cmp = [](const V& v, int u) -> float { return reinterpret_cast<const float*>(&v)[u]; };
    auto cmpr = [](V& v, int u) -> float& { return reinterpret_cast<float*>(&v)[u]; };
    V pc[S];
    if (a.proj) {
#pragma unroll
      for (int c = 0; c < S; ++c)
        if (c < s) pc[c] = __ldg(reinterpret_cast<const V*>(a.P + (int64_t)c * a.ldp) + gi);
    }
    V v0[GPC], vm[GPC], v1[GPC];
#pragma unroll
    for (int i = 0; i < GPC; ++i) {
      const int g = chunk * GPC + i;
      if (g > s) break;
      v0[i] = ld_v(col(g, 0));
      if (a.do_update) {
        vm[i] = ld_v(col(g, 1));
        v1[i] = ld_v(col(g, 2));
      }
    }
#pragma unroll
    for (int i = 0; i < GPC; ++i) {
      const int g = chunk * GPC + i;
      if (g > s) break;
      V out = v0[i];
      if (a.do_update) {
        V nv = v0[i], nm = vm[i];
#pragma unroll
        for (int u = 0; u < NR; ++u) {
          if (g == 0) {
            cmpr(nv, u) -= tau1 * cmp(v1[i], u);      // r = r^(0) - tau r^(1)
            cmpr(nm, u) += tau1 * cmp(v0[i], u);      // x = x + tau r^(0)
          } else {
            cmpr(nv, u) -= tau1 * cmp(v1[i], u);      // v_q = v_q^(0) - tau v_q^(1)
            cmpr(nm, u) -= tau1 * cmp(v0[i], u);      // u_q = v_q^(-1) - tau v_q^(0)
          }
        }
        st_v(col(g, 0), nv);
        st_v(col(g, 1), nm);
        if (g == 0 && a.xbak) st_v(a.xbak, nm);
        out = nv;
      }
      if (a.proj) {
#pragma unroll
        for (int c = 0; c < S; ++c) {
          if (c >= s) break;
#pragma unroll
          for (int u = 0; u < NR; ++u) acc[i * S + c] = fmaf(cmp(out, u), cmp(pc[c], u), acc[i * S + c]);
        }
        if (g == 0) {
#pragma unroll
          for (int u = 0; u < NR; ++u) acc[NL - 1] = fmaf(cmp(out, u), cmp(out, u), acc[NL - 1]);
        }
      }
    }
  };
  const int64_t quads = a.n / 4;
  const int64_t stride = (int64_t)gridDim.x * (32 * T1_SLABS);
  if constexpr (!LZ) {
    for (int64_t gi = (int64_t)blockIdx.x * (32 * T1_SLABS) + slab * 32 + lane; gi < quads; gi += stride)
      do_rows(float4{}, gi);
    if (blockIdx.x == 0 && slab == 0 && lane < a.n - quads * 4) do_rows(float{}, quads * 4 + lane);
  } else {
    // First the level -1 updates of level step 0 (lazy_update with k = 0):
    // x += V^(-1) gamma_0 and v_q^(-1) = r^(0) - [V^(0)_{0:q-1}, V^(-1)_{q:s-1}] eta_q, each
    // row with lazy_update's operations in its order; every chunk needs all of a row's V^(-1)
    // and V^(0) entries, so the slab's rows go through shared memory, between two barriers
    // of the slab's warps per iteration (n % 4 == 0, no tail).  The updated
    // x and V^(-1) then enter the degree-1 step in registers.
    // two staging buffers (dynamic shared memory), [buffer][slab][column][lane]: the
    // iteration after next writes a buffer only after every warp of the slab has passed
    // the next iteration's barrier, i.e. finished reading it, so one barrier per iteration
    extern __shared__ __align__(16) unsigned char t1_dyn[];
    float4* stgb = reinterpret_cast<float4*>(t1_dyn);
    auto stg = [&](int buf, int c) -> float4& { return stgb[((buf * T1_SLABS + slab) * (2 * S + 1) + c) * 32 + lane]; };
    __shared__ float gs[SMAX];
    __shared__ float es[SMAX * SMAX];
    if (threadIdx.x < s) gs[threadIdx.x] = (float)a.lgamma[threadIdx.x];
    for (int i = threadIdx.x; i < s * s; i += T1_NT) es[(i / s) * SMAX + (i % s)] = (float)a.leta[(i / s) * a.leta_ld + (i % s)];
    __syncthreads();
    // the T1_G warps of a slab meet at their own barrier (ids 1.., T1_G * 32 threads), so
    // that the slabs stream independently
    auto slab_sync = [&]() { asm volatile("bar.sync %0, %1;" ::"r"(1 + slab), "r"(T1_G * 32) : "memory"); };
    int it = 0;
    for (int64_t base = (int64_t)blockIdx.x * (32 * T1_SLABS); base < quads; base += stride, ++it) {
      const int buf = it & 1;
      const int64_t gi = base + slab * 32 + lane;
      const bool act = gi < quads;
      auto ld_v = [&](const float* p) -> float4 { return reinterpret_cast<const float4*>(p)[gi]; };
      auto st_v = [&](float* p, const float4& v) { reinterpret_cast<float4*>(p)[gi] = v; };
      float4 pc[S], v0[GPC], vm[GPC], v1[GPC];
      if (act) {
        if (a.proj) {
#pragma unroll
          for (int c = 0; c < S; ++c)
            if (c < s) pc[c] = __ldg(reinterpret_cast<const float4*>(a.P + (int64_t)c * a.ldp) + gi);
        }
#pragma unroll
        for (int i = 0; i < GPC; ++i) {
          const int g = chunk * GPC + i;
          if (g > s) break;
          v0[i] = ld_v(col(g, 0));
          vm[i] = ld_v(col(g, 1));
          v1[i] = ld_v(col(g, 2));
          if (g == 0)
            stg(buf, 2 * S) = v0[i];          // r^(0)
          else {
            stg(buf, g - 1) = vm[i];          // v_{g-1}^(-1), before the update
            stg(buf, S + g - 1) = v0[i];      // v_{g-1}^(0)
          }
        }
      }
      slab_sync();
      if (act) {
#pragma unroll
        for (int i = 0; i < GPC; ++i) {
          const int g = chunk * GPC + i;
          if (g > s) break;
          if (g == 0) {
            float4 xv = vm[i];
#pragma unroll
            for (int j = 0; j < S; ++j) {
              if (j >= s) break;
              fma4(xv, gs[j], stg(buf, j));
            }
            vm[i] = xv;
          } else {
            const int q = g - 1;
            float4 v = stg(buf, 2 * S);
#pragma unroll
            for (int j = 0; j < S; ++j) {
              if (j >= s) break;
              fnma4(v, es[q * SMAX + j], j < q ? stg(buf, S + j) : stg(buf, j));
            }
            vm[i] = v;
          }
        }
      }
      if (act) {
#pragma unroll
        for (int i = 0; i < GPC; ++i) {
          const int g = chunk * GPC + i;
          if (g > s) break;
          float4 nv = v0[i], nm = vm[i];
          if (g == 0) {
            nv.x -= tau1 * v1[i].x; nv.y -= tau1 * v1[i].y; nv.z -= tau1 * v1[i].z; nv.w -= tau1 * v1[i].w;
            nm.x += tau1 * v0[i].x; nm.y += tau1 * v0[i].y; nm.z += tau1 * v0[i].z; nm.w += tau1 * v0[i].w;
          } else {
            nv.x -= tau1 * v1[i].x; nv.y -= tau1 * v1[i].y; nv.z -= tau1 * v1[i].z; nv.w -= tau1 * v1[i].w;
            nm.x -= tau1 * v0[i].x; nm.y -= tau1 * v0[i].y; nm.z -= tau1 * v0[i].z; nm.w -= tau1 * v0[i].w;
          }
          st_v(col(g, 0), nv);
          st_v(col(g, 1), nm);
          if (g == 0 && a.xbak) st_v(a.xbak, nm);
          if (a.proj) {
#pragma unroll
            for (int c = 0; c < S; ++c) {
              if (c >= s) break;
              acc[i * S + c] = fmaf(nv.x, pc[c].x, acc[i * S + c]);
              acc[i * S + c] = fmaf(nv.y, pc[c].y, acc[i * S + c]);
              acc[i * S + c] = fmaf(nv.z, pc[c].z, acc[i * S + c]);
              acc[i * S + c] = fmaf(nv.w, pc[c].w, acc[i * S + c]);
            }
            if (g == 0) {
              acc[NL - 1] = fmaf(nv.x, nv.x, acc[NL - 1]);
              acc[NL - 1] = fmaf(nv.y, nv.y, acc[NL - 1]);
              acc[NL - 1] = fmaf(nv.z, nv.z, acc[NL - 1]);
              acc[NL - 1] = fmaf(nv.w, nv.w, acc[NL - 1]);
            }
          }
        }
      }
    }
  }
  if (!a.proj) return;
#pragma unroll
  for (int r0 = 0; r0 < NLP; r0 += 32) {
    float v[32];
#pragma unroll
    for (int i = 0; i < 32; ++i) v[i] = acc[r0 + i];
    RedScatterT<float, 32, 16, 32>::run(v, lane);
    const int idx = r0 + rs_index<32>(lane);
    if (idx < NL) wsum[w][idx] = widen_f32(v[0]);
  }
  __syncthreads();
  for (int i = threadIdx.x; i < NV; i += T1_NT) {
    int g, loc;
    if (i < S * S) {
      g = 1 + i / S;
      loc = ((g % GPC) * S) + (i % S);
    } else if (i < S * S + S) {
      g = 0;
      loc = i - S * S;
    } else {
      g = 0;
      loc = NL - 1;
    }
    double sum = 0.0;
#pragma unroll
    for (int sl = 0; sl < T1_SLABS; ++sl) sum += wsum[sl * T1_G + g / GPC][loc];
    bsum[i] = sum;
  }
  __syncthreads();
  // every block's NV sums, added in two stages so that no block adds many:
  // the last block to arrive of each group of GB consecutive blocks adds the
  // group's sums (blocks in order), the last group to finish adds the groups'
  // sums, each value by NJ threads over parts of the groups, then the parts in
  // order.  A fixed order: the result does not depend on which blocks are last.
  constexpr int NJ = T1_NT / NV;
  static_assert(NJ >= 1, "block too small for the value count");
  __shared__ double part[NJ][NV];
  double* bpart = a.rs.partials;                              // [block][NV]
  double* gpart = a.rs.partials + (size_t)MAXBLK * NV;        // [group][NV]
  const int nblk = gridDim.x;
  const int GB = (nblk + MAXGRP - 1) / MAXGRP > 8 ? (nblk + MAXGRP - 1) / MAXGRP : 8;
  const int ngrp = (nblk + GB - 1) / GB, grp = blockIdx.x / GB;
  const int gsize = (grp + 1) * GB <= nblk ? GB : nblk - grp * GB;
  for (int i = threadIdx.x; i < NV; i += T1_NT) bpart[(size_t)blockIdx.x * NV + i] = bsum[i];
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) s_last = atomicAdd(&a.rs.tickets[grp], 1u) == (unsigned)(gsize - 1);
  __syncthreads();
  if (!s_last) return;
  __threadfence();
  for (int i = threadIdx.x; i < NV; i += T1_NT) {
    double v = 0.0;
    int b = grp * GB;
    const int bend = b + gsize;
    for (; b + 8 <= bend; b += 8) {   // eight loads in flight, added in block order
      double r[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) r[u] = __ldcg(bpart + (size_t)(b + u) * NV + i);
#pragma unroll
      for (int u = 0; u < 8; ++u) v += r[u];
    }
    for (; b < bend; ++b) v += __ldcg(bpart + (size_t)b * NV + i);
    gpart[(size_t)grp * NV + i] = v;
  }
  if (threadIdx.x == 0) a.rs.tickets[grp] = 0u;
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) s_last = atomicAdd(&a.rs.tickets[MAXGRP], 1u) == (unsigned)(ngrp - 1);
  __syncthreads();
  if (!s_last) return;
  __threadfence();
  if (threadIdx.x < NJ * NV) {
    const int v = threadIdx.x % NV, j = threadIdx.x / NV;
    double c = 0.0;
    for (int g = j; g < ngrp; g += NJ) c += __ldcg(gpart + (size_t)g * NV + v);
    part[j][v] = c;
  }
  __syncthreads();
  if (threadIdx.x == 0) a.rs.tickets[MAXGRP] = 0u;
  DevState* st = a.st;
  for (int i = threadIdx.x; i < NV; i += T1_NT) {
    double v = part[0][i];
#pragma unroll
    for (int j = 1; j < NJ; ++j) v += part[j][i];
    if (i < S * S) {
      const int q = i / S, c = i % S;
      if (q < s && c < s) st->projV[q * SMAX + c] = v;
    } else if (i < S * S + S) {
      if (i - S * S < s) st->projR[i - S * S] = v;
    } else {
      st->rr = v;
    }
  }
  __threadfence();
  __syncthreads();
  if (threadIdx.x < 32) run_epilogue(a.epi, ew);
}

template <typename T, int L>
static void launch_tau(const Ctx& c, const TauArgs<T>& a) {
  static int cap = max_grid(tau_kernel<T, L>, c, MAXBLK);
  const int nt = a.s + 1;
  int64_t chunks = (a.n + NT - 1) / NT;
  int64_t capc = cap / nt;
  if (capc < 1) capc = 1;
  if (chunks > capc) chunks = capc;
  if (chunks < 1) chunks = 1;
  tau_kernel<T, L><<<(int)(chunks * nt), NT, 0, c.stream>>>(a);
}

template <int S, bool LZ>
static void launch_tau1(const Ctx& c, const TauArgs<float>& a, int64_t need) {
  constexpr size_t dyn = LZ ? sizeof(float4) * 2 * T1_SLABS * (2 * S + 1) * 32 : 0;
  static bool attr = !LZ || cudaFuncSetAttribute(tau1_f32_kernel<S, LZ>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                 (int)dyn) == cudaSuccess;
  (void)attr;
  static int cap = [&] {
    int nb = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, tau1_f32_kernel<S, LZ>, T1_NT, dyn) != cudaSuccess || nb < 1)
      nb = 1;
    return nb * c.sms > MAXBLK ? MAXBLK : nb * c.sms;
  }();
  tau1_f32_kernel<S, LZ><<<clamp_grid(need, cap), T1_NT, dyn, c.stream>>>(a);
}

template <typename T>
static bool tau1_applies(int n, int s, int ell, const T* R, const T* V, const T* x, const T* xbak, int64_t ld,
                         const T* P, int64_t ldp, const T* Pb) {
  (void)n;
  return sizeof(T) == 4 && ell == 1 && Pb == nullptr && s <= 8 && ld % 4 == 0 && ldp % 4 == 0 && aligned16(R) &&
         aligned16(V) && aligned16(x) && aligned16(P) && (xbak == nullptr || aligned16(xbak));
}

template <typename T>
bool tau_fuses_lazy(int n, int s, int ell, const T* R, const T* V, const T* x, const T* xbak, int64_t ld,
                    const T* P, int64_t ldp, const T* Pb) {
  return tau1_applies(n, s, ell, R, V, x, xbak, ld, P, ldp, Pb) && n % 4 == 0;
}

template <typename T>
cudaError_t tau_update(const Ctx& c, int n, int s, int ell, T* R, T* V, T* x, T* xbak, int64_t ld,
                       const double* tau, const T* P, int64_t ldp, int do_update, int proj, DevState* st,
                       Epi epi, const T* Pb, const T* Pil, int sp, const double* lgamma, const double* leta,
                       int leta_ld, int xonly) {
  TauArgs<T> a{n, s, ell, R, V, x, xbak, ld, tau ? tau : st->tau, P, ldp, do_update, proj, xonly, st, epi, c.rs,
               Pb, Pil, sp, lgamma, leta, leta_ld};
  if (xonly && (!do_update || tau1_applies(n, s, ell, R, V, x, xbak, ld, P, ldp, Pb))) return cudaErrorInvalidValue;
  if (lgamma && !(do_update && tau_fuses_lazy(n, s, ell, R, V, x, xbak, ld, P, ldp, Pb)))
    return cudaErrorInvalidValue;
  if constexpr (sizeof(T) == 4) {
    if (tau1_applies(n, s, ell, R, V, x, xbak, ld, P, ldp, Pb)) {
      const int64_t need = ((int64_t)n + T1_ROWS - 1) / T1_ROWS;
      if (s <= 4) {
        if (lgamma) launch_tau1<4, true>(c, a, need); else launch_tau1<4, false>(c, a, need);
      } else {
        if (lgamma) launch_tau1<8, true>(c, a, need); else launch_tau1<8, false>(c, a, need);
      }
      return cudaGetLastError();
    }
  }
  if (ell <= 1)
    launch_tau<T, 1>(c, a);
  else if (ell <= 2)
    launch_tau<T, 2>(c, a);
  else if (ell <= 4)
    launch_tau<T, 4>(c, a);
  else
    launch_tau<T, LMAX>(c, a);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// multi-dot with per-target groups
// ---------------------------------------------------------------------------
template <typename T>
struct MdArgs {
  MdCols<T> cols;
  int n, nt, ny, self, ostride;
  double* out;
  Epi epi;
  RedScratch rs;
};

// C: compile-time bound on ny; U rows per iteration, all their loads issued
// before the first multiply-add (a thread has few rows in flight otherwise:
// the loop is latency-bound).  Each accumulator still takes its rows in
// order and, within a row, the columns in order, so the sums are those of
// one row at a time.
template <typename T, int C, int U>
__global__ void __launch_bounds__(NT, 2) multidot_kernel(MdArgs<T> a) {
  __shared__ EpiScratch ew;
  __shared__ double smem_w[NWARP * MAXRED];
  __shared__ double red[MAXRED];
  __shared__ int s_last;
  const int t = blockIdx.x % a.nt;
  const int chunk = blockIdx.x / a.nt;
  const int nchunks = gridDim.x / a.nt;
  Acc<T, C + 1> acc;  // X_t . Y_c in slots 0..ny-1, X_t . X_t in slot C
  acc.zero();
  const T* xt = a.cols.x[t];
  const int stride = nchunks * NT;
  int row = chunk * NT + threadIdx.x;
  for (; row + (U - 1) * stride < a.n; row += U * stride) {
    T xv[U], yv[U][C];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      xv[u] = __ldg(xt + row + u * stride);
#pragma unroll
      for (int c = 0; c < C; ++c) {
        if (c >= a.ny) break;
        yv[u][c] = __ldg(a.cols.y[c] + row + u * stride);
      }
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
#pragma unroll
      for (int c = 0; c < C; ++c) {
        if (c >= a.ny) break;
        acc.add(c, xv[u], yv[u][c]);
      }
      if (a.self) acc.add(C, xv[u], xv[u]);
    }
  }
  for (; row < a.n; row += stride) {
    const T xv = __ldg(xt + row);
    T yv[C];
#pragma unroll
    for (int c = 0; c < C; ++c) {
      if (c >= a.ny) break;
      yv[c] = __ldg(a.cols.y[c] + row);
    }
#pragma unroll
    for (int c = 0; c < C; ++c) {
      if (c >= a.ny) break;
      acc.add(c, xv, yv[c]);
    }
    if (a.self) acc.add(C, xv, xv);
  }
  const int m = a.ny + a.self;
  if constexpr (sizeof(T) == 4) {
    // FP32 partials: FP32 warp stage over the C + 1 slots only
    constexpr int M = pow2_ge(C + 1);
    float fin[M];
#pragma unroll
    for (int i = 0; i < M; ++i) fin[i] = i < C && i < a.ny ? acc.v[i < C ? i : 0] : (i == a.ny ? acc.v[C] : 0.f);
    block_reduce_f32<M>(fin, m, smem_w, red);
  } else {
    double fin[32];
#pragma unroll
    for (int i = 0; i < 32; ++i)
      fin[i] = i < C && i < a.ny ? acc.get(i < C ? i : 0) : (i == a.ny ? acc.get(C) : 0.0);
    block_reduce<32>(fin, m, smem_w, red);
  }
  if (!grid_reduce(a.rs, t, chunk, nchunks, m, red, &s_last)) return;
  if (!groups_done(a.rs, t, a.nt, m, red, &s_last)) return;
  for (int i = threadIdx.x; i < a.nt * m; i += NT) {
    const int tt = i / m, cc = i % m;
    a.out[tt * a.ostride + cc] = __ldcg(a.rs.group_out + tt * MAXRED + cc);
  }
  __threadfence();
  __syncthreads();
  if (threadIdx.x < 32) run_epilogue(a.epi, ew);
}

// Two blocks per SM whatever the variant's occupancy: the row-to-thread map,
// and with it every partial sum, is then the same for all variants.
template <typename T, int C, int U>
static void launch_multidot(const Ctx& c, const MdArgs<T>& a) {
  const int cap = 2 * c.sms < MAXBLK ? 2 * c.sms : MAXBLK;
  int64_t chunks = (a.n + NT - 1) / NT;
  int64_t capc = cap / a.nt;
  if (capc < 1) capc = 1;
  if (chunks > capc) chunks = capc;
  if (chunks < 1) chunks = 1;
  multidot_kernel<T, C, U><<<(int)(chunks * a.nt), NT, 0, c.stream>>>(a);
}

template <typename T>
cudaError_t multidot(const Ctx& c, int n, const MdCols<T>& cols, int nt, int ny, int self, double* out,
                     int ostride, Epi epi) {
  if (nt < 1 || nt > MD_MAXT || ny < 0 || ny + self > MAXRED || ny > MD_MAXC) return cudaErrorInvalidValue;
  MdArgs<T> a{cols, n, nt, ny, self, ostride, out, epi, c.rs};
  if (ny <= 2)
    launch_multidot<T, 2, 8>(c, a);
  else if (ny <= 4)
    launch_multidot<T, 4, 4>(c, a);
  else if (ny <= 8)
    launch_multidot<T, 8, 2>(c, a);
  else
    launch_multidot<T, MD_MAXC, 1>(c, a);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Arnoldi / Cholesky QR helpers
// ---------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(NT) cols_axpy_kernel(int n, T* w, const T* U, int64_t ld, int nc,
                                                       const double* h) {
  __shared__ double hc[SMAX + 1];
  if (threadIdx.x < nc) hc[threadIdx.x] = h[threadIdx.x];
  __syncthreads();
  const int stride = gridDim.x * NT;
  for (int row = blockIdx.x * NT + threadIdx.x; row < n; row += stride) {
    double v = (double)w[row];
    for (int c = 0; c < nc; ++c) v -= hc[c] * (double)U[(int64_t)c * ld + row];
    w[row] = (T)v;
  }
}

template <typename T>
cudaError_t cols_axpy(const Ctx& c, int n, T* w, const T* U, int64_t ld, int nc, const double* h) {
  static int cap = max_grid(cols_axpy_kernel<T>, c);
  cols_axpy_kernel<T><<<clamp_grid((n + NT - 1) / NT, cap), NT, 0, c.stream>>>(n, w, U, ld, nc, h);
  return cudaGetLastError();
}

template <typename T>
__global__ void __launch_bounds__(NT) scale_rsqrt_kernel(int n, const T* x, T* y, const double* nrm2) {
  const double f = 1.0 / sqrt(*nrm2);
  const int stride = gridDim.x * NT;
  for (int row = blockIdx.x * NT + threadIdx.x; row < n; row += stride) y[row] = (T)((double)x[row] * f);
}

template <typename T>
cudaError_t scale_rsqrt(const Ctx& c, int n, const T* x, T* y, const double* nrm2) {
  static int cap = max_grid(scale_rsqrt_kernel<T>, c);
  scale_rsqrt_kernel<T><<<clamp_grid((n + NT - 1) / NT, cap), NT, 0, c.stream>>>(n, x, y, nrm2);
  return cudaGetLastError();
}

template <typename T>
__global__ void __launch_bounds__(NT) tri_apply_kernel(int n, int s, T* V, T* U, int64_t ld, const double* R) {
  __shared__ double r[SMAX * SMAX];
  for (int i = threadIdx.x; i < s * s; i += NT) r[i] = R[i];
  __syncthreads();
  const int stride = gridDim.x * NT;
  for (int row = blockIdx.x * NT + threadIdx.x; row < n; row += stride) {
    for (int pass = 0; pass < (U ? 2 : 1); ++pass) {
      T* M = pass == 0 ? V : U;
      double v[SMAX];
#pragma unroll
      for (int j = 0; j < SMAX; ++j)
        if (j < s) v[j] = (double)M[(int64_t)j * ld + row];
#pragma unroll
      for (int j = 0; j < SMAX; ++j) {
        if (j < s) {
          double t = v[j];
#pragma unroll
          for (int i = 0; i < SMAX; ++i)
            if (i < j) t -= v[i] * r[i * s + j];
          v[j] = t / r[j * s + j];
          M[(int64_t)j * ld + row] = (T)v[j];
        }
      }
    }
  }
}

template <typename T>
cudaError_t tri_apply(const Ctx& c, int n, int s, T* V, T* U, int64_t ld, const double* R) {
  static int cap = max_grid(tri_apply_kernel<T>, c);
  tri_apply_kernel<T><<<clamp_grid((n + NT - 1) / NT, cap), NT, 0, c.stream>>>(n, s, V, U, ld, R);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// single-thread small solves
// ---------------------------------------------------------------------------
__global__ void small_cholesky_kernel(int s, const double* G, double* R, int* flag) {
  double g[SMAX * SMAX], r[SMAX * SMAX];
  for (int i = 0; i < s * s; ++i) g[i] = G[i];
  const bool ok = cholesky_upper(g, r, s, CHOLQR_REL_TOL);
  for (int i = 0; i < s * s; ++i) R[i] = ok ? r[i] : (i % (s + 1) == 0 ? 1.0 : 0.0);
  if (!ok) *flag |= FLAG_CHOL;
}

cudaError_t small_cholesky(const Ctx& c, int s, const double* G, double* R, int* flag) {
  small_cholesky_kernel<<<1, 1, 0, c.stream>>>(s, G, R, flag);
  return cudaGetLastError();
}

// The warp-parallel elimination that the reduction epilogues use.
__global__ void small_lu_kernel(int n, const double* M, const double* rhs, double* z, int* flag) {
  __shared__ double a[SMAX * SMAX], y[SMAX], l[SMAX];
  for (int i = threadIdx.x; i < n * n; i += 32) a[i] = M[i];
  if (threadIdx.x < n) y[threadIdx.x] = rhs[threadIdx.x];
  __syncwarp();
  const bool ok = warp_lu_solve(a, y, n, l);
  if (threadIdx.x < n) z[threadIdx.x] = y[threadIdx.x];
  if (threadIdx.x == 0) *flag = ok ? 0 : 1;
}

cudaError_t small_lu(const Ctx& c, int n, const double* M, const double* rhs, double* z, int* flag) {
  small_lu_kernel<<<1, 32, 0, c.stream>>>(n, M, rhs, z, flag);
  return cudaGetLastError();
}

__global__ void small_tau_kernel(int ell, const double* G, double* tau) {
  double g[(LMAX + 1) * (LMAX + 1)], t[LMAX], wk[2 * LMAX * LMAX + 2 * LMAX];
  for (int i = 0; i < (ell + 1) * (ell + 1); ++i) g[i] = G[i];
  tau_from_gram(g, ell, t, wk);
  for (int i = 0; i < ell; ++i) tau[i] = t[i];
}

cudaError_t small_tau(const Ctx& c, int ell, const double* G, double* tau) {
  small_tau_kernel<<<1, 1, 0, c.stream>>>(ell, G, tau);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// precision conversions and vector helpers
// ---------------------------------------------------------------------------
__global__ void to_f32_scaled_kernel(int n, const double* x, float* y, double alpha) {
  const int stride = gridDim.x * NT;
  for (int row = blockIdx.x * NT + threadIdx.x; row < n; row += stride) y[row] = (float)(x[row] * alpha);
}

cudaError_t to_f32_scaled(const Ctx& c, int n, const double* x, float* y, double alpha) {
  static int cap = max_grid(to_f32_scaled_kernel, c);
  to_f32_scaled_kernel<<<clamp_grid((n + NT - 1) / NT, cap), NT, 0, c.stream>>>(n, x, y, alpha);
  return cudaGetLastError();
}

__global__ void axpy_f32_into_f64_kernel(int n, const float* x, double* y, double alpha) {
  const int stride = gridDim.x * NT;
  for (int row = blockIdx.x * NT + threadIdx.x; row < n; row += stride) y[row] += alpha * (double)x[row];
}

cudaError_t axpy_f32_into_f64(const Ctx& c, int n, const float* x, double* y, double alpha) {
  static int cap = max_grid(axpy_f32_into_f64_kernel, c);
  axpy_f32_into_f64_kernel<<<clamp_grid((n + NT - 1) / NT, cap), NT, 0, c.stream>>>(n, x, y, alpha);
  return cudaGetLastError();
}

__global__ void axpby_f64_kernel(int n, double alpha, const double* x, double beta, const double* z, double* y) {
  const int stride = gridDim.x * NT;
  for (int row = blockIdx.x * NT + threadIdx.x; row < n; row += stride) y[row] = alpha * x[row] + beta * z[row];
}

cudaError_t axpby_f64(const Ctx& c, int n, double alpha, const double* x, double beta, const double* z,
                      double* y) {
  static int cap = max_grid(axpby_f64_kernel, c);
  axpby_f64_kernel<<<clamp_grid((n + NT - 1) / NT, cap), NT, 0, c.stream>>>(n, alpha, x, beta, z, y);
  return cudaGetLastError();
}

__global__ void f64_to_f32_n_kernel(int64_t n, const double* x, float* y, double alpha) {
  const int64_t stride = (int64_t)gridDim.x * NT;
  for (int64_t i = blockIdx.x * (int64_t)NT + threadIdx.x; i < n; i += stride) y[i] = (float)(x[i] * alpha);
}

cudaError_t f64_to_f32_n(const Ctx& c, int64_t n, const double* x, float* y, double alpha) {
  static int cap = max_grid(f64_to_f32_n_kernel, c);
  f64_to_f32_n_kernel<<<clamp_grid((n + NT - 1) / NT, cap), NT, 0, c.stream>>>(n, x, y, alpha);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// explicit instantiations
// ---------------------------------------------------------------------------
#define MSK_INST(T)                                                                                       \
  template cudaError_t multidot<T>(const Ctx&, int, const MdCols<T>&, int, int, int, double*, int, Epi);  \
  template cudaError_t gamma_eager<T>(const Ctx&, int, int, T*, const T*, int64_t, int, const double*);   \
  template cudaError_t eta_eager<T>(const Ctx&, int, int, const T*, T*, int64_t, int, int, const double*); \
  template cudaError_t lazy_update<T>(const Ctx&, int, int, T*, T*, T*, int64_t, int, const double*,      \
                                      const double*, int);                                                \
  template cudaError_t tau_update<T>(const Ctx&, int, int, int, T*, T*, T*, T*, int64_t, const double*,   \
                                     const T*, int64_t, int, int, DevState*, Epi, const T*, const T*,    \
                                     int, const double*, const double*, int, int);                       \
  template bool tau_fuses_lazy<T>(int, int, int, const T*, const T*, const T*, const T*, int64_t, const T*,  \
                                  int64_t, const T*);                                                    \
  template cudaError_t cols_axpy<T>(const Ctx&, int, T*, const T*, int64_t, int, const double*);          \
  template cudaError_t scale_rsqrt<T>(const Ctx&, int, const T*, T*, const double*);                      \
  template cudaError_t tri_apply<T>(const Ctx&, int, int, T*, T*, int64_t, const double*);
MSK_INST(double)
MSK_INST(float)

}  // namespace msk

// Learned initial guess: a small 3D CNN trained on the solver's own
// (b^(i+1), x^(i)) -> x^(i+1) - x^(i) pairs (fed as the channels
// r0 = b^(i+1) - A x^(i) and x^(i)), with hand-written bfloat16 kernels
// that accumulate in FP32.  Not part of the paper: the workload's learned-x0
// form.  The network: 3x3x3 convolutions 2 -> 16 -> 16 -> 16 -> 1, "same"
// zero padding, bias, GELU (erf form) after the first three layers.
//
// Precision: weights, biases and every convolution operand (input volumes,
// hidden activations, gradients fed to the next contraction) are rounded to
// bfloat16 (round to nearest even); products are accumulated in FP32; the FP32
// master weights, Adam moments, pre-activations and the network output stay
// FP32.  Volumes are [batch][channel][z][y][x] with x fastest, as the solver's
// vectors.  Weight tap (dz, dy, dx) multiplies the input voxel at offset
// (dz-1, dy-1, dx-1) (cross-correlation).
//
// All reductions (weight gradients, loss, normalisation) are deterministic:
// per-block partials summed in block order.

#include <cuda_bf16.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include <cuda.h>          // CUtensorMap and its enums (types only: the encoder is fetched at run time)
#include <cudaTypedefs.h>

#include "launch.h"
#include "msstab.h"

namespace mcnn {

constexpr int NL = 4;
constexpr int CI_[NL] = {2, 16, 16, 16};
constexpr int CO_[NL] = {16, 16, 16, 1};
constexpr int WG_MAX_BLOCKS = 1024;   // rows of the weight-gradient partials (two blocks per SM are launched)

__host__ __device__ constexpr int n_params() {
  return 2 * 16 * 27 + 16 + 16 * 16 * 27 + 16 + 16 * 16 * 27 + 16 + 16 * 1 * 27 + 1;
}
inline int w_offset(int l) {
  int o = 0;
  for (int i = 0; i < l; ++i) o += CO_[i] * CI_[i] * 27 + CO_[i];
  return o;
}

enum Mode { FWD_HIDDEN = 0, FWD_LAST = 1, BWD_DATA = 2, INFER_HIDDEN = 3 };

__device__ __forceinline__ float gelu(float z) { return 0.5f * z * (1.0f + erff(z * 0.70710678118654752f)); }
__device__ __forceinline__ float gelu_grad(float z) {
  return 0.5f * (1.0f + erff(z * 0.70710678118654752f)) + z * expf(-0.5f * z * z) * 0.39894228040143268f;
}
__device__ __forceinline__ float bf(float v) { return __bfloat162float(__float2bfloat16_rn(v)); }

struct Dims {
  int X, Y, Z;
  __host__ __device__ int64_t vol() const { return (int64_t)X * Y * Z; }
};

// Layout of the bfloat16 volumes the convolutions read and write ("half-
// major"): channel c of voxel p of batch entry b of a C-channel batch sits at
// element ((b * halves(C) + c / 8) * vol + p) * 8 + c % 8.  Each voxel's 8
// channels of one half are one 16-byte row (zero channels when C < 8), so the
// halo of a tile is one tiled tensor copy per half that lands in shared memory
// already in the K-major operand layout of the MMAs.  FP32 volumes (pre-
// activations, outputs, targets) stay channel-planar.
__host__ __device__ constexpr int halves(int c) { return (c + 7) / 8; }

__device__ __forceinline__ uint32_t bf16_bits(float v) {
  return (uint32_t)__bfloat16_as_ushort(__float2bfloat16_rn(v));
}

// ---------------------------------------------------------------------------
// The 3x3x3 convolutions on the tensor cores (tcgen05), as an implicit GEMM:
// an output tile of 128 voxels (8 x-consecutive by 16 y-consecutive in one z
// plane) is the M dimension, the 16 output channels N, and each of the 27
// taps one K = 16 step over the 16 input channels (layers with fewer channels
// are padded with zero channels):
// D[m][co] = sum_tap sum_ci A_tap[m][ci] W_tap[ci][co].  Both operands sit in
// shared memory K-major without swizzle (core matrices of 8 rows x 16 bytes):
// the input halo (10 x 18 x 3 voxels) as two halves of 8 channels,
// [half][voxel][8], so that A_tap is the halo shifted by the tap -- 16 bytes
// between x-consecutive voxels, 160 bytes (one halo row) between the 8-row
// groups, 8640 bytes (one half) between the two K halves; the weights as
// [tap][half][co][8] -- 128 bytes between co groups, 256 between halves.
// A block is a two-stage pipeline: one thread of warp 4 issues the halo copy
// of the next tile and the 27 MMAs of a tile (kind::f16, BF16 operands, FP32
// accumulator of 128 lanes x 16 columns in tensor memory, two accumulators)
// and commits them to an mbarrier; warps 0-3 read their 32 rows of the other
// accumulator with tcgen05.ld for the epilogue (bias, GELU or GELU', bf16
// rounding) meanwhile.  Blocks are persistent (weights, tensor memory and the
// mbarriers set up once, tiles taken in a grid-stride loop).  A wait that runs
// out raises *flag and ends the block's loop; the copies and MMAs in flight get
// a second bounded wait, and tensor memory is freed before the block exits.
// ---------------------------------------------------------------------------
constexpr int CTX = 8, CTY = 16;
constexpr int CHX = CTX + 2, CHY = CTY + 2, CHZ = 3, CHV = CHX * CHY * CHZ;   // 540 halo voxels
constexpr int TC_A_HALF = CHV * 16;                 // bytes of one channel half of the halo (8640)
constexpr int TC_A_HSTRIDE = 8704;                  // the halves 128-byte aligned (tensor-copy destinations)
constexpr int TC_A_BYTES = 2 * TC_A_HSTRIDE;
constexpr int TC_B_BYTES = 27 * 512;                // weights of the 27 taps
constexpr int TC_SMEM = TC_B_BYTES + 2 * TC_A_BYTES + 128;   // weights, two halo stages, alignment slack
constexpr int TC_THREADS = 160;                     // warps 0-3: the epilogue; warp 4: copies and MMAs
constexpr long long TC_WAIT_LIMIT = 1LL << 22;
static_assert(TC_A_HALF <= TC_A_HSTRIDE && TC_A_HSTRIDE % 128 == 0, "halo halves");

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// shared-memory matrix descriptor: start, leading (K) and stride (M/N) byte
// offsets, descriptor version 1, no swizzle
__device__ __forceinline__ uint64_t umma_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
  return (uint64_t)((saddr >> 4) & 0x3FFF) | ((uint64_t)((lbo >> 4) & 0x3FFF) << 16) |
         ((uint64_t)((sbo >> 4) & 0x3FFF) << 32) | (1ull << 46);
}

__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t phase) {
  uint32_t done = 0;
  for (long long it = 0; it < TC_WAIT_LIMIT && !done; ++it)
    asm volatile("{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
                 "selp.u32 %0, 1, 0, p;\n\t}\n"
                 : "=r"(done) : "r"(bar), "r"(phase));
  return done != 0;
}

template <int CI, int CO, int MODE>
__global__ void __launch_bounds__(TC_THREADS) conv_tc_kernel(const __grid_constant__ CUtensorMap halo_map, Dims d,
                                                             int B, const __nv_bfloat16* __restrict__ w,
                                                             const float* __restrict__ bias, float* __restrict__ z,
                                                             __nv_bfloat16* __restrict__ act,
                                                             const float* __restrict__ zaux, int* flag) {
  extern __shared__ __align__(1024) unsigned char tsm_raw[];
  // the tensor copies want 128-byte aligned destinations
  unsigned char* tsm = tsm_raw + ((128u - (smem_u32(tsm_raw) & 127u)) & 127u);
  unsigned char* Bs = tsm;                  // weights
  unsigned char* As = tsm + TC_B_BYTES;     // halo stage s at As + s * TC_A_BYTES
  __shared__ __align__(8) uint64_t full[2];    // the halo copies of stage s have landed
  __shared__ __align__(8) uint64_t done[2];    // the MMAs into accumulator s (reading stage s) are complete
  __shared__ __align__(8) uint64_t freed[2];   // the four epilogue warps have read accumulator s
  __shared__ uint32_t tslot;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int tilesx = (d.X + CTX - 1) / CTX, tilesy = (d.Y + CTY - 1) / CTY;
  const int tiles = tilesx * tilesy * d.Z;
  const int jobs = tiles * B;
  const int nj = jobs > (int)blockIdx.x ? (jobs - 1 - (int)blockIdx.x) / (int)gridDim.x + 1 : 0;
  const int64_t vol = d.vol();
  // weights once per block: w[co][ci][tap] -> tap * 512 + (ci / 8) * 256 + co * 16 + (ci % 8) * 2,
  // zero for the padding channels (ci >= CI or co >= CO).  w is first copied
  // as it is into a halo stage (free until the first tile) with independent
  // 16-byte loads, all in flight at once (one element per load took a global
  // round trip per element, the bulk of a launch on a small volume), then
  // rearranged from there.
  constexpr int WBYTES = CO * CI * 27 * 2;
  static_assert(WBYTES % 16 == 0 && WBYTES <= TC_A_BYTES, "weights staged in a halo stage");
  {
    constexpr int NV = WBYTES / 16, PER = (NV + TC_THREADS - 1) / TC_THREADS;
    uint4 v[PER];
#pragma unroll
    for (int u = 0; u < PER; ++u)
      if (u * TC_THREADS + tid < NV) v[u] = __ldg(reinterpret_cast<const uint4*>(w) + u * TC_THREADS + tid);
#pragma unroll
    for (int u = 0; u < PER; ++u)
      if (u * TC_THREADS + tid < NV) reinterpret_cast<uint4*>(As)[u * TC_THREADS + tid] = v[u];
  }
  __syncthreads();
  const __nv_bfloat16* ws = reinterpret_cast<const __nv_bfloat16*>(As);
  for (int i = tid; i < 16 * 16 * 27; i += TC_THREADS) {
    const int co = i / (16 * 27), r = i % (16 * 27), ci = r / 27, tap = r % 27;
    const __nv_bfloat16 v = (co < CO && ci < CI) ? ws[(co * CI + ci) * 27 + tap] : __float2bfloat16_rn(0.f);
    *reinterpret_cast<__nv_bfloat16*>(Bs + tap * 512 + (ci >> 3) * 256 + co * 16 + (ci & 7) * 2) = v;
  }
  __syncthreads();   // the halo stages are overwritten below
  // fewer than 9 input channels: the second half of each halo stage stays zero
  // (the weights of those channels are zero too, and 0 * 0 keeps the sums finite)
  if (halves(CI) < 2)
    for (int st = 0; st < 2; ++st)
      for (int i = tid; i < TC_A_HALF / 16; i += TC_THREADS)
        reinterpret_cast<uint4*>(As + st * TC_A_BYTES + TC_A_HSTRIDE)[i] = make_uint4(0u, 0u, 0u, 0u);
  if (tid == 0) {
    for (int st = 0; st < 2; ++st) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(&full[st])), "r"(1));
      asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(&done[st])), "r"(1));
      asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(&freed[st])), "r"(4));
    }
    asm volatile("fence.mbarrier_init.release.cluster;");
  }
  asm volatile("fence.proxy.async.shared::cta;");
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tslot)),
                 "r"(32));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
  const uint32_t taddr = tslot;
  if (warp == 4) {
    // ---- producer: one thread issues the halo copies (one tile ahead) and
    // the 27 MMAs of each tile into accumulator i % 2 ----
    if (lane == 0) {
      // D f32, A and B bf16, both K-major, N = 16, M = 128
      const uint32_t idesc = (1u << 4) | (1u << 7) | (1u << 10) | ((16u >> 3) << 17) | ((128u >> 4) << 24);
      auto load = [&](int st, int job) {
        const int b = job / tiles, tile = job % tiles;
        const int tz0 = tile / (tilesx * tilesy);
        const int ty0 = ((tile / tilesx) % tilesy) * CTY;
        const int tx0 = (tile % tilesx) * CTX;
        // halo: one tiled tensor copy per channel half, box (8 channels, 10 x,
        // 18 y, 3 z) at (0, tx0 - 1, ty0 - 1, tz0 - 1, b * halves + half); the
        // copy fills out-of-range voxels with zeros
        const uint32_t bar = smem_u32(&full[st]);
        constexpr uint32_t bytes = (uint32_t)halves(CI) * TC_A_HALF;
        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
#pragma unroll
        for (int hf = 0; hf < halves(CI); ++hf)
          asm volatile(
              "cp.async.bulk.tensor.5d.shared::cluster.global.tile.mbarrier::complete_tx::bytes "
              "[%0], [%1, {%2, %3, %4, %5, %6}], [%7];"
              ::"r"(smem_u32(As + st * TC_A_BYTES + hf * TC_A_HSTRIDE)),
                "l"(reinterpret_cast<uint64_t>(&halo_map)), "r"(0), "r"(tx0 - 1), "r"(ty0 - 1), "r"(tz0 - 1),
                "r"(b * halves(CI) + hf), "r"(bar)
              : "memory");
      };
      int ok = 1;
      uint32_t lph[2] = {0u, 0u}, mph[2] = {0u, 0u}, fph[2] = {0u, 0u};
      bool lout[2] = {false, false}, mout[2] = {false, false};
      if (nj > 0) {
        load(0, blockIdx.x);
        lout[0] = true;
      }
      for (int i = 0; i < nj; ++i) {
        const int st = i & 1;
        if (i + 1 < nj) {
          if (mout[st ^ 1]) {   // the MMAs of tile i - 1 read the other stage
            if (!mbar_wait(smem_u32(&done[st ^ 1]), mph[st ^ 1])) {
              ok = 0;
              break;
            }
            mph[st ^ 1] ^= 1u;
            mout[st ^ 1] = false;
          }
          load(st ^ 1, blockIdx.x + (i + 1) * gridDim.x);
          lout[st ^ 1] = true;
        }
        if (!mbar_wait(smem_u32(&full[st]), lph[st])) {
          ok = 0;
          break;
        }
        lph[st] ^= 1u;
        lout[st] = false;
        if (i >= 2) {   // the epilogue of tile i - 2 has read accumulator st
          if (!mbar_wait(smem_u32(&freed[st]), fph[st])) {
            ok = 0;
            break;
          }
          fph[st] ^= 1u;
        }
        asm volatile("tcgen05.fence::after_thread_sync;");
        const uint32_t a0 = smem_u32(As + st * TC_A_BYTES), b0 = smem_u32(Bs);
        for (int tap = 0; tap < 27; ++tap) {
          const int dz = tap / 9, dy = (tap / 3) % 3, dx = tap % 3;
          const uint64_t ad = umma_desc(a0 + ((dz * CHY + dy) * CHX + dx) * 16, TC_A_HSTRIDE, CHX * 16);
          const uint64_t bd = umma_desc(b0 + tap * 512, 256, 128);
          const uint32_t accum = tap > 0;
          asm volatile("{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
                       "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n"
                       ::"r"(taddr + st * 16), "l"(ad), "l"(bd), "r"(idesc), "r"(accum));
        }
        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
                     ::"r"(smem_u32(&done[st])));
        mout[st] = true;
      }
      if (!ok) {
        // give the copies and MMAs in flight a second bounded wait before leaving
        atomicOr(flag, 1);
        for (int st = 0; st < 2; ++st) {
          if (lout[st]) mbar_wait(smem_u32(&full[st]), lph[st]);
          if (mout[st]) mbar_wait(smem_u32(&done[st]), mph[st]);
        }
      }
    }
  } else {
    // ---- epilogue warps: thread m holds output voxel m of each tile ----
    uint32_t dph[2] = {0u, 0u};
    for (int i = 0; i < nj; ++i) {
      const int st = i & 1;
      const int job = blockIdx.x + i * gridDim.x;
      const int b = job / tiles, tile = job % tiles;
      const int tz0 = tile / (tilesx * tilesy);
      const int ty0 = ((tile / tilesx) % tilesy) * CTY;
      const int tx0 = (tile % tilesx) * CTX;
      const int m = warp * 32 + lane;
      const int gx = tx0 + (m & 7), gy = ty0 + (m >> 3), gz = tz0;
      const bool inside = gx < d.X && gy < d.Y;
      const int64_t p = ((int64_t)gz * d.Y + gy) * d.X + gx;
      const int64_t ob = (int64_t)b * CO * vol;
      // the backward mode's pre-activations are loaded while the MMAs run
      float za[MODE == BWD_DATA ? CO : 1];
      if constexpr (MODE == BWD_DATA) {
#pragma unroll
        for (int co = 0; co < CO; ++co) za[co] = inside ? __ldg(zaux + ob + (int64_t)co * vol + p) : 0.f;
      }
      // one decision per warp (tcgen05.ld below is warp-collective)
      const bool got = __all_sync(0xffffffffu, mbar_wait(smem_u32(&done[st]), dph[st]));
      dph[st] ^= 1u;
      if (!got) {
        if (lane == 0) atomicOr(flag, 1);
        break;
      }
      asm volatile("tcgen05.fence::after_thread_sync;");
      uint32_t r[16];
      asm volatile(
          "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
          : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
            "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
          : "r"(taddr + ((uint32_t)(warp * 32) << 16) + (uint32_t)(st * 16)));
      asm volatile("tcgen05.wait::ld.sync.aligned;");
      asm volatile("tcgen05.fence::before_thread_sync;");
      __syncwarp();
      if (lane == 0) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(&freed[st])) : "memory");
      if (inside) {
        // bf16 outputs of the 16 channels, as two 16-byte half-major rows
        uint32_t packed[8];
#pragma unroll
        for (int co = 0; co < 16; ++co) {
          float out = 0.f;
          if (co < CO) {
            const float acc = __uint_as_float(r[co]) + (bias ? bias[co] : 0.f);
            const int64_t o = ob + (int64_t)co * vol + p;
            if (MODE == FWD_HIDDEN) {
              z[o] = acc;
              out = gelu(acc);
            } else if (MODE == FWD_LAST) {
              z[o] = acc;
            } else if (MODE == INFER_HIDDEN) {
              out = gelu(acc);
            } else {
              out = acc * gelu_grad(za[MODE == BWD_DATA ? co : 0]);
            }
          }
          if (co % 2 == 0)
            packed[co / 2] = bf16_bits(out);
          else
            packed[co / 2] |= bf16_bits(out) << 16;
        }
        if constexpr (MODE != FWD_LAST) {
          static_assert(MODE == FWD_LAST || CO == 16, "bf16 outputs have 16 channels");
          uint4* dst = reinterpret_cast<uint4*>(act);
          dst[((int64_t)b * 2 + 0) * vol + p] = make_uint4(packed[0], packed[1], packed[2], packed[3]);
          dst[((int64_t)b * 2 + 1) * vol + p] = make_uint4(packed[4], packed[5], packed[6], packed[7]);
        }
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(32));
}

// The tensor map of a half-major volume (B entries of nh halves): dimensions
// (8 channels, x, y, z, entry * nh + half), innermost first; box (8, bx, by,
// bz, 1): (8, 10, 18, 3, 1) is one halo half of a convolution tile, (8, 8, 16,
// 1, 1) one half of the tile itself; out-of-range elements read as zero.  The encoder is
// the driver's, fetched through the runtime (no link against the driver).
static cudaError_t half_major_map(CUtensorMap* m, const __nv_bfloat16* in, Dims d, int B, int nh, int bx, int by,
                                  int bz) {
  static PFN_cuTensorMapEncodeTiled_v12000 enc = nullptr;
  if (!enc) {
    void* fn = nullptr;
    cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
    const cudaError_t e = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q);
    if (e != cudaSuccess) return e;
    if (q != cudaDriverEntryPointSuccess || !fn) return cudaErrorNotSupported;
    enc = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
  }
  const cuuint64_t dims[5] = {8, (cuuint64_t)d.X, (cuuint64_t)d.Y, (cuuint64_t)d.Z, (cuuint64_t)B * nh};
  const cuuint64_t strides[4] = {16, 16ull * d.X, 16ull * d.X * d.Y, 16ull * d.X * d.Y * d.Z};
  const cuuint32_t box[5] = {8, (cuuint32_t)bx, (cuuint32_t)by, (cuuint32_t)bz, 1};
  const cuuint32_t estr[5] = {1, 1, 1, 1, 1};
  const CUresult r = enc(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 5, const_cast<__nv_bfloat16*>(in), dims, strides, box,
                         estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                         CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

static cudaError_t halo_map(CUtensorMap* m, const __nv_bfloat16* in, Dims d, int B, int nh) {
  return half_major_map(m, in, d, B, nh, CHX, CHY, CHZ);
}

template <int CI, int CO, int MODE>
static cudaError_t conv_tc(cudaStream_t st, const __nv_bfloat16* in, Dims d, int B, const __nv_bfloat16* w,
                           const float* bias, float* z, __nv_bfloat16* act, const float* zaux, int* flag) {
  // tensor-copy base and the weights' vector loads: 16-byte aligned
  if ((((uintptr_t)in | (uintptr_t)w) & 15u) != 0) return cudaErrorMisalignedAddress;
  CUtensorMap map;
  {
    const cudaError_t e = halo_map(&map, in, d, B, halves(CI));
    if (e != cudaSuccess) return e;
  }
  static bool attr = false;
  if (!attr) {
    cudaError_t e = cudaFuncSetAttribute(conv_tc_kernel<CI, CO, MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize, TC_SMEM);
    if (e != cudaSuccess) return e;
    attr = true;
  }
  static int cap = 0;
  if (!cap) {
    int dev = 0, sms = 0, nb = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess)
      e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, conv_tc_kernel<CI, CO, MODE>, TC_THREADS, (size_t)TC_SMEM);
    if (e != cudaSuccess) return e;
    // the occupancy query answers one block per SM for this kernel, although
    // shared memory (the binding limit) admits four; blocks beyond the
    // resident ones only queue (no block waits on another), so launch as many
    // as shared memory admits
    const int by_smem = (227 * 1024) / (TC_SMEM + 2048);
    nb = std::max(nb, std::min(8, by_smem));
    cap = nb * (sms > 0 ? sms : 1);
  }
  const int64_t jobs = (int64_t)((d.X + CTX - 1) / CTX) * ((d.Y + CTY - 1) / CTY) * d.Z * B;
  const int grid = (int)(jobs < cap ? jobs : cap);   // persistent blocks, tiles in a grid-stride loop
  conv_tc_kernel<CI, CO, MODE><<<grid, TC_THREADS, TC_SMEM, st>>>(map, d, B, w, bias, z, act, zaux, flag);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Layers with one or two input channels (the network's input layer and the
// backward-data pass of its one-channel output layer): the taps are packed
// into K.  Each thread writes its voxel's row of an im2col tile, K element
// k = tap * CI + ci (27 CI values, zero up to the next multiple of 16), so a
// tile takes ceil(27 CI / 16) MMAs (4 for two channels, 2 for one) instead of
// 27 with 16 - CI zero channels each: at N = 16 an MMA costs several times
// its arithmetic, and the MMA count bounded these layers.  Both operands
// K-major without swizzle: the tile [m/8][k/8][m%8][k%8] (128 bytes per
// 8-element K chunk, 1024 per group of 8 rows), the weights [co/8][k/8][co%8]
// [k%8] likewise.  Single-stage persistent blocks (as many per SM as shared
// memory admits overlap one another's copies, MMAs and epilogues); bounded
// waits; tensor memory freed on every path.
// ---------------------------------------------------------------------------
constexpr int TK_A_BYTES = 16 * 1024;     // 128 rows x 64 K elements
constexpr int TK_B_BYTES = 2 * 1024;      // 16 output channels x 64 K elements
constexpr int TK_SMEM = TC_A_HSTRIDE + TK_A_BYTES + TK_B_BYTES + 128;

template <int CI, int CO, int MODE>
__global__ void __launch_bounds__(128) conv_k_kernel(const __grid_constant__ CUtensorMap halo_map, Dims d, int B,
                                                     const __nv_bfloat16* __restrict__ w,
                                                     const float* __restrict__ bias, float* __restrict__ z,
                                                     __nv_bfloat16* __restrict__ act,
                                                     const float* __restrict__ zaux, int* flag) {
  static_assert(CI <= 2 && CO == 16, "taps packed into K: one or two input channels, 16 outputs");
  constexpr int KE = 27 * CI, KS = (KE + 15) / 16, KC = 2 * KS;   // K elements, MMAs, 8-element chunks
  extern __shared__ __align__(1024) unsigned char ksm_raw[];
  unsigned char* ksm = ksm_raw + ((128u - (smem_u32(ksm_raw) & 127u)) & 127u);
  unsigned char* Hs = ksm;                   // halo (channel half 0), tensor-copy destination
  unsigned char* As = ksm + TC_A_HSTRIDE;    // im2col tile
  unsigned char* Bs = As + TK_A_BYTES;       // weights
  __shared__ __align__(8) uint64_t mbar;
  __shared__ __align__(8) uint64_t tbar;
  __shared__ uint32_t tslot;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int tilesx = (d.X + CTX - 1) / CTX, tilesy = (d.Y + CTY - 1) / CTY;
  const int tiles = tilesx * tilesy * d.Z;
  const int64_t vol = d.vol();
  // weights: w[co][ci][tap] copied as it is into the halo buffer with 16-byte
  // loads, then rearranged to B[k][co], k = tap * CI + ci (zero for k >= KE)
  constexpr int WBYTES = CO * CI * 27 * 2;
  static_assert(WBYTES % 16 == 0 && WBYTES <= TC_A_HSTRIDE, "weights staged in the halo buffer");
  {
    constexpr int NV = WBYTES / 16, PER = (NV + 127) / 128;
    uint4 v[PER];
#pragma unroll
    for (int u = 0; u < PER; ++u)
      if (u * 128 + tid < NV) v[u] = __ldg(reinterpret_cast<const uint4*>(w) + u * 128 + tid);
#pragma unroll
    for (int u = 0; u < PER; ++u)
      if (u * 128 + tid < NV) reinterpret_cast<uint4*>(Hs)[u * 128 + tid] = v[u];
  }
  __syncthreads();
  {
    const __nv_bfloat16* ws = reinterpret_cast<const __nv_bfloat16*>(Hs);
    for (int i = tid; i < 16 * KC * 8; i += 128) {
      const int co = i / (KC * 8), k = i % (KC * 8), tap = k / CI, ci = k % CI;
      const __nv_bfloat16 v = k < KE ? ws[(co * CI + ci) * 27 + tap] : __float2bfloat16_rn(0.f);
      *reinterpret_cast<__nv_bfloat16*>(Bs + (co >> 3) * 1024 + (k >> 3) * 128 + (co & 7) * 16 + (k & 7) * 2) = v;
    }
  }
  __syncthreads();   // the halo buffer is overwritten below
  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(&mbar)), "r"(1));
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(&tbar)), "r"(1));
    asm volatile("fence.mbarrier_init.release.cluster;");
  }
  asm volatile("fence.proxy.async.shared::cta;");
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tslot)),
                 "r"(32));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
  const uint32_t taddr = tslot;
  // D f32, A and B bf16, both K-major, N = 16, M = 128
  const uint32_t idesc = (1u << 4) | (1u << 7) | (1u << 10) | ((16u >> 3) << 17) | ((128u >> 4) << 24);
  const int m = tid, mx = m & 7, my = m >> 3;
  bool ok = true;
  uint32_t phase = 0;
  for (int job = blockIdx.x; job < tiles * B && ok; job += gridDim.x, phase ^= 1u) {
    const int b = job / tiles, tile = job % tiles;
    const int tz0 = tile / (tilesx * tilesy);
    const int ty0 = ((tile / tilesx) % tilesy) * CTY;
    const int tx0 = (tile % tilesx) * CTX;
    // halo: one tiled tensor copy (channel half 0) at (0, tx0 - 1, ty0 - 1,
    // tz0 - 1, b); out-of-range voxels read as zero.  The previous tile's
    // im2col is complete (block barrier below), so the buffer is free.
    if (tid == 0) {
      asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(&tbar)), "r"(TC_A_HALF)
                   : "memory");
      asm volatile(
          "cp.async.bulk.tensor.5d.shared::cluster.global.tile.mbarrier::complete_tx::bytes "
          "[%0], [%1, {%2, %3, %4, %5, %6}], [%7];"
          ::"r"(smem_u32(Hs)), "l"(reinterpret_cast<uint64_t>(&halo_map)), "r"(0), "r"(tx0 - 1), "r"(ty0 - 1),
            "r"(tz0 - 1), "r"(b), "r"(smem_u32(&tbar))
          : "memory");
    }
    const bool halo_ok = mbar_wait(smem_u32(&tbar), phase);
    // the previous tile's MMAs (waited on) and tensor-memory reads are done
    asm volatile("tcgen05.fence::before_thread_sync;");
    const int all_loaded = __syncthreads_and((int)halo_ok);
    asm volatile("tcgen05.fence::after_thread_sync;");
    if (!all_loaded) {
      if (tid == 0) {
        atomicOr(flag, 1);
        mbar_wait(smem_u32(&tbar), phase);
      }
      __syncthreads();
      ok = false;
      break;
    }
    // this thread's im2col row: 16-bit K elements, two per word
    uint32_t kw[KC * 4];
#pragma unroll
    for (int j = 0; j < KC * 4; ++j) {
      uint32_t v = 0u;
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int k = 2 * j + h, tap = k / CI, ci = k % CI;
        if (k < KE) {
          const int dz = tap / 9, dy = (tap / 3) % 3, dx = tap % 3;
          const uint32_t e = *reinterpret_cast<const uint16_t*>(
              Hs + ((dz * CHY + my + dy) * CHX + mx + dx) * 16 + ci * 2);
          v |= e << (16 * h);
        }
      }
      kw[j] = v;
    }
#pragma unroll
    for (int c = 0; c < KC; ++c)
      *reinterpret_cast<uint4*>(As + (m >> 3) * 1024 + c * 128 + (m & 7) * 16) =
          make_uint4(kw[4 * c], kw[4 * c + 1], kw[4 * c + 2], kw[4 * c + 3]);
    // the tile, written by threads, is read by the tensor cores
    asm volatile("fence.proxy.async.shared::cta;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    if (tid == 0) {
      const uint32_t a0 = smem_u32(As), b0 = smem_u32(Bs);
#pragma unroll
      for (int kk = 0; kk < KS; ++kk) {
        const uint64_t ad = umma_desc(a0 + kk * 256, 128, 1024);
        const uint64_t bd = umma_desc(b0 + kk * 256, 128, 1024);
        asm volatile("{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
                     "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n"
                     ::"r"(taddr), "l"(ad), "l"(bd), "r"(idesc), "r"(kk > 0 ? 1 : 0));
      }
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
                   ::"r"(smem_u32(&mbar)));
    }
    const int gx = tx0 + mx, gy = ty0 + my, gz = tz0;
    const bool inside = gx < d.X && gy < d.Y;
    const int64_t p = ((int64_t)gz * d.Y + gy) * d.X + gx;
    const int64_t ob = (int64_t)b * CO * vol;
    float za[MODE == BWD_DATA ? CO : 1];
    if constexpr (MODE == BWD_DATA) {
#pragma unroll
      for (int co = 0; co < CO; ++co) za[co] = inside ? __ldg(zaux + ob + (int64_t)co * vol + p) : 0.f;
    }
    const bool done = mbar_wait(smem_u32(&mbar), phase);
    const int all_done = __syncthreads_and((int)done);
    asm volatile("tcgen05.fence::after_thread_sync;");
    if (!all_done) {
      if (tid == 0) atomicOr(flag, 1);
      ok = false;
      break;
    }
    uint32_t r[16];
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, "
                 "[%16];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
                   "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]),
                   "=r"(r[15])
                 : "r"(taddr + ((uint32_t)(warp * 32) << 16)));
    asm volatile("tcgen05.wait::ld.sync.aligned;");
    if (inside) {
      uint32_t packed[8];
#pragma unroll
      for (int co = 0; co < 16; ++co) {
        const float acc = __uint_as_float(r[co]) + (bias ? bias[co] : 0.f);
        const int64_t o = ob + (int64_t)co * vol + p;
        float out;
        if (MODE == FWD_HIDDEN) {
          z[o] = acc;
          out = gelu(acc);
        } else if (MODE == INFER_HIDDEN) {
          out = gelu(acc);
        } else {
          out = acc * gelu_grad(za[MODE == BWD_DATA ? co : 0]);
        }
        if (co % 2 == 0)
          packed[co / 2] = bf16_bits(out);
        else
          packed[co / 2] |= bf16_bits(out) << 16;
      }
      static_assert(MODE != FWD_LAST, "the packed-K layers have 16 bf16 outputs");
      uint4* dst = reinterpret_cast<uint4*>(act);
      dst[((int64_t)b * 2 + 0) * vol + p] = make_uint4(packed[0], packed[1], packed[2], packed[3]);
      dst[((int64_t)b * 2 + 1) * vol + p] = make_uint4(packed[4], packed[5], packed[6], packed[7]);
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(32));
}

template <int CI, int CO, int MODE>
static cudaError_t conv_k(cudaStream_t st, const __nv_bfloat16* in, Dims d, int B, const __nv_bfloat16* w,
                          const float* bias, float* z, __nv_bfloat16* act, const float* zaux, int* flag) {
  if ((((uintptr_t)in | (uintptr_t)w) & 15u) != 0) return cudaErrorMisalignedAddress;
  CUtensorMap map;
  {
    const cudaError_t e = halo_map(&map, in, d, B, halves(CI));
    if (e != cudaSuccess) return e;
  }
  static int cap = 0;
  if (!cap) {
    int dev = 0, sms = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(conv_k_kernel<CI, CO, MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize, TK_SMEM);
    if (e != cudaSuccess) return e;
    // as many blocks per SM as shared memory admits (at most 8: 32 tensor-memory columns each)
    cap = std::min(8, (227 * 1024) / (TK_SMEM + 2048)) * (sms > 0 ? sms : 1);
  }
  const int64_t jobs = (int64_t)((d.X + CTX - 1) / CTX) * ((d.Y + CTY - 1) / CTY) * d.Z * B;
  const int grid = (int)(jobs < cap ? jobs : cap);
  conv_k_kernel<CI, CO, MODE><<<grid, 128, TK_SMEM, st>>>(map, d, B, w, bias, z, act, zaux, flag);
  return cudaGetLastError();
}

// Every layer on the tensor cores: fewer than 16 input or output channels
// (2 -> 16, 16 -> 1, 1 -> 16) are padded with zero channels to K = 16 per tap
// and N = 16 (the MMAs cost little; the halo loads and the stores skip the
// padding).  Modes: FWD_HIDDEN writes z (FP32) and act = bf16(gelu(z));
// FWD_LAST z only; INFER_HIDDEN act only; BWD_DATA act = bf16(sum *
// gelu'(zaux)) (the gradient of the previous layer's pre-activation; w then
// holds that layer's weights transposed and flipped).  w: [CO][CI][27] bf16,
// bias: CO floats or NULL.
template <int CI, int CO, int MODE>
static cudaError_t conv(cudaStream_t st, const __nv_bfloat16* in, Dims d, int B, const __nv_bfloat16* w,
                        const float* bias, float* z, __nv_bfloat16* act, const float* zaux, int* flag) {
  static_assert(CI <= 16 && CO <= 16, "the tensor-core convolution takes up to 16 channels");
  if constexpr (CI <= 2)
    return conv_k<CI, CO, MODE>(st, in, d, B, w, bias, z, act, zaux, flag);
  else
    return conv_tc<CI, CO, MODE>(st, in, d, B, w, bias, z, act, zaux, flag);
}

// ---------------------------------------------------------------------------
// Weight and bias gradients on the tensor cores.  For each tap the weight
// gradient is a product with the voxels as the contraction:
//   dW_tap[co][ci] = sum_p a[ci][p + tap - 1] g[co][p],
// transposed: D = A_s . G with A_s (shifted input channels x voxels) and G
// (voxels x output channels).  Both operands are read MN-major, straight from
// the half-major tiles that the tensor copies land (8 consecutive voxels of
// one channel half are one 128-byte core matrix: 8 K-rows of 8 channels):
//   A_s:  the halo of the forward convolution; its 16 M-direction core
//         matrices 16 bytes (one voxel) apart, so that core n is the window
//         shifted by n voxels: n = dx + 10 dy' (a halo row is 10 voxels) puts
//         the taps dx = 0..2 of two consecutive dy in one MMA (cores 0..2 and
//         10..12, rows 8n .. 8n + 7 = the 8 channels of the half); the other
//         cores are products never read.  K: one halo row (160 bytes) per 8
//         voxels;
//   G:    the output-gradient tile [half][y 16][x 8][8]: 128 bytes per 8
//         voxels (K), 2048 bytes per channel half (N = 16).
// An MMA (kind::f16, M = 128, N = 16, K = 16) covers two tile rows; per K step
// 13 MMAs: 3 dz x 2 channel halves x (dy 0-1, dy 2), and the bias gradient
// (a 128 x 16 block of ones times G).  The issue of an MMA costs about the
// same whatever its shape (measured: M = 64..128, N = 16..128), so the taps
// share MMAs rather than padding the 16 output channels to M = 128.  The 13
// accumulators (16 columns each) stay in tensor memory over all tiles of the
// block; one thread issues the tensor copies of the next tile (two stages)
// and the MMAs of the current one.  Then each warp reads its lanes and writes
// the entries they hold of the block's partial sums: dW as [co][ci][tap], then
// the CO bias sums db[co] = sum_p g[co][p].  Waits are bounded: one that runs
// out raises *flag, the copies and MMAs in flight get a second bounded wait,
// and tensor memory is freed on every path.
// ---------------------------------------------------------------------------
constexpr int WG_G_HALF = CTX * CTY * 16;         // 2048: one channel half of the G tile
constexpr int WG_G_BYTES = 2 * WG_G_HALF;
constexpr int WG_STAGE = WG_G_BYTES + TC_A_BYTES; // G tile, then the halo (both halves)
constexpr int WG_ONES = 2 * WG_STAGE;             // 128 x 16 bf16 ones (4096 bytes)
constexpr int WG_HALO_REACH = 8704 + (2 * CHY + 2 * 7 + 2) * CHX * 16 + 15 * 16 + CHX * 16 + 128;
constexpr int WG_SMEM = 80 * 1024;                // at most two blocks per SM (256 tensor-memory columns each)
constexpr int WG_NCOL = 256;
constexpr int WG_REGIONS = 13;                    // 12 tap groups and the bias
static_assert(WG_STAGE % 128 == 0 && WG_STAGE + WG_G_BYTES + WG_HALO_REACH <= WG_ONES + 4096 &&
                  WG_ONES + 4096 + 128 <= WG_SMEM && WG_REGIONS * 16 <= WG_NCOL,
              "weight-gradient shared and tensor memory");

__device__ __forceinline__ void tma_5d(uint32_t dst, const CUtensorMap* map, int c1, int c2, int c3, int c4,
                                       uint32_t bar) {
  asm volatile(
      "cp.async.bulk.tensor.5d.shared::cluster.global.tile.mbarrier::complete_tx::bytes "
      "[%0], [%1, {%2, %3, %4, %5, %6}], [%7];"
      ::"r"(dst), "l"(reinterpret_cast<uint64_t>(map)), "r"(0), "r"(c1), "r"(c2), "r"(c3), "r"(c4), "r"(bar)
      : "memory");
}

__device__ __forceinline__ void mma_f16(uint32_t d, uint64_t ad, uint64_t bd, uint32_t idesc, uint32_t accum) {
  asm volatile("{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
               "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n"
               ::"r"(d), "l"(ad), "l"(bd), "r"(idesc), "r"(accum));
}

template <int CI, int CO>
__global__ void __launch_bounds__(128) wgrad_tc_kernel(const __grid_constant__ CUtensorMap halo_map,
                                                       const __grid_constant__ CUtensorMap g_map, Dims d, int B,
                                                       float* __restrict__ partials, int* flag) {
  constexpr int NV = CO * CI * 27 + CO;
  constexpr int HI = halves(CI);
  extern __shared__ __align__(1024) unsigned char wsm_raw[];
  unsigned char* sm = wsm_raw + ((128u - (smem_u32(wsm_raw) & 127u)) & 127u);
  __shared__ __align__(8) uint64_t lbar[2];   // tensor copies of a stage
  __shared__ __align__(8) uint64_t mbar[2];   // MMAs that read a stage
  __shared__ uint32_t tslot;
  __shared__ int s_ok;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int tilesx = (d.X + CTX - 1) / CTX, tilesy = (d.Y + CTY - 1) / CTY;
  const int tiles = tilesx * tilesy * d.Z;
  const int jobs = tiles * B;
  const int nj = jobs > (int)blockIdx.x ? (jobs - 1 - (int)blockIdx.x) / (int)gridDim.x + 1 : 0;
  // the ones of the bias gradient; a channel half of G that no copy fills is zero
  for (int i = tid; i < 2048; i += 128) reinterpret_cast<uint16_t*>(sm + WG_ONES)[i] = 0x3F80u;
  if (halves(CO) < 2)
    for (int st = 0; st < 2; ++st)
      for (int i = tid; i < WG_G_HALF / 16; i += 128)
        reinterpret_cast<uint4*>(sm + st * WG_STAGE + WG_G_HALF)[i] = make_uint4(0u, 0u, 0u, 0u);
  if (tid == 0) {
    for (int st = 0; st < 2; ++st) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(&lbar[st])), "r"(1));
      asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(&mbar[st])), "r"(1));
    }
    asm volatile("fence.mbarrier_init.release.cluster;");
  }
  asm volatile("fence.proxy.async.shared::cta;");
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tslot)),
                 "r"(WG_NCOL));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
  const uint32_t taddr = tslot;
  if (tid == 0) {
    // D f32, A and B bf16, both MN-major (bits 15, 16), N = 16, M = 128
    const uint32_t idesc = (1u << 4) | (1u << 7) | (1u << 10) | (1u << 15) | (1u << 16) | ((16u >> 3) << 17) |
                           ((128u >> 4) << 24);
    // MN-major descriptors: leading byte offset = the K step, stride byte
    // offset = the M/N step.  The start address is the low field in 16-byte
    // units (shared addresses stay below 2^18 bytes), so a descriptor moves
    // by adding the byte offset / 16.
    const uint64_t odesc = umma_desc(smem_u32(sm + WG_ONES), 128, 256);
    auto load = [&](int st, int job) {
      const int b = job / tiles, tile = job % tiles;
      const int tz0 = tile / (tilesx * tilesy);
      const int ty0 = ((tile / tilesx) % tilesy) * CTY;
      const int tx0 = (tile % tilesx) * CTX;
      const uint32_t bar = smem_u32(&lbar[st]);
      constexpr uint32_t bytes = (uint32_t)halves(CO) * WG_G_HALF + (uint32_t)HI * TC_A_HALF;
      asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
      unsigned char* base = sm + st * WG_STAGE;
#pragma unroll
      for (int hf = 0; hf < halves(CO); ++hf)
        tma_5d(smem_u32(base + hf * WG_G_HALF), &g_map, tx0, ty0, tz0, b * halves(CO) + hf, bar);
#pragma unroll
      for (int hf = 0; hf < HI; ++hf)
        tma_5d(smem_u32(base + WG_G_BYTES + hf * TC_A_HSTRIDE), &halo_map, tx0 - 1, ty0 - 1, tz0 - 1,
               b * HI + hf, bar);
    };
    int ok = 1;
    uint32_t lph[2] = {0u, 0u}, mph[2] = {0u, 0u};
    bool lout[2] = {false, false}, mout[2] = {false, false};
    int last = -1;   // stage of the latest committed MMAs
    if (nj > 0) {
      load(0, blockIdx.x);
      lout[0] = true;
    }
    for (int i = 0; i < nj; ++i) {
      const int st = i & 1;
      if (i + 1 < nj) {
        if (mout[st ^ 1]) {   // the MMAs of job i - 1 read the other stage
          if (!mbar_wait(smem_u32(&mbar[st ^ 1]), mph[st ^ 1])) {
            ok = 0;
            break;
          }
          mph[st ^ 1] ^= 1u;
          mout[st ^ 1] = false;
        }
        load(st ^ 1, blockIdx.x + (i + 1) * gridDim.x);
        lout[st ^ 1] = true;
      }
      if (!mbar_wait(smem_u32(&lbar[st]), lph[st])) {
        ok = 0;
        break;
      }
      lph[st] ^= 1u;
      lout[st] = false;
      asm volatile("tcgen05.fence::after_thread_sync;");
      const uint32_t g0 = smem_u32(sm + st * WG_STAGE), h0 = g0 + WG_G_BYTES;
      const uint64_t gdesc = umma_desc(g0, 128, WG_G_HALF);
      const uint64_t hdesc = umma_desc(h0, CHX * 16, 16);
#pragma unroll 1
      for (int j2 = 0; j2 < CTY / 2; ++j2) {
        const uint64_t gd = gdesc + (uint64_t)(j2 * 16);        // two tile rows: 256 bytes
        const uint32_t accum = (i > 0 || j2 > 0) ? 1u : 0u;
#pragma unroll
        for (int r = 0; r < 12; ++r) {
          // region r = (dz * 2 + half) * 2 + dyg: taps dz, dy = 2 dyg + (0, 1), dx = 0..2
          const int dz = r / 4, hf = (r / 2) % 2, dyg = r % 2;
          if (hf >= HI) continue;
          const uint64_t ad = hdesc + (uint64_t)((hf * TC_A_HSTRIDE) / 16 + (dz * CHY + 2 * j2 + 2 * dyg) * CHX);
          mma_f16(taddr + r * 16, ad, gd, idesc, accum);
        }
        mma_f16(taddr + 12 * 16, odesc, gd, idesc, accum);
      }
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
                   ::"r"(smem_u32(&mbar[st])));
      mout[st] = true;
      last = st;
    }
    // the MMAs complete in order: the latest commit covers the earlier ones
    if (last >= 0 && mout[last] && !mbar_wait(smem_u32(&mbar[last]), mph[last])) ok = 0;
    if (!ok) {
      atomicOr(flag, 1);
      for (int st = 0; st < 2; ++st)
        if (lout[st]) mbar_wait(smem_u32(&lbar[st]), lph[st]);
    }
    s_ok = ok;
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
  if (s_ok) {
    // row m of a region: core n = m / 8 (the window shifted by dx + 10 dy'),
    // channel m % 8 of the half; warp w holds rows 32 w .. 32 w + 31
    float* out = partials + (size_t)blockIdx.x * NV;
    const int m = warp * 32 + lane, n = m / 8, dx = n % 10, dyp = n / 10;
    for (int r = 0; r < WG_REGIONS; ++r) {
      if (r < 12 && r / 2 % 2 >= HI) continue;   // a channel half the layer does not have (uniform)
      uint32_t v[16];
      asm volatile(
          "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
          : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
            "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
          : "r"(taddr + ((uint32_t)(warp * 32) << 16) + (uint32_t)(r * 16)));
      asm volatile("tcgen05.wait::ld.sync.aligned;");
      if (r == 12) {
        if (m == 0)
#pragma unroll
          for (int co = 0; co < CO; ++co) out[CO * CI * 27 + co] = nj > 0 ? __uint_as_float(v[co]) : 0.f;
        continue;
      }
      const int dz = r / 4, hf = (r / 2) % 2, dyg = r % 2;
      const int ci = hf * 8 + m % 8, dy = 2 * dyg + dyp;
      if (n < 16 && dx < 3 && dy < 3 && dyp < 2 && ci < CI) {
        const int tap = (dz * 3 + dy) * 3 + dx;
#pragma unroll
        for (int co = 0; co < CO; ++co) out[(co * CI + ci) * 27 + tap] = nj > 0 ? __uint_as_float(v[co]) : 0.f;
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(WG_NCOL));
}

// The tensor-core weight gradient of a layer: a (input activations, CI
// channels) and g (gradient of the pre-activations, CO channels), both half-
// major bf16.  At most max_blocks blocks (the partials buffer's rows); the
// number launched goes to *nblocks.
template <int CI, int CO>
static cudaError_t wgrad_tc(cudaStream_t st, const __nv_bfloat16* a, const __nv_bfloat16* g, Dims d, int B,
                            float* partials, int max_blocks, int* nblocks, int* flag) {
  if ((((uintptr_t)a | (uintptr_t)g) & 15u) != 0) return cudaErrorMisalignedAddress;
  CUtensorMap amap, gmap;
  {
    cudaError_t e = half_major_map(&amap, a, d, B, halves(CI), CHX, CHY, CHZ);
    if (e == cudaSuccess) e = half_major_map(&gmap, g, d, B, halves(CO), CTX, CTY, 1);
    if (e != cudaSuccess) return e;
  }
  static int sms = 0;
  if (!sms) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(wgrad_tc_kernel<CI, CO>, cudaFuncAttributeMaxDynamicSharedMemorySize, WG_SMEM);
    if (e != cudaSuccess) {
      sms = 0;
      return e;
    }
  }
  const int64_t jobs = (int64_t)((d.X + CTX - 1) / CTX) * ((d.Y + CTY - 1) / CTY) * d.Z * B;
  int64_t grid = jobs < 2 * sms ? jobs : 2 * sms;   // two blocks per SM: two threads issue MMAs
  if (grid > max_blocks) grid = max_blocks;
  if (grid < 1) grid = 1;
  wgrad_tc_kernel<CI, CO><<<(int)grid, 128, WG_SMEM, st>>>(amap, gmap, d, B, partials, flag);
  *nblocks = (int)grid;
  return cudaGetLastError();
}

// grad[i] = sum over blocks of partials[blk][i] (FP64), in a fixed order: the
// blocks in RED_CHUNKS consecutive ranges summed in block order (one
// grid row per range), then the range sums in range order
constexpr int RED_CHUNKS = 32;
__global__ void reduce_partials_chunk_kernel(const float* partials, int nblocks, int nv, double* chunk_sums) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nv) return;
  const int per = (nblocks + RED_CHUNKS - 1) / RED_CHUNKS;
  const int b0 = blockIdx.y * per, b1 = min(nblocks, b0 + per);
  double s = 0.0;
  for (int b = b0; b < b1; ++b) s += (double)partials[(size_t)b * nv + i];
  chunk_sums[(size_t)blockIdx.y * nv + i] = s;
}

__global__ void reduce_partials_kernel(const double* chunk_sums, int nv, float* grad) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nv) return;
  double s = 0.0;
  for (int c = 0; c < RED_CHUNKS; ++c) s += chunk_sums[(size_t)c * nv + i];
  grad[i] = (float)s;
}

// ---------------------------------------------------------------------------
// loss, weight handling, data movement
// ---------------------------------------------------------------------------

// g = bf16(2 (out - t) / count); per-block partial sums of (out - t)^2
__global__ void loss_kernel(const float* out, const float* t, int64_t n, double inv_count, __nv_bfloat16* g,
                            double* partial) {
  __shared__ double red[32];
  double s = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const float dlt = out[i] - t[i];
    s += (double)dlt * dlt;
    reinterpret_cast<uint4*>(g)[i] = make_uint4(bf16_bits((float)(2.0 * (double)dlt * inv_count)), 0u, 0u, 0u);
  }
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double tot = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) tot += red[w];
    partial[blockIdx.x] = tot;
  }
}

// Operator-weighted loss: s = K * (out - t) on each D^3 crop (cross-
// correlation, zero outside the crop), per-block partial sums of s^2.
__global__ void stencil_fwd_kernel(const float* out, const float* t, int B, int D, const float* k27, float* s,
                                   double* partial) {
  __shared__ double red[32];
  __shared__ float k[27];
  if (threadIdx.x < 27) k[threadIdx.x] = k27[threadIdx.x];
  __syncthreads();
  const int64_t n = (int64_t)B * D * D * D;
  double acc2 = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const int x = (int)(i % D), y = (int)((i / D) % D), z = (int)((i / ((int64_t)D * D)) % D);
    const int64_t base = i - x - (int64_t)y * D - (int64_t)z * D * D;
    float v = 0.f;
    for (int dz = -1; dz <= 1; ++dz)
      for (int dy = -1; dy <= 1; ++dy)
        for (int dx = -1; dx <= 1; ++dx) {
          const float kk = k[(dz + 1) * 9 + (dy + 1) * 3 + (dx + 1)];
          const int zz = z + dz, yy = y + dy, xx = x + dx;
          if (kk == 0.f || zz < 0 || zz >= D || yy < 0 || yy >= D || xx < 0 || xx >= D) continue;
          const int64_t j = base + ((int64_t)zz * D + yy) * D + xx;
          v = fmaf(kk, out[j] - t[j], v);
        }
    s[i] = v;
    acc2 += (double)v * v;
  }
  for (int o = 16; o > 0; o >>= 1) acc2 += __shfl_xor_sync(0xffffffffu, acc2, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc2;
  __syncthreads();
  if (threadIdx.x == 0) {
    double tot = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) tot += red[w];
    partial[blockIdx.x] = tot;
  }
}

// g = bf16((2 / count) K^T * s): the gradient of mean(s^2) with respect to out
__global__ void stencil_bwd_kernel(const float* s, int B, int D, const float* k27, double inv_count,
                                   __nv_bfloat16* g) {
  __shared__ float k[27];
  if (threadIdx.x < 27) k[threadIdx.x] = k27[threadIdx.x];
  __syncthreads();
  const int64_t n = (int64_t)B * D * D * D;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const int x = (int)(i % D), y = (int)((i / D) % D), z = (int)((i / ((int64_t)D * D)) % D);
    const int64_t base = i - x - (int64_t)y * D - (int64_t)z * D * D;
    float v = 0.f;
    for (int dz = -1; dz <= 1; ++dz)
      for (int dy = -1; dy <= 1; ++dy)
        for (int dx = -1; dx <= 1; ++dx) {
          const float kk = k[(dz + 1) * 9 + (dy + 1) * 3 + (dx + 1)];
          const int zz = z - dz, yy = y - dy, xx = x - dx;   // the rows whose tap (dz, dy, dx) reads i
          if (kk == 0.f || zz < 0 || zz >= D || yy < 0 || yy >= D || xx < 0 || xx >= D) continue;
          v = fmaf(kk, s[base + ((int64_t)zz * D + yy) * D + xx], v);
        }
    reinterpret_cast<uint4*>(g)[i] = make_uint4(bf16_bits((float)(2.0 * (double)v * inv_count)), 0u, 0u, 0u);
  }
}

// bf16 copies of the weights (and transposed, flipped copies for the data
// gradient: wt[ci][co][26 - tap] = w[co][ci][tap]) and bf16-rounded biases
__global__ void quantize_kernel(const float* theta, __nv_bfloat16* wq, __nv_bfloat16* wt, float* bq, int ci, int co) {
  const int nw = co * ci * 27;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < nw + co; i += gridDim.x * blockDim.x) {
    if (i < nw) {
      const __nv_bfloat16 v = __float2bfloat16_rn(theta[i]);
      wq[i] = v;
      const int o = i / (ci * 27), r = i % (ci * 27), c = r / 27, tap = r % 27;
      wt[(c * co + o) * 27 + (26 - tap)] = v;
    } else {
      bq[i - nw] = bf(theta[i]);
    }
  }
}

__global__ void adam_kernel(float* theta, float* m, float* v, const float* grad, int n, float lr, float b1, float b2,
                            float eps, float c1, float c2) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float g = grad[i];
  const float mi = b1 * m[i] + (1.f - b1) * g;
  const float vi = b2 * v[i] + (1.f - b2) * g * g;
  m[i] = mi;
  v[i] = vi;
  theta[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
}

// batch of crops of pair k: in[b] = (bf16(sr_k r0), bf16(s_x x)), t[b] = c sr_k delta
// (sr_k = 1 / RMS of pair k's residual: the map r0 -> delta is linear, so each
// pair is presented at unit residual scale)
__global__ void gather_kernel(const float* pin, const float* pt, int64_t N, Dims full, const int* origins, int D,
                              const float* pair_sr, float s1, float c, __nv_bfloat16* in, float* t) {
  const int b = blockIdx.y;
  const int k = origins[4 * b], oz = origins[4 * b + 1], oy = origins[4 * b + 2], ox = origins[4 * b + 3];
  const float s0 = pair_sr[k], st = c * pair_sr[k];
  const int64_t v3 = (int64_t)D * D * D;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < v3; i += (int64_t)gridDim.x * blockDim.x) {
    const int x = (int)(i % D), y = (int)((i / D) % D), z = (int)(i / ((int64_t)D * D));
    const int64_t g = ((int64_t)(oz + z) * full.Y + (oy + y)) * full.X + (ox + x);
    const uint32_t c01 = bf16_bits(s0 * pin[((int64_t)k * 2 + 0) * N + g]) |
                         (bf16_bits(s1 * pin[((int64_t)k * 2 + 1) * N + g]) << 16);
    reinterpret_cast<uint4*>(in)[(int64_t)b * v3 + i] = make_uint4(c01, 0u, 0u, 0u);   // half-major, C = 2
    t[(int64_t)b * v3 + i] = st * pt[(int64_t)k * N + g];
  }
}

// store a training pair: the input channels (r0, x_prev) and the target
// x_next - x_prev, FP32
__global__ void pair_kernel(const double* r0, const double* xp, const double* xn, int64_t N, float* pin, float* pt) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x) {
    pin[i] = (float)r0[i];
    pin[N + i] = (float)xp[i];
    pt[i] = (float)(xn[i] - xp[i]);
  }
}

// inference input: bf16(s0 r0), bf16(s1 x_prev)
__global__ void infer_in_kernel(const double* r0, const double* xp, int64_t N, float s0, float s1,
                                __nv_bfloat16* in) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x) {
    const uint32_t c01 = bf16_bits(s0 * (float)r0[i]) | (bf16_bits(s1 * (float)xp[i]) << 16);
    reinterpret_cast<uint4*>(in)[i] = make_uint4(c01, 0u, 0u, 0u);   // half-major, C = 2
  }
}

// a batch of FP32 two-channel volumes [B][2][v3] as the half-major bf16 input
__global__ void pack_input_kernel(const float* x, int B, int64_t v3, __nv_bfloat16* in) {
  const int64_t n = (int64_t)B * v3;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t b = i / v3, p = i % v3;
    const uint32_t c01 = bf16_bits(x[(b * 2 + 0) * v3 + p]) | (bf16_bits(x[(b * 2 + 1) * v3 + p]) << 16);
    reinterpret_cast<uint4*>(in)[i] = make_uint4(c01, 0u, 0u, 0u);
  }
}

__global__ void infer_out_kernel(const float* out, int64_t N, double inv_st, double* delta) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x)
    delta[i] = (double)out[i] * inv_st;
}

// per-block sums of squares (deterministic: fixed mapping)
template <typename T>
__global__ void sumsq_kernel(const T* x, int64_t n, double* partial) {
  __shared__ double red[32];
  double s = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    s += (double)x[i] * x[i];
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double tot = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) tot += red[w];
    partial[blockIdx.x] = tot;
  }
}

__global__ void bf16_from_float_kernel(const float* x, int64_t n, __nv_bfloat16* y) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    y[i] = __float2bfloat16_rn(x[i]);
}

}  // namespace mcnn

// ===========================================================================
// handle
// ===========================================================================
using namespace mcnn;

struct msstab_cnn_s {
  Dims full{};
  std::vector<float> pair_sr;   // 1 / RMS of each stored pair's residual
  float* d_pair_sr = nullptr;
  int64_t N = 0;
  int max_pairs = 0, n_pairs = 0, max_batch = 0, crop = 0;
  cudaStream_t stream = nullptr;
  std::vector<void*> allocs;
  float* theta = nullptr;
  float* m = nullptr;
  float* v = nullptr;
  float* grad = nullptr;
  __nv_bfloat16* wq[NL] = {};
  __nv_bfloat16* wt[NL] = {};
  float* bq[NL] = {};
  float* pin = nullptr;   // [max_pairs][2][N]
  float* pt = nullptr;    // [max_pairs][N]
  // training buffers (batch of crops)
  __nv_bfloat16* act[NL] = {};  // input of layer l
  float* z[NL] = {};            // pre-activation of layer l
  __nv_bfloat16* dz[NL] = {};   // gradient of the pre-activation of layer l (bf16)
  float* tgt = nullptr;
  float* kst = nullptr;         // operator stencil of the loss (27 floats), or unused
  int* tcflag = nullptr;        // raised by a tensor-core convolution whose wait ran out
  bool use_stencil = false;
  float* sbuf = nullptr;        // K * (out - t) of the batch
  float* partials = nullptr;
  int partial_rows = 0;         // blocks whose weight-gradient partials fit in partials
  double* dpart = nullptr;
  double* chunk_sums = nullptr; // [RED_CHUNKS][values] of the weight-gradient reduction
  double* h_small = nullptr;
  int* origins = nullptr;
  // inference buffers (full grid)
  __nv_bfloat16* iin = nullptr;
  __nv_bfloat16* ia = nullptr;
  __nv_bfloat16* ib = nullptr;
  float* iout = nullptr;
  float scale[2] = {1.f, 1.f};   // s_x (x channel), c (target factor)
  int adam_t = 0;
  std::string err;
};

namespace {

thread_local std::string g_cnn_error;

msstab_status cfail(msstab_cnn_t h, msstab_status code, const std::string& what) {
  if (h) h->err = what;
  g_cnn_error = what;
  msk::set_global_error(what);
  return code;
}

#define CCK(call)                                                                              \
  do {                                                                                         \
    cudaError_t e_ = (call);                                                                   \
    if (e_ != cudaSuccess)                                                                     \
      return cfail(h, e_ == cudaErrorMemoryAllocation ? MSSTAB_ERR_OOM : MSSTAB_ERR_CUDA,      \
                   std::string(#call) + ": " + cudaGetErrorString(e_));                        \
  } while (0)

template <typename T>
msstab_status calloc_(msstab_cnn_t h, T** p, size_t count) {
  void* q = nullptr;
  cudaError_t e = cudaMalloc(&q, count * sizeof(T) + 256);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return cfail(h, MSSTAB_ERR_OOM, "cudaMalloc failed in the CNN handle");
  }
  h->allocs.push_back(q);
  *p = (T*)q;
  return MSSTAB_OK;
}

#define CKA(expr)                      \
  do {                                 \
    msstab_status s_ = (expr);         \
    if (s_ != MSSTAB_OK) return s_;    \
  } while (0)

int grid1(int64_t n) {
  int64_t g = (n + 255) / 256;
  return (int)(g < 4096 ? (g < 1 ? 1 : g) : 4096);
}

msstab_status quantize(msstab_cnn_t h) {
  for (int l = 0; l < NL; ++l) {
    const int o = w_offset(l);
    quantize_kernel<<<grid1(CO_[l] * CI_[l] * 27 + CO_[l]), 256, 0, h->stream>>>(h->theta + o, h->wq[l], h->wt[l],
                                                                                   h->bq[l], CI_[l], CO_[l]);
    CCK(cudaGetLastError());
  }
  return MSSTAB_OK;
}

// forward of the batch in h->act[0] (B crops of D^3): z[l], act[l+1]
msstab_status forward_batch(msstab_cnn_t h, int B, int D) {
  const Dims d{D, D, D};
  cudaStream_t st = h->stream;
  CCK((conv<2, 16, FWD_HIDDEN>(st, h->act[0], d, B, h->wq[0], h->bq[0], h->z[0], h->act[1], nullptr, h->tcflag)));
  CCK((conv<16, 16, FWD_HIDDEN>(st, h->act[1], d, B, h->wq[1], h->bq[1], h->z[1], h->act[2], nullptr, h->tcflag)));
  CCK((conv<16, 16, FWD_HIDDEN>(st, h->act[2], d, B, h->wq[2], h->bq[2], h->z[2], h->act[3], nullptr, h->tcflag)));
  CCK((conv<16, 1, FWD_LAST>(st, h->act[3], d, B, h->wq[3], h->bq[3], h->z[3], nullptr, nullptr, h->tcflag)));
  return MSSTAB_OK;
}

// loss of z[3] against tgt, gradient into h->grad; *loss on the host
// weight and bias gradients of one layer from the wgrad partials
msstab_status reduce_partials(msstab_cnn_t h, int nb, int nv, float* grad) {
  reduce_partials_chunk_kernel<<<dim3(grid1(nv), RED_CHUNKS), 256, 0, h->stream>>>(h->partials, nb, nv, h->chunk_sums);
  reduce_partials_kernel<<<grid1(nv), 256, 0, h->stream>>>(h->chunk_sums, nv, grad);
  CCK(cudaGetLastError());
  return MSSTAB_OK;
}

msstab_status backward_batch(msstab_cnn_t h, int B, int D, double* loss) {
  const Dims d{D, D, D};
  cudaStream_t st = h->stream;
  const int64_t n = (int64_t)B * D * D * D;
  const int lg = grid1(n) < 1024 ? grid1(n) : 1024;
  if (h->use_stencil) {
    stencil_fwd_kernel<<<lg, 256, 0, st>>>(h->z[3], h->tgt, B, D, h->kst, h->sbuf, h->dpart);
    CCK(cudaGetLastError());
    stencil_bwd_kernel<<<lg, 256, 0, st>>>(h->sbuf, B, D, h->kst, 1.0 / (double)n, h->dz[3]);
  } else {
    loss_kernel<<<lg, 256, 0, st>>>(h->z[3], h->tgt, n, 1.0 / (double)n, h->dz[3], h->dpart);
  }
  CCK(cudaGetLastError());
  int nb = 0;
  // layer 3 (16 -> 1)
  CCK((wgrad_tc<16, 1>(st, h->act[3], h->dz[3], d, B, h->partials, h->partial_rows, &nb, h->tcflag)));
  CKA(reduce_partials(h, nb, 16 * 27 + 1, h->grad + w_offset(3)));
  CCK((conv<1, 16, BWD_DATA>(st, h->dz[3], d, B, h->wt[3], nullptr, nullptr, h->dz[2], h->z[2], h->tcflag)));
  for (int l = 2; l >= 1; --l) {
    CCK((wgrad_tc<16, 16>(st, h->act[l], h->dz[l], d, B, h->partials, h->partial_rows, &nb, h->tcflag)));
    CKA(reduce_partials(h, nb, 16 * 16 * 27 + 16, h->grad + w_offset(l)));
    CCK((conv<16, 16, BWD_DATA>(st, h->dz[l], d, B, h->wt[l], nullptr, nullptr, h->dz[l - 1], h->z[l - 1], h->tcflag)));
  }
  CCK((wgrad_tc<2, 16>(st, h->act[0], h->dz[0], d, B, h->partials, h->partial_rows, &nb, h->tcflag)));
  CKA(reduce_partials(h, nb, 2 * 16 * 27 + 16, h->grad + w_offset(0)));
  CCK(cudaGetLastError());
  if (loss) {
    std::vector<double> part(lg);
    CCK(cudaMemcpyAsync(part.data(), h->dpart, sizeof(double) * lg, cudaMemcpyDeviceToHost, st));
    CCK(cudaStreamSynchronize(st));
    double s = 0.0;
    for (int i = 0; i < lg; ++i) s += part[i];
    *loss = s / (double)n;
  }
  return MSSTAB_OK;
}

template <typename T>
msstab_status sumsq(msstab_cnn_t h, const T* x, int64_t n, double* out) {
  const int g = 1024;
  sumsq_kernel<T><<<g, 256, 0, h->stream>>>(x, n, h->dpart);
  CCK(cudaGetLastError());
  std::vector<double> part(g);
  CCK(cudaMemcpyAsync(part.data(), h->dpart, sizeof(double) * g, cudaMemcpyDeviceToHost, h->stream));
  CCK(cudaStreamSynchronize(h->stream));
  double s = 0.0;
  for (int i = 0; i < g; ++i) s += part[i];
  *out = s;
  return MSSTAB_OK;
}

// after a synchronisation: a tensor-core convolution whose wait ran out
msstab_status tc_check(msstab_cnn_t h) {
  int f = 0;
  CCK(cudaMemcpy(&f, h->tcflag, sizeof(int), cudaMemcpyDeviceToHost));
  if (f) return cfail(h, MSSTAB_ERR_CUDA, "a tensor-core convolution timed out waiting for its MMAs");
  return MSSTAB_OK;
}

msstab_status check_batch(msstab_cnn_t h, int B, int D) {
  if (B < 1 || B > h->max_batch || D < 1 || D > h->crop)
    return cfail(h, MSSTAB_ERR_INVALID_ARG, "batch size or crop edge beyond the handle's capacity");
  return MSSTAB_OK;
}

}  // namespace

extern "C" {

int32_t msstab_cnn_num_params(void) { return n_params(); }

msstab_status msstab_cnn_destroy(msstab_cnn_t h) {
  if (!h) return MSSTAB_OK;
  cudaStreamSynchronize(h->stream);
  for (void* p : h->allocs) cudaFree(p);
  if (h->h_small) cudaFreeHost(h->h_small);
  delete h;
  return MSSTAB_OK;
}

msstab_status msstab_cnn_create(int32_t nx, int32_t ny, int32_t nz, const float* d_params, int32_t max_pairs,
                                int32_t max_batch, int32_t crop, void* stream, msstab_cnn_t* out) {
  if (!out) return cfail(nullptr, MSSTAB_ERR_INVALID_ARG, "out is NULL");
  *out = nullptr;
  if (nx < 1 || ny < 1 || nz < 1 || (int64_t)nx * ny * nz >= (1LL << 31) || max_pairs < 0 || max_batch < 1 ||
      crop < 1 || crop > nx || crop > ny || crop > nz || !d_params)
    return cfail(nullptr, MSSTAB_ERR_INVALID_ARG, "msstab_cnn_create: bad grid, capacity or NULL parameters");
  msstab_cnn_t h = new msstab_cnn_s();
  h->full = Dims{nx, ny, nz};
  h->N = (int64_t)nx * ny * nz;
  h->max_pairs = max_pairs;
  h->max_batch = max_batch;
  h->crop = crop;
  h->stream = (cudaStream_t)stream;
  auto fail_create = [&](msstab_status s) {
    g_cnn_error = h->err;
    msstab_cnn_destroy(h);
    return s;
  };
  const int np = n_params();
  const int64_t bv = (int64_t)max_batch * crop * crop * crop;
  msstab_status s = MSSTAB_OK;
#define CKC(expr)                      \
  if ((s = (expr)) != MSSTAB_OK) return fail_create(s)
  CKC(calloc_(h, &h->theta, np));
  CKC(calloc_(h, &h->m, np));
  CKC(calloc_(h, &h->v, np));
  CKC(calloc_(h, &h->grad, np));
  for (int l = 0; l < NL; ++l) {
    CKC(calloc_(h, &h->wq[l], CO_[l] * CI_[l] * 27));
    CKC(calloc_(h, &h->wt[l], CO_[l] * CI_[l] * 27));
    CKC(calloc_(h, &h->bq[l], CO_[l]));
    CKC(calloc_(h, &h->act[l], (size_t)8 * halves(CI_[l]) * bv));   // half-major bf16
    CKC(calloc_(h, &h->z[l], (size_t)CO_[l] * bv));
    CKC(calloc_(h, &h->dz[l], (size_t)8 * halves(CO_[l]) * bv));
  }
  CKC(calloc_(h, &h->tgt, bv));
  CKC(calloc_(h, &h->sbuf, bv));
  CKC(calloc_(h, &h->kst, 27));
  CKC(calloc_(h, &h->tcflag, 1));
  h->partial_rows = WG_MAX_BLOCKS;
  CKC(calloc_(h, &h->partials, (size_t)h->partial_rows * (16 * 16 * 27 + 16)));
  CKC(calloc_(h, &h->dpart, 4096));
  CKC(calloc_(h, &h->chunk_sums, (size_t)RED_CHUNKS * (16 * 16 * 27 + 16)));
  CKC(calloc_(h, &h->origins, 4 * (size_t)max_batch));
  if (max_pairs > 0) {
    CKC(calloc_(h, &h->pin, (size_t)max_pairs * 2 * h->N));
    CKC(calloc_(h, &h->pt, (size_t)max_pairs * h->N));
    CKC(calloc_(h, &h->d_pair_sr, (size_t)max_pairs));
  }
  CKC(calloc_(h, &h->iin, 8 * (size_t)h->N));
  CKC(calloc_(h, &h->ia, 16 * (size_t)h->N));
  CKC(calloc_(h, &h->ib, 16 * (size_t)h->N));
  CKC(calloc_(h, &h->iout, (size_t)h->N));
#undef CKC
  if (cudaMallocHost((void**)&h->h_small, 64 * sizeof(double)) != cudaSuccess) {
    h->h_small = nullptr;
    h->err = "cudaMallocHost failed";
    return fail_create(MSSTAB_ERR_OOM);
  }
  if (cudaMemsetAsync(h->tcflag, 0, sizeof(int), h->stream) != cudaSuccess ||
      cudaMemcpyAsync(h->theta, d_params, sizeof(float) * np, cudaMemcpyDeviceToDevice, h->stream) != cudaSuccess ||
      cudaMemsetAsync(h->m, 0, sizeof(float) * np, h->stream) != cudaSuccess ||
      cudaMemsetAsync(h->v, 0, sizeof(float) * np, h->stream) != cudaSuccess) {
    h->err = "copying the initial parameters failed";
    return fail_create(MSSTAB_ERR_CUDA);
  }
  if ((s = quantize(h)) != MSSTAB_OK) return fail_create(s);
  if (cudaStreamSynchronize(h->stream) != cudaSuccess) {
    h->err = "CNN set-up failed";
    return fail_create(MSSTAB_ERR_CUDA);
  }
  *out = h;
  return MSSTAB_OK;
}

msstab_status msstab_cnn_get_params(msstab_cnn_t h, float* d_params) {
  if (!h || !d_params) return cfail(h, MSSTAB_ERR_INVALID_ARG, "NULL argument");
  CCK(cudaMemcpyAsync(d_params, h->theta, sizeof(float) * n_params(), cudaMemcpyDeviceToDevice, h->stream));
  CCK(cudaStreamSynchronize(h->stream));
  return MSSTAB_OK;
}

msstab_status msstab_cnn_set_params(msstab_cnn_t h, const float* d_params) {
  if (!h || !d_params) return cfail(h, MSSTAB_ERR_INVALID_ARG, "NULL argument");
  CCK(cudaMemcpyAsync(h->theta, d_params, sizeof(float) * n_params(), cudaMemcpyDeviceToDevice, h->stream));
  CKA(quantize(h));
  CCK(cudaStreamSynchronize(h->stream));
  return MSSTAB_OK;
}

msstab_status msstab_cnn_set_scales(msstab_cnn_t h, float s_x, float c) {
  if (!h || !(s_x > 0.f) || !(c > 0.f)) return cfail(h, MSSTAB_ERR_INVALID_ARG, "scales must be positive");
  h->scale[0] = s_x;
  h->scale[1] = c;
  return MSSTAB_OK;
}

msstab_status msstab_cnn_set_loss_stencil(msstab_cnn_t h, const double* k27) {
  if (!h) return cfail(h, MSSTAB_ERR_INVALID_ARG, "NULL handle");
  if (!k27) {
    h->use_stencil = false;
    return MSSTAB_OK;
  }
  float k[27];
  bool any = false;
  for (int i = 0; i < 27; ++i) {
    if (!std::isfinite(k27[i])) return cfail(h, MSSTAB_ERR_INVALID_ARG, "stencil entries must be finite");
    k[i] = (float)k27[i];
    any |= k[i] != 0.f;
  }
  if (!any) return cfail(h, MSSTAB_ERR_INVALID_ARG, "stencil is zero");
  CCK(cudaMemcpyAsync(h->kst, k, sizeof(k), cudaMemcpyHostToDevice, h->stream));
  CCK(cudaStreamSynchronize(h->stream));
  h->use_stencil = true;
  return MSSTAB_OK;
}

msstab_status msstab_cnn_get_scales(msstab_cnn_t h, float* scales2) {
  if (!h || !scales2) return cfail(h, MSSTAB_ERR_INVALID_ARG, "NULL argument");
  std::memcpy(scales2, h->scale, sizeof(h->scale));
  return MSSTAB_OK;
}

msstab_status msstab_cnn_forward(msstab_cnn_t h, const float* d_in, int32_t B, int32_t D, float* d_out) {
  if (!h || !d_in || !d_out) return cfail(h, MSSTAB_ERR_INVALID_ARG, "NULL argument");
  CKA(check_batch(h, B, D));
  const int64_t v3 = (int64_t)D * D * D;
  pack_input_kernel<<<grid1((int64_t)B * v3), 256, 0, h->stream>>>(d_in, B, v3, h->act[0]);
  CCK(cudaGetLastError());
  CKA(forward_batch(h, B, D));
  CCK(cudaMemcpyAsync(d_out, h->z[3], sizeof(float) * B * D * D * D, cudaMemcpyDeviceToDevice, h->stream));
  CCK(cudaStreamSynchronize(h->stream));
  return tc_check(h);
}

msstab_status msstab_cnn_grad(msstab_cnn_t h, const float* d_in, const float* d_target, int32_t B, int32_t D,
                              float* d_grad, double* loss) {
  if (!h || !d_in || !d_target || !d_grad) return cfail(h, MSSTAB_ERR_INVALID_ARG, "NULL argument");
  CKA(check_batch(h, B, D));
  const int64_t v3 = (int64_t)D * D * D;
  pack_input_kernel<<<grid1((int64_t)B * v3), 256, 0, h->stream>>>(d_in, B, v3, h->act[0]);
  CCK(cudaGetLastError());
  CCK(cudaMemcpyAsync(h->tgt, d_target, sizeof(float) * B * D * D * D, cudaMemcpyDeviceToDevice, h->stream));
  CKA(forward_batch(h, B, D));
  CKA(backward_batch(h, B, D, loss));
  CCK(cudaMemcpyAsync(d_grad, h->grad, sizeof(float) * n_params(), cudaMemcpyDeviceToDevice, h->stream));
  CCK(cudaStreamSynchronize(h->stream));
  return tc_check(h);
}

msstab_status msstab_cnn_adam_step(msstab_cnn_t h, const float* d_grad, float lr) {
  if (!h || !d_grad || !(lr > 0.f)) return cfail(h, MSSTAB_ERR_INVALID_ARG, "bad Adam arguments");
  h->adam_t += 1;
  const float b1 = 0.9f, b2 = 0.999f;
  const float c1 = 1.f - powf(b1, (float)h->adam_t), c2 = 1.f - powf(b2, (float)h->adam_t);
  adam_kernel<<<grid1(n_params()), 256, 0, h->stream>>>(h->theta, h->m, h->v, d_grad, n_params(), lr, b1, b2, 1e-8f,
                                                        c1, c2);
  CCK(cudaGetLastError());
  CKA(quantize(h));
  return MSSTAB_OK;
}

msstab_status msstab_cnn_add_pair(msstab_cnn_t h, const double* d_r0, const double* d_x_prev,
                                  const double* d_x_next) {
  if (!h || !d_r0 || !d_x_prev || !d_x_next) return cfail(h, MSSTAB_ERR_INVALID_ARG, "NULL argument");
  if (h->n_pairs >= h->max_pairs) return cfail(h, MSSTAB_ERR_INVALID_ARG, "the pair store is full");
  const int k = h->n_pairs;
  pair_kernel<<<grid1(h->N), 256, 0, h->stream>>>(d_r0, d_x_prev, d_x_next, h->N, h->pin + (size_t)k * 2 * h->N,
                                                  h->pt + (size_t)k * h->N);
  CCK(cudaGetLastError());
  double ss = 0.0;
  CKA(sumsq<double>(h, d_r0, h->N, &ss));
  const double rms = std::sqrt(ss / (double)h->N);
  const float sr = rms > 0.0 && std::isfinite(rms) ? (float)(1.0 / rms) : 1.f;
  h->pair_sr.push_back(sr);
  CCK(cudaMemcpyAsync(h->d_pair_sr + k, &h->pair_sr.back(), sizeof(float), cudaMemcpyHostToDevice, h->stream));
  CCK(cudaStreamSynchronize(h->stream));
  h->n_pairs += 1;
  return MSSTAB_OK;
}

msstab_status msstab_cnn_fit_scales(msstab_cnn_t h) {
  if (!h || h->n_pairs < 1) return cfail(h, MSSTAB_ERR_INVALID_ARG, "no training pairs");
  double sx = 0.0, sd = 0.0;
  for (int k = 0; k < h->n_pairs; ++k) {
    double a = 0.0, d = 0.0;
    CKA(sumsq<float>(h, h->pin + ((size_t)k * 2 + 1) * h->N, h->N, &a));
    CKA(sumsq<float>(h, h->pt + (size_t)k * h->N, h->N, &d));
    sx += a;
    sd += d * (double)h->pair_sr[k] * (double)h->pair_sr[k];
  }
  const double cnt = (double)h->n_pairs * (double)h->N;
  const double rx = std::sqrt(sx / cnt), rd = std::sqrt(sd / cnt);
  h->scale[0] = rx > 0.0 ? (float)(1.0 / rx) : 1.f;
  h->scale[1] = rd > 0.0 ? (float)(1.0 / rd) : 1.f;
  return MSSTAB_OK;
}

msstab_status msstab_cnn_train(msstab_cnn_t h, int32_t iters, int32_t B, int32_t D, const int32_t* origins,
                               float lr, float* loss_history) {
  if (!h || !origins || iters < 0 || !(lr > 0.f)) return cfail(h, MSSTAB_ERR_INVALID_ARG, "bad training arguments");
  CKA(check_batch(h, B, D));
  if (h->n_pairs < 1) return cfail(h, MSSTAB_ERR_INVALID_ARG, "no training pairs");
  for (int it = 0; it < iters; ++it) {
    const int32_t* o = origins + (size_t)it * 4 * B;
    for (int b = 0; b < B; ++b)
      if (o[4 * b] < 0 || o[4 * b] >= h->n_pairs || o[4 * b + 1] < 0 || o[4 * b + 1] + D > h->full.Z ||
          o[4 * b + 2] < 0 || o[4 * b + 2] + D > h->full.Y || o[4 * b + 3] < 0 || o[4 * b + 3] + D > h->full.X)
        return cfail(h, MSSTAB_ERR_INVALID_ARG, "crop origin out of range");
    CCK(cudaMemcpyAsync(h->origins, o, sizeof(int32_t) * 4 * B, cudaMemcpyHostToDevice, h->stream));
    const int64_t v3 = (int64_t)D * D * D;
    gather_kernel<<<dim3(grid1(v3), B), 256, 0, h->stream>>>(h->pin, h->pt, h->N, h->full, h->origins, D,
                                                             h->d_pair_sr, h->scale[0], h->scale[1], h->act[0],
                                                             h->tgt);
    CCK(cudaGetLastError());
    CKA(forward_batch(h, B, D));
    double loss = 0.0;
    CKA(backward_batch(h, B, D, loss_history ? &loss : nullptr));
    if (loss_history) loss_history[it] = (float)loss;
    CKA(msstab_cnn_adam_step(h, h->grad, lr));
  }
  CCK(cudaStreamSynchronize(h->stream));
  return tc_check(h);
}

msstab_status msstab_cnn_infer(msstab_cnn_t h, const double* d_r0, const double* d_x_prev, double* d_delta) {
  if (!h || !d_r0 || !d_x_prev || !d_delta) return cfail(h, MSSTAB_ERR_INVALID_ARG, "NULL argument");
  cudaStream_t st = h->stream;
  double ss = 0.0;
  CKA(sumsq<double>(h, d_r0, h->N, &ss));
  const double rms = std::sqrt(ss / (double)h->N);
  const float sr = rms > 0.0 && std::isfinite(rms) ? (float)(1.0 / rms) : 1.f;
  infer_in_kernel<<<grid1(h->N), 256, 0, st>>>(d_r0, d_x_prev, h->N, sr, h->scale[0], h->iin);
  CCK(cudaGetLastError());
  CCK((conv<2, 16, INFER_HIDDEN>(st, h->iin, h->full, 1, h->wq[0], h->bq[0], nullptr, h->ia, nullptr, h->tcflag)));
  CCK((conv<16, 16, INFER_HIDDEN>(st, h->ia, h->full, 1, h->wq[1], h->bq[1], nullptr, h->ib, nullptr, h->tcflag)));
  CCK((conv<16, 16, INFER_HIDDEN>(st, h->ib, h->full, 1, h->wq[2], h->bq[2], nullptr, h->ia, nullptr, h->tcflag)));
  CCK((conv<16, 1, FWD_LAST>(st, h->ia, h->full, 1, h->wq[3], h->bq[3], h->iout, nullptr, nullptr, h->tcflag)));
  infer_out_kernel<<<grid1(h->N), 256, 0, st>>>(h->iout, h->N, 1.0 / ((double)h->scale[1] * (double)sr), d_delta);
  CCK(cudaGetLastError());
  return MSSTAB_OK;
}

const char* msstab_cnn_last_error(msstab_cnn_t h) { return h ? h->err.c_str() : g_cnn_error.c_str(); }

}  // extern "C"

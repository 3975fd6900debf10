// Tensor-core apply, F16X3: y_b = M x_b on tcgen05 with FP32 accumulation.
//
// The batched product Y[b][n] = sum_k X[b][k] M[n][k] (every block's
// coefficients times the precomputed operator of Eq. 11 / Eq. 20) is a GEMM
// with M = 128 blocks per tile, N = N^2 outputs, K = N^2 inputs.  At 8x8 it
// moves 512 bytes per block for 8192 flops, so it is bound by HBM; the
// tensor cores only have to keep up, which leaves room for a 3-product split
// that restores FP32-level accuracy from FP16 operands:
//   x = x_hi + x_lo, M 2^s = M_hi + M_lo (FP16, round to nearest),
//   y = (x_hi M_hi + [x_hi M_lo + x_lo M_hi]) 2^-s + M[:,0] x[0].
// The input DC coefficient x[0] is taken out of the tensor-core product and
// added in FP32 in the epilogue (it is the largest coefficient; keeping it
// out of the FP16 split and the long FP32 sums keeps pixel errors near
// 1e-5).  The bracketed correction is accumulated apart from the main term.
//
// Per CTA (one per SM, persistent over tiles t = blockIdx.x + i*gridDim.x):
//   warp 0      TMA producer: X tile (128 rows x 256 B, two SWIZZLE_128B
//               boxes) into a 3-stage shared-memory ring;
//   warp 1      MMA issuer: A from TMEM, B (M_hi | M_lo, resident in shared
//               memory for the whole launch), D in TMEM, double-buffered;
//   warp 2      TMEM allocator;
//   warps 4-7   converter: thread = block row; reads its row from the stage,
//               removes the DC term, splits hi/lo, tcgen05.st into TMEM (A);
//   warps 8-11  epilogue: tcgen05.ld of D, scale, + DC term, swizzled
//               shared-memory staging (2 stages), TMA store of 32 rows
//               per warp.
// TMEM per buffer (256 columns): A_hi 32, A_lo 32, D 128 (main 64, corr 64).
#include "sm100_ptx.cuh"

#include <mutex>

namespace dctf {
namespace {

using namespace ptx;

constexpr int kTile = 128;
constexpr int kInStages = 3;
constexpr int kOutStages = 2;
constexpr int kThreads = 384;
constexpr uint32_t kTmemCols = 512;
constexpr int kN2 = 64;                          // 8x8 blocks
constexpr int kRowBytes = kN2 * 4;               // 256
constexpr int kBoxBytes = kTile * 128;           // 16 KB: 128 rows x 32 floats
constexpr int kStageBytes = kTile * kRowBytes;   // 32 KB
constexpr int kBBytes = 2 * kN2 * 128;           // M_hi and M_lo, 128 rows x 128 B
constexpr int kSlabBytes = 32 * kRowBytes;       // one epilogue warp's 32 output rows
constexpr int kSlabBoxBytes = 32 * 128;          // 32 rows x 32 floats

// shared memory carve-up (from a 1024-aligned base)
constexpr int kOffIn = 0;
constexpr int kOffOut = kOffIn + kInStages * kStageBytes;
constexpr int kOffB = kOffOut + kOutStages * kStageBytes;
constexpr int kOffMdc = kOffB + kBBytes;
constexpr int kOffDc = kOffMdc + kN2 * 4;
constexpr int kOffBar = kOffDc + 4 * kTile * 4;
constexpr int kNumBars = 3 + 3 + 2 + 2 + 2 + 4;
constexpr int kOffMisc = kOffBar + kNumBars * 8;
constexpr int kSmemBytes = kOffMisc + 16 + 1024;   // + alignment slack

// roles for error codes
enum : uint32_t { kRoleProducer = 1, kRoleMma = 2, kRoleConv = 3, kRoleEpi = 4, kRoleDrain = 5 };

__global__ void __launch_bounds__(kThreads, 1)
apply_tc_f16x3_n8(const __grid_constant__ CUtensorMap tm_in,
                  const __grid_constant__ CUtensorMap tm_out, const uint4 *__restrict__ pieces,
                  const float *__restrict__ Mdc, float out_scale, int ntiles,
                  uint32_t *__restrict__ err) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t *base = reinterpret_cast<uint8_t *>(
      (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  uint8_t *s_in = base + kOffIn;
  uint8_t *s_out = base + kOffOut;
  uint8_t *s_b = base + kOffB;
  float *s_mdc = reinterpret_cast<float *>(base + kOffMdc);
  float *s_dc = reinterpret_cast<float *>(base + kOffDc);
  uint64_t *bars = reinterpret_cast<uint64_t *>(base + kOffBar);
  uint64_t *full_in = bars;          // [3] TMA -> converter
  uint64_t *empty_in = bars + 3;     // [3] converter -> TMA
  uint64_t *a_full = bars + 6;       // [2] converter -> MMA
  uint64_t *mma_done = bars + 8;     // [2] MMA -> converter (A free), epilogue (D full)
  uint64_t *d_empty = bars + 10;     // [2] epilogue -> MMA
  uint64_t *dc_full = bars + 12;     // [4] converter -> epilogue (DC ring)
  uint32_t *s_tmem = reinterpret_cast<uint32_t *>(base + kOffMisc);
  volatile int *s_abort = reinterpret_cast<volatile int *>(base + kOffMisc + 4);

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int my_tiles =
      blockIdx.x < ntiles ? (ntiles - (int)blockIdx.x + (int)gridDim.x - 1) / (int)gridDim.x : 0;

  if (tid == 0) {
    for (int s = 0; s < kInStages; ++s) { mbar_init(&full_in[s], 1); mbar_init(&empty_in[s], 128); }
    for (int b = 0; b < 2; ++b) {
      mbar_init(&a_full[b], 128); mbar_init(&mma_done[b], 1); mbar_init(&d_empty[b], 128);
    }
    for (int r = 0; r < 4; ++r) mbar_init(&dc_full[r], 128);
    *s_abort = 0;
    mbar_fence_init();
  }
  // resident operands: the B pieces (already in the swizzled layout) and M[:,0]
  for (int i = tid; i < kBBytes / 16; i += kThreads)
    reinterpret_cast<uint4 *>(s_b)[i] = __ldg(pieces + i);
  if (tid < kN2) s_mdc[tid] = __ldg(Mdc + tid);
  fence_async_smem();
  if (warp == 2) { tmem_alloc(s_tmem, kTmemCols); tmem_relinquish(); }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *s_tmem;

  if (warp == 0 && lane == 0) {
    // ------------------------------------------------------------ producer
    tma_prefetch_map(&tm_in);
    int issued = 0;
    for (int it = 0; it < my_tiles; ++it) {
      const int tile = blockIdx.x + it * gridDim.x;
      const int s = it % kInStages;
      const uint32_t ph = (it / kInStages) & 1;
      if (!wait_bounded(&empty_in[s], ph ^ 1, s_abort, err, kRoleProducer | (tile << 8))) break;
      mbar_arrive_expect_tx(&full_in[s], kStageBytes);
      uint8_t *dst = s_in + s * kStageBytes;
      tma_load_2d(&tm_in, &full_in[s], dst, 0, tile * kTile);
      tma_load_2d(&tm_in, &full_in[s], dst + kBoxBytes, 32, tile * kTile);
      ++issued;
    }
    // no copy may still be landing in shared memory when the CTA exits
    for (int it = issued > kInStages ? issued - kInStages : 0; it < issued; ++it)
      wait_drain(&full_in[it % kInStages], (it / kInStages) & 1, err, kRoleDrain);
  } else if (warp == 1 && lane == 0) {
    // ------------------------------------------------------------ MMA issuer
    constexpr uint32_t kIdescMain = idesc_f16(128, 2 * kN2, false);   // N = 128: hi | lo
    constexpr uint32_t kIdescCorr = idesc_f16(128, kN2, false);       // N = 64: hi
    const uint64_t bdesc = desc_sw128(smem_u32(s_b));
    int last = -1;
    for (int it = 0; it < my_tiles; ++it) {
      const int tile = blockIdx.x + it * gridDim.x;
      const int b = it & 1;
      const uint32_t ph = (it >> 1) & 1;
      if (!wait_bounded(&a_full[b], ph, s_abort, err, kRoleMma | (tile << 8))) break;
      if (!wait_bounded(&d_empty[b], ph ^ 1, s_abort, err, kRoleMma | (tile << 8))) break;
      tc_fence_after();
      const uint32_t t_a = tmem + b * 256, t_d = t_a + 128;
#pragma unroll
      for (int k = 0; k < kN2 / 16; ++k)   // D[0:128] = A_hi [M_hi; M_lo]^T
        mma_f16_ts(t_d, t_a + 8 * k, bdesc + 2 * k, kIdescMain, k > 0);
#pragma unroll
      for (int k = 0; k < kN2 / 16; ++k)   // D[64:128] += A_lo M_hi^T
        mma_f16_ts(t_d + 64, t_a + 32 + 8 * k, bdesc + 2 * k, kIdescCorr, 1);
      tc_commit(&mma_done[b]);
      last = it;
    }
    if (last >= 0) wait_drain(&mma_done[last & 1], (last >> 1) & 1, err, kRoleDrain);
  } else if (warp >= 4 && warp < 8) {
    // ------------------------------------------------------------ converter
    const int row = tid - 128;                       // block row in the tile = TMEM lane
    const uint32_t lane_base = (uint32_t)((warp & 3) * 32) << 16;
    for (int it = 0; it < my_tiles; ++it) {
      const int tile = blockIdx.x + it * gridDim.x;
      const int s = it % kInStages, b = it & 1, r4 = it & 3;
      const uint32_t ps = (it / kInStages) & 1, pb = (it >> 1) & 1;
      if (!warp_wait_bounded(&full_in[s], ps, s_abort, err, kRoleConv | (tile << 8))) break;
      const uint8_t *st = s_in + s * kStageBytes + row * 128;
      float v[64];
#pragma unroll
      for (int u = 0; u < 16; ++u) {
        const float4 q = *reinterpret_cast<const float4 *>(
            st + (u >> 3) * kBoxBytes + (((u & 7) ^ (row & 7)) << 4));
        v[4 * u] = q.x; v[4 * u + 1] = q.y; v[4 * u + 2] = q.z; v[4 * u + 3] = q.w;
      }
      mbar_arrive(&empty_in[s]);        // every thread: its reads of stage s are done
      const float x0 = v[0];
      v[0] = 0.f;
      // A buffer b is free once the MMAs of tile it-2 completed
      if (!warp_wait_bounded(&mma_done[b], pb ^ 1, s_abort, err, kRoleConv | (tile << 8))) break;
      s_dc[r4 * kTile + row] = x0;
      mbar_arrive(&dc_full[r4]);
      tc_fence_after();
      const uint32_t t_a = tmem + lane_base + b * 256;
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        uint32_t hi[16], lo[16];
#pragma unroll
        for (int c = 0; c < 16; ++c) {
          const float a0 = v[32 * h + 2 * c], a1 = v[32 * h + 2 * c + 1];
          const __half2 h2 = __floats2half2_rn(a0, a1);     // .x (low half) = element 2c
          const float2 hf = __half22float2(h2);
          const __half2 l2 = __floats2half2_rn(a0 - hf.x, a1 - hf.y);
          hi[c] = *reinterpret_cast<const uint32_t *>(&h2);
          lo[c] = *reinterpret_cast<const uint32_t *>(&l2);
        }
        tmem_st16(t_a + 16 * h, hi);
        tmem_st16(t_a + 32 + 16 * h, lo);
      }
      tmem_st_wait();
      tc_fence_before();
      mbar_arrive(&a_full[b]);
    }
  } else if (warp >= 8) {
    // ------------------------------------------------------------ epilogue
    // Each warp owns 32 rows of the tile and stores them with its own TMA
    // copies, so no synchronisation wider than a warp is needed.
    const int row = tid - 256, wr = warp & 3, r32 = lane;
    const uint32_t lane_base = (uint32_t)(wr * 32) << 16;
    for (int it = 0; it < my_tiles; ++it) {
      const int tile = blockIdx.x + it * gridDim.x;
      const int b = it & 1, o = it & 1, r4 = it & 3;
      const uint32_t pb = (it >> 1) & 1, p4 = (it >> 2) & 1;
      if (!warp_wait_bounded(&mma_done[b], pb, s_abort, err, kRoleEpi | (tile << 8))) break;
      tc_fence_after();
      if (!warp_wait_bounded(&dc_full[r4], p4, s_abort, err, kRoleEpi | (tile << 8))) break;
      const float x0 = s_dc[r4 * kTile + row];
      // this warp's slab of staging buffer o is free once its TMA store of
      // tile it-2 has read it
      if (lane == 0) bulk_wait_read<kOutStages - 1>();
      __syncwarp();
      uint8_t *slab = s_out + o * kStageBytes + wr * kSlabBytes;
      const uint32_t t_d = tmem + lane_base + b * 256 + 128;
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        uint32_t dm[32], dc[32];
        tmem_ld32(t_d + 32 * h, dm);
        tmem_ld32(t_d + 64 + 32 * h, dc);
#pragma unroll
        for (int u = 0; u < 8; ++u) {
          float4 q;
          float *qq = reinterpret_cast<float *>(&q);
#pragma unroll
          for (int e = 0; e < 4; ++e) {
            const int c = 4 * u + e;
            const float acc = __uint_as_float(dm[c]) + __uint_as_float(dc[c]);
            qq[e] = fmaf(s_mdc[32 * h + c], x0, acc * out_scale);
          }
          *reinterpret_cast<float4 *>(slab + h * kSlabBoxBytes + r32 * 128 +
                                      ((u ^ (r32 & 7)) << 4)) = q;
        }
      }
      tc_fence_before();
      mbar_arrive(&d_empty[b]);         // every thread: its TMEM reads of D[b] are done
      fence_async_smem();
      __syncwarp();
      if (lane == 0) {
        const int y0 = tile * kTile + wr * 32;
        tma_store_2d(&tm_out, slab, 0, y0);
        tma_store_2d(&tm_out, slab + kSlabBoxBytes, 32, y0);
        bulk_commit();
      }
    }
    if (lane == 0) bulk_wait<0>();
  }

  tc_fence_before();
  __syncthreads();
  if (warp == 2) {
    tc_fence_after();
    tmem_dealloc(tmem, kTmemCols);
  }
}

// ---------------------------------------------------------------- host side
typedef CUresult (*EncodeTiledFn)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *,
                                  const cuuint64_t *, const cuuint64_t *, const cuuint32_t *,
                                  const cuuint32_t *, CUtensorMapInterleave, CUtensorMapSwizzle,
                                  CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encode_fn() {
  static EncodeTiledFn fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void *p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                         &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<EncodeTiledFn>(p);
  });
  return fn;
}

// [nblocks][n2] FP32 rows seen as a 2-D tensor (inner dim n2), boxes of
// 32 floats x box_rows rows with 128-byte swizzle.
cudaError_t make_rows_map(CUtensorMap *m, const void *ptr, int64_t nblocks, int n2,
                          int box_rows) {
  EncodeTiledFn enc = encode_fn();
  if (enc == nullptr) return cudaErrorNotSupported;
  cuuint64_t dims[2] = {(cuuint64_t)n2, (cuuint64_t)nblocks};
  cuuint64_t strides[1] = {(cuuint64_t)n2 * 4};
  cuuint32_t box[2] = {32, (cuuint32_t)box_rows};
  cuuint32_t es[2] = {1, 1};
  CUresult r = enc(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<void *>(ptr), dims, strides,
                   box, es, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                   CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

}  // namespace

bool tc_supported(int n, dctf_precision p) { return n == 8 && p == DCTF_F16X3; }

cudaError_t launch_apply_tc(const dctf_operator *op, const float *x, int64_t nblocks, float *y,
                            cudaStream_t s) {
  if (!tc_supported(op->n, op->precision)) return cudaErrorNotSupported;
  CUtensorMap tin, tout;
  cudaError_t e = make_rows_map(&tin, x, nblocks, op->n2, kTile);
  if (e != cudaSuccess) return e;
  e = make_rows_map(&tout, y, nblocks, op->n2, 32);
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(apply_tc_f16x3_n8, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           kSmemBytes);
  if (e != cudaSuccess) return e;
  const int ntiles = (int)((nblocks + kTile - 1) / kTile);
  int grid = sm_count(op->device);
  if (grid > ntiles) grid = ntiles;
  if (grid < 1) grid = 1;
  const float out_scale = ldexpf(1.0f, -op->f16_scale_exp);
  apply_tc_f16x3_n8<<<grid, kThreads, kSmemBytes, s>>>(
      tin, tout, reinterpret_cast<const uint4 *>(op->d_f16), op->d_Mdc, out_scale, ntiles,
      op->d_err);
  return cudaGetLastError();
}

}  // namespace dctf

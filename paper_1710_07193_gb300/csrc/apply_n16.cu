// Tensor-core apply for 16x16 blocks (N^2 = 256): y_b = M x_b, F16X3 split.
//
// Same arithmetic as the 8x8 kernel (apply_group.cu): x and M 2^s split into
// FP16 hi/lo, y = (x_hi M_lo + x_lo M_hi + x_hi M_hi) 2^-s + M[:,0] x[0] with
// FP32 accumulation in TMEM and the input DC coefficient in FP32.  What
// changes at 16x16 is size: M is 256 x 256, its two FP16 pieces 256 KB,
// more than one SM's shared memory, and a 128-block tile is 128 KB in and
// 128 KB out.  So:
//
//  * Output split.  Each 128-block tile is processed by a pair of CTAs; CTA
//    (pair, half) computes output coefficients [128 half, 128 half + 128).
//    Its 128 rows of M_hi and M_lo (128 KB) stay resident in shared memory
//    for the whole launch.  Both CTAs of a pair read the same input tile
//    (the second read is an L2 hit); each writes its own half of the output.
//  * K chunks.  The tile's input is streamed in eight 32-coefficient chunks
//    (16 KB, one SWIZZLE_128B box) through a TMA ring; the converter turns
//    each chunk into FP16 hi/lo A operands in an 8-deep TMEM ring (one whole
//    tile), and the MMA warp accumulates 128 x 128 x 16 MMAs into two TMEM
//    accumulators, one per K half, correction products before the main
//    product (tensor-core FP32 accumulation truncates; this order and the
//    split keep the error near the 8x8 kernel's).
//  * Output chunks.  The epilogue reads D 32 columns at a time and TMA-stores
//    32 x 32 boxes, double-buffered per warp.
//
// Roles (384 threads): warp 0 TMA producer, warp 1 MMA issuer, warp 2 TMEM
// allocator, warps 4-7 converter (thread = tile row), warps 8-11 epilogue.
// All waits bounded, warp-uniform in multi-lane roles (sm100_ptx.cuh).
#include "sm100_ptx.cuh"

#include <mutex>

namespace dctf {
namespace {

using namespace ptx;

constexpr int kThreads = 384;
constexpr int kTile = 128;
constexpr int kN2 = 256;                 // coefficients per block
constexpr int kOut = 128;                // outputs per CTA (half of kN2)
constexpr int kChunkK = 32;              // K per input chunk (one 128-byte box row)
constexpr int kChunks = kN2 / kChunkK;   // 8
constexpr int kStages = 3;               // input chunk stages
constexpr int kABufs = 8;                // TMEM A ring (one chunk each: hi 16 | lo 16 columns)
constexpr int kGroups = 2;               // K halves, each with its own 128-column accumulator
constexpr int kDcRing = 8;
constexpr uint32_t kTmemCols = 512;

constexpr int kChunkBytes = kTile * kChunkK * 4;    // 16 KB: one box (32 floats x 128 rows)
constexpr int kBChunks = kN2 / 64;                  // 64-wide K blocks of the B layout
constexpr int kBPieceChunk = kOut * 128;            // 16 KB: 128 rows x 64 fp16
constexpr int kBBytes = 2 * kBChunks * kBPieceChunk; // 128 KB: [piece][kb][128 rows][128 B]
constexpr int kOutSlab = 32 * 128;                  // one warp's 32 x 32 floats box
constexpr int kOffB = 0;
constexpr int kOffIn = kOffB + kBBytes;
constexpr int kOffOut = kOffIn + kStages * kChunkBytes;
constexpr int kOffMdc = kOffOut + 2 * 4 * kOutSlab;
constexpr int kOffDc = kOffMdc + kOut * 4;
constexpr int kOffBar = kOffDc + kDcRing * kTile * 4;
constexpr int kNumBars = 2 * kStages + 2 * kABufs + 2 + kDcRing;
constexpr int kOffMisc = kOffBar + kNumBars * 8;
constexpr int kSmem = kOffMisc + 16 + 1024;
static_assert(kSmem <= 232448, "shared memory");

enum : uint32_t { kRoleProducer = 1, kRoleMma = 2, kRoleConv = 3, kRoleEpi = 4, kRoleDrain = 5 };

__global__ void __launch_bounds__(kThreads, 1)
apply_n16_f16x3_kernel(const __grid_constant__ CUtensorMap tm_in,
                       const __grid_constant__ CUtensorMap tm_out, const uint4 *__restrict__ pieces,
                       const float *__restrict__ Mdc, float out_scale, int ntiles,
                       uint32_t *__restrict__ err) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t *base = reinterpret_cast<uint8_t *>(
      (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  uint8_t *s_b = base + kOffB;
  uint8_t *s_in = base + kOffIn;
  uint8_t *s_out = base + kOffOut;
  float *s_mdc = reinterpret_cast<float *>(base + kOffMdc);
  float *s_dc = reinterpret_cast<float *>(base + kOffDc);
  uint64_t *bars = reinterpret_cast<uint64_t *>(base + kOffBar);
  uint64_t *full_in = bars;                     // [kStages]
  uint64_t *empty_in = full_in + kStages;       // [kStages]
  uint64_t *a_full = empty_in + kStages;        // [kABufs]
  uint64_t *a_done = a_full + kABufs;           // [kABufs] MMA finished reading the chunk
  uint64_t *d_full = a_done + kABufs;           // [1]
  uint64_t *d_empty = d_full + 1;               // [1]
  uint64_t *dc_full = d_empty + 1;              // [kDcRing]
  uint32_t *s_tmem = reinterpret_cast<uint32_t *>(base + kOffMisc);
  volatile int *s_abort = reinterpret_cast<volatile int *>(base + kOffMisc + 4);

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int half = blockIdx.x & 1;
  const int pair = blockIdx.x >> 1, npairs = gridDim.x >> 1;
  const int my_tiles = pair < ntiles ? (ntiles - pair + npairs - 1) / npairs : 0;

  if (tid == 0) {
    for (int s = 0; s < kStages; ++s) { mbar_init(&full_in[s], 1); mbar_init(&empty_in[s], 128); }
    for (int a = 0; a < kABufs; ++a) { mbar_init(&a_full[a], 128); mbar_init(&a_done[a], 1); }
    mbar_init(d_full, 1);
    mbar_init(d_empty, 128);
    for (int r = 0; r < kDcRing; ++r) mbar_init(&dc_full[r], 128);
    *s_abort = 0;
    mbar_fence_init();
    tma_prefetch_map(&tm_in);
  }
  // resident B: for each piece (hi, lo) and K chunk, this half's 128 rows
  // (a contiguous 16 KB block of the operator's piece image)
  for (int i = tid; i < kBBytes / 16; i += kThreads) {
    const int blk = i / (kBPieceChunk / 16), off = i % (kBPieceChunk / 16);
    const int piece = blk / kBChunks, kc = blk % kBChunks;
    // source image: [kc][512 rows: hi 0..255, lo 256..511][128 B]
    const size_t src_row0 = (size_t)kc * 512 + piece * 256 + half * kOut;
    reinterpret_cast<uint4 *>(s_b)[i] = __ldg(pieces + src_row0 * 8 + off);
  }
  if (tid < kOut) s_mdc[tid] = __ldg(Mdc + half * kOut + tid);
  fence_async_smem();
  if (warp == 2) { tmem_alloc(s_tmem, kTmemCols); tmem_relinquish(); }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *s_tmem;   // A ring: columns 0..255, D0: 256..383, D1: 384..511

  if (warp == 0 && lane == 0) {
    // ---------------------------------------------------------- producer
    int q = 0, issued = 0;
    for (int it = 0; it < my_tiles; ++it) {
      const int tile = pair + it * npairs;
      for (int kc = 0; kc < kChunks; ++kc, ++q) {
        const int s = q % kStages;
        if (!wait_bounded(&empty_in[s], ((q / kStages) & 1) ^ 1, s_abort, err,
                          kRoleProducer | (q << 8)))
          goto producer_done;
        mbar_arrive_expect_tx(&full_in[s], kChunkBytes);
        tma_load_2d(&tm_in, &full_in[s], s_in + s * kChunkBytes, kc * kChunkK, tile * kTile);
        ++issued;
      }
    }
  producer_done:
    for (int k = issued > kStages ? issued - kStages : 0; k < issued; ++k)
      wait_drain(&full_in[k % kStages], (k / kStages) & 1, err, kRoleDrain);
  } else if (warp == 1 && lane == 0) {
    // ---------------------------------------------------------- MMA issuer
    // Tile t: for each K half g, D_g = sum over its 4 chunks of the two
    // correction products, then of the main product.  Tensor-core FP32
    // accumulation truncates, so small terms go in while D_g is still small,
    // and each accumulator sees half the K steps; the epilogue adds D_0 + D_1
    // with round-to-nearest.  The chunk's A buffer is released after its main
    // product.
    constexpr uint32_t kIdesc = idesc_f16(128, kOut, false);
    int q = 0, last_q = -1;
    for (int it = 0; it < my_tiles; ++it) {
      if (!wait_bounded(d_empty, (it & 1) ^ 1, s_abort, err, kRoleMma | (it << 8)))
        goto mma_done_label;
      for (int g = 0; g < kGroups; ++g) {
        const uint32_t t_d = tmem + 256 + g * kOut;
        const int q0 = q + g * (kChunks / kGroups);
        for (int c = 0; c < kChunks / kGroups; ++c) {
          const int qc = q0 + c, a = qc % kABufs, kc = g * (kChunks / kGroups) + c;
          if (!wait_bounded(&a_full[a], (qc / kABufs) & 1, s_abort, err, kRoleMma | (qc << 8)))
            goto mma_done_label;
          tc_fence_after();
          const uint32_t t_a = tmem + a * 32;
          // chunk kc covers K [32 kc, 32 kc + 32): 64-wide block kc / 2 of the
          // B layout, starting 64 bytes into its rows for odd kc
          const int kb = kc >> 1, kofs = (kc & 1) * 4;      // in 16-byte descriptor units
          const uint64_t b_hi = desc_sw128(smem_u32(s_b + (0 * kBChunks + kb) * kBPieceChunk)) + kofs;
          const uint64_t b_lo = desc_sw128(smem_u32(s_b + (1 * kBChunks + kb) * kBPieceChunk)) + kofs;
#pragma unroll
          for (int kk = 0; kk < kChunkK / 16; ++kk)
            mma_f16_ts(t_d, t_a + 8 * kk, b_lo + 2 * kk, kIdesc, (c > 0 || kk > 0) ? 1u : 0u);
#pragma unroll
          for (int kk = 0; kk < kChunkK / 16; ++kk)
            mma_f16_ts(t_d, t_a + 16 + 8 * kk, b_hi + 2 * kk, kIdesc, 1);
        }
        for (int c = 0; c < kChunks / kGroups; ++c) {
          const int qc = q0 + c, a = qc % kABufs, kc = g * (kChunks / kGroups) + c;
          const uint32_t t_a = tmem + a * 32;
          const int kb = kc >> 1, kofs = (kc & 1) * 4;
          const uint64_t b_hi = desc_sw128(smem_u32(s_b + (0 * kBChunks + kb) * kBPieceChunk)) + kofs;
#pragma unroll
          for (int kk = 0; kk < kChunkK / 16; ++kk)
            mma_f16_ts(t_d, t_a + 8 * kk, b_hi + 2 * kk, kIdesc, 1);
          tc_commit(&a_done[a]);
          last_q = qc;
        }
      }
      q += kChunks;
      tc_commit(d_full);
    }
  mma_done_label:
    if (last_q >= 0) wait_drain(&a_done[last_q % kABufs], (last_q / kABufs) & 1, err, kRoleDrain);
  } else if (warp >= 4 && warp < 8) {
    // ---------------------------------------------------------- converter
    const int row = tid - 128;
    const uint32_t lane_base = (uint32_t)((warp & 3) * 32) << 16;
    int q = 0;
    for (int it = 0; it < my_tiles; ++it) {
      for (int kc = 0; kc < kChunks; ++kc, ++q) {
        const int s = q % kStages, a = q % kABufs;
        if (!warp_wait_bounded(&full_in[s], (q / kStages) & 1, s_abort, err, kRoleConv | (q << 8)))
          goto conv_done;
        float v[32];
        const uint8_t *st = s_in + s * kChunkBytes + row * 128;
#pragma unroll
        for (int u = 0; u < 8; ++u) {
          const float4 f = *reinterpret_cast<const float4 *>(st + ((u ^ (row & 7)) << 4));
          v[4 * u] = f.x; v[4 * u + 1] = f.y; v[4 * u + 2] = f.z; v[4 * u + 3] = f.w;
        }
        mbar_arrive(&empty_in[s]);
        if (kc == 0) {
          const int r = it % kDcRing;
          s_dc[r * kTile + row] = v[0];     // ring slot free: see the epilogue's d_empty chain
          v[0] = 0.f;
          mbar_arrive(&dc_full[r]);
        }
        // A buffer a is free once the MMAs of chunk q - kABufs completed
        if (!warp_wait_bounded(&a_done[a], ((q / kABufs) & 1) ^ 1, s_abort, err,
                               kRoleConv | (q << 8)))
          goto conv_done;
        tc_fence_after();
        const uint32_t t_a = tmem + lane_base + a * 32;
        {
          uint32_t hi[16], lo[16];
#pragma unroll
          for (int c = 0; c < 16; ++c) {
            const float a0 = v[2 * c], a1 = v[2 * c + 1];
            const __half2 h2 = __floats2half2_rn(a0, a1);
            const float2 hf = __half22float2(h2);
            const __half2 l2 = __floats2half2_rn(a0 - hf.x, a1 - hf.y);
            hi[c] = *reinterpret_cast<const uint32_t *>(&h2);
            lo[c] = *reinterpret_cast<const uint32_t *>(&l2);
          }
          tmem_st16(t_a, hi);
          tmem_st16(t_a + 16, lo);
        }
        tmem_st_wait();
        tc_fence_before();
        mbar_arrive(&a_full[a]);
      }
    }
  conv_done:;
  } else if (warp >= 8) {
    // ---------------------------------------------------------- epilogue
    const int row = tid - 256, wr = warp & 3, r32 = lane;
    const uint32_t lane_base = (uint32_t)(wr * 32) << 16;
    int o = 0;
    for (int it = 0; it < my_tiles; ++it) {
      const int tile = pair + it * npairs;
      const int r = it % kDcRing;
      if (!warp_wait_bounded(d_full, it & 1, s_abort, err, kRoleEpi | (it << 8))) break;
      tc_fence_after();
      if (!warp_wait_bounded(&dc_full[r], (it / kDcRing) & 1, s_abort, err, kRoleEpi | (it << 8)))
        break;
      const float x0 = s_dc[r * kTile + row];
      const uint32_t t_d = tmem + lane_base + 256;
      for (int j = 0; j < kOut / 32; ++j, ++o) {
        uint32_t d0[32], d1[32];
        tmem_ld32x2(t_d + 32 * j, t_d + kOut + 32 * j, d0, d1);
        if (j == kOut / 32 - 1) {
          tc_fence_before();
          mbar_arrive(d_empty);                // every column of D_0 and D_1 has been read
        }
        if (lane == 0) bulk_wait_read<1>();   // staging box o & 1 free
        __syncwarp();
        uint8_t *slab = s_out + ((o & 1) * 4 + wr) * kOutSlab;
#pragma unroll
        for (int u = 0; u < 8; ++u) {
          const float4 md = reinterpret_cast<const float4 *>(s_mdc)[8 * j + u];
          float4 y;
          y.x = fmaf(__uint_as_float(d0[4 * u]) + __uint_as_float(d1[4 * u]), out_scale, md.x * x0);
          y.y = fmaf(__uint_as_float(d0[4 * u + 1]) + __uint_as_float(d1[4 * u + 1]), out_scale,
                     md.y * x0);
          y.z = fmaf(__uint_as_float(d0[4 * u + 2]) + __uint_as_float(d1[4 * u + 2]), out_scale,
                     md.z * x0);
          y.w = fmaf(__uint_as_float(d0[4 * u + 3]) + __uint_as_float(d1[4 * u + 3]), out_scale,
                     md.w * x0);
          *reinterpret_cast<float4 *>(slab + r32 * 128 + ((u ^ (r32 & 7)) << 4)) = y;
        }
        fence_async_smem();
        __syncwarp();
        if (lane == 0) {
          tma_store_2d(&tm_out, slab, half * kOut + 32 * j, tile * kTile + wr * 32);
          bulk_commit();
        }
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

// [nblocks][256] FP32 rows; boxes of 32 floats x box_rows rows, 128-byte swizzle.
cudaError_t make_map(CUtensorMap *m, const void *ptr, int64_t nblocks, int box_rows) {
  EncodeTiledFn enc = encode_fn();
  if (enc == nullptr) return cudaErrorNotSupported;
  cuuint64_t dims[2] = {(cuuint64_t)kN2, (cuuint64_t)nblocks};
  cuuint64_t strides[1] = {(cuuint64_t)kN2 * 4};
  cuuint32_t box[2] = {32, (cuuint32_t)box_rows};
  cuuint32_t es[2] = {1, 1};
  CUresult r = enc(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<void *>(ptr), dims, strides,
                   box, es, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                   CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

}  // namespace

cudaError_t launch_apply_n16(const dctf_operator *op, const float *x, int64_t nblocks, float *y,
                             cudaStream_t s) {
  CUtensorMap tin, tout;
  cudaError_t e = make_map(&tin, x, nblocks, kTile);
  if (e == cudaSuccess) e = make_map(&tout, y, nblocks, 32);
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(apply_n16_f16x3_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           kSmem);
  if (e != cudaSuccess) return e;
  const int ntiles = (int)((nblocks + kTile - 1) / kTile);
  int pairs = sm_count(op->device) / 2;
  if (pairs > ntiles) pairs = ntiles;
  if (pairs < 1) pairs = 1;
  apply_n16_f16x3_kernel<<<2 * pairs, kThreads, kSmem, s>>>(
      tin, tout, reinterpret_cast<const uint4 *>(op->d_f16), op->d_Mdc,
      ldexpf(1.0f, -op->f16_scale_exp), ntiles, op->d_err);
  return cudaGetLastError();
}

}  // namespace dctf

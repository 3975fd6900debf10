// Tensor-core apply for 16x16 blocks (N^2 = 256): y_b = M x_b with a split
// precision, one kernel template per split.
//
// Every split writes x (the input coefficients, FP32) and M as sums of
// low-precision pieces, x = sum_i x_i and M = sum_j m_j, and accumulates
// the products x_i m_j^T that carry the result to FP32 accuracy, in FP32 in
// TMEM; the input DC coefficient is left out of the products and added as
// M[:,0] x[0] in FP32 in the epilogue (it is ~16x the block mean, by far the
// largest input).  The splits:
//
//   F16X3  : x, M 2^s in FP16 hi + lo; hi.lo, lo.hi, hi.hi          (kind::f16)
//   BF16X6 : x, M in three BF16 pieces; the six products with
//            i + j <= 2                                              (kind::f16, bf16)
//   TF32X3 : x, M in TF32 hi + lo; hi.lo, lo.hi, hi.hi              (kind::tf32)
//   TF32X1 : x, M rounded to TF32 once; one product (not exact)     (kind::tf32)
//   BF16X3 : x, M in BF16 hi + lo; hi.lo, lo.hi, hi.hi (~16 bits,
//            not exact)                                              (kind::f16, bf16)
//
// Tensor-core FP32 accumulation truncates, so the order matters: per K half
// of 128 inputs, each with its own accumulator, the correction products go
// in first (while the accumulator is small), the main product x_0 m_0 last;
// the epilogue adds the two halves with round-to-nearest.  BF16X6 instead
// keeps one accumulator per order i + j of its products (SplitBf16x6S
// below): each holds terms of one magnitude, so no order is needed, and its
// pieces stack into 3 wider MMAs per K step instead of 6.  TF32X3 does the
// same with its order 0 still split by K half (SplitTf32x3S): 2 MMAs per K
// step instead of 3.
//
// What 16x16 changes against the 8x8 kernel (apply_group.cu) is size: M is
// 256 x 256, its pieces 256-512 KB, more than one SM's shared memory, and a
// 128-block tile is 128 KB in and 128 KB out.  So:
//
//  * Output split.  A 128-block tile is processed by kParts = 256 / kOut
//    CTAs; CTA (group, part) computes output coefficients
//    [kOut part, kOut part + kOut).  Its kOut rows of every M piece stay
//    resident in shared memory for the whole launch (96-128 KB).  The CTAs
//    of a group read the same input tile (the later reads are L2 hits); each
//    writes its own slice of the output.
//  * K chunks.  The tile's input is streamed in eight 32-coefficient chunks
//    (16 KB, one SWIZZLE_128B box) through a TMA ring; the converter turns
//    each chunk into the A pieces in a TMEM ring, and the MMA warp issues
//    128 x kOut x K MMAs into the two accumulators of the tile.
//  * Output chunks.  Eight epilogue warps, two per TMEM lane quarter, each
//    reading half of the tile's output columns 32 at a time and TMA-storing
//    them as 32 x 8 boxes through one 1 KB staging box per warp; two warps
//    per quarter halve the time the (single-buffered, for kOut = 128)
//    accumulators are held after the MMAs (16x16 F16X3: 150 -> 133 us at
//    8192^2), and each warp releases them as soon as it has read its slices
//    (-> 128 us).
//
// Roles (512 threads): warp 0 TMA producer, warp 1 MMA issuer, warp 2 TMEM
// allocator, warps 4-7 converter (thread = tile row), warps 8-15 epilogue.
// All waits bounded, warp-uniform in multi-lane roles (sm100_ptx.cuh).
#include "sm100_ptx.cuh"

#include <mutex>

namespace dctf {
namespace {

using namespace ptx;

// ------------------------------------------------------------ the splits
// kPieces     : pieces of x and of M
// kImgPieces  : pieces stacked per chunk in the operator's piece image
// kTf32       : TF32 pieces (kind::tf32), else 16-bit pieces (kind::f16)
// kOut, kDBufs: outputs per CTA, accumulator sets (tiles) in TMEM
// kCorr       : correction products; corr_x(j), corr_m(j) their pieces
struct SplitF16x3 {
  static constexpr int kPieces = 2, kImgPieces = 2, kOut = 128, kDBufs = 1, kCorr = 2;
  static constexpr bool kTf32 = false, kBf16 = false;
  static constexpr bool kStacked = false, kHalvedOrder0 = false;
  __device__ static constexpr int corr_x(int j) { return j; }
  __device__ static constexpr int corr_m(int j) { return 1 - j; }
};
struct SplitBf16x3 {     // the first two BF16X6 pieces of M
  static constexpr int kPieces = 2, kImgPieces = 3, kOut = 128, kDBufs = 1, kCorr = 2;
  static constexpr bool kTf32 = false, kBf16 = true;
  static constexpr bool kStacked = false, kHalvedOrder0 = false;
  __device__ static constexpr int corr_x(int j) { return j; }
  __device__ static constexpr int corr_m(int j) { return 1 - j; }
};
// Stacked form of BF16X6: the products x_i m_j go into one accumulator per
// order i + j (1, 2^-8, 2^-16 of the result), each holding terms of one
// magnitude, so chunks need no ordering and a two-chunk A ring suffices; M's
// three pieces are stacked along N in each K block, so x_i [m_0 | ... |
// m_(2-i)] is one MMA of N = (3 - i) 64: 3 MMAs per K step instead of 6.
// Accumulator columns of a tile: [order 0 | order 1 | order 2].
struct SplitBf16x6S {
  static constexpr int kPieces = 3, kImgPieces = 3, kOut = 64, kDBufs = 2;
  static constexpr bool kTf32 = false, kBf16 = true;
  static constexpr bool kStacked = true, kHalvedOrder0 = false;
};
// Stacked form of TF32X3 with order 0 split by K half, since one order-0
// accumulator over all 256 inputs (32 truncating MMA additions) missed the
// error bar.  Accumulator columns of a tile: [order 0, K half 0 | order 1 |
// order 0, K half 1].  M's two pieces are stacked along N in each K block,
// [m_hi | m_lo] in the first K half and [m_lo | m_hi] in the second, so
// x_hi against both is one MMA of N = 128 into [A0 | O1], then [O1 | A1];
// x_lo m_hi is one of N = 64 into O1.  One accumulator set leaves TMEM a
// five-chunk A ring.
struct SplitTf32x3S {
  static constexpr int kPieces = 2, kImgPieces = 2, kOut = 64, kDBufs = 1;
  static constexpr bool kTf32 = true, kBf16 = false;
  static constexpr bool kStacked = true, kHalvedOrder0 = true;
};
struct SplitTf32x1 {
  static constexpr int kPieces = 1, kImgPieces = 2, kOut = 128, kDBufs = 1, kCorr = 0;
  static constexpr bool kTf32 = true, kBf16 = false;
  static constexpr bool kStacked = false, kHalvedOrder0 = false;
  __device__ static constexpr int corr_x(int) { return 0; }
  __device__ static constexpr int corr_m(int) { return 0; }
};

constexpr int kThreads = 512;
constexpr int kTile = 128;
constexpr int kN2 = 256;                 // coefficients per block
constexpr int kChunkK = 32;              // K per input chunk (one 128-byte box row)
constexpr int kChunks = kN2 / kChunkK;   // 8
constexpr int kGroups = 2;               // K halves, each with its own accumulator
// input chunk stages: see Layout::kStages
constexpr int kDcRing = 8;
constexpr uint32_t kTmemCols = 512;
constexpr uint32_t kRingCols = 256;      // A ring: columns 0..255; accumulators 256..511
constexpr int kChunkBytes = kTile * kChunkK * 4;    // 16 KB: one box (32 floats x 128 rows)
constexpr int kOutSlab = 32 * 32;                   // one warp's 32 x 8 floats box (SWIZZLE_32B)

template <class S>
struct Layout {
  // Input chunks arrive ~2,100 cycles after their TMA load is issued, and a
  // stage is issued again only once the converter has read it, so the
  // chunk rate is stages / (load latency + conversion): the two-CTA splits
  // (M's 128 output rows resident, 128 KB) fit five stages because each
  // epilogue warp stages its output in 32 x 8 quarters through 1 KB (16x16
  // F16X3 at 8192^2: 117 us with three stages, 109 with four, 94.5 with
  // five); the four-CTA splits keep three.
  static constexpr int kStages = S::kOut == 128 ? 5 : 3;
  static constexpr int kElem = S::kTf32 ? 4 : 2;            // bytes per piece element
  static constexpr int kRowElems = 128 / kElem;             // K per 128-byte B row
  static constexpr int kBlocksK = kN2 / kRowElems;          // 128-byte K blocks of B
  static constexpr int kPieceCols = kChunkK * kElem / 4;    // TMEM columns per A piece per chunk
  static constexpr int kABufCols = S::kPieces * kPieceCols;
  // accumulator columns a tile: two K halves of kOut, or (stacked) one of
  // kOut per order; the A ring takes the rest of TMEM
  static constexpr int kAccCols =
      S::kStacked ? (S::kHalvedOrder0 ? 3 : S::kPieces) * S::kOut : kGroups * S::kOut;
  static constexpr uint32_t kRing = kTmemCols - S::kDBufs * kAccCols;
  static constexpr int kABufs = kRing / kABufCols;
  static constexpr int kKStep = S::kTf32 ? 8 : 16;          // K per MMA
  static constexpr int kParts = kN2 / S::kOut;
  static constexpr int kBBlock = S::kOut * 128;             // one (piece, K block) of B
  static constexpr int kBBytes = S::kPieces * kBlocksK * kBBlock;
  static constexpr int kOffB = 0;
  static constexpr int kOffIn = kOffB + kBBytes;
  static constexpr int kOffOut = kOffIn + kStages * kChunkBytes;
  static constexpr int kOffMdc = kOffOut + 2 * 4 * kOutSlab;
  static constexpr int kOffDc = kOffMdc + S::kOut * 4;
  static constexpr int kOffBar = kOffDc + kDcRing * kTile * 4;
  static constexpr int kNumBars = 2 * kStages + 2 * kABufs + 2 * S::kDBufs + kDcRing + 1;
  static constexpr int kOffMisc = kOffBar + kNumBars * 8;
  static constexpr int kSmem = kOffMisc + 16 + 1024;
  static_assert(kSmem <= 232448, "shared memory");
  static_assert(S::kStacked ? kABufs >= 2 : kABufs >= kChunks / kGroups,
                "a K half's chunks must fit the A ring");
  static_assert(S::kStacked || kRing == kRingCols, "TMEM split");
  static_assert(kDcRing >= S::kDBufs + 2, "DC ring depth");
  static_assert(!(S::kTf32 && S::kBf16), "one piece type");
};

enum : uint32_t { kRoleProducer = 1, kRoleMma = 2, kRoleConv = 3, kRoleEpi = 4, kRoleDrain = 5 };

// Split one chunk row (32 FP32 inputs) into the A pieces and store them to
// this lane's TMEM row at column t_a (piece p at t_a + p kPieceCols).
template <class S>
__device__ __forceinline__ void convert_store(const float (&v)[32], uint32_t t_a) {
  if constexpr (S::kTf32) {
    uint32_t hi[32];
#pragma unroll
    for (int c = 0; c < 32; ++c) hi[c] = tf32_rna(v[c]);
    tmem_st32(t_a, hi);
    if constexpr (S::kPieces == 2) {
      uint32_t lo[32];
#pragma unroll
      for (int c = 0; c < 32; ++c) lo[c] = tf32_rna(v[c] - __uint_as_float(hi[c]));
      tmem_st32(t_a + 32, lo);
    }
  } else if constexpr (S::kBf16 && S::kPieces == 2) {
    // x ~ x0 + x1 (16 of FP32's 24 bits)
    uint32_t p0[16], p1[16];
#pragma unroll
    for (int c = 0; c < 16; ++c) {
      const float a0 = v[2 * c], a1 = v[2 * c + 1];
      const __nv_bfloat162 b0 = __floats2bfloat162_rn(a0, a1);
      const float2 f0 = __bfloat1622float2(b0);
      const __nv_bfloat162 b1 = __floats2bfloat162_rn(a0 - f0.x, a1 - f0.y);
      p0[c] = *reinterpret_cast<const uint32_t *>(&b0);
      p1[c] = *reinterpret_cast<const uint32_t *>(&b1);
    }
    tmem_st16(t_a, p0);
    tmem_st16(t_a + 16, p1);
  } else if constexpr (S::kBf16) {
    // x = x0 + x1 + x2 exactly (FP32 has 24 bits, each BF16 piece takes 8)
    uint32_t p0[16], p1[16], p2[16];
#pragma unroll
    for (int c = 0; c < 16; ++c) {
      const float a0 = v[2 * c], a1 = v[2 * c + 1];
      const __nv_bfloat162 b0 = __floats2bfloat162_rn(a0, a1);
      const float2 f0 = __bfloat1622float2(b0);
      const float r0 = a0 - f0.x, r1 = a1 - f0.y;
      const __nv_bfloat162 b1 = __floats2bfloat162_rn(r0, r1);
      const float2 f1 = __bfloat1622float2(b1);
      const __nv_bfloat162 b2 = __floats2bfloat162_rn(r0 - f1.x, r1 - f1.y);
      p0[c] = *reinterpret_cast<const uint32_t *>(&b0);
      p1[c] = *reinterpret_cast<const uint32_t *>(&b1);
      p2[c] = *reinterpret_cast<const uint32_t *>(&b2);
    }
    tmem_st16(t_a, p0);
    tmem_st16(t_a + 16, p1);
    tmem_st16(t_a + 32, p2);
  } else {
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
}

// Stacked splits: x_i [m_0 | ... | m_(P-1-i)], N = (P - i) kOut.
template <class S, int I>
__device__ __forceinline__ void mma_stacked(uint32_t d, uint32_t a, uint64_t b, uint32_t acc) {
  constexpr int kN = (S::kPieces - I) * S::kOut;
  if constexpr (S::kTf32)
    mma_tf32_ts(d, a, b, idesc_tf32(128, kN), acc);
  else
    mma_f16_ts(d, a, b, idesc_f16(128, kN, S::kBf16), acc);
}

template <class S, int N>
__device__ __forceinline__ void mma_n(uint32_t d, uint32_t a, uint64_t b, uint32_t acc) {
  if constexpr (S::kTf32)
    mma_tf32_ts(d, a, b, idesc_tf32(128, N), acc);
  else
    mma_f16_ts(d, a, b, idesc_f16(128, N, S::kBf16), acc);
}

template <class S>
__device__ __forceinline__ void mma_ts(uint32_t d, uint32_t a, uint64_t b, uint32_t acc) {
  if constexpr (S::kTf32)
    mma_tf32_ts(d, a, b, idesc_tf32(128, S::kOut), acc);
  else
    mma_f16_ts(d, a, b, idesc_f16(128, S::kOut, S::kBf16), acc);
}

template <class S>
__global__ void __launch_bounds__(kThreads, 1)
apply_n16_kernel(const __grid_constant__ CUtensorMap tm_in, const __grid_constant__ CUtensorMap tm_out,
                 const uint4 *__restrict__ pieces, const float *__restrict__ Mdc, float out_scale,
                 int ntiles, uint32_t *__restrict__ err) {
  using L = Layout<S>;
  constexpr int kOut = S::kOut, kABufs = L::kABufs, kDBufs = S::kDBufs, kStages = L::kStages;
  extern __shared__ uint8_t smem_raw[];
  uint8_t *base = reinterpret_cast<uint8_t *>(
      (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  uint8_t *s_b = base + L::kOffB;
  uint8_t *s_in = base + L::kOffIn;
  uint8_t *s_out = base + L::kOffOut;
  float *s_mdc = reinterpret_cast<float *>(base + L::kOffMdc);
  float *s_dc = reinterpret_cast<float *>(base + L::kOffDc);
  uint64_t *bars = reinterpret_cast<uint64_t *>(base + L::kOffBar);
  uint64_t *full_in = bars;                     // [kStages]
  uint64_t *empty_in = full_in + kStages;       // [kStages]
  uint64_t *a_full = empty_in + kStages;        // [kABufs]
  uint64_t *a_done = a_full + kABufs;           // [kABufs] MMA finished reading the chunk
  uint64_t *d_full = a_done + kABufs;           // [kDBufs]
  uint64_t *d_empty = d_full + kDBufs;          // [kDBufs]
  uint64_t *dc_full = d_empty + kDBufs;         // [kDcRing]
  uint64_t *b_full = dc_full + kDcRing;         // the resident pieces have landed
  uint32_t *s_tmem = reinterpret_cast<uint32_t *>(base + L::kOffMisc);
  volatile int *s_abort = reinterpret_cast<volatile int *>(base + L::kOffMisc + 4);

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int part = blockIdx.x % L::kParts;
  const int grp = blockIdx.x / L::kParts, ngroups = gridDim.x / L::kParts;
  const int my_tiles = grp < ntiles ? (ntiles - grp + ngroups - 1) / ngroups : 0;

  if (tid == 0) {
    for (int s = 0; s < kStages; ++s) { mbar_init(&full_in[s], 1); mbar_init(&empty_in[s], 128); }
    for (int a = 0; a < kABufs; ++a) { mbar_init(&a_full[a], 128); mbar_init(&a_done[a], 1); }
    for (int d = 0; d < kDBufs; ++d) { mbar_init(&d_full[d], 1); mbar_init(&d_empty[d], 256); }
    for (int r = 0; r < kDcRing; ++r) mbar_init(&dc_full[r], 128);
    mbar_init(b_full, 1);
    *s_abort = 0;
    mbar_fence_init();
    tma_prefetch_map(&tm_in);
  }
  if (tid < kOut) s_mdc[tid] = __ldg(Mdc + part * kOut + tid);
  fence_async_smem();
  if (warp == 2) { tmem_alloc(s_tmem, kTmemCols); tmem_relinquish(); }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *s_tmem;
  // A launch of this kernel that follows on the stream may be scheduled now
  // (it only does so when launched for programmatic stream serialisation).
  if (tid == 0) pdl_launch_dependents();

  if (warp == 0 && lane == 0) {
    // ---------------------------------------------------------- producer
    // resident B first: for each piece and 128-byte K block, this part's
    // kOut rows, a contiguous 16 KB (kOut = 128) or 8 KB block of the
    // operator's piece image (K block kb holds kImgPieces * 256 rows: piece
    // p's output t at row p * 256 + t), copied in the background while the
    // first input chunks load and convert; the MMA warp waits for it.  (A
    // thread-by-thread copy before the roles start cost ~7 us a launch.)
    mbar_arrive_expect_tx(b_full, L::kBBytes);
    for (int blk = 0; blk < S::kPieces * L::kBlocksK; ++blk) {
      // piece-major blocks; stacked: K-block-major, the pieces adjacent
      const int kb = S::kStacked ? blk / S::kPieces : blk % L::kBlocksK;
      // (halved order 0: the pieces in reverse order in the second K half)
      const int slot = blk % S::kPieces;
      const int piece = !S::kStacked ? blk / L::kBlocksK
                        : (S::kHalvedOrder0 && kb >= L::kBlocksK / 2) ? S::kPieces - 1 - slot
                                                                       : slot;
      const size_t src_row0 = (size_t)kb * S::kImgPieces * kN2 + piece * kN2 + part * kOut;
      bulk_load(s_b + blk * L::kBBlock, pieces + src_row0 * 8, L::kBBlock, b_full);
    }
    int q = 0, issued = 0;
    for (int it = 0; it < my_tiles; ++it) {
      const int tile = grp + it * ngroups;
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
    wait_drain(b_full, 0, err, kRoleDrain);
    for (int k = issued > kStages ? issued - kStages : 0; k < issued; ++k)
      wait_drain(&full_in[k % kStages], (k / kStages) & 1, err, kRoleDrain);
  } else if (warp == 1 && lane == 0) {
    // ---------------------------------------------------------- MMA issuer
    // Tile t, K half g: D_g = sum over its 4 chunks of the correction
    // products, then of the main product; a chunk's A buffer is released
    // after its main product.
    int q = 0, last_q = -1;
    if (my_tiles > 0 && !wait_bounded(b_full, 0, s_abort, err, kRoleMma))
      goto mma_done_label;
    if constexpr (S::kStacked) {
      // Tile t: the accumulator of order o (columns o kOut ..) gets every
      // x_i m_j with i + j = o, chunk by chunk; a chunk's A buffer is
      // released after its MMAs
      for (int it = 0; it < my_tiles; ++it) {
        const int db = it % kDBufs;
        if (!wait_bounded(&d_empty[db], ((it / kDBufs) & 1) ^ 1, s_abort, err,
                          kRoleMma | (it << 8)))
          goto mma_done_label;
        const uint32_t t_d = tmem + L::kRing + db * L::kAccCols;
        for (int kc = 0; kc < kChunks; ++kc, ++q) {
          const int a = q % kABufs;
          if (!wait_bounded(&a_full[a], (q / kABufs) & 1, s_abort, err, kRoleMma | (q << 8)))
            goto mma_done_label;
          tc_fence_after();
          const uint32_t t_a = tmem + a * L::kABufCols;
          const int kb = kc * kChunkK / L::kRowElems;
          const int kofs = (kc * kChunkK % L::kRowElems) * L::kElem / 16;   // 16-byte units
          // K block kb: the pieces' kOut rows stacked, m_0 first
          const uint32_t s_blk = smem_u32(s_b + kb * S::kPieces * L::kBBlock);
          const uint64_t b = desc_sw128(s_blk) + kofs;
          if constexpr (S::kHalvedOrder0) {
            // K half 0: B = [m_hi | m_lo] -> [A0 | O1]; half 1: [m_lo | m_hi] -> [O1 | A1]
            const bool h1 = kc >= kChunks / 2;
            const uint64_t b_second = desc_sw128(s_blk + L::kBBlock) + kofs;
            const uint64_t b_mhi = h1 ? b_second : b;
#pragma unroll
            for (int kk = 0; kk < kChunkK / L::kKStep; ++kk) {
              if (kc == kChunks / 2 && kk == 0) {
                // A1 starts here while O1 goes on: the pair as two MMAs
                mma_n<S, kOut>(t_d + kOut, t_a, b, 1u);                 // x_hi m_lo -> O1
                mma_n<S, kOut>(t_d + 2 * kOut, t_a, b_second, 0u);      // x_hi m_hi -> A1
              } else {
                mma_n<S, 2 * kOut>(h1 ? t_d + kOut : t_d, t_a + 8 * kk, b + 2 * kk,
                                   (kc > 0 || kk > 0) ? 1u : 0u);
              }
              mma_n<S, kOut>(t_d + kOut, t_a + L::kPieceCols + 8 * kk, b_mhi + 2 * kk, 1u);
            }
          } else {
#pragma unroll
            for (int kk = 0; kk < kChunkK / L::kKStep; ++kk) {
              mma_stacked<S, 0>(t_d, t_a + 8 * kk, b + 2 * kk, (kc > 0 || kk > 0) ? 1u : 0u);
              mma_stacked<S, 1>(t_d + kOut, t_a + L::kPieceCols + 8 * kk, b + 2 * kk, 1u);
              mma_stacked<S, 2>(t_d + 2 * kOut, t_a + 2 * L::kPieceCols + 8 * kk, b + 2 * kk, 1u);
            }
          }
          tc_commit(&a_done[a]);
          last_q = q;
        }
        tc_commit(&d_full[db]);
      }
    } else {
    for (int it = 0; it < my_tiles; ++it) {
      const int db = it % kDBufs;
      if (!wait_bounded(&d_empty[db], ((it / kDBufs) & 1) ^ 1, s_abort, err, kRoleMma | (it << 8)))
        goto mma_done_label;
      for (int g = 0; g < kGroups; ++g) {
        const uint32_t t_d = tmem + kRingCols + (db * kGroups + g) * kOut;
        const int q0 = q + g * (kChunks / kGroups);
        for (int c = 0; c < kChunks / kGroups; ++c) {
          const int qc = q0 + c, a = qc % kABufs, kc = g * (kChunks / kGroups) + c;
          if (!wait_bounded(&a_full[a], (qc / kABufs) & 1, s_abort, err, kRoleMma | (qc << 8)))
            goto mma_done_label;
          tc_fence_after();
          const uint32_t t_a = tmem + a * L::kABufCols;
          // chunk kc covers K [32 kc, 32 kc + 32): K block kc * 32 / kRowElems
          // of B, starting (kc * 32 % kRowElems) elements into its rows
          const int kb = kc * kChunkK / L::kRowElems;
          const int kofs = (kc * kChunkK % L::kRowElems) * L::kElem / 16;   // 16-byte units
#pragma unroll
          for (int j = 0; j < S::kCorr; ++j) {
            const uint64_t b = desc_sw128(smem_u32(
                                   s_b + (S::corr_m(j) * L::kBlocksK + kb) * L::kBBlock)) + kofs;
#pragma unroll
            for (int kk = 0; kk < kChunkK / L::kKStep; ++kk)
              mma_ts<S>(t_d, t_a + S::corr_x(j) * L::kPieceCols + 8 * kk, b + 2 * kk,
                        (c > 0 || j > 0 || kk > 0) ? 1u : 0u);
          }
        }
        for (int c = 0; c < kChunks / kGroups; ++c) {
          const int qc = q0 + c, a = qc % kABufs, kc = g * (kChunks / kGroups) + c;
          const uint32_t t_a = tmem + a * L::kABufCols;
          const int kb = kc * kChunkK / L::kRowElems;
          const int kofs = (kc * kChunkK % L::kRowElems) * L::kElem / 16;
          const uint64_t b = desc_sw128(smem_u32(s_b + kb * L::kBBlock)) + kofs;
#pragma unroll
          for (int kk = 0; kk < kChunkK / L::kKStep; ++kk)
            mma_ts<S>(t_d, t_a + 8 * kk, b + 2 * kk, (S::kCorr > 0 || c > 0 || kk > 0) ? 1u : 0u);
          tc_commit(&a_done[a]);
          last_q = qc;
        }
      }
      q += kChunks;
      tc_commit(&d_full[db]);
    }
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
          // ring slot it % kDcRing is free: to get here the converter waited
          // for the MMAs of a chunk of tile it - 2 or later, which began
          // after the epilogue had read tile it - 2 - kDBufs, so at most
          // kDBufs + 1 earlier tiles still hold slots (kDcRing >= kDBufs + 2)
          const int r = it % kDcRing;
          s_dc[r * kTile + row] = v[0];
          v[0] = 0.f;
          mbar_arrive(&dc_full[r]);
        }
        // A buffer a is free once the MMAs of chunk q - kABufs completed
        if (!warp_wait_bounded(&a_done[a], ((q / kABufs) & 1) ^ 1, s_abort, err,
                               kRoleConv | (q << 8)))
          goto conv_done;
        tc_fence_after();
        convert_store<S>(v, tmem + lane_base + a * L::kABufCols);
        tmem_st_wait();
        tc_fence_before();
        mbar_arrive(&a_full[a]);
      }
    }
  conv_done:;
  } else if (warp >= 8) {
    // ---------------------------------------------------------- epilogue
    // eight warps: warp 8 + 4 h + q reads TMEM lanes 32 q.. (its rows) and
    // output columns [h kOut / 2, (h + 1) kOut / 2)
    const int ew = warp - 8, wr = warp & 3, hc = ew >> 2, r32 = lane, row = wr * 32 + lane;
    const uint32_t lane_base = (uint32_t)(wr * 32) << 16;
    constexpr int kJ = kOut / 64;              // 32-column slices per warp
    // Under programmatic dependent launch the loads may run while the
    // previous kernel on the stream finishes; no output is written before
    // that kernel has completed (it may still read the output buffer).
    if (lane == 0) pdl_wait();
    __syncwarp();
    for (int it = 0; it < my_tiles; ++it) {
      const int tile = grp + it * ngroups;
      const int r = it % kDcRing, db = it % kDBufs;
      if (!warp_wait_bounded(&d_full[db], (it / kDBufs) & 1, s_abort, err, kRoleEpi | (it << 8)))
        break;
      tc_fence_after();
      if (!warp_wait_bounded(&dc_full[r], (it / kDcRing) & 1, s_abort, err, kRoleEpi | (it << 8)))
        break;
      const float x0 = s_dc[r * kTile + row];
      const uint32_t t_d = tmem + lane_base + L::kRing + db * L::kAccCols;
      // read this warp's slices of both K-half accumulators (stacked: of
      // every order, the smallest first) and add them, then release D before
      // staging and storing, so the next tile's MMAs need not wait for the
      // stores (16x16 F16X3: 135 -> 128 us at 8192^2)
      float acc[kJ][32];
#pragma unroll
      for (int jj = 0; jj < kJ; ++jj) {
        const int j = hc * kJ + jj;
        uint32_t d0[32], d1[32];
        if constexpr (S::kStacked) {
          tmem_ld32x2(t_d + 2 * kOut + 32 * j, t_d + kOut + 32 * j, d0, d1);
#pragma unroll
          for (int c = 0; c < 32; ++c) acc[jj][c] = __uint_as_float(d0[c]) + __uint_as_float(d1[c]);
          tmem_ld32(t_d + 32 * j, d0);
#pragma unroll
          for (int c = 0; c < 32; ++c) acc[jj][c] += __uint_as_float(d0[c]);
        } else {
          tmem_ld32x2(t_d + 32 * j, t_d + kOut + 32 * j, d0, d1);
#pragma unroll
          for (int c = 0; c < 32; ++c) acc[jj][c] = __uint_as_float(d0[c]) + __uint_as_float(d1[c]);
        }
      }
      tc_fence_before();
      mbar_arrive(&d_empty[db]);               // this warp's columns of D have been read
#pragma unroll
      for (int jj = 0; jj < kJ; ++jj) {
        const int j = hc * kJ + jj;
        // four 32 x 8 quarters of the slice through the warp's 1 KB box
#pragma unroll
        for (int hh = 0; hh < 4; ++hh) {
          if (lane == 0) bulk_wait_read<0>();   // the warp's staging box is free
          __syncwarp();
          uint8_t *slab = s_out + ew * kOutSlab;
#pragma unroll
          for (int u = 0; u < 2; ++u) {
            const int uu = 2 * hh + u;
            const float4 md = reinterpret_cast<const float4 *>(s_mdc)[8 * j + uu];
            float4 y;
            y.x = fmaf(acc[jj][4 * uu], out_scale, md.x * x0);
            y.y = fmaf(acc[jj][4 * uu + 1], out_scale, md.y * x0);
            y.z = fmaf(acc[jj][4 * uu + 2], out_scale, md.z * x0);
            y.w = fmaf(acc[jj][4 * uu + 3], out_scale, md.w * x0);
            // SWIZZLE_32B: 16-byte chunk u of 32-byte row r32 at u ^ ((r32 >> 2) & 1)
            *reinterpret_cast<float4 *>(slab + r32 * 32 + ((u ^ ((r32 >> 2) & 1)) << 4)) = y;
          }
          fence_async_smem();
          __syncwarp();
          if (lane == 0) {
            tma_store_2d(&tm_out, slab, part * kOut + 32 * j + 8 * hh, tile * kTile + wr * 32);
            bulk_commit();
          }
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

// [nblocks][256] FP32 rows; boxes of box_cols floats x box_rows rows (32
// floats: 128-byte swizzle, the input chunks; 16 floats: 64-byte swizzle,
// the output halves).
cudaError_t make_map(CUtensorMap *m, const void *ptr, int64_t nblocks, int box_rows,
                     int box_cols = 32) {
  EncodeTiledFn enc = encode_fn();
  if (enc == nullptr) return cudaErrorNotSupported;
  cuuint64_t dims[2] = {(cuuint64_t)kN2, (cuuint64_t)nblocks};
  cuuint64_t strides[1] = {(cuuint64_t)kN2 * 4};
  cuuint32_t box[2] = {(cuuint32_t)box_cols, (cuuint32_t)box_rows};
  cuuint32_t es[2] = {1, 1};
  CUresult r = enc(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<void *>(ptr), dims, strides,
                   box, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
                   box_cols == 32   ? CU_TENSOR_MAP_SWIZZLE_128B
                   : box_cols == 16 ? CU_TENSOR_MAP_SWIZZLE_64B
                                    : CU_TENSOR_MAP_SWIZZLE_32B,
                   CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

template <class S>
cudaError_t launch(const dctf_operator *op, const void *pieces, float out_scale,
                   const CUtensorMap &tin, const CUtensorMap &tout, int ntiles, cudaStream_t s,
                   bool pdl) {
  using L = Layout<S>;
  cudaError_t e = cudaFuncSetAttribute(apply_n16_kernel<S>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, L::kSmem);
  if (e != cudaSuccess) return e;
  int groups = sm_count(op->device) / L::kParts;
  if (groups > ntiles) groups = ntiles;
  if (groups < 1) groups = 1;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(L::kParts * groups);
  cfg.blockDim = dim3(kThreads);
  cfg.dynamicSmemBytes = L::kSmem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  if (pdl) {
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
  }
  e = cudaLaunchKernelEx(&cfg, apply_n16_kernel<S>, tin, tout,
                         reinterpret_cast<const uint4 *>(pieces), op->d_Mdc, out_scale, ntiles,
                         op->d_err);
  if (e != cudaSuccess) return e;
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_apply_n16(const dctf_operator *op, const float *x, int64_t nblocks, float *y,
                             cudaStream_t s, bool pdl) {
  if (op->d_f16 == nullptr || op->d_bf16 == nullptr || op->d_tf32 == nullptr)
    return cudaErrorInvalidValue;
  CUtensorMap tin, tout;
  cudaError_t e = make_map(&tin, x, nblocks, kTile);
  if (e == cudaSuccess) e = make_map(&tout, y, nblocks, 32, 8);
  if (e != cudaSuccess) return e;
  const int ntiles = (int)((nblocks + kTile - 1) / kTile);
  switch (op->precision) {
    case DCTF_F16X3:
      return launch<SplitF16x3>(op, op->d_f16, ldexpf(1.0f, -op->f16_scale_exp), tin, tout, ntiles, s, pdl);
    case DCTF_BF16X6:
      return launch<SplitBf16x6S>(op, op->d_bf16, 1.0f, tin, tout, ntiles, s, pdl);
    case DCTF_TF32X3:
      return launch<SplitTf32x3S>(op, op->d_tf32, 1.0f, tin, tout, ntiles, s, pdl);
    case DCTF_TF32X1:
      return launch<SplitTf32x1>(op, op->d_tf32, 1.0f, tin, tout, ntiles, s, pdl);
    case DCTF_BF16X3:
      return launch<SplitBf16x3>(op, op->d_bf16, 1.0f, tin, tout, ntiles, s, pdl);
    default:
      return cudaErrorInvalidValue;
  }
}

}  // namespace dctf

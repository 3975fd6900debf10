// Persistent grouped tensor-core apply: many (image, operator) items, one
// launch.  y_b = M_item x_b for every block b of every item (Eq. 11 / 20).
//
// The batched product Y[b][n] = sum_k X[b][k] M[n][k] is a GEMM with M = 128
// blocks per tile, N = 64 outputs, K = 64 inputs.  It moves 512 bytes per
// block for 8192 flops, so it is bound by HBM; the tensor cores only have to
// keep up, which leaves room for a 3-product split that restores FP32-level
// accuracy from FP16 operands:
//   x = x_hi + x_lo, M 2^s = M_hi + M_lo (FP16, round to nearest),
//   y = (x_hi M_hi + x_hi M_lo + x_lo M_hi) 2^-s + M[:,0] x[0],
// accumulated in FP32 in TMEM.  The input DC coefficient x[0] (by far the
// largest) is kept out of the split and the long sums and applied in FP32 in
// the epilogue, which keeps pixel errors near 1e-5.  dctf_apply runs this
// kernel with one item; the grouped entry points with many.  Features:
//
//  * Work items.  Each item has its own operator (B pieces and M[:,0] in
//    global memory), its own coefficient arrays (TMA tensor maps kept in the
//    item descriptor), and, for quantised I/O, its own quantisation tables.
//  * Balanced contiguous schedule.  The blocks of all items form one sequence
//    of 64-block half tiles; CTA c takes the contiguous range
//    [c H / G, (c+1) H / G).  Inside an item, consecutive halves pair up into
//    128-row MMA tiles; a range or item boundary can leave a 64-row tile.
//    The part of a range inside one item is a "segment".
//  * Operator slots.  A loader warp copies each segment's B pieces, M[:,0]
//    and quantisation tables into one of two shared-memory slots
//    (cp.async.bulk), one segment ahead, so operator switches overlap the
//    previous segment's tiles.
//  * Quantised I/O (IoT = int16_t): the converter dequantises x = Q q_in
//    before the split, the epilogue requantises round_half_away(y / q_out)
//    with int16 saturation, so int16 coefficients go HBM -> HBM directly.
//  * Pixel output (kMode = kModePixels): the operator is G = H K^T, which takes a block's
//    DCT coefficients straight to its filtered pixels (K^T K = I, so
//    K^T M = H K^T, Eq. 3 applied after Eq. 7); the epilogue rounds half
//    away from zero, saturates to [0, 255] and writes the block's 8 x 8
//    bytes into the image (Sec. III's conversion), 64 B per block instead
//    of 256 B of coefficients.  One image goes through kModePixelsHalf:
//    the same arithmetic in CTAs of half an SM, two per SM, so a CTA of the
//    next launch fills an SM while the other CTA there drains.
//  * Image-plane layout (kMode = kModePlanar): the coefficients of block
//    (by, bx) sit at rows 8 by + u, columns 8 bx + v of an image-shaped FP32
//    array (the layout of a JPEG decoder's coefficient plane).  A 2-D TMA
//    view moves boxes of 256 floats x 8 rows (32 blocks of one block row,
//    1 KB runs): four per 128-block tile on load, one per epilogue warp on
//    store; block rows are padded to a multiple of 128 blocks in the tile
//    walk (the padding is outside the tensor: zero-filled on load, clipped
//    or skipped on store).
//  * Host-direct I/O (kMode = kModeHost): the coefficients stay in page-locked
//    host memory mapped into the device address space.  The whole producer
//    warp copies each 32 KB input tile with 16-byte cp.async into the same
//    swizzled stage layout the TMA box gives (zero-filled past the last
//    block), and the epilogue warps write their staged outputs to host
//    memory with coalesced 16-byte stores.  Every byte crosses the host link
//    once each way, with no device buffer and no copy engine.
//
// Roles (384 threads; 512 in the pixel mode): warp 0 TMA producer, warp 1
// MMA issuer, warp 2 TMEM allocator, warp 3 slot loader, warps 4-7
// converter (thread = tile row), warps 8-11 epilogue (each warp stores its
// own 32 rows; the pixel mode adds warps 12-15, the two sets of four taking
// alternate tiles).  TMEM holds a ring of four [A_hi 32 | A_lo 32 | D 64]
// column buffers (two in the half-SM pixel mode), so the MMA can run up to
// four tiles ahead of the epilogue, which frees its buffer right after one
// paired TMEM load.  Launched for programmatic stream serialisation, a CTA
// lets the next launch be scheduled once it is set up, and its epilogue
// writes nothing before the previous kernel has completed.  Every wait is bounded (see sm100_ptx.cuh); waits in
// multi-lane roles are warp-uniform.
#include "apply_group.cuh"

#include <mutex>

namespace dctf {
namespace {

using namespace ptx;

constexpr int kTile = 128;
constexpr int kHalf = 64;
constexpr int kN2 = 64;
constexpr uint32_t kTmemCols = 512;

template <typename IoT> struct Io;
template <> struct Io<float> {
  static constexpr int kRowBytes = kN2 * 4;                 // 256
  static constexpr int kBoxCols = 32;                       // 128-byte swizzle rows
  static constexpr int kBoxesPerRow = 2;
};
template <> struct Io<int16_t> {
  static constexpr int kRowBytes = kN2 * 2;                 // 128
  static constexpr int kBoxCols = 64;
  static constexpr int kBoxesPerRow = 1;
};

constexpr int kBufs = 4;        // TMEM ring: [A_hi 32 | A_lo 32 | D 64] columns each
                                // (DC ring: twice as deep, Layout::kDcRing)

// S input stages, NS operator slots (1 for a single item, 2 for groups), OB
// output staging buffers (2; 0 for the pixel output, which stores from
// registers and spends that shared memory on input stages instead)
template <typename IoT, int S, int NS, int OB = 2, int NB = kBufs> struct Layout {
  static constexpr int kDcRing = 2 * NB;
  static constexpr int kStageBytes = kTile * Io<IoT>::kRowBytes;
  static constexpr int kBoxBytes = kTile * 128;              // one 128-row box
  static constexpr int kSlabBytes = 32 * Io<IoT>::kRowBytes; // one warp's output rows
  static constexpr int kSlabBoxBytes = 32 * 128;
  static constexpr int kOffIn = 0;
  static constexpr int kOffOut = kOffIn + S * kStageBytes;
  static constexpr int kOffSlot = kOffOut + OB * kStageBytes;
  static constexpr int kOffDc = kOffSlot + NS * kSlotBytes;
  static constexpr int kOffBar = kOffDc + kDcRing * kTile * 4;
  static constexpr int kNumBars = 2 * S + 3 * NB + kDcRing + 2 * NS;
  static constexpr int kOffMisc = kOffBar + kNumBars * 8;
  static constexpr int kSmem = kOffMisc + 16 + 1024;
  static_assert(kSmem <= 232448, "shared memory");
};

enum : uint32_t { kRoleProducer = 1, kRoleMma = 2, kRoleConv = 3, kRoleEpi = 4, kRoleDrain = 5,
                  kRoleLoader = 6 };

struct Tile {
  int item;
  int seg;
  bool seg_first, seg_last;
  int row0;      // first block of the tile inside its item
  int rows;      // 64 or 128
};

// Walks this CTA's tiles; every role runs its own copy and sees the same
// sequence.  Contiguous mode (groups): CTA c owns half tiles
// [c H / G, (c+1) H / G), pairing them into 128-row tiles inside each item.
// Interleaved mode (one item): full 128-row tiles are dealt round-robin
// (tile k of CTA c is tile k G + c) while every CTA gets one; the remaining
// halves are dealt one per CTA, so no CTA carries more than half a tile of
// extra work.
struct TileWalk {
  const GroupItem *items;
  int nitems;
  int64_t h, h1;          // contiguous mode: current / end half index (global)
  int max_take;           // halves per tile: 2 (128-row tiles) or 1 (64-row tiles)
  bool interleaved;
  int64_t k, full_rounds, rem_base, H;   // interleaved mode
  int rem_step;
  int item;
  int64_t ih0, ih1;       // current item's global half range
  int seg;
  int64_t seg_h0;
  bool started;

  __device__ void init(const GroupItem *it, int n, int64_t total, int take, bool inter) {
    items = it;
    nitems = n;
    max_take = take;
    interleaved = inter;
    seg = 0;
    started = false;
    if (interleaved) {
      H = total;
      const int64_t G = gridDim.x;
      full_rounds = take == 2 ? H / (2 * G) : 0;
      k = 0;
      rem_base = full_rounds * 2 * G;
      rem_step = 0;
      item = 0;
      load_item();
      return;
    }
    h = total * blockIdx.x / gridDim.x;
    h1 = total * (blockIdx.x + 1) / gridDim.x;
    // the item holding half h (half_begin is increasing)
    int lo = 0, hi = n - 1;
    while (lo < hi) {
      int mid = (lo + hi + 1) >> 1;
      if (items[mid].half_begin <= h) lo = mid; else hi = mid - 1;
    }
    item = lo;
    load_item();
    seg_h0 = h;
  }
  __device__ void load_item() {
    ih0 = items[item].half_begin;
    ih1 = ih0 + (items[item].nblocks + kHalf - 1) / kHalf;
  }
  __device__ bool next_interleaved(Tile &t) {
    const int64_t G = gridDim.x;
    int64_t half;
    int take;
    if (k < full_rounds) {
      half = 2 * (k * G + blockIdx.x);
      take = 2;
      ++k;
    } else {
      half = rem_base + blockIdx.x + (int64_t)rem_step * G;
      if (half >= H) return false;
      take = 1;
      ++rem_step;
    }
    t.item = 0;
    t.seg = 0;
    t.seg_first = !started;
    started = true;
    t.row0 = (int)(half * kHalf);
    t.rows = take * kHalf;
    // last tile of this CTA?
    bool more;
    if (k < full_rounds) more = true;
    else more = rem_base + blockIdx.x + (int64_t)rem_step * G < H;
    t.seg_last = !more;
    return true;
  }
  __device__ bool next(Tile &t) {
    if (interleaved) return next_interleaved(t);
    if (h >= h1) return false;
    while (h >= ih1) {          // skips items without blocks as well
      if (item + 1 >= nitems) return false;
      ++item;
      load_item();
      ++seg;
      seg_h0 = h;
    }
    const int64_t end = ih1 < h1 ? ih1 : h1;
    const int take = (end - h >= 2 && max_take == 2) ? 2 : 1;
    t.item = item;
    t.seg = seg;
    t.seg_first = (h == seg_h0);
    t.row0 = (int)((h - ih0) * kHalf);
    t.rows = take * kHalf;
    h += take;
    t.seg_last = (h == end);
    return true;
  }
};

// uint8 of a filtered pixel: round half away from zero and saturate to
// [0, 255] (Sec. III's conversion), on the FMA/ALU pipes only: clamp, add
// 0.5, then add 2^23 rounding toward zero, which leaves floor(p + 0.5) in
// the low mantissa bits.  (Rounding and float-to-integer conversion
// instructions run on the slower XU pipe, which made the pixel epilogue
// the bottleneck of the fused kernel.)  A value within one FP32 ulp below
// a .5 boundary may round up: inside the 1e-4 tie band.  The pixel is the
// low byte of the result (the higher bits hold the exponent of 2^23); the
// caller packs low bytes with PRMT, so no mask is needed.
__device__ __forceinline__ uint32_t pixel_u8_low_byte(float p) {
  const float c = fminf(fmaxf(p, 0.f), 255.f) + 0.5f;
  return __float_as_uint(__fadd_rz(c, 8388608.0f));
}

// FP32 I/O: at most 152 registers a thread (58,368 of the SM's 65,536 for 384
// threads), so the small FP64 operator-build kernels of the next image can
// run on the same SMs while this kernel streams.
enum : int { kModeBlocks = 0, kModePixels = 1, kModePlanar = 2, kModeHost = 3, kModePixelsHalf = 4 };

// kModePixelsHalf: the pixel output of one image in CTAs of half an SM (384
// threads x 80 registers, two input stages, two TMEM buffers of the ring,
// 256 columns, ~85 KB of shared memory), two per SM.  One launch of whole-SM
// CTAs loses its first load's latency and its last tiles' drain, which no
// CTA of the next launch can fill; with two CTAs an SM, a CTA of the next
// launch starts on an SM as soon as one of this launch's CTAs there has
// left, so fills and drains overlap.
__host__ __device__ constexpr bool is_pixels(int mode) {
  return mode == kModePixels || mode == kModePixelsHalf;
}
__host__ __device__ constexpr int ring_bufs(int mode) { return mode == kModePixelsHalf ? 2 : kBufs; }
__host__ __device__ constexpr uint32_t ring_cols(int mode) {
  return mode == kModePixelsHalf ? 256u : kTmemCols;
}

// The pixel mode runs eight epilogue warps in two sets of four (one warp per
// TMEM lane quarter), the sets taking alternate tiles, so two tiles' 64
// roundings and packings a block are in flight at once: its per-tile
// epilogue is a latency chain (TMEM load, DC value, rounding, stores) that
// bounds it otherwise.  Its 512 threads get 128 registers each.
__host__ __device__ constexpr int epi_warps(int mode) { return mode == kModePixels ? 8 : 4; }
// threads that release an accumulator buffer (four warps, one per lane
// quarter, in every mode)
constexpr int kEpiReleaseThreads = 128;
__host__ __device__ constexpr int block_threads(int mode) { return 256 + 32 * epi_warps(mode); }

template <typename IoT, int S, int NS, bool kGroup, int kMode>
__global__ void __maxnreg__(kMode == kModePixelsHalf ? 80
                            : kMode == kModePixels ? 128
                            : sizeof(IoT) == 4 ? 152 : 168)
apply_group_kernel(const GroupItem *__restrict__ gitems, const __grid_constant__ GroupItem single,
                   int nitems, int64_t total_halves, int max_take, int interleaved,
                   uint32_t *__restrict__ err) {
  using L = Layout<IoT, S, NS, is_pixels(kMode) ? 0 : 2, ring_bufs(kMode)>;
  // the TMEM ring of this mode (these shadow the whole-SM constants)
  constexpr int kBufs = ring_bufs(kMode);
  constexpr int kDcRing = L::kDcRing;
  constexpr uint32_t kTmemCols = ring_cols(kMode);
  extern __shared__ uint8_t smem_raw[];
  uint8_t *base = reinterpret_cast<uint8_t *>(
      (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  uint8_t *s_in = base + L::kOffIn;
  uint8_t *s_out = base + L::kOffOut;
  uint8_t *s_slot = base + L::kOffSlot;
  float *s_dc = reinterpret_cast<float *>(base + L::kOffDc);
  uint64_t *bars = reinterpret_cast<uint64_t *>(base + L::kOffBar);
  uint64_t *full_in = bars;                    // [S]    TMA -> converter
  uint64_t *empty_in = bars + S;               // [S]    converter -> TMA
  uint64_t *a_full = bars + 2 * S;             // [4]    converter -> MMA
  uint64_t *mma_done = a_full + kBufs;         // [4]    MMA -> converter (A free), epilogue (D full)
  uint64_t *d_empty = mma_done + kBufs;        // [4]    epilogue -> MMA
  uint64_t *dc_full = d_empty + kBufs;         // [8]    converter -> epilogue (DC values)
  uint64_t *slot_full = dc_full + kDcRing;     // [NS]   loader -> all
  uint64_t *slot_empty = slot_full + NS;       // [NS]   all -> loader
  uint32_t *s_tmem = reinterpret_cast<uint32_t *>(base + L::kOffMisc);
  volatile int *s_abort = reinterpret_cast<volatile int *>(base + L::kOffMisc + 4);

  const GroupItem *items = kGroup ? gitems : &single;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

  if (tid == 0) {
    // host-direct input: one cp.async arrival per producer lane
    for (int s = 0; s < S; ++s) {
      mbar_init(&full_in[s], kMode == kModeHost ? 32 : 1);
      mbar_init(&empty_in[s], 128);
    }
    for (int b = 0; b < kBufs; ++b) {
      mbar_init(&a_full[b], 128); mbar_init(&mma_done[b], 1);
      mbar_init(&d_empty[b], kEpiReleaseThreads);
    }
    for (int r = 0; r < kDcRing; ++r) mbar_init(&dc_full[r], 128);
    for (int k = 0; k < NS; ++k) {   // released by the converter, the epilogue and the MMA
      mbar_init(&slot_full[k], 1);
      mbar_init(&slot_empty[k], 128 + 32 * epi_warps(kMode) + 1);
    }
    *s_abort = 0;
    mbar_fence_init();
  }
  if (warp == 2) { tmem_alloc(s_tmem, kTmemCols); tmem_relinquish(); }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *s_tmem;
  // A launch of this kernel that follows on the stream may be scheduled now
  // (it only does so when launched for programmatic stream serialisation).
  if (tid == 0) pdl_launch_dependents();

  TileWalk walk;
  walk.init(items, nitems, total_halves, max_take, interleaved != 0);
  Tile t;

  if (kMode == kModeHost && warp == 0) {
    // ---------------------------------------------------------- host producer
    // The tile's rows are contiguous: chunk c (16 bytes) of the tile is chunk
    // c % kCPR of row c / kCPR (kCPR = 16 for FP32 rows, 8 for int16), and
    // lane l copies chunks l, l + 32, ...  (a warp reads 512 contiguous bytes
    // per step).  Each chunk lands where the 128-byte-swizzled TMA box would
    // put it.
    constexpr int kCPR = Io<IoT>::kRowBytes / 16;
    int it = 0;
    while (walk.next(t)) {
      const int s = it % S;
      const uint32_t ph = (it / S) & 1;
      if (!warp_wait_bounded(&empty_in[s], ph ^ 1, s_abort, err, kRoleProducer | (it << 8))) break;
      const GroupItem &gi = items[t.item];
      const int64_t left = gi.nblocks - t.row0;
      const int valid = left < t.rows ? (int)left : t.rows;     // rows past the end: zeros
      const uint4 *src = reinterpret_cast<const uint4 *>(gi.hin) + (int64_t)t.row0 * kCPR;
      const uint32_t dst = smem_u32(s_in + s * L::kStageBytes);
      const int nchunks = t.rows * kCPR;
#pragma unroll 8
      for (int c = lane; c < nchunks; c += 32) {
        const int r = c / kCPR, u = c % kCPR;
        const uint32_t d = dst + (u >> 3) * L::kBoxBytes + r * 128 + (((u & 7) ^ (r & 7)) << 4);
        const bool ok = r < valid;
        cp_async_16(d, ok ? src + c : src, ok ? 16u : 0u);
      }
      cp_async_arrive(&full_in[s]);
      ++it;
    }
    cp_async_wait_all();
    if (lane == 0)
      for (int q = it > S ? it - S : 0; q < it; ++q)
        wait_drain(&full_in[q % S], (q / S) & 1, err, kRoleDrain);
  } else if (kMode != kModeHost && warp == 0 && lane == 0) {
    // ---------------------------------------------------------- producer
    int it = 0, issued = 0;
    while (walk.next(t)) {
      const int s = it % S;
      const uint32_t ph = (it / S) & 1;
      if (!wait_bounded(&empty_in[s], ph ^ 1, s_abort, err, kRoleProducer | (it << 8))) break;
      const GroupItem &gi = items[t.item];
      mbar_arrive_expect_tx(&full_in[s], t.rows * Io<IoT>::kRowBytes);
      uint8_t *dst = s_in + s * L::kStageBytes;
      if constexpr (kMode == kModePlanar) {
        // t.rows / 32 boxes of (256 floats, 8 rows): 32 blocks of one block
        // row each, shared [box][u][32 blocks][v]; the rows of a box are
        // 1 KB runs of the plane
        const int by = t.row0 / (int)gi.bw, bx0 = t.row0 % (int)gi.bw;
        for (int k = 0; k < t.rows / 32; ++k)
          tma_load_2d(&gi.tm_in, &full_in[s], dst + k * 8192, (bx0 + 32 * k) * 8, by * 8);
      } else {
        const void *map = t.rows == kTile ? (const void *)&gi.tm_in : (const void *)&gi.tm_in_half;
#pragma unroll
        for (int bx = 0; bx < Io<IoT>::kBoxesPerRow; ++bx)
          tma_load_2d(map, &full_in[s], dst + bx * L::kBoxBytes, bx * Io<IoT>::kBoxCols, t.row0);
      }
      ++issued;
      ++it;
    }
    for (int q = issued > S ? issued - S : 0; q < issued; ++q)
      wait_drain(&full_in[q % S], (q / S) & 1, err, kRoleDrain);
  } else if (warp == 3 && lane == 0) {
    // ---------------------------------------------------------- slot loader
    int last = -1;
    while (walk.next(t)) {
      if (!t.seg_first) continue;
      const int k = t.seg % NS;
      const int use = t.seg / NS;                 // how many times slot k was filled before
      if (use >= 1 &&
          !wait_bounded(&slot_empty[k], (use - 1) & 1, s_abort, err, kRoleLoader))
        break;
      const GroupItem &gi = items[t.item];
      uint8_t *slot = s_slot + k * kSlotBytes;
      const uint32_t bytes = kSlotPieces + kSlotMdc + (Io<IoT>::kBoxesPerRow == 1 ? 2 * kSlotQ : 0);
      mbar_arrive_expect_tx(&slot_full[k], bytes);
      bulk_load(slot, gi.pieces, kSlotPieces, &slot_full[k]);
      bulk_load(slot + kSlotPieces, gi.mdc, kSlotMdc, &slot_full[k]);
      if (Io<IoT>::kBoxesPerRow == 1) {
        bulk_load(slot + kSlotPieces + kSlotMdc, gi.qin, kSlotQ, &slot_full[k]);
        bulk_load(slot + kSlotPieces + kSlotMdc + kSlotQ, gi.qout, kSlotQ, &slot_full[k]);
      }
      last = t.seg;
    }
    for (int sg = last - NS + 1 > 0 ? last - NS + 1 : 0; sg <= last; ++sg)
      wait_drain(&slot_full[sg % NS], (sg / NS) & 1, err, kRoleDrain);
  } else if (warp == 1 && lane == 0) {
    // ---------------------------------------------------------- MMA issuer
    // D (64 columns) = A_hi M_lo^T + A_lo M_hi^T + A_hi M_hi^T, 12 MMAs of
    // 128 x 64 x 16; the three products share one FP32 accumulator.
    constexpr uint32_t kIdesc = idesc_f16(128, kN2, false);
    int it = 0, last = -1;
    while (walk.next(t)) {
      const int b = it % kBufs, k = t.seg % NS;
      const uint32_t ph = (it / kBufs) & 1;
      if (t.seg_first &&
          !wait_bounded(&slot_full[k], (t.seg / NS) & 1, s_abort, err, kRoleMma | (it << 8)))
        break;
      if (!wait_bounded(&a_full[b], ph, s_abort, err, kRoleMma | (it << 8))) break;
      if (!wait_bounded(&d_empty[b], ph ^ 1, s_abort, err, kRoleMma | (it << 8))) break;
      tc_fence_after();
      const uint64_t b_hi = desc_sw128(smem_u32(s_slot + k * kSlotBytes));
      const uint64_t b_lo = desc_sw128(smem_u32(s_slot + k * kSlotBytes + kN2 * 128));
      const uint32_t t_a = tmem + b * 128, t_d = t_a + 64;
      // the two small correction products first, so they accumulate at
      // their own magnitude before the main product is added
#pragma unroll
      for (int kk = 0; kk < kN2 / 16; ++kk)
        mma_f16_ts(t_d, t_a + 8 * kk, b_lo + 2 * kk, kIdesc, kk > 0);
#pragma unroll
      for (int kk = 0; kk < kN2 / 16; ++kk)
        mma_f16_ts(t_d, t_a + 32 + 8 * kk, b_hi + 2 * kk, kIdesc, 1);
#pragma unroll
      for (int kk = 0; kk < kN2 / 16; ++kk)
        mma_f16_ts(t_d, t_a + 8 * kk, b_hi + 2 * kk, kIdesc, 1);
      tc_commit(&mma_done[b]);
      if (t.seg_last) tc_commit(&slot_empty[k]);   // slot free once these MMAs finish
      last = it;
      ++it;
    }
    if (last >= 0) wait_drain(&mma_done[last % kBufs], (last / kBufs) & 1, err, kRoleDrain);
  } else if (warp >= 4 && warp < 8) {
    // ---------------------------------------------------------- converter
    const int row = tid - 128;
    const uint32_t lane_base = (uint32_t)((warp & 3) * 32) << 16;
    int it = 0;
    while (walk.next(t)) {
      const int s = it % S, b = it % kBufs, r = it % kDcRing, k = t.seg % NS;
      const uint32_t ps = (it / S) & 1, pb = (it / kBufs) & 1;
      // every role that releases a slot first waits for it to be filled, so
      // its release can never count toward the slot's previous use
      if (t.seg_first &&
          !warp_wait_bounded(&slot_full[k], (t.seg / NS) & 1, s_abort, err, kRoleConv | (it << 8)))
        break;
      if (!warp_wait_bounded(&full_in[s], ps, s_abort, err, kRoleConv | (it << 8))) break;
      if constexpr (kMode == kModePixelsHalf) {
        // the same split, 32 inputs at a time (80 registers a thread): box
        // row 0 is split and stored once A buffer b is free, then box row 1
        // (the stage is released after it)
        const uint8_t *st = s_in + s * L::kStageBytes + row * 128;
        const uint32_t t_a = tmem + lane_base + b * 128;
        bool ok = true;
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          float v[32];
#pragma unroll
          for (int u = 0; u < 8; ++u) {
            const float4 q =
                *reinterpret_cast<const float4 *>(st + h * L::kBoxBytes + ((u ^ (row & 7)) << 4));
            v[4 * u] = q.x; v[4 * u + 1] = q.y; v[4 * u + 2] = q.z; v[4 * u + 3] = q.w;
          }
          if (h == 1) mbar_arrive(&empty_in[s]);
          if (row >= t.rows) {
#pragma unroll
            for (int c = 0; c < 32; ++c) v[c] = 0.f;   // rows past the tile: not stored
          }
          if (h == 0) {
            const float x0 = v[0];
            v[0] = 0.f;
            // A buffer b is free once the MMAs of tile it - kBufs completed
            if (!warp_wait_bounded(&mma_done[b], pb ^ 1, s_abort, err, kRoleConv | (it << 8))) {
              ok = false;
              break;
            }
            s_dc[r * kTile + row] = x0;
            mbar_arrive(&dc_full[r]);
            tc_fence_after();
          }
          uint32_t hi[16], lo[16];
#pragma unroll
          for (int c = 0; c < 16; ++c) {
            const __half2 h2 = __floats2half2_rn(v[2 * c], v[2 * c + 1]);
            const float2 hf = __half22float2(h2);
            const __half2 l2 = __floats2half2_rn(v[2 * c] - hf.x, v[2 * c + 1] - hf.y);
            hi[c] = *reinterpret_cast<const uint32_t *>(&h2);
            lo[c] = *reinterpret_cast<const uint32_t *>(&l2);
          }
          tmem_st16(t_a + 16 * h, hi);
          tmem_st16(t_a + 32 + 16 * h, lo);
        }
        if (!ok) break;
        tmem_st_wait();
        tc_fence_before();
        mbar_arrive(&a_full[b]);
        if (t.seg_last) mbar_arrive(&slot_empty[k]);
        ++it;
        continue;
      }
      float v[64];
      const uint8_t *st = s_in + s * L::kStageBytes + row * 128;
      if constexpr (kMode == kModePlanar) {
        // shared [box][u][32 blocks][v]: this block's row u is 32 bytes at
        // (row / 32) 8192 + u 1024 + (row % 32) 32.  Lanes 4 apart hit the
        // same banks; taking the two 16-byte halves in an order that flips
        // with bit 2 of the row removes the conflicts.
        const uint8_t *sp = s_in + s * L::kStageBytes + (row >> 5) * 8192 + (row & 31) * 32;
        const int sw = (row >> 2) & 1;
#pragma unroll
        for (int u = 0; u < 8; ++u) {
          const float4 *q = reinterpret_cast<const float4 *>(sp + u * 1024);
          const float4 f = q[sw], g = q[sw ^ 1];
          const float4 a = sw ? g : f, b = sw ? f : g;
          v[8 * u] = a.x; v[8 * u + 1] = a.y; v[8 * u + 2] = a.z; v[8 * u + 3] = a.w;
          v[8 * u + 4] = b.x; v[8 * u + 5] = b.y; v[8 * u + 6] = b.z; v[8 * u + 7] = b.w;
        }
      } else if constexpr (Io<IoT>::kBoxesPerRow == 2) {
#pragma unroll
        for (int u = 0; u < 16; ++u) {
          const float4 q = *reinterpret_cast<const float4 *>(
              st + (u >> 3) * L::kBoxBytes + (((u & 7) ^ (row & 7)) << 4));
          v[4 * u] = q.x; v[4 * u + 1] = q.y; v[4 * u + 2] = q.z; v[4 * u + 3] = q.w;
        }
      } else {
        // quantised input: x = Q * q_in (exact in FP32)
        const uint16_t *qin = reinterpret_cast<const uint16_t *>(
            s_slot + k * kSlotBytes + kSlotPieces + kSlotMdc);
#pragma unroll
        for (int u = 0; u < 8; ++u) {
          const uint4 q = *reinterpret_cast<const uint4 *>(st + (((u & 7) ^ (row & 7)) << 4));
          const uint4 qq = *reinterpret_cast<const uint4 *>(qin + 8 * u);
          const uint32_t w[4] = {q.x, q.y, q.z, q.w};
          const uint32_t m[4] = {qq.x, qq.y, qq.z, qq.w};
#pragma unroll
          for (int e = 0; e < 4; ++e) {
            v[8 * u + 2 * e] = (float)(int16_t)(w[e] & 0xffffu) * (float)(m[e] & 0xffffu);
            v[8 * u + 2 * e + 1] = (float)(int16_t)(w[e] >> 16) * (float)(m[e] >> 16);
          }
        }
      }
      mbar_arrive(&empty_in[s]);
      if (row >= t.rows) {
#pragma unroll
        for (int c = 0; c < 64; ++c) v[c] = 0.f;     // rows past the tile: not stored
      }
      const float x0 = v[0];
      v[0] = 0.f;
      // A buffer b is free once the MMAs of tile it - kBufs completed
      if (!warp_wait_bounded(&mma_done[b], pb ^ 1, s_abort, err, kRoleConv | (it << 8))) break;
      s_dc[r * kTile + row] = x0;
      mbar_arrive(&dc_full[r]);
      tc_fence_after();
      const uint32_t t_a = tmem + lane_base + b * 128;
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
      if (t.seg_last) mbar_arrive(&slot_empty[k]);
      ++it;
    }
  } else if (warp >= 8) {
    // ---------------------------------------------------------- epilogue
    const int wr = warp & 3, row = wr * 32 + lane, r32 = lane;
    const uint32_t lane_base = (uint32_t)(wr * 32) << 16;
    // Under programmatic dependent launch the loads above may run while the
    // previous kernel on the stream finishes; no output is written before
    // that kernel has completed (it may still read the output buffer).
    if (lane == 0) pdl_wait();
    __syncwarp();
    int it = 0;
    while (walk.next(t)) {
      const int b = it % kBufs, o = it & 1, r = it % kDcRing, k = t.seg % NS;
      const uint32_t pb = (it / kBufs) & 1, pr = (it / kDcRing) & 1;
      if (t.seg_first &&
          !warp_wait_bounded(&slot_full[k], (t.seg / NS) & 1, s_abort, err, kRoleEpi | (it << 8)))
        break;
      if constexpr (kMode == kModePixelsHalf) {
        // warp 8 + wr: TMEM lanes 32 wr.. (its blocks), every tile, the 64
        // pixels of a block in two halves of 32 (80 registers a thread)
        if (!warp_wait_bounded(&mma_done[b], pb, s_abort, err, kRoleEpi | (it << 8))) break;
        tc_fence_after();
        // the DC value is read before D[b] is released
        if (!warp_wait_bounded(&dc_full[r], pr, s_abort, err, kRoleEpi | (it << 8))) break;
        const float x0 = s_dc[r * kTile + row];
        const GroupItem &gi = items[t.item];
        const float out_scale = gi.out_scale;
        const int bk = t.row0 + row, bw = (int)gi.bw;
        const bool live = row < t.rows && bk < gi.nblocks;
        const int by = bk / bw, bx = bk - by * bw;
#pragma unroll
        for (int hc = 0; hc < 2; ++hc) {   // pixel rows 4 hc .. 4 hc + 3
          uint32_t d[32];
          tmem_ld32(tmem + lane_base + b * 128 + 64 + 32 * hc, d);
          if (hc == 1) {
            tc_fence_before();
            mbar_arrive(&d_empty[b]);
          }
          const float4 *mdc4 =
              reinterpret_cast<const float4 *>(s_slot + k * kSlotBytes + kSlotPieces) + 8 * hc;
          float px[32];
#pragma unroll
          for (int u = 0; u < 8; ++u) {
            const float4 md = mdc4[u];
            px[4 * u] = fmaf(__uint_as_float(d[4 * u]), out_scale, md.x * x0);
            px[4 * u + 1] = fmaf(__uint_as_float(d[4 * u + 1]), out_scale, md.y * x0);
            px[4 * u + 2] = fmaf(__uint_as_float(d[4 * u + 2]), out_scale, md.z * x0);
            px[4 * u + 3] = fmaf(__uint_as_float(d[4 * u + 3]), out_scale, md.w * x0);
          }
          if (live) {
            uint8_t *dst = gi.img + ((int64_t)by * 8 + 4 * hc) * gi.pitch + (int64_t)bx * 8;
#pragma unroll
            for (int i = 0; i < 4; ++i) {
              uint32_t w[2];
#pragma unroll
              for (int h = 0; h < 2; ++h) {
                const float *a = px + 8 * i + 4 * h;
                w[h] = __byte_perm(
                    __byte_perm(pixel_u8_low_byte(a[0]), pixel_u8_low_byte(a[1]), 0x0040),
                    __byte_perm(pixel_u8_low_byte(a[2]), pixel_u8_low_byte(a[3]), 0x0040), 0x5410);
              }
              *reinterpret_cast<uint2 *>(dst + i * gi.pitch) = make_uint2(w[0], w[1]);
            }
          }
        }
        if (t.seg_last) mbar_arrive(&slot_empty[k]);   // done with this slot's G[:,0]
        ++it;
        continue;
      }
      if constexpr (kMode == kModePixels) {
        // warp 8 + 4 set + wr: TMEM lanes 32 wr.. (its blocks), every output
        // column, tiles it with it % 2 == set (TMEM buffers b of that parity)
        const int set = (warp - 8) >> 2;
        if ((it & 1) != set) {
          if (t.seg_last) mbar_arrive(&slot_empty[k]);   // the other set's tile
          ++it;
          continue;
        }
        if (!warp_wait_bounded(&mma_done[b], pb, s_abort, err, kRoleEpi | (it << 8))) break;
        tc_fence_after();
        uint32_t d[2][32];
        tmem_ld32x2(tmem + lane_base + b * 128 + 64, tmem + lane_base + b * 128 + 96, d[0], d[1]);
        // the DC value is read before D[b] is released (see below)
        if (!warp_wait_bounded(&dc_full[r], pr, s_abort, err, kRoleEpi | (it << 8))) break;
        const float x0 = s_dc[r * kTile + row];
        tc_fence_before();
        mbar_arrive(&d_empty[b]);
        const GroupItem &gi = items[t.item];
        const float out_scale = gi.out_scale;
        // block bk of the item covers image rows 8 (bk / bw) + 0..7 and
        // columns 8 (bk % bw) + 0..7; its pixel (i, j) is output i * 8 + j.
        // The lanes of a warp hold consecutive blocks, so each row's 8-byte
        // stores of a warp are contiguous.
        // 32-bit block coordinates: an item has fewer than 2^31 blocks
        const int bk = t.row0 + row, bw = (int)gi.bw;
        const bool live = row < t.rows && bk < gi.nblocks;
        const int by = bk / bw, bx = bk - by * bw;
#pragma unroll
        for (int hc = 0; hc < 2; ++hc) {   // pixel rows 4 hc .. 4 hc + 3
          const float4 *mdc4 =
              reinterpret_cast<const float4 *>(s_slot + k * kSlotBytes + kSlotPieces) + 8 * hc;
          float px[32];
#pragma unroll
          for (int u = 0; u < 8; ++u) {
            const float4 md = mdc4[u];
            px[4 * u] = fmaf(__uint_as_float(d[hc][4 * u]), out_scale, md.x * x0);
            px[4 * u + 1] = fmaf(__uint_as_float(d[hc][4 * u + 1]), out_scale, md.y * x0);
            px[4 * u + 2] = fmaf(__uint_as_float(d[hc][4 * u + 2]), out_scale, md.z * x0);
            px[4 * u + 3] = fmaf(__uint_as_float(d[hc][4 * u + 3]), out_scale, md.w * x0);
          }
          if (live) {
            uint8_t *dst = gi.img + ((int64_t)by * 8 + 4 * hc) * gi.pitch + (int64_t)bx * 8;
#pragma unroll
            for (int i = 0; i < 4; ++i) {
              uint32_t w[2];
#pragma unroll
              for (int h = 0; h < 2; ++h) {
                const float *a = px + 8 * i + 4 * h;
                // bytes b0..b3 into one word (PRMT: low bytes of four words)
                w[h] = __byte_perm(
                    __byte_perm(pixel_u8_low_byte(a[0]), pixel_u8_low_byte(a[1]), 0x0040),
                    __byte_perm(pixel_u8_low_byte(a[2]), pixel_u8_low_byte(a[3]), 0x0040), 0x5410);
              }
              *reinterpret_cast<uint2 *>(dst + i * gi.pitch) = make_uint2(w[0], w[1]);
            }
          }
        }
        if (t.seg_last) mbar_arrive(&slot_empty[k]);   // done with this slot's G[:,0]
        ++it;
        continue;
      }
      if (!warp_wait_bounded(&mma_done[b], pb, s_abort, err, kRoleEpi | (it << 8))) break;
      tc_fence_after();
      float acc[64];
      {
        uint32_t d0[32], d1[32];
        tmem_ld32x2(tmem + lane_base + b * 128 + 64, tmem + lane_base + b * 128 + 96, d0, d1);
#pragma unroll
        for (int c = 0; c < 32; ++c) {
          acc[c] = __uint_as_float(d0[c]);
          acc[32 + c] = __uint_as_float(d1[c]);
        }
      }
      // the DC value is read before D[b] is released: the converter rewrites
      // this ring slot for tile it + 8 only after the MMAs of tile it + 4,
      // which wait for that release
      if (!warp_wait_bounded(&dc_full[r], pr, s_abort, err, kRoleEpi | (it << 8))) break;
      const float x0 = s_dc[r * kTile + row];
      tc_fence_before();
      mbar_arrive(&d_empty[b]);                      // D[b] may be overwritten now
      const GroupItem &gi = items[t.item];
      const float out_scale = gi.out_scale;
      const uint8_t *slot = s_slot + k * kSlotBytes;
      const float4 *mdc4 = reinterpret_cast<const float4 *>(slot + kSlotPieces);
#pragma unroll
      for (int u = 0; u < 16; ++u) {
        const float4 md = mdc4[u];
        acc[4 * u] = fmaf(acc[4 * u], out_scale, md.x * x0);
        acc[4 * u + 1] = fmaf(acc[4 * u + 1], out_scale, md.y * x0);
        acc[4 * u + 2] = fmaf(acc[4 * u + 2], out_scale, md.z * x0);
        acc[4 * u + 3] = fmaf(acc[4 * u + 3], out_scale, md.w * x0);
      }
      const bool store = wr * 32 < t.rows;
      uint8_t *slab = s_out + o * L::kStageBytes + wr * L::kSlabBytes;
      // slab o is free: the TMA store of tile it - 2 has read it (host mode:
      // the lanes' copies of tile it - 2 came before the previous __syncwarp)
      if (kMode != kModeHost && lane == 0) bulk_wait_read<1>();
      __syncwarp();
      if constexpr (kMode == kModePlanar) {
        // shared [u][32][v] for this warp's 32 blocks (halves in the
        // converter's bank-friendly order)
        const int sw = (r32 >> 2) & 1;
#pragma unroll
        for (int u = 0; u < 8; ++u) {
          float4 *q = reinterpret_cast<float4 *>(slab + (u * 32 + r32) * 32);
          const float4 a = make_float4(acc[8 * u], acc[8 * u + 1], acc[8 * u + 2], acc[8 * u + 3]);
          const float4 b =
              make_float4(acc[8 * u + 4], acc[8 * u + 5], acc[8 * u + 6], acc[8 * u + 7]);
          q[sw] = sw ? b : a;
          q[sw ^ 1] = sw ? a : b;
        }
      } else if constexpr (Io<IoT>::kBoxesPerRow == 2) {
#pragma unroll
        for (int u = 0; u < 16; ++u)
          *reinterpret_cast<float4 *>(slab + (u >> 3) * L::kSlabBoxBytes + r32 * 128 +
                                      (((u & 7) ^ (r32 & 7)) << 4)) =
              make_float4(acc[4 * u], acc[4 * u + 1], acc[4 * u + 2], acc[4 * u + 3]);
      } else {
        // requantise: round_half_away(y / q_out), saturated to int16
        const uint16_t *qout = reinterpret_cast<const uint16_t *>(
            slot + kSlotPieces + kSlotMdc + kSlotQ);
#pragma unroll
        for (int u = 0; u < 8; ++u) {
          const uint4 qq = *reinterpret_cast<const uint4 *>(qout + 8 * u);
          const uint32_t m[4] = {qq.x, qq.y, qq.z, qq.w};
          uint32_t w[4];
#pragma unroll
          for (int e = 0; e < 4; ++e) {
            float a = roundf(__fdiv_rn(acc[8 * u + 2 * e], (float)(m[e] & 0xffffu)));
            float c = roundf(__fdiv_rn(acc[8 * u + 2 * e + 1], (float)(m[e] >> 16)));
            a = fminf(fmaxf(a, -32768.f), 32767.f);
            c = fminf(fmaxf(c, -32768.f), 32767.f);
            w[e] = ((uint32_t)(uint16_t)(int16_t)a) | ((uint32_t)(uint16_t)(int16_t)c << 16);
          }
          *reinterpret_cast<uint4 *>(slab + r32 * 128 + ((u ^ (r32 & 7)) << 4)) =
              make_uint4(w[0], w[1], w[2], w[3]);
        }
      }
      fence_async_smem();
      __syncwarp();
      if (t.seg_last) mbar_arrive(&slot_empty[k]);   // done with this slot's M[:,0], q_out
      if constexpr (kMode == kModeHost) {
        // copy the staged rows to host memory: chunk c = lane + 32 i is chunk
        // c % kCPR of row c / kCPR, so a warp writes 512 contiguous bytes per
        // step
        constexpr int kCPR = Io<IoT>::kRowBytes / 16;
        const int64_t y0 = (int64_t)t.row0 + wr * 32;
        const int64_t left = gi.nblocks - y0;
        const int lim = t.rows - wr * 32 < 32 ? t.rows - wr * 32 : 32;
        const int nrows = (int)(left < lim ? left : lim);     // <= 0: nothing to store
        uint4 *dst = reinterpret_cast<uint4 *>(gi.hout) + y0 * kCPR;
#pragma unroll
        for (int i = 0; i < kCPR; ++i) {
          const int c = lane + 32 * i, r = c / kCPR, u = c % kCPR;
          if (r < nrows)
            __stcs(dst + c, *reinterpret_cast<const uint4 *>(
                                slab + (u >> 3) * L::kSlabBoxBytes + r * 128 + (((u & 7) ^ (r & 7)) << 4)));
        }
        ++it;
        continue;
      }
      if (lane == 0) {
        if (store) {
          const int y0 = t.row0 + wr * 32;
          if constexpr (kMode == kModePlanar) {
            // one (256 floats, 8 rows) box: this warp's 32 blocks; a box
            // past the image's right edge is clipped, one wholly past it
            // is skipped
            const int bx = y0 % (int)gi.bw, by = y0 / (int)gi.bw;
            if (bx < gi.pitch) tma_store_2d(&gi.tm_out, slab, bx * 8, by * 8);
          } else {
#pragma unroll
            for (int bx = 0; bx < Io<IoT>::kBoxesPerRow; ++bx)
              tma_store_2d(&gi.tm_out, slab + bx * L::kSlabBoxBytes, bx * Io<IoT>::kBoxCols, y0);
          }
        }
        bulk_commit();
      }
      ++it;
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

// [nblocks][64] rows (FP32 or int16) as a 2-D tensor; boxes of 128 bytes
// (32 floats or 64 int16) x box_rows rows, 128-byte swizzle.
cudaError_t make_map(CUtensorMap *m, const void *ptr, int64_t nblocks, bool i16, int box_rows) {
  EncodeTiledFn enc = encode_fn();
  if (enc == nullptr) return cudaErrorNotSupported;
  const int esz = i16 ? 2 : 4;
  cuuint64_t dims[2] = {(cuuint64_t)kN2, (cuuint64_t)nblocks};
  cuuint64_t strides[1] = {(cuuint64_t)kN2 * esz};
  cuuint32_t box[2] = {(cuuint32_t)(128 / esz), (cuuint32_t)box_rows};
  cuuint32_t es[2] = {1, 1};
  CUresult r = enc(m, i16 ? CU_TENSOR_MAP_DATA_TYPE_UINT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2,
                   const_cast<void *>(ptr), dims, strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
                   CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                   CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

template <typename IoT, int S, int NS, bool kGroup, int kMode = kModeBlocks>
cudaError_t launch_cfg(const GroupItem *d_items, const GroupItem &single, int nitems,
                       int64_t total_halves, int grid, int max_take, int interleaved,
                       uint32_t *err, cudaStream_t s, bool pdl) {
  auto kern = apply_group_kernel<IoT, S, NS, kGroup, kMode>;
  constexpr int smem = Layout<IoT, S, NS, is_pixels(kMode) ? 0 : 2, ring_bufs(kMode)>::kSmem;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e != cudaSuccess) return e;
  if (kMode == kModePixelsHalf) {   // room for two CTAs an SM
    e = cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
    if (e != cudaSuccess) return e;
  }
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(block_threads(kMode));
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  if (pdl) {
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
  }
  e = cudaLaunchKernelEx(&cfg, kern, d_items, single, nitems, total_halves, max_take, interleaved,
                         err);
  if (e != cudaSuccess) return e;
  return cudaGetLastError();
}

}  // namespace

cudaError_t fill_group_item(GroupItem *gi, const dctf_operator *op, const void *in, void *out,
                            int64_t nblocks, bool i16, const uint16_t *qin,
                            const uint16_t *qout) {
  memset(gi, 0, sizeof *gi);
  cudaError_t e = make_map(&gi->tm_in, in, nblocks, i16, kTile);
  if (e == cudaSuccess) e = make_map(&gi->tm_in_half, in, nblocks, i16, kHalf);
  if (e == cudaSuccess) e = make_map(&gi->tm_out, out, nblocks, i16, 32);
  if (e != cudaSuccess) return e;
  gi->pieces = op->d_f16;
  gi->mdc = op->d_Mdc;
  gi->qin = qin;
  gi->qout = qout;
  gi->out_scale = ldexpf(1.0f, -op->f16_scale_exp);
  gi->nblocks = nblocks;
  return cudaSuccess;
}

cudaError_t fill_group_item_host(GroupItem *gi, const dctf_operator *op, const void *hin,
                                 void *hout, int64_t nblocks, const uint16_t *qin,
                                 const uint16_t *qout) {
  memset(gi, 0, sizeof *gi);
  if (((reinterpret_cast<uintptr_t>(hin) | reinterpret_cast<uintptr_t>(hout)) & 15) != 0)
    return cudaErrorInvalidValue;
  gi->pieces = op->d_f16;
  gi->mdc = op->d_Mdc;
  gi->qin = qin;
  gi->qout = qout;
  gi->out_scale = ldexpf(1.0f, -op->f16_scale_exp);
  gi->nblocks = nblocks;
  gi->hin = hin;
  gi->hout = hout;
  return cudaSuccess;
}

cudaError_t launch_apply_pixels(const GroupItem &single, int64_t total_halves, int grid,
                                uint32_t *err, cudaStream_t s, bool pdl) {
  if (total_halves <= 0) return cudaSuccess;
  int64_t g = grid > 0 ? grid : 0;
  if (g > total_halves) g = total_halves;
  if (g < 1) g = 1;
  // two half-SM CTAs an SM, two input stages each, interleaved schedule
  // (giving the two CTAs of an SM unequal shares, so that their drains fall
  // apart, measured slower: 16.1-19.0 us against 15.9).  A small image
  // launched for programmatic serialisation takes one CTA an SM instead:
  // the next launch's CTAs then start beside this one's and load while it
  // runs, which saves more than one CTA's lower rate costs (back to back,
  // 2048^2: 5.7 us against 6.8; 4096^2: 17.1 against 15.8).
  constexpr int64_t kOnePerSmHalves = 2048;   // 131,072 blocks
  if (!pdl || total_halves > kOnePerSmHalves) g = 2 * g > total_halves ? total_halves : 2 * g;
  return launch_cfg<float, 2, 1, false, kModePixelsHalf>(nullptr, single, 1, total_halves, (int)g,
                                                         2, 1, err, s, pdl);
}

// Image-plane coefficients: the 2-D view of an FP32 array of `height` rows
// of `pitch` floats (`width` of them used); boxes of 256 floats x 8 rows,
// i.e. 32 blocks of one block row, each box row a 1 KB run of the plane.
static cudaError_t make_planar_map(CUtensorMap *m, const void *ptr, int height, int width,
                                   int64_t pitch) {
  EncodeTiledFn enc = encode_fn();
  if (enc == nullptr) return cudaErrorNotSupported;
  cuuint64_t dims[2] = {(cuuint64_t)width, (cuuint64_t)height};
  cuuint64_t strides[1] = {(cuuint64_t)pitch * 4};
  cuuint32_t box[2] = {256, 8};
  cuuint32_t es[2] = {1, 1};
  CUresult r = enc(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<void *>(ptr), dims, strides,
                   box, es, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                   CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

cudaError_t launch_apply_planar(const dctf_operator *op, const float *in, int height, int width,
                                int64_t in_pitch, float *out, int64_t out_pitch, uint32_t *err,
                                cudaStream_t s, bool pdl) {
  GroupItem gi;
  memset(&gi, 0, sizeof gi);
  cudaError_t e = make_planar_map(&gi.tm_in, in, height, width, in_pitch);
  if (e == cudaSuccess) e = make_planar_map(&gi.tm_out, out, height, width, out_pitch);
  if (e != cudaSuccess) return e;
  const int64_t bw_pad = (width / 8 + kTile - 1) / kTile * kTile;
  gi.pieces = op->d_f16;
  gi.mdc = op->d_Mdc;
  gi.out_scale = ldexpf(1.0f, -op->f16_scale_exp);
  gi.bw = bw_pad;
  gi.pitch = width / 8;                              // the plane's width in blocks
  gi.nblocks = (int64_t)(height / 8) * bw_pad;      // tile walk over padded block rows
  const int64_t total_halves = gi.nblocks / kHalf;
  int64_t g = sm_count(op->device);
  if (g > total_halves) g = total_halves;
  if (g < 1) g = 1;
  return launch_cfg<float, 4, 1, false, kModePlanar>(nullptr, gi, 1, total_halves, (int)g, 2, 1,
                                                     err, s, pdl);
}

// Input stages and operator slots of the grouped launches, per variant
// (the autotuner's third axis).  Shared memory bounds the product: an FP32
// stage is 32 KB and a slot 17 KB, so one slot leaves room for a stage more.
int group_variant_stages(int kind, int variant) {
  static const int kStagesOf[3][kGroupVariants] = {{3, 2, 4}, {4, 6, 8}, {4, 5, 6}};
  return kStagesOf[kind][variant];
}
int group_variant_slots(int, int variant) { return variant == 2 ? 1 : 2; }

cudaError_t launch_apply_group_pixels(const GroupItem *d_items, int nitems, int64_t total_halves,
                                      int grid, int max_take, uint32_t *err, cudaStream_t s,
                                      int variant, bool pdl) {
  if (total_halves <= 0) return cudaSuccess;
  int64_t g = grid > 0 ? grid : 0;
  if (g > total_halves) g = total_halves;
  if (g < 1) g = 1;
  static const GroupItem kEmpty = {};
  const int take = max_take == 1 ? 1 : 2;
  switch (variant) {
    case 1:
      return launch_cfg<float, 5, 2, true, kModePixels>(d_items, kEmpty, nitems, total_halves,
                                                        (int)g, take, 0, err, s, pdl);
    case 2:
      return launch_cfg<float, 6, 1, true, kModePixels>(d_items, kEmpty, nitems, total_halves,
                                                        (int)g, take, 0, err, s, pdl);
    default:
      return launch_cfg<float, 4, 2, true, kModePixels>(d_items, kEmpty, nitems, total_halves,
                                                        (int)g, take, 0, err, s, pdl);
  }
}

cudaError_t launch_apply_host_direct(const GroupItem &single, int64_t total_halves, int grid,
                                     uint32_t *err, cudaStream_t s) {
  if (total_halves <= 0) return cudaSuccess;
  int64_t g = grid > 0 ? grid : 0;
  if (g > total_halves) g = total_halves;
  if (g < 1) g = 1;
  // 64-block tiles dealt round-robin: the CTAs work on adjacent tiles, so the
  // host memory in flight stays one compact window
  return launch_cfg<float, 4, 1, false, kModeHost>(nullptr, single, 1, total_halves, (int)g, 1, 1,
                                                   err, s, false);
}

cudaError_t launch_apply_group_host(const GroupItem *d_items, int nitems, int64_t total_halves,
                                    int grid, uint32_t *err, cudaStream_t s) {
  if (total_halves <= 0) return cudaSuccess;
  int64_t g = grid > 0 ? grid : 0;
  if (g > total_halves) g = total_halves;
  if (g < 1) g = 1;
  static const GroupItem kEmpty = {};
  // 128-row tiles: each stage holds a whole tile, so twice the host reads
  // are in flight per CTA as with 64-row tiles (serving stream: 42k req/s
  // sustained against 23-25k with 64-row tiles)
  return launch_cfg<int16_t, 4, 2, true, kModeHost>(d_items, kEmpty, nitems, total_halves, (int)g, 2,
                                                    0, err, s, false);
}

cudaError_t launch_apply_group(const GroupItem *d_items, const GroupItem *single, int nitems,
                               int64_t total_halves, bool i16, int grid, int max_take,
                               uint32_t *err, cudaStream_t s, bool pdl, int variant) {
  if (total_halves <= 0) return cudaSuccess;
  int64_t g = grid > 0 ? grid : 0;
  if (g > total_halves) g = total_halves;
  if (g < 1) g = 1;
  static const GroupItem kEmpty = {};
  const int take = max_take == 1 ? 1 : 2;
  if (single != nullptr) {   // one item: interleaved schedule, one operator slot, 4 stages
    return i16 ? launch_cfg<int16_t, 4, 1, false>(nullptr, *single, 1, total_halves, (int)g, take,
                                                 1, err, s, pdl)
               : launch_cfg<float, 4, 1, false>(nullptr, *single, 1, total_halves, (int)g, take, 1,
                                               err, s, pdl);
  }
  if (i16) {
    switch (variant) {
      case 1:
        return launch_cfg<int16_t, 6, 2, true>(d_items, kEmpty, nitems, total_halves, (int)g, take,
                                               0, err, s, pdl);
      case 2:
        return launch_cfg<int16_t, 8, 1, true>(d_items, kEmpty, nitems, total_halves, (int)g, take,
                                               0, err, s, pdl);
      default:
        return launch_cfg<int16_t, 4, 2, true>(d_items, kEmpty, nitems, total_halves, (int)g, take,
                                               0, err, s, pdl);
    }
  }
  switch (variant) {
    case 1:
      return launch_cfg<float, 2, 2, true>(d_items, kEmpty, nitems, total_halves, (int)g, take, 0,
                                           err, s, pdl);
    case 2:
      return launch_cfg<float, 4, 1, true>(d_items, kEmpty, nitems, total_halves, (int)g, take, 0,
                                           err, s, pdl);
    default:
      return launch_cfg<float, 3, 2, true>(d_items, kEmpty, nitems, total_halves, (int)g, take, 0,
                                           err, s, pdl);
  }
}

}  // namespace dctf

// Paper-form apply on tensor cores: the operator as a sum of Kronecker
// products, M = sum_t A_t kron B_t, applied to each 16x16 block as the
// sandwich products Y = sum_t A_t X B_t^T (Sec. II.B Eq. 11-12, Sec. II.C
// Eq. 20), with the F16X3 split and FP32 accumulation in TMEM.
//
// Per block the sandwich form costs r * 2 * 2 N^3 flops against 2 N^4 for the
// dense product (r = rank of the mask), 8x fewer for a separable mask at
// N = 16.  On tensor cores its two halves are small GEMMs over a unit of 8
// blocks (128 MMA rows):
//
//  pass 1  Z_t = X B_t^T for every term: rows (block b, row k of X), K = the
//          16 columns of X, N = (term, j).  The B operand holds the hi pieces
//          of B_t 2^sB, then the lo pieces, so
//            D1 = x_hi B_lo^T + x_lo B_hi^T + x_hi B_hi^T
//          (corrections first, while the sum is small) is three MMAs of
//          N = 16 ng per group of up to four terms.
//  transpose  pass 2 contracts over k, which pass 1 leaves in TMEM lanes.
//          A transposer thread (lane (b, k)) reads its row of Z_t, puts it
//          through a padded 16 x 20 shared-memory tile of its block, reads
//          back column j = its row index (now lane (b, j)), re-splits it
//          into FP16 hi/lo (Z 2^sZ, scaled so it cannot overflow FP16) and
//          stores it to its own TMEM lane as pass 2's A operand.  Two warp
//          sets take alternate steps, so one set's latency hides under the
//          other's work.
//  pass 2  Y = sum_t A_t Z_t: rows (block b, column j), K = (term, k),
//          N = (piece, i); B = the hi and lo pieces of A_t 2^sA stacked along
//          N, so per term
//            D2[:, 0:32] (+)= Z_hi [A_hi | A_lo]^T   (N = 32)
//            D2[:, 32:48] (+)= Z_lo A_hi^T           (N = 16).
//          The main product Z_hi A_hi has its 16 columns to itself: tensor-
//          core FP32 accumulation truncates, and keeping the corrections in
//          their own columns halves the chain of truncating adds that reach
//          the largest sums (a full-rank 16x16 mask: 16 instead of 32).
//  epilogue  y[b][i][j] = (D2[i] + (D2[16 + i] + D2[32 + i])) 2^-(sZ + sA)
//          + M[(i,j), 0] x0,
//          the DC term kept out of the products and applied in FP32 as in
//          the dense kernels; each lane stores its block's column straight
//          from registers.
//
// So a unit costs 3 + 2 r MMAs (r <= 4; 3 more per further group of four
// terms), against the dense kernel's 3 x 256 x 256 MAC per block, and the
// data movement stays the dense kernel's 2 KB a block.  The factors' pieces
// and scales come from the FP64 device build (kron.cu); the number of terms
// is read on the device.
//
// Roles (640 threads): warp 0 TMA producer (one 8 KB box per unit), warp 1
// pass-1 MMA issuer, warp 2 TMEM allocator, warp 3 pass-2 MMA issuer, warps
// 4-7 converter (thread = row (b, k): DC out, FP16 split, A1 to TMEM), warps
// 8-11 and 16-19 transposer (even and odd steps), warps 12-15 epilogue.  The
// two passes have their own issuing threads, so pass 1 runs ahead of the
// transposers instead of waiting behind pass 2.  Every wait is bounded
// (sm100_ptx.cuh).
#include "sm100_ptx.cuh"

#include <mutex>

namespace dctf {
namespace {

using namespace ptx;

constexpr int kN2 = 256;
constexpr int kThreads = 640;
constexpr int kUnit = 8;                      // blocks per unit: 128 MMA rows
constexpr int kUnitBytes = kUnit * kN2 * 4;   // 8 KB: one TMA box of 32 floats x 64 lines
constexpr int kStages = 12;
constexpr int kMaxTerms = 16;
constexpr int kDcRing = 8;
// TMEM columns (512 allocated), every buffer aligned to 16 columns
constexpr int kA1Bufs = 4;
constexpr uint32_t kColA1 = 0;      // 4 x 16: x hi (8) | x lo (8)
constexpr uint32_t kColD2 = 64;     // 2 x 48: main | Z_hi A_lo | Z_lo A_hi
constexpr uint32_t kColD1 = 160;    // 2 x 64: pass-1 accumulators (16 per term)
constexpr uint32_t kColA2 = 288;    // 2 x 64: Z hi (32) | Z lo (32), four terms
constexpr uint32_t kTmemCols = 512;
// shared memory
constexpr int kTRow = 20;                     // transposer tile row (floats)
constexpr int kTBlk = 16 * kTRow + 16;        // per block: banks of a warp's 2 blocks disjoint
constexpr int kOffIn = 0;
constexpr int kOffB1 = kOffIn + kStages * kUnitBytes;     // 16 KB pass-1 pieces
constexpr int kOffB2 = kOffB1 + kKronPieceBytes / 2;      // 16 KB pass-2 pieces
constexpr int kOffT = kOffB2 + kKronPieceBytes / 2;
constexpr int kOffMdc = kOffT + 2 * 4 * 2 * kTBlk * 4;   // two transposer sets
constexpr int kOffDc = kOffMdc + kN2 * 4;
constexpr int kOffBar = kOffDc + kDcRing * kUnit * 4;
constexpr int kNumBars = 2 * kStages + 2 * kA1Bufs + 6 * 2 + 2 * kDcRing + 1;
constexpr int kOffMisc = kOffBar + kNumBars * 8;
constexpr int kSmem = kOffMisc + 16 + 1024;
static_assert(kSmem <= 232448, "shared memory");
static_assert(kOffB1 % 1024 == 0 && kOffB2 % 1024 == 0, "swizzle atoms");

enum : uint32_t { kRoleProducer = 1, kRoleMma = 2, kRoleConv = 3, kRoleEpi = 4, kRoleDrain = 5,
                  kRoleTrans = 7 };

// 16 FP32 values -> FP16 hi = rn(v), lo = rn(v - hi), packed in pairs
__device__ __forceinline__ void split16(const float (&v)[16], uint32_t (&hi)[8],
                                        uint32_t (&lo)[8]) {
#pragma unroll
  for (int c = 0; c < 8; ++c) {
    const __half2 h2 = __floats2half2_rn(v[2 * c], v[2 * c + 1]);
    const float2 hf = __half22float2(h2);
    const __half2 l2 = __floats2half2_rn(v[2 * c] - hf.x, v[2 * c + 1] - hf.y);
    hi[c] = *reinterpret_cast<const uint32_t *>(&h2);
    lo[c] = *reinterpret_cast<const uint32_t *>(&l2);
  }
}

__global__ void __launch_bounds__(kThreads, 1)
apply_kron_tc_kernel(const __grid_constant__ CUtensorMap tm_in, float *__restrict__ y,
                     int64_t nblocks, const uint4 *__restrict__ pieces,
                     const float *__restrict__ Mdc, const int *__restrict__ rank_in,
                     const float *__restrict__ kscale, uint32_t *__restrict__ err) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t *base = reinterpret_cast<uint8_t *>(
      (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  uint8_t *s_in = base + kOffIn;
  uint8_t *s_b1 = base + kOffB1;
  uint8_t *s_b2 = base + kOffB2;
  float *s_t = reinterpret_cast<float *>(base + kOffT);
  float *s_mdc = reinterpret_cast<float *>(base + kOffMdc);
  float *s_dc = reinterpret_cast<float *>(base + kOffDc);
  uint64_t *bars = reinterpret_cast<uint64_t *>(base + kOffBar);
  uint64_t *full_in = bars;                   // [kStages] TMA -> converter
  uint64_t *empty_in = full_in + kStages;     // [kStages] converter -> TMA
  uint64_t *a1_full = empty_in + kStages;     // [kA1Bufs] converter -> MMA
  uint64_t *a1_empty = a1_full + kA1Bufs;     // [kA1Bufs] MMA (pass 1 done) -> converter
  uint64_t *d1_full = a1_empty + kA1Bufs;     // [2] MMA -> transposer
  uint64_t *d1_empty = d1_full + 2;           // [2] transposer -> MMA
  uint64_t *a2_full = d1_empty + 2;           // [2] transposer -> MMA
  uint64_t *a2_empty = a2_full + 2;           // [2] MMA (pass 2 done) -> transposer
  uint64_t *d2_full = a2_empty + 2;           // [2] MMA -> epilogue
  uint64_t *d2_empty = d2_full + 2;           // [2] epilogue -> MMA
  uint64_t *dc_full = d2_empty + 2;           // [kDcRing] converter -> epilogue
  uint64_t *dc_empty = dc_full + kDcRing;     // [kDcRing] epilogue -> converter
  uint64_t *b_full = dc_empty + kDcRing;      // the pieces images have landed
  uint32_t *s_tmem = reinterpret_cast<uint32_t *>(base + kOffMisc);
  volatile int *s_abort = reinterpret_cast<volatile int *>(base + kOffMisc + 4);

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int64_t nunits = (nblocks + kUnit - 1) / kUnit;
  const int G = gridDim.x, cta = blockIdx.x;
  const int my_units = cta < nunits ? (int)((nunits - cta + G - 1) / G) : 0;
  const int rank = min(max(*rank_in, 0), kMaxTerms);
  const int NG = (rank + 3) / 4;                // term groups: steps per unit
  const bool terms = rank > 0;
  const int nsteps = my_units * NG;

  if (tid == 0) {
    for (int s = 0; s < kStages; ++s) { mbar_init(&full_in[s], 1); mbar_init(&empty_in[s], 128); }
    for (int b = 0; b < kA1Bufs; ++b) { mbar_init(&a1_full[b], 128); mbar_init(&a1_empty[b], 1); }
    for (int b = 0; b < 2; ++b) {
      mbar_init(&d1_full[b], 1);   mbar_init(&d1_empty[b], 128);
      mbar_init(&a2_full[b], 128); mbar_init(&a2_empty[b], 1);
      mbar_init(&d2_full[b], 1);   mbar_init(&d2_empty[b], 128);
    }
    for (int r = 0; r < kDcRing; ++r) { mbar_init(&dc_full[r], 128); mbar_init(&dc_empty[r], 128); }
    mbar_init(b_full, 1);
    *s_abort = 0;
    mbar_fence_init();
    tma_prefetch_map(&tm_in);
  }
  if (tid < kN2) s_mdc[tid] = __ldg(Mdc + tid);   // M[:, 0]
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
    // both pieces images first (32 KB, already in the swizzled B layout), in
    // the background of the first input loads; the issuers wait for them
    mbar_arrive_expect_tx(b_full, kKronPieceBytes);
    for (int h = 0; h < 2; ++h)
      bulk_load(s_b1 + h * (kKronPieceBytes / 2), pieces + h * (kKronPieceBytes / 32),
                kKronPieceBytes / 2, b_full);
    int issued = 0;
    for (int k = 0; k < my_units; ++k) {
      const int s = k % kStages;
      if (!wait_bounded(&empty_in[s], ((k / kStages) & 1) ^ 1, s_abort, err,
                        kRoleProducer | (k << 8)))
        break;
      mbar_arrive_expect_tx(&full_in[s], kUnitBytes);
      const int64_t unit = cta + (int64_t)k * G;
      tma_load_2d(&tm_in, &full_in[s], s_in + s * kUnitBytes, 0, (int)(unit * 64));
      ++issued;
    }
    for (int k = issued > kStages ? issued - kStages : 0; k < issued; ++k)
      wait_drain(&full_in[k % kStages], (k / kStages) & 1, err, kRoleDrain);
    wait_drain(b_full, 0, err, kRoleDrain);
  } else if (warp == 1 && lane == 0 && terms) {
    // ---------------------------------------------------------- pass-1 issuer
    // D1 = x_hi B_lo^T + x_lo B_hi^T + x_hi B_hi^T for every step, in order
    uint64_t *last_bar = nullptr;
    uint32_t last_ph = 0;
    const bool b_ok = nsteps == 0 || wait_bounded(b_full, 0, s_abort, err, kRoleMma);
    for (int st = 0; b_ok && st < nsteps; ++st) {
      const int k = st / NG, g = st % NG, ng = min(4, rank - 4 * g);
      const int ab = k % kA1Bufs, db = st & 1;
      if (g == 0 && !wait_bounded(&a1_full[ab], (k / kA1Bufs) & 1, s_abort, err,
                                  kRoleMma | (st << 8)))
        break;
      if (!wait_bounded(&d1_empty[db], ((st >> 1) & 1) ^ 1, s_abort, err, kRoleMma | (st << 8)))
        break;
      tc_fence_after();
      const uint32_t t_a1 = tmem + kColA1 + ab * 16, t_d1 = tmem + kColD1 + db * 64;
      const uint32_t idesc = idesc_f16(128, 16 * ng, false);
      const uint64_t b_hi = desc_sw128(smem_u32(s_b1)) + 2 * g;              // K slot g
      const uint64_t b_lo = desc_sw128(smem_u32(s_b1 + 16 * ng * 128)) + 2 * g;
      mma_f16_ts(t_d1, t_a1, b_lo, idesc, 0u);          // x_hi B_lo
      mma_f16_ts(t_d1, t_a1 + 8, b_hi, idesc, 1u);      // x_lo B_hi
      mma_f16_ts(t_d1, t_a1, b_hi, idesc, 1u);          // x_hi B_hi
      tc_commit(&d1_full[db]);
      last_bar = &d1_full[db]; last_ph = (st >> 1) & 1;
      if (g == NG - 1) tc_commit(&a1_empty[ab]);
    }
    // every MMA issued so far has completed once the last commit arrived
    if (last_bar != nullptr) wait_drain(last_bar, last_ph, err, kRoleDrain);
  } else if (warp == 3 && lane == 0 && terms) {
    // ---------------------------------------------------------- pass-2 issuer
    // per term, D2[0:32] (+)= Z_hi [A_hi | A_lo]^T, D2[32:48] (+)= Z_lo A_hi^T
    uint64_t *last_bar = nullptr;
    uint32_t last_ph = 0;
    const bool b_ok = nsteps == 0 || wait_bounded(b_full, 0, s_abort, err, kRoleMma);
    for (int st = 0; b_ok && st < nsteps; ++st) {
      const int k = st / NG, g = st % NG, ng = min(4, rank - 4 * g);
      const int a2b = st & 1, d2b = k & 1;
      if (!wait_bounded(&a2_full[a2b], (st >> 1) & 1, s_abort, err, kRoleMma | (st << 8)))
        break;
      if (g == 0 && !wait_bounded(&d2_empty[d2b], ((k >> 1) & 1) ^ 1, s_abort, err,
                                  kRoleMma | (st << 8)))
        break;
      tc_fence_after();
      const uint32_t t_a2 = tmem + kColA2 + a2b * 64, t_d2 = tmem + kColD2 + d2b * 48;
      const uint64_t b2 = desc_sw128(smem_u32(s_b2 + g * 4096));   // K block g
      for (int tt = 0; tt < ng; ++tt) {
        const uint32_t acc = (g > 0 || tt > 0) ? 1u : 0u;
        mma_f16_ts(t_d2, t_a2 + 8 * tt, b2 + 2 * tt, idesc_f16(128, 32, false), acc);
        mma_f16_ts(t_d2 + 32, t_a2 + 32 + 8 * tt, b2 + 2 * tt, idesc_f16(128, 16, false), acc);
      }
      tc_commit(&a2_empty[a2b]);
      last_bar = &a2_empty[a2b]; last_ph = (st >> 1) & 1;
      if (g == NG - 1) {
        tc_commit(&d2_full[d2b]);
      }
    }
    if (last_bar != nullptr) wait_drain(last_bar, last_ph, err, kRoleDrain);
  } else if (warp >= 4 && warp < 8) {
    // ---------------------------------------------------------- converter
    const int m = tid - 128, lb = m >> 4, r = m & 15;
    const uint32_t lane_base = (uint32_t)((warp & 3) * 32) << 16;
    for (int k = 0; k < my_units; ++k) {
      const int s = k % kStages;
      if (!warp_wait_bounded(&full_in[s], (k / kStages) & 1, s_abort, err, kRoleConv | (k << 8)))
        break;
      // row m of the unit: 64 bytes, half of the 128-byte line m / 2 of the
      // SWIZZLE_128B box (16-byte chunk c of the line at chunk c ^ (line & 7))
      float v[16];
      const int line = m >> 1;
      const uint8_t *row = s_in + s * kUnitBytes + line * 128;
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        const int chunk = ((m & 1) * 4 + c) ^ (line & 7);
        const float4 f = *reinterpret_cast<const float4 *>(row + chunk * 16);
        v[4 * c] = f.x; v[4 * c + 1] = f.y; v[4 * c + 2] = f.z; v[4 * c + 3] = f.w;
      }
      mbar_arrive(&empty_in[s]);
      const float x0 = v[0];
      if (r == 0) v[0] = 0.f;             // the DC coefficient stays out of the products
      const int slot = k % kDcRing;
      if (!warp_wait_bounded(&dc_empty[slot], ((k / kDcRing) & 1) ^ 1, s_abort, err,
                             kRoleConv | (k << 8)))
        break;
      if (r == 0) s_dc[slot * kUnit + lb] = x0;
      mbar_arrive(&dc_full[slot]);
      if (!terms) continue;
      if (!warp_wait_bounded(&a1_empty[k % kA1Bufs], ((k / kA1Bufs) & 1) ^ 1, s_abort, err,
                             kRoleConv | (k << 8)))
        break;
      tc_fence_after();
      uint32_t hi[8], lo[8];
      split16(v, hi, lo);
      const uint32_t t_a1 = tmem + lane_base + kColA1 + (k % kA1Bufs) * 16;
      tmem_st8(t_a1, hi);
      tmem_st8(t_a1 + 8, lo);
      tmem_st_wait();
      tc_fence_before();
      mbar_arrive(&a1_full[k % kA1Bufs]);
    }
  } else if (((warp >= 8 && warp < 12) || warp >= 16) && terms) {
    // ---------------------------------------------------------- transposer
    // warps 8-11 take the even steps (D1 and A2 buffers 0), warps 16-19
    // the odd ones (buffers 1)
    const int q = warp & 3, lb = lane >> 4, r = lane & 15, db = warp >= 16 ? 1 : 0;
    const uint32_t lane_base = (uint32_t)(q * 32) << 16;
    const float zscale = __ldg(kscale);
    float *tile = s_t + ((db * 4 + q) * 2 + lb) * kTBlk;
    const uint32_t t_d1 = tmem + lane_base + kColD1 + db * 64;
    const uint32_t t_a2 = tmem + lane_base + kColA2 + db * 64;
    for (int st = db; st < nsteps; st += 2) {
      const int g = st % NG, ng = min(4, rank - 4 * g);
      if (!warp_wait_bounded(&d1_full[db], (st >> 1) & 1, s_abort, err, kRoleTrans | (st << 8)))
        break;
      tc_fence_after();
      if (!warp_wait_bounded(&a2_empty[db], ((st >> 1) & 1) ^ 1, s_abort, err,
                             kRoleTrans | (st << 8)))
        break;
      for (int tt = 0; tt < ng; ++tt) {
        uint32_t a[16];
        tmem_ld16(t_d1 + 16 * tt, a);
        if (tt == ng - 1) {            // every read of this step's D1 is done
          tc_fence_before();
          mbar_arrive(&d1_empty[db]);
        }
        // row r of Z_t (this lane is row (b, k = r)), scaled to Z 2^sZ
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          float4 z;
          z.x = __uint_as_float(a[4 * u]) * zscale;
          z.y = __uint_as_float(a[4 * u + 1]) * zscale;
          z.z = __uint_as_float(a[4 * u + 2]) * zscale;
          z.w = __uint_as_float(a[4 * u + 3]) * zscale;
          *reinterpret_cast<float4 *>(tile + r * kTRow + 4 * u) = z;
        }
        __syncwarp();
        // column j = r of Z_t: this lane's row (b, j) of pass 2's A operand
        float zc[16];
#pragma unroll
        for (int c = 0; c < 16; ++c) zc[c] = tile[c * kTRow + r];
        __syncwarp();                    // the tile is rewritten by the next term
        uint32_t hi[8], lo[8];
        split16(zc, hi, lo);
        tmem_st8(t_a2 + 8 * tt, hi);
        tmem_st8(t_a2 + 32 + 8 * tt, lo);
      }
      tmem_st_wait();
      tc_fence_before();
      mbar_arrive(&a2_full[db]);
    }
  } else if (warp >= 12 && warp < 16) {
    // ---------------------------------------------------------- epilogue
    // lane (b, j) holds column j of block b's Y: it stores y[b][i][j] for
    // every i straight from registers (a warp's store covers two 64-byte
    // runs, whole sectors), with M[(i, j), 0] for the DC term in registers
    const int q = warp & 3, lb = lane >> 4, j = lane & 15;
    const uint32_t lane_base = (uint32_t)(q * 32) << 16;
    const float oscale = __ldg(kscale + 1);
    float mdc[16];
#pragma unroll
    for (int i = 0; i < 16; ++i) mdc[i] = s_mdc[i * 16 + j];
    // no output is written before the previous kernel on the stream has
    // completed (under programmatic dependent launch)
    if (lane == 0) pdl_wait();
    __syncwarp();
    for (int k = 0; k < my_units; ++k) {
      const int64_t unit = cta + (int64_t)k * G;
      float acc[16];
      if (terms) {
        if (!warp_wait_bounded(&d2_full[k & 1], (k >> 1) & 1, s_abort, err, kRoleEpi | (k << 8)))
          break;
        tc_fence_after();
        uint32_t dm[16], c1[16], c2[16];
        const uint32_t t_d2 = tmem + lane_base + kColD2 + (k & 1) * 48;
        tmem_ld16x3(t_d2, t_d2 + 16, t_d2 + 32, dm, c1, c2);
        tc_fence_before();
        mbar_arrive(&d2_empty[k & 1]);
#pragma unroll
        for (int i = 0; i < 16; ++i)
          acc[i] = (__uint_as_float(dm[i]) + (__uint_as_float(c1[i]) + __uint_as_float(c2[i]))) *
                   oscale;
      } else {
#pragma unroll
        for (int i = 0; i < 16; ++i) acc[i] = 0.f;
      }
      const int slot = k % kDcRing;
      if (!warp_wait_bounded(&dc_full[slot], (k / kDcRing) & 1, s_abort, err, kRoleEpi | (k << 8)))
        break;
      const float x0 = s_dc[slot * kUnit + 2 * q + lb];
      mbar_arrive(&dc_empty[slot]);
      const int64_t gb = unit * kUnit + 2 * q + lb;
      if (gb < nblocks) {
        float *dst = y + gb * kN2 + j;
#pragma unroll
        for (int i = 0; i < 16; ++i) __stcs(dst + i * 16, fmaf(mdc[i], x0, acc[i]));
      }
    }
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

}  // namespace

cudaError_t launch_apply_kron_tc(const dctf_operator *op, const float *x, int64_t nblocks,
                                 float *y, cudaStream_t s, bool pdl) {
  if (op->n != 16 || op->d_kpieces == nullptr || nblocks * 8 >= ((int64_t)1 << 31))
    return cudaErrorInvalidValue;
  EncodeTiledFn enc = encode_fn();
  if (enc == nullptr) return cudaErrorNotSupported;
  // the input as lines of 32 floats (128 B, two rows of a block); one box is
  // 64 lines = one unit of 8 blocks; lines past the end read as zeros
  CUtensorMap tm;
  cuuint64_t dims[2] = {32, (cuuint64_t)nblocks * 8};
  cuuint64_t strides[1] = {128};
  cuuint32_t box[2] = {32, 64};
  cuuint32_t es[2] = {1, 1};
  if (enc(&tm, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<float *>(x), dims, strides, box, es,
          CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
          CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
    return cudaErrorInvalidValue;
  cudaError_t e = cudaFuncSetAttribute(apply_kron_tc_kernel,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, kSmem);
  if (e != cudaSuccess) return e;
  const int64_t nunits = (nblocks + kUnit - 1) / kUnit;
  int grid = sm_count(op->device);
  if (grid > nunits) grid = (int)nunits;
  if (grid < 1) grid = 1;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(kThreads);
  cfg.dynamicSmemBytes = kSmem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  if (pdl) {
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
  }
  e = cudaLaunchKernelEx(&cfg, apply_kron_tc_kernel, tm, y, nblocks,
                         reinterpret_cast<const uint4 *>(op->d_kpieces), op->d_Mdc,
                         op->d_krank, op->d_kscale, op->d_err);
  if (e != cudaSuccess) return e;
  return cudaGetLastError();
}

}  // namespace dctf

// Plain FP32 CUDA-core apply: y_b = M x_b (Eq. 11 / Eq. 20) with FP32 FMA.
//
// The comparison kernel of the library.  A CTA keeps a tile of TB blocks
// resident in shared memory (so in-place filtering is safe: every input of
// the tile is read before any output of it is written) and sweeps the
// outputs in TN-wide chunks and the inputs in TK-wide chunks of M.  Each
// thread owns an RB x RN register tile (blocks strided by TB/RB, outputs by
// TN/RN, which keeps the 16-byte shared loads of a warp on distinct banks).
// The input DC coefficient x_b[0] is left out of the running sums and added
// last as M[:,0] x_b[0]: it is the largest coefficient by far, and adding it
// once to an accumulator of the AC terms keeps the rounding error of the
// sums near one ulp of the output instead of growing with the DC magnitude.
// For 8x8 blocks with FP32 input at full size, apply_simt_db_kernel runs the
// same arithmetic with the next tile's loads overlapped (cp.async into a
// second X buffer); for 16x16 blocks, apply_simt16_db_kernel overlaps the
// loads of the next chunk of M the same way.
#include "dctf_internal.cuh"
#include "sm100_ptx.cuh"

namespace dctf {
namespace {
using namespace ptx;

template <typename Tin> __device__ inline float4 load4(const Tin *p);
template <> __device__ inline float4 load4<float>(const float *p) {
  return __ldg(reinterpret_cast<const float4 *>(p));
}
template <> __device__ inline float4 load4<double>(const double *p) {
  double2 a = __ldg(reinterpret_cast<const double2 *>(p));
  double2 b = __ldg(reinterpret_cast<const double2 *>(p) + 1);
  return make_float4((float)a.x, (float)a.y, (float)b.x, (float)b.y);
}

template <int N2, int TB, int TN, int TK, int RB, int RN>
struct SimtCfg {
  static constexpr int kThreads = (TB / RB) * (TN / RN);
  static constexpr int kXP = N2 + 4;        // X row pitch (floats)
  static constexpr int kMP = TK + 4;        // M chunk row pitch
  static constexpr int kYP = TN + 4;        // Y staging pitch
  static constexpr bool kMResident = (TN == N2 && TK == N2);
  static constexpr bool kYAliasX = (TN == N2);
  static constexpr int kXFloats = TB * kXP;
  static constexpr int kMFloats = TN * kMP;
  static constexpr int kYFloats = kYAliasX ? 0 : TB * kYP;
  static constexpr size_t kSmem = (size_t)(kXFloats + kMFloats + kYFloats + TB) * 4;
  static_assert(kThreads == 128, "128 threads per CTA");
  static_assert(!kYAliasX || TB * kYP <= kXFloats, "Y staging must fit in X");
};

template <typename Tin, int N2, int TB, int TN, int TK, int RB, int RN>
__global__ void __launch_bounds__(128)
apply_simt_kernel(const float *__restrict__ M32, const float *__restrict__ Mdc,
                  const Tin *__restrict__ x, int64_t nblocks, float *y) {
  using Cfg = SimtCfg<N2, TB, TN, TK, RB, RN>;
  constexpr int TPB = TB / RB;   // thread rows (blocks)
  constexpr int TPN = TN / RN;   // thread columns (outputs)
  extern __shared__ __align__(16) float smem[];
  float *Xs = smem;
  float *Ms = Xs + Cfg::kXFloats;
  float *Ys = Cfg::kYAliasX ? Xs : Ms + Cfg::kMFloats;
  float *x0s = Ms + Cfg::kMFloats + Cfg::kYFloats;
  const int t = threadIdx.x, tb = t / TPN, tn = t % TPN;
  const int64_t ntiles = (nblocks + TB - 1) / TB;

  if (Cfg::kMResident) {
    for (int idx = t; idx < N2 * N2 / 4; idx += 128) {
      int r = idx / (N2 / 4), c4 = idx % (N2 / 4);
      *reinterpret_cast<float4 *>(&Ms[r * Cfg::kMP + 4 * c4]) =
          __ldg(reinterpret_cast<const float4 *>(M32 + (size_t)r * N2) + c4);
    }
  }

  for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const int64_t b0 = tile * TB;
    __syncthreads();   // previous tile's readers of Xs / Ys are done
    for (int idx = t; idx < TB * N2 / 4; idx += 128) {
      int r = idx / (N2 / 4), c4 = idx % (N2 / 4);
      int64_t b = b0 + r;
      float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
      if (b < nblocks) v = load4<Tin>(x + b * N2 + 4 * c4);
      if (c4 == 0) { x0s[r] = v.x; v.x = 0.f; }
      *reinterpret_cast<float4 *>(&Xs[r * Cfg::kXP + 4 * c4]) = v;
    }
    for (int n0 = 0; n0 < N2; n0 += TN) {
      float acc[RB][RN];
#pragma unroll
      for (int i = 0; i < RB; ++i)
#pragma unroll
        for (int j = 0; j < RN; ++j) acc[i][j] = 0.f;
      for (int k0 = 0; k0 < N2; k0 += TK) {
        if (!Cfg::kMResident) {
          __syncthreads();
          for (int idx = t; idx < TN * TK / 4; idx += 128) {
            int r = idx / (TK / 4), c4 = idx % (TK / 4);
            *reinterpret_cast<float4 *>(&Ms[r * Cfg::kMP + 4 * c4]) =
                __ldg(reinterpret_cast<const float4 *>(M32 + (size_t)(n0 + r) * N2 + k0) + c4);
          }
        }
        __syncthreads();
#pragma unroll 2
        for (int k4 = 0; k4 < TK; k4 += 4) {
          float4 xa[RB], ma[RN];
#pragma unroll
          for (int i = 0; i < RB; ++i)
            xa[i] = *reinterpret_cast<const float4 *>(&Xs[(tb + TPB * i) * Cfg::kXP + k0 + k4]);
#pragma unroll
          for (int j = 0; j < RN; ++j)
            ma[j] = *reinterpret_cast<const float4 *>(&Ms[(tn + TPN * j) * Cfg::kMP + k4]);
#pragma unroll
          for (int i = 0; i < RB; ++i)
#pragma unroll
            for (int j = 0; j < RN; ++j) {
              acc[i][j] = fmaf(xa[i].x, ma[j].x, acc[i][j]);
              acc[i][j] = fmaf(xa[i].y, ma[j].y, acc[i][j]);
              acc[i][j] = fmaf(xa[i].z, ma[j].z, acc[i][j]);
              acc[i][j] = fmaf(xa[i].w, ma[j].w, acc[i][j]);
            }
        }
      }
      // the DC input term, last (see the file comment)
#pragma unroll
      for (int j = 0; j < RN; ++j) {
        float md = __ldg(Mdc + n0 + tn + TPN * j);
#pragma unroll
        for (int i = 0; i < RB; ++i) acc[i][j] = fmaf(md, x0s[tb + TPB * i], acc[i][j]);
      }
      __syncthreads();   // all reads of Xs (aliased by Ys) / Ys are done
#pragma unroll
      for (int i = 0; i < RB; ++i)
#pragma unroll
        for (int j = 0; j < RN; ++j) Ys[(tb + TPB * i) * Cfg::kYP + tn + TPN * j] = acc[i][j];
      __syncthreads();
      for (int idx = t; idx < TB * TN / 4; idx += 128) {
        int r = idx / (TN / 4), c4 = idx % (TN / 4);
        int64_t b = b0 + r;
        if (b < nblocks)
          *reinterpret_cast<float4 *>(y + b * N2 + n0 + 4 * c4) =
              *reinterpret_cast<const float4 *>(&Ys[r * Cfg::kYP + 4 * c4]);
      }
    }
  }
}

// FP32 input, M resident (TN = TK = N2): the same tile walk and arithmetic
// as apply_simt_kernel, but the next tile's input streams into a second X
// buffer with cp.async while the current tile computes, so the tile loads
// leave the critical path.  Each output sums the same terms in the same
// order: the bits equal apply_simt_kernel's.
template <int N2, int TB, int RB, int RN>
struct SimtDbCfg {
  static constexpr int kThreads = (TB / RB) * (N2 / RN);
  static constexpr int kXP = N2 + 4;
  static constexpr int kXFloats = TB * kXP;
  static constexpr size_t kSmem = (size_t)(2 * kXFloats + N2 * kXP + TB) * 4;
  static_assert(kThreads == 128 && TB == 128, "128 threads, one tile row each");
};

template <int N2, int TB, int RB, int RN>
__global__ void __launch_bounds__(128)
apply_simt_db_kernel(const float *__restrict__ M32, const float *__restrict__ Mdc,
                     const float *__restrict__ x, int64_t nblocks, float *y) {
  using Cfg = SimtDbCfg<N2, TB, RB, RN>;
  constexpr int kXP = Cfg::kXP;
  constexpr int TPB = TB / RB, TPN = N2 / RN;
  extern __shared__ __align__(16) float smem[];
  float *Ms = smem + 2 * Cfg::kXFloats;
  float *x0s = Ms + N2 * kXP;
  const int t = threadIdx.x, tb = t / TPN, tn = t % TPN;
  const int64_t ntiles = (nblocks + TB - 1) / TB;

  for (int idx = t; idx < N2 * N2 / 4; idx += 128) {
    int r = idx / (N2 / 4), c4 = idx % (N2 / 4);
    *reinterpret_cast<float4 *>(&Ms[r * kXP + 4 * c4]) =
        __ldg(reinterpret_cast<const float4 *>(M32 + (size_t)r * N2) + c4);
  }
  // tile `tl` into buffer `buf`: 16-byte copies, zero-filled past nblocks
  auto issue = [&](int64_t tl, int buf) {
    float *dst = smem + buf * Cfg::kXFloats;
    const int64_t b0 = tl * TB;
    for (int idx = t; idx < TB * N2 / 4; idx += 128) {
      const int r = idx / (N2 / 4), c4 = idx % (N2 / 4);
      const bool ok = b0 + r < nblocks;
      cp_async_16(smem_u32(dst + r * kXP + 4 * c4), ok ? x + (b0 + r) * N2 + 4 * c4 : x,
                  ok ? 16u : 0u);
    }
    cp_async_commit();
  };

  int c = 0;
  if ((int64_t)blockIdx.x < ntiles) issue(blockIdx.x, 0);
  for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x, c ^= 1) {
    const int64_t b0 = tile * TB;
    float *Xs = smem + c * Cfg::kXFloats;
    __syncthreads();   // the previous tile's output stores have read buffer c ^ 1
    const bool more = tile + gridDim.x < ntiles;
    if (more) issue(tile + gridDim.x, c ^ 1);
    if (more) cp_async_wait_group<1>(); else cp_async_wait_group<0>();
    __syncthreads();   // every thread's copies of this tile have landed
    x0s[t] = Xs[t * kXP];   // the DC input term, added last
    Xs[t * kXP] = 0.f;
    __syncthreads();
    float acc[RB][RN];
#pragma unroll
    for (int i = 0; i < RB; ++i)
#pragma unroll
      for (int j = 0; j < RN; ++j) acc[i][j] = 0.f;
#pragma unroll 2
    for (int k4 = 0; k4 < N2; k4 += 4) {
      float4 xa[RB], ma[RN];
#pragma unroll
      for (int i = 0; i < RB; ++i)
        xa[i] = *reinterpret_cast<const float4 *>(&Xs[(tb + TPB * i) * kXP + k4]);
#pragma unroll
      for (int j = 0; j < RN; ++j)
        ma[j] = *reinterpret_cast<const float4 *>(&Ms[(tn + TPN * j) * kXP + k4]);
#pragma unroll
      for (int i = 0; i < RB; ++i)
#pragma unroll
        for (int j = 0; j < RN; ++j) {
          acc[i][j] = fmaf(xa[i].x, ma[j].x, acc[i][j]);
          acc[i][j] = fmaf(xa[i].y, ma[j].y, acc[i][j]);
          acc[i][j] = fmaf(xa[i].z, ma[j].z, acc[i][j]);
          acc[i][j] = fmaf(xa[i].w, ma[j].w, acc[i][j]);
        }
    }
#pragma unroll
    for (int j = 0; j < RN; ++j) {
      float md = __ldg(Mdc + tn + TPN * j);
#pragma unroll
      for (int i = 0; i < RB; ++i) acc[i][j] = fmaf(md, x0s[tb + TPB * i], acc[i][j]);
    }
    __syncthreads();   // all reads of Xs done: it stages the outputs now
#pragma unroll
    for (int i = 0; i < RB; ++i)
#pragma unroll
      for (int j = 0; j < RN; ++j) Xs[(tb + TPB * i) * kXP + tn + TPN * j] = acc[i][j];
    __syncthreads();
    for (int idx = t; idx < TB * N2 / 4; idx += 128) {
      int r = idx / (N2 / 4), c4 = idx % (N2 / 4);
      if (b0 + r < nblocks)
        *reinterpret_cast<float4 *>(y + (b0 + r) * N2 + 4 * c4) =
            *reinterpret_cast<const float4 *>(&Xs[r * kXP + 4 * c4]);
    }
  }
}

// 16x16 blocks, FP32 input: M (256 KB) does not fit shared memory, so it
// streams in 128 x 32 chunks, 16 per 64-block tile (two passes of 128
// outputs, eight 32-input chunks each).  The chunk sequence is the same for
// every tile, so the next chunk is always known: it is copied with cp.async
// into the second of two chunk buffers while the current one computes, and
// one barrier a chunk both publishes its copies and retires the previous
// chunk's readers.  Each thread holds an 8 x 8 register tile (8 blocks x 8
// outputs: 16 shared-memory loads per 256 FMAs); each output still sums its
// inputs in order k = 0..255 with one FMA chain (the DC term last), so the
// bits equal apply_simt_kernel's.  Outputs go straight from registers to
// global memory (for each of a thread's outputs, the 16 threads of its block
// row store 64 contiguous bytes), so no staging buffer: 101 KB of shared
// memory a CTA, two CTAs per SM (a 4 x 8 register tile with three CTAs per
// SM measured 8% slower).
struct Simt16Db {
  static constexpr int N2 = 256, TB = 64, TN = 128, TK = 32, RB = 8, RN = 8;
  static constexpr int TPB = TB / RB, TPN = TN / RN;     // 8 x 16 = 128 threads
  static constexpr int kXP = N2 + 4, kMP = TK + 4;
  static constexpr int kChunks = (N2 / TN) * (N2 / TK);  // 16 per tile
  static constexpr int kXFloats = TB * kXP, kMFloats = TN * kMP;
  static constexpr size_t kSmem = (size_t)(kXFloats + 2 * kMFloats + TB) * 4;
  static_assert(TPB * TPN == 128, "128 threads");
};

__global__ void __launch_bounds__(128, 2)
apply_simt16_db_kernel(const float *__restrict__ M32, const float *__restrict__ Mdc,
                       const float *__restrict__ x, int64_t nblocks, float *y) {
  using C = Simt16Db;
  extern __shared__ __align__(16) float smem[];
  float *Xs = smem;
  float *Mb = Xs + C::kXFloats;                  // two chunk buffers
  float *x0s = Mb + 2 * C::kMFloats;
  const int t = threadIdx.x, tb = t / C::TPN, tn = t % C::TPN;
  const int64_t ntiles = (nblocks + C::TB - 1) / C::TB;
  if ((int64_t)blockIdx.x >= ntiles) return;
  // chunk c of a tile: outputs (c / 8) * 128.., inputs (c % 8) * 32..
  auto issue_m = [&](int c, int buf) {
    const int n0 = (c / (C::N2 / C::TK)) * C::TN, k0 = (c % (C::N2 / C::TK)) * C::TK;
    float *dst = Mb + buf * C::kMFloats;
    for (int idx = t; idx < C::TN * C::TK / 4; idx += 128) {
      const int r = idx / (C::TK / 4), c4 = idx % (C::TK / 4);
      cp_async_16(smem_u32(dst + r * C::kMP + 4 * c4), M32 + (size_t)(n0 + r) * C::N2 + k0 + 4 * c4,
                  16u);
    }
    cp_async_commit();
  };
  int cnt = 0;                                   // chunks computed so far by this CTA
  issue_m(0, 0);
  for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const int64_t b0 = tile * C::TB;
    __syncthreads();   // the previous tile's readers of Xs / Ys are done
    for (int idx = t; idx < C::TB * C::N2 / 4; idx += 128) {
      const int r = idx / (C::N2 / 4), c4 = idx % (C::N2 / 4);
      const int64_t b = b0 + r;
      float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
      if (b < nblocks) v = __ldg(reinterpret_cast<const float4 *>(x + b * C::N2) + c4);
      if (c4 == 0) { x0s[r] = v.x; v.x = 0.f; }
      *reinterpret_cast<float4 *>(&Xs[r * C::kXP + 4 * c4]) = v;
    }
    for (int n0 = 0; n0 < C::N2; n0 += C::TN) {
      float acc[C::RB][C::RN];
#pragma unroll
      for (int i = 0; i < C::RB; ++i)
#pragma unroll
        for (int j = 0; j < C::RN; ++j) acc[i][j] = 0.f;
      for (int k0 = 0; k0 < C::N2; k0 += C::TK, ++cnt) {
        cp_async_wait_group<0>();   // this thread's copies of chunk cnt (the only ones in flight)
        __syncthreads();            // every thread's have landed, and chunk cnt - 1 is read
        issue_m((cnt + 1) % C::kChunks, (cnt + 1) & 1);
        const float *Ms = Mb + (cnt & 1) * C::kMFloats;
#pragma unroll 2
        for (int k4 = 0; k4 < C::TK; k4 += 4) {
          float4 xa[C::RB], ma[C::RN];
#pragma unroll
          for (int i = 0; i < C::RB; ++i)
            xa[i] = *reinterpret_cast<const float4 *>(&Xs[(tb + C::TPB * i) * C::kXP + k0 + k4]);
#pragma unroll
          for (int j = 0; j < C::RN; ++j)
            ma[j] = *reinterpret_cast<const float4 *>(&Ms[(tn + C::TPN * j) * C::kMP + k4]);
#pragma unroll
          for (int i = 0; i < C::RB; ++i)
#pragma unroll
            for (int j = 0; j < C::RN; ++j) {
              acc[i][j] = fmaf(xa[i].x, ma[j].x, acc[i][j]);
              acc[i][j] = fmaf(xa[i].y, ma[j].y, acc[i][j]);
              acc[i][j] = fmaf(xa[i].z, ma[j].z, acc[i][j]);
              acc[i][j] = fmaf(xa[i].w, ma[j].w, acc[i][j]);
            }
        }
      }
#pragma unroll
      for (int j = 0; j < C::RN; ++j) {
        const float md = __ldg(Mdc + n0 + tn + C::TPN * j);
#pragma unroll
        for (int i = 0; i < C::RB; ++i) acc[i][j] = fmaf(md, x0s[tb + C::TPB * i], acc[i][j]);
      }
      // in place is safe: the whole tile's input is in Xs already
#pragma unroll
      for (int i = 0; i < C::RB; ++i) {
        const int64_t b = b0 + tb + C::TPB * i;
        if (b < nblocks) {
#pragma unroll
          for (int j = 0; j < C::RN; ++j) y[b * C::N2 + n0 + tn + C::TPN * j] = acc[i][j];
        }
      }
    }
  }
  cp_async_wait_group<0>();   // the prefetch of a chunk no tile uses
}

cudaError_t launch_simt16_db(const dctf_operator *op, const float *x, int64_t nblocks, float *y,
                             cudaStream_t s) {
  using C = Simt16Db;
  cudaError_t e = cudaFuncSetAttribute(apply_simt16_db_kernel,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)C::kSmem);
  if (e != cudaSuccess) return e;
  int per_sm = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, apply_simt16_db_kernel, 128, C::kSmem);
  if (e != cudaSuccess) return e;
  if (per_sm < 1) per_sm = 1;
  const int64_t ntiles = (nblocks + C::TB - 1) / C::TB;
  int64_t grid = (int64_t)per_sm * sm_count(op->device);
  if (grid > ntiles) grid = ntiles;
  if (grid < 1) grid = 1;
  apply_simt16_db_kernel<<<(unsigned)grid, 128, C::kSmem, s>>>(op->d_M32, op->d_Mdc, x, nblocks, y);
  return cudaGetLastError();
}

template <int N2, int TB, int RB, int RN>
cudaError_t launch_db(const dctf_operator *op, const float *x, int64_t nblocks, float *y,
                      cudaStream_t s) {
  using Cfg = SimtDbCfg<N2, TB, RB, RN>;
  auto kern = apply_simt_db_kernel<N2, TB, RB, RN>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)Cfg::kSmem);
  if (e != cudaSuccess) return e;
  int per_sm = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, 128, Cfg::kSmem);
  if (e != cudaSuccess) return e;
  if (per_sm < 1) per_sm = 1;
  int64_t ntiles = (nblocks + TB - 1) / TB;
  int64_t grid = (int64_t)per_sm * sm_count(op->device);
  if (grid > ntiles) grid = ntiles;
  if (grid < 1) grid = 1;
  kern<<<(unsigned)grid, 128, Cfg::kSmem, s>>>(op->d_M32, op->d_Mdc, x, nblocks, y);
  return cudaGetLastError();
}

template <typename Tin, int N2, int TB, int TN, int TK, int RB, int RN>
cudaError_t launch_cfg(const dctf_operator *op, const Tin *x, int64_t nblocks, float *y,
                       cudaStream_t s) {
  using Cfg = SimtCfg<N2, TB, TN, TK, RB, RN>;
  auto kern = apply_simt_kernel<Tin, N2, TB, TN, TK, RB, RN>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)Cfg::kSmem);
  if (e != cudaSuccess) return e;
  int per_sm = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, 128, Cfg::kSmem);
  if (e != cudaSuccess) return e;
  if (per_sm < 1) per_sm = 1;
  int64_t ntiles = (nblocks + TB - 1) / TB;
  int64_t grid = (int64_t)per_sm * sm_count(op->device);
  if (grid > ntiles) grid = ntiles;
  if (grid < 1) grid = 1;
  kern<<<(unsigned)grid, 128, Cfg::kSmem, s>>>(op->d_M32, op->d_Mdc, x, nblocks, y);
  return cudaGetLastError();
}

template <typename Tin>
cudaError_t dispatch(const dctf_operator *op, const Tin *x, int64_t nblocks, float *y,
                     cudaStream_t s) {
  switch (op->n) {
    case 4:  return launch_cfg<Tin, 16, 128, 16, 16, 8, 2>(op, x, nblocks, y, s);
    case 8:
      // fewer blocks than 128-block tiles can spread over the SMs (the
      // 256 x 256 workload has 1,024): 16-block tiles, 8x the CTAs.  Each
      // output sums the same K chunks in the same order, so the bits match.
      if (nblocks < (int64_t)128 * sm_count(op->device))
        return launch_cfg<Tin, 64, 16, 64, 64, 2, 4>(op, x, nblocks, y, s);
      // FP32 input (16-byte aligned, checked by the caller): double-buffered
      if constexpr (sizeof(Tin) == 4)
        return launch_db<64, 128, 8, 8>(op, reinterpret_cast<const float *>(x), nblocks, y, s);
      else
        return launch_cfg<Tin, 64, 128, 64, 64, 8, 8>(op, x, nblocks, y, s);
    case 16:
      // FP32 input: the M chunks double-buffered (same bits)
      if constexpr (sizeof(Tin) == 4)
        return launch_simt16_db(op, reinterpret_cast<const float *>(x), nblocks, y, s);
      else
        return launch_cfg<Tin, 256, 32, 128, 64, 4, 8>(op, x, nblocks, y, s);
  }
  return cudaErrorInvalidValue;
}

}  // namespace

cudaError_t launch_apply_simt(const dctf_operator *op, const float *x, const double *x64,
                              int64_t nblocks, float *y, cudaStream_t s) {
  if (x64 != nullptr) return dispatch<double>(op, x64, nblocks, y, s);
  return dispatch<float>(op, x, nblocks, y, s);
}

}  // namespace dctf

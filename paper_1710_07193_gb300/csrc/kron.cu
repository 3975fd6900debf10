// Paper-form apply: the operator as a sum of Kronecker products,
// M = sum_t A_t kron B_t, applied to each block as sandwich products
// Y = sum_t A_t X B_t^T (Sec. II.B Eq. 11-12, Sec. II.C Eq. 20), in FP32 on
// CUDA cores.
//
// The paper builds its 3x3 filters as three (zero padding) or nine
// (replication) sandwich products of shift and Toeplitz matrices.  The same
// structure holds for any mask: a separable mask u v^T filters the block's
// columns and rows independently, and both paddings act on each axis on its
// own (a pixel is dropped when either coordinate leaves the block;
// replication clamps each coordinate), so its H is H_u kron H_v.  Writing
// the mask as a sum of r = rank(w) separable terms gives
//   M = sum_t (C H_{u_t} C^T) kron (C H_{v_t} C^T),
// and vec(A X B^T) = (A kron B) vec(X) for the row-major vec.  Per block
// that is r * 2 N^3 multiply-adds instead of N^4: 8x fewer for a separable
// mask at N = 16, the same as the dense product at r = N / 2.
//
// Build, all on the device in FP64: one CTA per (term, side).  Every CTA
// first splits the mask into rank-1 terms by Gaussian elimination with
// complete pivoting (the same deterministic steps in every CTA, so all agree
// on the split; exact up to FP64 rounding, stopping at the numerical rank),
// then, if its term exists, forms the 1-D filter matrix of its side and its
// DCT form C H C^T, stored in FP64 and FP32; CTA 0 records the rank.  For
// 16x16 blocks one more CTA then writes the FP16 pieces of every factor for
// the tensor-core form (kron_tc.cu) and their scales.
//
// Apply: 256 threads, thread = (block, rows i and i + N/2).  Per term:
// U = X B_t^T row by row (the two X rows in registers, B_t from shared
// memory by broadcast), U to shared memory, then Y[r, :] += sum_k A_t[r, k]
// U[k, :] (a block's threads sit in one warp, so warp-level
// synchronisation is enough).  FP32 throughout;
// as in the dense kernels the input DC coefficient (~N x the block mean) is
// kept out of the products and added last as M[:,0] x[0], which keeps the
// FP32 error near 1e-4 (without it, 1.2e-3 on the 4096^2 workload's mask).
#include <cmath>
#include <cstring>

#include "dctf_internal.cuh"

namespace dctf {
namespace {

constexpr int kMaxTerms = kMaxN;
constexpr int kBuildThreads = 256;

// Gaussian elimination with complete pivoting on the mask, by all threads of
// the CTA: each step takes the largest remaining |R[p][q]| (the first in
// row-major order among equals) as pivot, emits u = R[:, q] / R[p][q],
// v = R[p, :] and subtracts u v^T; it stops when the largest remainder is
// not above 1e-13 of the mask's largest entry (the numerical rank).  Returns
// the number of terms; u[t][r], v[t][c] in shared memory.
__device__ int split_mask(const MaskParams &mp, double (*R)[kMaxN], double (*u)[kMaxN],
                          double (*v)[kMaxN], double *s_val, int *s_idx) {
  const int mh = mp.mh, mw = mp.mw, n = mh * mw, tid = threadIdx.x;
  const int lane = tid & 31, warp = tid >> 5, nwarps = kBuildThreads / 32;
  if (tid < n) R[tid / mw][tid % mw] = mp.w[tid];
  __syncthreads();
  // argmax of |R| over the mask, ties to the lower index; returns the index
  auto argmax = [&](double *best) -> int {
    double val = tid < n ? fabs(R[tid / mw][tid % mw]) : -1.0;
    int idx = tid < n ? tid : n;
    for (int o = 16; o > 0; o >>= 1) {
      const double ov = __shfl_down_sync(0xffffffffu, val, o);
      const int oi = __shfl_down_sync(0xffffffffu, idx, o);
      if (ov > val || (ov == val && oi < idx)) { val = ov; idx = oi; }
    }
    if (lane == 0) { s_val[warp] = val; s_idx[warp] = idx; }
    __syncthreads();
    double bv = s_val[0];
    int bi = s_idx[0];
    for (int w = 1; w < nwarps; ++w)
      if (s_val[w] > bv || (s_val[w] == bv && s_idx[w] < bi)) { bv = s_val[w]; bi = s_idx[w]; }
    __syncthreads();            // s_val / s_idx are reused by the next call
    *best = bv;
    return bi;
  };
  double wmax;
  argmax(&wmax);
  int rank = 0;
  const int steps = mh < mw ? mh : mw;
  for (int k = 0; k < steps; ++k) {
    double best;
    const int pq = argmax(&best);
    if (!(best > 1e-13 * wmax)) break;
    const int p = pq / mw, q = pq % mw;
    const double piv = R[p][q];
    if (tid < mh) u[rank][tid] = R[tid][q] / piv;
    if (tid < mw) v[rank][tid] = R[p][tid];
    __syncthreads();
    if (tid < n) R[tid / mw][tid % mw] -= u[rank][tid / mw] * v[rank][tid % mw];
    __syncthreads();
    ++rank;
  }
  return rank;
}

// A_t (side 0) or B_t (side 1) of term t = blockIdx.x / 2: the 1-D filter
// matrix H[i][s] = sum_r f[r] [P(i + r - a) = s], then C H C^T (Eq. 7).
__global__ void __launch_bounds__(kBuildThreads)
kron_build_kernel(const MaskParams mp, const double *__restrict__ C, float *__restrict__ A,
                  float *__restrict__ B, double *__restrict__ A64, double *__restrict__ B64,
                  int *__restrict__ rank_out) {
  __shared__ double cs[kMaxN][kMaxN + 1], hs[kMaxN][kMaxN + 1], ts[kMaxN][kMaxN + 1];
  __shared__ double R[kMaxN][kMaxN], su[kMaxTerms][kMaxN], sv[kMaxTerms][kMaxN];
  __shared__ double s_val[kBuildThreads / 32];
  __shared__ int s_idx[kBuildThreads / 32];
  const int rank = split_mask(mp, R, su, sv, s_val, s_idx);
  if (blockIdx.x == 0 && threadIdx.x == 0) *rank_out = rank;
  const int n = mp.n, t = blockIdx.x >> 1, side = blockIdx.x & 1;
  if (t >= rank) return;
  const int i = threadIdx.x / n, j = threadIdx.x % n;
  const bool live = threadIdx.x < n * n;
  const double *f = side ? sv[t] : su[t];
  const int len = side ? mp.mw : mp.mh, a = side ? mp.ac : mp.ar;
  if (live) {
    cs[i][j] = C[i * n + j];
    double h = 0.0;                       // entry (i, s = j)
    for (int r = 0; r < len; ++r) {
      int s = i + r - a;
      if (mp.boundary == DCTF_ZERO) {
        if (s < 0 || s >= n) continue;
      } else {
        s = min(max(s, 0), n - 1);
      }
      if (s == j) h += f[r];
    }
    hs[i][j] = h;
  }
  __syncthreads();
  if (live) {                             // T = H C^T
    double acc = 0.0;
    for (int q = 0; q < n; ++q) acc += hs[i][q] * cs[j][q];
    ts[i][j] = acc;
  }
  __syncthreads();
  if (live) {                             // C T = C H C^T
    double acc = 0.0;
    for (int p = 0; p < n; ++p) acc += cs[i][p] * ts[p][j];
    const size_t o = (size_t)t * n * n + i * n + j;
    (side ? B : A)[o] = (float)acc;
    (side ? B64 : A64)[o] = acc;
  }
}

// n = 16: the FP16 pieces of the factors for the tensor-core form
// (kron_tc.cu), in the K-major SWIZZLE_128B B-operand layout, and their
// power-of-two scales.
//  * Pass 1 operand (16 KB, 128 rows): terms in groups of four; group g uses
//    the 32-byte K slot g of every 128-byte row, with rows
//    p * 16 ng + tt * 16 + j for piece p (0 = hi, 1 = lo) of
//    B_t[j][:] 2^sB, t = 4 g + tt, ng the group's term count.
//  * Pass 2 operand (16 KB): K block g (4 KB, 32 rows) holds rows p * 16 + i,
//    elements (tt, k) of piece p of A_t[i][k] 2^sA, t = 4 g + tt.
//  * sB, sA put the largest factor entry near 2^10, so the lo pieces stay
//    normal FP16 numbers; sZ makes |Z 2^sZ| <= max |x| for the intermediate
//    Z_t = X B_t^T (row sums of |B_t| at most 2^-sZ), so the FP16 re-split of
//    Z cannot overflow where x itself fits FP16.
//  scale[0] = 2^(sZ - sB) (pass 1 result -> Z 2^sZ), scale[1] = 2^-(sZ + sA).
__global__ void __launch_bounds__(kBuildThreads)
kron_pieces_kernel(const double *__restrict__ A64, const double *__restrict__ B64,
                   const int *__restrict__ rank_in, uint8_t *__restrict__ pieces,
                   float *__restrict__ scale) {
  constexpr int n = 16, n2 = 256;
  __shared__ double red[3][kBuildThreads];
  const int tid = threadIdx.x, rank = *rank_in;
  for (int e = tid; e < kKronPieceBytes / 16; e += kBuildThreads)
    reinterpret_cast<uint4 *>(pieces)[e] = make_uint4(0, 0, 0, 0);
  double ma = 0.0, mb = 0.0, rs = 0.0;
  for (int e = tid; e < rank * n2; e += kBuildThreads) {
    ma = fmax(ma, fabs(A64[e]));
    mb = fmax(mb, fabs(B64[e]));
  }
  for (int e = tid; e < rank * n; e += kBuildThreads) {    // row sums of |B_t|
    double r = 0.0;
    for (int l = 0; l < n; ++l) r += fabs(B64[(size_t)e * n + l]);
    rs = fmax(rs, r);
  }
  red[0][tid] = ma; red[1][tid] = mb; red[2][tid] = rs;
  __syncthreads();
  for (int w = kBuildThreads / 2; w > 0; w >>= 1) {
    if (tid < w)
      for (int k = 0; k < 3; ++k) red[k][tid] = fmax(red[k][tid], red[k][tid + w]);
    __syncthreads();
  }
  ma = red[0][0]; mb = red[1][0]; rs = red[2][0];
  auto clampi = [](int e) { return e < -40 ? -40 : (e > 40 ? 40 : e); };
  const int sA = ma > 0.0 ? clampi(10 - (int)ceil(log2(ma))) : 0;
  const int sB = mb > 0.0 ? clampi(10 - (int)ceil(log2(mb))) : 0;
  const int sZ = rs > 0.0 ? clampi(-(int)ceil(log2(rs))) : 0;
  if (tid == 0) {
    scale[0] = (float)ldexp(1.0, sZ - sB);
    scale[1] = (float)ldexp(1.0, -(sZ + sA));
  }
  __syncthreads();     // the zero fill is complete before the pieces land
  for (int e = tid; e < rank * n2; e += kBuildThreads) {
    const int t = e / n2, r = (e / n) % n, c = e % n;      // factor row r, column c
    const int g = t >> 2, tt = t & 3, ng = min(4, rank - 4 * g);
    // pass 1: B_t[j = r][l = c]
    {
      const double x = ldexp(B64[e], sB);
      const __half hi = __double2half(x), lo = __double2half(x - (double)__half2float(hi));
      const int byte = 32 * g + 2 * c;
      *reinterpret_cast<__half *>(pieces + sw128_offset(tt * 16 + r, byte, 128, 0)) = hi;
      *reinterpret_cast<__half *>(pieces + sw128_offset(16 * ng + tt * 16 + r, byte, 128, 0)) = lo;
    }
    // pass 2: A_t[i = r][k = c]
    {
      const double x = ldexp(A64[e], sA);
      const __half hi = __double2half(x), lo = __double2half(x - (double)__half2float(hi));
      const int byte = 2 * (tt * 16 + c);
      uint8_t *p2 = pieces + kKronPieceBytes / 2;
      *reinterpret_cast<__half *>(p2 + sw128_offset(r, byte, 32, g)) = hi;
      *reinterpret_cast<__half *>(p2 + sw128_offset(16 + r, byte, 32, g)) = lo;
    }
  }
}

constexpr int kThreads = 256;

// Thread = (block, row pair i, i + N/2): every shared-memory load of B_t or
// of a U row feeds two rows' multiply-adds.
template <int N>
__global__ void __launch_bounds__(kThreads, 2)
apply_kron_kernel(const float *__restrict__ x, float *__restrict__ y, int64_t nblocks,
                  const float *__restrict__ A, const float *__restrict__ B,
                  const float *__restrict__ Mdc, const int *__restrict__ rank_in, int max_rank) {
  // the number of terms, from the device build (at most max_rank, which
  // sized the shared memory)
  const int rank = min(*rank_in, max_rank);
  constexpr int H = N / 2;                // threads per block
  constexpr int BPC = kThreads / H;       // blocks per pass
  constexpr int LD = N + 4;               // padded row (16-byte aligned, fewer bank conflicts)
  // one block's U, padded by 4 floats: N * LD is a multiple of 32 banks, so
  // unpadded the blocks of a warp would read their U rows from the same
  // banks (4-way conflicts at N = 16 on every 16-byte load)
  constexpr int UB = N * LD + 4;
  extern __shared__ __align__(16) float smem_f[];
  float *sA = smem_f;                     // [rank][N][LD]
  float *sB = sA + rank * N * LD;         // [rank][N][N]
  float *sU = sB + rank * N * N;          // [BPC][UB]
  float *sDc = sU + BPC * UB;             // [N * N]: M[:, 0]
  for (int e = threadIdx.x; e < rank * N * N; e += kThreads) {
    const int t = e / (N * N), r = (e / N) % N, c = e % N;
    sA[(t * N + r) * LD + c] = A[e];
    sB[e] = B[e];
  }
  for (int e = threadIdx.x; e < N * N; e += kThreads) sDc[e] = Mdc[e];
  __syncthreads();
  const int lb = threadIdx.x / H, i = threadIdx.x % H;   // rows i and i + H
  float *u_blk = sU + lb * UB;
  for (int64_t b0 = (int64_t)blockIdx.x * BPC; b0 < nblocks; b0 += (int64_t)gridDim.x * BPC) {
    const int64_t b = b0 + lb;
    const bool live = b < nblocks;
    float x0r[N], x1r[N], y0r[N], y1r[N];
    if (live) {
      const float4 *s0 = reinterpret_cast<const float4 *>(x + b * N * N + i * N);
      const float4 *s1 = reinterpret_cast<const float4 *>(x + b * N * N + (i + H) * N);
#pragma unroll
      for (int q = 0; q < N / 4; ++q) {
        const float4 v = __ldcs(s0 + q), w = __ldcs(s1 + q);
        x0r[4 * q] = v.x; x0r[4 * q + 1] = v.y; x0r[4 * q + 2] = v.z; x0r[4 * q + 3] = v.w;
        x1r[4 * q] = w.x; x1r[4 * q + 1] = w.y; x1r[4 * q + 2] = w.z; x1r[4 * q + 3] = w.w;
      }
    } else {
#pragma unroll
      for (int k = 0; k < N; ++k) { x0r[k] = 0.f; x1r[k] = 0.f; }
    }
    // the block's DC coefficient, from its row-0 thread (first lane of the block)
    const float xdc = __shfl_sync(0xffffffffu, x0r[0], (threadIdx.x & 31) & ~(H - 1));
    if (i == 0) x0r[0] = 0.f;
#pragma unroll
    for (int k = 0; k < N; ++k) { y0r[k] = 0.f; y1r[k] = 0.f; }
    for (int t = 0; t < rank; ++t) {
      // U[r][j] = sum_k X[r][k] B_t[j][k] for r = i, i + H
      const float *bt = sB + t * N * N;
#pragma unroll
      for (int jq = 0; jq < N / 4; ++jq) {
        float u0[4], u1[4];
#pragma unroll
        for (int e = 0; e < 4; ++e) {
          const int j = 4 * jq + e;
          float a0 = 0.f, a1 = 0.f;
#pragma unroll
          for (int q = 0; q < N / 4; ++q) {
            const float4 bv = *reinterpret_cast<const float4 *>(bt + j * N + 4 * q);
            a0 = fmaf(x0r[4 * q], bv.x, a0); a1 = fmaf(x1r[4 * q], bv.x, a1);
            a0 = fmaf(x0r[4 * q + 1], bv.y, a0); a1 = fmaf(x1r[4 * q + 1], bv.y, a1);
            a0 = fmaf(x0r[4 * q + 2], bv.z, a0); a1 = fmaf(x1r[4 * q + 2], bv.z, a1);
            a0 = fmaf(x0r[4 * q + 3], bv.w, a0); a1 = fmaf(x1r[4 * q + 3], bv.w, a1);
          }
          u0[e] = a0; u1[e] = a1;
        }
        *reinterpret_cast<float4 *>(u_blk + i * LD + 4 * jq) = make_float4(u0[0], u0[1], u0[2], u0[3]);
        *reinterpret_cast<float4 *>(u_blk + (i + H) * LD + 4 * jq) =
            make_float4(u1[0], u1[1], u1[2], u1[3]);
      }
      __syncwarp();
      // Y[r][:] += sum_k A_t[r][k] U[k][:]
      const float *at0 = sA + (t * N + i) * LD, *at1 = sA + (t * N + i + H) * LD;
#pragma unroll
      for (int kq = 0; kq < N / 4; ++kq) {
        const float4 p4 = *reinterpret_cast<const float4 *>(at0 + 4 * kq);
        const float4 q4 = *reinterpret_cast<const float4 *>(at1 + 4 * kq);
        const float av0[4] = {p4.x, p4.y, p4.z, p4.w}, av1[4] = {q4.x, q4.y, q4.z, q4.w};
#pragma unroll
        for (int e = 0; e < 4; ++e) {
          const int k = 4 * kq + e;
#pragma unroll
          for (int q = 0; q < N / 4; ++q) {
            const float4 uv = *reinterpret_cast<const float4 *>(u_blk + k * LD + 4 * q);
            y0r[4 * q] = fmaf(av0[e], uv.x, y0r[4 * q]);
            y0r[4 * q + 1] = fmaf(av0[e], uv.y, y0r[4 * q + 1]);
            y0r[4 * q + 2] = fmaf(av0[e], uv.z, y0r[4 * q + 2]);
            y0r[4 * q + 3] = fmaf(av0[e], uv.w, y0r[4 * q + 3]);
            y1r[4 * q] = fmaf(av1[e], uv.x, y1r[4 * q]);
            y1r[4 * q + 1] = fmaf(av1[e], uv.y, y1r[4 * q + 1]);
            y1r[4 * q + 2] = fmaf(av1[e], uv.z, y1r[4 * q + 2]);
            y1r[4 * q + 3] = fmaf(av1[e], uv.w, y1r[4 * q + 3]);
          }
        }
      }
      __syncwarp();                       // U is rewritten by the next term
    }
#pragma unroll
    for (int k = 0; k < N; ++k) {
      y0r[k] = fmaf(sDc[i * N + k], xdc, y0r[k]);
      y1r[k] = fmaf(sDc[(i + H) * N + k], xdc, y1r[k]);
    }
    if (live) {
      float4 *d0 = reinterpret_cast<float4 *>(y + b * N * N + i * N);
      float4 *d1 = reinterpret_cast<float4 *>(y + b * N * N + (i + H) * N);
#pragma unroll
      for (int q = 0; q < N / 4; ++q) {
        __stcs(d0 + q, make_float4(y0r[4 * q], y0r[4 * q + 1], y0r[4 * q + 2], y0r[4 * q + 3]));
        __stcs(d1 + q, make_float4(y1r[4 * q], y1r[4 * q + 1], y1r[4 * q + 2], y1r[4 * q + 3]));
      }
    }
  }
}

template <int N>
cudaError_t launch_apply(const dctf_operator *op, const float *x, int64_t nblocks, float *y,
                         cudaStream_t s) {
  constexpr int BPC = kThreads / (N / 2), LD = N + 4, UB = N * LD + 4;
  const int smem =
      (op->krank_bound * N * LD + op->krank_bound * N * N + BPC * UB + N * N) * (int)sizeof(float);
  cudaError_t e = cudaFuncSetAttribute(apply_kron_kernel<N>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e != cudaSuccess) return e;
  int64_t grid = (nblocks + BPC - 1) / BPC;
  const int64_t cap = 2LL * sm_count(op->device);
  if (grid > cap) grid = cap;
  if (grid < 1) grid = 1;
  apply_kron_kernel<N><<<(unsigned)grid, kThreads, smem, s>>>(x, y, nblocks, op->d_kA, op->d_kB,
                                                             op->d_Mdc, op->d_krank,
                                                             op->krank_bound);
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_kron_build(dctf_operator *op, const MaskParams &mp, cudaStream_t s) {
  op->krank_bound = mp.mh < mp.mw ? mp.mh : mp.mw;
  kron_build_kernel<<<2 * op->krank_bound, kBuildThreads, 0, s>>>(
      mp, op->d_C64, op->d_kA, op->d_kB, op->d_kA64, op->d_kB64, op->d_krank);
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess && op->d_kpieces != nullptr) {
    kron_pieces_kernel<<<1, kBuildThreads, 0, s>>>(op->d_kA64, op->d_kB64, op->d_krank,
                                                   op->d_kpieces, op->d_kscale);
    e = cudaGetLastError();
  }
  return e;
}

cudaError_t launch_apply_kron(const dctf_operator *op, const float *x, int64_t nblocks, float *y,
                              cudaStream_t s) {
  switch (op->n) {
    case 4: return launch_apply<4>(op, x, nblocks, y, s);
    case 8: return launch_apply<8>(op, x, nblocks, y, s);
    case 16: return launch_apply<16>(op, x, nblocks, y, s);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace dctf

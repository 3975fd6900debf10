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
// Build: the host splits the mask into rank-1 terms by Gaussian elimination
// with complete pivoting (exact up to FP64 rounding, stops at the numerical
// rank); one CTA per (term, side) forms the 1-D filter matrix and its DCT
// form C H C^T in FP64 and stores it in FP32.
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

struct KronParams {
  double u[kMaxTerms][kMaxN];   // column factor of term t (mask rows)
  double v[kMaxTerms][kMaxN];   // row factor of term t (mask columns)
  int rank, mh, mw, ar, ac, n, boundary;
};

// A_t (side 0) or B_t (side 1) of term t = blockIdx.x / 2: the 1-D filter
// matrix H[i][s] = sum_r f[r] [P(i + r - a) = s], then C H C^T (Eq. 7).
__global__ void kron_build_kernel(const KronParams kp, const double *__restrict__ C,
                                  float *__restrict__ A, float *__restrict__ B) {
  __shared__ double cs[kMaxN][kMaxN + 1], hs[kMaxN][kMaxN + 1], ts[kMaxN][kMaxN + 1];
  const int n = kp.n, t = blockIdx.x >> 1, side = blockIdx.x & 1;
  const int i = threadIdx.x / n, j = threadIdx.x % n;
  const bool live = threadIdx.x < n * n;
  const double *f = side ? kp.v[t] : kp.u[t];
  const int len = side ? kp.mw : kp.mh, a = side ? kp.ac : kp.ar;
  if (live) {
    cs[i][j] = C[i * n + j];
    double h = 0.0;                       // entry (i, s = j)
    for (int r = 0; r < len; ++r) {
      int s = i + r - a;
      if (kp.boundary == DCTF_ZERO) {
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
    (side ? B : A)[(size_t)t * n * n + i * n + j] = (float)acc;
  }
}

constexpr int kThreads = 256;

// Thread = (block, row pair i, i + N/2): every shared-memory load of B_t or
// of a U row feeds two rows' multiply-adds.
template <int N>
__global__ void __launch_bounds__(kThreads, 2)
apply_kron_kernel(const float *__restrict__ x, float *__restrict__ y, int64_t nblocks,
                  const float *__restrict__ A, const float *__restrict__ B,
                  const float *__restrict__ Mdc, int rank) {
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
      (op->krank * N * LD + op->krank * N * N + BPC * UB + N * N) * (int)sizeof(float);
  cudaError_t e = cudaFuncSetAttribute(apply_kron_kernel<N>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e != cudaSuccess) return e;
  int64_t grid = (nblocks + BPC - 1) / BPC;
  const int64_t cap = 2LL * sm_count(op->device);
  if (grid > cap) grid = cap;
  if (grid < 1) grid = 1;
  apply_kron_kernel<N><<<(unsigned)grid, kThreads, smem, s>>>(x, y, nblocks, op->d_kA, op->d_kB,
                                                             op->d_Mdc, op->krank);
  return cudaGetLastError();
}

}  // namespace

// Split the mask into rank-1 terms, w = sum_t u_t v_t^T, by Gaussian
// elimination with complete pivoting: each step takes the largest remaining
// entry w[p][q] as pivot, emits u = R[:, q] / R[p][q], v = R[p, :] and
// subtracts u v^T.  Stops when the remainder is below 1e-13 of the mask's
// largest entry (the numerical rank).  Returns the number of terms.
int kron_split_mask(const MaskParams &mp, double (*u)[kMaxN], double (*v)[kMaxN]) {
  const int mh = mp.mh, mw = mp.mw;
  double R[kMaxN][kMaxN];
  double wmax = 0.0;
  for (int r = 0; r < mh; ++r)
    for (int c = 0; c < mw; ++c) {
      R[r][c] = mp.w[r * mw + c];
      wmax = fmax(wmax, fabs(R[r][c]));
    }
  int rank = 0;
  const int steps = mh < mw ? mh : mw;
  for (int k = 0; k < steps; ++k) {
    int p = 0, q = 0;
    double best = -1.0;
    for (int r = 0; r < mh; ++r)
      for (int c = 0; c < mw; ++c)
        if (fabs(R[r][c]) > best) { best = fabs(R[r][c]); p = r; q = c; }
    if (!(best > 1e-13 * wmax)) break;
    const double piv = R[p][q];
    for (int r = 0; r < mh; ++r) u[rank][r] = R[r][q] / piv;
    for (int c = 0; c < mw; ++c) v[rank][c] = R[p][c];
    for (int r = 0; r < mh; ++r)
      for (int c = 0; c < mw; ++c) R[r][c] -= u[rank][r] * v[rank][c];
    ++rank;
  }
  return rank;
}

cudaError_t launch_kron_build(dctf_operator *op, const MaskParams &mp, cudaStream_t s) {
  KronParams kp;
  memset(&kp, 0, sizeof kp);
  kp.rank = kron_split_mask(mp, kp.u, kp.v);
  kp.mh = mp.mh; kp.mw = mp.mw; kp.ar = mp.ar; kp.ac = mp.ac;
  kp.n = mp.n; kp.boundary = mp.boundary;
  op->krank = kp.rank;
  if (kp.rank == 0) return cudaSuccess;   // zero mask: nothing to apply, output zeros
  kron_build_kernel<<<2 * kp.rank, kMaxN2, 0, s>>>(kp, op->d_C64, op->d_kA, op->d_kB);
  return cudaGetLastError();
}

cudaError_t launch_apply_kron(const dctf_operator *op, const float *x, int64_t nblocks, float *y,
                              cudaStream_t s) {
  if (op->krank == 0) return cudaMemsetAsync(y, 0, (size_t)nblocks * op->n2 * sizeof(float), s);
  switch (op->n) {
    case 4: return launch_apply<4>(op, x, nblocks, y, s);
    case 8: return launch_apply<8>(op, x, nblocks, y, s);
    case 16: return launch_apply<16>(op, x, nblocks, y, s);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace dctf

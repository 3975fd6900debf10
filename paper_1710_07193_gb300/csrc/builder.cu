// FP64 operator builder: H (spatial filter), M = K H K^T (DCT domain), and the
// low-precision pieces the apply kernels consume.
//
// Sec. II.B-C build the filter of a 3x3 mask from shift/Toeplitz matrices and
// move each to the DCT domain once per mask (Eq. 7); here the whole filter is
// one spatial operator H on the row-major vectorised block, and Eq. 7 applied
// to it gives M = K H K^-1 = K H K^T with K = C kron C (Eq. 1-2).  K is never
// formed: a product with K is the separable 2-D DCT C X C^T of the vector
// reshaped to N x N, so M costs 4 N^5 multiply-adds instead of 2 N^6.
//
// Two launches, both one CTA per row/column of an N^2 x N^2 matrix:
//   build_hg: row p of H (a1) and row p of G = H K^T (first half of a2);
//   build_m : column q of M = K G (second half of a2), its FP32 copy and the
//             FP16 hi/lo pieces (a3), written in the tensor-core B layout.
#include "dctf_internal.cuh"

namespace dctf {
namespace {

__device__ inline void dct_matrix_smem(double (*cs)[kMaxN + 1], int n) {
  // C[u][x] = alpha(u) cos(pi (2x + 1) u / (2n)), Sec. II.A (Eq. 1-2)
  for (int t = threadIdx.x; t < n * n; t += blockDim.x) {
    int u = t / n, x = t % n;
    double alpha = (u == 0) ? sqrt(1.0 / n) : sqrt(2.0 / n);
    cs[u][x] = alpha * cos(M_PI * (2 * x + 1) * u / (2 * n));
  }
}

// out = vec(C mat(in) C^T) for one n x n matrix held row-major in smem;
// thread t < n*n produces element t.  tmp is n*n scratch.
__device__ inline double dct2_vec(const double *in, double *tmp,
                                  const double (*cs)[kMaxN + 1], int n, int t) {
  int a = t / n, b = t % n;
  if (t < n * n) {
    double acc = 0.0;
    for (int s = 0; s < n; ++s) acc += cs[a][s] * in[s * n + b];
    tmp[t] = acc;
  }
  __syncthreads();
  double r = 0.0;
  if (t < n * n)
    for (int s = 0; s < n; ++s) r += tmp[a * n + s] * cs[b][s];
  return r;
}

__global__ void build_hg_kernel(const MaskParams mp, double *__restrict__ H,
                                double *__restrict__ G) {
  __shared__ double cs[kMaxN][kMaxN + 1];
  __shared__ double hrow[kMaxN2];
  __shared__ double tmp[kMaxN2];
  const int n = mp.n, n2 = n * n, p = blockIdx.x, t = threadIdx.x;
  const int i = p / n, j = p % n;
  dct_matrix_smem(cs, n);
  if (t < n2) hrow[t] = 0.0;
  __syncthreads();
  if (t == 0) {
    // Row (i, j) of H: mask entry (r, c) reads pixel (i + r - ar, j + c - ac)
    // of the same block (Eq. 5 as a correlation); zero padding drops the
    // pixels outside the block (Sec. II.B), border replication moves them to
    // the nearest edge pixel, clamping each axis (Sec. II.C, Eq. 13-18).
    for (int r = 0; r < mp.mh; ++r)
      for (int c = 0; c < mp.mw; ++c) {
        int s = i + r - mp.ar, u = j + c - mp.ac;
        if (mp.boundary == DCTF_ZERO) {
          if (s < 0 || s >= n || u < 0 || u >= n) continue;
        } else {
          s = min(max(s, 0), n - 1);
          u = min(max(u, 0), n - 1);
        }
        hrow[s * n + u] += mp.w[r * mp.mw + c];
      }
  }
  __syncthreads();
  if (t < n2) H[(size_t)p * n2 + t] = hrow[t];
  // G[p][:] = (H K^T)[p][:] = K H[p][:]^T = vec(C mat(H[p][:]) C^T)
  double g = dct2_vec(hrow, tmp, cs, n, t);
  if (t < n2) G[(size_t)p * n2 + t] = g;
}

__global__ void build_m_kernel(int n, int f16_scale_exp, const double *__restrict__ G,
                               double *__restrict__ M64, float *__restrict__ M32,
                               float *__restrict__ Mdc, __half *__restrict__ f16) {
  __shared__ double cs[kMaxN][kMaxN + 1];
  __shared__ double gcol[kMaxN2];
  __shared__ double tmp[kMaxN2];
  const int n2 = n * n, q = blockIdx.x, t = threadIdx.x;
  dct_matrix_smem(cs, n);
  if (t < n2) gcol[t] = G[(size_t)t * n2 + q];
  __syncthreads();
  // M[:][q] = K G[:][q] = vec(C mat(G[:][q]) C^T)
  double m = dct2_vec(gcol, tmp, cs, n, t);
  if (t >= n2) return;
  M64[(size_t)t * n2 + q] = m;
  M32[(size_t)t * n2 + q] = (float)m;
  if (q == 0) Mdc[t] = (float)m;
  if (f16 != nullptr) {
    // M * 2^s split as hi = rn16(M 2^s), lo = rn16(M 2^s - hi); row t of the
    // stacked B operand is output coefficient t (hi), row n2 + t its lo part.
    double ms = ldexp(m, f16_scale_exp);
    __half hi = __double2half(ms);
    __half lo = __double2half(ms - (double)__half2float(hi));
    int chunk = q >> 6, byte = (q & 63) * 2;
    char *base = reinterpret_cast<char *>(f16);
    *reinterpret_cast<__half *>(base + sw128_offset(t, byte, 2 * n2, chunk)) = hi;
    *reinterpret_cast<__half *>(base + sw128_offset(n2 + t, byte, 2 * n2, chunk)) = lo;
  }
}

}  // namespace

cudaError_t launch_build(dctf_operator *op, const MaskParams &mp, cudaStream_t s) {
  const int n2 = op->n2;
  build_hg_kernel<<<n2, n2, 0, s>>>(mp, op->d_H64, op->d_G64);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  build_m_kernel<<<n2, n2, 0, s>>>(op->n, op->f16_scale_exp, op->d_G64, op->d_M64,
                                   op->d_M32, op->d_Mdc, op->d_f16);
  return cudaGetLastError();
}

}  // namespace dctf

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
// One launch, one CTA per column q of the N^2 x N^2 operator:
//   row q of H (a1, kept for download);
//   column q of G = H K^T: G[p][q] = sum_b H[p][b] K[q][b] is the spatial
//     filter applied to DCT basis image q, so it comes straight from the mask
//     taps (first half of a2);
//   column q of M = K G (second half of a2), its FP32 copy and the
//     low-precision pieces (a3) in the tensor-core B layout: FP16 hi/lo, and
//     for 16x16 blocks also three BF16 pieces and TF32 hi/lo; for 8x8 blocks
//     the FP16 pieces of the pixel operator G.
#include <cmath>
#include <cstring>
#include <mutex>

#include "sm100_ptx.cuh"

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

// C (Eq. 1-2) into global memory, once per operator: the FP64 cosines are
// costly on this part, so the per-mask build kernels only copy the table.
__global__ void dct_matrix_kernel(int n, double *__restrict__ C) {
  const int t = threadIdx.x;
  if (t < n * n) {
    int u = t / n, x = t % n;
    double alpha = (u == 0) ? sqrt(1.0 / n) : sqrt(2.0 / n);
    C[t] = alpha * cos(M_PI * (2 * x + 1) * u / (2 * n));
  }
}

__device__ inline void load_c(double (*cs)[kMaxN + 1], const double *__restrict__ C, int n) {
  for (int t = threadIdx.x; t < n * n; t += blockDim.x) cs[t / n][t % n] = C[t];
}

// Column q, entry t of M (m) and of G (gq): the FP64 and FP32 copies and
// every low-precision piece, in the layouts the apply kernels read.
__device__ __forceinline__ void write_pieces(int n, int q, int t, int f16_scale_exp, double m,
                                             double gq, double *__restrict__ M64,
                                             float *__restrict__ M32, float *__restrict__ Mdc,
                                             __half *__restrict__ f16,
                                             __nv_bfloat16 *__restrict__ bf16,
                                             uint32_t *__restrict__ tf32,
                                             __half *__restrict__ f16_pix,
                                             float *__restrict__ Gdc) {
  const int n2 = n * n;
  if (f16_pix != nullptr) {
    // the pixel operator G = H K^T (coefficients -> filtered pixels), split
    // like M: G 2^s = hi + lo in FP16 (|G| obeys the same bound as |M|)
    const double gs = ldexp(gq, f16_scale_exp);
    const __half hi = __double2half(gs);
    const __half lo = __double2half(gs - (double)__half2float(hi));
    const int chunk = q >> 6, byte = (q & 63) * 2;
    char *base = reinterpret_cast<char *>(f16_pix);
    *reinterpret_cast<__half *>(base + sw128_offset(t, byte, 2 * n2, chunk)) = hi;
    *reinterpret_cast<__half *>(base + sw128_offset(n2 + t, byte, 2 * n2, chunk)) = lo;
    if (q == 0) Gdc[t] = (float)gq;
  }
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
  if (bf16 != nullptr) {
    // M = m0 + m1 + m2 + O(2^-24 |M|), each piece the BF16 rounding of the
    // remainder (FP64 arithmetic, so every remainder is exact); rows
    // p n2 + t, 64 inputs per 128-byte row.  BF16 has FP32's exponent range,
    // so no scaling.
    const __nv_bfloat16 b0 = __double2bfloat16(m);
    const double r1 = m - (double)__bfloat162float(b0);
    const __nv_bfloat16 b1 = __double2bfloat16(r1);
    const __nv_bfloat16 b2 = __double2bfloat16(r1 - (double)__bfloat162float(b1));
    const int chunk = q >> 6, byte = (q & 63) * 2;
    char *base = reinterpret_cast<char *>(bf16);
    *reinterpret_cast<__nv_bfloat16 *>(base + sw128_offset(t, byte, 3 * n2, chunk)) = b0;
    *reinterpret_cast<__nv_bfloat16 *>(base + sw128_offset(n2 + t, byte, 3 * n2, chunk)) = b1;
    *reinterpret_cast<__nv_bfloat16 *>(base + sw128_offset(2 * n2 + t, byte, 3 * n2, chunk)) = b2;
  }
  if (tf32 != nullptr) {
    // M = hi + lo + O(2^-22 |M|) in TF32 (FP32 bit patterns, low 13 bits
    // clear); rows p n2 + t, 32 inputs per 128-byte row.
    const uint32_t hi = ptx::tf32_rna((float)m);
    const uint32_t lo = ptx::tf32_rna((float)(m - (double)__uint_as_float(hi)));
    const int chunk = q >> 5, byte = (q & 31) * 4;
    char *base = reinterpret_cast<char *>(tf32);
    *reinterpret_cast<uint32_t *>(base + sw128_offset(t, byte, 2 * n2, chunk)) = hi;
    *reinterpret_cast<uint32_t *>(base + sw128_offset(n2 + t, byte, 2 * n2, chunk)) = lo;
  }
}

// Fused build: see the file comment.  Thread t < n2 owns entry t of the
// column (and of H's row q).
__global__ void build_kernel(const MaskParams mp, int f16_scale_exp, const double *__restrict__ C,
                             double *__restrict__ H, double *__restrict__ M64,
                             float *__restrict__ M32, float *__restrict__ Mdc,
                             __half *__restrict__ f16, __nv_bfloat16 *__restrict__ bf16,
                             uint32_t *__restrict__ tf32, __half *__restrict__ f16_pix,
                             float *__restrict__ Gdc) {
  __shared__ double cs[kMaxN][kMaxN + 1];
  __shared__ double gcol[kMaxN2];
  __shared__ double tmp[kMaxN2];
  const int n = mp.n, n2 = n * n, q = blockIdx.x, t = threadIdx.x;
  load_c(cs, C, n);
  __syncthreads();
  if (t < n2) {
    // Row q of H (as a1: mask entry (r, c) of output pixel q reads pixel
    // (qi + r - ar, qj + c - ac) of the block, Eq. 5 as a correlation; zero
    // padding drops pixels outside the block, replication clamps each axis,
    // Sec. II.B-C); thread t owns column t.
    const int qi = q / n, qj = q % n;
    double h = 0.0;
    for (int r = 0; r < mp.mh; ++r)
      for (int c = 0; c < mp.mw; ++c) {
        int s = qi + r - mp.ar, u = qj + c - mp.ac;
        if (mp.boundary == DCTF_ZERO) {
          if (s < 0 || s >= n || u < 0 || u >= n) continue;
        } else {
          s = min(max(s, 0), n - 1);
          u = min(max(u, 0), n - 1);
        }
        if (s * n + u == t) h += mp.w[r * mp.mw + c];
      }
    H[(size_t)q * n2 + t] = h;
    // G[t][q]: output pixel t = (i, j) of the filter applied to basis image
    // q = (fu, fv), whose pixel (a, b) is K[q][(a, b)] = C[fu][a] C[fv][b]
    const int i = t / n, j = t % n, fu = q / n, fv = q % n;
    double g = 0.0;
    for (int r = 0; r < mp.mh; ++r)
      for (int c = 0; c < mp.mw; ++c) {
        int s = i + r - mp.ar, u = j + c - mp.ac;
        if (mp.boundary == DCTF_ZERO) {
          if (s < 0 || s >= n || u < 0 || u >= n) continue;
        } else {
          s = min(max(s, 0), n - 1);
          u = min(max(u, 0), n - 1);
        }
        g += mp.w[r * mp.mw + c] * (cs[fu][s] * cs[fv][u]);
      }
    gcol[t] = g;
  }
  __syncthreads();
  // M[:][q] = K G[:][q] = vec(C mat(G[:][q]) C^T)
  const double m = dct2_vec(gcol, tmp, cs, n, t);
  if (t >= n2) return;
  write_pieces(n, q, t, f16_scale_exp, m, gcol[t], M64, M32, Mdc, f16, bf16, tf32, f16_pix, Gdc);
}

}  // namespace

cudaError_t launch_dct_matrix(dctf_operator *op, cudaStream_t s) {
  dct_matrix_kernel<<<1, op->n2, 0, s>>>(op->n, op->d_C64);
  return cudaGetLastError();
}

cudaError_t launch_build(dctf_operator *op, const MaskParams &mp, cudaStream_t s) {
  const int n2 = op->n2;
  build_kernel<<<n2, n2, 0, s>>>(mp, op->f16_scale_exp, op->d_C64, op->d_H64, op->d_M64, op->d_M32,
                                 op->d_Mdc, op->d_f16, op->d_bf16, op->d_tf32, op->d_f16_pix,
                                 op->d_Gdc);
  return cudaGetLastError();
}

}  // namespace dctf

// ---------------------------------------------------------------------------
// Allocation-free build of M into caller memory.
//
// For callers that may not allocate device memory: code running inside a
// framework that owns every byte of the GPU through its own pool, real-time
// paths where cudaMalloc's implicit device synchronisation is not allowed,
// or plug-ins handed only the buffers they read and write.  It runs the
// build in its two-pass form, which needs scratch: rows of H and of
// G = H K^T, then columns of M = K G read back from G.  That scratch (G, and
// H when the caller does not want it) lives in this file-scope array instead
// of an allocation.  It is 1 MiB, sized for the
// largest block (n = 16: two 256 x 256 FP64 matrices), and every GPU that
// loads the library holds it until the process exits.
static __device__ __align__(256) double dctf_build_scratch[2 * dctf::kMaxN2 * dctf::kMaxN2];

namespace dctf {
namespace {

constexpr size_t kScratchDoubles = 2 * (size_t)kMaxN2 * kMaxN2;

// Pass 1: row p of H (mask entries added in (r, c) order, as in build_kernel,
// so H is bit-identical) and row p of G = H K^T = vec(C mat(H[p]) C^T).
__global__ void build_hg_noalloc_kernel(const MaskParams mp, double *__restrict__ H,
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
  if (t < n2 && H != nullptr) H[(size_t)p * n2 + t] = hrow[t];
  double g = dct2_vec(hrow, tmp, cs, n, t);
  if (t < n2) G[(size_t)p * n2 + t] = g;
}

// Pass 2: column q of M = K G (FP64 only).
__global__ void build_m_noalloc_kernel(int n, const double *__restrict__ G,
                                       double *__restrict__ M64) {
  __shared__ double cs[kMaxN][kMaxN + 1];
  __shared__ double gcol[kMaxN2];
  __shared__ double tmp[kMaxN2];
  const int n2 = n * n, q = blockIdx.x, t = threadIdx.x;
  dct_matrix_smem(cs, n);
  if (t < n2) gcol[t] = G[(size_t)t * n2 + q];
  __syncthreads();
  double m = dct2_vec(gcol, tmp, cs, n, t);
  if (t < n2) M64[(size_t)t * n2 + q] = m;
}

// Driver entry points fetched at run time (libcuda is not linked).
template <class Fn>
Fn driver_fn(const char *name) {
  void *f = nullptr;
  cudaDriverEntryPointQueryResult q;
  if (cudaGetDriverEntryPointByVersion(name, &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
      q == cudaDriverEntryPointSuccess)
    return reinterpret_cast<Fn>(f);
  return nullptr;
}
typedef CUresult (*CtxGetCurrentFn)(CUcontext *);
typedef CUresult (*CtxGetIdFn)(CUcontext, unsigned long long *);

struct ScratchAddr {
  unsigned long long ctx_id;
  double *addr;
};
std::mutex g_scratch_mu;
ScratchAddr g_scratch_addr[64];   // one per context seen; a full table starts over
int g_scratch_n = 0;

// Device address of the static scratch in the current context.  Host code
// cannot use the symbol itself as a device pointer: the address is looked up
// with cudaGetSymbolAddress once per context (the first call on a device)
// and cached under the context's ID, which CUDA never reuses within a
// process, so a context made after a device reset gets its own lookup.
cudaError_t scratch_on_current_device(double **out) {
  static CtxGetCurrentFn get_cur = nullptr;
  static CtxGetIdFn get_id = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    get_cur = driver_fn<CtxGetCurrentFn>("cuCtxGetCurrent");
    get_id = driver_fn<CtxGetIdFn>("cuCtxGetId");
  });
  if (get_cur == nullptr || get_id == nullptr) return cudaErrorNotSupported;
  CUcontext ctx = nullptr;
  if (get_cur(&ctx) != CUDA_SUCCESS) return cudaErrorDeviceUninitialized;
  if (ctx == nullptr) {
    // no context on this thread yet: make the current device's primary
    // context current (cudaSetDevice initialises it; nothing is allocated)
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaSetDevice(dev);
    if (e != cudaSuccess) return e;
    if (get_cur(&ctx) != CUDA_SUCCESS || ctx == nullptr) return cudaErrorDeviceUninitialized;
  }
  unsigned long long id = 0;
  if (get_id(ctx, &id) != CUDA_SUCCESS) return cudaErrorDeviceUninitialized;
  std::lock_guard<std::mutex> lock(g_scratch_mu);
  for (int i = 0; i < g_scratch_n; ++i)
    if (g_scratch_addr[i].ctx_id == id) {
      *out = g_scratch_addr[i].addr;
      return cudaSuccess;
    }
  void *p = nullptr;
  const cudaError_t e = cudaGetSymbolAddress(&p, dctf_build_scratch);
  if (e != cudaSuccess) return e;
  if (g_scratch_n == 64) g_scratch_n = 0;
  g_scratch_addr[g_scratch_n++] = {id, static_cast<double *>(p)};
  *out = static_cast<double *>(p);
  return cudaSuccess;
}

}  // namespace
}  // namespace dctf

extern "C" dctf_status dctf_build_matrix_noalloc(const double *mask, int mh, int mw,
                                                 const int anchor[2], int n,
                                                 dctf_boundary boundary, double *M_out,
                                                 double *H_out, dctf_stream_t stream) {
  using namespace dctf;
  // the scratch holds G and H, 2 n^4 doubles: a block side beyond its size
  // is refused before anything else is looked at
  if (n < 1) return set_error(DCTF_EINVAL, "block size n=%d: must be positive", n);
  const size_t n2 = (size_t)n * n;
  if (n > kMaxN || 2 * n2 * n2 > kScratchDoubles)
    return set_error(DCTF_EINVAL,
                     "n=%d needs %zu doubles of build scratch; the static scratch holds %zu "
                     "(n <= %d)",
                     n, 2 * n2 * n2, kScratchDoubles, kMaxN);
  MaskParams mp;
  const dctf_status st = check_mask(mask, mh, mw, anchor, n, boundary, &mp);
  if (st != DCTF_OK) return st;
  if (M_out == nullptr) return set_error(DCTF_EINVAL, "M_out must not be NULL");
  if ((reinterpret_cast<uintptr_t>(M_out) & 15) || (reinterpret_cast<uintptr_t>(H_out) & 15))
    return set_error(DCTF_EINVAL, "M_out and H_out must be 16-byte aligned");
  double *scratch = nullptr;
  cudaError_t e = scratch_on_current_device(&scratch);
  if (e != cudaSuccess) return cuda_error(e, "device address of the static build scratch");
  double *G = scratch;                                  // first half
  double *H = H_out != nullptr ? H_out : scratch + n2 * n2;
  build_hg_noalloc_kernel<<<(unsigned)n2, (unsigned)n2, 0, stream>>>(mp, H, G);
  e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_error(e, "no-alloc build launch");
  build_m_noalloc_kernel<<<(unsigned)n2, (unsigned)n2, 0, stream>>>(n, G, M_out);
  e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_error(e, "no-alloc build launch");
  return DCTF_OK;
}

// Pixels <-> block-DCT coefficients on the device (Sec. II.A, Eq. 1 and 3).
//
// forward: uint8 image -> BLOCK = C block C^T per N x N block, raster block
//          order, FP32 or FP64 coefficients [nblocks][N^2];
// inverse: coefficients -> block = C^T BLOCK C -> uint8 by rounding half
//          away from zero and saturating (the conversion of Sec. III).
// One CTA handles kBlocksPerCta blocks, one thread per coefficient; the two
// 1-D passes go through shared memory, in FP64.
#include "dctf_internal.cuh"

namespace dctf {
namespace {

template <int N>
__device__ inline void load_c(double (*cs)[N + 1]) {
  for (int t = threadIdx.x; t < N * N; t += blockDim.x) {
    int u = t / N, x = t % N;
    double alpha = (u == 0) ? sqrt(1.0 / N) : sqrt(2.0 / N);
    cs[u][x] = alpha * cos(M_PI * (2 * x + 1) * u / (2 * N));
  }
}

template <int N> constexpr int blocks_per_cta() { return N == 16 ? 1 : (N == 8 ? 4 : 16); }

template <int N, typename Tout>
__global__ void forward_dct_kernel(const uint8_t *__restrict__ img, int height, int width,
                                   int64_t pitch, Tout *__restrict__ out) {
  constexpr int N2 = N * N, BPC = blocks_per_cta<N>();
  __shared__ double cs[N][N + 1];
  __shared__ double xs[BPC][N2], ts[BPC][N2];
  load_c<N>(cs);
  const int bl = threadIdx.x / N2, t = threadIdx.x % N2, u = t / N, v = t % N;
  const int bw = width / N;
  const int64_t nblocks = (int64_t)(height / N) * bw;
  const int64_t b = (int64_t)blockIdx.x * BPC + bl;
  const bool live = b < nblocks;
  if (live) {
    const int64_t by = b / bw, bx = b % bw;
    xs[bl][t] = img[(by * N + u) * pitch + bx * N + v];
  }
  __syncthreads();
  if (live) {   // ts[u][j] = sum_i C[u][i] x[i][j]   (here v plays j)
    double a = 0.0;
    for (int i = 0; i < N; ++i) a += cs[u][i] * xs[bl][i * N + v];
    ts[bl][t] = a;
  }
  __syncthreads();
  if (live) {   // Y[u][v] = sum_j ts[u][j] C[v][j]
    double a = 0.0;
    for (int j = 0; j < N; ++j) a += ts[bl][u * N + j] * cs[v][j];
    out[b * N2 + t] = (Tout)a;
  }
}

// Forward DCT then JPEG-style quantisation: Q = sat_int16(round_half_away(
// BLOCK / q)) with a per-coefficient table q (input preparation for the
// quantised path).
template <int N>
__global__ void forward_dct_q16_kernel(const uint8_t *__restrict__ img, int height, int width,
                                       int64_t pitch, const uint16_t *__restrict__ q,
                                       int16_t *__restrict__ out) {
  constexpr int N2 = N * N, BPC = blocks_per_cta<N>();
  __shared__ double cs[N][N + 1];
  __shared__ double xs[BPC][N2], ts[BPC][N2];
  load_c<N>(cs);
  const int bl = threadIdx.x / N2, t = threadIdx.x % N2, u = t / N, v = t % N;
  const int bw = width / N;
  const int64_t nblocks = (int64_t)(height / N) * bw;
  const int64_t b = (int64_t)blockIdx.x * BPC + bl;
  const bool live = b < nblocks;
  if (live) {
    const int64_t by = b / bw, bx = b % bw;
    xs[bl][t] = img[(by * N + u) * pitch + bx * N + v];
  }
  __syncthreads();
  if (live) {
    double a = 0.0;
    for (int i = 0; i < N; ++i) a += cs[u][i] * xs[bl][i * N + v];
    ts[bl][t] = a;
  }
  __syncthreads();
  if (live) {
    double a = 0.0;
    for (int j = 0; j < N; ++j) a += ts[bl][u * N + j] * cs[v][j];
    double r = a / (double)q[t];
    r = r < 0.0 ? -floor(-r + 0.5) : floor(r + 0.5);
    r = r < -32768.0 ? -32768.0 : (r > 32767.0 ? 32767.0 : r);
    out[b * N2 + t] = (int16_t)r;
  }
}

template <int N>
__global__ void inverse_dct_u8_kernel(const float *__restrict__ coeffs, int height, int width,
                                      uint8_t *__restrict__ img, int64_t pitch) {
  constexpr int N2 = N * N, BPC = blocks_per_cta<N>();
  __shared__ double cs[N][N + 1];
  __shared__ double ys[BPC][N2], ts[BPC][N2];
  load_c<N>(cs);
  const int bl = threadIdx.x / N2, t = threadIdx.x % N2, i = t / N, j = t % N;
  const int bw = width / N;
  const int64_t nblocks = (int64_t)(height / N) * bw;
  const int64_t b = (int64_t)blockIdx.x * BPC + bl;
  const bool live = b < nblocks;
  if (live) ys[bl][t] = coeffs[b * N2 + t];
  __syncthreads();
  if (live) {   // ts[i][v] = sum_u C[u][i] Y[u][v]
    double a = 0.0;
    for (int u = 0; u < N; ++u) a += cs[u][i] * ys[bl][u * N + j];
    ts[bl][t] = a;
  }
  __syncthreads();
  if (live) {   // p[i][j] = sum_v ts[i][v] C[v][j]
    double p = 0.0;
    for (int v = 0; v < N; ++v) p += ts[bl][i * N + v] * cs[v][j];
    double r = p < 0.0 ? -floor(-p + 0.5) : floor(p + 0.5);
    r = r < 0.0 ? 0.0 : (r > 255.0 ? 255.0 : r);
    const int64_t by = b / bw, bx = b % bw;
    img[(by * N + i) * pitch + bx * N + j] = (uint8_t)r;
  }
}

template <typename Tout>
cudaError_t launch_forward(const uint8_t *img, int h, int w, int64_t pitch, int n, Tout *out,
                           cudaStream_t s) {
  const int64_t nblocks = (int64_t)(h / n) * (w / n);
  switch (n) {
    case 4: forward_dct_kernel<4, Tout><<<(unsigned)((nblocks + 15) / 16), 256, 0, s>>>(img, h, w, pitch, out); break;
    case 8: forward_dct_kernel<8, Tout><<<(unsigned)((nblocks + 3) / 4), 256, 0, s>>>(img, h, w, pitch, out); break;
    case 16: forward_dct_kernel<16, Tout><<<(unsigned)nblocks, 256, 0, s>>>(img, h, w, pitch, out); break;
  }
  return cudaGetLastError();
}

}  // namespace
}  // namespace dctf

using namespace dctf;

static dctf_status check_image(const void *img, int h, int w, int64_t pitch, int n,
                               const void *c) {
  if (n != 4 && n != 8 && n != 16) return set_error(DCTF_EINVAL, "n=%d must be 4, 8 or 16", n);
  if (img == nullptr || c == nullptr) return set_error(DCTF_EINVAL, "NULL buffer");
  if (h <= 0 || w <= 0 || h % n || w % n)
    return set_error(DCTF_EINVAL, "image %dx%d: sides must be positive multiples of %d", h, w, n);
  if (pitch < w) return set_error(DCTF_EINVAL, "pitch %lld < width %d", (long long)pitch, w);
  if ((int64_t)(h / n) * (w / n) > ((int64_t)1 << 31)) return set_error(DCTF_EINVAL, "image too large");
  return DCTF_OK;
}

extern "C" {

dctf_status dctf_forward_dct(const uint8_t *image, int height, int width, int64_t pitch, int n,
                             float *coeffs, dctf_stream_t stream) {
  dctf_status st = check_image(image, height, width, pitch, n, coeffs);
  if (st != DCTF_OK) return st;
  cudaError_t e = launch_forward<float>(image, height, width, pitch, n, coeffs, stream);
  return e == cudaSuccess ? DCTF_OK : cuda_error(e, "forward DCT launch");
}

dctf_status dctf_forward_dct_f64(const uint8_t *image, int height, int width, int64_t pitch,
                                 int n, double *coeffs, dctf_stream_t stream) {
  dctf_status st = check_image(image, height, width, pitch, n, coeffs);
  if (st != DCTF_OK) return st;
  cudaError_t e = launch_forward<double>(image, height, width, pitch, n, coeffs, stream);
  return e == cudaSuccess ? DCTF_OK : cuda_error(e, "forward DCT launch");
}

dctf_status dctf_forward_dct_i16(const uint8_t *image, int height, int width, int64_t pitch,
                                 int n, const uint16_t *q, int16_t *coeffs,
                                 dctf_stream_t stream) {
  dctf_status st = check_image(image, height, width, pitch, n, coeffs);
  if (st != DCTF_OK) return st;
  if (q == nullptr) return set_error(DCTF_EINVAL, "quantisation table is NULL");
  const int64_t nblocks = (int64_t)(height / n) * (width / n);
  switch (n) {
    case 4: forward_dct_q16_kernel<4><<<(unsigned)((nblocks + 15) / 16), 256, 0, stream>>>(image, height, width, pitch, q, coeffs); break;
    case 8: forward_dct_q16_kernel<8><<<(unsigned)((nblocks + 3) / 4), 256, 0, stream>>>(image, height, width, pitch, q, coeffs); break;
    case 16: forward_dct_q16_kernel<16><<<(unsigned)nblocks, 256, 0, stream>>>(image, height, width, pitch, q, coeffs); break;
  }
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? DCTF_OK : cuda_error(e, "forward DCT launch");
}

dctf_status dctf_inverse_dct_u8(const float *coeffs, int height, int width, int n,
                                uint8_t *image, int64_t pitch, dctf_stream_t stream) {
  dctf_status st = check_image(image, height, width, pitch, n, coeffs);
  if (st != DCTF_OK) return st;
  const int64_t nblocks = (int64_t)(height / n) * (width / n);
  switch (n) {
    case 4: inverse_dct_u8_kernel<4><<<(unsigned)((nblocks + 15) / 16), 256, 0, stream>>>(coeffs, height, width, image, pitch); break;
    case 8: inverse_dct_u8_kernel<8><<<(unsigned)((nblocks + 3) / 4), 256, 0, stream>>>(coeffs, height, width, image, pitch); break;
    case 16: inverse_dct_u8_kernel<16><<<(unsigned)nblocks, 256, 0, stream>>>(coeffs, height, width, image, pitch); break;
  }
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? DCTF_OK : cuda_error(e, "inverse DCT launch");
}

}  // extern "C"

// Internal declarations shared by the library's translation units.
#pragma once

#include <cuda.h>              // CUtensorMap (type only; the driver entry is
                               // fetched at run time, libcuda is not linked)
#include <cuda_runtime.h>
#include <cuda_fp16.h>
#include <cuda_bf16.h>
#include <cstdint>
#include <cstdio>
#include <mutex>
#include <string>

#include "dctf.h"

namespace dctf {

// ------------------------------------------------------------ host errors
dctf_status set_error(dctf_status s, const char *fmt, ...);
dctf_status cuda_error(cudaError_t e, const char *what);

#define DCTF_CUDA(call)                                                     \
  do {                                                                      \
    cudaError_t e__ = (call);                                               \
    if (e__ != cudaSuccess) return ::dctf::cuda_error(e__, #call);          \
  } while (0)

// Largest mask the build kernels take (parameters travel by value).
constexpr int kMaxN = 16;
constexpr int kMaxN2 = kMaxN * kMaxN;

struct MaskParams {
  double w[kMaxN * kMaxN];   // row-major mh x mw
  int mh, mw, ar, ac, n, boundary;
};

// Argument checks shared by every entry point that takes a mask (capi.cu):
// n in {4, 8, 16}, non-NULL mask and anchor, 1 <= mh, mw <= n, anchor inside
// the mask, a known boundary, finite entries.  Fills *mp; EINVAL otherwise.
dctf_status check_mask(const double *mask, int mh, int mw, const int anchor[2], int n,
                       int boundary, MaskParams *mp);

// Byte layout of the tensor-core B operand ("pieces"): for every 64-element
// chunk kc of the input index k, R stacked rows of 128 bytes (64 fp16/bf16,
// or 32 fp32), 16-byte units XOR-swizzled by (row & 7), i.e. the canonical
// K-major SWIZZLE_128B layout, so a linear copy into 1024-aligned shared
// memory is directly usable by tcgen05.mma.
__host__ __device__ inline size_t sw128_offset(int row, int byte_in_row,
                                               int rows, int chunk) {
  int unit = byte_in_row >> 4;
  return ((size_t)chunk * rows + row) * 128 + (size_t)(((unit ^ (row & 7)) << 4) | (byte_in_row & 15));
}

}  // namespace dctf

// The opaque operator handle.
struct dctf_operator {
  int device;
  int n, n2;
  int mh, mw, ar, ac;
  int boundary;
  dctf_precision precision;
  uint32_t flags;           // DCTF_APPLY_* flags
  int f16_scale_exp;        // pieces hold M * 2^f16_scale_exp
  // one device allocation, carved:
  void *d_base;
  size_t bytes;
  double *d_C64;            // [n][n] DCT matrix C (Eq. 1-2), made once at creation
  double *d_M64;            // [n2][n2] FP64 operator, row = output coefficient
  double *d_H64;            // [n2][n2] spatial operator
  float *d_M32;             // [n2][n2] FP32 copy of M
  float *d_Mdc;             // [n2] M[:, 0] in FP32
  __half *d_f16;            // F16X3 pieces: rows 0..n2-1 hi, n2..2n2-1 lo (sw128)
  __half *d_f16_pix;        // n = 8: F16X3 pieces of the pixel operator G = H K^T
  float *d_Gdc;             // n = 8: G[:, 0] in FP32
  __nv_bfloat16 *d_bf16;    // n = 16: BF16 pieces m0, m1, m2 (3 n2 rows per 64-chunk;
                            //   BF16X3 uses m0, m1)
  uint32_t *d_tf32;         // n = 16: TF32 pieces hi, lo (2 n2 rows per 32-chunk)
  bool kron;                // built with DCTF_BUILD_KRON: Kronecker factors kept
  int krank_bound;          //   min(mh, mw) of the last build: at least the number of terms
  int *d_krank;             //   device: number of terms of M = sum_t A_t kron B_t
  float *d_kscale;          //   device, n = 16: [0] 2^(sZ - sB), [1] 2^-(sZ + sA)
  float *d_kA, *d_kB;       //   [kMaxN][n][n] FP32 each (DCT-domain 1-D filters)
  double *d_kA64, *d_kB64;  //   the same in FP64
  uint8_t *d_kpieces;       //   n = 16: FP16 hi/lo pieces of B_t (16 KB) and A_t (16 KB)
                            //   in the tcgen05 B-operand layout (kron_tc.cu)
  uint32_t *d_err;          // device status word
  // dctf_apply_host staging (lazily allocated): kHostPipes streams, each
  // with an input and an output chunk buffer
  static constexpr int kHostPipes = 4;
  float *d_stage[kHostPipes][2];
  size_t stage_blocks;
  cudaStream_t host_streams[kHostPipes];
  void *h_pipe_items;       // 8x8 F16X3: each pipe's full-chunk work item, encoded once
  std::mutex host_mu;       // serialises dctf_apply_host calls on this operator
};

namespace dctf {

// builder.cu
cudaError_t launch_dct_matrix(dctf_operator *op, cudaStream_t s);
cudaError_t launch_build(dctf_operator *op, const MaskParams &mp, cudaStream_t s);

// apply_simt.cu
cudaError_t launch_apply_simt(const dctf_operator *op, const float *x,
                              const double *x64, int64_t nblocks, float *y,
                              cudaStream_t s);

// tensor-core kernels exist for these (n, precision): apply_group.cu (n = 8,
// F16X3) and apply_n16.cu (n = 16, every split precision)
inline bool tc_supported(int n, dctf_precision p) {
  if (n == 8) return p == DCTF_F16X3;
  return n == 16 && (p == DCTF_F16X3 || p == DCTF_BF16X6 || p == DCTF_TF32X1 || p == DCTF_TF32X3 ||
                     p == DCTF_BF16X3);
}
// pdl: launch with programmatic stream serialisation (the input and the
// operator must not be written by the preceding kernel on the stream)
cudaError_t launch_apply_n16(const dctf_operator *op, const float *x, int64_t nblocks,
                             float *y, cudaStream_t s, bool pdl);

// kron.cu: the Kronecker (sandwich-product) form of the operator, built on
// the device (rank split, factors, and for n = 16 the tensor-core pieces)
constexpr int kKronPieceBytes = 32768;
cudaError_t launch_kron_build(dctf_operator *op, const MaskParams &mp, cudaStream_t s);
cudaError_t launch_apply_kron(const dctf_operator *op, const float *x, int64_t nblocks, float *y,
                              cudaStream_t s);
// kron_tc.cu: the sandwich products on tensor cores (n = 16, F16X3)
cudaError_t launch_apply_kron_tc(const dctf_operator *op, const float *x, int64_t nblocks,
                                 float *y, cudaStream_t s, bool pdl);

int sm_count(int device);

// Host memory a kernel can read and write directly: page-locked, mapped into
// the device address space, [p, p + bytes) inside one allocation.  Returns
// the device address of p, or nullptr.
void *mapped_host(const void *p, size_t bytes);

}  // namespace dctf

// C-ABI entry points: argument checks, operator lifetime, dispatch.
#include <cmath>
#include <cstdarg>
#include <cstring>
#include <mutex>
#include <new>

#include "apply_group.cuh"

namespace dctf {

static thread_local std::string g_last_error;

dctf_status set_error(dctf_status s, const char *fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  g_last_error = buf;
  return s;
}

dctf_status cuda_error(cudaError_t e, const char *what) {
  if (e == cudaErrorMemoryAllocation)
    return set_error(DCTF_ENOMEM, "%s: %s", what, cudaGetErrorString(e));
  return set_error(DCTF_ECUDA, "%s: %s", what, cudaGetErrorString(e));
}

int sm_count(int device) {
  static std::mutex mu;
  static int cache[64] = {0};
  std::lock_guard<std::mutex> lock(mu);
  if (device < 0 || device >= 64) return 0;
  if (cache[device] == 0) {
    int v = 0;
    if (cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, device) != cudaSuccess) return 0;
    cache[device] = v;
  }
  return cache[device];
}

static bool aligned16(const void *p) { return (reinterpret_cast<uintptr_t>(p) & 15) == 0; }

// Host memory a kernel can read and write directly: page-locked
// (cudaHostAlloc, cudaHostRegister), mapped into the device address space,
// with [p, p + bytes) inside one allocation.  Returns the device address of
// p, or nullptr (pageable memory, a range past the allocation, or a failed
// query).
typedef CUresult (*PointerAttrFn)(void *, CUpointer_attribute, CUdeviceptr);
static PointerAttrFn pointer_attr_fn() {
  static PointerAttrFn fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void *f = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuPointerGetAttribute", &f, 12000, cudaEnableDefault,
                                         &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PointerAttrFn>(f);
  });
  return fn;
}
// CTAs of the host-direct launch.  The host link, not the SMs, bounds it
// (~330 GB/s both directions together on GB300, by copy engine or by kernel
// loads alike); measured on 262,144 blocks, 16-48 CTAs reach it (412-435 us)
// while one CTA per SM (152) gives 525 us: fewer concurrent request streams
// over a narrower window of host memory move faster.
constexpr int kHostDirectCtas = 32;

void *mapped_host(const void *p, size_t bytes) {
  if (p == nullptr) return nullptr;
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  if (a.type != cudaMemoryTypeHost || a.devicePointer == nullptr) return nullptr;
  PointerAttrFn f = pointer_attr_fn();
  if (f == nullptr) return nullptr;
  CUdeviceptr start = 0;
  size_t size = 0;
  const CUdeviceptr q = reinterpret_cast<CUdeviceptr>(p);
  if (f(&start, CU_POINTER_ATTRIBUTE_RANGE_START_ADDR, q) != CUDA_SUCCESS ||
      f(&size, CU_POINTER_ATTRIBUTE_RANGE_SIZE, q) != CUDA_SUCCESS)
    return nullptr;
  if (q < start || q - start > size || bytes > size - (q - start)) return nullptr;
  return a.devicePointer;
}

dctf_status check_mask(const double *mask, int mh, int mw, const int anchor[2], int n,
                       int boundary, MaskParams *mp) {
  if (n != 4 && n != 8 && n != 16)
    return set_error(DCTF_EINVAL, "block size n=%d: must be 4, 8 or 16", n);
  if (mask == nullptr || anchor == nullptr)
    return set_error(DCTF_EINVAL, "mask and anchor must not be NULL");
  if (mh < 1 || mw < 1 || mh > n || mw > n)
    return set_error(DCTF_EINVAL, "mask %dx%d must fit in the %dx%d block", mh, mw, n, n);
  if (anchor[0] < 0 || anchor[0] >= mh || anchor[1] < 0 || anchor[1] >= mw)
    return set_error(DCTF_EINVAL, "anchor (%d,%d) outside the %dx%d mask", anchor[0], anchor[1], mh, mw);
  if (boundary != DCTF_ZERO && boundary != DCTF_REPLICATE)
    return set_error(DCTF_EINVAL, "boundary %d: must be DCTF_ZERO or DCTF_REPLICATE", boundary);
  memset(mp, 0, sizeof *mp);
  for (int k = 0; k < mh * mw; ++k) {
    if (!std::isfinite(mask[k])) return set_error(DCTF_EINVAL, "mask entry %d is not finite", k);
    mp->w[k] = mask[k];
  }
  mp->mh = mh; mp->mw = mw; mp->ar = anchor[0]; mp->ac = anchor[1];
  mp->n = n; mp->boundary = boundary;
  return DCTF_OK;
}

// Power of two s with |M 2^s| <= 2^14: ||M||_2 = ||H||_2 <= sum|w| * n, a
// bound on every entry, so the FP16 pieces neither overflow nor lose the lo
// part to subnormals.
static int f16_scale_exponent(const MaskParams &mp) {
  double s = 0.0;
  for (int k = 0; k < mp.mh * mp.mw; ++k) s += fabs(mp.w[k]);
  double bound = s * mp.n;
  if (bound <= 0.0) return 0;
  int e = 14 - (int)ceil(log2(bound));
  return e < -24 ? -24 : (e > 24 ? 24 : e);
}

static size_t align_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

}  // namespace dctf

using namespace dctf;

extern "C" {

int dctf_version(void) { return 400; }   // 0.4.0

const char *dctf_last_error(void) { return g_last_error.c_str(); }

static dctf_status build_operator(const double *mask, int mh, int mw, const int anchor[2], int n,
                                  dctf_boundary boundary, bool kron, dctf_stream_t stream,
                                  dctf_operator **out) {
  if (out == nullptr) return set_error(DCTF_EINVAL, "out must not be NULL");
  *out = nullptr;
  MaskParams mp;
  dctf_status st = check_mask(mask, mh, mw, anchor, n, boundary, &mp);
  if (st != DCTF_OK) return st;

  dctf_operator *op = new (std::nothrow) dctf_operator();
  if (op == nullptr) return set_error(DCTF_ENOMEM, "host allocation of the operator failed");
  DCTF_CUDA(cudaGetDevice(&op->device));
  op->n = n; op->n2 = n * n;
  const size_t n2 = op->n2, sq = n2 * n2;
  const bool pieces = tc_supported(n, DCTF_F16X3);
  const bool wide = n == 16;                  // BF16 and TF32 pieces too
  const bool pix = n == 8;                    // pixel operator pieces too
  size_t off = 0, o_C64, o_M64, o_H64, o_M32, o_Mdc, o_f16 = 0, o_bf16 = 0, o_tf32 = 0,
         o_pix = 0, o_gdc = 0, o_kA = 0, o_kB = 0, o_kA64 = 0, o_kB64 = 0, o_kmisc = 0,
         o_kpieces = 0, o_err;
  o_C64 = off; off = align_up(off + n2 * 8, 1024);
  o_M64 = off; off = align_up(off + sq * 8, 1024);
  o_H64 = off; off = align_up(off + sq * 8, 1024);
  o_M32 = off; off = align_up(off + sq * 4, 1024);
  o_Mdc = off; off = align_up(off + n2 * 4, 1024);
  if (pieces) { o_f16 = off; off = align_up(off + 2 * sq * 2, 1024); }
  if (pix) {
    o_pix = off; off = align_up(off + 2 * sq * 2, 1024);
    o_gdc = off; off = align_up(off + n2 * 4, 1024);
  }
  if (wide) {
    o_bf16 = off; off = align_up(off + 3 * sq * 2, 1024);
    o_tf32 = off; off = align_up(off + 2 * sq * 4, 1024);
  }
  if (kron) {
    o_kA = off; off = align_up(off + (size_t)kMaxN * n2 * 4, 1024);
    o_kB = off; off = align_up(off + (size_t)kMaxN * n2 * 4, 1024);
    o_kA64 = off; off = align_up(off + (size_t)kMaxN * n2 * 8, 1024);
    o_kB64 = off; off = align_up(off + (size_t)kMaxN * n2 * 8, 1024);
    o_kmisc = off; off = align_up(off + 256, 1024);
    if (wide) { o_kpieces = off; off = align_up(off + kKronPieceBytes, 1024); }
  }
  o_err = off; off = align_up(off + 256, 1024);
  cudaError_t e = cudaMalloc(&op->d_base, off);
  if (e != cudaSuccess) { delete op; return cuda_error(e, "cudaMalloc(operator)"); }
  op->bytes = off;
  char *b = static_cast<char *>(op->d_base);
  op->d_C64 = reinterpret_cast<double *>(b + o_C64);
  op->d_M64 = reinterpret_cast<double *>(b + o_M64);
  op->d_H64 = reinterpret_cast<double *>(b + o_H64);
  op->d_M32 = reinterpret_cast<float *>(b + o_M32);
  op->d_Mdc = reinterpret_cast<float *>(b + o_Mdc);
  op->d_f16 = pieces ? reinterpret_cast<__half *>(b + o_f16) : nullptr;
  op->d_f16_pix = pix ? reinterpret_cast<__half *>(b + o_pix) : nullptr;
  op->d_Gdc = pix ? reinterpret_cast<float *>(b + o_gdc) : nullptr;
  op->d_bf16 = wide ? reinterpret_cast<__nv_bfloat16 *>(b + o_bf16) : nullptr;
  op->d_tf32 = wide ? reinterpret_cast<uint32_t *>(b + o_tf32) : nullptr;
  op->kron = kron;
  op->d_kA = kron ? reinterpret_cast<float *>(b + o_kA) : nullptr;
  op->d_kB = kron ? reinterpret_cast<float *>(b + o_kB) : nullptr;
  op->d_kA64 = kron ? reinterpret_cast<double *>(b + o_kA64) : nullptr;
  op->d_kB64 = kron ? reinterpret_cast<double *>(b + o_kB64) : nullptr;
  op->d_krank = kron ? reinterpret_cast<int *>(b + o_kmisc) : nullptr;
  op->d_kscale = kron ? reinterpret_cast<float *>(b + o_kmisc + 16) : nullptr;
  op->d_kpieces = kron && wide ? reinterpret_cast<uint8_t *>(b + o_kpieces) : nullptr;
  op->d_err = reinterpret_cast<uint32_t *>(b + o_err);
  op->precision = pieces ? DCTF_F16X3 : DCTF_FP32_SIMT;

  e = cudaMemsetAsync(op->d_err, 0, 256, stream);
  if (e == cudaSuccess && pieces) e = cudaMemsetAsync(op->d_f16, 0, 2 * sq * 2, stream);
  if (e == cudaSuccess) e = launch_dct_matrix(op, stream);
  if (e != cudaSuccess) { dctf_release_operator(op); return cuda_error(e, "operator set-up"); }
  st = dctf_operator_rebuild(op, mask, mh, mw, anchor, boundary, stream);
  if (st != DCTF_OK) { dctf_release_operator(op); return st; }
  *out = op;
  return DCTF_OK;
}

dctf_status dctf_build_operator(const double *mask, int mh, int mw, const int anchor[2],
                                int n, dctf_boundary boundary, dctf_stream_t stream,
                                dctf_operator **out) {
  return build_operator(mask, mh, mw, anchor, n, boundary, false, stream, out);
}

dctf_status dctf_build_operator_ex(const double *mask, int mh, int mw, const int anchor[2], int n,
                                   dctf_boundary boundary, uint32_t flags, dctf_stream_t stream,
                                   dctf_operator **out) {
  if (flags & ~(uint32_t)(DCTF_MASK_CONVOLUTION | DCTF_BUILD_KRON))
    return set_error(DCTF_EINVAL, "unknown flags");
  const bool kron = (flags & DCTF_BUILD_KRON) != 0;
  if (!(flags & DCTF_MASK_CONVOLUTION))
    return build_operator(mask, mh, mw, anchor, n, boundary, kron, stream, out);
  // convolution with w, anchor a = correlation with w rotated by 180 degrees
  // and the anchor mirrored: (mh - 1 - ar, mw - 1 - ac)
  if (mask == nullptr || anchor == nullptr || mh < 1 || mw < 1 || mh > kMaxN || mw > kMaxN)
    return set_error(DCTF_EINVAL, "bad mask");
  double rot[kMaxN2];
  for (int r = 0; r < mh; ++r)
    for (int c = 0; c < mw; ++c) rot[(mh - 1 - r) * mw + (mw - 1 - c)] = mask[r * mw + c];
  const int a2[2] = {mh - 1 - anchor[0], mw - 1 - anchor[1]};
  return build_operator(rot, mh, mw, a2, n, boundary, kron, stream, out);
}

dctf_status dctf_operator_rebuild(dctf_operator *op, const double *mask, int mh, int mw,
                                  const int anchor[2], dctf_boundary boundary,
                                  dctf_stream_t stream) {
  if (op == nullptr) return set_error(DCTF_EINVAL, "operator is NULL");
  MaskParams mp;
  dctf_status st = check_mask(mask, mh, mw, anchor, op->n, boundary, &mp);
  if (st != DCTF_OK) return st;
  op->mh = mh; op->mw = mw; op->ar = anchor[0]; op->ac = anchor[1];
  op->boundary = boundary;
  op->f16_scale_exp = f16_scale_exponent(mp);
  cudaError_t e = launch_build(op, mp, stream);
  if (e == cudaSuccess && op->kron) e = launch_kron_build(op, mp, stream);
  if (e != cudaSuccess) return cuda_error(e, "operator build launch");
  return DCTF_OK;
}

dctf_status dctf_operator_set_precision(dctf_operator *op, dctf_precision p) {
  if (op == nullptr) return set_error(DCTF_EINVAL, "operator is NULL");
  if (p == DCTF_FP32_SIMT) { op->precision = p; return DCTF_OK; }
  if (p == DCTF_KRON_FP32 || p == DCTF_KRON_F16X3) {
    if (!op->kron)
      return set_error(DCTF_EUNSUPPORTED, "the Kronecker form needs an operator built with "
                                          "DCTF_BUILD_KRON");
    if (p == DCTF_KRON_F16X3 && op->n != 16)
      return set_error(DCTF_EUNSUPPORTED, "DCTF_KRON_F16X3 has a kernel for n=16 only");
    op->precision = p;
    return DCTF_OK;
  }
  if (p < DCTF_FP32_SIMT || (p > DCTF_TF32X3 && p != DCTF_BF16X3))
    return set_error(DCTF_EINVAL, "unknown precision %d", (int)p);
  if (!tc_supported(op->n, p))
    return set_error(DCTF_EUNSUPPORTED, "precision %d has no kernel for n=%d", (int)p, op->n);
  op->precision = p;
  return DCTF_OK;
}

dctf_status dctf_operator_set_flags(dctf_operator *op, uint32_t flags) {
  if (op == nullptr) return set_error(DCTF_EINVAL, "operator is NULL");
  if (flags & ~(uint32_t)DCTF_APPLY_INPUTS_READY) return set_error(DCTF_EINVAL, "unknown flags");
  op->flags = flags;
  return DCTF_OK;
}

dctf_status dctf_operator_kron_rank(const dctf_operator *op, int *rank) {
  if (op == nullptr || rank == nullptr) return set_error(DCTF_EINVAL, "NULL argument");
  if (!op->kron) return set_error(DCTF_EUNSUPPORTED, "operator built without DCTF_BUILD_KRON");
  DCTF_CUDA(cudaDeviceSynchronize());     // the rank is found by the device build
  DCTF_CUDA(cudaMemcpy(rank, op->d_krank, sizeof(int), cudaMemcpyDeviceToHost));
  return DCTF_OK;
}

dctf_status dctf_operator_download(const dctf_operator *op, double *M_host, double *H_host) {
  if (op == nullptr || M_host == nullptr) return set_error(DCTF_EINVAL, "NULL argument");
  size_t bytes = (size_t)op->n2 * op->n2 * sizeof(double);
  DCTF_CUDA(cudaDeviceSynchronize());
  DCTF_CUDA(cudaMemcpy(M_host, op->d_M64, bytes, cudaMemcpyDeviceToHost));
  if (H_host) DCTF_CUDA(cudaMemcpy(H_host, op->d_H64, bytes, cudaMemcpyDeviceToHost));
  return DCTF_OK;
}

dctf_status dctf_operator_status(dctf_operator *op, uint32_t *code, int clear) {
  if (op == nullptr || code == nullptr) return set_error(DCTF_EINVAL, "NULL argument");
  DCTF_CUDA(cudaDeviceSynchronize());
  DCTF_CUDA(cudaMemcpy(code, op->d_err, sizeof(uint32_t), cudaMemcpyDeviceToHost));
  if (clear) {
    DCTF_CUDA(cudaMemset(op->d_err, 0, sizeof(uint32_t)));
    DCTF_CUDA(cudaDeviceSynchronize());
  }
  return DCTF_OK;
}

void dctf_release_operator(dctf_operator *op) {
  if (op == nullptr) return;
  for (int i = 0; i < dctf_operator::kHostPipes; ++i) {
    if (op->host_streams[i]) cudaStreamDestroy(op->host_streams[i]);
    for (int j = 0; j < 2; ++j)
      if (op->d_stage[i][j]) cudaFree(op->d_stage[i][j]);
  }
  if (op->d_base) cudaFree(op->d_base);
  delete[] static_cast<GroupItem *>(op->h_pipe_items);
  delete op;
}

static dctf_status check_apply(const dctf_operator *op, const void *in, size_t in_elem,
                               int64_t nblocks, const float *out) {
  if (op == nullptr) return set_error(DCTF_EINVAL, "operator is NULL");
  if (nblocks < 0) return set_error(DCTF_EINVAL, "nblocks=%lld < 0", (long long)nblocks);
  if (nblocks == 0) return DCTF_OK;
  if (in == nullptr || out == nullptr) return set_error(DCTF_EINVAL, "coefficient pointer is NULL");
  if (!aligned16(in) || !aligned16(out))
    return set_error(DCTF_EINVAL, "coefficient pointers must be 16-byte aligned");
  if (nblocks > (int64_t)1 << 31) return set_error(DCTF_EINVAL, "nblocks too large");
  const char *a = static_cast<const char *>(in);
  const char *b = reinterpret_cast<const char *>(out);
  size_t la = (size_t)nblocks * op->n2 * in_elem, lb = (size_t)nblocks * op->n2 * sizeof(float);
  if (a != b && a < b + lb && b < a + la)
    return set_error(DCTF_EINVAL, "input and output overlap without being equal");
  return DCTF_OK;
}

static dctf_status apply_impl(const dctf_operator *op, const float *coeffs, int64_t nblocks,
                              float *out, dctf_stream_t stream, bool allow_pdl) {
  dctf_status st = check_apply(op, coeffs, sizeof(float), nblocks, out);
  if (st != DCTF_OK || nblocks == 0) return st;
  cudaError_t e;
  if (op->precision == DCTF_FP32_SIMT) {
    e = launch_apply_simt(op, coeffs, nullptr, nblocks, out, stream);
  } else if (op->precision == DCTF_KRON_FP32) {
    e = launch_apply_kron(op, coeffs, nblocks, out, stream);   // in place is fine: a thread
                                                               // writes only the row it read
  } else if (op->precision == DCTF_KRON_F16X3) {
    // in place is fine: a unit of 8 blocks is read before its output is written
    e = launch_apply_kron_tc(op, coeffs, nblocks, out, stream,
                             allow_pdl && (op->flags & DCTF_APPLY_INPUTS_READY) != 0);
  } else if (op->n == 16) {
    if (static_cast<const void *>(coeffs) == static_cast<const void *>(out))
      return set_error(DCTF_EINVAL,
                       "16x16 tensor-core apply cannot run in place (use DCTF_FP32_SIMT)");
    e = launch_apply_n16(op, coeffs, nblocks, out, stream,
                         allow_pdl && (op->flags & DCTF_APPLY_INPUTS_READY) != 0);
  } else {
    // one item of the persistent tensor-core kernel, descriptor by value
    GroupItem gi;
    e = fill_group_item(&gi, op, coeffs, out, nblocks, false, nullptr, nullptr);
    if (e == cudaSuccess)
      e = launch_apply_group(nullptr, &gi, 1, (nblocks + 63) / 64, false, sm_count(op->device), 2,
                             op->d_err, stream,
                             allow_pdl && (op->flags & DCTF_APPLY_INPUTS_READY) != 0);
  }
  if (e != cudaSuccess) return cuda_error(e, "dctf_apply launch");
  return DCTF_OK;
}

dctf_status dctf_apply(const dctf_operator *op, const float *coeffs, int64_t nblocks,
                       float *out, dctf_stream_t stream) {
  return apply_impl(op, coeffs, nblocks, out, stream, true);
}

dctf_status dctf_apply_pixels(const dctf_operator *op, const float *coeffs, int height,
                              int width, uint8_t *image, int64_t pitch, dctf_stream_t stream) {
  if (op == nullptr || coeffs == nullptr || image == nullptr)
    return set_error(DCTF_EINVAL, "NULL argument");
  if (op->n != 8 || op->d_f16_pix == nullptr)
    return set_error(DCTF_EUNSUPPORTED, "the fused pixel apply needs an 8x8 operator");
  if (height <= 0 || width <= 0 || height % 8 || width % 8)
    return set_error(DCTF_EINVAL, "image %dx%d: sides must be positive multiples of 8", height,
                     width);
  if (pitch < width || pitch % 8)
    return set_error(DCTF_EINVAL, "pitch %lld: must be >= width and a multiple of 8",
                     (long long)pitch);
  if (!aligned16(coeffs) || (reinterpret_cast<uintptr_t>(image) & 7))
    return set_error(DCTF_EINVAL, "coeffs must be 16-byte and image 8-byte aligned");
  const int64_t nblocks = (int64_t)(height / 8) * (width / 8);
  if (nblocks > ((int64_t)1 << 31) - 128) return set_error(DCTF_EINVAL, "image too large");
  const char *a = reinterpret_cast<const char *>(coeffs);
  const char *b = reinterpret_cast<const char *>(image);
  const size_t la = (size_t)nblocks * 64 * sizeof(float), lb = (size_t)(height - 1) * pitch + width;
  if (a < b + lb && b < a + la) return set_error(DCTF_EINVAL, "coefficients and image overlap");
  GroupItem gi;   // (its coefficient output map is not used: pointed at the input)
  cudaError_t e = fill_group_item(&gi, op, coeffs, const_cast<float *>(coeffs), nblocks, false,
                                  nullptr, nullptr);
  if (e == cudaSuccess) {
    gi.pieces = op->d_f16_pix;
    gi.mdc = op->d_Gdc;
    gi.img = image;
    gi.pitch = pitch;
    gi.bw = width / 8;
    e = launch_apply_pixels(gi, (nblocks + 63) / 64, sm_count(op->device), op->d_err, stream,
                            (op->flags & DCTF_APPLY_INPUTS_READY) != 0);
  }
  if (e != cudaSuccess) return cuda_error(e, "dctf_apply_pixels launch");
  return DCTF_OK;
}

dctf_status dctf_apply_planar(const dctf_operator *op, const float *coeffs, int height, int width,
                              int64_t pitch, float *out, int64_t out_pitch,
                              dctf_stream_t stream) {
  if (op == nullptr || coeffs == nullptr || out == nullptr)
    return set_error(DCTF_EINVAL, "NULL argument");
  if (op->n != 8 || op->d_f16 == nullptr)
    return set_error(DCTF_EUNSUPPORTED, "the image-plane apply needs an 8x8 operator");
  if (height <= 0 || width <= 0 || height % 8 || width % 8)
    return set_error(DCTF_EINVAL, "plane %dx%d: sides must be positive multiples of 8", height,
                     width);
  if (pitch < width || out_pitch < width || pitch % 4 || out_pitch % 4)
    return set_error(DCTF_EINVAL, "pitches must be >= width and multiples of 4 floats");
  if (!aligned16(coeffs) || !aligned16(out))
    return set_error(DCTF_EINVAL, "planes must be 16-byte aligned");
  // the tile walk runs over block rows padded to 128 blocks, in 32-bit indices
  if ((int64_t)(height / 8) * ((width / 8 + 127) / 128 * 128) > ((int64_t)1 << 31) - 128)
    return set_error(DCTF_EINVAL, "plane too large");
  const char *a = reinterpret_cast<const char *>(coeffs);
  const char *b = reinterpret_cast<const char *>(out);
  const size_t la = ((size_t)(height - 1) * pitch + width) * 4;
  const size_t lb = ((size_t)(height - 1) * out_pitch + width) * 4;
  if (a != b && a < b + lb && b < a + la)
    return set_error(DCTF_EINVAL, "input and output planes overlap without being equal");
  if (a == b && pitch != out_pitch)
    return set_error(DCTF_EINVAL, "in place needs equal pitches");
  cudaError_t e = launch_apply_planar(op, coeffs, height, width, pitch, out, out_pitch, op->d_err,
                                      stream, (op->flags & DCTF_APPLY_INPUTS_READY) != 0);
  if (e != cudaSuccess) return cuda_error(e, "dctf_apply_planar launch");
  return DCTF_OK;
}

dctf_status dctf_apply_f64in(const dctf_operator *op, const double *coeffs, int64_t nblocks,
                             float *out, dctf_stream_t stream) {
  dctf_status st = check_apply(op, coeffs, sizeof(double), nblocks, out);
  if (st != DCTF_OK || nblocks == 0) return st;
  if (static_cast<const void *>(coeffs) == static_cast<const void *>(out))
    return set_error(DCTF_EINVAL, "FP64 input cannot be filtered in place into FP32");
  cudaError_t e = launch_apply_simt(op, nullptr, coeffs, nblocks, out, stream);
  if (e != cudaSuccess) return cuda_error(e, "dctf_apply_f64in launch");
  return DCTF_OK;
}

int dctf_host_buffer_direct(const void *p, int64_t bytes) {
  return bytes >= 0 && mapped_host(p, (size_t)bytes) != nullptr ? 1 : 0;
}

dctf_status dctf_apply_host(dctf_operator *op, const float *host_in, int64_t nblocks,
                            float *host_out) {
  if (op == nullptr) return set_error(DCTF_EINVAL, "operator is NULL");
  if (nblocks < 0) return set_error(DCTF_EINVAL, "nblocks < 0");
  if (nblocks == 0) return DCTF_OK;
  if (host_in == nullptr || host_out == nullptr) return set_error(DCTF_EINVAL, "NULL buffer");
  if (nblocks > ((int64_t)1 << 31) - 128) return set_error(DCTF_EINVAL, "nblocks too large");
  const size_t row = (size_t)op->n2 * sizeof(float);
  {
    const char *a = reinterpret_cast<const char *>(host_in), *b = reinterpret_cast<char *>(host_out);
    const size_t len = (size_t)nblocks * row;
    if (a != b && a < b + len && b < a + len)
      return set_error(DCTF_EINVAL, "input and output overlap without being equal");
  }
  std::lock_guard<std::mutex> lock(op->host_mu);   // the streams and staging are per operator
  constexpr int P = dctf_operator::kHostPipes;
  if (op->host_streams[0] == nullptr)
    for (int i = 0; i < P; ++i)
      DCTF_CUDA(cudaStreamCreateWithFlags(&op->host_streams[i], cudaStreamDefault));
  // 8x8 F16X3 on page-locked mapped host memory: one host-direct launch
  // reads the input and writes the output over the host link itself (no
  // device staging, no copy-engine pipeline to fill and drain)
  if (op->n == 8 && op->precision == DCTF_F16X3 && aligned16(host_in) && aligned16(host_out)) {
    const void *din = mapped_host(host_in, (size_t)nblocks * row);
    void *dout = din ? mapped_host(host_out, (size_t)nblocks * row) : nullptr;
    if (dout != nullptr) {
      GroupItem gi;
      memset(&gi, 0, sizeof gi);
      gi.pieces = op->d_f16;
      gi.mdc = op->d_Mdc;
      gi.out_scale = ldexpf(1.0f, -op->f16_scale_exp);
      gi.nblocks = nblocks;
      gi.hin = static_cast<const float *>(din);
      gi.hout = static_cast<float *>(dout);
      cudaStream_t s = op->host_streams[0];
      cudaError_t e = launch_apply_host_direct(gi, (nblocks + 63) / 64, kHostDirectCtas,
                                               op->d_err, s);
      if (e != cudaSuccess) return cuda_error(e, "dctf_apply_host launch");
      DCTF_CUDA(cudaStreamSynchronize(s));
      return DCTF_OK;
    }
  }
  const int64_t chunk = (int64_t)((8u << 20) / row);    // 8 MB of coefficients per chunk (4 MB measured slower)
  if (op->d_stage[0][0] == nullptr) {
    for (int i = 0; i < P; ++i)
      for (int j = 0; j < 2; ++j) DCTF_CUDA(cudaMalloc(&op->d_stage[i][j], chunk * row));
    op->stage_blocks = chunk;
  }
  // 8x8 F16X3: each pipe's work item (tensor maps of its fixed staging
  // buffers) is encoded once, so a full chunk costs one launch call
  const bool cached = op->n == 8 && op->precision == DCTF_F16X3;
  if (cached && op->h_pipe_items == nullptr) {
    GroupItem *items = new (std::nothrow) GroupItem[P];
    if (items == nullptr) return set_error(DCTF_ENOMEM, "host allocation");
    for (int k = 0; k < P; ++k) {
      cudaError_t e = fill_group_item(&items[k], op, op->d_stage[k][0], op->d_stage[k][1], chunk,
                                      false, nullptr, nullptr);
      if (e != cudaSuccess) { delete[] items; return cuda_error(e, "tensor map encode"); }
    }
    op->h_pipe_items = items;
  }
  // chunk c runs on pipe c % P: its host->device copy, the apply and its
  // device->host copy are ordered on that stream, and the P pipes overlap,
  // so both copy engines and the SMs stay busy.  The apply follows a copy
  // on its stream, so it never uses programmatic dependent launch.
  const int64_t nchunks = (nblocks + chunk - 1) / chunk;
  for (int64_t c = 0; c < nchunks; ++c) {
    const int k = (int)(c % P);
    const int64_t b0 = c * chunk, nb = nblocks - b0 < chunk ? nblocks - b0 : chunk;
    cudaStream_t s = op->host_streams[k];
    DCTF_CUDA(cudaMemcpyAsync(op->d_stage[k][0], host_in + b0 * op->n2, nb * row,
                              cudaMemcpyHostToDevice, s));
    dctf_status st = DCTF_OK;
    if (cached && nb == chunk) {
      GroupItem gi = static_cast<GroupItem *>(op->h_pipe_items)[k];
      gi.out_scale = ldexpf(1.0f, -op->f16_scale_exp);    // follows rebuilds
      cudaError_t e = launch_apply_group(nullptr, &gi, 1, (nb + 63) / 64, false,
                                         sm_count(op->device), 2, op->d_err, s, false);
      if (e != cudaSuccess) st = cuda_error(e, "dctf_apply_host launch");
    } else {
      st = apply_impl(op, op->d_stage[k][0], nb, op->d_stage[k][1], s, false);
    }
    if (st != DCTF_OK) return st;
    DCTF_CUDA(cudaMemcpyAsync(host_out + b0 * op->n2, op->d_stage[k][1], nb * row,
                              cudaMemcpyDeviceToHost, s));
  }
  for (int k = 0; k < P; ++k) DCTF_CUDA(cudaStreamSynchronize(op->host_streams[k]));
  return DCTF_OK;
}

}  // extern "C"

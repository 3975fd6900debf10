// Self-test of the device-side failure handling used by the tensor-core
// kernels: a wait that can never complete must give up after its limit,
// record a status code, and make every other role of the CTA leave its loop
// through the abort flag, so the kernel returns and the context stays
// usable.  Nothing here faults, traps or waits without a bound.
#include "sm100_ptx.cuh"

namespace dctf {
namespace {

using namespace ptx;

// Warp 0, lane 0 waits (bounded, limit_ns) on a barrier nobody arrives at:
// it times out and records code 0x101.  Warp 1 waits warp-uniformly, with a
// limit 1000x longer, on another barrier nobody arrives at: it must leave
// through the abort flag set by warp 0, long before its own limit.
__global__ void selftest_timeout_kernel(uint32_t *err, uint64_t limit_ns, uint32_t *left_by_abort) {
  __shared__ uint64_t bars[2];
  __shared__ int abort_flag;
  volatile int *ab = &abort_flag;
  if (threadIdx.x == 0) {
    mbar_init(&bars[0], 1);
    mbar_init(&bars[1], 1);
    *ab = 0;
    mbar_fence_init();
  }
  __syncthreads();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (warp == 0 && lane == 0) {
    wait_bounded_ns(&bars[0], 0, ab, err, 0x101u, limit_ns);
  } else if (warp == 1) {
    const bool ok = __all_sync(0xffffffffu,
                               wait_bounded_ns(&bars[1], 0, ab, err, 0x202u, limit_ns * 1000));
    if (!ok && lane == 0 && *ab) *left_by_abort = 1;
  }
  __syncthreads();
}

}  // namespace
}  // namespace dctf

using namespace dctf;

extern "C" dctf_status dctf_selftest_wait_timeout(uint32_t limit_us, uint32_t *code,
                                                  uint32_t *other_role_aborted) {
  if (code == nullptr || other_role_aborted == nullptr)
    return set_error(DCTF_EINVAL, "NULL argument");
  if (limit_us == 0 || limit_us > 100000)
    return set_error(DCTF_EINVAL, "limit_us must be in 1..100000");
  uint32_t *d = nullptr;
  DCTF_CUDA(cudaMalloc(&d, 2 * sizeof(uint32_t)));
  cudaError_t e = cudaMemset(d, 0, 2 * sizeof(uint32_t));
  if (e == cudaSuccess) {
    selftest_timeout_kernel<<<1, 64>>>(d, (uint64_t)limit_us * 1000, d + 1);
    e = cudaGetLastError();
  }
  uint32_t h[2] = {0, 0};
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  if (e == cudaSuccess) e = cudaMemcpy(h, d, sizeof h, cudaMemcpyDeviceToHost);
  cudaFree(d);
  if (e != cudaSuccess) return cuda_error(e, "self-test");
  *code = h[0];
  *other_role_aborted = h[1];
  return h[0] != 0 ? DCTF_ETIMEOUT : DCTF_OK;
}

// aa_selftest.cu -- self-test of the bounded device-side wait that every
// streaming pass uses on its mbarriers (no counterpart in the paper).
//
// A one-CTA kernel arms an mbarrier with an expected transaction count and
// issues no copy, so the phase never completes; mbar_wait_bounded gives up
// after its iteration limit (about a second), the kernel records the
// timeout code and returns normally.  The host checks that the error came
// back as a status and that the context is still usable.
#include "../../include/aa.h"
#include "aa_passes.cuh"

namespace {
__global__ void wait_timeout_kernel(int *status) {
  __shared__ __align__(8) uint64_t bar;
  if (threadIdx.x == 0) {
    aa::mbar_init(&bar, 1);
    aa::fence_mbar_init();
    aa::mbar_arrive_expect_tx(&bar, 16);  // 16 bytes that no copy will deliver
    *status = aa::mbar_wait_bounded(&bar, 0) ? 0 : aa::DEV_ETIMEOUT;
  }
}
}  // namespace

extern "C" int aa_selftest_wait_timeout(void *stream) {
  int *d = nullptr;
  if (cudaMalloc(&d, sizeof(int)) != cudaSuccess) {
    cudaGetLastError();
    return AA_ENOMEM;
  }
  int h = 1;
  cudaStream_t s = (cudaStream_t)stream;
  cudaError_t e = cudaMemcpyAsync(d, &h, sizeof(int), cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) {
    wait_timeout_kernel<<<1, 32, 0, s>>>(d);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaMemcpyAsync(&h, d, sizeof(int), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  cudaFree(d);
  if (e != cudaSuccess) return AA_ECUDA;
  return h == aa::DEV_ETIMEOUT ? AA_ETIMEOUT : (h == 0 ? AA_OK : AA_ECUDA);
}

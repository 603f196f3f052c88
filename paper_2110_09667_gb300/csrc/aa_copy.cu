// aa_copy.cu -- a copy kernel for moving iterates between page-locked host
// memory and the device.
//
// On this part the host memory sits behind NVLink-C2C, and the SMs can load
// and store page-locked host memory directly through its device address.
// A grid of 16-byte loads and stores from every SM keeps more transfers in
// flight than the copy engines do.  The kernel runs only when
// cudaPointerGetAttributes reports a device address for both sides (device
// memory, or host memory from cudaHostAlloc / cudaHostRegister); anything
// else (pageable host memory, unaligned pointers) goes to cudaMemcpyAsync.
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/aa.h"

namespace {

constexpr int COPY_THREADS = 512;
constexpr int COPY_UNROLL = 4;  // 16-byte transfers in flight per thread

__global__ void __launch_bounds__(COPY_THREADS)
    copy16_kernel(uint4 *__restrict__ dst, const uint4 *__restrict__ src, size_t n16) {
  const size_t stride = (size_t)gridDim.x * COPY_THREADS;
  size_t i = (size_t)blockIdx.x * COPY_THREADS + threadIdx.x;
  for (; i + (COPY_UNROLL - 1) * stride < n16; i += COPY_UNROLL * stride) {
    uint4 v[COPY_UNROLL];
#pragma unroll
    for (int u = 0; u < COPY_UNROLL; ++u) v[u] = src[i + u * stride];
#pragma unroll
    for (int u = 0; u < COPY_UNROLL; ++u) dst[i + u * stride] = v[u];
  }
  for (; i < n16; i += stride) dst[i] = src[i];
}

__global__ void copy_tail_kernel(unsigned char *__restrict__ dst, const unsigned char *__restrict__ src,
                                 size_t n) {
  for (size_t i = threadIdx.x; i < n; i += blockDim.x) dst[i] = src[i];
}

// The address the device uses for p, or null when the device cannot
// address it (pageable host memory, an unknown pointer).
const void *device_address(const void *p) {
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    (void)cudaGetLastError();  // clear the error an unknown pointer leaves
    return nullptr;
  }
  if (at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged ||
      at.type == cudaMemoryTypeHost)
    return at.devicePointer;
  return nullptr;
}

int sm_count() {
  int dev = 0, n = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return 0;
  return n;
}

}  // namespace

extern "C" int aa_copy_path(const void *dst, const void *src) {
  const void *ds = device_address(src), *dd = device_address(dst);
  return (ds && dd && ((((uintptr_t)ds | (uintptr_t)dd) & 15u) == 0)) ? 1 : 0;
}

extern "C" int aa_copy(void *dst, const void *src, size_t bytes, void *stream) {
  if (bytes == 0) return AA_OK;
  if (!dst || !src) return AA_EINVAL;
  cudaStream_t s = (cudaStream_t)stream;
  const void *ds = device_address(src);
  void *dd = const_cast<void *>(device_address(dst));
  const bool aligned = (((uintptr_t)ds | (uintptr_t)dd) & 15u) == 0;
  const int nsm = sm_count();
  if (!ds || !dd || !aligned || nsm <= 0) {
    return cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDefault, s) == cudaSuccess ? AA_OK
                                                                                : AA_ECUDA;
  }
  const size_t n16 = bytes / 16;
  if (n16 > 0) {
    size_t blocks = (n16 + COPY_THREADS - 1) / COPY_THREADS;
    const size_t cap = (size_t)nsm * 4;  // four CTAs of 512 threads per SM
    if (blocks > cap) blocks = cap;
    copy16_kernel<<<(unsigned)blocks, COPY_THREADS, 0, s>>>((uint4 *)dd, (const uint4 *)ds, n16);
    if (cudaGetLastError() != cudaSuccess) return AA_ECUDA;
  }
  const size_t tail = bytes - n16 * 16;
  if (tail) {
    copy_tail_kernel<<<1, 32, 0, s>>>((unsigned char *)dd + n16 * 16,
                                       (const unsigned char *)ds + n16 * 16, tail);
    if (cudaGetLastError() != cudaSuccess) return AA_ECUDA;
  }
  return AA_OK;
}

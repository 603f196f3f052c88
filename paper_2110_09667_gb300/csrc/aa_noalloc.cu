// aa_noalloc.cu -- aa_mdot_noalloc: the multi-column dot product of aa_mdot
// with its reduction scratch in a statically sized device array, for callers
// that must not allocate device memory.
//
// Some callers cannot call cudaMalloc from the code that needs the product:
// frameworks that own all device memory through their own pool and forbid
// allocations behind the pool's back, processes running close to the
// device's memory limit where a fresh allocation could fail in the middle of
// a solve, and latency-critical loops where cudaMalloc/cudaFree would
// synchronize the device.  This entry point gives them the same deterministic two-stage
// reduction as aa_mdot without any allocation: the per-CTA partial sums and
// the reduction state live in g_mdot_scratch below, a file-scope array that
// every GPU which loads the library holds until the process exits.
#include <cuda_runtime.h>
#include <string.h>

#include <mutex>

#include "../../include/aa.h"
#include "aa_passes.cuh"

namespace {

using namespace aa;

// Largest grid this entry point launches (2 CTAs on each of 152 SMs; also
// enough to saturate HBM for a streaming multi-dot).
constexpr int NA_GRID = 304;
constexpr size_t NA_STATE_BYTES = (sizeof(DevState) + 255) / 256 * 256;
constexpr size_t NA_PARTIAL_BYTES = (size_t)NA_GRID * NDOT_MAX * sizeof(double);
// Total scratch: the reduction state plus NA_GRID x 256 partial sums
// (about 0.76 MB).
constexpr size_t NA_BYTES = NA_STATE_BYTES + NA_PARTIAL_BYTES;

static __device__ __align__(256) unsigned char g_mdot_scratch[NA_BYTES];

// Device address of g_mdot_scratch for each device, looked up with that
// device current (in host code the symbol name is only a host-side stand-in).
// The address belongs to the context the module was loaded into, so the
// cache is keyed on the current context as well: after cudaDeviceReset (a new
// primary context) the address is looked up again instead of reusing a
// pointer into the destroyed context.
constexpr int NA_MAX_DEVICES = 64;
std::mutex g_na_mutex;
void *g_na_ptr[NA_MAX_DEVICES];
void *g_na_ctx[NA_MAX_DEVICES];

typedef int (*ctx_get_current_fn)(void **);  // cuCtxGetCurrent(CUcontext *)

void *current_context() {
  static ctx_get_current_fn fn = nullptr;
  static bool tried = false;
  if (!tried) {
    void *p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = (ctx_get_current_fn)p;
    cudaGetLastError();
    tried = true;
  }
  void *ctx = nullptr;
  if (fn && fn(&ctx) != 0) ctx = nullptr;
  return ctx;
}

int scratch_for_current_device(void **out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= NA_MAX_DEVICES) return AA_ECUDA;
  std::lock_guard<std::mutex> lock(g_na_mutex);
  // (A thread whose runtime has not bound a context yet reads NULL here; the
  // look-up below binds it, and the context is read again after it.)
  void *ctx = current_context();
  if (!g_na_ptr[dev] || ctx != g_na_ctx[dev]) {
    void *p = nullptr;
    if (cudaGetSymbolAddress(&p, g_mdot_scratch) != cudaSuccess || !p) {
      cudaGetLastError();
      return AA_ECUDA;
    }
    g_na_ptr[dev] = p;
    g_na_ctx[dev] = current_context();
  }
  *out = g_na_ptr[dev];
  return AA_OK;
}

template <int DPW>
cudaError_t launch_na(const PassArgs &a, int grid, size_t smem, int nstages, cudaStream_t s) {
  auto kern = pass_kernel<double, DPW>;
  cudaError_t e =
      cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024 - 8 * 1024);
  if (e != cudaSuccess) return e;
  kern<<<grid, NT, smem, s>>>(a, nstages);
  return cudaGetLastError();
}

}  // namespace

extern "C" int aa_mdot_noalloc(const double *A, int64_t lda, int k, const double *V, int64_t ldv,
                               int nv, int64_t n, double *out_dev, void *stream) {
  if (!A || !V || !out_dev) return AA_EINVAL;
  if (n < 1 || k < 1 || nv < 1 || lda < n || ldv < n) return AA_EINVAL;
  if (k * nv > NDOT_MAX || k + nv > MAXCOL) return AA_EINVAL;  // beyond the scratch's capacity
  if (n > (int64_t)2147483647 * TR) return AA_EINVAL;
  for (int j = 0; j < k; ++j)
    if (((uintptr_t)(A + (size_t)j * lda) & 15u) != 0) return AA_EINVAL;
  for (int v = 0; v < nv; ++v)
    if (((uintptr_t)(V + (size_t)v * ldv) & 15u) != 0) return AA_EINVAL;
  void *scratch = nullptr;
  if (scratch_for_current_device(&scratch) != AA_OK) return AA_ECUDA;
  DevState *st = (DevState *)scratch;
  double *partials = (double *)((unsigned char *)scratch + NA_STATE_BYTES);
  cudaStream_t s = (cudaStream_t)stream;

  PassArgs a;
  memset(&a, 0, sizeof a);
  a.kind = K_MDOT;
  a.n = n;
  a.ntiles = (int)((n + TR - 1) / TR);
  a.m = 1;
  a.ncol = k + nv;
  a.qbase = a.ncol;  // every column is FP64
  for (int j = 0; j < k; ++j) a.col[j] = A + (size_t)j * lda;
  for (int v = 0; v < nv; ++v) a.col[k + v] = V + (size_t)v * ldv;
  for (int j = 0; j < k; ++j)
    for (int v = 0; v < nv; ++v) {
      a.dot_a[a.ndots] = (uint8_t)j;
      a.dot_b[a.ndots] = (uint8_t)(k + v);
      a.ndots++;
    }
  a.st = st;
  a.partials = partials;
  a.result_host_dev = out_dev;

  // The ticket that elects the last CTA and the device status word must
  // start at zero; the array keeps whatever the previous call left.
  if (cudaMemsetAsync(&st->ticket, 0, sizeof(st->ticket), s) != cudaSuccess ||
      cudaMemsetAsync(&st->st, 0, sizeof(st->st), s) != cudaSuccess) {
    cudaGetLastError();
    return AA_ECUDA;
  }
  const size_t stage = (size_t)a.ncol * TR * 8;
  const size_t budget = 227 * 1024 - 8 * 1024;
  const int nstages = (stage * 2 <= budget) ? 2 : 1;
  size_t smem = stage * nstages;
  const size_t epi = epi_doubles(1) * sizeof(double);
  if (smem < epi) smem = epi;
  int grid = NA_GRID;
  if (grid > a.ntiles) grid = a.ntiles;
  const int dpw = (a.ndots + NWARP - 1) / NWARP;
  cudaError_t e;
  if (dpw <= 1) e = launch_na<1>(a, grid, smem, nstages, s);
  else if (dpw <= 4) e = launch_na<4>(a, grid, smem, nstages, s);
  else if (dpw <= 16) e = launch_na<16>(a, grid, smem, nstages, s);
  else e = launch_na<32>(a, grid, smem, nstages, s);
  return e == cudaSuccess ? AA_OK : AA_ECUDA;
}

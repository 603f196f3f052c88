// aa_passes_bf16.cu -- streaming-pass kernels instantiated for __nv_bfloat16 history
// storage (one translation unit per storage type so that they compile in
// parallel).
#include "aa_passes.cuh"

namespace aa {
cudaError_t launch_pass_bf16(const PassArgs &a, int nsm, int *grid_out, cudaStream_t stream) {
  return launch_q<__nv_bfloat16>(a, nsm, grid_out, stream);
}
}  // namespace aa

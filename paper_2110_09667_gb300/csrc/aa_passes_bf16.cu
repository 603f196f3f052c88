// aa_passes_bf16.cu -- streaming-pass kernels instantiated for __nv_bfloat16 history
// storage; every n-space operation runs on the FP32/INT pipes (MODE 2).
// (One translation unit per storage type so that they compile in parallel.)
#include "aa_passes.cuh"

namespace aa {
cudaError_t launch_pass_bf16(const PassArgs &a, int nsm, int *grid_out, cudaStream_t stream) {
  return launch_qm<__nv_bfloat16, 2>(a, nsm, grid_out, stream);
}
}  // namespace aa

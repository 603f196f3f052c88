// aa_passes.cu -- dispatch of the streaming-pass kernels by history
// storage type (the kernels themselves are in aa_passes.cuh, instantiated in
// aa_passes_f64.cu, aa_passes_f32.cu and aa_passes_bf16.cu).
#include <cuda_runtime.h>

#include "aa_common.h"

namespace aa {
cudaError_t launch_pass_f64(const PassArgs &a, int nsm, int *grid_out, cudaStream_t stream);
cudaError_t launch_pass_f32(const PassArgs &a, int nsm, int *grid_out, cudaStream_t stream);
cudaError_t launch_pass_bf16(const PassArgs &a, int nsm, int *grid_out, cudaStream_t stream);

// storage: 0 fp64, 1 fp32, 2 bf16
cudaError_t launch_pass(const PassArgs &a, int storage, int nsm, int *grid_out,
                        cudaStream_t stream) {
  if (storage == 1) return launch_pass_f32(a, nsm, grid_out, stream);
  if (storage == 2) return launch_pass_bf16(a, nsm, grid_out, stream);
  return launch_pass_f64(a, nsm, grid_out, stream);
}

int max_grid(int nsm) { return nsm * 8; }
}  // namespace aa

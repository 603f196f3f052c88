// aa_passes_f64.cu -- streaming-pass kernels instantiated for double history
// storage (one translation unit per storage type so that they compile in
// parallel).
#include "aa_passes.cuh"

namespace aa {
cudaError_t launch_pass_f64(const PassArgs &a, int nsm, int *grid_out, cudaStream_t stream) {
  return launch_q<double>(a, nsm, grid_out, stream);
}
}  // namespace aa

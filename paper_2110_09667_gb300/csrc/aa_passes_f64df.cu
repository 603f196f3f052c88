// aa_passes_f64df.cu -- streaming-pass kernels for FP64 history storage with
// the n-space arithmetic in (hi, lo) float arithmetic on the FP32/INT pipes
// (AA_FLAG_DF_ARITH, MODE 3).  Own translation unit so that it compiles in
// parallel with the other storage types.
#include "aa_passes.cuh"

namespace aa {
cudaError_t launch_pass_f64df(const PassArgs &a, int nsm, int *grid_out, cudaStream_t stream) {
  return launch_qm<double, 3>(a, nsm, grid_out, stream);
}
}  // namespace aa

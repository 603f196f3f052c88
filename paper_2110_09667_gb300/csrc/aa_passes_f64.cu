// aa_passes_f64.cu -- streaming-pass kernels instantiated for FP64 history
// storage: the exact FP64 path and the variant with FP32-pipe dot products.
// (One translation unit per storage type so that they compile in parallel.)
#include "aa_passes.cuh"

namespace aa {
cudaError_t launch_pass_f64df(const PassArgs &a, int nsm, int *grid_out, cudaStream_t stream);

cudaError_t launch_pass_f64(const PassArgs &a, int nsm, int *grid_out, cudaStream_t stream) {
  // AA_FLAG_DF_ARITH moves only the first pass (rotation, differences, first
  // dot block: the FP64-pipe-bound one) to (hi, lo) float arithmetic; the
  // projection and update passes, which split every FP64 operand and do one
  // multiply-add with it, issue more slowly in that form than on the FP64 pipe.
  if ((a.flags & 0x10u) && a.kind == K_A) return launch_pass_f64df(a, nsm, grid_out, stream);
  // AA_FLAG_FP32_DOTS: the first pass of an add and the CGS-2 middle pass,
  // when they carry more than RD dot products, move those products to the
  // FP32 pipe; passes with a few products keep their FP64 row-local sums.
  if ((a.flags & 0x8u) && a.ndots > RD && (a.kind == K_A || a.kind == K_CGS2B))
    return launch_qm<double, 1>(a, nsm, grid_out, stream);
  return launch_qm<double, 0>(a, nsm, grid_out, stream);
}
}  // namespace aa

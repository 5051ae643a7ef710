// D2Q37 fused step kernels with bf16 population storage.
#include "step2d.cuh"

namespace hlbm {
cudaError_t launch_step2d_bf16(const StepArgs& a, int kind, bool mom, int rows, cudaStream_t s) {
  return launch_step2d_st<ST_BF16>(a, kind, mom, rows, s);
}
}  // namespace hlbm

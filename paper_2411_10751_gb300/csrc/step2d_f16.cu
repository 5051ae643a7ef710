// D2Q37 fused step kernels with f16 population storage.
#include "step2d.cuh"

namespace hlbm {
cudaError_t launch_step2d_f16(const StepArgs& a, int kind, bool mom, int rows, cudaStream_t s) {
  return launch_step2d_st<ST_F16>(a, kind, mom, rows, s);
}
}  // namespace hlbm

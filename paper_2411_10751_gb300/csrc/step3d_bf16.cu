// D3Q39 fused step kernels with bf16 population storage.
#include "step3d.cuh"

namespace hlbm {
cudaError_t launch_step3d_bf16(const StepArgs& a, int kind, bool mom, int rows, int npt, const CUtensorMap* tm,
                              cudaStream_t s) {
  return launch_step3d_st<ST_BF16>(a, kind, mom, rows, npt, tm, s);
}
}  // namespace hlbm

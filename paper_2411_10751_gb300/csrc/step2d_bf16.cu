// D2Q37 fused step kernels with bf16 population storage.
#include "step2d.cuh"

namespace hlbm {
cudaError_t launch_step2d_bf16(const StepArgs& a, int kind, bool mom, int rows, int npt, const CUtensorMap* tm,
                              cudaStream_t s) {
  return launch_step2d_st<ST_BF16>(a, kind, mom, rows, npt, tm, s, nullptr, nullptr);
}
void box_step2d_bf16(int kind, bool mom, int rows, int* wb, int* hb, int* ob) {
  launch_step2d_st<ST_BF16>(StepArgs{}, kind, mom, rows, 1, nullptr, nullptr, wb, hb, ob);
}
cudaError_t configure_step2d_bf16() { return configure_step2d_st<ST_BF16>(); }
}  // namespace hlbm

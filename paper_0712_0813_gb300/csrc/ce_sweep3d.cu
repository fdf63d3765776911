// ce_sweep3d.cu -- 3D z-sweep step kernel (placeholder until the tiled kernel lands).
#include "ce_internal.h"

namespace ce {
bool sweep_supported(int, int64_t, int, int) { return false; }
SweepPlan sweep_plan(int64_t, int, int) { return SweepPlan{}; }
template <typename T>
cudaError_t launch_step_sweep(const StepArgs<T>&, const SweepPlan&, cudaStream_t) {
  return cudaErrorNotSupported;
}
template cudaError_t launch_step_sweep<float>(const StepArgs<float>&, const SweepPlan&, cudaStream_t);
template cudaError_t launch_step_sweep<double>(const StepArgs<double>&, const SweepPlan&, cudaStream_t);
}  // namespace ce

// Instantiations of the fused step kernel (lbm_step_kernel.cuh) for one storage family.
#include "lbm_step_kernel.cuh"

namespace lbm {

cudaError_t launch_step_f32(int cfg, const StepArgs& a, bool reduce, cudaStream_t st) {
    return launch_step_cfg<float, false>(cfg, a, reduce, st);
}

cudaError_t launch_step_f32s(int cfg, const StepArgs& a, bool reduce, cudaStream_t st) {
    return launch_step_cfg<float, true>(cfg, a, reduce, st);
}

}  // namespace lbm

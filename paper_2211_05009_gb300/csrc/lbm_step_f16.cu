// Instantiations of the fused step kernel (lbm_step_kernel.cuh) for one storage family.
#include "lbm_step_kernel.cuh"

namespace lbm {

cudaError_t launch_step_f16s(int cfg, const StepArgs& a, bool reduce, cudaStream_t st) {
    return launch_step_cfg<__half, true>(cfg, a, reduce, st);
}

cudaError_t launch_step_bf16s(int cfg, const StepArgs& a, bool reduce, cudaStream_t st) {
    return launch_step_cfg<__nv_bfloat16, true>(cfg, a, reduce, st);
}

cudaError_t launch_step_q16s(int cfg, const StepArgs& a, bool reduce, cudaStream_t st) {
    return launch_step_cfg<q16, true>(cfg, a, reduce, st);
}

}  // namespace lbm

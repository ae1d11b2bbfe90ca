// Instantiations of the fused power-iteration kernel for bfloat16 storage
// (bf16 -> bf16 for intermediate steps, bf16 -> float32 for the final step).
#include "spmm.cuh"

namespace fsc {
cudaError_t launch_step_bf16(int LP, int G, bool weighted, const StepArgs& a, cudaStream_t s) {
    return launch_step_any<__nv_bfloat16, __nv_bfloat16>(LP, G, weighted, a, s);
}
cudaError_t launch_step_bf16_to_f32(int LP, int G, bool weighted, const StepArgs& a, cudaStream_t s) {
    return launch_step_any<__nv_bfloat16, float>(LP, G, weighted, a, s);
}
FSC_BOUNDS_READER(spmm_bf16)
}  // namespace fsc

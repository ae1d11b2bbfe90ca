// Instantiations of the fused power-iteration kernel for float32 storage.
#include "spmm.cuh"

namespace fsc {
cudaError_t launch_step_f32(int LP, int G, bool weighted, const StepArgs& a, cudaStream_t s) {
    return launch_step_any<float, float>(LP, G, weighted, a, s);
}
FSC_BOUNDS_READER(spmm_f32)
}  // namespace fsc

// Compiled variant f32 (8, 56, 8): the step with the CUDA-core propagation.
#include "dpf_wide_launch.cuh"

namespace dpf {
template dpf_status wide_launch<float, 8, 56, 8, false>(Ctx&, StepArgs<float>&, cudaStream_t);
}  // namespace dpf

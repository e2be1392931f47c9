// Compiled variant f32 (8, 56, 8): the step with the tensor-core propagation.
#include "dpf_wide_launch.cuh"

namespace dpf {
template dpf_status wide_launch<float, 8, 56, 8, true>(Ctx&, StepArgs<float>&, cudaStream_t);
}  // namespace dpf

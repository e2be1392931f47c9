// Compiled variant: precision float, d1 = 8, d2 = 56, dy = 8 (constants in device
// memory, tensor-core propagation).
#include "dpf_variant_wide.cuh"

namespace dpf {
Variant make_v_f32_8_56_8() { return WideVariantImpl<float, 8, 56, 8>::make(DPF_F32); }
}  // namespace dpf

// Compiled variant: precision float, d1 = 2, d2 = 8, dy = 2.
#include "dpf_variant.cuh"

namespace dpf {
Variant make_v_f32_2_8_2() { return VariantImpl<float, 2, 8, 2>::make(DPF_F32); }
}  // namespace dpf

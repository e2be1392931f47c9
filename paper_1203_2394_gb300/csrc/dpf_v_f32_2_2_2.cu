// Compiled variant: precision float, d1 = 2, d2 = 2, dy = 2.
#include "dpf_variant.cuh"

namespace dpf {
Variant make_v_f32_2_2_2() { return VariantImpl<float, 2, 2, 2>::make(DPF_F32); }
}  // namespace dpf
